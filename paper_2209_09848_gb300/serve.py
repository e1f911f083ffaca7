"""Serving loop for matched-filter search requests (not in the paper).

Requests -- cutouts of uneven size and frame count, each with its own
trajectory grid -- arrive at any time.  The server admits them by device
memory footprint against a budget, uploads each admitted stack into device
memory where it stays until its search is done, and runs the searches on a
pool of CUDA streams, so requests admitted while others are on the GPU
overlap with them on the device (continuous batching: a request starts as
soon as memory and a stream slot are free, not when a batch fills).  Every
search runs through the CUDA library (mf_prf_table_create, mf_search,
mf_rescore_topk); this module only schedules.

Latency of a request = time from arrival (submit) to its results being in
host memory.

Each search reports whether all of its bounded device waits completed
through its own status slot (mf_search_status), copied back with its
results; a request whose search gave up is failed with MFError(MF_ETIMEOUT)
while the requests around it complete normally.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor

import numpy as np
import torch

from . import binding as mf


@dataclasses.dataclass
class Request:
    """One search.  Host tensors (pinned for fast uploads): stack [T, H, W]
    float32 / bfloat16 / float16, sigma [H, W] float32, mask [H, W] uint8 or
    None, frame_scale [T] float32 or None; velocities vx, vy (px/frame);
    optionally the frames' times [T] and pointing jitter [T, 2] (the filter
    bank then follows them), the PRF kind (2: shift-stack filter) and
    phase_steps (Q > 0: the phase-quantised bank)."""
    stack: torch.Tensor
    sigma: torch.Tensor
    vx: np.ndarray
    vy: np.ndarray
    mask: torch.Tensor | None = None
    frame_scale: torch.Tensor | None = None
    k_top: int = 0
    sigma_px: float = 0.7
    tag: object = None
    times: np.ndarray | None = None
    jitter: np.ndarray | None = None
    kind: int = 0
    phase_steps: int = 0
    # for tests of the failure path: enqueue, after this request's search, a
    # bounded device wait that runs out and records its code in the search's
    # status slot, so the request must come back failed (MF_ETIMEOUT)
    probe_timeout: bool = False


@dataclasses.dataclass
class Result:
    snr_max: np.ndarray
    argmax: np.ndarray
    candidates: np.ndarray | None
    arrival: float
    admitted: float
    done: float
    footprint: int
    tag: object = None
    gpu_start_ms: float = 0.0  # device timeline of the request's work, from the server's start event
    gpu_end_ms: float = 0.0
    kernel_start_ms: float = 0.0  # the same for its kernels alone (after its uploads, before its downloads)
    kernel_end_ms: float = 0.0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint_bytes(req: Request, table) -> int:
    """Device bytes a request holds while admitted: its stack, noise map, mask
    and frame scales, the search workspace (sized by the library), the
    outputs, the filter bank and, if asked, the rescore workspace and
    candidate list."""
    T, H, W = req.stack.shape
    n = T * H * W * req.stack.element_size() + H * W * 4
    n += H * W if req.mask is not None else 0
    n += T * 4 if req.frame_scale is not None else 0
    n += mf.search_workspace_size((T, H, W), table, req.stack.dtype) + H * W * 8 + table.info()["device_bytes"]
    if req.k_top:
        n += mf.rescore_workspace_size(H, W, req.k_top) + req.k_top * mf.CANDIDATE_BYTES + 4
    return int(n)


class Server:
    """Admission by footprint, device-resident stacks, overlapping searches.

    budget_bytes: device memory the admitted requests may hold together.
    streams: searches that may be in flight at once.
    planners: host threads building filter banks (the planner is C++ and
    releases the GIL)."""

    def __init__(self, budget_bytes: int, streams: int = 4, planners: int = 4, device=None, skip_ahead: int = 8):
        dev = torch.device(device if device is not None else "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.budget = int(budget_bytes)
        self.used = 0
        self.peak = 0
        self.skip_ahead = skip_ahead
        self._pending = collections.deque()
        self._cv = threading.Condition()
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self._free_streams = list(range(streams))
        self._inflight = collections.deque()
        self._planner = ThreadPoolExecutor(max_workers=planners)
        self._stop = False
        self._active = 0  # admitted and not yet completed
        self._t0 = torch.cuda.Event(enable_timing=True)  # origin of the device timeline
        self._t0.record(torch.cuda.current_stream(self.device))
        self.rejected = 0
        self.failed = 0  # requests whose search reported a device wait that gave up
        self._sched = threading.Thread(target=self._schedule_loop, daemon=True)
        self._done = threading.Thread(target=self._complete_loop, daemon=True)
        self._sched.start()
        self._done.start()

    # ------------------------------------------------------------- public
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        arrival = time.perf_counter()
        plan = self._planner.submit(self._plan, req)
        with self._cv:
            self._pending.append((req, fut, arrival, plan))
            self._cv.notify_all()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()
        self._done.join()
        self._planner.shutdown(wait=True)

    # ------------------------------------------------------------ planning
    def _plan(self, req: Request):
        torch.cuda.set_device(self.device)
        T = req.stack.shape[0]
        table = mf.prf_table_create(req.vx, req.vy, T, sigma_px=req.sigma_px, kind=req.kind, times=req.times,
                                    jitter=req.jitter, phase_steps=req.phase_steps)
        return table, footprint_bytes(req, table)

    # ----------------------------------------------------------- admission
    def _pick(self):
        """First of the next `skip_ahead` pending requests whose plan is ready
        and whose footprint fits; a request larger than the whole budget is
        failed with MemoryError.  Called with the lock held."""
        for i, (req, fut, arrival, plan) in enumerate(list(self._pending)[: self.skip_ahead]):
            if not plan.done():
                continue
            try:
                table, fp = plan.result()
            except Exception as e:  # planning failed: report it on the request
                del self._pending[i]
                fut.set_exception(e)
                return "again"
            if fp > self.budget:
                del self._pending[i]
                self.rejected += 1
                fut.set_exception(MemoryError("request needs %d bytes, budget is %d" % (fp, self.budget)))
                return "again"
            if self.used + fp <= self.budget:
                del self._pending[i]
                return req, fut, arrival, table, fp
        return None

    def _schedule_loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                while True:
                    if self._stop and not self._pending:
                        return
                    picked = self._pick() if self._free_streams else None
                    if picked == "again":
                        continue
                    if picked is not None:
                        break
                    self._cv.wait(timeout=0.002)
                req, fut, arrival, table, fp = picked
                self.used += fp
                self.peak = max(self.peak, self.used)
                self._active += 1
                sidx = self._free_streams.pop(0)
            try:
                job = self._launch(req, table, self._streams[sidx])
            except Exception as e:
                with self._cv:
                    self.used -= fp
                    self._active -= 1
                    self._free_streams.append(sidx)
                    self._cv.notify_all()
                fut.set_exception(e)
                continue
            with self._cv:
                self._inflight.append((job, fut, arrival, time.perf_counter(), fp, sidx, req.tag))
                self._cv.notify_all()

    def _launch(self, req: Request, table, stream):
        T, H, W = req.stack.shape
        dev = self.device
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            stack = torch.empty((T, H, W), dtype=req.stack.dtype, device=dev)
            stack.copy_(req.stack, non_blocking=True)
            sigma = req.sigma.to(dev, non_blocking=True)
            mask = None if req.mask is None else req.mask.to(dev, non_blocking=True)
            fs = None if req.frame_scale is None else req.frame_scale.to(dev, non_blocking=True)
            ws = torch.empty(mf.search_workspace_size((T, H, W), table, req.stack.dtype), dtype=torch.uint8,
                             device=dev)
            snr_max = torch.empty((H, W), dtype=torch.float32, device=dev)
            argmax = torch.empty((H, W), dtype=torch.int32, device=dev)
            evk0 = torch.cuda.Event(enable_timing=True)
            evk0.record(stream)
            mf.search(stack, sigma, table, mask=mask, frame_scale=fs, workspace=ws, out=(snr_max, argmax, None),
                      stream=stream)
            if req.probe_timeout:
                mf.wait_probe_search(ws, stream=stream)
            cand = None
            if req.k_top:
                raw, n = mf.rescore_topk(stack, sigma, table, snr_max, argmax, req.k_top, mask=mask,
                                         frame_scale=fs, stream=stream)
                cand = (raw, n)
            evk1 = torch.cuda.Event(enable_timing=True)
            evk1.record(stream)
            status = torch.zeros(1, dtype=torch.int32, pin_memory=True)
            mf.search_status(ws, status, stream=stream)
            out_max = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
            out_arg = torch.empty((H, W), dtype=torch.int32, pin_memory=True)
            out_max.copy_(snr_max, non_blocking=True)
            out_arg.copy_(argmax, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        # device tensors stay referenced until the job completes
        return dict(ev=ev, ev0=ev0, evk=(evk0, evk1), keep=(stack, sigma, mask, fs, ws, snr_max, argmax, table),
                    out=(out_max, out_arg), cand=cand, status=status)

    # ---------------------------------------------------------- completion
    def _complete_loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self._cv:
                while not self._inflight:
                    if self._stop and not self._pending and self._active == 0:
                        return
                    self._cv.wait(timeout=0.002)
                item = None
                for j, it in enumerate(self._inflight):
                    if it[0]["ev"].query():
                        item = it
                        del self._inflight[j]
                        break
            if item is None:
                time.sleep(0.0002)
                continue
            job, fut, arrival, admitted, fp, sidx, tag = item
            done = time.perf_counter()
            code = int(job["status"][0])
            res = err = None
            if code != 0:
                # a bounded wait of this request's search gave up: its maps
                # are not valid; the other requests are not affected
                self.failed += 1
                err = mf.MFError(mf.MF_ETIMEOUT, "request %r: a device wait of its search gave up (code %d)"
                                 % (tag, code))
            else:
                cands = None
                if job["cand"] is not None:
                    raw, n = job["cand"]
                    cands = mf.decode_candidates(raw, int(n.item()))
                res = Result(job["out"][0].numpy().copy(), job["out"][1].numpy().copy(), cands, arrival, admitted,
                             done, fp, tag, self._t0.elapsed_time(job["ev0"]), self._t0.elapsed_time(job["ev"]),
                             self._t0.elapsed_time(job["evk"][0]), self._t0.elapsed_time(job["evk"][1]))
            del job
            with self._cv:
                self.used -= fp
                self._active -= 1
                self._free_streams.append(sidx)
                self._cv.notify_all()
            if err is not None:
                fut.set_exception(err)
            else:
                fut.set_result(res)


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)
