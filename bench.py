#!/usr/bin/env python3
"""Benchmark of the trajectory matched filter (Ganapathi 2022, Section 3.2).

Workload: the paper-shaped search -- 1000 frames of 2048 x 2048 float32
residuals, log-normal per-pixel sigma, 1 % clustered star mask, 200 injected
linear movers, 100 trajectories on a 10 x 10 velocity grid over +-0.1 px/frame
(synthetic stand-ins for TESS full-frame images; seeded).

One step = one pass of the hot path over that stack: mf_search (inverse
variance, weighted stack, FP64-accumulated denominator, FP32 numerator
stencil, SNR max/argmax over the filter bank) followed by mf_rescore_topk
(top 4096 candidates re-scored in FP64).  The filter-bank table is built once
before timing.  Metric: trajectory x pixel x frame updates per second.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank searches its own stack (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "traj*pixel*frame/s at 1000x2048^2x100 traj"
UNIT = "traj*pixel*frame/s"
T_FR, HH, WW, NXG, NYG, VMAX = 1000, 2048, 2048, 10, 10, 0.1
# the paper's own figure for this search (Abstract): 100 trajectories on
# 1000 frames of 2048 x 2048 in 5 minutes on one NVIDIA A100
PAPER_RATE = NXG * NYG * T_FR * HH * WW / 300.0
K_TOP = 4096
FLOP_PER_UNIT_GENERAL = 50  # 25 FP32 FMAs per (trajectory, pixel, frame): the general 5x5 footprint
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


def _sm_count():
    """Streaming multiprocessors of the GPU the benchmark runs on."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def _fp32_peak_tflops(sm_mhz, sms=None):
    """FFMA peak from unit counts and clock: SMs x FP32 lanes x 2 flop x clock."""
    sms = _sm_count() if sms is None else sms
    return sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
                power.append(float(parts[3].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, dist=None, device=None) -> float:
    """Max of a per-rank number over all ranks (the slowest rank sets the
    whole job's time); identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Weak scaling: every rank processes its own units; the job's throughput
    is all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def flop_per_unit(kernel: int, vx, taps: int = 5) -> float:
    """Algorithmic FP32 flops per (trajectory, pixel, frame) of the numerator
    form the plan uses.  General 5 x 5 footprint: 25 FMAs.  Factored form
    (separable footprint): a `taps`-tap column pass per trajectory, plus a
    `taps`-tap row pass shared by all trajectories with the same v_x, i.e.
    taps * C / K FMAs per unit for C distinct v_x among K trajectories (halo
    rows and columns, and classes split over several CTAs, are overhead, not
    algorithmic work); taps = 1 for the shift-stack filter."""
    if kernel != 2:
        return float(FLOP_PER_UNIT_GENERAL)
    K = len(vx)
    C = len(set(float(v) for v in vx))
    return 2.0 * (taps + taps * C / K)


def _traffic_from_profiles(kernel: int = 2):
    """DRAM bytes of the numerator per traj*pixel*frame (all its launches),
    from the committed ncu summary of the kernel the plan uses: measured on a
    small case of the same plan (counters beyond the launch time are not
    taken on the full workload), to be scaled by the units of a step."""
    name = "k_numerator_fac_paper_shaped.md" if kernel == 2 else "k_numerator_paper_shaped.md"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_unit:"):
                    v = line.split(":", 1)[1].strip()
                    return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


def cpu_oracle_sample(res_dev, sigma_np, mask_np, vx, vy, T, budget_s=15.0, threads=None, kind=0):
    """Time the FP64 oracle on host cores over a crop of the same workload:
    all trajectories and frames, start pixels in a centred square sized for
    about `budget_s` seconds of CPU work.  Returns (units/s, cores, sample text,
    (oracle snr, crop origin, side))."""
    import numpy as np

    import oracle
    oracle.build()
    cores = threads or oracle.threads()
    H, W = sigma_np.shape
    shifts, taps = oracle.trajectory_table(vx, vy, T, kind=kind)
    halo = int(np.abs(shifts).max()) + 3

    def run(side):
        y0, x0 = (H - side) // 2, (W - side) // 2
        ya, yb = max(0, y0 - halo), min(H, y0 + side + halo)
        xa, xb = max(0, x0 - halo), min(W, x0 + side + halo)
        sub = res_dev[:, ya:yb, xa:xb].contiguous().cpu().numpy()
        sig = np.ascontiguousarray(sigma_np[ya:yb, xa:xb])
        msk = None if mask_np is None else np.ascontiguousarray(mask_np[ya:yb, xa:xb])
        lam = oracle.inverse_variance(sig, msk)
        ys, xs = np.meshgrid(np.arange(y0 - ya, y0 - ya + side), np.arange(x0 - xa, x0 - xa + side),
                             indexing="ij")
        K = len(vx)
        ys = np.repeat(ys.ravel(), K)
        xs = np.repeat(xs.ravel(), K)
        ks = np.tile(np.arange(K), side * side)
        t0 = time.perf_counter()
        N, D = oracle.search_points(sub, lam, shifts, taps, ys, xs, ks)
        dt = time.perf_counter() - t0
        return dt, N.reshape(side, side, K), D.reshape(side, side, K), (y0, x0)

    dt, *_ = run(8)
    per_px = dt / 64.0
    side = int(max(8, min(256, (budget_s / max(per_px, 1e-9)) ** 0.5)))
    dt, N, D, origin = run(side)
    units = side * side * len(vx) * T
    sample = "%dx%d start pixels x %d trajectories x %d frames (crop of the same stack)" % (side, side, len(vx), T)
    return units / dt, cores, sample, (N, D, origin, side)


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, each step a bounded
    sample of the same workload (generated on the host with the same recipe)."""
    import numpy as np

    import oracle
    from paper_2209_09848_gb300 import synth
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    oracle.build()
    side = int(os.environ.get("MF_REF_SIDE", "48"))
    vx, vy = synth.velocity_grid(NXG, NYG, -VMAX, VMAX)
    shifts, taps = oracle.trajectory_table(vx, vy, T_FR)
    halo = int(np.abs(shifts).max()) + 3
    hs = side + 2 * halo
    rng = np.random.default_rng(7)
    sigma = np.exp(0.3 * rng.standard_normal((hs, hs))).astype(np.float32)
    mask = synth.star_mask(hs, hs, rng, 0.01)
    res = (sigma[None] * rng.standard_normal((T_FR, hs, hs), dtype=np.float32)).astype(np.float32)
    lam = oracle.inverse_variance(sigma, mask)
    K = len(vx)
    yy, xx = np.meshgrid(np.arange(halo, halo + side), np.arange(halo, halo + side), indexing="ij")
    ys, xs = np.repeat(yy.ravel(), K), np.repeat(xx.ravel(), K)
    ks = np.tile(np.arange(K), side * side)
    for _ in range(args.warmup):
        oracle.search_points(res, lam, shifts, taps, ys[:K * 4], xs[:K * 4], ks[:K * 4])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        N, D = oracle.search_points(res, lam, shifts, taps, ys, xs, ks)
        snr, valid, smax, amax = oracle.snr_and_best(N.reshape(side * side, K).T[:, :, None],
                                                     D.reshape(side * side, K).T[:, :, None])
        times.append(time.perf_counter() - t0)
    units = side * side * K * T_FR
    dt = sum(times) / len(times)
    value = units / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "paper-shaped search, 1000 frames x 2048^2 px x 100 trajectories (FP64 oracle "
                               "on a %dx%d start-pixel sample per step)" % (side, side),
                   "frames": T_FR, "height": HH, "width": WW, "trajectories": K},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": "%dx%d start pixels x %d trajectories x %d frames per step" % (side, side, K,
                                                                                                   T_FR)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the search runs only in the CUDA library)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2209_09848_gb300 import _build
    _build.build()
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import synth

    T, H, W = args.frames, args.size, args.size
    # 200 movers on the 2048 x 2048 frame; a smaller frame gets them in proportion to its area
    n_mov = max(1, int(round(200 * H * W / (HH * WW))))
    case = synth.paper_case_gpu(T=T, H=H, W=W, n_movers=n_mov, seed=1 + rank, device=dev)
    vx, vy = synth.velocity_grid(NXG, NYG, -args.vmax, args.vmax)
    K = len(vx)
    kind = 2 if args.prf == "shiftstack" else 0
    table = mf.prf_table_create(vx, vy, T, kind=kind, kernel=args.kernel or None)
    info = table.info()
    res, sigma, mask = case["res"], case["sigma"], case["mask"]
    ws_search = torch.empty(mf.search_workspace_size((T, H, W), table), dtype=torch.uint8, device=dev)
    ws_rescore = torch.empty(mf.rescore_workspace_size(H, W, K_TOP), dtype=torch.uint8, device=dev)
    snr_max = torch.empty((H, W), dtype=torch.float32, device=dev)
    argmax = torch.empty((H, W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        mf.search(res, sigma, table, mask=mask, workspace=ws_search, out=(snr_max, argmax, None), stream=stream)
        if not args.no_rescore:
            mf.rescore_topk(res, sigma, table, snr_max, argmax, K_TOP, mask=mask, workspace=ws_rescore,
                            stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if mf.device_status() != 0:
        raise SystemExit("device status word set during warm-up")
    mf.profile_enable(True)
    mf.profile_read(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = mf.profile_read(reset=True)
    mf.profile_enable(False)
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist, dev)
    units_rank = K * T * H * W
    value = job_throughput(units_rank, ws, ms * 1e-3)

    peaks, peak_src = _peaks()
    # numerator time per step (a factored plan with time segments makes one
    # launch per segment)
    num_launches, num_ms_total = prof["k_numerator"]
    num_ms = num_ms_total / args.steps
    peak_tf = _fp32_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
    fpu = flop_per_unit(info["kernel"], vx, info.get("taps", 5))
    achieved_tf = units_rank * fpu / (num_ms * 1e-3) / 1e12
    # the committed ncu figure holds for the profiled workload only: the
    # default paper-shaped search with the Gaussian footprint
    profiled = (T, H, args.vmax, kind) == (T_FR, HH, VMAX, 0)
    traffic_per_unit = _traffic_from_profiles(info["kernel"]) if profiled else None
    traffic = None if traffic_per_unit is None else traffic_per_unit * units_rank
    kernel_ms = {k: round(v[1] / args.steps, 3) for k, v in prof.items() if k != "_launches" and v[0]}
    launches = int(prof["_launches"])

    # end to end through the host-buffer entry point (mf_search_host): every
    # step uploads its stack from pinned host memory, searches, re-scores and
    # downloads the maps and candidates; uploads go on a copy stream and steps
    # alternate two workspaces (ordered by one event each), so one step's
    # upload overlaps the previous step's kernels on the compute stream (each
    # step's copies stay inside the timed region)
    e2e = None
    if not args.no_e2e:
        host = torch.empty((T, H, W), dtype=torch.float32, pin_memory=True)
        host.copy_(res)
        k_top = 0 if args.no_rescore else K_TOP
        comp, copy = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        frees = [torch.cuda.Event(), torch.cuda.Event()]
        wss = [torch.empty(mf.search_host_workspace_size(host, table, k_top), dtype=torch.uint8, device=dev)
               for _ in frees]
        outs = [(torch.empty((H, W), dtype=torch.float32, pin_memory=True),
                 torch.empty((H, W), dtype=torch.int32, pin_memory=True),
                 torch.zeros((k_top, mf.CANDIDATE_BYTES), dtype=torch.uint8, pin_memory=True) if k_top else None,
                 torch.zeros(1, dtype=torch.int32, pin_memory=True) if k_top else None) for _ in frees]
        # a streaming rate: the first step's upload (the pipeline fill, about
        # 80 ms at the host link's ~211 GB/s) is inside the timed region and
        # is spread over the run, so the run is long enough to amortise it
        e2e_steps = max(20, args.steps)
        # one untimed pass through each stream and workspace
        for i in range(2):
            mf.search_host(host, sigma, table, mask=mask, k_top=k_top, workspace=wss[i], out=outs[i],
                           stream=comp, copy_stream=copy, ws_free=frees[i])
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            j = i % 2
            mf.search_host(host, sigma, table, mask=mask, k_top=k_top, workspace=wss[j], out=outs[j],
                           stream=comp, copy_stream=copy, ws_free=frees[j])
        torch.cuda.synchronize(dev)
        e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dist, dev)
        same = bool(torch.equal(outs[(e2e_steps - 1) % 2][0], snr_max.cpu()))
        e2e = {"value": job_throughput(units_rank, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": T * H * W * 4,
               "d2h_bytes_per_step": H * W * 8 + (k_top * mf.CANDIDATE_BYTES + 4 if k_top else 0),
               "steps": e2e_steps, "call": "mf_search_host (pinned host stack in, host maps and candidates out)",
               "pipelined": "copy stream + compute stream, 2 workspaces: a step's upload overlaps the previous "
                            "step's kernels; the first upload (pipeline fill) is inside the timed region",
               "maps_equal_device_timed_run": same}
        del host, wss

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        sig_np = case["sigma_np"]
        msk_np = case["mask_np"]
        rate, cores, sample, (N, D, (y0, x0), side) = cpu_oracle_sample(res, sig_np, msk_np, vx, vy, T,
                                                                        budget_s=args.cpu_budget, kind=kind)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        # the same crop searched on the GPU just above: report the agreement
        import oracle
        snr = np.where(D > 0, N / np.sqrt(np.where(D > 0, D, 1)), -np.inf)
        o_max = snr.max(axis=2)
        g_max = snr_max[y0:y0 + side, x0:x0 + side].cpu().numpy().astype(np.float64)
        err = np.abs(g_max - o_max) / np.maximum(1.0, np.abs(o_max))
        parity = {"crop": [int(y0), int(x0), int(side)], "max_rel_err_snr_max": float(err.max()),
                  "tolerance": 1e-5}

    # the serving form and the precision form, each measured on its own after
    # the timed search (rank 0 at N = 1: they are single-GPU workloads)
    serve = precision = None
    if rank == 0 and ws == 1 and (not args.no_serve or not args.no_precision):
        del case, res, sigma, mask, ws_search, ws_rescore, snr_max, argmax
        torch.cuda.empty_cache()
        if not args.no_precision:
            precision = precision_measure(args, dev, T, H, W, 2, args.precision_px)
            precision["phase_quantised"] = quantised_measure(args, dev, T, H, W)
        if not args.no_serve:
            serve = serve_measure(args, dev, args.serve_duration, args.pool, extra_rates=(2 * args.rate,))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_RATE if profiled else None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper-shaped search: %d frames x %dx%d px float32, %d trajectories "
                                   "(%dx%d grid, |v|<=%.2f px/frame), sigma log-normal, 1%% star mask, "
                                   "200 movers; search + top-%d FP64 rescore per step%s" % (
                                       T, H, W, K, NXG, NYG, args.vmax, K_TOP,
                                       "; shift-stack filter (one tap per frame, Section 3.2)" if kind == 2 else ""),
                       "frames": T, "height": H, "width": W, "trajectories": K,
                       "l2": "inputs larger than L2 (%.1f GB stack per step)" % (T * H * W * 4 / 1e9),
                       "plan": {k: info[k] for k in ("kernel", "groups", "warps_per_group", "tile_h", "tile_w",
                                                      "window_pitch", "window_rows", "stages")},
                       "parallelism": "weak scaling: independent stack per GPU" if ws > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "kernel": "k_numerator_fac" if info["kernel"] == 2 else "k_numerator",
                         "achieved": achieved_tf, "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": achieved_tf / peak_tf, "traffic": traffic,
                         "traffic_source": None if traffic is None else (
                             "DRAM bytes per step: %.4f bytes per traj*pixel*frame from the ncu capture of the same "
                             "plan on 1000 x 512^2 (profiles/), times this step's units" % traffic_per_unit),
                         "peak_source": "%d SMs (device properties) x 128 FP32 lanes x 2 flop x %.0f MHz "
                                        "(sm_max_mhz, %s)" % (_sm_count(), float(peaks.get("sm_max_mhz", 2070.0)),
                                                              peak_src),
                         "flop_per_unit": fpu,
                         # the same launches counted at the general 5 x 5 form's
                         # 50 flop per unit: a rate of the search, not of the FP32 pipe
                         "general_form_equivalent_tflops": units_rank * FLOP_PER_UNIT_GENERAL / (num_ms * 1e-3) / 1e12,
                         "numerator_ms_per_step": num_ms,
                         "numerator_launches_per_step": num_launches // args.steps},
            "kernel_ms_per_step": kernel_ms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if parity:
            line["parity"] = parity
        if precision:
            line["precision"] = precision
        if serve:
            line["serve"] = serve
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _cutout(rng, dev, side, T, K, dtype, seed):
    """One cutout of the batched / serving workloads: config-2 statistics
    scaled to the cutout (movers in proportion to its area, at least 1)."""
    import torch

    from paper_2209_09848_gb300 import synth
    n_mov = max(1, int(round(200 * side * side / (2048 * 2048))))
    case = synth.paper_case_gpu(T=T, H=side, W=side, n_movers=n_mov, seed=seed, device=dev)
    nx = max(1, int(round(np.sqrt(K))))
    ny = max(1, int(round(K / nx)))
    vx, vy = synth.velocity_grid(nx, ny, -VMAX, VMAX)
    res = case["res"]
    if dtype == "bf16":
        res = res.to(torch.bfloat16)
    return dict(res=res, sigma=case["sigma"], mask=case["mask"], vx=vx, vy=vy, T=T, side=side)


def run_batch(args):
    """Batched form: uneven cutouts in one graph-captured persistent launch,
    layouts picked by the autotuner, against the same searches launched one
    at a time."""
    import torch

    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import _build, autotune
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(4)
    items = []
    for i in range(args.items):
        side = int(rng.choice([256, 512, 768, 1024]))
        T = int(rng.integers(300, 1301))
        K = int(rng.integers(50, 401))
        dt = "bf16" if rng.random() < 0.5 else "f32"
        items.append(_cutout(rng, dev, side, T, K, dt, 100 + i))
    units = sum(len(it["vx"]) * it["T"] * it["side"] ** 2 for it in items)
    t0 = time.perf_counter()
    for it in items:
        dtype = it["res"].dtype
        it["table"] = autotune.tuned_table(it["vx"], it["vy"], it["T"], it["side"], it["side"], dtype=dtype,
                                           crop=256, reps=1)
    tune_s = time.perf_counter() - t0
    b = mf.Batch()
    for it in items:
        b.add(it["res"], it["sigma"], it["table"], mask=it["mask"])
    b.prepare(device=dev)
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / args.steps
    # the same searches, one launch sequence per cutout
    e0.record()
    for it in items:
        mf.search(it["res"], it["sigma"], it["table"], mask=it["mask"])
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    ok = all(torch.equal(o[0], mf.search(it["res"], it["sigma"], it["table"], mask=it["mask"])[0])
             for o, it in list(zip(b.outputs, items))[:4])
    line = {"metric": "traj*pixel*frame/s, %d uneven cutouts in one graph-captured persistent launch" % len(items),
            "value": units / (ms_batch * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 and bf16 storage, f32 arithmetic", "data": "synthetic",
            "config": {"workload": "batched form: sides {256,512,768,1024}^2, frames 300-1300, 50-400 "
                                   "trajectories each, fp32 or bf16 (coin flip), sigma/mask/movers as the "
                                   "paper-shaped stack", "items": len(items), "units": units,
                       "autotune_s": tune_s, "info": b.info()},
            "one_launch_per_cutout": {"value": units / (ms_seq * 1e-3), "ms": ms_seq},
            "speedup_vs_one_launch_per_cutout": ms_seq / ms_batch,
            "batch_equals_single_search": bool(ok)}
    print(json.dumps(line), flush=True)
    return 0


def serve_measure(args, dev, duration, pool_n, rate=None, extra_rates=()):
    """Serving form: Poisson request stream, admission by footprint against
    a memory budget, continuous batching on several streams; p50/p99 latency
    and throughput, against the same stream served one request at a time.
    Requests are drawn from `pool_n` distinct pregenerated cutouts (each a
    config-2-like stack of its own size, frame count and trajectory grid).
    `extra_rates`: further mean arrival rates run on the same pool (to show
    how the two schedules hold up as the offered load grows)."""
    import torch

    from paper_2209_09848_gb300.serve import Request, Server, percentile
    rate = args.rate if rate is None else rate
    rng = np.random.default_rng(5)
    pool = []
    for i in range(pool_n):
        side = int(rng.choice([256, 512, 768, 1024]))
        T = int(rng.integers(300, 1301))
        K = int(rng.integers(10, 201))
        dt = "bf16" if rng.random() < 0.5 else "f32"
        c = _cutout(rng, dev, side, T, K, dt, 500 + i)
        req = Request(stack=c["res"].cpu().pin_memory(), sigma=c["sigma"].cpu().pin_memory(),
                      vx=c["vx"], vy=c["vy"], mask=c["mask"].cpu().pin_memory(), k_top=64,
                      tag=(len(c["vx"]) * T * side * side))
        pool.append(req)
        del c
    torch.cuda.empty_cache()

    def serve(streams, arrivals, picks):
        srv = Server(budget_bytes=int(args.budget_gb * 1e9), streams=streams, planners=8, device=dev)
        # warm the planners and the allocator on one request
        srv.submit(pool[0]).result()
        futs = []
        t0 = time.perf_counter()
        for t_arr, k in zip(arrivals, picks):
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            futs.append(srv.submit(pool[k]))
        res = [f.result() for f in futs]
        srv.close()
        lat = [r.latency * 1e3 for r in res]
        span = max(r.done for r in res) - min(r.arrival for r in res)
        units = sum(r.tag for r in res)
        return {"p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "mean_ms": float(np.mean(lat)),
                "throughput": units / span, "unit": UNIT, "requests": len(res), "span_s": span,
                "peak_bytes": srv.peak, "failed": srv.failed}

    def stream(r, dur):
        n_req = int(r * dur)
        arrivals = np.cumsum(rng.exponential(1.0 / r, n_req))
        picks = rng.integers(0, len(pool), n_req)
        offered = sum(pool[k].tag for k in picks) / dur
        return arrivals, picks, offered

    arr, picks, offered = stream(rate, duration)
    mix = serve(args.streams, arr, picks)
    one = serve(1, arr, picks)
    out = {"p50_ms": mix["p50_ms"], "p99_ms": mix["p99_ms"], "throughput": mix["throughput"], "unit": UNIT,
           "workload": "Poisson %.0f req/s for %.0f s (%d requests), cutouts as the batched form (sides "
                       "{256,512,768,1024}, 300-1300 frames, fp32 or bf16) with 10-200 trajectories, top-64 FP64 "
                       "rescore each, budget %.0f GB, %d streams; requests drawn from %d distinct pregenerated "
                       "cutouts" % (rate, duration, len(picks), args.budget_gb, args.streams, pool_n),
           "offered": offered, "distinct_requests": pool_n, "served": mix, "one_request_at_a_time": one}
    for r2 in extra_rates:
        arr, picks, offered = stream(r2, duration)
        out["at_%g_per_s" % r2] = {"offered": offered, "served": serve(args.streams, arr, picks),
                                   "one_request_at_a_time": serve(1, arr, picks)}
    del pool
    torch.cuda.empty_cache()
    return out


def run_serve(args):
    """The serving form alone, as its own JSON line."""
    import torch

    from paper_2209_09848_gb300 import _build
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = serve_measure(args, dev, args.duration, args.pool)
    mix = r["served"]
    line = {"metric": "serve p50/p99 latency (ms) and traj*pixel*frame/s under a Poisson request stream",
            "value": mix["throughput"], "unit": UNIT, "n_gpus": 1, "steps": mix["requests"],
            "warmup": 1, "ms_per_step": mix["mean_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 and bf16 storage, f32 arithmetic", "data": "synthetic",
            "config": {"workload": "serving form: " + r["workload"], "distinct_requests": args.pool},
            "serve": mix, "one_request_at_a_time": r["one_request_at_a_time"]}
    print(json.dumps(line), flush=True)
    return 0


def precision_measure(args, dev, T, H, W, steps, n_px):
    """Precision form: the paper-shaped stack stored as FP32, BF16 (scale 1)
    and FP16 (per-frame scale max|r_t| / 2^14), 1000 trajectories (40 x 25
    grid), FP32 accumulation; a bf16 / fp16 stack's weighted copy stays
    16-bit.  For each form: its rate, its workspace and stack bytes, and on
    sampled start pixels (every trajectory) the SNR error against the FP64
    oracle evaluated on the FP32 master (the error the storage costs) and
    against the oracle of the form itself (the oracle's 16-bit weighted
    stack: the kernel's own error); plus the FP64 re-score from the FP32
    master on 64 pixels chosen from a host-generated score map."""
    import torch

    import oracle
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import synth
    oracle.build()
    case = synth.paper_case_gpu(T=T, H=H, W=W, seed=3, device=dev)
    vx, vy = synth.velocity_grid(40, 25, -args.vmax, args.vmax)
    K = len(vx)
    table = mf.prf_table_create(vx, vy, T)
    master = case["res"]
    scale16 = (master.abs().amax(dim=(1, 2)) / 2.0 ** 14).float().contiguous()
    forms = {"f32": (master, None), "bf16": (master.to(torch.bfloat16), None),
             "f16": ((master / scale16[:, None, None]).to(torch.float16), scale16)}
    rng = np.random.default_rng(11)
    ys = rng.integers(0, H, n_px).astype(np.int32)
    xs = rng.integers(0, W, n_px).astype(np.int32)
    pys, pxs = np.repeat(ys, K), np.repeat(xs, K)
    pks = np.tile(np.arange(K, dtype=np.int32), n_px)
    res_host = master.cpu().numpy()
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(case["sigma_np"], case["mask_np"])

    def best(N, D):
        N = N.reshape(n_px, K)
        D = D.reshape(n_px, K)
        snr = np.where(D > 0, N / np.sqrt(np.where(D > 0, D, 1.0)), 0.0)
        return np.where(D > 0, snr, -np.inf).max(axis=1)

    t0 = time.perf_counter()
    o_max = best(*oracle.search_points(res_host, lam, sh, tp, pys, pxs, pks))
    oracle_s = time.perf_counter() - t0
    chk_s, chk_a = synth.score_map(H, W, seed=21, K=K, mask_frac=0.0)
    chk_want = oracle.topk_order(chk_s, chk_a, 64)
    Nc, Dc = oracle.search_points(res_host, lam, sh, tp, (chk_want // W).astype(np.int32),
                                  (chk_want % W).astype(np.int32), chk_a.ravel()[chk_want])
    out = {}
    peaks, _ = _peaks()
    peak_tf = _fp32_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)))
    units = K * T * H * W
    mf.profile_enable(True)
    for name, (stack, fs) in forms.items():
        ws_bytes = mf.search_workspace_size((T, H, W), table, stack.dtype)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        smax = torch.empty((H, W), device=dev)
        amax = torch.empty((H, W), dtype=torch.int32, device=dev)
        mf.search(stack, case["sigma"], table, mask=case["mask"], frame_scale=fs, workspace=ws, out=(smax, amax, None))
        torch.cuda.synchronize()
        mf.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            mf.search(stack, case["sigma"], table, mask=case["mask"], frame_scale=fs, workspace=ws,
                      out=(smax, amax, None))
            raw, n = mf.rescore_topk(master, case["sigma"], table, smax, amax, K_TOP, mask=case["mask"])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = mf.profile_read(reset=True)
        num_ms = prof["k_numerator"][1] / steps  # per step: one launch per time segment
        g_max = smax.cpu().numpy()[ys, xs].astype(np.float64)
        err = np.abs(g_max - o_max) / np.maximum(1.0, np.abs(o_max))
        form_err = None
        if name != "f32":
            # the oracle of the precision form: its 16-bit weighted stack
            q, beta = oracle.weighted_stack16(stack.float().cpu().numpy(), case["sigma_np"], case["mask_np"],
                                              None if fs is None else fs.cpu().numpy(),
                                              "bf16" if name == "bf16" else "fp16")
            f_max = best(*oracle.search_weighted_points(q, beta, lam, sh, tp, pys, pxs, pks))
            del q
            form_err = float((np.abs(g_max - f_max) / np.maximum(1.0, np.abs(f_max))).max())
        # the FP64 re-score on 64 pixels chosen from a host-generated score
        # map (the oracle is evaluated at its own selection of them)
        raw64, n64 = mf.rescore_topk(master, case["sigma"], table, torch.from_numpy(chk_s).to(dev),
                                     torch.from_numpy(chk_a).to(dev), 64, mask=case["mask"])
        cands = mf.decode_candidates(raw64, int(n64.item()))
        ok = Dc > 0
        rerr = np.abs(cands["snr"][ok] - Nc[ok] / np.sqrt(Dc[ok])) / np.maximum(1.0, np.abs(Nc[ok] / np.sqrt(Dc[ok])))
        y_bytes = T * H * W * (4 if name == "f32" or table.info()["kernel"] != 2 else 2)
        out[name] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "numerator_ms": num_ms,
                     "frac": units * flop_per_unit(table.info()["kernel"], vx) / (num_ms * 1e-3) / 1e12 / peak_tf,
                     "stack_gb": stack.numel() * stack.element_size() / 1e9,
                     "workspace_gb": ws_bytes / 1e9, "weighted_stack_gb": y_bytes / 1e9,
                     "numerator_algorithmic_dram_gb": y_bytes / 1e9,
                     "snr_max_rel_err_vs_fp64_oracle_on_fp32_master": {"max": float(err.max()),
                                                                       "median": float(np.median(err))},
                     "snr_max_rel_err_vs_oracle_of_this_form": form_err,
                     "fp64_rescore_rel_err": float(rerr.max()) if ok.any() else None,
                     "rescore_selection_equals_oracle": bool(np.array_equal(
                         cands["y"].astype(np.int64) * W + cands["x"], chk_want))}
        del ws
        torch.cuda.empty_cache()
    mf.profile_enable(False)
    del case, master, forms
    torch.cuda.empty_cache()
    return {"workload": "%d frames x %dx%d, %d trajectories (40x25 grid, |v|<=%.2f), search + top-%d FP64 rescore "
                        "from the FP32 master; %d steps per form" % (T, H, W, K, args.vmax, K_TOP, steps),
            "error_sample": "%d random start pixels x all trajectories, FP64 oracle on the FP32 master (%.1f s)"
                            % (n_px, oracle_s),
            "forms": out}


def quantised_measure(args, dev, T, H, W, Q=4, steps=1):
    """The phase-quantised bank on the 1000-trajectory grid (40 x 25, the
    precision form's): the exact bank with column passes, the quantised bank
    (phases rounded to multiples of 1/Q) with column passes and with the
    precompute-then-gather numerator (phase planes); the quantisation loss
    as the SNR at the 200 injected movers' start pixels, quantised over
    exact (the movers' velocities are off the grid, as in the paper's
    injections)."""
    import torch

    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import synth
    case = synth.paper_case_gpu(T=T, H=H, W=W, seed=3, device=dev)
    vx, vy = synth.velocity_grid(40, 25, -args.vmax, args.vmax)
    K = len(vx)
    units = K * T * H * W
    mv = case["movers"]
    my = np.clip(np.round(mv[:, 0]).astype(np.int64), 0, H - 1)
    mx = np.clip(np.round(mv[:, 1]).astype(np.int64), 0, W - 1)
    out, at_movers = {}, {}
    mf.profile_enable(True)
    for name, kw in (("exact_column_passes", {}), ("quantised_column_passes", dict(phase_steps=Q, kernel=2)),
                     ("quantised_phase_planes", dict(phase_steps=Q, kernel=3))):
        tab = mf.prf_table_create(vx, vy, T, **kw)
        ws = torch.empty(mf.search_workspace_size((T, H, W), tab), dtype=torch.uint8, device=dev)
        smax = torch.empty((H, W), device=dev)
        amax = torch.empty((H, W), dtype=torch.int32, device=dev)
        mf.search(case["res"], case["sigma"], tab, mask=case["mask"], workspace=ws, out=(smax, amax, None))
        torch.cuda.synchronize()
        mf.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            mf.search(case["res"], case["sigma"], tab, mask=case["mask"], workspace=ws, out=(smax, amax, None))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = mf.profile_read(reset=True)
        info = tab.info()
        out[name] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "numerator_ms": prof["k_numerator"][1] / steps, "phase_planes": info["phase_planes"],
                     "plan": {x: info[x] for x in ("groups", "warps_per_group", "tile_h", "window_rows")}}
        at_movers[name] = smax.cpu().numpy()[my, mx].astype(np.float64)
        del ws, tab
        torch.cuda.empty_cache()
    mf.profile_enable(False)
    del case
    torch.cuda.empty_cache()
    ratio = at_movers["quantised_column_passes"] / np.where(at_movers["exact_column_passes"] > 0,
                                                             at_movers["exact_column_passes"], np.nan)
    return {"workload": "%d frames x %dx%d float32, %d trajectories (40x25 grid), Q = %d, search only, %d step(s)"
                        % (T, H, W, K, Q, steps), "forms": out,
            "quantisation_loss": {"snr_max_at_movers_quantised_over_exact_median": float(np.nanmedian(ratio)),
                                  "min": float(np.nanmin(ratio)), "movers": int(len(my))}}


def run_precision(args):
    """The precision forms alone, as their own JSON line."""
    import torch

    from paper_2209_09848_gb300 import _build
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    T, H, W = args.frames, args.size, args.size
    r = precision_measure(args, dev, T, H, W, args.steps, args.sample_px)
    out = r["forms"]
    K = 1000
    line = {"metric": "traj*pixel*frame/s, precision forms at %dx%d^2x%d traj" % (T, H, K), "value": out["bf16"]["value"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": out["bf16"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 storage (f32 and f16 alongside), f32 arithmetic", "data": "synthetic",
            "config": {"workload": "precision form: " + r["workload"], "error_sample": r["error_sample"]},
            "forms": out, "phase_quantised": quantised_measure(args, dev, T, H, W)}
    print(json.dumps(line), flush=True)
    return 0


def run_refit(args):
    """Per-pixel background re-fit (Section 3.1): 1000 raw frames of 2048 x
    2048 (synthetic scene: scattered light on a 64 x 64 grid, background
    with jitter Taylor terms, noise, outliers), Huber delta 1.345, 10
    clipped steps after the least-squares start.  Device timing with CUDA
    events (16.8 GB of frames, far above L2); parity on sampled pixels
    against the FP64 oracle; end to end with the frames uploaded from pinned
    host memory and the coefficient maps read back each step."""
    import torch

    import oracle
    from oracle import background as ob
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import _build, synth
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    T, H, W = args.frames, args.size, args.size
    M, delta = 10, 1.345
    c = synth.background_case_gpu(T=T, H=H, W=W, seed=7, n=64, device=dev)
    D, S, jit = c["D"], c["S"], c["jitter"]
    R = torch.empty_like(D)
    ws = torch.empty(mf.refit_workspace_size(T), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return mf.background_refit(D, jit, delta, M, scatter=S, resid=R, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if mf.device_status() != 0:
        raise SystemExit("device status word set during warm-up")
    mf.profile_enable(True)
    mf.profile_read(reset=True)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, coef = step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = mf.profile_read(reset=True)
    mf.profile_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    units = T * H * W
    # parity on sampled pixels
    rng = np.random.default_rng(3)
    ys = rng.integers(0, H, args.sample_px)
    xs = rng.integers(0, W, args.sample_px)
    iy, ix = torch.as_tensor(ys, device=dev), torch.as_tensor(xs, device=dev)
    Dp = D[:, iy, ix].cpu().numpy()
    Rp = R[:, iy, ix].cpu().numpy()
    Sh = S.cpu().numpy()
    t0 = time.perf_counter()
    co, Ro = ob.refit_points(Dp, ys, xs, H, W, jit, delta, M, S=Sh)
    cpu_s = time.perf_counter() - t0
    err = float(np.abs(Rp.astype(np.float64) - Ro).max())
    tol = 2e-6 * float(np.abs(Dp).max())
    # end to end: frames from pinned host memory, coefficients back
    D_h = D.cpu().pin_memory()
    coef_h = torch.empty((H, W, 6), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(e2e_steps):
        D.copy_(D_h, non_blocking=True)
        _, coef = step()
        coef_h.copy_(coef, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3) / e2e_steps
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    k_ms = prof["k_refit"][1] / args.steps
    alg_bytes = (M + 3) * 4.0  # M + 2 reads of the series, one write of the residual
    line = {"metric": "pixel*frame/s, per-pixel background re-fit (Huber, jitter Taylor basis)",
            "value": units / (ms * 1e-3), "unit": "pixel*frame/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (basis and coefficients f64 on the host)", "data": "synthetic",
            "config": {"workload": "background re-fit: %d frames x %dx%d raw, scattered light on 64x64, "
                                   "delta %.3f, %d clipped steps" % (T, H, W, delta, M),
                       "l2": "inputs larger than L2 (%.1f GB of frames)" % (units * 4 / 1e9)},
            "roofline": {"bound": "hbm", "kernel": "k_refit",
                         "achieved": alg_bytes * units / (k_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg_bytes * units / (k_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                         "peak_source": peak_src, "bytes_per_unit": alg_bytes,
                         "implementation_bytes_per_unit": (M + 4) * 4.0, "kernel_ms": k_ms},
            "parity": {"pixels": int(args.sample_px), "max_abs_err_residual": err, "tolerance": tol},
            "cpu_baseline": {"value": args.sample_px * T / cpu_s, "unit": "pixel*frame/s", "cores": 1,
                             "kind": "oracle", "sample": "%d random pixels x %d frames (numpy FP64)"
                                                         % (args.sample_px, T)},
            "e2e": {"value": units / (e2e_ms * 1e-3), "unit": "pixel*frame/s", "h2d_bytes_per_step": units * 4,
                    "d2h_bytes_per_step": H * W * 6 * 4},
            "gpu_launches": int(prof["_launches"]), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_detect(args):
    """Detection stage (Section 3.3): a 2048 x 2048 best-score map (the
    search's output shape; synthetic score statistics) normalised by the
    local 255 x 255 sigma, 3 sigma candidates grouped into detections.
    Device timing with CUDA events per step, L2 flushed between steps (the
    256 MB of intermediate maps exceed L2, the 32 MB input does not);
    end to end through mf_detect with the maps uploaded from pinned host
    memory and the detections and counts read back each step."""
    import torch

    import oracle
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import _build, synth
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H = W = args.size
    window, thr, max_out = 255, 3.0, 4096
    s_np, a_np = synth.score_map(H, W, seed=3, K=100)
    s_h = torch.from_numpy(s_np).pin_memory()
    a_h = torch.from_numpy(a_np).pin_memory()
    smax, amax = s_h.to(dev), a_h.to(dev)
    z = torch.empty((H, W), dtype=torch.float32, device=dev)
    ws = torch.empty(mf.detect_workspace_size(H, W, max_out), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return mf.detect(smax, amax, window=window, threshold=thr, max_out=max_out, z_out=z, workspace=ws,
                         stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if mf.device_status() != 0:
        raise SystemExit("device status word set during warm-up")
    mf.profile_enable(True)
    mf.profile_read(reset=True)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    steps = max(args.steps, 20)
    total = 0.0
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        raw, n = step()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    clocks = sampler.stop()
    prof = mf.profile_read(reset=True)
    mf.profile_enable(False)
    ms = total / steps
    found, written = (int(v) for v in n.cpu().tolist())
    # end to end: upload the maps, detect, read the detections and counts back
    out_h = torch.empty((max_out, mf.DETECTION_BYTES), dtype=torch.uint8, pin_memory=True)
    n_h = torch.empty(2, dtype=torch.int32, pin_memory=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        smax.copy_(s_h, non_blocking=True)
        amax.copy_(a_h, non_blocking=True)
        raw, n = step()
        out_h.copy_(raw[:max_out], non_blocking=True)
        n_h.copy_(n, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / steps
    # oracle on the host cores: the same map once
    t0 = time.perf_counter()
    det_o, _, _ = oracle.detections(s_np, a_np, window=window, threshold=thr)
    cpu_s = time.perf_counter() - t0
    det_g = mf.decode_detections(raw, written)
    P = H * W
    peaks, peak_src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    stats_ms = prof["k_det_stats"][1] / steps
    # algorithmic bytes of the stage: the score and argmax maps read once, the
    # z map written once (12 B per pixel); the statistics kernels' share of it
    line = {"metric": "pixel/s, detection stage (local 255x255 sigma, 3 sigma, 8-connected detections)",
            "value": P / (ms * 1e-3), "unit": "pixel/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 statistics, f32 z", "data": "synthetic",
            "config": {"workload": "detection: %dx%d best-score map (noise ~2.5 +- 0.45 with a gradient, 1%% masked, "
                                   "%d compact sources), window %d, threshold %.1f, mean subtracted, max_out %d"
                                   % (H, W, min(200, P // 400), window, thr, max_out),
                       "l2": "flushed between steps (256 MB write)"},
            "roofline": {"bound": "hbm", "kernel": "k_det_cols + k_det_rows",
                         "achieved": 12.0 * P / (stats_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": 12.0 * P / (stats_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                         "peak_source": peak_src, "bytes_per_pixel": 12, "stats_ms": stats_ms},
            "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in prof.items()
                                   if not k.startswith("_") and v[0]},
            "detections": {"found": found, "written": written, "oracle_found": int(len(det_o)),
                           "peaks_equal_oracle_top64": bool(np.array_equal(
                               (det_g["y"][:64], det_g["x"][:64]), (det_o["y"][:64], det_o["x"][:64])))},
            "cpu_baseline": {"value": P / cpu_s, "unit": "pixel/s", "cores": 1, "kind": "oracle",
                             "sample": "the whole %dx%d map once (numpy summed-area tables, scipy labels)" % (H, W)},
            "e2e": {"value": P / (e2e_ms * 1e-3), "unit": "pixel/s", "h2d_bytes_per_step": 8 * P,
                    "d2h_bytes_per_step": max_out * mf.DETECTION_BYTES + 8},
            "gpu_launches": int(prof["_launches"]), "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=T_FR)
    ap.add_argument("--size", type=int, default=HH)
    ap.add_argument("--vmax", type=float, default=VMAX, help="velocity grid half-range, px/frame")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-rescore", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--prf", choices=["gauss", "shiftstack"], default="gauss",
                    help="filter footprint: the Gaussian PRF, or the single-tap shift-stack filter")
    ap.add_argument("--kernel", type=int, choices=[0, 1, 2], default=0,
                    help="numerator: 0 planner's choice, 1 general 5x5, 2 factored")
    ap.add_argument("--workload", choices=["search", "batch", "serve", "precision", "detect", "refit"],
                    default="search",
                    help="search: the paper-shaped search (default); batch / serve: the batched and serving forms")
    ap.add_argument("--items", type=int, default=64, help="batch: cutouts in the batch")
    ap.add_argument("--pool", type=int, default=32, help="serve: distinct pregenerated requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve workload: seconds of arrivals")
    ap.add_argument("--serve-duration", type=float, default=15.0,
                    help="seconds of arrivals of the serving form in the default line")
    ap.add_argument("--no-serve", action="store_true", help="default line without the serving form")
    ap.add_argument("--no-precision", action="store_true", help="default line without the precision forms")
    ap.add_argument("--precision-px", type=int, default=128,
                    help="start pixels of the precision forms' error sample in the default line")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve: admission budget")
    ap.add_argument("--streams", type=int, default=4, help="serve: searches in flight")
    ap.add_argument("--sample-px", type=int, default=256, help="precision: start pixels checked against the oracle")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "detect":
        return run_detect(args)
    if args.workload == "refit":
        return run_refit(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
