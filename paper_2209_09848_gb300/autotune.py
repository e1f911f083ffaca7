"""Autotuner for the numerator's layout (not in the paper).

For a filter bank and a cutout size it times candidate layouts the library
can hold in shared memory -- the factored numerator with the planner's
geometry and with each tile width, and the general numerator with the
planner's CTA shape and with each frame hand-off -- on a sample stack of the
same frame count and dtype, and keeps the fastest.  Results are cached per
(frames, sample size, trajectories, dtype, velocity span) bucket, so a stream
of similar requests is tuned once.  Timing uses CUDA events around
mf_search; every candidate runs the library's kernels.
"""
from __future__ import annotations

import threading

import numpy as np
import torch

from . import binding as mf

CANDIDATES = [
    {"kernel": 2},
    {"kernel": 2, "tile_w": 32},
    {"kernel": 2, "tile_w": 64},
    {"kernel": 1, "lockstep": 0},
    {"kernel": 1, "lockstep": 1},
]
_cache: dict = {}
_lock = threading.Lock()


def _key(vx, vy, T, H, W, dtype, crop):
    span = float(max(np.ptp(vx) if len(vx) else 0.0, np.ptp(vy) if len(vy) else 0.0) * T)
    return (int(T) // 50, min(H, crop) // 64, min(W, crop) // 64, (len(vx) + 7) // 8, str(dtype),
            int(span // 8))


def tune(vx, vy, T, H, W, dtype=torch.float32, crop=512, reps=2, sigma_px=0.7, device="cuda", verbose=False):
    """Return (best layout options, timings {candidate index: ms}) for this
    bank and cutout size; cached by bucket.  The options are keyword
    arguments of prf_table_create."""
    key = _key(vx, vy, T, H, W, dtype, crop)
    with _lock:
        if key in _cache:
            return _cache[key]
    h, w = min(H, crop), min(W, crop)
    g = torch.Generator(device=device)
    g.manual_seed(1234)
    stack = torch.randn((T, h, w), generator=g, device=device).to(dtype)
    sigma = torch.ones((h, w), device=device)
    timings = {}
    seen = set()
    for i, opts in enumerate(CANDIDATES):
        try:
            table = mf.prf_table_create(vx, vy, T, sigma_px=sigma_px, **opts)
        except mf.MFError:
            continue  # this layout cannot hold the windows
        inf = table.info()
        sig = (inf["kernel"], inf["warps_per_group"], inf["tile_h"], inf["tile_w"], inf["lockstep"], inf["stages"])
        if sig in seen:
            continue  # the same layout as an earlier candidate
        seen.add(sig)
        ws = torch.empty(mf.search_workspace_size((T, h, w), table), dtype=torch.uint8, device=device)
        out = (torch.empty((h, w), device=device), torch.empty((h, w), dtype=torch.int32, device=device), None)
        mf.search(stack, sigma, table, workspace=ws, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            mf.search(stack, sigma, table, workspace=ws, out=out)
        e1.record()
        torch.cuda.synchronize()
        timings[i] = e0.elapsed_time(e1) / reps
        del table, ws
    if not timings:
        raise mf.MFError(5, "no numerator layout fits this filter bank")
    best = min(timings, key=timings.get)
    res = (dict(CANDIDATES[best]), timings)
    if verbose:
        print("autotune", key, "->", CANDIDATES[best], {i: round(v, 3) for i, v in timings.items()})
    with _lock:
        _cache[key] = res
    return res


def tuned_table(vx, vy, T, H, W, dtype=torch.float32, sigma_px=0.7, **kw):
    """Filter bank built with the layout the autotuner picked."""
    opts, _ = tune(vx, vy, T, H, W, dtype=dtype, sigma_px=sigma_px, **kw)
    return mf.prf_table_create(vx, vy, T, sigma_px=sigma_px, **opts)


def clear_cache():
    with _lock:
        _cache.clear()
