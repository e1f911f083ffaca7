"""Autotuner for the numerator's CTA layout (not in the paper).

For a filter bank and a cutout size it times every layout the library can
hold in shared memory -- CTA shape (trajectories per CTA x 32 x 32 sub-tiles)
and frame hand-off (last-warp refill or CTA barrier) -- on a sample stack of
the same frame count and dtype, and keeps the fastest.  Results are cached
per (frames, sample size, trajectories, dtype, velocity span) bucket, so a
stream of similar requests is tuned once.  Timing uses CUDA events around
mf_search; every candidate runs the library's kernels.
"""
from __future__ import annotations

import threading

import numpy as np
import torch

from . import binding as mf

CANDIDATES = [(shape, lock) for shape in (0, 1, 2, 3) for lock in (0, 1)]
_cache: dict = {}
_lock = threading.Lock()


def _key(vx, vy, T, H, W, dtype, crop):
    span = float(max(np.ptp(vx) if len(vx) else 0.0, np.ptp(vy) if len(vy) else 0.0) * T)
    return (int(T) // 50, min(H, crop) // 64, min(W, crop) // 64, (len(vx) + 7) // 8, str(dtype),
            int(span // 8))


def tune(vx, vy, T, H, W, dtype=torch.float32, crop=512, reps=2, sigma_px=0.7, device="cuda", verbose=False):
    """Return (best options dict, timings {(shape, lockstep): ms}) for this
    bank and cutout size; cached by bucket."""
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
    for shape, lock in CANDIDATES:
        try:
            table = mf.prf_table_create(vx, vy, T, sigma_px=sigma_px, shape=shape, lockstep=lock)
        except mf.MFError:
            continue  # this layout cannot hold the windows
        ws = torch.empty(mf.search_workspace_size((T, h, w), table), dtype=torch.uint8, device=device)
        out = (torch.empty((h, w), device=device), torch.empty((h, w), dtype=torch.int32, device=device), None)
        mf.search(stack, sigma, table, workspace=ws, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            mf.search(stack, sigma, table, workspace=ws, out=out)
        e1.record()
        torch.cuda.synchronize()
        timings[(shape, lock)] = e0.elapsed_time(e1) / reps
        del table, ws
    if not timings:
        raise mf.MFError(5, "no numerator layout fits this filter bank")
    best = min(timings, key=timings.get)
    res = ({"shape": best[0], "lockstep": best[1]}, timings)
    if verbose:
        print("autotune", key, "->", best, {k: round(v, 3) for k, v in timings.items()})
    with _lock:
        _cache[key] = res
    return res


def tuned_table(vx, vy, T, H, W, dtype=torch.float32, sigma_px=0.7, **kw):
    """Filter bank built with the layout the autotuner picked."""
    opts, _ = tune(vx, vy, T, H, W, dtype=dtype, sigma_px=sigma_px, **kw)
    return mf.prf_table_create(vx, vy, T, sigma_px=sigma_px, shape=opts["shape"], lockstep=opts["lockstep"])


def clear_cache():
    with _lock:
        _cache.clear()
