"""FP64 CPU oracle for the trajectory matched filter of Ganapathi (2022).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module.  It shares no code with the CUDA library; the C part
(``mf_oracle.c``) includes only the C standard library.

Functions and the passages they follow:

* ``prf_taps``, ``trajectory_table`` -- Section 2 (the PRF spreads a point
  source over neighbouring pixels; trajectories are straight lines in pixel
  space) and Section 3.2 (a filter is the trajectory line convolved with the
  PRF).  Gaussian PRF of width ``sigma_prf``, 5x5 footprint, renormalised;
  kind 2 is the shift-stack filter (Section 3.2: a single 1 in the pixel
  holding the source's centre).
* ``trajectory_table_quantised`` -- the filter bank of a phase-quantised
  precompute-then-gather search (Section 3.2 expects a sparse formulation
  to be much faster): footprints at phases rounded to multiples of 1/Q;
  ``search_quantised_gather`` computes that search in its own order (each
  frame correlated once per rounded phase, then one gather per trajectory).
* ``trajectory_table_frames`` -- the same with each frame's time (Fig. 3:
  the downlink gap makes time jump) and the pointing jitter (Section 2.1;
  Section 3.2: the filter follows the trajectory including the jitter).
* ``inverse_variance`` -- Section 3.2 (Gaussian noise of known width; bright
  pixels are clipped, read here as excluded: weight 0).  A pixel whose noise
  is not a finite number above 0 is excluded the same way.
* ``search_full`` / ``search_points`` -- Section 3.2, Eq. 5 (dot product of
  the filter with the data at every pixel location), in the C oracle.
* ``snr_and_best`` -- Section 3.2 (maximum score over the filter bank gives
  the most likely trajectory); score normalised to SNR = N / sqrt(D).
* ``dense_template`` / ``search_dense`` -- a second, paper-literal
  implementation for tiny inputs: it builds each filter as a full T x H x W
  tensor (Section 3.2: F in R^{R x C x T}) and takes the dot product.
* ``inject`` -- Section 4.1 (injection adds a filter times a flux).
* ``weighted_stack16`` / ``search_weighted`` -- the precision form (not in
  the paper; 16-bit storage of the stack): the inverse-variance weighted
  residual of Section 3.2 formed in FP32 and rounded to the stack's 16-bit
  type, then the matched filter on it.
* ``search_numpy`` -- a third implementation of the same definition, with
  numpy slicing over whole frames (used to cross-check the C loops).

Parity is pinned by ``tests/test_oracle.py`` against closed forms, library
routines (scipy quadrature and 2-D correlation), brute force and the
statistics of the matched filter on pure noise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "prf_taps", "trajectory_table", "trajectory_table_frames", "trajectory_table_quantised",
    "inverse_variance", "search_full",
    "search_points", "snr_and_best", "dense_template", "search_dense", "inject",
    "search_numpy", "search_quantised_gather", "topk_order", "threads", "round_to_bf16", "weighted_stack16",
    "search_weighted", "search_weighted_points",
]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over output pixels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i = ctypes.c_int
            d = ctypes.c_double
            lib.orc_prf_taps.argtypes = [d, d, d, i, P]
            lib.orc_pixel_integrated_gauss.argtypes = [i, d, d]
            lib.orc_pixel_integrated_gauss.restype = d
            lib.orc_trajectory_table.argtypes = [i, i, P, P, d, i, P, P]
            lib.orc_trajectory_table_frames.argtypes = [i, i, P, P, P, P, P, d, i, i, P, P]
            lib.orc_trajectory_table_quantised.argtypes = [i, i, P, P, d, i, i, P, P]
            lib.orc_inverse_variance.argtypes = [i, i, P, P, P]
            lib.orc_search_full.argtypes = [i, i, i, P, P, P, i, P, P, P, P]
            lib.orc_search_points.argtypes = [i, i, i, P, P, P, P, P, ctypes.c_long,
                                              P, P, P, P, P]
            _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the C oracle will use."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pixel_integrated_gauss(a: int, phase: float, sigma: float) -> float:
    return _load().orc_pixel_integrated_gauss(int(a), float(phase), float(sigma))


def prf_taps(phx: float, phy: float, sigma: float = 0.7, kind: int = 0) -> np.ndarray:
    """5x5 PRF footprint, ``out[dy + 2, dx + 2]``; sums to 1."""
    out = np.zeros(25, np.float64)
    _load().orc_prf_taps(float(phx), float(phy), float(sigma), int(kind), _ptr(out))
    return out.reshape(5, 5)


def trajectory_table(vx, vy, T: int, sigma: float = 0.7, kind: int = 0):
    """Filter bank in sparse form for linear trajectories.

    Returns ``shifts`` int32 [K, T, 2] (s_x, s_y) and ``taps`` float64
    [K, T, 5, 5] with ``taps[k, t, dy + 2, dx + 2]``.
    """
    vx = np.ascontiguousarray(vx, np.float64)
    vy = np.ascontiguousarray(vy, np.float64)
    K = vx.shape[0]
    shifts = np.zeros((K, T, 2), np.int32)
    taps = np.zeros((K, T, 5, 5), np.float64)
    _load().orc_trajectory_table(K, int(T), _ptr(vx), _ptr(vy), float(sigma), int(kind),
                                 _ptr(shifts), _ptr(taps))
    return shifts, taps


def trajectory_table_frames(vx, vy, T: int, times=None, jitter=None, sigma: float = 0.7, kind: int = 0,
                            Q: int = 0):
    """As ``trajectory_table`` with frame times and pointing jitter (Section
    2.1 and Fig. 3): position c = v * times[t] + jitter[t].  ``times`` [T]
    in frame cadences (None: 0..T-1); ``jitter`` [T, 2] as (x, y) pixels
    (None: 0); Q > 0: phases rounded to multiples of 1/Q as in
    ``trajectory_table_quantised``."""
    vx = np.ascontiguousarray(vx, np.float64)
    vy = np.ascontiguousarray(vy, np.float64)
    K = vx.shape[0]
    tm = None if times is None else np.ascontiguousarray(times, np.float64)
    jx = jy = None
    if jitter is not None:
        j = np.asarray(jitter, np.float64).reshape(T, 2)
        jx, jy = np.ascontiguousarray(j[:, 0]), np.ascontiguousarray(j[:, 1])
    shifts = np.zeros((K, T, 2), np.int32)
    taps = np.zeros((K, T, 5, 5), np.float64)
    _load().orc_trajectory_table_frames(K, int(T), _ptr(vx), _ptr(vy), _ptr(tm), _ptr(jx), _ptr(jy),
                                        float(sigma), int(kind), int(Q), _ptr(shifts), _ptr(taps))
    return shifts, taps


def trajectory_table_quantised(vx, vy, T: int, Q: int, sigma: float = 0.7, kind: int = 0):
    """The filter bank of the phase-quantised search: as ``trajectory_table``
    with each footprint's sub-pixel phase rounded to a multiple of 1/Q."""
    vx = np.ascontiguousarray(vx, np.float64)
    vy = np.ascontiguousarray(vy, np.float64)
    K = vx.shape[0]
    shifts = np.zeros((K, T, 2), np.int32)
    taps = np.zeros((K, T, 5, 5), np.float64)
    _load().orc_trajectory_table_quantised(K, int(T), _ptr(vx), _ptr(vy), float(sigma), int(kind), int(Q),
                                           _ptr(shifts), _ptr(taps))
    return shifts, taps


def inverse_variance(sigma, mask=None) -> np.ndarray:
    sigma = np.ascontiguousarray(sigma, np.float32)
    H, W = sigma.shape
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lam = np.zeros((H, W), np.float64)
    _load().orc_inverse_variance(H, W, _ptr(sigma), _ptr(m), _ptr(lam))
    return lam


def search_full(res, lam, shifts, taps, frame_scale=None):
    """N[k, y, x] and D[k, y, x] for every filter and start pixel (FP64)."""
    res = np.ascontiguousarray(res, np.float32)
    T, H, W = res.shape
    lam = np.ascontiguousarray(lam, np.float64)
    shifts = np.ascontiguousarray(shifts, np.int32)
    taps = np.ascontiguousarray(taps, np.float64)
    K = shifts.shape[0]
    assert shifts.shape == (K, T, 2) and taps.shape == (K, T, 5, 5)
    fs = None if frame_scale is None else np.ascontiguousarray(frame_scale, np.float64)
    N = np.zeros((K, H, W), np.float64)
    D = np.zeros((K, H, W), np.float64)
    _load().orc_search_full(T, H, W, _ptr(res), _ptr(fs), _ptr(lam), K, _ptr(shifts),
                            _ptr(taps), _ptr(N), _ptr(D))
    return N, D


def search_points(res, lam, shifts, taps, ys, xs, ks, frame_scale=None):
    """N and D at the listed (y, x, k) triples (FP64)."""
    res = np.ascontiguousarray(res, np.float32)
    T, H, W = res.shape
    lam = np.ascontiguousarray(lam, np.float64)
    shifts = np.ascontiguousarray(shifts, np.int32)
    taps = np.ascontiguousarray(taps, np.float64)
    ys = np.ascontiguousarray(ys, np.int32)
    xs = np.ascontiguousarray(xs, np.int32)
    ks = np.ascontiguousarray(ks, np.int32)
    n = ys.shape[0]
    fs = None if frame_scale is None else np.ascontiguousarray(frame_scale, np.float64)
    N = np.zeros(n, np.float64)
    D = np.zeros(n, np.float64)
    _load().orc_search_points(T, H, W, _ptr(res), _ptr(fs), _ptr(lam), _ptr(shifts),
                              _ptr(taps), n, _ptr(ys), _ptr(xs), _ptr(ks), _ptr(N), _ptr(D))
    return N, D


def round_to_bf16(x) -> np.ndarray:
    """FP32 values rounded to the nearest bfloat16 (the upper 16 bits of an
    FP32), ties to even, returned as FP32.  From the definition: add half
    of the dropped part's unit (0x7FFF, plus 1 when the kept part is odd) and
    truncate the low 16 bits."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    keep_odd = (b >> 16) & 1
    r = ((b + 0x7FFF + keep_odd) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def weighted_stack16(stored, sigma, mask=None, frame_scale=None, dtype="bf16"):
    """The precision form's weighted stack (not in the paper: residuals
    stored in 16 bits to halve the stack's bytes, spec extension).

    The inverse-variance weighted residual y_t = lambda * (alpha_t * r_t) of
    Section 3.2's noise model is formed in FP32 -- lambda = 1 / sigma^2
    rounded to FP32 (0 where masked or sigma unusable), alpha_t the frame
    scale, r_t the stored 16-bit value -- and stored in the stack's own
    16-bit type: bf16 as it is (scale beta_t = 1); fp16 divided by beta_t,
    the power of two at or above lambda_max * |alpha_t| (lambda_max the
    largest lambda), which keeps every stored value within fp16's range and
    makes the division exact.  Rounding is to nearest, ties to even.

    Returns (q, beta): q [T, H, W] float32 holding the 16-bit values,
    beta [T] float64, so that the weighted residual is beta_t * q_t.  The
    matched filter of the precision form is then N = sum W beta q (weights
    already applied) and D = sum W^2 lambda as usual (``search_weighted``)."""
    stored = np.ascontiguousarray(stored, np.float32)
    T = stored.shape[0]
    s = np.asarray(sigma, np.float64)
    usable = (s > 0) & np.isfinite(s)
    if mask is not None:
        usable &= np.asarray(mask) == 0
    lam = np.where(usable, 1.0 / np.where(usable, s * s, 1.0), 0.0).astype(np.float32)
    alpha = np.ones(T, np.float32) if frame_scale is None else np.asarray(frame_scale, np.float32)
    y = lam[None] * (alpha[:, None, None] * stored)  # FP32 products, in this order
    if dtype == "bf16":
        return round_to_bf16(y), np.ones(T, np.float64)
    if dtype != "fp16":
        raise ValueError(dtype)
    lmax = np.float32(lam.max())
    x = (lmax * np.abs(alpha)).astype(np.float32)
    e = np.minimum((x.view(np.uint32) >> 23) & 0xFF, 253).astype(np.int64)  # x = 1.m 2^(e - 127)
    beta = np.where(x > 0, np.ldexp(1.0, e - 126), 1.0)
    inv = np.where(x > 0, np.ldexp(1.0, 126 - e), 1.0).astype(np.float32)
    q = (y * inv[:, None, None]).astype(np.float16).astype(np.float32)
    return q, beta


def search_weighted(q, beta, lam, shifts, taps):
    """Matched filter on a weighted stack whose values already carry lambda:
    N = sum_t sum_{a,b} W beta_t q_t(q) over the footprint pixels inside the
    frame (lambda is not applied again), D = sum W^2 lambda (Section 3.2,
    Eq. 5 with the weights moved into the stored stack)."""
    q = np.ascontiguousarray(q, np.float32)
    T, H, W = q.shape
    ones = np.ones((H, W), np.float64)
    N, _ = search_full(q, ones, shifts, taps, frame_scale=np.asarray(beta, np.float64))
    _, D = search_full(q, lam, shifts, taps)  # D does not depend on the stack's values
    return N, D


def search_weighted_points(q, beta, lam, shifts, taps, ys, xs, ks):
    """``search_weighted`` at the listed (y, x, k) triples."""
    q = np.ascontiguousarray(q, np.float32)
    T, H, W = q.shape
    ones = np.ones((H, W), np.float64)
    N, _ = search_points(q, ones, shifts, taps, ys, xs, ks, frame_scale=np.asarray(beta, np.float64))
    _, D = search_points(q, lam, shifts, taps, ys, xs, ks)  # D does not depend on the stack's values
    return N, D


def snr_and_best(N, D):
    """SNR_k = N_k / sqrt(D_k) where D_k > 0, and the best filter per pixel.

    Section 3.2: the maximum over the filter bank names the most likely
    trajectory.  Ties go to the smallest k.  A pixel where no filter has
    D > 0 gets snr_max = 0 and argmax = -1.  Returns (snr, valid, snr_max,
    argmax) with snr = 0 where D = 0.
    """
    N = np.asarray(N, np.float64)
    D = np.asarray(D, np.float64)
    valid = D > 0
    snr = np.zeros_like(N)
    snr[valid] = N[valid] / np.sqrt(D[valid])
    masked = np.where(valid, snr, -np.inf)
    argmax = np.argmax(masked, axis=0).astype(np.int32)  # first maximum = smallest k
    snr_max = np.take_along_axis(masked, argmax[None], axis=0)[0]
    none = ~valid.any(axis=0)
    snr_max = np.where(none, 0.0, snr_max)
    argmax = np.where(none, -1, argmax).astype(np.int32)
    return snr, valid, snr_max, argmax


def topk_order(snr_max, argmax, k_top):
    """Candidate order: SNR descending, then flat pixel index ascending.

    Pixels with argmax = -1 are never candidates.  Returns flat indices.
    """
    s = np.asarray(snr_max, np.float64).ravel()
    ok = np.asarray(argmax).ravel() >= 0
    idx = np.nonzero(ok)[0]
    order = np.lexsort((idx, -s[idx]))
    return idx[order[:k_top]]


def dense_template(H, W, shifts_k, taps_k, py, px):
    """Filter of one trajectory for start pixel (py, px) as a dense T x H x W
    tensor (Section 3.2: the trajectory line convolved with the PRF).  Footprint
    pixels that fall outside the frame are dropped."""
    T = shifts_k.shape[0]
    F = np.zeros((T, H, W), np.float64)
    for t in range(T):
        sx, sy = int(shifts_k[t, 0]), int(shifts_k[t, 1])
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                qy, qx = py + sy + dy, px + sx + dx
                if 0 <= qy < H and 0 <= qx < W:
                    F[t, qy, qx] += taps_k[t, dy + 2, dx + 2]
    return F


def search_dense(res, lam, shifts, taps, frame_scale=None):
    """Paper-literal brute force for tiny inputs: for each filter and each start
    pixel, build the dense filter and take <F, lambda r> and <F^2, lambda>."""
    res = np.asarray(res, np.float64)
    if frame_scale is not None:
        res = res * np.asarray(frame_scale, np.float64)[:, None, None]
    T, H, W = res.shape
    K = shifts.shape[0]
    N = np.zeros((K, H, W))
    D = np.zeros((K, H, W))
    y = res * lam[None]
    for k in range(K):
        for py in range(H):
            for px in range(W):
                F = dense_template(H, W, shifts[k], taps[k], py, px)
                N[k, py, px] = np.sum(F * y)
                D[k, py, px] = np.sum(F * F * lam[None])
    return N, D


def _shifted(img, oy, ox):
    """out[y, x] = img[y + oy, x + ox], zero where that falls outside."""
    H, W = img.shape
    out = np.zeros_like(img)
    y0, y1 = max(0, -oy), min(H, H - oy)
    x0, x1 = max(0, -ox), min(W, W - ox)
    if y0 < y1 and x0 < x1:
        out[y0:y1, x0:x1] = img[y0 + oy:y1 + oy, x0 + ox:x1 + ox]
    return out


def search_numpy(res, lam, shifts, taps, frame_scale=None):
    """Same definition with whole-frame numpy slicing (loops over k, t, dy, dx)."""
    res = np.asarray(res, np.float64)
    if frame_scale is not None:
        res = res * np.asarray(frame_scale, np.float64)[:, None, None]
    T, H, W = res.shape
    K = shifts.shape[0]
    N = np.zeros((K, H, W))
    D = np.zeros((K, H, W))
    for k in range(K):
        for t in range(T):
            sx, sy = int(shifts[k, t, 0]), int(shifts[k, t, 1])
            yt = res[t] * lam
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    w = taps[k, t, dy + 2, dx + 2]
                    N[k] += w * _shifted(yt, sy + dy, sx + dx)
                    D[k] += w * w * _shifted(lam, sy + dy, sx + dx)
    return N, D


def search_quantised_gather(res, lam, vx, vy, Q: int, sigma: float = 0.7, kind: int = 0, frame_scale=None):
    """The phase-quantised search in its own order, precompute then gather:
    frame t is correlated once with the footprint of every rounded phase
    n / Q (n = floor(phi Q + 1/2) per axis) that some trajectory takes in
    that frame, over the frame plus a 2-pixel halo (the footprint still
    overlaps the frame there), for the numerator (lambda r) and the
    denominator (lambda, with squared taps); every trajectory then adds the
    plane of its phase at its start pixel plus its base shift.  Returns
    N, D [K, H, W]; the same sums as ``search_full`` on
    ``trajectory_table_quantised``, in another order."""
    res = np.asarray(res, np.float64)
    if frame_scale is not None:
        res = res * np.asarray(frame_scale, np.float64)[:, None, None]
    T, H, W = res.shape
    lam = np.asarray(lam, np.float64)
    vx = np.asarray(vx, np.float64)
    vy = np.asarray(vy, np.float64)
    K = vx.shape[0]
    N = np.zeros((K, H, W))
    D = np.zeros((K, H, W))
    lam_p = np.pad(lam, 4)
    for t in range(T):
        y_p = np.pad(res[t] * lam, 4)
        planes = {}
        for k in range(K):
            cx, cy = vx[k] * t, vy[k] * t
            sx, sy = np.floor(cx + 0.5), np.floor(cy + 0.5)
            n = (np.floor((cx - sx) * Q + 0.5), np.floor((cy - sy) * Q + 0.5))
            if n not in planes:
                w = prf_taps(n[0] / Q, n[1] / Q, sigma, kind)
                # plane index i holds position i - 2: rows -2 .. H + 1
                C = np.zeros((H + 4, W + 4))
                E = np.zeros((H + 4, W + 4))
                for b in range(-2, 3):
                    for a in range(-2, 3):
                        wab = w[b + 2, a + 2]
                        C += wab * y_p[2 + b:2 + b + H + 4, 2 + a:2 + a + W + 4]
                        E += wab * wab * lam_p[2 + b:2 + b + H + 4, 2 + a:2 + a + W + 4]
                planes[n] = (C, E)
            C, E = planes[n]
            N[k] += _window(C, int(sy) + 2, int(sx) + 2, H, W)
            D[k] += _window(E, int(sy) + 2, int(sx) + 2, H, W)
    return N, D


def _window(plane, oy, ox, H, W):
    """out[y, x] = plane[y + oy, x + ox] for an H x W output, zero where that
    falls outside the plane."""
    out = np.zeros((H, W))
    Hp, Wp = plane.shape
    y0, y1 = max(0, -oy), min(H, Hp - oy)
    x0, x1 = max(0, -ox), min(W, Wp - ox)
    if y0 < y1 and x0 < x1:
        out[y0:y1, x0:x1] = plane[y0 + oy:y1 + oy, x0 + ox:x1 + ox]
    return out


def inject(res, shifts_k, taps_k, py, px, flux):
    """Add flux times the filter of one trajectory started at (py, px)
    (Section 4.1: injection adds a filter times a flux).  In place on a float64
    array; footprint pixels outside the frame are dropped."""
    T, H, W = res.shape
    for t in range(T):
        sx, sy = int(shifts_k[t, 0]), int(shifts_k[t, 1])
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                qy, qx = py + sy + dy, px + sx + dx
                if 0 <= qy < H and 0 <= qx < W:
                    res[t, qy, qx] += flux * taps_k[t, dy + 2, dx + 2]
    return res
