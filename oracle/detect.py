"""FP64 CPU oracle for score normalisation and candidate extraction.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  It shares no code
with the CUDA library.

Section 3.3 of Ganapathi (2022) turns the per-pixel best score into
candidates: the standard deviation of the scores in the 255 x 255 square
centred on a pixel is that pixel's sigma, scores are expressed in units of
it, and scores above 3 sigma (5 sigma for the recovery figure of Section
4.1) are candidates.  The readings taken where the text is silent:

* the square is clipped to the image, and pixels without a score (no
  trajectory reached them with weight: argmax -1) neither enter a window's
  statistics nor become candidates;
* sigma is the population standard deviation (divide by the pixel count n);
* the normalised score is z = (s - mean) / sigma, the mean taken over the
  same square; ``subtract_mean=False`` gives the literal z = s / sigma;
* a pixel with n < 2, or whose window is constant, gets z = 0; a window
  counts as constant when sigma^2 <= 1e-12 (mean^2 + sigma^2), the
  resolution of the variance as the mean square minus the squared mean;
* a candidate is a pixel with z > threshold; candidates that touch (8
  neighbours) are one detection, reported at its largest z (smallest flat
  index among equal z) with the number of pixels it covers.

Functions:

* ``local_stats_direct`` -- the definition: for every pixel, the explicit
  window, its mean and the two-pass variance.  Small inputs only.
* ``local_stats`` -- the same sums through summed-area tables (FP64
  cumulative sums); pinned to ``local_stats_direct`` by the tests.
* ``normalise`` -- z and the candidate flags.
* ``components`` -- 8-connected labels of the candidate flags
  (``scipy.ndimage.label``), pinned by a flood fill in the tests.
* ``detections`` -- the detections ordered by (z rounded to FP32
  descending, flat index ascending), and their total count.
"""
from __future__ import annotations

import numpy as np

__all__ = ["local_stats_direct", "local_stats", "normalise", "components", "detections",
           "DETECTION_FIELDS"]

# one detection: peak pixel, the trajectory there, pixels in the component,
# normalised score, snr_max, local mean and sigma at the peak
DETECTION_FIELDS = ("y", "x", "k", "npix", "z", "snr", "mean", "sigma")


def _valid(argmax):
    return np.asarray(argmax) >= 0


def local_stats_direct(score, argmax, window: int):
    """Per pixel: valid count n, mean and population standard deviation of
    the scores in the window x window square centred on it (clipped to the
    image, valid pixels only), straight from the definition."""
    s = np.asarray(score, dtype=np.float64)
    v = _valid(argmax)
    H, W = s.shape
    R = window // 2
    n = np.zeros((H, W), dtype=np.int64)
    mean = np.zeros((H, W))
    sd = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            y0, y1, x0, x1 = max(0, y - R), min(H, y + R + 1), max(0, x - R), min(W, x + R + 1)
            vals = s[y0:y1, x0:x1][v[y0:y1, x0:x1]]
            n[y, x] = vals.size
            if vals.size:
                m = vals.sum() / vals.size
                mean[y, x] = m
                sd[y, x] = np.sqrt(((vals - m) ** 2).sum() / vals.size)
    return n, mean, sd


def _box(a, R):
    """Sum of `a` over the (2R+1)^2 square around each element, clipped to
    the array: differences of a summed-area table."""
    H, W = a.shape
    S = np.zeros((H + 1, W + 1), dtype=a.dtype)
    S[1:, 1:] = np.cumsum(np.cumsum(a, axis=0), axis=1)
    ys = np.arange(H)
    xs = np.arange(W)
    y0 = np.clip(ys - R, 0, H)[:, None]
    y1 = np.clip(ys + R + 1, 0, H)[:, None]
    x0 = np.clip(xs - R, 0, W)[None, :]
    x1 = np.clip(xs + R + 1, 0, W)[None, :]
    return S[y1, x1] - S[y0, x1] - S[y1, x0] + S[y0, x0]


def local_stats(score, argmax, window: int):
    """As ``local_stats_direct``, from window sums of the valid scores,
    their squares and the valid count: mean = S1 / n, variance = S2 / n -
    mean^2 (clamped at 0)."""
    s = np.asarray(score, dtype=np.float64)
    v = _valid(argmax)
    R = window // 2
    x = np.where(v, s, 0.0)
    n = _box(v.astype(np.int64), R)
    s1 = _box(x, R)
    s2 = _box(x * x, R)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(n > 0, s1 / np.maximum(n, 1), 0.0)
        var = np.where(n > 0, s2 / np.maximum(n, 1) - mean * mean, 0.0)
    return n, mean, np.sqrt(np.maximum(var, 0.0))


def normalise(score, argmax, n, mean, sd, threshold: float, subtract_mean: bool = True):
    """z = (s - mean) / sigma (or s / sigma) at valid pixels with n >= 2 and
    a window that is not constant, else 0; candidate flags z > threshold."""
    s = np.asarray(score, dtype=np.float64)
    ok = _valid(argmax) & (n >= 2) & (sd * sd > 1e-12 * (mean * mean + sd * sd))
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.where(ok, (s - (mean if subtract_mean else 0.0)) / np.where(ok, sd, 1.0), 0.0)
    return z, ok & (z > threshold)


def components(flag):
    """8-connected labels (0 = not a candidate, 1.. per component)."""
    from scipy import ndimage
    lab, count = ndimage.label(np.asarray(flag, dtype=bool), structure=np.ones((3, 3), dtype=int))
    return lab, int(count)


def detections(score, argmax, window: int = 255, threshold: float = 3.0, subtract_mean: bool = True,
               stats=None):
    """All detections as a structured array ordered by (float32(z)
    descending, flat index ascending), plus z and the flags."""
    s = np.asarray(score)
    a = np.asarray(argmax)
    H, W = s.shape
    n, mean, sd = stats if stats is not None else local_stats(s, a, window)
    z, flag = normalise(s, a, n, mean, sd, threshold, subtract_mean)
    lab, count = components(flag)
    dt = np.dtype([("y", np.int32), ("x", np.int32), ("k", np.int32), ("npix", np.int32),
                   ("z", np.float64), ("snr", np.float32), ("mean", np.float64), ("sigma", np.float64)])
    out = np.zeros(count, dtype=dt)
    if count:
        flat = lab.ravel()
        zf = z.ravel()
        idx = np.flatnonzero(flat)
        labs = flat[idx]
        # peak of each component: largest z, then smallest flat index
        order = np.lexsort((idx, -zf[idx], labs))
        first = np.ones(order.size, dtype=bool)
        first[1:] = labs[order][1:] != labs[order][:-1]
        peaks = idx[order][first]
        npix = np.bincount(labs, minlength=count + 1)[1:]
        pl = flat[peaks]
        out["y"] = peaks // W
        out["x"] = peaks % W
        out["k"] = a.ravel()[peaks]
        out["npix"] = npix[pl - 1]
        out["z"] = zf[peaks]
        out["snr"] = s.ravel()[peaks]
        out["mean"] = mean.ravel()[peaks]
        out["sigma"] = sd.ravel()[peaks]
        rank = np.lexsort((peaks, -out["z"].astype(np.float32)))
        out = out[rank]
    return out, z, flag
