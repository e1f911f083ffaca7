"""FP64 CPU oracle for the per-pixel background re-fit (Section 3.1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  It shares no code
with the CUDA library.

Section 3.1 models frame t as D_t = U(S_t) + B + B_theta theta_t^k + noise
(Eq. 1): U(S_t) the low-resolution scattered light upsampled bilinearly,
B the background and B_theta its second-order Taylor expansion in the
jitter theta_t = (x_t, y_t), theta_t^k = (x_t, y_t, x_t^2, y_t^2, x_t y_t).
With S_t fixed, the Huber loss (Eqs. 2-4) separates into one regression per
pixel on the same six basis values phi_t = (1, x_t, y_t, x_t^2, y_t^2,
x_t y_t), so the Gram matrix G = sum_t phi_t phi_t^T and its inverse are
shared; the Huber fit is reached by repeated least-squares solves with
clipped residuals (Huber 1977, "modified residuals").  Readings:

* Eq. 4 is garbled; the Huber loss is L(a) = a^2 / 2 for |a| <= delta and
  delta (|a| - delta / 2) otherwise; its clipped residual is
  psi(a) = min(max(a, -delta), delta);
* the iteration starts at the least-squares fit and takes `iterations`
  steps beta <- beta + G^-1 sum_t phi_t psi(y_t - phi_t . beta), with
  y_t = D_t - U(S_t); the output residual is r_t = y_t - phi_t . beta, the
  matched filter's input;
* U maps an n x n grid to H x W with pixel centres aligned: low-resolution
  coordinate u = (i + 1/2) n / H - 1/2 for row i (likewise for columns),
  clamped to [0, n - 1], then linear interpolation between the two nearest
  grid points in each direction; no scattered light (S absent) means U = 0.

Functions: ``basis`` (phi), ``upsample`` (U), ``refit`` (coefficients and
residuals), ``refit_points`` (the same for sampled pixels of a large
image), ``huber_loss`` (the objective, for the pins).
"""
from __future__ import annotations

import numpy as np

__all__ = ["basis", "upsample", "refit", "refit_points", "huber_loss"]


def basis(jitter):
    """phi_t = (1, x, y, x^2, y^2, x y) for jitter [T, 2] = (x_t, y_t)."""
    j = np.asarray(jitter, dtype=np.float64)
    x, y = j[:, 0], j[:, 1]
    return np.stack([np.ones_like(x), x, y, x * x, y * y, x * y], axis=1)


def upsample(S, H: int, W: int):
    """Bilinear upsampling of S [T, n, n] (or [n, n]) to [T, H, W]."""
    S = np.asarray(S, dtype=np.float64)
    squeeze = S.ndim == 2
    if squeeze:
        S = S[None]
    n_y, n_x = S.shape[1], S.shape[2]

    def axis(N, n):
        u = np.clip((np.arange(N) + 0.5) * n / N - 0.5, 0.0, n - 1)
        i0 = np.floor(u).astype(np.int64)
        i1 = np.minimum(i0 + 1, n - 1)
        return i0, i1, u - i0

    y0, y1, fy = axis(H, n_y)
    x0, x1, fx = axis(W, n_x)
    top = S[:, y0][:, :, x0] * (1 - fx) + S[:, y0][:, :, x1] * fx
    bot = S[:, y1][:, :, x0] * (1 - fx) + S[:, y1][:, :, x1] * fx
    out = top * (1 - fy)[None, :, None] + bot * fy[None, :, None]
    return out[0] if squeeze else out


def huber_loss(a, delta):
    a = np.abs(np.asarray(a, dtype=np.float64))
    return np.where(a <= delta, 0.5 * a * a, delta * (a - 0.5 * delta))


def refit(D, jitter, delta: float, iterations: int, S=None):
    """Per-pixel Huber fit of D_t - U(S_t) on phi_t: returns (coef [H, W, 6],
    residual [T, H, W]) in FP64."""
    D = np.asarray(D, dtype=np.float64)
    T, H, W = D.shape
    Y = D - (upsample(S, H, W) if S is not None else 0.0)
    Phi = basis(jitter)
    Ginv = np.linalg.inv(Phi.T @ Phi)
    Yf = Y.reshape(T, H * W)
    beta = Ginv @ (Phi.T @ Yf)
    for _ in range(int(iterations)):
        E = Yf - Phi @ beta
        beta = beta + Ginv @ (Phi.T @ np.clip(E, -delta, delta))
    R = Yf - Phi @ beta
    return beta.T.reshape(H, W, 6), R.reshape(T, H, W)


def refit_points(D_pts, ys, xs, H: int, W: int, jitter, delta: float, iterations: int, S=None):
    """``refit`` for the pixels (ys[m], xs[m]) of an H x W image: D_pts
    [T, m] their time series; U evaluated at those pixels only."""
    D_pts = np.asarray(D_pts, dtype=np.float64)
    ys = np.asarray(ys)
    xs = np.asarray(xs)
    if S is not None:
        S = np.asarray(S, dtype=np.float64)
        n_y, n_x = S.shape[1], S.shape[2]
        u = np.clip((ys + 0.5) * n_y / H - 0.5, 0.0, n_y - 1)
        v = np.clip((xs + 0.5) * n_x / W - 0.5, 0.0, n_x - 1)
        y0 = np.floor(u).astype(np.int64)
        x0 = np.floor(v).astype(np.int64)
        y1 = np.minimum(y0 + 1, n_y - 1)
        x1 = np.minimum(x0 + 1, n_x - 1)
        fy, fx = u - y0, v - x0
        top = S[:, y0, x0] * (1 - fx) + S[:, y0, x1] * fx
        bot = S[:, y1, x0] * (1 - fx) + S[:, y1, x1] * fx
        D_pts = D_pts - (top * (1 - fy) + bot * fy)
    T, m = D_pts.shape
    coef, R = refit(D_pts.reshape(T, 1, m), jitter, delta, iterations)
    return coef.reshape(m, 6), R.reshape(T, m)
