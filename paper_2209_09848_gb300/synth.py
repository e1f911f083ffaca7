"""Seeded synthetic inputs shaped like the paper's workloads.

Stand-ins for TESS full-frame images, which are not available here:
background-subtracted residual stacks of T frames x H x W pixels (Section 2:
2048 x 2048 CCDs, about 1000 frames per sector), Gaussian noise with a
per-pixel sigma, a mask of saturated-star residuals (Section 3.2 clips bright
pixels), and injected linear movers (Section 4.1: a grid of injected sources
20 px apart vertically and 80 px horizontally).

The scene model draws each mover with a circular Gaussian PRF integrated over
pixels, on the 5 x 5 pixels around its nearest pixel, renormalised.  This
module is shared by the oracle tests and the GPU path only as an input
generator: it holds none of the matched filter's arithmetic, and it imports
neither the oracle nor the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------ velocities --

def velocity_grid(nx: int, ny: int, lo: float = -0.1, hi: float = 0.1):
    """Cartesian grid of velocities (px/frame), x varying fastest."""
    gx = np.linspace(lo, hi, nx)
    gy = np.linspace(lo, hi, ny)
    vx = np.tile(gx, ny)
    vy = np.repeat(gy, nx)
    return vx.astype(np.float64), vy.astype(np.float64)


def small_grid_velocities():
    """4 x 4 grid, vx, vy in {-0.15, -0.05, 0.05, 0.15} px/frame (16 filters)."""
    g = np.array([-0.15, -0.05, 0.05, 0.15])
    return np.tile(g, 4), np.repeat(g, 4)


# ----------------------------------------------------------- scene model --

def _pixel_gauss_np(d, phase, sigma):
    from scipy.special import erf
    s = sigma * math.sqrt(2.0)
    return 0.5 * (erf((d + 0.5 - phase) / s) - erf((d - 0.5 - phase) / s))


def render_movers_np(T, H, W, movers, sigma_prf=0.7):
    """Flux image stack (float64 [T, H, W]) of linear movers.

    movers: iterable of (y0, x0, vy, vx, flux) with start position in pixels
    (pixel centres at integers) and velocity in px/frame.
    """
    out = np.zeros((T, H, W))
    d = np.arange(-2, 3)
    for (y0, x0, vy, vx, flux) in movers:
        for t in range(T):
            cy, cx = y0 + vy * t, x0 + vx * t
            by, bx = math.floor(cy + 0.5), math.floor(cx + 0.5)
            gy = _pixel_gauss_np(d, cy - by, sigma_prf)
            gx = _pixel_gauss_np(d, cx - bx, sigma_prf)
            w = np.outer(gy, gx)
            w /= w.sum()
            for i in range(5):
                qy = by + i - 2
                if not (0 <= qy < H):
                    continue
                for j in range(5):
                    qx = bx + j - 2
                    if 0 <= qx < W:
                        out[t, qy, qx] += flux * w[i, j]
    return out


def star_mask(H, W, rng, frac=0.01):
    """Clustered mask of saturated-star residuals: square blobs of 3..7 px
    around random star centres until `frac` of the pixels is covered."""
    m = np.zeros((H, W), np.uint8)
    target = frac * H * W
    covered = 0
    while covered < target:
        cy, cx = rng.integers(0, H), rng.integers(0, W)
        r = int(rng.integers(1, 4))  # half width 1..3 -> 3x3 .. 7x7
        y0, y1 = max(0, cy - r), min(H, cy + r + 1)
        x0, x1 = max(0, cx - r), min(W, cx + r + 1)
        m[y0:y1, x0:x1] = 1
        covered = int(m.sum()) if covered + (2 * r + 1) ** 2 >= target else covered + (2 * r + 1) ** 2
    return m


def lattice_starts(H, W, n, rng, dy=20, dx=80, margin=4):
    """Start pixels on a jittered lattice whose sites stay at least dy rows and
    dx columns apart (Section 4.1 injection grid)."""
    sy, sx = dy + 10, dx + 20
    ys = np.arange(margin + 5, H - margin - 5, sy)
    xs = np.arange(margin + 10, W - margin - 10, sx)
    sites = np.array([(y, x) for y in ys for x in xs])
    if len(sites) < n:
        raise ValueError("frame too small for %d movers" % n)
    pick = rng.choice(len(sites), size=n, replace=False)
    jy = rng.integers(-5, 6, size=n)
    jx = rng.integers(-10, 11, size=n)
    return sites[pick, 0] + jy, sites[pick, 1] + jx


# ------------------------------------------------------------ small cases --

def small_case(T, H, W, seed, sigma_kind="lognormal", mask_frac=0.0, movers=0, flux=(0.5, 2.0),
               vx=None, vy=None, speed=(0.003, 0.1)):
    """Host (numpy) stack for tests: returns dict with res float32 [T,H,W],
    sigma float32 [H,W], mask uint8 [H,W] or None, movers list."""
    rng = np.random.default_rng(seed)
    if sigma_kind == "uniform":
        sigma = np.ones((H, W), np.float32)
    else:
        sigma = np.exp(0.3 * rng.standard_normal((H, W))).astype(np.float32)
    mask = star_mask(H, W, rng, mask_frac) if mask_frac > 0 else None
    res = sigma[None].astype(np.float64) * rng.standard_normal((T, H, W))
    mv = []
    for _ in range(movers):
        y0 = float(rng.integers(0, H))
        x0 = float(rng.integers(0, W))
        if vx is not None:
            k = int(rng.integers(0, len(vx)))
            mvx, mvy = float(vx[k]), float(vy[k])
        else:
            sp = rng.uniform(*speed)
            ang = rng.uniform(0, 2 * np.pi)
            mvx, mvy = sp * math.cos(ang), sp * math.sin(ang)
        mv.append((y0, x0, mvy, mvx, float(rng.uniform(*flux))))
    if mv:
        res += render_movers_np(T, H, W, mv)
    return dict(res=res.astype(np.float32), sigma=sigma, mask=mask, movers=mv)


def small_config(seed=0):
    """32 frames x 128 x 128, sigma = 1, no mask, 3 movers at grid velocities
    with per-frame flux 0.5..2, 16 filters on the 4 x 4 grid."""
    vx, vy = small_grid_velocities()
    c = small_case(32, 128, 128, seed, sigma_kind="uniform", movers=3, flux=(0.5, 2.0), vx=vx, vy=vy)
    c["vx"], c["vy"] = vx, vy
    return c


# --------------------------------------------------------- paper-shaped ---

def paper_case_gpu(T=1000, H=2048, W=2048, n_movers=200, seed=1, device="cuda", dtype=None, mask_frac=0.01):
    """Paper-shaped stack generated on the GPU with torch (seeded Philox):
    log-normal sigma (median 1, log-std 0.3), 1 % clustered star mask, 200
    linear movers with per-frame flux 0.05..1 and speed 0.003..0.1 px/frame in
    random directions, on a jittered 20 x 80 px lattice.  Returns dict with
    torch tensors res [T,H,W] float32 (device), sigma, mask and numpy movers."""
    import torch
    rng = np.random.default_rng(seed)
    sigma = np.exp(0.3 * rng.standard_normal((H, W))).astype(np.float32)
    mask = star_mask(H, W, rng, mask_frac) if mask_frac > 0 else None
    ys, xs = lattice_starts(H, W, n_movers, rng)
    sp = rng.uniform(0.003, 0.1, n_movers)
    ang = rng.uniform(0, 2 * np.pi, n_movers)
    flux = rng.uniform(0.05, 1.0, n_movers)
    movers = np.stack([ys, xs, sp * np.sin(ang), sp * np.cos(ang), flux], 1)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    res = torch.empty((T, H, W), dtype=torch.float32, device=device)
    sig_t = torch.from_numpy(sigma).to(device)
    chunk = max(1, (1 << 28) // (H * W))
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        res[t0:t1].normal_(generator=g)
        res[t0:t1].mul_(sig_t)
    add_movers_torch(res, movers)
    out = dict(res=res, sigma=sig_t, mask=None if mask is None else torch.from_numpy(mask).to(device),
               movers=movers, sigma_np=sigma, mask_np=mask)
    return out


def add_movers_torch(res, movers, sigma_prf=0.7):
    """Add linear movers to a [T, H, W] float32 torch tensor in place (scene model)."""
    import torch
    T, H, W = res.shape
    dev = res.device
    m = torch.as_tensor(np.asarray(movers, np.float64), device=dev)
    if m.numel() == 0:
        return res
    t = torch.arange(T, device=dev, dtype=torch.float64)
    cy = m[:, 0:1] + m[:, 2:3] * t[None]          # [M, T]
    cx = m[:, 1:2] + m[:, 3:4] * t[None]
    by = torch.floor(cy + 0.5)
    bx = torch.floor(cx + 0.5)
    d = torch.arange(-2, 3, device=dev, dtype=torch.float64)
    s = sigma_prf * math.sqrt(2.0)

    def g(ph):
        return 0.5 * (torch.erf((d + 0.5 - ph[..., None]) / s) - torch.erf((d - 0.5 - ph[..., None]) / s))

    gy, gx = g(cy - by), g(cx - bx)                # [M, T, 5]
    w = gy[..., :, None] * gx[..., None, :]          # [M, T, 5, 5]
    w = w / w.sum(dim=(-1, -2), keepdim=True)
    val = (w * m[:, 4, None, None, None]).float()
    qy = by[..., None, None] + d[:, None]
    qx = bx[..., None, None] + d[None, :]
    qy, qx = torch.broadcast_tensors(qy, qx)
    tt = torch.broadcast_to(t[None, :, None, None], qy.shape)
    ok = (qy >= 0) & (qy < H) & (qx >= 0) & (qx < W)
    flat = (tt[ok].long() * H + qy[ok].long()) * W + qx[ok].long()
    res.view(-1).index_add_(0, flat, val[ok])
    return res


# ---------------------------------------------------------- score maps --

def score_map(H, W, seed, K=100, mask_frac=0.01, n_sources=200, level=2.5, spread=0.45, peak=(2.0, 12.0),
              gradient=0.5):
    """A best-score map shaped like the search's output, for the detection
    stage: snr_max [H, W] float32 and argmax [H, W] int32.  Noise pixels
    scatter around `level` (the maximum over K trajectories of unit-normal
    scores sits above 0) with a slow gradient across the image; sources add
    compact bumps (3 x 3 to 5 x 5, heights in `peak`) at uniform random
    centres (at most one per 400 pixels; nearby ones may touch); masked
    pixels (clustered blobs) have argmax -1 and score 0."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    s = level + spread * rng.standard_normal((H, W)) + gradient * (yy / max(H, 1) - 0.5)
    a = rng.integers(0, K, size=(H, W)).astype(np.int32)
    n_src = min(n_sources, H * W // 400)
    if n_src > 0:
        ys = rng.integers(0, H, size=n_src)
        xs = rng.integers(0, W, size=n_src)
        for y, x in zip(ys, xs):
            r = int(rng.integers(1, 3))
            h = rng.uniform(*peak)
            y0, y1, x0, x1 = max(0, y - r), min(H, y + r + 1), max(0, x - r), min(W, x + r + 1)
            dy = (np.arange(y0, y1) - y)[:, None]
            dx = (np.arange(x0, x1) - x)[None, :]
            s[y0:y1, x0:x1] += h * np.exp(-(dy * dy + dx * dx) / 1.5)
            a[y0:y1, x0:x1] = int(rng.integers(0, K))
    if mask_frac > 0:
        m = star_mask(H, W, rng, mask_frac).astype(bool)
        s[m] = 0.0
        a[m] = -1
    return s.astype(np.float32), a


# ------------------------------------------------------ background scenes --

def background_case(T, H, W, seed, n=64, noise=1.0, jitter_amp=0.15, n_movers=0, outlier_frac=0.002):
    """Raw frames for the per-pixel background re-fit (Section 3.1, Eq. 1):
    D_t = scattered light + B + B_theta theta_t^k + noise (+ movers and rare
    outliers).  The scattered light is a smooth field (a few low-frequency
    waves whose amplitudes drift with t) evaluated at the pixel centres; S
    holds the same field sampled on an n x n grid of cell centres, so the
    low-resolution model misses it slightly, as it would on sky data.  The
    jitter theta_t = (x_t, y_t) is a bounded random walk of `jitter_amp` px.
    Returns dict(D float32 [T,H,W], S float32 [T,n,n], jitter float64 [T,2],
    coef float64 [H,W,6] (B and the five Taylor terms))."""
    rng = np.random.default_rng(seed)
    steps = rng.normal(0.0, jitter_amp / 4, size=(T, 2))
    jit = np.clip(np.cumsum(steps, axis=0), -jitter_amp, jitter_amp)
    waves = rng.uniform(0.2, 1.0, size=(4, 2))
    phase = rng.uniform(0, 2 * np.pi, size=4)
    amp0 = rng.uniform(5, 20, size=4)
    drift = rng.normal(0, 0.2, size=(T, 4)).cumsum(axis=0) * 0.05

    def field(yy, xx, t):
        a = amp0 * (1 + drift[t])
        return sum(a[i] * np.cos(2 * np.pi * (waves[i, 0] * yy + waves[i, 1] * xx) + phase[i]) for i in range(4))

    py = (np.arange(H) + 0.5) / H
    px = (np.arange(W) + 0.5) / W
    gy = (np.arange(n) + 0.5) / n
    YY, XX = np.meshgrid(py, px, indexing="ij")
    GY, GX = np.meshgrid(gy, gy, indexing="ij")
    coef = np.zeros((H, W, 6))
    coef[..., 0] = 100 + 20 * rng.standard_normal((H, W))
    coef[..., 1:3] = 5 * rng.standard_normal((H, W, 2))
    coef[..., 3:] = 2 * rng.standard_normal((H, W, 3))
    x, y = jit[:, 0], jit[:, 1]
    phi = np.stack([np.ones(T), x, y, x * x, y * y, x * y], axis=1)
    D = np.empty((T, H, W), np.float32)
    S = np.empty((T, n, n), np.float32)
    for t in range(T):
        D[t] = field(YY, XX, t) + coef @ phi[t] + noise * rng.standard_normal((H, W))
        S[t] = field(GY, GX, t)
    if outlier_frac > 0:
        m = rng.random((T, H, W)) < outlier_frac
        D[m] += rng.uniform(20, 200, size=int(m.sum())) * noise
    if n_movers:
        ys = rng.uniform(0, H, n_movers)
        xs = rng.uniform(0, W, n_movers)
        vs = rng.uniform(-0.1, 0.1, size=(n_movers, 2))
        movers = [(ys[i], xs[i], vs[i, 0], vs[i, 1], rng.uniform(2, 10) * noise) for i in range(n_movers)]
        D += render_movers_np(T, H, W, movers).astype(np.float32)
    return {"D": D, "S": S, "jitter": jit, "coef": coef}


def background_case_gpu(T=1000, H=2048, W=2048, seed=1, n=64, noise=1.0, jitter_amp=0.15, outlier_frac=0.001,
                        device="cuda"):
    """``background_case`` at full size, generated on the GPU with torch
    (seeded Philox): D float32 [T, H, W] and S float32 [T, n, n] on the
    device, jitter float64 [T, 2] on the host.  Same scene model: drifting
    low-frequency scattered light at the pixel centres (S samples it on the
    n x n cell centres), a background with jitter Taylor terms, Gaussian
    noise and rare bright outliers."""
    import torch
    rng = np.random.default_rng(seed)
    steps = rng.normal(0.0, jitter_amp / 4, size=(T, 2))
    jit = np.clip(np.cumsum(steps, axis=0), -jitter_amp, jitter_amp)
    waves = rng.uniform(0.2, 1.0, size=(4, 2))
    phase = rng.uniform(0, 2 * np.pi, size=4)
    amp0 = rng.uniform(5, 20, size=4)
    drift = rng.normal(0, 0.2, size=(T, 4)).cumsum(axis=0) * 0.05
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    py = (torch.arange(H, device=device, dtype=torch.float32) + 0.5) / H
    px = (torch.arange(W, device=device, dtype=torch.float32) + 0.5) / W
    gy = (torch.arange(n, device=device, dtype=torch.float32) + 0.5) / n
    modes = [torch.cos(2 * np.pi * (float(waves[i, 0]) * py[:, None] + float(waves[i, 1]) * px[None, :])
                       + float(phase[i])) for i in range(4)]
    gmodes = [torch.cos(2 * np.pi * (float(waves[i, 0]) * gy[:, None] + float(waves[i, 1]) * gy[None, :])
                        + float(phase[i])) for i in range(4)]
    coef = torch.randn((6, H, W), generator=g, device=device)
    coef[0] = 100 + 20 * coef[0]
    coef[1:3] *= 5
    coef[3:] *= 2
    D = torch.empty((T, H, W), dtype=torch.float32, device=device)
    S = torch.empty((T, n, n), dtype=torch.float32, device=device)
    x, y = jit[:, 0], jit[:, 1]
    for t in range(T):
        a = amp0 * (1 + drift[t])
        ph = (1.0, float(x[t]), float(y[t]), float(x[t] ** 2), float(y[t] ** 2), float(x[t] * y[t]))
        frame = torch.randn((H, W), generator=g, device=device) * noise
        for i in range(4):
            frame.add_(modes[i], alpha=float(a[i]))
        for k in range(6):
            frame.add_(coef[k], alpha=ph[k])
        if outlier_frac > 0:
            hit = torch.rand((H, W), generator=g, device=device) < outlier_frac
            frame.add_(hit * (20 + 180 * torch.rand((H, W), generator=g, device=device)) * noise)
        D[t] = frame
        S[t] = sum(float(a[i]) * gmodes[i] for i in range(4))
    return {"D": D, "S": S, "jitter": jit}
