"""Pins for the FP64 oracle, each against something other than the oracle.

Section references are to Ganapathi (2022).  A plausible mistake in the
oracle (a dropped term, a flipped sign, a transposed tap index, a wrong
normalisation) fails at least one of these:

* PRF pixel integral vs scipy quadrature; footprint orientation via the
  centroid and via hand-placed sources;
* hand-worked base pixels and phases (tests/golden/trajectory_shifts.txt);
* a paper-literal dense-template brute force and a whole-frame numpy
  implementation vs the C loops;
* v = 0 vs scipy.signal.correlate2d; integer velocities and the single-tap
  (shift-stack, Section 3.2) filter vs numpy roll-and-add;
* noiseless injection (Section 4.1): flux estimate N/D equals the injected
  flux and SNR = f sqrt(D);
* linearity, noise scaling, mask invariance, translation equivariance;
* on pure Gaussian noise with the right sigma, SNR has mean 0 and variance 1
  (the matched filter is the maximum-likelihood detector, Section 3.2);
* injected movers are recovered at their start pixel and trajectory.
"""
import os

import numpy as np
import pytest
from scipy import integrate, signal, stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- PRF ----

@pytest.mark.parametrize("a,phase,sigma", [(0, 0.0, 0.7), (1, 0.3, 0.7), (-2, -0.45, 0.7),
                                           (2, 0.5, 1.3), (-1, 0.1, 0.35)])
def test_pixel_integral_matches_quadrature(oracle, a, phase, sigma):
    pdf = stats.norm(loc=phase, scale=sigma).pdf
    want, _ = integrate.quad(pdf, a - 0.5, a + 0.5, epsabs=1e-15, epsrel=1e-13)
    got = oracle.oracle.pixel_integrated_gauss(a, phase, sigma)
    assert abs(got - want) < 1e-13


def test_prf_taps_from_quadrature(oracle):
    phx, phy, sig = 0.31, -0.22, 0.7
    pdf_x = stats.norm(loc=phx, scale=sig).pdf
    pdf_y = stats.norm(loc=phy, scale=sig).pdf
    want = np.zeros((5, 5))
    for dy in range(-2, 3):
        iy, _ = integrate.quad(pdf_y, dy - 0.5, dy + 0.5, epsabs=1e-15)
        for dx in range(-2, 3):
            ix, _ = integrate.quad(pdf_x, dx - 0.5, dx + 0.5, epsabs=1e-15)
            want[dy + 2, dx + 2] = ix * iy
    want /= want.sum()
    got = oracle.prf_taps(phx, phy, sig, 0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
def test_prf_orientation_and_symmetry(oracle, kind):
    d = np.arange(-2, 3)
    w = oracle.prf_taps(0.4, 0.0, 0.7, kind)
    assert abs(w.sum() - 1) < 1e-14
    # a source displaced towards +x puts its mass at larger column index
    assert (w * d[None, :]).sum() > 0.2
    assert abs((w * d[:, None]).sum()) < 1e-14
    w2 = oracle.prf_taps(0.0, -0.3, 0.7, kind)
    assert (w2 * d[:, None]).sum() < -0.15
    np.testing.assert_allclose(oracle.prf_taps(0.1, 0.35, 0.7, kind),
                               oracle.prf_taps(0.35, 0.1, 0.7, kind).T, atol=1e-15)
    np.testing.assert_allclose(oracle.prf_taps(0.2, -0.4, 0.7, kind),
                               oracle.prf_taps(-0.2, 0.4, 0.7, kind)[::-1, ::-1], atol=1e-15)


def test_point_sampled_kind(oracle):
    w = oracle.prf_taps(0.0, 0.0, 0.7, 1)
    # ratio of neighbour to centre of a sampled Gaussian is exp(-1/(2 s^2))
    assert abs(w[2, 3] / w[2, 2] - np.exp(-1 / (2 * 0.49))) < 1e-14
    assert abs(w[3, 3] / w[2, 2] - np.exp(-2 / (2 * 0.49))) < 1e-14


# ---------------------------------------------------------- trajectories --

def _golden_shifts():
    rows = []
    with open(os.path.join(HERE, "golden", "trajectory_shifts.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                v, t, s, ph = line.split()
                rows.append((float(v), int(t), int(s), float(ph)))
    return rows


def test_trajectory_shifts_golden(oracle):
    rows = _golden_shifts()
    assert len(rows) >= 20
    for v, t, s, ph in rows:
        T = t + 1
        shifts, taps = oracle.trajectory_table([v, 0.0], [0.0, v], T, 0.7, 0)
        assert shifts[0, t, 0] == s and shifts[0, t, 1] == 0, (v, t)
        assert shifts[1, t, 1] == s and shifts[1, t, 0] == 0, (v, t)
        np.testing.assert_allclose(taps[0, t], oracle.prf_taps(ph, 0.0), atol=1e-14)
        np.testing.assert_allclose(taps[1, t], oracle.prf_taps(0.0, ph), atol=1e-14)


# ------------------------------------------------------ implementations --

def _random_case(seed, T=3, H=7, W=9, K=3, smax=4, custom=True):
    g = _rng(seed)
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.15).astype(np.uint8)
    if custom:
        shifts = g.integers(-smax, smax + 1, size=(K, T, 2)).astype(np.int32)
        taps = g.random((K, T, 5, 5))  # not separable, not symmetric
    else:
        vx = g.uniform(-0.6, 0.6, K)
        vy = g.uniform(-0.6, 0.6, K)
        shifts, taps = None, None
        return res, sigma, mask, vx, vy
    return res, sigma, mask, shifts, taps


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_c_oracle_matches_dense_template(oracle, seed):
    res, sigma, mask, shifts, taps = _random_case(seed)
    lam = oracle.inverse_variance(sigma, mask)
    N, D = oracle.search_full(res, lam, shifts, taps)
    Nd, Dd = oracle.search_dense(res, lam, shifts, taps)
    np.testing.assert_allclose(N, Nd, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D, Dd, rtol=1e-12, atol=1e-12)
    Nn, Dn = oracle.search_numpy(res, lam, shifts, taps)
    np.testing.assert_allclose(N, Nn, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D, Dn, rtol=1e-12, atol=1e-12)


def test_gaussian_table_dense_and_points(oracle):
    res, sigma, mask, vx, vy = _random_case(5, T=6, H=8, W=10, K=4, custom=False)
    shifts, taps = oracle.trajectory_table(vx, vy, 6)
    lam = oracle.inverse_variance(sigma, mask)
    fs = np.linspace(0.5, 2.0, 6)
    N, D = oracle.search_full(res, lam, shifts, taps, frame_scale=fs)
    Nd, Dd = oracle.search_dense(res, lam, shifts, taps, frame_scale=fs)
    np.testing.assert_allclose(N, Nd, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D, Dd, rtol=1e-12, atol=1e-12)
    g = _rng(9)
    ys, xs, ks = g.integers(0, 8, 40), g.integers(0, 10, 40), g.integers(0, 4, 40)
    Np, Dp = oracle.search_points(res, lam, shifts, taps, ys, xs, ks, frame_scale=fs)
    np.testing.assert_array_equal(Np, N[ks, ys, xs])
    np.testing.assert_array_equal(Dp, D[ks, ys, xs])


def test_frame_scale_equals_scaled_data(oracle):
    res, sigma, mask, shifts, taps = _random_case(11, T=4)
    lam = oracle.inverse_variance(sigma, mask)
    fs = np.array([0.5, 2.0, 4.0, 0.25])  # powers of two: scaling is exact
    N1, D1 = oracle.search_full(res, lam, shifts, taps, frame_scale=fs)
    N2, D2 = oracle.search_full(res * fs[:, None, None].astype(np.float32), lam, shifts, taps)
    np.testing.assert_allclose(N1, N2, rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(D1, D2)


# ------------------------------------------------- library special cases --

def test_zero_velocity_is_correlation_of_weighted_sum(oracle):
    g = _rng(3)
    T, H, W = 5, 13, 11
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.1).astype(np.uint8)
    w0 = g.random((5, 5))  # asymmetric: catches a flipped or transposed kernel
    shifts = np.zeros((1, T, 2), np.int32)
    taps = np.broadcast_to(w0, (1, T, 5, 5)).copy()
    lam = oracle.inverse_variance(sigma, mask)
    N, D = oracle.search_full(res, lam, shifts, taps)
    ysum = (res.astype(np.float64) * lam[None]).sum(0)
    wantN = signal.correlate2d(ysum, w0, mode="same", boundary="fill")
    wantD = T * signal.correlate2d(lam, w0 * w0, mode="same", boundary="fill")
    np.testing.assert_allclose(N[0], wantN, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D[0], wantD, rtol=1e-12, atol=1e-12)


def test_zero_velocity_gaussian_is_prf_convolved_mean_stack(oracle):
    g = _rng(4)
    T, H, W = 7, 12, 12
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.ones((H, W), np.float32)
    shifts, taps = oracle.trajectory_table([0.0], [0.0], T)
    lam = oracle.inverse_variance(sigma)
    N, D = oracle.search_full(res, lam, shifts, taps)
    w0 = oracle.prf_taps(0.0, 0.0)
    mean = res.astype(np.float64).mean(0)
    np.testing.assert_allclose(N[0], T * signal.correlate2d(mean, w0, mode="same"),
                               rtol=1e-12, atol=1e-12)
    # uniform sigma, no mask: D is T * sum(w0^2) away from the borders
    assert np.allclose(D[0, 2:-2, 2:-2], T * (w0 ** 2).sum(), rtol=1e-13)


def _roll_zero(img, oy, ox):
    """img shifted so that out[y, x] = img[y + oy, x + ox], zero fill, via np.roll on a padded copy."""
    H, W = img.shape
    pad = max(abs(oy), abs(ox)) + 1
    big = np.pad(img, pad)
    big = np.roll(big, (-oy, -ox), axis=(0, 1))
    return big[pad:pad + H, pad:pad + W]


def test_single_tap_filter_is_shift_and_add(oracle):
    """Section 3.2: shift-stacking is the matched filter with one unit tap per frame."""
    g = _rng(6)
    T, H, W = 9, 16, 14
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.2 * g.standard_normal((H, W))).astype(np.float32)
    lam = oracle.inverse_variance(sigma)
    for vx, vy in [(1, 0), (0, -1), (1, 1), (-1, 1)]:
        shifts = np.zeros((1, T, 2), np.int32)
        shifts[0, :, 0] = vx * np.arange(T)
        shifts[0, :, 1] = vy * np.arange(T)
        taps = np.zeros((1, T, 5, 5))
        taps[0, :, 2, 2] = 1.0
        N, D = oracle.search_full(res, lam, shifts, taps)
        want = np.zeros((H, W))
        wantD = np.zeros((H, W))
        for t in range(T):
            want += _roll_zero(res[t].astype(np.float64) * lam, vy * t, vx * t)
            wantD += _roll_zero(lam, vy * t, vx * t)
        np.testing.assert_allclose(N[0], want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(D[0], wantD, rtol=1e-12, atol=1e-12)


def test_integer_velocity_gaussian_is_shifted_correlation(oracle):
    g = _rng(7)
    T, H, W = 6, 15, 15
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.ones((H, W), np.float32)
    lam = oracle.inverse_variance(sigma)
    shifts, taps = oracle.trajectory_table([1.0, -1.0, 0.0], [0.0, 1.0, -1.0], T)
    N, D = oracle.search_full(res, lam, shifts, taps)
    w0 = oracle.prf_taps(0.0, 0.0)
    for k, (vx, vy) in enumerate([(1, 0), (-1, 1), (0, -1)]):
        want = np.zeros((H, W))
        for t in range(T):
            # correlate on a zero-padded frame so that shifted footprints that
            # straddle the border keep their in-frame part
            big = signal.correlate2d(np.pad(res[t].astype(np.float64), 8), w0, mode="same")
            want += _shift_padded(big, vy * t, vx * t, 8, H, W)
        np.testing.assert_allclose(N[k], want, rtol=1e-12, atol=1e-12)


def _shift_padded(big, oy, ox, pad, H, W):
    return big[pad + oy:pad + oy + H, pad + ox:pad + ox + W]


# ---------------------------------------------------------- closed forms --

@pytest.mark.parametrize("seed", [0, 1])
def test_noiseless_injection_closed_form(oracle, seed):
    """Section 4.1: injection adds flux times the filter.  With no noise the
    matched filter at the injected start pixel returns the flux (N/D = f) and
    SNR = f sqrt(D) = sqrt(sum f^2 w^2 / sigma^2)."""
    g = _rng(seed)
    T, H, W = 12, 20, 24
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.05).astype(np.uint8)
    vx = np.array([0.35, -0.2, 0.05])
    vy = np.array([-0.15, 0.3, 0.0])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma, mask)
    for k in range(3):
        py, px, f = 9, 11, 2.5
        res = np.zeros((T, H, W))
        oracle.inject(res, shifts[k], taps[k], py, px, f)
        N, D = oracle.search_points(res.astype(np.float32), lam, shifts, taps, [py], [px], [k])
        # injection values are float64; the float32 copy adds a relative 6e-8 per term
        assert abs(N[0] / D[0] - f) < 1e-6 * f
        direct = 0.0
        for t in range(T):
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    qy, qx = py + shifts[k, t, 1] + dy, px + shifts[k, t, 0] + dx
                    direct += (f * taps[k, t, dy + 2, dx + 2]) ** 2 / float(sigma[qy, qx]) ** 2 \
                        * (1 - mask[qy, qx])
        snr = N[0] / np.sqrt(D[0])
        assert abs(snr - np.sqrt(direct)) < 1e-6 * np.sqrt(direct)


def test_injection_float64_exact(oracle):
    """Same closed form with data exactly representable in float32."""
    T, H, W = 8, 16, 16
    sigma = np.full((H, W), 2.0, np.float32)
    lam = oracle.inverse_variance(sigma)
    shifts = np.zeros((1, T, 2), np.int32)
    shifts[0, :, 0] = np.arange(T) // 2
    taps = np.zeros((1, T, 5, 5))
    taps[0, :, 1:4, 1:4] = [[0.0625, 0.125, 0.0625], [0.125, 0.25, 0.125], [0.0625, 0.125, 0.0625]]
    res = np.zeros((T, H, W))
    oracle.inject(res, shifts[0], taps[0], 6, 5, 4.0)
    N, D = oracle.search_points(res.astype(np.float32), lam, shifts, taps, [6], [5], [0])
    w2 = (taps[0, 0] ** 2).sum()  # 0.140625
    assert D[0] == T * w2 / 4.0
    assert N[0] == 4.0 * D[0]


# -------------------------------------------------------------- invariants

def test_linearity_scaling_mask_translation(oracle):
    g = _rng(12)
    T, H, W = 5, 18, 18
    # dyadic values with few bits: 2 r1 - r2 / 2 is exact in float32
    r1 = (np.round(64 * g.standard_normal((T, H, W))) / 64).astype(np.float32)
    r2 = (np.round(64 * g.standard_normal((T, H, W))) / 64).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.1).astype(np.uint8)
    vx = np.array([0.4, -0.3])
    vy = np.array([0.1, 0.45])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma, mask)
    N1, D1 = oracle.search_full(r1, lam, shifts, taps)
    N2, _ = oracle.search_full(r2, lam, shifts, taps)
    N12, D12 = oracle.search_full((2 * r1 - 0.5 * r2).astype(np.float32), lam, shifts, taps)
    np.testing.assert_allclose(N12, 2 * N1 - 0.5 * N2, atol=1e-10)
    np.testing.assert_array_equal(D12, D1)
    # sigma -> c sigma: SNR -> SNR / c
    c = 2.0
    lam_c = oracle.inverse_variance(sigma * np.float32(c), mask)
    Nc, Dc = oracle.search_full(r1, lam_c, shifts, taps)
    s1 = oracle.snr_and_best(N1, D1)[0]
    sc = oracle.snr_and_best(Nc, Dc)[0]
    np.testing.assert_allclose(sc, s1 / c, rtol=1e-12, atol=1e-12)
    # values under the mask do not matter
    r3 = r1.copy()
    r3[:, mask.astype(bool)] = 1e6
    N3, _ = oracle.search_full(r3, lam, shifts, taps)
    np.testing.assert_allclose(N3, N1, atol=1e-9)
    # translation: shifting data and noise map shifts the output (interior)
    oy, ox = 2, 3
    rs = np.zeros_like(r1)
    rs[:, oy:, ox:] = r1[:, :H - oy, :W - ox]
    ls = np.zeros_like(lam)
    ls[oy:, ox:] = lam[:H - oy, :W - ox]
    Ns, Ds = oracle.search_full(rs, ls, shifts, taps)
    m = 6
    np.testing.assert_allclose(Ns[:, oy + m:H - m, ox + m:W - m], N1[:, m:H - m - oy, m:W - m - ox],
                               atol=1e-10)
    np.testing.assert_allclose(Ds[:, oy + m:H - m, ox + m:W - m], D1[:, m:H - m - oy, m:W - m - ox],
                               rtol=1e-13)


def test_unusable_sigma_counts_as_masked(oracle):
    """A pixel whose noise is 0, negative, NaN or infinite carries no usable
    measurement: it weighs 0 in N and D, exactly as if it were masked (the
    mask excludes pixels, Section 3.2).  Hand-built map: the bad values are
    planted at known pixels and the search is compared with a plain run in
    which those pixels hold sigma = 1 and are masked instead."""
    g = _rng(31)
    T, H, W = 6, 14, 16
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.05).astype(np.uint8)
    bad = {(3, 4): 0.0, (7, 9): -1.0, (10, 2): np.nan, (5, 13): np.inf, (0, 0): -np.inf, (12, 15): -0.0}
    sig_bad = sigma.copy()
    sig_ok = sigma.copy()
    mask_ok = mask.copy()
    for (y, x), v in bad.items():
        sig_bad[y, x] = v
        sig_ok[y, x] = 1.0
        mask_ok[y, x] = 1
    lam_bad = oracle.inverse_variance(sig_bad, mask)
    lam_ok = oracle.inverse_variance(sig_ok, mask_ok)
    for (y, x) in bad:
        assert lam_bad[y, x] == 0.0
    assert np.all(np.isfinite(lam_bad))
    np.testing.assert_array_equal(lam_bad, lam_ok)
    # every other pixel keeps 1 / sigma^2 (or 0 where masked)
    keep = np.ones((H, W), bool)
    for (y, x) in bad:
        keep[y, x] = False
    want = np.where(mask.astype(bool), 0.0, 1.0 / sigma.astype(np.float64) ** 2)
    np.testing.assert_array_equal(lam_bad[keep], want[keep])
    vx = np.array([0.3, -0.2])
    vy = np.array([0.15, 0.4])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    N1, D1 = oracle.search_full(res, lam_bad, shifts, taps)
    N2, D2 = oracle.search_full(res, lam_ok, shifts, taps)
    np.testing.assert_array_equal(N1, N2)
    np.testing.assert_array_equal(D1, D2)
    assert np.all(np.isfinite(N1)) and np.all(np.isfinite(D1))


# ------------------------------------------------- precision form (16-bit) --

def test_bf16_rounding_is_round_to_nearest_even(oracle):
    # the oracle's bf16 rounding (written from the definition) against the
    # library conversion of torch, on random values, exact ties with an odd
    # and an even kept part, negatives, zeros and subnormals
    torch = pytest.importorskip("torch")
    g = _rng(41)
    x = (g.standard_normal(20000) * np.exp(g.uniform(-30, 30, 20000))).astype(np.float32)
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0xBF818000, 0x00018000, 0x7F7F7FFF], np.uint32)
    x = np.concatenate([x, ties.view(np.float32), np.array([0.0, -0.0, 1e-42, -1e-42], np.float32)])
    got = oracle.round_to_bf16(x)
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes to the even 1
    assert got[-10] == np.float32(1.0) and got[-9] == np.float32(1.0 + 2.0 ** -6)


def test_weighted_stack16_exact_when_representable(oracle):
    # lambda and the frame scales powers of two and small integer residuals:
    # lambda * alpha * r is exact in 16 bits, so the stored stack times beta
    # equals it and the weighted search equals the plain one exactly
    g = _rng(42)
    T, H, W = 7, 19, 23
    r = g.integers(-60, 61, size=(T, H, W)).astype(np.float32)
    sigma = (2.0 ** g.integers(-2, 3, size=(H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.05).astype(np.uint8)
    alpha = (2.0 ** g.integers(-3, 4, size=T)).astype(np.float32)
    vx = np.array([0.3, -0.25, 0.0])
    vy = np.array([0.1, 0.2, -0.35])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma, mask)
    N0, D0 = oracle.search_full(r, lam, shifts, taps, frame_scale=alpha.astype(np.float64))
    for dt in ("bf16", "fp16"):
        q, beta = oracle.weighted_stack16(r, sigma, mask, alpha, dt)
        y = lam[None] * alpha[:, None, None, ] * r.astype(np.float64)
        np.testing.assert_array_equal(q * beta[:, None, None], y)
        N, D = oracle.search_weighted(q, beta, lam, shifts, taps)
        np.testing.assert_allclose(N, N0, rtol=1e-13, atol=1e-13)
        np.testing.assert_array_equal(D, D0)


def test_fp16_frame_scale_bounds(oracle):
    # beta_t is the power of two with beta / 2 < lambda_max * |alpha_t| <=
    # beta: the largest storable residual at the largest weight stays finite
    # (negative frame scales included)
    g = _rng(43)
    T, H, W = 9, 12, 14
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    alpha = (np.exp(g.uniform(-12, 12, T)) * np.where(np.arange(T) % 3 == 0, -1, 1)).astype(np.float32)
    r = np.full((T, H, W), 65504.0, np.float32)
    r[:, 0, 0] = -65504.0
    q, beta = oracle.weighted_stack16(r, sigma, None, alpha, "fp16")
    lam = oracle.inverse_variance(sigma)
    x = (np.float32(lam.astype(np.float32).max()) * np.abs(alpha)).astype(np.float64)
    m, e = np.frexp(beta)
    assert np.all(m == 0.5)  # powers of two
    assert np.all((beta / 2 < x) & (x <= beta))
    assert np.all(np.isfinite(q)) and np.abs(q).max() <= 65504


def test_weighted_stack16_rounding_error_bound(oracle):
    # each stored value is the weighted residual to within half a unit in
    # the last place of its 16-bit type: relative 2^-8 for bf16 (8
    # significant bits), 2^-11 for normal fp16 values (11 bits), so N moves
    # by at most that times sum |W y|
    g = _rng(44)
    T, H, W = 10, 30, 33
    r = (g.standard_normal((T, H, W)) * 40).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    alpha = np.exp(g.uniform(-2, 2, T)).astype(np.float32)
    vx = np.array([0.2, -0.4])
    vy = np.array([0.15, 0.05])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma)
    y = lam.astype(np.float32)[None] * (alpha[:, None, None] * r)
    N0, _ = oracle.search_full(r, lam, shifts, taps, frame_scale=alpha.astype(np.float64))
    Nabs, _ = oracle.search_full(np.abs(y), np.ones((H, W)), shifts, np.abs(taps))
    for dt, u in (("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)):
        q, beta = oracle.weighted_stack16(r, sigma, None, alpha, dt)
        big = np.abs(y) > 1e-3 * beta[:, None, None]  # fp16: normal range
        rel = np.abs(q * beta[:, None, None] - y.astype(np.float64)) / np.abs(y)
        assert rel[big].max() <= u * (1 + 1e-6)
        assert rel[big].max() > u / 4  # the bound is attained in order of magnitude
        N, _ = oracle.search_weighted(q, beta, lam, shifts, taps)
        assert np.all(np.abs(N - N0) <= (u + 1e-6) * Nabs + 1e-12)


# ------------------------------------------------------------ statistics --

def test_pure_noise_snr_is_standard_normal(oracle):
    """Matched filter with the right noise model: SNR ~ N(0, 1) on pure noise.

    Samples are independent: start pixels 16 px apart (farther than a
    trajectory's footprint over the stack) and a fresh noise draw each time.
    """
    g = _rng(21)
    T, H, W = 24, 64, 64
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.01).astype(np.uint8)
    vx = np.array([0.0, 0.3, -0.25, 0.1])
    vy = np.array([0.0, 0.1, 0.2, -0.3])
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma, mask)
    grid = np.array([8, 24, 40, 56])
    ys, xs = [a.ravel() for a in np.meshgrid(grid, grid, indexing="ij")]
    ys4, xs4 = np.repeat(ys, 4), np.repeat(xs, 4)
    ks4 = np.tile(np.arange(4), ys.size)
    draws = 200
    snr = np.zeros((draws, ys.size, 4))
    for d in range(draws):
        res = (sigma[None] * g.standard_normal((T, H, W))).astype(np.float32)
        N, D = oracle.search_points(res, lam, shifts, taps, ys4, xs4, ks4)
        snr[d] = (N / np.sqrt(D)).reshape(ys.size, 4)
    n = draws * ys.size
    for k in range(4):
        v = snr[:, :, k].ravel()
        assert abs(v.mean()) < 4 / np.sqrt(n)
        assert abs(v.var() - 1.0) < 4 * np.sqrt(2 / n)
    # the same statistic with a wrong normalisation is far off
    assert abs((snr / np.sqrt(2.0)).var() - 1.0) > 0.4


def test_injected_movers_recovered(oracle):
    """Section 4.1 protocol on Gaussian noise: movers on a 20 x 80 px grid at
    grid velocities are found at their start pixel with their trajectory."""
    g = _rng(31)
    T, H, W = 40, 48, 176
    sigma = np.ones((H, W), np.float32)
    vx = np.array([-0.15, -0.05, 0.05, 0.15] * 4)
    vy = np.repeat([-0.15, -0.05, 0.05, 0.15], 4)
    shifts, taps = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma)
    res = g.standard_normal((T, H, W))
    truth = []
    for iy, py in enumerate([14, 34]):
        for ix, px in enumerate([20, 100]):
            k = int(g.integers(0, 16))
            oracle.inject(res, shifts[k], taps[k], py, px, 5.0)  # SNR about 10
            truth.append((py, px, k))
    N, D = oracle.search_full(res.astype(np.float32), lam, shifts, taps)
    snr, valid, smax, amax = oracle.snr_and_best(N, D)
    for py, px, k in truth:
        assert smax[py, px] > 8
        assert amax[py, px] == k
        win = smax[py - 3:py + 4, px - 3:px + 4]
        assert win.max() == smax[py, px]


# ----------------------------------------------------------- selection ---

def test_best_tie_and_empty_rules(oracle):
    N = np.array([[[1.0, 0.0]], [[1.0, 0.0]], [[0.5, 0.0]]])  # K=3, H=1, W=2
    D = np.array([[[1.0, 0.0]], [[1.0, 0.0]], [[1.0, 0.0]]])
    snr, valid, smax, amax = oracle.snr_and_best(N, D)
    assert amax[0, 0] == 0 and smax[0, 0] == 1.0  # tie -> smallest k
    assert amax[0, 1] == -1 and smax[0, 1] == 0.0  # no filter with D > 0
    N = np.array([[[-3.0]], [[-2.0]]])
    D = np.array([[[1.0]], [[0.0]]])
    snr, valid, smax, amax = oracle.snr_and_best(N, D)
    assert amax[0, 0] == 0 and smax[0, 0] == -3.0  # k with D = 0 is not a candidate


def test_topk_order_rule(oracle):
    smax = np.array([[3.0, 5.0, 3.0], [5.0, 1.0, 0.0]])
    amax = np.array([[0, 1, 2], [3, 0, -1]])
    assert list(oracle.topk_order(smax, amax, 4)) == [1, 3, 0, 2]
    assert list(oracle.topk_order(smax, amax, 10)) == [1, 3, 0, 2, 4]


# ------------------------------------------- frame times and jitter (NEXT) --

def _golden_frames():
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "trajectory_frames.txt")
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            v, tau, j, s, ph = (float(x) for x in line)
            rows.append((v, tau, j, int(s), ph))
    return rows


def test_trajectory_frames_golden(oracle):
    rows = _golden_frames()
    assert len(rows) >= 10
    for v, tau, j, s, ph in rows:
        sx, tx = oracle.trajectory_table_frames([v], [0.0], 1, times=[tau], jitter=[[j, 0.0]])
        assert (sx[0, 0, 0], sx[0, 0, 1]) == (s, 0), (v, tau, j)
        np.testing.assert_allclose(tx[0, 0], oracle.prf_taps(ph, 0.0), atol=1e-14)
        sy, ty = oracle.trajectory_table_frames([0.0], [v], 1, times=[tau], jitter=[[0.0, j]])
        assert (sy[0, 0, 0], sy[0, 0, 1]) == (0, s), (v, tau, j)
        np.testing.assert_allclose(ty[0, 0], oracle.prf_taps(0.0, ph), atol=1e-14)


def test_frames_reduce_to_linear_and_select_rows(oracle):
    # frames at 0..T-1 without jitter: the linear table; integer times with a
    # gap: the rows of the linear table at those times (missing frames drop out)
    vx, vy = [0.3, -0.17, 0.0], [0.11, 0.0, -0.42]
    s0, t0 = oracle.trajectory_table(vx, vy, 40)
    s1, t1 = oracle.trajectory_table_frames(vx, vy, 40)
    assert np.array_equal(s0, s1) and np.array_equal(t0, t1)
    tau = np.array([0, 1, 2, 3, 17, 18, 19, 39])
    s2, t2 = oracle.trajectory_table_frames(vx, vy, len(tau), times=tau.astype(float))
    assert np.array_equal(s2, s0[:, tau]) and np.array_equal(t2, t0[:, tau])


def test_integer_jitter_moves_the_base_pixel_only(oracle):
    g = _rng(8)
    T = 12
    j = g.integers(-3, 4, size=(T, 2)).astype(float)
    vx, vy = g.uniform(-0.4, 0.4, 5), g.uniform(-0.4, 0.4, 5)
    s0, t0 = oracle.trajectory_table(vx, vy, T)
    s1, t1 = oracle.trajectory_table_frames(vx, vy, T, jitter=j)
    assert np.array_equal(s1, s0 + j.astype(np.int32)[None])
    np.testing.assert_allclose(t1, t0, atol=1e-15)


def test_jittered_gapped_injection_closed_form(oracle):
    """A source rendered by the scene model (independent PRF code in synth) at
    p + v tau_t + j_t in each frame: the matched filter built with the same
    times and jitter returns N/D = f and SNR = f sqrt(D) at p (Section 4.1
    injection, Section 2.1 jitter, Fig. 3 time jump)."""
    from paper_2209_09848_gb300 import synth
    g = _rng(4)
    T, H, W = 14, 30, 34
    tau = np.sort(g.choice(np.arange(40), size=T, replace=False)).astype(float)
    jit = g.uniform(-0.3, 0.3, size=(T, 2))
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    lam = oracle.inverse_variance(sigma)
    vx, vy = np.array([0.21, -0.13]), np.array([-0.08, 0.17])
    shifts, taps = oracle.trajectory_table_frames(vx, vy, T, times=tau, jitter=jit)
    py, px, f = 15, 16, 3.0
    for k in range(2):
        res = np.zeros((T, H, W))
        for t in range(T):
            cy = py + vy[k] * tau[t] + jit[t, 1]
            cx = px + vx[k] * tau[t] + jit[t, 0]
            res[t] = synth.render_movers_np(1, H, W, [(cy, cx, 0.0, 0.0, f)])[0]
        N, D = oracle.search_points(res.astype(np.float32), lam, shifts, taps, [py], [px], [k])
        assert abs(N[0] / D[0] - f) < 1e-6 * f
        # the linear table without times and jitter misses part of the flux
        s_lin, t_lin = oracle.trajectory_table(vx, vy, T)
        N2, D2 = oracle.search_points(res.astype(np.float32), lam, s_lin, t_lin, [py], [px], [k])
        assert N2[0] / D2[0] < 0.9 * f


def test_shift_stack_kind_is_single_tap_shift_and_add(oracle):
    """Section 3.2: the shift-stack filter of Rice et al. has one value of 1
    per frame, in the pixel holding the source's centre; N is then the sum of
    the weighted frames shifted along the trajectory (numpy roll-and-add)."""
    for ph in [(0.0, 0.0), (0.49, -0.3), (-0.5, 0.2)]:
        t = oracle.prf_taps(*ph, kind=2)
        assert t[2, 2] == 1.0 and t.sum() == 1.0
    g = _rng(12)
    T, H, W = 9, 30, 34
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    vx, vy = np.array([0.37, -0.61]), np.array([0.22, 0.45])
    shifts, taps = oracle.trajectory_table(vx, vy, T, kind=2)
    lam = oracle.inverse_variance(sigma)
    N, D = oracle.search_full(res, lam, shifts, taps)
    wr = res.astype(np.float64) * lam[None]
    for k in range(2):
        n = np.zeros((H, W))
        d = np.zeros((H, W))
        for t in range(T):
            sx = int(np.floor(vx[k] * t + 0.5))
            sy = int(np.floor(vy[k] * t + 0.5))
            n += np.roll(wr[t], (-sy, -sx), axis=(0, 1))
            d += np.roll(lam, (-sy, -sx), axis=(0, 1))
        inner = (slice(6, H - 6), slice(6, W - 6))
        np.testing.assert_allclose(N[k][inner], n[inner], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(D[k][inner], d[inner], rtol=1e-12, atol=1e-12)


# ------------------------------------------------ phase-quantised (NEXT) --

def test_quantised_table_hand_worked(oracle):
    # v = 0.3, Q = 4: phases 0, 0.3, -0.4, -0.1, 0.2 round to 0, 0.25, -0.5,
    # 0, 0.25 (halves up); base pixels as for the exact table
    sh, tp = oracle.trajectory_table_quantised([0.3], [0.0], 5, 4)
    assert list(sh[0, :, 0]) == [0, 0, 1, 1, 1]
    for t, ph in enumerate([0.0, 0.25, -0.5, 0.0, 0.25]):
        np.testing.assert_allclose(tp[0, t], oracle.prf_taps(ph, 0.0), atol=1e-15)


def test_quantised_table_on_grid_and_converging(oracle):
    # phases already on the 1/Q grid: the exact table; otherwise the taps
    # approach the exact ones as 1/Q
    s0, t0 = oracle.trajectory_table([0.25, -0.125], [0.5, 0.375], 16)
    s1, t1 = oracle.trajectory_table_quantised([0.25, -0.125], [0.5, 0.375], 16, 8)
    assert np.array_equal(s0, s1) and np.array_equal(t0, t1)
    g = _rng(21)
    vx, vy = g.uniform(-0.5, 0.5, 6), g.uniform(-0.5, 0.5, 6)
    s0, t0 = oracle.trajectory_table(vx, vy, 40)
    errs = []
    for Q in (2, 4, 8, 16, 32):
        sq, tq = oracle.trajectory_table_quantised(vx, vy, 40, Q)
        assert np.array_equal(sq, s0)
        errs.append(np.abs(tq - t0).max())
        assert errs[-1] <= 0.5 / Q  # |dW/dphase| < 1 for the sigma = 0.7 footprint
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_quantised_filter_never_beats_exact_on_injection(oracle):
    """A noiseless source injected with the exact filter: a mismatched
    (quantised) template gives N_q / sqrt(D_q) <= f sqrt(D) (Cauchy-Schwarz),
    and loses little at Q = 4."""
    g = _rng(22)
    T, H, W = 30, 24, 28
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    lam = oracle.inverse_variance(sigma)
    vx, vy = np.array([0.23, -0.31]), np.array([0.17, 0.05])
    sh, tp = oracle.trajectory_table(vx, vy, T)
    py, px, f = 11, 13, 2.0
    for k in range(2):
        res = np.zeros((T, H, W))
        oracle.inject(res, sh[k], tp[k], py, px, f)
        N, D = oracle.search_points(res.astype(np.float32), lam, sh, tp, [py], [px], [k])
        exact = N[0] / np.sqrt(D[0])
        for Q in (2, 4, 8):
            sq, tq = oracle.trajectory_table_quantised(vx, vy, T, Q)
            Nq, Dq = oracle.search_points(res.astype(np.float32), lam, sq, tq, [py], [px], [k])
            snr_q = Nq[0] / np.sqrt(Dq[0])
            assert snr_q <= exact * (1 + 1e-6)
            if Q >= 4:
                assert snr_q >= 0.97 * exact


@pytest.mark.parametrize("T,H,W,Q,vmax,masked", [
    (7, 13, 17, 4, 0.4, False),
    (9, 11, 9, 3, 1.6, True),     # odd Q; shifts that carry start pixels out of the frame
    (5, 6, 21, 8, 0.9, True),
])
def test_quantised_gather_equals_quantised_bank(oracle, T, H, W, Q, vmax, masked):
    # precompute-then-gather (planes per rounded phase, one gather per
    # trajectory) against the plain loops on the quantised filter bank
    g = _rng(T * 31 + W)
    res = g.standard_normal((T, H, W)).astype(np.float32)
    sigma = np.exp(0.3 * g.standard_normal((H, W))).astype(np.float32)
    mask = (g.random((H, W)) < 0.1).astype(np.uint8) if masked else None
    lam = oracle.inverse_variance(sigma, mask)
    vx, vy = g.uniform(-vmax, vmax, 6), g.uniform(-vmax, vmax, 6)
    vx[0], vy[0] = 0.0, 0.0
    sh, tp = oracle.trajectory_table_quantised(vx, vy, T, Q)
    N0, D0 = oracle.search_full(res, lam, sh, tp)
    N1, D1 = oracle.search_quantised_gather(res, lam, vx, vy, Q)
    np.testing.assert_allclose(N1, N0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D1, D0, rtol=1e-12, atol=1e-12)
    assert (D0 > 0).any()


def test_quantised_gather_on_grid_is_exact_search(oracle):
    # velocities whose phases all lie on the 1/Q grid: the exact search
    g = _rng(23)
    T, H, W = 12, 10, 14
    res = g.standard_normal((T, H, W)).astype(np.float32)
    lam = oracle.inverse_variance(np.ones((H, W), np.float32))
    vx, vy = np.array([0.25, -0.5, 0.125]), np.array([0.375, 0.0, -0.25])
    sh, tp = oracle.trajectory_table(vx, vy, T)
    N0, D0 = oracle.search_numpy(res, lam, sh, tp)
    N1, D1 = oracle.search_quantised_gather(res, lam, vx, vy, 8)
    np.testing.assert_allclose(N1, N0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D1, D0, rtol=1e-12, atol=1e-12)


def test_quantised_frames_reduce_to_quantised_table(oracle):
    # the frame model with quantised phases: no times and no jitter is the
    # linear quantised bank, zero jitter and times 0..T-1 likewise
    g = _rng(24)
    vx, vy = g.uniform(-0.6, 0.6, 7), g.uniform(-0.6, 0.6, 7)
    T = 33
    for Q in (1, 3, 4):
        s0, t0 = oracle.trajectory_table_quantised(vx, vy, T, Q)
        s1, t1 = oracle.trajectory_table_frames(vx, vy, T, Q=Q)
        s2, t2 = oracle.trajectory_table_frames(vx, vy, T, times=np.arange(T, dtype=float),
                                                jitter=np.zeros((T, 2)), Q=Q)
        assert np.array_equal(s0, s1) and np.array_equal(t0, t1)
        assert np.array_equal(s0, s2) and np.array_equal(t0, t2)
    # integer jitter moves the base pixel and leaves the rounded phase alone
    s0, t0 = oracle.trajectory_table_frames(vx, vy, T, Q=4)
    j = np.tile([[2.0, -3.0]], (T, 1))
    s1, t1 = oracle.trajectory_table_frames(vx, vy, T, jitter=j, Q=4)
    assert np.array_equal(s1 - s0, np.broadcast_to([2, -3], s0.shape)) and np.array_equal(t0, t1)
