"""Pins of the background re-fit oracle (Section 3.1, Eqs. 1-4): the
bilinear upsampling against torch's, the least-squares limit against
numpy's lstsq, exact recovery of noise-free models, the converged Huber
fit against a general-purpose minimiser of the Huber loss, monotone loss
and bounded influence of an outlier."""
import numpy as np
import pytest

from oracle import background as ob


def test_upsample_matches_torch_bilinear():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(0)
    S = g.normal(size=(3, 8, 8))
    for H, W in [(64, 64), (50, 37), (8, 8), (3, 5)]:
        want = torch.nn.functional.interpolate(torch.from_numpy(S)[None], size=(H, W), mode="bilinear",
                                               align_corners=False)[0].numpy()
        np.testing.assert_allclose(ob.upsample(S, H, W), want, rtol=0, atol=1e-12)
    assert np.allclose(ob.upsample(np.full((4, 4), 2.5), 17, 9), 2.5)


def test_least_squares_limit():
    g = np.random.default_rng(1)
    T, H, W = 40, 3, 4
    jit = g.uniform(-0.2, 0.2, size=(T, 2))
    D = g.normal(50, 3, size=(T, H, W))
    coef, R = ob.refit(D, jit, np.inf, 3)
    Phi = ob.basis(jit)
    want = np.linalg.lstsq(Phi, D.reshape(T, -1), rcond=None)[0].T.reshape(H, W, 6)
    np.testing.assert_allclose(coef, want, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(R, D - np.einsum("tk,hwk->thw", Phi, want), atol=1e-9)


def test_noise_free_model_recovered_exactly():
    g = np.random.default_rng(2)
    T, H, W = 30, 2, 3
    jit = g.uniform(-0.15, 0.15, size=(T, 2))
    truth = g.normal(size=(H, W, 6)) * [10, 3, 3, 1, 1, 1]
    D = np.einsum("tk,hwk->thw", ob.basis(jit), truth)
    for delta in (0.01, 1.0, np.inf):
        coef, R = ob.refit(D, jit, delta, 5)
        np.testing.assert_allclose(coef, truth, rtol=1e-8, atol=1e-8)
        assert np.abs(R).max() < 1e-9


def test_converged_fit_minimises_huber_loss():
    from scipy import optimize
    g = np.random.default_rng(3)
    T = 80
    jit = g.uniform(-0.2, 0.2, size=(T, 2))
    Phi = ob.basis(jit)
    truth = np.array([100.0, 4.0, -3.0, 1.0, 0.5, -0.7])
    y = Phi @ truth + g.normal(size=T)
    y[g.choice(T, 6, replace=False)] += g.uniform(30, 80, 6)  # outliers: movers, cosmic rays
    delta = 1.345
    coef, _ = ob.refit(y.reshape(T, 1, 1), jit, delta, 400)
    b = coef[0, 0]
    res = optimize.minimize(lambda beta: ob.huber_loss(y - Phi @ beta, delta).sum(),
                            np.linalg.lstsq(Phi, y, rcond=None)[0], method="BFGS",
                            options={"gtol": 1e-10, "maxiter": 10000})
    assert ob.huber_loss(y - Phi @ b, delta).sum() <= res.fun + 1e-7
    np.testing.assert_allclose(b, res.x, rtol=1e-4, atol=1e-4)


def test_loss_decreases_and_outlier_influence_is_bounded():
    g = np.random.default_rng(4)
    T = 60
    jit = g.uniform(-0.2, 0.2, size=(T, 2))
    Phi = ob.basis(jit)
    y = Phi @ np.array([10.0, 1, 1, 0, 0, 0]) + g.normal(size=T)
    delta = 1.0
    losses = [ob.huber_loss(y - Phi @ ob.refit(y.reshape(T, 1, 1), jit, delta, m)[0][0, 0], delta).sum()
              for m in range(8)]
    assert all(b <= a + 1e-12 for a, b in zip(losses, losses[1:]))
    # one outlier of growing size: least squares follows it; the Huber fit
    # sees it only through its clipped residual delta (the estimating
    # equation sum_t phi_t psi(e_t) = 0), so any size beyond the clip gives
    # the same fit (the iteration walks from the least-squares start in steps
    # of at most G^-1 sum |phi| delta, so a larger outlier needs more steps)
    fits = []
    for big in (1e2, 3e2):
        z = y.copy()
        z[7] += big
        ls = ob.refit(z.reshape(T, 1, 1), jit, np.inf, 0)[0][0, 0]
        fits.append(ob.refit(z.reshape(T, 1, 1), jit, delta, 3000)[0][0, 0])
        base = ob.refit(y.reshape(T, 1, 1), jit, np.inf, 0)[0][0, 0]
        assert abs(ls[0] - base[0]) > 1e-3 * big
    np.testing.assert_allclose(fits[0], fits[1], rtol=1e-6, atol=1e-6)


def test_scene_generator_and_refit_end_to_end():
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(60, 48, 40, seed=5, n=16, noise=1.0)
    coef, R = ob.refit(c["D"], c["jitter"], 1.345, 10, S=c["S"])
    # the residual is noise plus the low-resolution model's misfit of the
    # smooth scattered light (largest at the borders, where U extrapolates)
    inner = (slice(None), slice(4, -4), slice(4, -4))
    assert np.median(np.abs(R[inner])) < 1.0
    # the intercept is the well-determined coefficient (the jitter spans
    # +-0.15 px, so the Taylor terms are weakly constrained); pixels hit by a
    # strong outlier are still converging after 10 steps
    err = np.abs(coef[4:-4, 4:-4, 0] - c["coef"][4:-4, 4:-4, 0])
    assert np.median(err) < 1.0 and np.mean(err > 3.0) < 0.02


def test_points_match_full_image():
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(40, 30, 26, seed=6, n=8)
    coef, R = ob.refit(c["D"], c["jitter"], 1.345, 6, S=c["S"])
    g = np.random.default_rng(0)
    ys, xs = g.integers(0, 30, 20), g.integers(0, 26, 20)
    cp, Rp = ob.refit_points(c["D"][:, ys, xs], ys, xs, 30, 26, c["jitter"], 1.345, 6, S=c["S"])
    np.testing.assert_allclose(cp, coef[ys, xs], rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(Rp, R[:, ys, xs], rtol=1e-10, atol=1e-9)
