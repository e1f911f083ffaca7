"""mf_background_refit (Section 3.1: per-pixel Huber fit of the background
and its jitter Taylor terms, with the low-resolution scattered light
subtracted) against the FP64 oracle.  The kernel sums in FP32 over an
orthonormal basis; residuals agree to |delta r| <= 2e-6 max|D| (the
rounding of FP32 frames of that size), and the fitted background phi . beta
(the coefficients themselves are ill-conditioned in the Taylor basis) to
the same bound."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    assert torch.cuda.is_available()
    m.load()
    return m


def _check(mf, c, delta, M, scatter=True, in_place=False):
    from oracle import background as ob
    D = torch.from_numpy(c["D"]).cuda()
    S = torch.from_numpy(c["S"]).cuda() if scatter else None
    out = D if in_place else None
    R, coef = mf.background_refit(D.clone() if not in_place else D, c["jitter"], delta, M, scatter=S,
                                  resid=out if in_place else None)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    co, Ro = ob.refit(c["D"], c["jitter"], delta, M, S=c["S"] if scatter else None)
    tol = 2e-6 * max(1.0, float(np.abs(c["D"]).max()))
    err = np.abs(R.cpu().numpy().astype(np.float64) - Ro)
    assert err.max() <= tol, "residual max err %.3g > %.3g" % (err.max(), tol)
    phi = ob.basis(c["jitter"])
    fit_g = np.einsum("tk,hwk->thw", phi, coef.cpu().numpy().astype(np.float64))
    fit_o = np.einsum("tk,hwk->thw", phi, co)
    assert np.abs(fit_g - fit_o).max() <= 4 * tol
    return R, coef


@pytest.mark.parametrize("T,H,W,n,M,delta", [
    (100, 64, 48, 8, 10, 1.345),
    (300, 37, 53, 4, 5, 1.0),        # pixel count not a multiple of the CTA, > 1 basis chunk
    (6, 20, 30, 2, 3, 1.345),         # the smallest frame count
    (64, 33, 17, 16, 0, 1.345),       # least-squares start only
    (80, 40, 40, 8, 4, float("inf")),  # least squares throughout
    (600, 16, 16, 8, 20, 0.5),       # many clipped residuals, three basis chunks
])
def test_refit_matches_oracle(mf, T, H, W, n, M, delta):
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(T, H, W, seed=T + H, n=n, n_movers=2)
    _check(mf, c, delta, M)


def test_refit_without_scatter_and_in_place(mf):
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(50, 30, 40, seed=3, n=4)
    _check(mf, c, 1.345, 6, scatter=False)
    _check(mf, c, 1.345, 6, in_place=True)


def test_refit_removes_background_and_keeps_movers(mf):
    # a bright mover survives in the residual; the background does not
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(200, 64, 64, seed=8, n=8, n_movers=4, outlier_frac=0.0)
    R, coef = mf.background_refit(torch.from_numpy(c["D"]).cuda(), c["jitter"], 1.345, 10,
                                  scatter=torch.from_numpy(c["S"]).cuda())
    r = R.cpu().numpy()
    inner = r[:, 8:-8, 8:-8]
    assert abs(np.median(inner)) < 0.1 and np.percentile(np.abs(inner), 50) < 1.0
    assert r.max() > 1.0  # the movers


def test_refit_deterministic(mf):
    from paper_2209_09848_gb300 import synth
    c = synth.background_case(90, 50, 50, seed=9, n=8)
    D = torch.from_numpy(c["D"]).cuda()
    a = mf.background_refit(D, c["jitter"], 1.345, 5, scatter=torch.from_numpy(c["S"]).cuda())
    b = mf.background_refit(D, c["jitter"], 1.345, 5, scatter=torch.from_numpy(c["S"]).cuda())
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_refit_rejects_bad_arguments(mf):
    D = torch.zeros((10, 4, 4), device="cuda")
    jit = np.random.default_rng(0).uniform(-0.2, 0.2, size=(10, 2))
    for kw in (dict(delta=0.0), dict(delta=float("nan")), dict(iterations=-1), dict(iterations=1001)):
        args = dict(delta=1.0, iterations=2)
        args.update(kw)
        with pytest.raises(mf.MFError):
            mf.background_refit(D, jit, args["delta"], args["iterations"])
    with pytest.raises(mf.MFError):  # constant jitter: x and x^2 collinear with 1
        mf.background_refit(D, np.zeros((10, 2)), 1.0, 2)
    with pytest.raises(mf.MFError):  # fewer frames than coefficients
        mf.background_refit(torch.zeros((5, 4, 4), device="cuda"), jit[:5], 1.0, 2)
    bad = jit.copy()
    bad[3, 1] = np.inf
    with pytest.raises(mf.MFError):
        mf.background_refit(D, bad, 1.0, 2)
