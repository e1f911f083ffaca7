"""Filter banks with frame times and pointing jitter (Section 2.1: the
filter follows the trajectory including the jitter; Fig. 3: the downlink
gap makes time jump) through mf_prf_table_create_frames, against the FP64
oracle's own table with the same frame model.  Same bar as the linear
search: |delta SNR| <= 1e-5 max(1, |SNR|), identical argmax where the two
best filters differ by more than 1e-3."""
import numpy as np
import pytest

from _util import check_search

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    assert torch.cuda.is_available()
    m.load()
    return m


def _frames(T, seed, gap=0, jit=0.3, frac=False):
    g = np.random.default_rng(seed)
    tau = np.arange(T, dtype=np.float64)
    if gap:
        tau[T // 2:] += gap  # frames missing while the spacecraft downlinks
    if frac:
        tau += g.uniform(-0.2, 0.2, T)  # mid-exposure times off the cadence
    jitter = g.uniform(-jit, jit, size=(T, 2))
    return tau, jitter


def _search(mf, c, table):
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = None if c["mask"] is None else torch.from_numpy(c["mask"]).cuda()
    smax, amax, sall = mf.search(r, s, table, mask=m, want_all=True)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    return smax.cpu().numpy(), amax.cpu().numpy(), sall.cpu().numpy()


@pytest.mark.parametrize("T,H,W,gap,jit,frac,layout", [
    (24, 90, 120, 0, 0.3, False, {}),                 # jitter only, factored numerator
    (30, 77, 101, 200, 0.25, False, {}),              # a 200-frame gap, factored
    (30, 77, 101, 200, 0.25, True, {"kernel": 1}),    # fractional times, general numerator
    (40, 131, 97, 37, 1.7, True, {"segments": 3}),    # multi-pixel jitter, time segments
    (9, 40, 60, 5, 0.45, False, {"kernel": 2, "group": 2, "tile_w": 64}),
])
def test_frames_search_matches_oracle(mf, oracle, T, H, W, gap, jit, frac, layout):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, T + H, mask_frac=0.02, movers=3)
    vx, vy = synth.velocity_grid(4, 5, -0.3, 0.3)
    tau, jitter = _frames(T, T * 7 + W, gap, jit, frac)
    table = mf.prf_table_create(vx, vy, T, times=tau, jitter=jitter, **layout)
    info = table.info()
    if layout.get("kernel"):
        assert info["kernel"] == layout["kernel"]
    sh_g, tp_g = table.export()
    sh, tp = oracle.trajectory_table_frames(vx, vy, T, times=tau, jitter=jitter)
    assert np.array_equal(sh_g, sh)
    np.testing.assert_allclose(tp_g, tp, rtol=0, atol=1e-15)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _search(mf, c, table)
    check_search(smax, amax, sall, N, D, oracle, label="frames %s" % ((T, H, W, gap, jit, layout),))


def test_frames_default_equals_linear_table(mf):
    from paper_2209_09848_gb300 import synth
    T = 12
    vx, vy = synth.velocity_grid(3, 3, -0.2, 0.2)
    a = mf.prf_table_create(vx, vy, T)
    b = mf.prf_table_create(vx, vy, T, times=np.arange(T, dtype=float), jitter=np.zeros((T, 2)))
    sa, ta = a.export()
    sb, tb = b.export()
    assert np.array_equal(sa, sb) and np.array_equal(ta, tb)


def test_frames_rescore_uses_the_frame_model(mf, oracle):
    # the FP64 re-score reads the table's shifts and taps: the jittered ones
    # (candidates picked from a host-generated score map)
    from paper_2209_09848_gb300 import synth
    T, H, W = 16, 48, 64
    c = synth.small_case(T, H, W, 3, mask_frac=0.01, movers=2)
    vx, vy = synth.velocity_grid(3, 2, -0.25, 0.25)
    tau, jitter = _frames(T, 11, gap=50, jit=0.4, frac=True)
    table = mf.prf_table_create(vx, vy, T, times=tau, jitter=jitter)
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    s_max, a_max = synth.score_map(H, W, seed=12, K=len(vx), mask_frac=0.0)
    raw, n = mf.rescore_topk(r, s, table, torch.from_numpy(s_max).cuda(), torch.from_numpy(a_max).cuda(), 32,
                             mask=m)
    torch.cuda.synchronize()
    cand = mf.decode_candidates(raw, int(n.item()))
    want = oracle.topk_order(s_max, a_max, 32)
    assert np.array_equal(cand["y"].astype(np.int64) * W + cand["x"], want)
    sh, tp = oracle.trajectory_table_frames(vx, vy, T, times=tau, jitter=jitter)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_points(c["res"], lam, sh, tp, (want // W).astype(np.int32), (want % W).astype(np.int32),
                                a_max.ravel()[want])
    ok = D > 0
    np.testing.assert_allclose(cand["snr"][ok], N[ok] / np.sqrt(D[ok]), rtol=1e-9, atol=1e-12)


def test_frames_rejects_bad_models(mf):
    vx = vy = np.zeros(2)
    with pytest.raises(mf.MFError):
        mf.prf_table_create(vx, vy, 3, times=np.array([0.0, np.nan, 2.0]))
    with pytest.raises(mf.MFError):
        mf.prf_table_create(vx, vy, 3, jitter=np.array([[0.0, 0.0], [np.inf, 0.0], [0.0, 0.0]]))
    with pytest.raises(mf.MFError):
        mf.prf_table_create(np.array([1.0]), np.array([0.0]), 2, times=np.array([0.0, 3e6]))
    with pytest.raises(ValueError):
        mf.prf_table_create(vx, vy, 3, times=np.zeros(4))

