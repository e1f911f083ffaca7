"""mf_rescore_topk: candidate selection is exact integer work (bit-exact against
the oracle's ordering rule on the same snr_max/argmax maps, generated on the
host), and the FP64 re-score matches the FP64 oracle, evaluated at the
oracle's own selection, to 1e-9 relative (two FP64 sums in different
order)."""
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


@pytest.mark.parametrize("k_top,T,H,W,mask_frac", [(64, 20, 70, 90, 0.02), (500, 12, 48, 64, 0.0),
                                                   (4096, 8, 64, 80, 0.01), (1, 5, 16, 16, 0.0)])
def test_rescore_matches_oracle(mf, oracle, k_top, T, H, W, mask_frac):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, 17 + k_top, mask_frac=mask_frac, movers=4)
    vx, vy = synth.velocity_grid(4, 3, -0.3, 0.3)
    K = len(vx)
    table = mf.prf_table_create(vx, vy, T)
    # a best-score map and its trajectories from the host generator: the
    # selection and the re-score read them, not a search's output
    s_max, a_max = synth.score_map(H, W, seed=k_top + H, K=K, mask_frac=mask_frac)
    dev = "cuda"
    r = torch.from_numpy(c["res"]).to(dev)
    s = torch.from_numpy(c["sigma"]).to(dev)
    m = None if c["mask"] is None else torch.from_numpy(c["mask"]).to(dev)
    k_eff = min(k_top, H * W)
    raw, n = mf.rescore_topk(r, s, table, torch.from_numpy(s_max).to(dev), torch.from_numpy(a_max).to(dev),
                             k_eff, mask=m)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    n = int(n.item())
    cands = mf.decode_candidates(raw, n)
    want = oracle.topk_order(s_max, a_max, k_eff)
    assert n == len(want)
    got_idx = cands["y"].astype(np.int64) * W + cands["x"]
    assert np.array_equal(got_idx, want)
    wy, wx = want // W, want % W
    wk = a_max.ravel()[want]
    assert np.array_equal(cands["k"], wk)
    assert np.array_equal(cands["snr_search"], s_max.ravel()[want])
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_points(c["res"], lam, sh, tp, wy.astype(np.int32), wx.astype(np.int32), wk)
    ok = D > 0
    np.testing.assert_allclose(cands["snr"][ok], N[ok] / np.sqrt(D[ok]), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(cands["flux"][ok], N[ok] / D[ok], rtol=1e-9, atol=1e-12)
    assert np.all(cands["snr"][~ok] == 0) and np.all(cands["flux"][~ok] == 0)


def test_rescore_reads_bf16_master_as_stored(mf, oracle):
    from paper_2209_09848_gb300 import synth
    T, H, W = 10, 40, 56
    c = synth.small_case(T, H, W, 5, mask_frac=0.01, movers=3)
    vx, vy = synth.velocity_grid(3, 3, -0.2, 0.2)
    table = mf.prf_table_create(vx, vy, T)
    q = torch.from_numpy(c["res"]).to(torch.bfloat16)
    r = q.cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    s_max, a_max = synth.score_map(H, W, seed=6, K=len(vx), mask_frac=0.0)
    raw, n = mf.rescore_topk(r, s, table, torch.from_numpy(s_max).cuda(), torch.from_numpy(a_max).cuda(), 50,
                             mask=m)
    torch.cuda.synchronize()
    cands = mf.decode_candidates(raw, int(n.item()))
    want = oracle.topk_order(s_max, a_max, 50)
    assert np.array_equal(cands["y"].astype(np.int64) * W + cands["x"], want)
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_points(q.float().numpy(), lam, sh, tp, (want // W).astype(np.int32),
                                (want % W).astype(np.int32), a_max.ravel()[want])
    ok = D > 0
    np.testing.assert_allclose(cands["snr"][ok], N[ok] / np.sqrt(D[ok]), rtol=1e-9, atol=1e-12)


def test_rescore_argument_errors(mf):
    T, H, W = 4, 8, 8
    table = mf.prf_table_create([0.1], [0.0], T)
    r = torch.zeros((T, H, W), device="cuda")
    s = torch.ones((H, W), device="cuda")
    smax = torch.zeros((H, W), device="cuda")
    amax = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    with pytest.raises(mf.MFError):
        mf.rescore_topk(r, s, table, smax, amax, 0)
    with pytest.raises(mf.MFError):
        mf.rescore_topk(r, s, table, smax, amax, H * W + 1)
