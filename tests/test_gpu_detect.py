"""mf_detect (Section 3.3: scores in units of the local 255 x 255 sigma,
candidates above a threshold, one detection per group of touching
candidates) against the FP64 oracle on the same snr_max / argmax maps.

z is FP64 on both sides with sums in different orders: |dz| <= 1e-9 max(1,
|z|).  The candidate decision z > threshold is compared exactly away from
the threshold (|z - threshold| > 1e-9 max(1, |z|) on the oracle side);
detections, pixel counts, peaks and trajectories are integer results and
compared exactly for every component with no pixel in that band; the order
(z rounded to FP32 descending, flat index ascending) is checked on the GPU
list and against the oracle's where the FP32 keys agree."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

Z_TOL = 1e-9


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    assert torch.cuda.is_available()
    m.load()
    return m


def _run(mf, s, a, window, threshold, subtract_mean=True, max_out=16384):
    smax = torch.from_numpy(s).cuda()
    amax = torch.from_numpy(a).cuda()
    z = torch.empty(s.shape, dtype=torch.float32, device="cuda")
    raw, n = mf.detect(smax, amax, window=window, threshold=threshold, subtract_mean=subtract_mean,
                       max_out=max_out, z_out=z)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    found, written = (int(v) for v in n.cpu().tolist())
    det = mf.decode_detections(raw, written)
    return z.cpu().numpy(), det.copy(), found, written


def _compare(mf, oracle, s, a, window, threshold, subtract_mean=True, max_out=16384):
    z_g, det_g, found, written = _run(mf, s, a, window, threshold, subtract_mean, max_out)
    det_o, z_o, flag_o = oracle.detections(s, a, window=window, threshold=threshold, subtract_mean=subtract_mean)
    H, W = s.shape
    # z map: FP32 copy of the FP64 z
    err = np.abs(z_g.astype(np.float64) - z_o) / np.maximum(1.0, np.abs(z_o))
    assert err.max() <= 6e-8 + Z_TOL, "z max rel err %.3g" % err.max()
    # components whose every pixel is decided away from the threshold
    band = np.abs(z_o - threshold) <= Z_TOL * np.maximum(1.0, np.abs(z_o))
    band &= a >= 0
    lab, count = oracle.components(flag_o)
    lab_band = set(np.unique(lab[band & flag_o]).tolist()) - {0}
    near = band & ~flag_o  # pixels the GPU may flag: they can join or make components
    if not near.any() and not lab_band:
        assert found == count
    assert written == min(found, max_out)
    # decided components: identical peak, k, npix and FP64 z / stats
    p_o = det_o["y"].astype(np.int64) * W + det_o["x"]
    p_g = det_g["y"].astype(np.int64) * W + det_g["x"]
    by_g = {int(p): d for p, d in zip(p_g, det_g)}
    near_dil = np.zeros_like(near)
    if near.any():
        from scipy import ndimage
        near_dil = ndimage.binary_dilation(near, structure=np.ones((3, 3), bool))
    checked = 0
    for p, d in zip(p_o, det_o):
        L = lab.ravel()[p]
        if L in lab_band or near_dil[lab == L].any():
            continue
        if int(p) not in by_g:
            assert written < found, "detection at %d missing" % p
            continue
        g = by_g[int(p)]
        assert (g["k"], g["npix"]) == (d["k"], d["npix"]), (p, g, d)
        assert abs(g["z"] - d["z"]) <= Z_TOL * max(1.0, abs(d["z"]))
        assert abs(g["mean"] - d["mean"]) <= 1e-12 * max(1.0, abs(d["mean"]))
        assert abs(g["sigma"] - d["sigma"]) <= 1e-9 * max(1.0, abs(d["sigma"]))
        assert g["snr"] == np.float32(d["snr"])
        checked += 1
    # order on the GPU list: FP32 z descending, flat index ascending
    k32 = det_g["z"].astype(np.float32)
    assert np.all((k32[:-1] > k32[1:]) | ((k32[:-1] == k32[1:]) & (p_g[:-1] < p_g[1:])))
    # the GPU list is the oracle's prefix wherever the keys agree
    if not near.any() and not lab_band and written == len(det_o[:max_out]):
        same = det_o["z"][:written].astype(np.float32) == k32
        if same.all():
            assert np.array_equal(p_g, p_o[:written])
    return checked, found


@pytest.mark.parametrize("H,W,window,threshold,subtract_mean", [
    (200, 300, 255, 3.0, True),
    (257, 1100, 63, 3.0, True),      # two row tiles, ragged tail
    (64, 2100, 255, 2.0, True),      # three row tiles, window wider than the image height
    (300, 257, 31, 3.0, False),      # literal z = s / sigma
    (33, 45, 3, 1.0, True),
    (90, 70, 1, 0.0, True),          # one pixel per window: z = 0 everywhere, nothing found
])
def test_detect_matches_oracle(mf, oracle, H, W, window, threshold, subtract_mean):
    from paper_2209_09848_gb300 import synth
    s, a = synth.score_map(H, W, seed=H * 7 + W, K=40)
    if not subtract_mean:
        threshold = 7.0  # s / sigma of a score map around 2.5 with sigma ~0.45
    checked, found = _compare(mf, oracle, s, a, window, threshold, subtract_mean)
    if window > 1:
        assert found > 0 and checked > 0
    else:
        assert found == 0


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (41, 1), (2, 2)])
def test_detect_degenerate_shapes(mf, oracle, H, W):
    g = np.random.default_rng(H * 100 + W)
    s = g.normal(2.5, 0.5, size=(H, W)).astype(np.float32)
    a = np.zeros((H, W), dtype=np.int32)
    _compare(mf, oracle, s, a, 255, 0.5)


def test_detect_empty_and_constant(mf, oracle):
    H, W = 50, 60
    s = np.full((H, W), 2.5, np.float32)
    a = np.zeros((H, W), np.int32)
    z, det, found, written = _run(mf, s, a, 255, 3.0)
    assert found == written == 0 and (z == 0).all()
    a[:] = -1
    z, det, found, written = _run(mf, np.random.default_rng(0).normal(size=(H, W)).astype(np.float32), a, 255, -5.0)
    assert found == written == 0 and (z == 0).all()


def test_detect_one_large_component(mf, oracle):
    # every valid pixel with sigma > 0 is a candidate: the union-find joins
    # the whole image (minus masked holes) into few components
    from paper_2209_09848_gb300 import synth
    s, a = synth.score_map(400, 500, seed=9, K=10)
    checked, found = _compare(mf, oracle, s, a, 63, -1e6)
    assert found >= 1 and checked >= 1


def test_detect_checkerboard_is_one_component(mf):
    # candidates touching only at corners are one detection (8 neighbours)
    H, W = 64, 64
    yy, xx = np.mgrid[0:H, 0:W]
    s = np.where((yy + xx) % 2 == 0, 10.0, 0.0).astype(np.float32)
    s[0, 0] = 11.0
    a = np.zeros((H, W), np.int32)
    z, det, found, written = _run(mf, s, a, 255, 0.5)
    assert found == 1 and written == 1
    assert (det[0]["y"], det[0]["x"], det[0]["npix"]) == (0, 0, H * W // 2)


def test_detect_max_out_and_counts_only(mf, oracle):
    from paper_2209_09848_gb300 import synth
    s, a = synth.score_map(256, 256, seed=4, K=20)
    z, det_all, found, written = _run(mf, s, a, 255, 3.0)
    assert written == found > 10
    z2, det5, found5, written5 = _run(mf, s, a, 255, 3.0, max_out=5)
    assert found5 == found and written5 == 5
    assert np.array_equal(det5, det_all[:5])
    z3, det0, found0, written0 = _run(mf, s, a, 255, 3.0, max_out=0)
    assert found0 == found and written0 == 0
    np.testing.assert_array_equal(z, z3)


def test_detect_is_deterministic(mf):
    from paper_2209_09848_gb300 import synth
    s, a = synth.score_map(512, 700, seed=11, K=30)
    r1 = _run(mf, s, a, 255, 2.5)
    r2 = _run(mf, s, a, 255, 2.5)
    np.testing.assert_array_equal(r1[0], r2[0])
    assert r1[2:] == r2[2:]
    assert r1[1].tobytes() == r2[1].tobytes()


def test_detect_rejects_bad_arguments(mf):
    s = torch.zeros((16, 16), device="cuda")
    a = torch.zeros((16, 16), dtype=torch.int32, device="cuda")
    for kw in (dict(window=4), dict(window=0), dict(window=2049), dict(threshold=float("nan")),
               dict(max_out=-1)):
        with pytest.raises(mf.MFError):
            mf.detect(s, a, **kw)
    with pytest.raises(mf.MFError):
        mf.detect(s, a, max_out=16385)


def test_detect_full_size_paper_shaped(mf, oracle):
    # 2048 x 2048, window 255, 3 sigma: every detection against the oracle
    from paper_2209_09848_gb300 import synth
    s, a = synth.score_map(2048, 2048, seed=3, K=100)
    checked, found = _compare(mf, oracle, s, a, 255, 3.0)
    assert found > 1000 and checked > 0.95 * found
