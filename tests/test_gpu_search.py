"""Parity of mf_search (CUDA, through the C ABI) with the FP64 oracle.

Element-by-element on seeded inputs at sizes the oracle finishes in seconds,
spanning several tiles and ragged tails; the bar is |delta SNR| <= 1e-5 *
max(1, |SNR|) and identical argmax wherever the two best filters differ by
more than 1e-3."""
import numpy as np
import pytest

from _util import check_search

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    m.load()
    return m


def _run(mf, res, sigma, mask, table, want_all=True, frame_scale=None, dtype=torch.float32):
    dev = "cuda"
    r = torch.from_numpy(res).to(dev).to(dtype)
    s = torch.from_numpy(sigma).to(dev)
    m = None if mask is None else torch.from_numpy(mask).to(dev)
    fs = None if frame_scale is None else torch.as_tensor(frame_scale, dtype=torch.float32, device=dev)
    smax, amax, sall = mf.search(r, s, table, mask=m, frame_scale=fs, want_all=want_all)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    return smax.cpu().numpy(), amax.cpu().numpy(), None if sall is None else sall.cpu().numpy()


def test_small_config_full_cube(mf, oracle):
    from paper_2209_09848_gb300 import synth
    c = synth.small_config(0)
    table = mf.prf_table_create(c["vx"], c["vy"], 32)
    sh, tp = table.export()
    sh_o, tp_o = oracle.trajectory_table(c["vx"], c["vy"], 32)
    assert np.array_equal(sh, sh_o)
    np.testing.assert_allclose(tp, tp_o, rtol=0, atol=1e-15)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh_o, tp_o)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="small config")


CASES = [
    # T, H, W, K, seed, mask_frac, max speed, custom
    (1, 37, 45, 1, 1, 0.0, 0.5, False),
    (2, 64, 96, 7, 2, 0.02, 0.6, False),
    (33, 50, 70, 16, 3, 0.01, 0.3, False),
    (5, 100, 33, 9, 4, 0.05, 1.2, False),
    (17, 41, 77, 11, 5, 0.02, 0.0, True),
    (40, 70, 130, 24, 6, 0.01, 0.15, False),
]


@pytest.mark.parametrize("T,H,W,K,seed,mask_frac,vmax,custom", CASES)
def test_random_shapes(mf, oracle, T, H, W, K, seed, mask_frac, vmax, custom):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, seed, mask_frac=mask_frac, movers=2)
    g = np.random.default_rng(100 + seed)
    if custom:
        sh = g.integers(-6, 7, size=(K, T, 2)).astype(np.int32)
        tp = g.uniform(-0.2, 1.0, size=(K, T, 5, 5))  # arbitrary footprints
        table = mf.prf_table_create_custom(sh, tp)
    else:
        vx = g.uniform(-vmax, vmax, K)
        vy = g.uniform(-vmax, vmax, K)
        table = mf.prf_table_create(vx, vy, T)
        sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="case %s" % ((T, H, W, K),))


@pytest.mark.parametrize("T,H,W,grid,vmax,layout", [
    (12, 48, 80, (3, 3), 0.3, {}),
    (41, 203, 157, (5, 7), 0.45, {}),                                         # several tiles, ragged edges
    (23, 70, 130, (4, 2), 0.3, dict(kernel=2, group=2, tile_w=64)),           # 64-column tiles
    (40, 96, 100, (3, 3), 0.6, dict(kernel=2, segments=3)),                   # time segments
])
def test_frame_scale_and_half_precision_storage(mf, oracle, T, H, W, grid, vmax, layout):
    # bf16 / fp16 stacks: the factored numerator reads the weighted stack in
    # the stack's own 16-bit type (the precision form); the oracle forms that
    # stack from its definition and the matched filter on it
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, 7, mask_frac=0.01, movers=2)
    vx, vy = synth.velocity_grid(*grid, -vmax, vmax)
    table = mf.prf_table_create(vx, vy, T, **layout)
    assert table.info()["kernel"] == 2
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    for dt, name in ((torch.bfloat16, "bf16"), (torch.float16, "fp16")):
        # fp16: max|r_t| / 2^14, negative on every third frame (the stored
        # values flip with it); bf16: any positive scale
        scale = (np.abs(c["res"]).max(axis=(1, 2)) / 2.0 ** 14 * np.where(np.arange(T) % 3 == 0, -1, 1)).astype(
            np.float32) if dt == torch.float16 else np.exp(np.random.default_rng(T).uniform(-1, 1, T)).astype(np.float32)
        q = torch.from_numpy(c["res"] / scale[:, None, None]).to(dt)
        deq = q.float().numpy()  # the stored values
        y16, beta = oracle.weighted_stack16(deq, c["sigma"], c["mask"], scale, name)
        N, D = oracle.search_weighted(y16, beta, lam, sh, tp)
        smax, amax, sall = _run(mf, deq, c["sigma"], c["mask"], table, frame_scale=scale, dtype=dt)
        check_search(smax, amax, sall, N, D, oracle, label="%s %s" % (name, (T, H, W)))


def test_half_precision_storage_general_kernel(mf, oracle):
    # the general numerator keeps an FP32 weighted stack: it matches the
    # oracle on the stored values exactly as the FP32 path does
    from paper_2209_09848_gb300 import synth
    T, H, W = 12, 48, 80
    c = synth.small_case(T, H, W, 7, mask_frac=0.01, movers=2)
    vx, vy = synth.velocity_grid(3, 3, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T, kernel=1)
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    for dt in (torch.bfloat16, torch.float16):
        scale = (np.abs(c["res"]).max(axis=(1, 2)) / 2.0 ** 14).astype(np.float32) if dt == torch.float16 \
            else np.ones(T, np.float32)
        q = torch.from_numpy(c["res"] / scale[:, None, None]).to(dt)
        deq = q.float().numpy()
        N, D = oracle.search_full(deq, lam, sh, tp, frame_scale=scale.astype(np.float64))
        smax, amax, sall = _run(mf, deq, c["sigma"], c["mask"], table, frame_scale=scale, dtype=dt)
        check_search(smax, amax, sall, N, D, oracle, label=str(dt))


def test_half_precision_shift_stack(mf, oracle):
    # single-tap footprints read the 16-bit stage directly (no row pass)
    from paper_2209_09848_gb300 import synth
    T, H, W = 30, 77, 101
    c = synth.small_case(T, H, W, 19, mask_frac=0.02, movers=2)
    vx, vy = synth.velocity_grid(4, 3, -0.4, 0.4)
    table = mf.prf_table_create(vx, vy, T, kind=2)
    assert table.info()["taps"] == 1
    sh, tp = oracle.trajectory_table(vx, vy, T, kind=2)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    for dt, name in ((torch.bfloat16, "bf16"), (torch.float16, "fp16")):
        scale = (np.abs(c["res"]).max(axis=(1, 2)) / 2.0 ** 12).astype(np.float32)
        q = torch.from_numpy(c["res"] / scale[:, None, None]).to(dt)
        deq = q.float().numpy()
        y16, beta = oracle.weighted_stack16(deq, c["sigma"], c["mask"], scale, name)
        N, D = oracle.search_weighted(y16, beta, lam, sh, tp)
        smax, amax, sall = _run(mf, deq, c["sigma"], c["mask"], table, frame_scale=scale, dtype=dt)
        check_search(smax, amax, sall, N, D, oracle, label="shift-stack " + name)


def test_velocity_zero_and_single_pixel_frames(mf, oracle):
    from paper_2209_09848_gb300 import synth
    for (T, H, W) in [(3, 1, 1), (4, 1, 40), (2, 33, 1), (1, 5, 5)]:
        c = synth.small_case(T, H, W, 9)
        vx = np.array([0.0, 0.4, -0.7])
        vy = np.array([0.0, -0.2, 0.9])
        table = mf.prf_table_create(vx, vy, T)
        sh, tp = oracle.trajectory_table(vx, vy, T)
        lam = oracle.inverse_variance(c["sigma"], None)
        N, D = oracle.search_full(c["res"], lam, sh, tp)
        smax, amax, sall = _run(mf, c["res"], c["sigma"], None, table)
        check_search(smax, amax, sall, N, D, oracle, label="tiny %s" % ((T, H, W),))


def test_fully_masked_gives_minus_one(mf):
    T, H, W = 4, 20, 20
    res = np.random.default_rng(0).standard_normal((T, H, W)).astype(np.float32)
    sigma = np.ones((H, W), np.float32)
    mask = np.ones((H, W), np.uint8)
    table = mf.prf_table_create([0.1, -0.1], [0.0, 0.2], T)
    smax, amax, sall = _run(mf, res, sigma, mask, table)
    assert np.all(amax == -1) and np.all(smax == 0) and np.all(sall == 0)


def test_unusable_sigma_is_masked(mf, oracle):
    # sigma of 0, -1, NaN, +-inf at unmasked pixels: excluded like masked
    # pixels on both sides (the oracle's rule is pinned without a GPU)
    from paper_2209_09848_gb300 import synth
    T, H, W = 14, 57, 83
    c = synth.small_case(T, H, W, 13, mask_frac=0.02, movers=2)
    sigma = c["sigma"].copy()
    g = np.random.default_rng(77)
    flat = g.choice(H * W, size=60, replace=False)
    vals = np.array([0.0, -1.0, np.nan, np.inf, -np.inf, -0.0], np.float32)
    sigma.reshape(-1)[flat] = vals[np.arange(flat.size) % vals.size]
    vx, vy = synth.velocity_grid(3, 4, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T)
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(sigma, c["mask"])
    assert np.all(np.isfinite(lam))
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], sigma, c["mask"], table)
    assert np.all(np.isfinite(smax)) and np.all(np.isfinite(sall))
    check_search(smax, amax, sall, N, D, oracle, label="unusable sigma")
    # and with the general kernel
    table_g = mf.prf_table_create(vx, vy, T, kernel=1)
    smax, amax, sall = _run(mf, c["res"], sigma, c["mask"], table_g)
    check_search(smax, amax, sall, N, D, oracle, label="unusable sigma, general kernel")
    # the FP64 re-score applies the same rule
    dev = "cuda"
    raw, n = mf.rescore_topk(torch.from_numpy(c["res"]).to(dev), torch.from_numpy(sigma).to(dev), table,
                             torch.from_numpy(smax).to(dev), torch.from_numpy(amax).to(dev), 200,
                             mask=torch.from_numpy(c["mask"]).to(dev))
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    cands = mf.decode_candidates(raw, int(n.item()))
    Nc, Dc = oracle.search_points(c["res"], lam, sh, tp, cands["y"].astype(np.int32), cands["x"].astype(np.int32),
                                  cands["k"].astype(np.int32))
    ok = Dc > 0
    np.testing.assert_allclose(cands["snr"][ok], Nc[ok] / np.sqrt(Dc[ok]), rtol=1e-9, atol=1e-12)


def test_denominator_staged_and_unstaged(mf, oracle):
    # the paper's slow movers: each CTA stages the lambda box its trajectory
    # reaches in shared memory, in tiles of 32, 16 or 8 rows as the box
    # allows; movers so fast that the box cannot fit go through the unstaged
    # denominator -- all match the oracle, for widths with a ragged last
    # 256-column tile that are (292: 16-byte row stores) and are not (290) a
    # multiple of four
    from paper_2209_09848_gb300 import synth
    T = 30
    for H, W in ((70, 290), (45, 292)):
        c = synth.small_case(T, H, W, 23, mask_frac=0.03, movers=2)
        lam = oracle.inverse_variance(c["sigma"], c["mask"])
        for vx, vy, th in (([0.3, -0.2, 0.1, 0.0], [0.1, 0.25, -0.3, 0.05], 32),
                           ([0.3, 0.0], [0.1, 6.0], 16),
                           ([0.3, 0.0], [0.1, -6.3], 8),
                           ([8.0, -7.0, 0.3], [8.0, 6.0, -0.2], 0)):
            table = mf.prf_table_create(vx, vy, T)
            assert table.info()["den_tile_h"] == th
            sh, tp = oracle.trajectory_table(vx, vy, T)
            N, D = oracle.search_full(c["res"], lam, sh, tp)
            smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
            check_search(smax, amax, sall, N, D, oracle, label="denominator tile %d, %d x %d" % (th, H, W))


def test_empty_frame_is_a_no_op(mf):
    table = mf.prf_table_create([0.1], [0.0], 3)
    r = torch.zeros((3, 0, 7), device="cuda")
    s = torch.ones((0, 7), device="cuda")
    smax, amax, _ = mf.search(r, s, table)
    torch.cuda.synchronize()
    assert smax.numel() == 0 and amax.numel() == 0


def test_invalid_arguments_enqueue_nothing(mf):
    T, H, W = 4, 16, 16
    table = mf.prf_table_create([0.1], [0.0], T)
    r = torch.zeros((T + 1, H, W), device="cuda")
    s = torch.ones((H, W), device="cuda")
    with pytest.raises(mf.MFError) as e:
        mf.search(r, s, table)
    assert e.value.status == 1 and "T=" in str(e.value)
    r = torch.zeros((T, H, W), device="cuda")
    with pytest.raises(mf.MFError):
        mf.search(r, s, table, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(mf.MFError):
        mf.prf_table_create([float("nan")], [0.0], T)
    with pytest.raises(mf.MFError):
        mf.prf_table_create([0.1], [0.0], T, sigma_px=-1.0)
    with pytest.raises(mf.MFError):
        mf.prf_table_create([0.1], [0.0], T, kind=7)


def test_deterministic_reruns(mf):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(20, 64, 64, 11, mask_frac=0.01, movers=3)
    vx, vy = synth.velocity_grid(4, 4, -0.2, 0.2)
    table = mf.prf_table_create(vx, vy, 20)
    a = _run(mf, c["res"], c["sigma"], c["mask"], table)
    b = _run(mf, c["res"], c["sigma"], c["mask"], table)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("lockstep", [0, 1])
@pytest.mark.parametrize("vec", [1, 2, 4])
@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_every_cta_shape(mf, oracle, shape, vec, lockstep):
    """Each numerator CTA layout (trajectories x sub-tiles) and shared-memory
    load width gives the oracle's answer, on a ragged frame that spans several
    tiles of every layout (odd velocities exercise every window alignment)."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 24, 150, 141
    c = synth.small_case(T, H, W, 40 + shape, mask_frac=0.02, movers=3)
    vx, vy = synth.velocity_grid(5, 4, -0.25, 0.25)
    vx = vx + 0.013 * np.arange(vx.size) / vx.size
    table = mf.prf_table_create(vx, vy, T, shape=shape, vec=vec, lockstep=lockstep)
    info = table.info()
    assert info["warps_per_group"] == [16, 8, 4, 2][shape] and info["vec"] == vec
    assert info["lockstep"] == lockstep
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="shape %d" % shape)


FACTORED = [
    # group, tile_h, tile_w, stages, segments (0 = planner's choice)
    (1, 0, 32, 0, 1),
    (1, 0, 64, 0, 2),
    (2, 0, 64, 2, 0),
    (3, 0, 32, 0, 3),
    (4, 128, 32, 4, 1),
    (5, 96, 32, 6, 5),
    (6, 64, 32, 5, 2),
    (8, 64, 32, 3, 4),
    (16, 32, 32, 2, 1),
    (2, 32, 64, 0, 3),
    (4, 64, 32, 3, 5),
    # 20 warps, the most a CTA has: whole classes on 64-row tiles (the paper
    # grid's layout), on 32 x 64 tiles, on 32-row tiles with empty slots, and
    # 5 trajectories on 128-row tiles
    (10, 64, 32, 0, 2),
    (10, 32, 64, 0, 0),
    (20, 32, 32, 2, 3),
    (5, 128, 32, 3, 0),
]


@pytest.mark.parametrize("group,tile_h,tile_w,stages,segments", FACTORED)
def test_factored_layouts(mf, oracle, group, tile_h, tile_w, stages, segments):
    """The factored numerator (row pass shared by the trajectories of one v_x,
    column pass per trajectory) gives the oracle's answer for every CTA
    geometry, stage count and number of time segments (segments of 8 to 40
    frames), on a ragged frame spanning several tiles, with more frames than a
    record chunk and a frame block, and a grid whose v_y spread makes the
    window rows differ from frame to frame."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 40, 203, 157
    c = synth.small_case(T, H, W, 60 + group, mask_frac=0.02, movers=3)
    gx = np.array([-0.61, -0.2, 0.05, 0.33, 0.9])
    gy = np.linspace(-0.8, 0.7, 7)
    vx = np.repeat(gx, gy.size)
    vy = np.tile(gy, gx.size)
    table = mf.prf_table_create(vx, vy, T, kernel=2, group=group, tile_h=tile_h or None, tile_w=tile_w,
                                stages=stages or None, segments=segments or None)
    info = table.info()
    if segments:
        assert info["time_segments"] == segments
    assert info["kernel"] == 2 and info["warps_per_group"] == group and info["tile_w"] == tile_w
    if tile_h:
        assert info["tile_h"] == tile_h
    if stages:
        assert info["stages"] == stages
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="factored %s" % ((group, tile_h, tile_w, stages),))


def test_factored_is_default_and_matches_general(mf):
    """Tables built from velocities use the factored numerator by default; the
    general kernel on the same table gives the same SNR up to FP32 rounding
    and the same argmax."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 30, 130, 170
    c = synth.small_case(T, H, W, 77, mask_frac=0.01, movers=4)
    vx, vy = synth.velocity_grid(6, 5, -0.3, 0.3)
    fac = mf.prf_table_create(vx, vy, T)
    gen = mf.prf_table_create(vx, vy, T, kernel=1)
    assert fac.info()["kernel"] == 2 and gen.info()["kernel"] == 1
    a = _run(mf, c["res"], c["sigma"], c["mask"], fac)
    b = _run(mf, c["res"], c["sigma"], c["mask"], gen)
    assert np.all(np.abs(a[0] - b[0]) <= 2e-5 * np.maximum(1, np.abs(b[0])))
    assert np.all(np.abs(a[2] - b[2]) <= 2e-5 * np.maximum(1, np.abs(b[2])))
    top2 = np.sort(b[2], axis=0)[-2:]
    clear = (top2[1] - top2[0]) > 1e-3
    assert np.array_equal(a[1][clear], b[1][clear])


def test_factored_needs_separable_table(mf):
    g = np.random.default_rng(5)
    sh = g.integers(-3, 4, size=(3, 4, 2)).astype(np.int32)
    tp = g.uniform(0, 1, size=(3, 4, 5, 5))
    t = mf.prf_table_create_custom(sh, tp)
    assert t.info()["kernel"] == 1
    with pytest.raises(mf.MFError):
        mf.prf_table_create(np.zeros(2), np.zeros(2), 4, kernel=2, group=21)


@pytest.mark.parametrize("layout", [{}, {"kernel": 1}, {"kernel": 2, "group": 3, "tile_w": 64},
                                    {"kernel": 2, "segments": 3}])
def test_shift_stack_matches_oracle(mf, oracle, layout):
    """The shift-stack filter (Section 3.2: one 1 per frame in the pixel
    holding the source): the factored numerator runs its single-tap passes,
    the general one its 25 taps with 24 zeros; both give the oracle's
    answer."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 36, 133, 150
    c = synth.small_case(T, H, W, 71, mask_frac=0.02, movers=3)
    vx, vy = synth.velocity_grid(5, 4, -0.45, 0.45)
    table = mf.prf_table_create(vx, vy, T, kind=2, **layout)
    info = table.info()
    if info["kernel"] == 2:
        assert info["taps"] == 1
    sh, tp = oracle.trajectory_table(vx, vy, T, kind=2)
    sg, tg = table.export()
    assert np.array_equal(sg, sh) and np.array_equal(tg, tp)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="shift-stack %s" % layout)


def test_shift_stack_single_tap_equals_batch(mf):
    """The batched launch runs the five-tap passes on the same single-tap
    table; zero taps add exact zeros, so the maps are bit-identical."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 24, 96, 112
    c = synth.small_case(T, H, W, 5, mask_frac=0.01, movers=2)
    vx, vy = synth.velocity_grid(4, 4, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T, kind=2)
    assert table.info()["taps"] == 1
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    smax, amax, _ = mf.search(r, s, table, mask=m)
    b = mf.Batch()
    b.add(r, s, table, mask=m)
    b.prepare()
    b.run()
    torch.cuda.synchronize()
    bmax, bamax, _ = b.outputs[0]
    assert torch.equal(smax, bmax) and torch.equal(amax, bamax)
    assert mf.prf_table_create(vx, vy, T).info()["taps"] == 5

