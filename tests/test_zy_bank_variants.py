"""Filter-bank variants on the GPU: the phase-quantised bank (footprints at
phases rounded to multiples of 1/Q) searched exactly against the FP64
oracle's search over its own quantised table (same bar as the linear
search: |delta SNR| <= 1e-5 max(1, |SNR|), identical argmax where the two
best filters differ by more than 1e-3), and the host-only plan of a
frame-model bank against the layout of the table created on the device.
Collected after the other GPU files but before the static-scratch search,
so that a run stopping at its first failure has run the core parity tests."""
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


def _run(mf, res, sigma, mask, table):
    r = torch.from_numpy(res).cuda()
    s = torch.from_numpy(sigma).cuda()
    m = None if mask is None else torch.from_numpy(mask).cuda()
    smax, amax, sall = mf.search(r, s, table, mask=m, want_all=True)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    return smax.cpu().numpy(), amax.cpu().numpy(), sall.cpu().numpy()


def _frames(T, seed, gap=0, jit=0.3, frac=False):
    g = np.random.default_rng(seed)
    tau = np.arange(T, dtype=np.float64)
    if gap:
        tau[T // 2:] += gap
    if frac:
        tau += g.uniform(-0.2, 0.2, T)
    return tau, g.uniform(-jit, jit, size=(T, 2))


@pytest.mark.parametrize("Q,layout", [(4, {}), (2, {"kernel": 1}), (8, {"kernel": 2, "tile_w": 64, "segments": 2})])
def test_phase_quantised_bank_matches_oracle(mf, oracle, Q, layout):
    """The phase-quantised filter bank (footprints at phases rounded to
    multiples of 1/Q) searched exactly: the table equals the oracle's
    quantised table and the maps match the oracle's search over it."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 20, 70, 90
    c = synth.small_case(T, H, W, 17 + Q, mask_frac=0.02, movers=2)
    vx, vy = synth.velocity_grid(4, 3, -0.45, 0.45)
    table = mf.prf_table_create(vx, vy, T, phase_steps=Q, **layout)
    if layout.get("kernel"):
        assert table.info()["kernel"] == layout["kernel"]
    sh, tp = oracle.trajectory_table_quantised(vx, vy, T, Q)
    sg, tg = table.export()
    assert np.array_equal(sg, sh)
    np.testing.assert_allclose(tg, tp, rtol=0, atol=1e-15)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="quantised Q=%d %s" % (Q, layout))


@pytest.mark.parametrize("Q,T,H,W,grid,vmax,layout", [
    (4, 24, 77, 101, (3, 8), 0.45, {}),                                   # 8 trajectories per v_x class
    (3, 20, 64, 70, (2, 12), 0.4, {"group": 12}),                         # odd Q, whole classes
    (2, 40, 96, 60, (4, 6), 0.3, {"tile_w": 64, "segments": 2}),          # 64 columns, time segments
    (5, 9, 33, 47, (1, 10), 0.6, {"group": 5, "tile_h": 32}),             # ragged tiles, fast movers
])
def test_phase_planes_match_oracle(mf, oracle, Q, T, H, W, grid, vmax, layout):
    """The precompute-then-gather numerator (kernel 3): per frame one column
    pass per rounded y-phase over the window, then one add per (trajectory,
    pixel).  Its maps match the oracle's search over the quantised table and
    the oracle's own precompute-then-gather order, for odd and even Q, with
    masks and borders (start pixels whose trajectories leave the frame)."""
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, 29 + Q, mask_frac=0.03, movers=2)
    vx, vy = synth.velocity_grid(*grid, -vmax, vmax)
    table = mf.prf_table_create(vx, vy, T, phase_steps=Q, kernel=3, **layout)
    info = table.info()
    assert info["kernel"] == 2 and info["phase_planes"] == min(info["warps_per_group"], Q + 1)
    sh, tp = oracle.trajectory_table_quantised(vx, vy, T, Q)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    Ng, Dg = oracle.search_quantised_gather(c["res"], lam, vx, vy, Q)
    np.testing.assert_allclose(Ng, N, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Dg, D, rtol=1e-10, atol=1e-12)
    smax, amax, sall = _run(mf, c["res"], c["sigma"], c["mask"], table)
    check_search(smax, amax, sall, N, D, oracle, label="phase planes Q=%d %s" % (Q, layout))
    # and the column-pass numerator on the same bank
    smax2, amax2, sall2 = _run(mf, c["res"], c["sigma"], c["mask"],
                               mf.prf_table_create(vx, vy, T, phase_steps=Q, kernel=2, **layout))
    check_search(smax2, amax2, sall2, N, D, oracle, label="column passes Q=%d" % Q)


def test_phase_planes_reject_exact_banks_and_batches(mf):
    T = 8
    with pytest.raises(mf.MFError) as e:
        mf.prf_table_create([0.1, 0.2], [0.0, 0.1], T, kernel=3)  # phase_steps = 0
    assert e.value.status == 1
    table = mf.prf_table_create([0.1, 0.2], [0.0, 0.1], T, phase_steps=4, kernel=3)
    b = mf.Batch()
    with pytest.raises(mf.MFError) as e:
        b.add(torch.zeros((T, 16, 16), device="cuda"), torch.ones((16, 16), device="cuda"), table)
    assert e.value.status == 5
    b.destroy()


def test_host_plan_equals_created_table(mf):
    # mf_prf_plan_frames (host only) describes the layout that
    # mf_prf_table_create_frames builds on the device
    from paper_2209_09848_gb300 import synth
    T = 60
    vx, vy = synth.velocity_grid(4, 3, -0.3, 0.3)
    tau, jitter = _frames(T, 5, gap=90, jit=0.6, frac=True)
    for kw in ({}, {"times": tau, "jitter": jitter}, {"times": tau, "jitter": jitter, "kernel": 1}):
        assert mf.prf_plan(vx, vy, T, **kw) == mf.prf_table_create(vx, vy, T, **kw).info()
