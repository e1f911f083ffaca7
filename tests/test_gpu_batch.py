"""Batched searches (one CUDA graph, persistent numerator): every search in a
batch of uneven cutouts gives exactly the maps mf_search gives for it alone
(same per-tile code and summation order), on the first run and on graph
replays; one search is also checked against the FP64 oracle."""
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


def _items(mf):
    from paper_2209_09848_gb300 import synth
    # T, H, W, grid, vmax, dtype, mask, layout (None: planner; shape: general
    # kernel; factored layouts of different warp counts share one launch)
    specs = [
        (24, 96, 130, (3, 3), 0.3, torch.float32, 0.02, None),
        (9, 64, 64, (2, 2), 0.5, torch.bfloat16, 0.0, None),
        (31, 150, 90, (4, 2), 0.2, torch.float32, 0.01, dict(shape=0)),
        (16, 70, 200, (5, 3), 0.25, torch.float16, 0.02, dict(shape=3)),
        (5, 33, 47, (1, 1), 0.1, torch.float32, 0.0, None),
        (40, 128, 128, (3, 4), 0.15, torch.float32, 0.01, dict(shape=1)),
        (20, 77, 140, (2, 5), 0.4, torch.float32, 0.01, dict(kernel=2, group=5, tile_h=64, tile_w=32)),
        (12, 100, 61, (3, 3), 0.3, torch.float32, 0.0, dict(kernel=2, group=1, tile_h=32, tile_w=32)),
        (18, 90, 150, (2, 3), 0.3, torch.float32, 0.02, dict(kernel=2, group=3, tile_w=64)),
        (22, 140, 70, (3, 4), 0.3, torch.bfloat16, 0.01, dict(kernel=2, group=10, tile_h=64)),  # 20 warps
    ]
    out = []
    for i, (T, H, W, (nx, ny), vm, dt, mfrac, layout) in enumerate(specs):
        c = synth.small_case(T, H, W, 200 + i, mask_frac=mfrac, movers=2)
        vx, vy = synth.velocity_grid(nx, ny, -vm, vm)
        table = mf.prf_table_create(vx, vy, T, **(layout or {}))
        scale = None
        if dt == torch.float16:
            scale = (np.abs(c["res"]).max(axis=(1, 2)) / 2.0 ** 14).astype(np.float32)
            data = torch.from_numpy(c["res"] / scale[:, None, None]).to(dt).cuda()
            scale = torch.from_numpy(scale).cuda()
        else:
            data = torch.from_numpy(c["res"]).to(dt).cuda()
        s = torch.from_numpy(c["sigma"]).cuda()
        m = None if c["mask"] is None else torch.from_numpy(c["mask"]).cuda()
        out.append(dict(c=c, vx=vx, vy=vy, table=table, data=data, sigma=s, mask=m, scale=scale))
    return out


def test_batch_equals_individual_searches(mf, oracle):
    items = _items(mf)
    b = mf.Batch()
    for it in items:
        b.add(it["data"], it["sigma"], it["table"], mask=it["mask"], frame_scale=it["scale"], want_all=True)
    b.prepare()
    info = b.info()
    assert info["items"] == len(items) and info["shape_groups"] >= 4 and not info["graph_ready"]
    assert {it["table"].info()["kernel"] for it in items} == {1, 2}
    alone = [mf.search(it["data"], it["sigma"], it["table"], mask=it["mask"], frame_scale=it["scale"],
                       want_all=True) for it in items]
    torch.cuda.synchronize()
    for run in range(3):
        for o in b.outputs:  # scribble over the outputs: every replay must rewrite them
            o[0].fill_(-7.0)
            o[1].fill_(-7)
            o[2].fill_(-7.0)
        b.run()
        for _ in range(200000):  # poll until the device is done (never blocks)
            if b.poll():
                break
        assert b.poll()
        torch.cuda.synchronize()
        assert mf.device_status() == 0
        assert b.info()["graph_ready"]
        for (gm, ga, gall), (am, aa, aall) in zip(b.outputs, alone):
            assert torch.equal(gm, am) and torch.equal(ga, aa) and torch.equal(gall, aall)
    # and one of them against the FP64 oracle
    it = items[0]
    sh, tp = oracle.trajectory_table(it["vx"], it["vy"], it["data"].shape[0])
    lam = oracle.inverse_variance(it["c"]["sigma"], it["c"]["mask"])
    N, D = oracle.search_full(it["c"]["res"], lam, sh, tp)
    gm, ga, gall = b.outputs[0]
    check_search(gm.cpu().numpy(), ga.cpu().numpy(), gall.cpu().numpy(), N, D, oracle, label="batch item 0")
    # and the bf16 item (factored numerator on the 16-bit weighted stack)
    it = items[1]
    assert it["table"].info()["kernel"] == 2
    sh, tp = oracle.trajectory_table(it["vx"], it["vy"], it["data"].shape[0])
    lam = oracle.inverse_variance(it["c"]["sigma"], it["c"]["mask"])
    q, beta = oracle.weighted_stack16(it["data"].float().cpu().numpy(), it["c"]["sigma"], it["c"]["mask"], None,
                                      "bf16")
    N, D = oracle.search_weighted(q, beta, lam, sh, tp)
    gm, ga, gall = b.outputs[1]
    check_search(gm.cpu().numpy(), ga.cpu().numpy(), gall.cpu().numpy(), N, D, oracle, label="batch item 1 (bf16)")
    # and the 20-warp bf16 item (whole v_x classes on 64-row tiles)
    it = items[-1]
    inf = it["table"].info()
    assert (inf["kernel"], inf["warps_per_group"], inf["tile_h"], inf["tile_w"]) == (2, 10, 64, 32)
    sh, tp = oracle.trajectory_table(it["vx"], it["vy"], it["data"].shape[0])
    lam = oracle.inverse_variance(it["c"]["sigma"], it["c"]["mask"])
    q, beta = oracle.weighted_stack16(it["data"].float().cpu().numpy(), it["c"]["sigma"], it["c"]["mask"], None,
                                      "bf16")
    N, D = oracle.search_weighted(q, beta, lam, sh, tp)
    gm, ga, gall = b.outputs[-1]
    check_search(gm.cpu().numpy(), ga.cpu().numpy(), gall.cpu().numpy(), N, D, oracle, label="batch item (20 warps)")
    b.destroy()


def test_batch_argument_errors(mf):
    b = mf.Batch()
    assert b.poll()  # nothing launched yet
    with pytest.raises(mf.MFError):
        b.run()  # not prepared
    with pytest.raises(mf.MFError):
        b.prepare()  # no items
    T = 4
    table = mf.prf_table_create([0.1], [0.0], T)
    r = torch.zeros((T + 1, 8, 8), device="cuda")
    with pytest.raises(mf.MFError):
        b.add(r, torch.ones((8, 8), device="cuda"), table)  # T mismatch
    b.destroy()


def test_batch_splits_launches_past_the_parameter_limit(mf):
    # a persistent launch carries at most 192 searches in its parameters: 200
    # searches of one layout take two launches of one time segment, and every
    # output equals the search on its own
    from paper_2209_09848_gb300 import synth
    T, H, W = 10, 24, 40
    vx, vy = synth.velocity_grid(2, 2, -0.2, 0.2)
    table = mf.prf_table_create(vx, vy, T, kernel=2)
    assert table.info()["time_segments"] == 1
    b = mf.Batch()
    ins = []
    for i in range(200):
        c = synth.small_case(T, H, W, 500 + i, movers=1)
        r = torch.from_numpy(c["res"]).cuda()
        s = torch.from_numpy(c["sigma"]).cuda()
        ins.append((r, s))
        b.add(r, s, table)
    b.prepare()
    b.run()
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    for (r, s), (gm, ga, _) in zip(ins, b.outputs):
        am, aa, _ = mf.search(r, s, table)
        torch.cuda.synchronize()
        assert torch.equal(gm, am) and torch.equal(ga, aa)
    b.destroy()


def test_autotuner_picks_a_timed_layout(mf, oracle):
    """The autotuner times the factored and general layouts, caches the
    winner per bucket, and the tuned table searches correctly."""
    from paper_2209_09848_gb300 import autotune, synth
    autotune.clear_cache()
    T, H, W = 20, 120, 140
    vx, vy = synth.velocity_grid(3, 4, -0.3, 0.3)
    opts, timings = autotune.tune(vx, vy, T, H, W, crop=128)
    assert timings and opts in autotune.CANDIDATES
    assert {autotune.CANDIDATES[i]["kernel"] for i in timings} == {1, 2}
    assert autotune.tune(vx, vy, T, H, W, crop=128)[0] is not None  # cached
    table = autotune.tuned_table(vx, vy, T, H, W, crop=128)
    c = synth.small_case(T, H, W, 31, mask_frac=0.01, movers=2)
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    smax, amax, sall = mf.search(torch.from_numpy(c["res"]).cuda(), torch.from_numpy(c["sigma"]).cuda(), table,
                                 mask=torch.from_numpy(c["mask"]).cuda(), want_all=True)
    torch.cuda.synchronize()
    check_search(smax.cpu().numpy(), amax.cpu().numpy(), sall.cpu().numpy(), N, D, oracle, label="tuned")
