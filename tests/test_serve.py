"""Serving loop: admission never exceeds the memory budget, a request larger
than the whole budget fails alone without disturbing the others, and every
request's result is the same served alone and in an overlapping mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _requests(n, seed=0, sides=(256, 384, 512), frames=(60, 160)):
    """Requests big enough (a few ms of GPU work each) for overlap to show."""
    from paper_2209_09848_gb300 import synth
    from paper_2209_09848_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        side = int(rng.choice(sides))
        T = int(rng.integers(*frames))
        g = np.random.default_rng(1000 + i)
        sigma = np.exp(0.3 * g.standard_normal((side, side))).astype(np.float32)
        res = (sigma[None] * g.standard_normal((T, side, side), dtype=np.float32)).astype(np.float32)
        mask = synth.star_mask(side, side, g, 0.01)
        nx, ny = int(rng.integers(4, 8)), int(rng.integers(4, 8))
        vx, vy = synth.velocity_grid(nx, ny, -0.3, 0.3)
        reqs.append(Request(stack=torch.from_numpy(res).pin_memory(), sigma=torch.from_numpy(sigma).pin_memory(),
                            vx=vx, vy=vy, mask=torch.from_numpy(mask).pin_memory(), k_top=16, tag=i))
    return reqs


def test_alone_equals_mix_and_budget_holds():
    from paper_2209_09848_gb300.serve import Server
    import paper_2209_09848_gb300 as mf
    reqs = _requests(12)
    alone = []
    srv = Server(budget_bytes=1 << 34, streams=1, planners=1)
    for r in reqs:
        alone.append(srv.submit(r).result(timeout=120))
    srv.close()
    # a budget that holds only a few requests at once forces queueing
    budget = 3 * max(a.footprint for a in alone)
    srv = Server(budget_bytes=budget, streams=4, planners=4)
    futs = [srv.submit(r) for r in reqs]
    mix = [f.result(timeout=120) for f in futs]
    srv.close()
    assert srv.peak <= budget
    assert mf.device_status() == 0
    # device-side overlap: two requests' GPU work intervals intersect
    overlapped = sum(1 for i in range(len(mix)) for j in range(i + 1, len(mix))
                     if mix[i].gpu_start_ms < mix[j].gpu_end_ms and mix[j].gpu_start_ms < mix[i].gpu_end_ms)
    assert overlapped > 0, "no two requests were on the GPU at the same time"
    for a, m in zip(alone, mix):
        assert a.tag == m.tag
        assert np.array_equal(a.snr_max, m.snr_max) and np.array_equal(a.argmax, m.argmax)
        assert np.array_equal(a.candidates, m.candidates)


def test_oversized_request_fails_alone():
    from paper_2209_09848_gb300.serve import Server
    reqs = _requests(3, seed=5)
    srv = Server(budget_bytes=1 << 34, streams=2)
    fp = srv.submit(reqs[0]).result(timeout=120).footprint
    srv.close()
    srv = Server(budget_bytes=fp + 1024, streams=2)
    big = _requests(1, seed=9, sides=(128,), frames=(10, 11))[0]
    big.stack = torch.zeros((400, 512, 512)).pin_memory()
    big.sigma = torch.ones((512, 512)).pin_memory()
    big.mask = None
    futs = [srv.submit(reqs[0]), srv.submit(big), srv.submit(reqs[0])]
    assert futs[0].result(timeout=120).snr_max.shape == reqs[0].sigma.shape
    with pytest.raises(MemoryError):
        futs[1].result(timeout=120)
    assert futs[2].result(timeout=120).snr_max.shape == reqs[0].sigma.shape
    srv.close()
    assert srv.rejected == 1


def test_request_with_frame_model_and_shift_stack():
    # a request carrying frame times, jitter and the shift-stack kind is
    # searched with that filter bank: its result equals mf.search on a table
    # built the same way
    from paper_2209_09848_gb300.serve import Server
    import paper_2209_09848_gb300 as mf
    r = _requests(1, seed=3, sides=(192,), frames=(40, 41))[0]
    T = r.stack.shape[0]
    g = np.random.default_rng(4)
    r.times = np.arange(T, dtype=np.float64) + np.where(np.arange(T) >= T // 2, 30.0, 0.0)
    r.jitter = g.uniform(-0.2, 0.2, size=(T, 2))
    r.kind = 2
    srv = Server(budget_bytes=1 << 34, streams=2)
    res = srv.submit(r).result(timeout=120)
    srv.close()
    table = mf.prf_table_create(r.vx, r.vy, T, kind=2, times=r.times, jitter=r.jitter)
    smax, amax, _ = mf.search(r.stack.cuda(), r.sigma.cuda(), table, mask=r.mask.cuda())
    torch.cuda.synchronize()
    assert np.array_equal(res.snr_max, smax.cpu().numpy()) and np.array_equal(res.argmax, amax.cpu().numpy())
