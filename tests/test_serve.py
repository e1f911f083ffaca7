"""Serving loop: admission never exceeds the memory budget, a request larger
than the whole budget fails alone without disturbing the others, every
request's result is the same served alone and in an overlapping mix, served
results match the FP64 oracle, and a request whose search reports a device
wait that gave up fails alone."""
import numpy as np
import pytest

from _util import check_search

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
    # device-side overlap of kernels: two requests' kernel intervals (after
    # their uploads, before their downloads) intersect
    overlapped = sum(1 for i in range(len(mix)) for j in range(i + 1, len(mix))
                     if mix[i].kernel_start_ms < mix[j].kernel_end_ms and mix[j].kernel_start_ms < mix[i].kernel_end_ms)
    assert overlapped > 0, "no two requests' kernels were on the GPU at the same time"
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


def _oracle_requests(seed=21):
    """Mixed requests small enough for the FP64 oracle: float32, bf16 and
    scaled fp16 storage, uneven sizes and frame counts, linear and
    frame-model (gaps, jitter) filter banks, masks and candidates."""
    from paper_2209_09848_gb300 import synth
    from paper_2209_09848_gb300.serve import Request
    rng = np.random.default_rng(seed)
    specs = [(torch.float32, None), (torch.bfloat16, None), (torch.float16, "scale"), (torch.float32, "frames"),
             (torch.bfloat16, "frames"), (torch.float32, None), (torch.float16, "scale"), (torch.float32, "frames")]
    reqs, meta = [], []
    for i, (dt, extra) in enumerate(specs):
        H = int(rng.integers(40, 150))
        W = int(rng.integers(40, 150))
        T = int(rng.integers(12, 48))
        c = synth.small_case(T, H, W, 300 + i, mask_frac=0.02, movers=2)
        nx, ny = int(rng.integers(2, 5)), int(rng.integers(2, 5))
        vx, vy = synth.velocity_grid(nx, ny, -0.3, 0.3)
        scale = None
        res = c["res"]
        if extra == "scale":
            scale = (np.abs(res).max(axis=(1, 2)) / 2.0 ** 14).astype(np.float32)
            res = res / scale[:, None, None]
        q = torch.from_numpy(np.ascontiguousarray(res, np.float32)).to(dt)
        times = jitter = None
        if extra == "frames":
            g = np.random.default_rng(400 + i)
            times = np.arange(T, dtype=np.float64) + np.where(np.arange(T) >= T // 2, 17.5, 0.0)
            jitter = g.uniform(-0.4, 0.4, size=(T, 2))
        reqs.append(Request(stack=q.pin_memory(), sigma=torch.from_numpy(c["sigma"]).pin_memory(), vx=vx, vy=vy,
                            mask=torch.from_numpy(c["mask"]).pin_memory(),
                            frame_scale=None if scale is None else torch.from_numpy(scale).pin_memory(),
                            k_top=24, tag=i, times=times, jitter=jitter))
        meta.append(dict(deq=q.float().numpy(), sigma=c["sigma"], mask=c["mask"], vx=vx, vy=vy, T=T, times=times,
                         jitter=jitter, scale=scale, dtype=dt))
    return reqs, meta


def _oracle_maps(oracle, m):
    if m["times"] is not None:
        sh, tp = oracle.trajectory_table_frames(m["vx"], m["vy"], m["T"], times=m["times"], jitter=m["jitter"])
    else:
        sh, tp = oracle.trajectory_table(m["vx"], m["vy"], m["T"])
    lam = oracle.inverse_variance(m["sigma"], m["mask"])
    fs = None if m["scale"] is None else m["scale"].astype(np.float64)
    return sh, tp, lam, fs


def _oracle_search(oracle, m, sh, tp, lam, fs):
    # 16-bit requests are searched in the precision form (the weighted stack
    # in 16 bits); float32 ones with the plain definition
    if m["dtype"] == torch.float32:
        return oracle.search_full(m["deq"], lam, sh, tp, frame_scale=fs)
    name = "bf16" if m["dtype"] == torch.bfloat16 else "fp16"
    q, beta = oracle.weighted_stack16(m["deq"], m["sigma"], m["mask"], m["scale"], name)
    return oracle.search_weighted(q, beta, lam, sh, tp)


def test_served_results_match_the_oracle(oracle):
    # requests submitted at once through the server, overlapping on four
    # streams; every served map and candidate list is checked against the
    # FP64 oracle, not the library
    from paper_2209_09848_gb300.serve import Server
    import paper_2209_09848_gb300 as mf
    reqs, meta = _oracle_requests()
    srv = Server(budget_bytes=1 << 30, streams=4, planners=4)
    futs = [srv.submit(r) for r in reqs]
    out = [f.result(timeout=300) for f in futs]
    srv.close()
    assert mf.device_status() == 0 and srv.failed == 0
    for res, m in zip(out, meta):
        sh, tp, lam, fs = _oracle_maps(oracle, m)
        N, D = _oracle_search(oracle, m, sh, tp, lam, fs)
        check_search(res.snr_max, res.argmax, None, N, D, oracle, label="served request %d" % res.tag)
        c = res.candidates
        assert len(c) > 0
        # the candidates are the top pixels of the served map, re-scored in FP64
        H, W = res.snr_max.shape
        want = oracle.topk_order(res.snr_max, res.argmax, 24)
        assert np.array_equal(c["y"].astype(np.int64) * W + c["x"], want)
        Nc, Dc = oracle.search_points(m["deq"], lam, sh, tp, c["y"].astype(np.int32), c["x"].astype(np.int32),
                                      c["k"].astype(np.int32), frame_scale=fs)
        ok = Dc > 0
        np.testing.assert_allclose(c["snr"][ok], Nc[ok] / np.sqrt(Dc[ok]), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(c["flux"][ok], Nc[ok] / Dc[ok], rtol=1e-9, atol=1e-12)


def test_a_request_whose_search_times_out_fails_alone(oracle):
    # one request's search is made to report a device wait that gave up (a
    # bounded wait aimed at its status slot); it comes back failed with
    # MF_ETIMEOUT while the requests around it, on other streams, match the
    # oracle
    from paper_2209_09848_gb300.serve import Server
    import paper_2209_09848_gb300 as mf
    reqs, meta = _oracle_requests(seed=22)
    reqs, meta = reqs[:5], meta[:5]
    reqs[2].probe_timeout = True
    srv = Server(budget_bytes=1 << 30, streams=4, planners=2)
    futs = [srv.submit(r) for r in reqs]
    for i, (f, m) in enumerate(zip(futs, meta)):
        if i == 2:
            with pytest.raises(mf.MFError) as e:
                f.result(timeout=300)
            assert e.value.status == mf.MF_ETIMEOUT
            continue
        res = f.result(timeout=300)
        sh, tp, lam, fs = _oracle_maps(oracle, m)
        N, D = _oracle_search(oracle, m, sh, tp, lam, fs)
        check_search(res.snr_max, res.argmax, None, N, D, oracle, label="request %d beside a failed one" % i)
    srv.close()
    assert srv.failed == 1
    # the probe also recorded its code in the device-wide word; reading clears it
    assert mf.device_status() == mf.MF_ETIMEOUT
    assert mf.device_status() == 0
