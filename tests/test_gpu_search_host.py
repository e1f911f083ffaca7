"""mf_search_host (stack in host memory): the same maps and candidates as
the device-stack calls, for contiguous and strided pinned stacks and for
pageable memory; the FP64 oracle on one case."""
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


def _case(T=21, H=90, W=77, seed=5):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, seed, mask_frac=0.02, movers=3)
    vx, vy = synth.velocity_grid(4, 3, -0.4, 0.4)
    return c, vx, vy


@pytest.mark.parametrize("layout", ["pinned", "strided", "pageable"])
def test_host_stack_matches_device_stack(mf, layout):
    c, vx, vy = _case()
    T, H, W = c["res"].shape
    table = mf.prf_table_create(vx, vy, T)
    sigma = torch.from_numpy(c["sigma"]).cuda()
    mask = torch.from_numpy(c["mask"]).cuda()
    res = torch.from_numpy(c["res"])
    if layout == "strided":
        big = torch.zeros((T, H + 3, W + 5), dtype=torch.float32).pin_memory()
        big[:, 1:H + 1, 2:W + 2] = res
        host = big[:, 1:H + 1, 2:W + 2]
    elif layout == "pinned":
        host = res.clone().pin_memory()
    else:
        host = res.clone()
    k_top = 50
    smax, amax, cand, n = mf.search_host(host, sigma, table, mask=mask, k_top=k_top)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    dm, da, _ = mf.search(res.cuda(), sigma, table, mask=mask)
    raw, dn = mf.rescore_topk(res.cuda(), sigma, table, dm, da, k_top, mask=mask)
    torch.cuda.synchronize()
    assert torch.equal(smax, dm.cpu()) and torch.equal(amax, da.cpu())
    assert int(n.item()) == int(dn.item())
    assert torch.equal(cand, raw.cpu())


def test_host_stack_against_oracle_and_errors(mf, oracle):
    c, vx, vy = _case(T=12, H=64, W=70, seed=9)
    T, H, W = c["res"].shape
    table = mf.prf_table_create(vx, vy, T)
    sigma = torch.from_numpy(c["sigma"]).cuda()
    mask = torch.from_numpy(c["mask"]).cuda()
    host = torch.from_numpy(c["res"]).pin_memory()
    smax, amax, _, _ = mf.search_host(host, sigma, table, mask=mask)
    torch.cuda.synchronize()
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    check_search(smax.numpy(), amax.numpy(), None, N, D, oracle, label="search_host")
    with pytest.raises(mf.MFError):  # workspace too small
        mf.search_host(host, sigma, table, mask=mask, workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    with pytest.raises(mf.MFError):  # k_top beyond the pixels
        mf.search_host(host, sigma, table, mask=mask, k_top=H * W + 1)


def test_pipelined_calls_keep_their_own_results(mf):
    """Uploads on a copy stream, kernels on one compute stream, two
    workspaces alternating with one event each: four different stacks in
    flight give exactly their own device-stack results."""
    from paper_2209_09848_gb300 import synth
    T, H, W = 18, 70, 66
    vx, vy = synth.velocity_grid(3, 3, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T)
    cases = [synth.small_case(T, H, W, 40 + i, mask_frac=0.01, movers=2) for i in range(4)]
    sigma = torch.from_numpy(cases[0]["sigma"]).cuda()
    hosts = [torch.from_numpy(c["res"]).pin_memory() for c in cases]
    comp, copy = torch.cuda.Stream(), torch.cuda.Stream()
    frees = [torch.cuda.Event(), torch.cuda.Event()]
    wss = [torch.empty(mf.search_host_workspace_size(hosts[0], table, 20), dtype=torch.uint8, device="cuda")
           for _ in frees]
    outs = []
    for i, h in enumerate(hosts):
        outs.append(mf.search_host(h, sigma, table, k_top=20, workspace=wss[i % 2], stream=comp,
                                   copy_stream=copy, ws_free=frees[i % 2]))
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    for h, (smax, amax, cand, n) in zip(hosts, outs):
        dm, da, _ = mf.search(h.cuda(), sigma, table)
        raw, dn = mf.rescore_topk(h.cuda(), sigma, table, dm, da, 20)
        torch.cuda.synchronize()
        assert torch.equal(smax, dm.cpu()) and torch.equal(amax, da.cpu())
        assert torch.equal(cand, raw.cpu()) and int(n.item()) == int(dn.item())


def test_host_search_status_slot(mf):
    # the host-stack search's workspace starts with its search's status
    # slot: mf_search_status reads it there (0 for a clean search, the probe's
    # code when a wait aimed at it runs out)
    c, vx, vy = _case(T=9, H=40, W=52, seed=13)
    T, H, W = c["res"].shape
    table = mf.prf_table_create(vx, vy, T)
    sigma = torch.from_numpy(c["sigma"]).cuda()
    host = torch.from_numpy(c["res"]).clone().pin_memory()
    ws = torch.empty(mf.search_host_workspace_size(host, table, 0), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    mf.search_host(host, sigma, table, workspace=ws)
    mf.search_status(ws, st)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    mf.search_host(host, sigma, table, workspace=ws)
    mf.wait_probe_search(ws)
    mf.search_status(ws, st)
    torch.cuda.synchronize()
    assert int(st[0]) == 4
    assert mf.device_status() == mf.MF_ETIMEOUT and mf.device_status() == 0
