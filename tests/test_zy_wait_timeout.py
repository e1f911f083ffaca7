"""The failure path of the bounded device waits, on the GPU: mf_wait_probe
launches one CTA whose wait on an mbarrier that nothing completes runs out
of the bound every kernel's waits use (about a second).  The status word
then reports MF_ETIMEOUT with the probe's code, reading it clears it, and
the context keeps working: a search right after matches the oracle.
Nothing faults, traps or hangs."""
import time

import pytest

from _util import check_search

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_wait_runs_out_and_the_context_survives(oracle):
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import synth
    assert torch.cuda.is_available()
    mf.load()
    assert mf.device_status() == 0
    t0 = time.perf_counter()
    mf.wait_probe()
    status = mf.device_status()  # synchronises the device, then reads and clears
    waited = time.perf_counter() - t0
    assert status == mf.binding.MF_ETIMEOUT
    assert "code 4" in mf.last_error()
    assert 0.3 < waited < 60.0  # 2^31 SM cycles
    assert mf.device_status() == 0
    T, H, W = 8, 40, 48
    c = synth.small_case(T, H, W, 3, mask_frac=0.02, movers=1)
    vx, vy = synth.velocity_grid(3, 2, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T)
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    smax, amax, sall = mf.search(r, s, table, mask=m, want_all=True)
    torch.cuda.synchronize()
    assert mf.device_status() == 0
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    check_search(smax.cpu().numpy(), amax.cpu().numpy(), sall.cpu().numpy(), N, D, oracle, label="after the probe")


def test_search_status_slot_is_per_search(oracle):
    # each search reports through its own status slot: 0 after a clean
    # search; the probe aimed at one search's workspace makes that search
    # (and only it) report code 4, read without synchronising the device;
    # a search enqueued after the failure on another workspace is unaffected
    import paper_2209_09848_gb300 as mf
    from paper_2209_09848_gb300 import synth
    mf.load()
    assert mf.device_status() == 0
    T, H, W = 10, 48, 64
    c = synth.small_case(T, H, W, 8, mask_frac=0.02, movers=1)
    vx, vy = synth.velocity_grid(3, 3, -0.3, 0.3)
    table = mf.prf_table_create(vx, vy, T)
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    nbytes = mf.search_workspace_size((T, H, W), table)
    ws_a = torch.full((nbytes,), 0xAB, dtype=torch.uint8, device="cuda")  # stale bytes: the search clears its slot
    ws_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st_a = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    st_b = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    mf.search(r, s, table, mask=m, workspace=ws_a)
    mf.search_status(ws_a, st_a)
    torch.cuda.synchronize()
    assert int(st_a[0]) == 0 and mf.device_status() == 0
    mf.search(r, s, table, mask=m, workspace=ws_a)
    mf.wait_probe_search(ws_a)
    mf.search_status(ws_a, st_a)
    smax, amax, sall = mf.search(r, s, table, mask=m, workspace=ws_b, want_all=True)
    mf.search_status(ws_b, st_b)
    torch.cuda.synchronize()
    assert int(st_a[0]) == 4 and int(st_b[0]) == 0
    sh, tp = oracle.trajectory_table(vx, vy, T)
    lam = oracle.inverse_variance(c["sigma"], c["mask"])
    N, D = oracle.search_full(c["res"], lam, sh, tp)
    check_search(smax.cpu().numpy(), amax.cpu().numpy(), sall.cpu().numpy(), N, D, oracle, label="beside a failure")
    # the probe also wrote the device-wide word; reading it clears it
    assert mf.device_status() == mf.MF_ETIMEOUT
    assert mf.device_status() == 0
    # a device status slot copied into device memory works the same way
    dst = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    mf.search(r, s, table, mask=m, workspace=ws_a)
    mf.search_status(ws_a, dst)
    torch.cuda.synchronize()
    assert int(dst.item()) == 0
