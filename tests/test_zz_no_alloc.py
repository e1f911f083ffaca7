"""mf_search_noalloc: the search for callers that cannot allocate device
memory -- plug-ins whose host application owns every device allocation, or
real-time loops that must not call cudaMalloc because it can synchronise the
device.  It keeps its scratch in one static device array inside libmf, shared
by every call, so each call must give the same maps as mf_search with a
caller-owned workspace whatever the previous call left in that array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from _util import SNR_TOL, snr_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    m.load()
    return m


def _case(mf, seed, T, H, W, nx, ny, vmax, mask_frac):
    from paper_2209_09848_gb300 import synth
    c = synth.small_case(T, H, W, seed, mask_frac=mask_frac, movers=3)
    vx, vy = synth.velocity_grid(nx, ny, -vmax, vmax)
    table = mf.prf_table_create(vx, vy, T)
    r = torch.from_numpy(c["res"]).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = None if c["mask"] is None else torch.from_numpy(c["mask"]).cuda()
    return table, r, s, m


def test_noalloc_matches_workspace_search_on_two_calls(mf):
    # a larger search first, then a smaller one: the second call meets the
    # scratch array holding the first call's data
    cases = [(1, 24, 120, 150, 4, 4, 0.3, 0.02), (2, 9, 40, 70, 3, 2, 0.5, 0.0)]
    for args in cases:
        table, r, s, m = _case(mf, *args)
        want_max, want_arg, want_all = mf.search(r, s, table, mask=m, want_all=True)
        got_max, got_arg, got_all = mf.search_noalloc(r, s, table, mask=m, want_all=True)
        torch.cuda.synchronize()
        assert mf.device_status() == 0
        _, ok = snr_close(got_all.cpu().numpy(), want_all.cpu().numpy(), SNR_TOL)
        assert ok
        _, ok = snr_close(got_max.cpu().numpy(), want_max.cpu().numpy(), SNR_TOL)
        assert ok
        assert np.array_equal(got_arg.cpu().numpy(), want_arg.cpu().numpy())


def test_noalloc_bf16_frame_scale_on_a_side_stream(mf):
    # scaled bf16 storage, searched on a non-default stream by both entry
    # points (one after the other on that stream)
    from paper_2209_09848_gb300 import synth
    T, H, W = 18, 96, 130
    c = synth.small_case(T, H, W, 41, mask_frac=0.01, movers=3)
    vx, vy = synth.velocity_grid(4, 3, -0.25, 0.25)
    table = mf.prf_table_create(vx, vy, T)
    scale = (np.abs(c["res"]).max(axis=(1, 2)) / 64.0).astype(np.float32)
    q = torch.from_numpy(c["res"] / scale[:, None, None]).to(torch.bfloat16).cuda()
    s = torch.from_numpy(c["sigma"]).cuda()
    m = torch.from_numpy(c["mask"]).cuda()
    fs = torch.from_numpy(scale).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        want_max, want_arg, want_all = mf.search(q, s, table, mask=m, frame_scale=fs, want_all=True, stream=side)
        got_max, got_arg, got_all = mf.search_noalloc(q, s, table, mask=m, frame_scale=fs, want_all=True,
                                                      stream=side)
    side.synchronize()
    assert mf.device_status() == 0
    _, ok = snr_close(got_all.cpu().numpy(), want_all.cpu().numpy(), SNR_TOL)
    assert ok
    _, ok = snr_close(got_max.cpu().numpy(), want_max.cpu().numpy(), SNR_TOL)
    assert ok
    assert np.array_equal(got_arg.cpu().numpy(), want_arg.cpu().numpy())


def test_noalloc_rejects_a_search_larger_than_its_scratch(mf):
    T, H, W = 80, 512, 512  # the denominator and numerator planes alone exceed 64 MiB
    table = mf.prf_table_create([0.05, -0.05, 0.02, -0.02, 0.0, 0.01, -0.01, 0.03, -0.03, 0.04] * 4,
                                [0.0, 0.1, -0.1, 0.05, -0.05, 0.0, 0.02, -0.02, 0.07, -0.07] * 4, T)
    r = torch.zeros((T, H, W), device="cuda")
    s = torch.ones((H, W), device="cuda")
    # outputs hold a sentinel: a rejected call enqueues nothing
    out = (torch.full((H, W), 7.25, device="cuda"), torch.full((H, W), 1234, dtype=torch.int32, device="cuda"),
           None)
    with pytest.raises(mf.MFError) as e:
        mf.search_noalloc(r, s, table, out=out)
    assert e.value.status == 1 and "scratch" in str(e.value)
    torch.cuda.synchronize()
    assert bool((out[0] == 7.25).all()) and bool((out[1] == 1234).all())
    assert mf.device_status() == 0
