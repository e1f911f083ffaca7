"""mf_prf_bank (no GPU): the filter bank the library builds on the host --
base shifts and FP64 footprints -- against the FP64 oracle's own tables:
linear trajectories (Section 2) for every PRF kind, the frame model (frame
times with gaps and fractional values, pointing jitter; Section 2.1, Fig. 3)
and the phase-quantised bank.  Shifts are integers and must be identical;
footprints agree to FP64 rounding (the two sides normalise in different
orders)."""
import os

import numpy as np
import pytest

mf = pytest.importorskip("paper_2209_09848_gb300")

TAP_TOL = 1e-15


def _vel(seed, n, vmax):
    g = np.random.default_rng(seed)
    vx, vy = g.uniform(-vmax, vmax, n), g.uniform(-vmax, vmax, n)
    vx[0], vy[0] = 0.0, 0.0
    vx[1], vy[1] = 0.25, -0.5  # phases on a quarter-pixel grid, halves included
    return vx, vy


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("T,vmax", [(1, 0.3), (37, 0.6), (400, 0.1), (50, 3.7)])
def test_linear_bank_equals_oracle(oracle, kind, T, vmax):
    vx, vy = _vel(T + kind, 9, vmax)
    s0, t0 = oracle.trajectory_table(vx, vy, T, kind=kind)
    s1, t1 = mf.prf_bank(vx, vy, T, kind=kind)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(t1, t0, rtol=0, atol=TAP_TOL)


@pytest.mark.parametrize("sigma", [0.45, 0.7, 1.3])
def test_prf_width(oracle, sigma):
    vx, vy = _vel(5, 6, 0.4)
    s0, t0 = oracle.trajectory_table(vx, vy, 30, sigma=sigma)
    s1, t1 = mf.prf_bank(vx, vy, 30, sigma_px=sigma)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(t1, t0, rtol=0, atol=TAP_TOL)


@pytest.mark.parametrize("gap,jit,frac", [(0, 0.3, False), (200, 0.25, True), (37, 1.7, True)])
def test_frame_model_bank_equals_oracle(oracle, gap, jit, frac):
    T = 60
    g = np.random.default_rng(gap + 1)
    tau = np.arange(T, dtype=np.float64)
    tau[T // 2:] += gap
    if frac:
        tau += g.uniform(-0.2, 0.2, T)
    jitter = g.uniform(-jit, jit, size=(T, 2))
    vx, vy = _vel(gap, 8, 0.4)
    s0, t0 = oracle.trajectory_table_frames(vx, vy, T, times=tau, jitter=jitter)
    s1, t1 = mf.prf_bank(vx, vy, T, times=tau, jitter=jitter)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(t1, t0, rtol=0, atol=TAP_TOL)
    # times alone and jitter alone
    s0, t0 = oracle.trajectory_table_frames(vx, vy, T, times=tau)
    s1, t1 = mf.prf_bank(vx, vy, T, times=tau)
    assert np.array_equal(s0, s1) and np.abs(t1 - t0).max() <= TAP_TOL
    s0, t0 = oracle.trajectory_table_frames(vx, vy, T, jitter=jitter)
    s1, t1 = mf.prf_bank(vx, vy, T, jitter=jitter)
    assert np.array_equal(s0, s1) and np.abs(t1 - t0).max() <= TAP_TOL


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 16, 4096])
def test_quantised_bank_equals_oracle(oracle, Q):
    vx, vy = _vel(Q, 10, 0.7)
    T = 80
    s0, t0 = oracle.trajectory_table_quantised(vx, vy, T, Q)
    s1, t1 = mf.prf_bank(vx, vy, T, phase_steps=Q)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(t1, t0, rtol=0, atol=TAP_TOL)


def test_quantised_bank_plans_the_factored_numerator():
    # quantised footprints are still separable, and trajectories of one v_x
    # share their x-phases: the factored layout of the exact bank
    g = np.linspace(-0.1, 0.1, 10)
    vx, vy = np.repeat(g, 10), np.tile(g, 10)
    exact = mf.prf_plan(vx, vy, 1000)
    quant = mf.prf_plan(vx, vy, 1000, phase_steps=4)
    assert quant["kernel"] == 2 and quant["taps"] == 5
    assert {k: quant[k] for k in ("groups", "warps_per_group", "tile_h", "tile_w", "time_segments")} == \
        {k: exact[k] for k in ("groups", "warps_per_group", "tile_h", "tile_w", "time_segments")}


def test_bank_arguments_rejected():
    vx = vy = np.zeros(2)
    for q in (-1, 4097):
        with pytest.raises(mf.MFError) as e:
            mf.prf_bank(vx, vy, 3, phase_steps=q)
        assert e.value.status == 1 and "phase_steps" in str(e.value)
    with pytest.raises(mf.MFError):
        mf.prf_bank(np.array([np.nan]), np.array([0.0]), 3)
    with pytest.raises(mf.MFError):
        mf.prf_bank(vx, vy, 3, times=np.array([0.0, np.inf, 2.0]))
    with pytest.raises(ValueError):
        mf.prf_bank(vx, np.zeros(3), 3)
    # the outputs are optional at the C level
    assert mf.load().mf_prf_bank(mf.binding.PrfParams(0, 0, 0.7), vx.ctypes.data_as(mf.binding.ctypes.c_void_p),
                                 vy.ctypes.data_as(mf.binding.ctypes.c_void_p), 2, 3, None, None, None) == 0


@pytest.mark.parametrize("Q", [2, 4, 7])
def test_quantised_frame_model_bank_equals_oracle(oracle, Q):
    T = 48
    g = np.random.default_rng(Q)
    tau = np.arange(T, dtype=np.float64) + np.where(np.arange(T) >= T // 3, 55.0, 0.0) + g.uniform(-0.2, 0.2, T)
    jitter = g.uniform(-0.8, 0.8, size=(T, 2))
    vx, vy = _vel(Q + 100, 8, 0.5)
    s0, t0 = oracle.trajectory_table_frames(vx, vy, T, times=tau, jitter=jitter, Q=Q)
    s1, t1 = mf.prf_bank(vx, vy, T, times=tau, jitter=jitter, phase_steps=Q)
    assert np.array_equal(s0, s1)
    np.testing.assert_allclose(t1, t0, rtol=0, atol=TAP_TOL)


def _quantised_golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "trajectory_quantised.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            v, t, q, s, ph = line.split()
            rows.append((float(v), int(t), int(q), int(s), float(ph)))
    return rows


def test_quantised_golden(oracle):
    # hand-worked base pixels and rounded phases, both axes, on the oracle
    # and on the library's host-built bank
    for v, t, Q, s, ph in _quantised_golden():
        want = oracle.prf_taps(ph, 0.0)
        for build in (lambda a, b: oracle.trajectory_table_quantised(a, b, t + 1, Q),
                      lambda a, b: mf.prf_bank(a, b, t + 1, phase_steps=Q)):
            sh, tp = build([v], [0.0])
            assert sh[0, t, 0] == s and sh[0, t, 1] == 0, (v, t, Q)
            np.testing.assert_allclose(tp[0, t], want, rtol=0, atol=1e-15)
            sh, tp = build([0.0], [v])
            assert sh[0, t, 1] == s and sh[0, t, 0] == 0, (v, t, Q)
            np.testing.assert_allclose(tp[0, t], want.T, rtol=0, atol=1e-15)
