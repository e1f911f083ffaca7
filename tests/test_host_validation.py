"""Argument validation of the C ABI, on the host: every call below is
rejected before the library touches a device (no GPU needed), with the
status its header documents."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    m.load()
    return m


EINVAL, EUNSUPPORTED = 1, 5
FAKE = ctypes.c_void_p(0x1000)  # never dereferenced: the calls fail validation first


def _detect(mf, H=16, W=16, window=255, threshold=3.0, max_out=8, ws_bytes=None, n_out=FAKE, snr=FAKE):
    lib = mf.load()
    opts = mf.binding.DetectOpts(window, 1, threshold)
    need = ctypes.c_size_t()
    if H >= 1 and W >= 1 and max_out >= 0 and H * W < (1 << 31):
        lib.mf_detect_workspace_size(H, W, max(max_out, 0), ctypes.byref(need))
    ws = ws_bytes if ws_bytes is not None else need.value
    return lib.mf_detect(snr, FAKE, H, W, ctypes.byref(opts), None, FAKE, max_out, n_out, ctypes.c_void_p(0x100000),
                         ws, None)


def test_detect_validation(mf):
    assert _detect(mf, window=4) == EINVAL
    assert _detect(mf, window=0) == EINVAL
    assert _detect(mf, window=2049) == EINVAL
    assert _detect(mf, threshold=float("nan")) == EINVAL
    assert _detect(mf, threshold=float("inf")) == EINVAL
    assert _detect(mf, max_out=-1) == EINVAL
    assert _detect(mf, max_out=16385) == EUNSUPPORTED
    assert _detect(mf, H=0) == EINVAL
    assert _detect(mf, H=1 << 16, W=1 << 15) == EINVAL  # 2^31 pixels
    assert _detect(mf, ws_bytes=16) == EINVAL
    assert _detect(mf, n_out=None) == EINVAL
    assert _detect(mf, snr=None) == EINVAL


def _refit(mf, T=10, H=4, W=4, jitter=None, iterations=3, delta=1.0, n=4, scatter=True, ws_bytes=None):
    lib = mf.load()
    if jitter is None:
        jitter = np.random.default_rng(0).uniform(-0.2, 0.2, size=(T, 2))
    jitter = np.ascontiguousarray(jitter, np.float64)
    opts = mf.binding.RefitOpts(iterations, 0, delta)
    need = ctypes.c_size_t()
    lib.mf_refit_workspace_size(max(T, 6), ctypes.byref(need))
    ws = ws_bytes if ws_bytes is not None else need.value
    return lib.mf_background_refit(FAKE, T, H, W, FAKE if scatter else None, n,
                                   jitter.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts), FAKE, None,
                                   ctypes.c_void_p(0x100000), ws, None)


def test_refit_validation(mf):
    assert _refit(mf, T=5, jitter=np.zeros((5, 2)) + [[0.1, 0.2]]) == EINVAL  # fewer frames than coefficients
    assert _refit(mf, jitter=np.zeros((10, 2))) == EINVAL  # singular Gram matrix
    j = np.random.default_rng(1).uniform(-0.2, 0.2, size=(10, 2))
    j[4, 0] = np.nan
    assert _refit(mf, jitter=j) == EINVAL
    assert _refit(mf, delta=0.0) == EINVAL
    assert _refit(mf, delta=float("nan")) == EINVAL
    assert _refit(mf, iterations=-1) == EINVAL
    assert _refit(mf, iterations=1001) == EINVAL
    assert _refit(mf, n=0) == EINVAL
    assert _refit(mf, W=0) == EINVAL
    assert _refit(mf, ws_bytes=8) == EINVAL
    need = ctypes.c_size_t()
    assert mf.load().mf_refit_workspace_size(5, ctypes.byref(need)) == EINVAL


def test_frames_validation(mf):
    lib = mf.load()
    prm = mf.binding.PrfParams(0, 0, 0.7)
    vx = np.array([0.1, -0.2])
    vy = np.array([0.0, 0.3])
    T = 4
    out = ctypes.c_void_p()

    def call(times=None, jitter=None, kind=0):
        prm.kind = kind
        tm = None if times is None else np.ascontiguousarray(times, np.float64)
        jt = None if jitter is None else np.ascontiguousarray(jitter, np.float64)
        fr = mf.binding.Frames(None if tm is None else tm.ctypes.data_as(ctypes.c_void_p),
                               None if jt is None else jt.ctypes.data_as(ctypes.c_void_p))
        return lib.mf_prf_table_create_frames(ctypes.byref(prm), vx.ctypes.data_as(ctypes.c_void_p),
                                              vy.ctypes.data_as(ctypes.c_void_p), 2, T, ctypes.byref(fr), None,
                                              ctypes.byref(out))

    assert call(times=[0, 1, np.inf, 3]) == EINVAL
    assert call(jitter=[[0, 0], [0, np.nan], [0, 0], [0, 0]]) == EINVAL
    assert call(times=[0, 1, 2, 1e7]) == EINVAL  # 0.1 px/cadence x 1e7 cadences: beyond 2^20 px
    assert call(kind=3) == EINVAL
