"""The binding's checks of tensors passed as device pointers (no GPU): the
library cannot tell a host pointer from a device one, so host tensors, wrong
dtypes and wrong shapes must raise ValueError before anything reaches it."""
import numpy as np
import pytest
import torch

import paper_2209_09848_gb300 as mf


class _Bank:
    """Stands in for a filter bank handle: the checks read only K."""
    K = 3
    handle = None


T, H, W = 4, 8, 10


def _host():
    return (torch.zeros((T, H, W)), torch.ones((H, W)), torch.zeros((H, W), dtype=torch.uint8))


def test_search_rejects_host_tensors():
    r, s, m = _host()
    with pytest.raises(ValueError, match="stack must be a CUDA tensor"):
        mf.search(r, s, _Bank(), mask=m)
    with pytest.raises(ValueError, match="stack must be a CUDA tensor"):
        mf.search_noalloc(r, s, _Bank())
    with pytest.raises(ValueError, match="stack must be a CUDA tensor"):
        mf.rescore_topk(r, s, _Bank(), s, torch.zeros((H, W), dtype=torch.int32), 4)


def test_search_host_wants_device_sigma():
    r, s, m = _host()
    with pytest.raises(ValueError, match="sigma must be a CUDA tensor"):
        mf.search_host(r, s, _Bank(), mask=m)


def test_detect_checks():
    s = torch.zeros((H, W))
    a = torch.zeros((H, W), dtype=torch.int32)
    with pytest.raises(ValueError, match="snr_max must be a CUDA tensor"):
        mf.detect(s, a)
    with pytest.raises(ValueError, match=r"snr_max must be \[H, W\]"):
        mf.detect(torch.zeros((2, H, W)), a)


def test_refit_checks():
    jit = np.zeros((T, 2))
    with pytest.raises(ValueError, match="data must be a CUDA tensor"):
        mf.background_refit(torch.zeros((T, H, W)), jit, 1.0, 2)
    with pytest.raises(ValueError, match=r"data must be \[T, H, W\]"):
        mf.background_refit(torch.zeros((H, W)), jit, 1.0, 2)


def test_device_arg_rules():
    # the checks themselves, on tensors that need no GPU
    chk = mf.binding._device_arg
    chk("x", None)  # optional and absent
    with pytest.raises(ValueError, match="x is required"):
        chk("x", None, optional=False)
    with pytest.raises(ValueError, match="x must be a CUDA tensor"):
        chk("x", np.zeros(3))
    with pytest.raises(ValueError, match="x must be a CUDA tensor"):
        chk("x", torch.zeros(3))
    meta = torch.empty((H, W), device="meta")  # a non-CUDA device with no storage
    with pytest.raises(ValueError, match="CUDA"):
        chk("x", meta, dtype=torch.float32, shape=(H, W))


class _OnCuda(torch.Tensor):
    """A host tensor that reports a CUDA device: reaches the checks after
    the device check without a GPU (never passed to the library)."""

    @property
    def device(self):
        return torch.device("cuda", 0)


def _cuda_like(t):
    return t.as_subclass(_OnCuda)


def test_device_arg_dtype_shape_layout():
    chk = mf.binding._device_arg
    x = _cuda_like(torch.zeros((H, W)))
    chk("x", x, torch.device("cuda", 0), torch.float32, (H, W))
    with pytest.raises(ValueError, match="x must be on cuda:1"):
        chk("x", x, torch.device("cuda", 1))
    with pytest.raises(ValueError, match="x must be torch.int32"):
        chk("x", x, dtype=torch.int32)
    with pytest.raises(ValueError, match=r"x must have shape \(10, 8\)"):
        chk("x", x, shape=(W, H))
    xt = _cuda_like(torch.zeros((W, H)).t())
    with pytest.raises(ValueError, match="x must be contiguous"):
        chk("x", xt, shape=(H, W))
    chk("x", xt, shape=(H, W), contiguous=False)


def test_search_argument_rules_before_the_library():
    # a stack on the (reported) GPU: sigma, mask and frame_scale must match it
    r = _cuda_like(torch.zeros((T, H, W)))
    s = _cuda_like(torch.ones((H, W)))
    m = _cuda_like(torch.zeros((H, W), dtype=torch.uint8))
    chk = mf.binding._check_search_inputs
    chk(r, s, m, _cuda_like(torch.ones(T)))
    with pytest.raises(ValueError, match="sigma must be a CUDA tensor"):
        chk(r, torch.ones((H, W)), m, None)
    with pytest.raises(ValueError, match="sigma must be torch.float32"):
        chk(r, _cuda_like(torch.ones((H, W), dtype=torch.float64)), m, None)
    with pytest.raises(ValueError, match="mask must be torch.uint8"):
        chk(r, s, _cuda_like(torch.zeros((H, W), dtype=torch.bool)), None)
    with pytest.raises(ValueError, match=r"mask must have shape \(8, 10\)"):
        chk(r, s, _cuda_like(torch.zeros((H, W + 1), dtype=torch.uint8)), None)
    with pytest.raises(ValueError, match=r"frame_scale must have shape \(4,\)"):
        chk(r, s, m, _cuda_like(torch.ones((T, 1))))
    with pytest.raises(ValueError, match="sigma is required"):
        chk(r, None, m, None)
    # a host stack (mf_search_host): the device arguments on the given device
    chk(torch.zeros((T, H, W)), s, m, None, device=torch.device("cuda", 0))
    out = mf.binding._check_search_outputs
    out(s, _cuda_like(torch.zeros((H, W), dtype=torch.int32)), None, _Bank(), H, W, torch.device("cuda", 0))
    with pytest.raises(ValueError, match="argmax must be torch.int32"):
        out(s, s, None, _Bank(), H, W, torch.device("cuda", 0))
    with pytest.raises(ValueError, match=r"snr_all must have shape \(3, 8, 10\)"):
        out(s, _cuda_like(torch.zeros((H, W), dtype=torch.int32)), _cuda_like(torch.zeros((2, H, W))), _Bank(), H,
            W, torch.device("cuda", 0))


class _StubLib:
    """Records the library calls a binding function makes (returns MF_OK)."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


class _Stream:
    cuda_stream = 0


def test_valid_calls_reach_the_library(monkeypatch):
    # arguments shaped like the bench's and the tests' GPU calls pass every
    # check and reach the library (stubbed: nothing runs)
    stub = _StubLib()
    monkeypatch.setattr(mf.binding, "load", lambda: stub)
    r = _cuda_like(torch.zeros((T, H, W)))
    s = _cuda_like(torch.ones((H, W)))
    m = _cuda_like(torch.zeros((H, W), dtype=torch.uint8))
    fs = _cuda_like(torch.ones(T))
    ws = _cuda_like(torch.zeros(64, dtype=torch.uint8))
    out = (_cuda_like(torch.zeros((H, W))), _cuda_like(torch.zeros((H, W), dtype=torch.int32)), None)
    mf.search(r, s, _Bank(), mask=m, frame_scale=fs, workspace=ws, out=out, stream=_Stream())
    # a strided stack (rows contiguous) is accepted as the ABI allows
    big = _cuda_like(torch.zeros((T, H + 2, W + 3)))[:, 1:H + 1, 1:W + 1]
    mf.search(big, s, _Bank(), workspace=ws, out=out, stream=_Stream())
    mf.search_noalloc(r, s, _Bank(), mask=m, out=out, stream=_Stream())
    D = _cuda_like(torch.zeros((8, H, W)))
    S = _cuda_like(torch.zeros((8, 4, 4)))
    jit = np.random.default_rng(0).uniform(-0.1, 0.1, (8, 2))
    mf.background_refit(D, jit, 1.0, 2, scatter=S, resid=D, want_coef=False, workspace=ws, stream=_Stream())
    assert stub.calls == ["mf_search_workspace_size", "mf_search", "mf_search_workspace_size", "mf_search",
                          "mf_search_noalloc", "mf_refit_workspace_size", "mf_background_refit"]
