"""ctypes binding for libmf (include/mf.h).  Argument marshalling only: every
step of the search runs in the CUDA library.  PyTorch supplies device memory
and streams.  Function names follow the C entry points without the ``mf_``
prefix."""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libmf.so")
_lib = None
_lock = threading.Lock()

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_ETIMEOUT, MF_EUNSUPPORTED = range(6)
MF_F32, MF_BF16, MF_F16 = 0, 1, 2
_DTYPES = {torch.float32: MF_F32, torch.bfloat16: MF_BF16, torch.float16: MF_F16}


class MFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libmf status %d: %s" % (status, msg))
        self.status = status


class PrfParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("phase_steps", ctypes.c_int32), ("sigma_px", ctypes.c_double)]


class Stack(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("T", ctypes.c_int64), ("H", ctypes.c_int64), ("W", ctypes.c_int64),
                ("frame_stride", ctypes.c_int64), ("row_stride", ctypes.c_int64),
                ("frame_scale", ctypes.c_void_p)]


class Candidate(ctypes.Structure):
    _fields_ = [("y", ctypes.c_int32), ("x", ctypes.c_int32), ("k", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("snr", ctypes.c_double), ("flux", ctypes.c_double),
                ("snr_search", ctypes.c_float), ("reserved2", ctypes.c_float)]


CANDIDATE_BYTES = ctypes.sizeof(Candidate)


class Frames(ctypes.Structure):
    _fields_ = [("times", ctypes.c_void_p), ("jitter", ctypes.c_void_p)]


class RefitOpts(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("reserved", ctypes.c_int32), ("delta", ctypes.c_double)]


class DetectOpts(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("subtract_mean", ctypes.c_int32), ("threshold", ctypes.c_double)]


class Detection(ctypes.Structure):
    _fields_ = [("y", ctypes.c_int32), ("x", ctypes.c_int32), ("k", ctypes.c_int32), ("npix", ctypes.c_int32),
                ("z", ctypes.c_double), ("mean", ctypes.c_double), ("sigma", ctypes.c_double),
                ("snr", ctypes.c_float), ("reserved", ctypes.c_int32)]


DETECTION_BYTES = ctypes.sizeof(Detection)


class PlanOpts(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("vec", ctypes.c_int32), ("lockstep", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("group", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("stages", ctypes.c_int32), ("segments", ctypes.c_int32)]


_LAYOUT_KEYS = ("shape", "vec", "lockstep", "kernel", "group", "tile_h", "tile_w", "stages", "segments")


def _opts(**kw):
    """mf_plan_opts from keyword layout options; None when all are None."""
    if all(kw.get(k) is None for k in _LAYOUT_KEYS):
        return None
    o = PlanOpts()
    o.shape = -1 if kw.get("shape") is None else int(kw["shape"])
    o.vec = 0 if kw.get("vec") is None else int(kw["vec"])
    o.lockstep = -1 if kw.get("lockstep") is None else int(kw["lockstep"])
    for k in ("kernel", "group", "tile_h", "tile_w", "stages", "segments"):
        setattr(o, k, 0 if kw.get(k) is None else int(kw[k]))
    return ctypes.byref(o)


class TableInfo(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("T", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("warps_per_group", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("window_pitch", ctypes.c_int32),
                ("window_rows", ctypes.c_int32), ("segments", ctypes.c_int32),
                ("max_abs_shift", ctypes.c_int32), ("g_nnz", ctypes.c_int64), ("smem_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("cost", ctypes.c_double), ("vec", ctypes.c_int32),
                ("lockstep", ctypes.c_int32), ("kernel", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("time_segments", ctypes.c_int32), ("taps", ctypes.c_int32), ("den_tile_h", ctypes.c_int32),
                ("phase_planes", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("reserved", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("k", KernelStat * 16)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libmf.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libmf.so not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "mf_prf_table_create": ([ctypes.POINTER(PrfParams), P, P, I32, I32, pp], ctypes.c_int),
            "mf_prf_table_create_ex": ([ctypes.POINTER(PrfParams), P, P, I32, I32, ctypes.POINTER(PlanOpts), pp],
                                       ctypes.c_int),
            "mf_prf_table_create_custom": ([P, P, I32, I32, pp], ctypes.c_int),
            "mf_prf_table_create_frames": ([ctypes.POINTER(PrfParams), P, P, I32, I32, ctypes.POINTER(Frames),
                                            ctypes.POINTER(PlanOpts), pp], ctypes.c_int),
            "mf_prf_table_destroy": ([P], None),
            "mf_prf_table_dims": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
            "mf_prf_table_export": ([P, P, P], ctypes.c_int),
            "mf_prf_table_info": ([P, ctypes.POINTER(TableInfo)], ctypes.c_int),
            "mf_prf_plan": ([ctypes.POINTER(PrfParams), P, P, I32, I32, ctypes.POINTER(PlanOpts),
                             ctypes.POINTER(TableInfo)], ctypes.c_int),
            "mf_prf_plan_frames": ([ctypes.POINTER(PrfParams), P, P, I32, I32, ctypes.POINTER(Frames),
                                    ctypes.POINTER(PlanOpts), ctypes.POINTER(TableInfo)], ctypes.c_int),
            "mf_prf_bank": ([ctypes.POINTER(PrfParams), P, P, I32, I32, ctypes.POINTER(Frames), P, P],
                            ctypes.c_int),
            "mf_search_workspace_size": ([ctypes.POINTER(Stack), P, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_search": ([ctypes.POINTER(Stack), P, P, P, P, P, P, P, SZ, P], ctypes.c_int),
            "mf_search_noalloc": ([ctypes.POINTER(Stack), P, P, P, P, P, P, P], ctypes.c_int),
            "mf_rescore_workspace_size": ([I64, I64, I32, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_rescore_topk": ([ctypes.POINTER(Stack), P, P, P, P, P, I32, P, P, P, SZ, P], ctypes.c_int),
            "mf_search_host_workspace_size": ([ctypes.POINTER(Stack), P, I32, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_search_host": ([ctypes.POINTER(Stack), P, P, P, P, P, I32, P, P, P, SZ, P, P, P], ctypes.c_int),
            "mf_refit_workspace_size": ([I64, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_background_refit": ([P, I64, I64, I64, P, I32, P, ctypes.POINTER(RefitOpts), P, P, P, SZ, P],
                                    ctypes.c_int),
            "mf_detect_workspace_size": ([I64, I64, I32, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_detect": ([P, P, I64, I64, ctypes.POINTER(DetectOpts), P, P, I32, P, P, SZ, P], ctypes.c_int),
            "mf_profile_enable": ([I32], ctypes.c_int),
            "mf_profile_read": ([ctypes.POINTER(Profile), I32], ctypes.c_int),
            "mf_batch_create": ([pp], ctypes.c_int),
            "mf_batch_add": ([P, ctypes.POINTER(Stack), P, P, P, P, P, P, ctypes.POINTER(I32)], ctypes.c_int),
            "mf_batch_workspace_size": ([P, ctypes.POINTER(SZ)], ctypes.c_int),
            "mf_batch_prepare": ([P, P, SZ], ctypes.c_int),
            "mf_batch_run": ([P, P], ctypes.c_int),
            "mf_batch_poll": ([P, ctypes.POINTER(I32)], ctypes.c_int),
            "mf_batch_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
            "mf_batch_destroy": ([P], None),
            "mf_last_error": ([], ctypes.c_char_p),
            "mf_device_status": ([], ctypes.c_int),
            "mf_wait_probe": ([P], ctypes.c_int),
            "mf_wait_probe_search": ([P, P], ctypes.c_int),
            "mf_search_status": ([P, P, P], ctypes.c_int),
            "mf_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load().mf_last_error().decode()


def version() -> str:
    return load().mf_version().decode()


def _check(status):
    if status != MF_OK:
        raise MFError(status, last_error())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _device_arg(name, t, device=None, dtype=None, shape=None, contiguous=True, optional=True):
    """Check a tensor the library takes as a device pointer: a CUDA tensor
    (on `device` when given) of `dtype` and `shape`, contiguous.  The library
    cannot tell a host pointer from a device one, so this is where such a
    mistake becomes a ValueError instead of a kernel reading host memory."""
    if t is None:
        if optional:
            return
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and t.device != device:
        raise ValueError("%s must be on %s, not %s" % (name, device, t.device))
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, not %s" % (name, dtype, t.dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, not %s" % (name, tuple(shape), tuple(t.shape)))
    if contiguous and not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class PrfTable:
    """Filter bank handle (mf_prf_table)."""

    def __init__(self, handle):
        self._h = handle
        K, T = ctypes.c_int32(), ctypes.c_int32()
        _check(load().mf_prf_table_dims(self._h, ctypes.byref(K), ctypes.byref(T)))
        self.K, self.T = K.value, T.value

    @property
    def handle(self):
        return self._h

    def export(self):
        import numpy as np
        shifts = np.zeros((self.K, self.T, 2), np.int32)
        taps = np.zeros((self.K, self.T, 5, 5), np.float64)
        _check(load().mf_prf_table_export(self._h, shifts.ctypes.data_as(ctypes.c_void_p),
                                          taps.ctypes.data_as(ctypes.c_void_p)))
        return shifts, taps

    def info(self) -> dict:
        inf = TableInfo()
        _check(load().mf_prf_table_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def destroy(self):
        if self._h:
            load().mf_prf_table_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _bank_args(vx, vy, T, sigma_px, kind, phase_steps, times, jitter):
    """Marshal a velocity filter bank's arguments: (PrfParams, vx, vy, Frames
    or None, arrays to keep alive during the call)."""
    import numpy as np
    vx = np.ascontiguousarray(vx, np.float64)
    vy = np.ascontiguousarray(vy, np.float64)
    if vx.shape != vy.shape or vx.ndim != 1:
        raise ValueError("vx and vy must be 1-D of equal length")
    prm = PrfParams(int(kind), int(phase_steps), float(sigma_px))
    if times is None and jitter is None:
        return prm, vx, vy, None, ()
    tm = None if times is None else np.ascontiguousarray(times, np.float64)
    jt = None if jitter is None else np.ascontiguousarray(jitter, np.float64)
    if tm is not None and tm.shape != (int(T),):
        raise ValueError("times must have shape (T,)")
    if jt is not None and jt.shape != (int(T), 2):
        raise ValueError("jitter must have shape (T, 2)")
    fr = Frames(None if tm is None else tm.ctypes.data_as(ctypes.c_void_p),
                None if jt is None else jt.ctypes.data_as(ctypes.c_void_p))
    return prm, vx, vy, fr, (tm, jt)


def _vptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def prf_table_create(vx, vy, T, sigma_px=0.7, kind=0, times=None, jitter=None, phase_steps=0,
                     **layout) -> PrfTable:
    """mf_prf_table_create, or mf_prf_table_create_ex when layout options are
    given: shape, vec, lockstep (general numerator), kernel (1 general,
    2 factored), group, tile_h, tile_w, stages, segments (factored
    numerator); None or absent = automatic.  times ([T] frame times in
    cadences) and jitter ([T, 2] (x, y) pointing offsets in pixels) select
    mf_prf_table_create_frames.  phase_steps = Q > 0 builds the
    phase-quantised bank (phases rounded to multiples of 1/Q)."""
    bad = set(layout) - set(_LAYOUT_KEYS)
    if bad:
        raise TypeError("unknown layout option(s) %s" % sorted(bad))
    prm, vx, vy, fr, _keep = _bank_args(vx, vy, T, sigma_px, kind, phase_steps, times, jitter)
    h = ctypes.c_void_p()
    opts = _opts(**layout)
    if fr is not None:
        _check(load().mf_prf_table_create_frames(ctypes.byref(prm), _vptr(vx), _vptr(vy), vx.shape[0], int(T),
                                                 ctypes.byref(fr), opts, ctypes.byref(h)))
    elif opts is None:
        _check(load().mf_prf_table_create(ctypes.byref(prm), _vptr(vx), _vptr(vy), vx.shape[0], int(T),
                                          ctypes.byref(h)))
    else:
        _check(load().mf_prf_table_create_ex(ctypes.byref(prm), _vptr(vx), _vptr(vy), vx.shape[0], int(T),
                                             opts, ctypes.byref(h)))
    return PrfTable(h)


def prf_plan(vx, vy, T, sigma_px=0.7, kind=0, times=None, jitter=None, phase_steps=0, **layout) -> dict:
    """mf_prf_plan (mf_prf_plan_frames with times / jitter): host-only layout
    of a Gaussian-PRF filter bank (no GPU needed)."""
    bad = set(layout) - set(_LAYOUT_KEYS)
    if bad:
        raise TypeError("unknown layout option(s) %s" % sorted(bad))
    prm, vx, vy, fr, _keep = _bank_args(vx, vy, T, sigma_px, kind, phase_steps, times, jitter)
    inf = TableInfo()
    if fr is not None:
        _check(load().mf_prf_plan_frames(ctypes.byref(prm), _vptr(vx), _vptr(vy), vx.shape[0], int(T),
                                         ctypes.byref(fr), _opts(**layout), ctypes.byref(inf)))
    else:
        _check(load().mf_prf_plan(ctypes.byref(prm), _vptr(vx), _vptr(vy), vx.shape[0], int(T), _opts(**layout),
                                  ctypes.byref(inf)))
    return inf.as_dict()


def prf_bank(vx, vy, T, sigma_px=0.7, kind=0, times=None, jitter=None, phase_steps=0):
    """mf_prf_bank: the filter bank's base shifts int32 [K, T, 2] and FP64
    footprints [K, T, 5, 5], built on the host (no GPU needed)."""
    import numpy as np
    prm, vx, vy, fr, _keep = _bank_args(vx, vy, T, sigma_px, kind, phase_steps, times, jitter)
    K = vx.shape[0]
    shifts = np.zeros((K, int(T), 2), np.int32)
    taps = np.zeros((K, int(T), 5, 5), np.float64)
    _check(load().mf_prf_bank(ctypes.byref(prm), _vptr(vx), _vptr(vy), K, int(T),
                              None if fr is None else ctypes.byref(fr), _vptr(shifts), _vptr(taps)))
    return shifts, taps


def prf_table_create_custom(shifts, taps) -> PrfTable:
    """shifts int32 [K, T, 2] as (s_x, s_y); taps float64 [K, T, 5, 5] as [.., dy+2, dx+2]."""
    import numpy as np
    shifts = np.ascontiguousarray(shifts, np.int32)
    taps = np.ascontiguousarray(taps, np.float64)
    K, T = shifts.shape[:2]
    if shifts.shape != (K, T, 2) or taps.shape != (K, T, 5, 5):
        raise ValueError("shifts must be [K, T, 2] and taps [K, T, 5, 5]")
    h = ctypes.c_void_p()
    _check(load().mf_prf_table_create_custom(shifts.ctypes.data_as(ctypes.c_void_p),
                                             taps.ctypes.data_as(ctypes.c_void_p), K, T, ctypes.byref(h)))
    return PrfTable(h)


def make_stack(data: torch.Tensor, frame_scale: torch.Tensor | None = None) -> Stack:
    if data.dim() != 3:
        raise ValueError("stack must be [T, H, W]")
    if data.dtype not in _DTYPES:
        raise ValueError("stack dtype must be float32, bfloat16 or float16")
    if data.stride(2) != 1:
        raise ValueError("stack rows must be contiguous")
    T, H, W = data.shape
    if frame_scale is not None:
        if frame_scale.dtype != torch.float32 or frame_scale.numel() != T or not frame_scale.is_contiguous():
            raise ValueError("frame_scale must be a contiguous float32 tensor of length T")
    return Stack(data.data_ptr(), _DTYPES[data.dtype], 0, T, H, W, data.stride(0), data.stride(1),
                 None if frame_scale is None else frame_scale.data_ptr())


def search_workspace_size(shape, table: PrfTable, dtype=torch.float32) -> int:
    """mf_search_workspace_size for a stack of this shape and dtype (a bf16 /
    fp16 stack may need less: its weighted stack can be 16-bit)."""
    T, H, W = shape
    st = Stack(None, _DTYPES[dtype], 0, T, H, W, H * W, W, None)
    n = ctypes.c_size_t()
    _check(load().mf_search_workspace_size(ctypes.byref(st), table.handle, ctypes.byref(n)))
    return n.value


def _workspace(nbytes, device, workspace):
    if workspace is not None:
        return workspace  # size and alignment are checked by the library
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def _check_search_inputs(stack, sigma, mask, frame_scale, device=None):
    """The device arguments of a search: stack [T, H, W] (rows contiguous,
    any frame and row stride), sigma float32 and mask uint8 [H, W] and
    frame_scale float32 [T] on the stack's device (`device` for a host
    stack)."""
    T, H, W = stack.shape
    if device is None:
        _device_arg("stack", stack, contiguous=False)
        device = stack.device
    _device_arg("sigma", sigma, device, torch.float32, (H, W), optional=False)
    _device_arg("mask", mask, device, torch.uint8, (H, W))
    _device_arg("frame_scale", frame_scale, device, torch.float32, (T,))


def _check_search_outputs(snr_max, argmax, snr_all, table, H, W, device):
    _device_arg("snr_max", snr_max, device, torch.float32, (H, W), optional=False)
    _device_arg("argmax", argmax, device, torch.int32, (H, W), optional=False)
    _device_arg("snr_all", snr_all, device, torch.float32, (table.K, H, W))


def search(stack: torch.Tensor, sigma: torch.Tensor, table: PrfTable, mask: torch.Tensor | None = None,
           frame_scale: torch.Tensor | None = None, want_all: bool = False, workspace=None, out=None,
           stream=None):
    """mf_search: returns (snr_max [H, W] f32, argmax [H, W] i32, snr_all [K, H, W] f32 or None)."""
    st = make_stack(stack, frame_scale)
    T, H, W = stack.shape
    dev = stack.device
    _check_search_inputs(stack, sigma, mask, frame_scale)
    if out is None:
        snr_max = torch.empty((H, W), dtype=torch.float32, device=dev)
        argmax = torch.empty((H, W), dtype=torch.int32, device=dev)
        snr_all = torch.empty((table.K, H, W), dtype=torch.float32, device=dev) if want_all else None
    else:
        snr_max, argmax, snr_all = out
        _check_search_outputs(snr_max, argmax, snr_all, table, H, W, dev)
    _device_arg("workspace", workspace, dev)
    nbytes = search_workspace_size((T, H, W), table, stack.dtype)
    ws = _workspace(nbytes, dev, workspace)
    _check(load().mf_search(ctypes.byref(st), _ptr(sigma), _ptr(mask), table.handle, _ptr(snr_max),
                            _ptr(argmax), _ptr(snr_all), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream_ptr(stream)))
    return snr_max, argmax, snr_all


def search_noalloc(stack: torch.Tensor, sigma: torch.Tensor, table: PrfTable, mask: torch.Tensor | None = None,
                   frame_scale: torch.Tensor | None = None, want_all: bool = False, out=None, stream=None):
    """mf_search_noalloc: mf_search with the library's static scratch (no workspace argument)."""
    st = make_stack(stack, frame_scale)
    T, H, W = stack.shape
    dev = stack.device
    _check_search_inputs(stack, sigma, mask, frame_scale)
    if out is None:
        snr_max = torch.empty((H, W), dtype=torch.float32, device=dev)
        argmax = torch.empty((H, W), dtype=torch.int32, device=dev)
        snr_all = torch.empty((table.K, H, W), dtype=torch.float32, device=dev) if want_all else None
    else:
        snr_max, argmax, snr_all = out
        _check_search_outputs(snr_max, argmax, snr_all, table, H, W, dev)
    _check(load().mf_search_noalloc(ctypes.byref(st), _ptr(sigma), _ptr(mask), table.handle, _ptr(snr_max),
                                    _ptr(argmax), _ptr(snr_all), _stream_ptr(stream)))
    return snr_max, argmax, snr_all


def search_host_workspace_size(stack: torch.Tensor, table: PrfTable, k_top: int = 0) -> int:
    """mf_search_host_workspace_size for a host stack tensor."""
    st = make_stack(stack, None)
    n = ctypes.c_size_t()
    _check(load().mf_search_host_workspace_size(ctypes.byref(st), table.handle, int(k_top), ctypes.byref(n)))
    return n.value


def search_host(stack: torch.Tensor, sigma: torch.Tensor, table: PrfTable, mask: torch.Tensor | None = None,
                frame_scale: torch.Tensor | None = None, k_top: int = 0, workspace=None, out=None, stream=None,
                copy_stream=None, ws_free=None):
    """mf_search_host: the stack is a CPU tensor (pinned for asynchronous
    upload), sigma / mask / frame_scale live on the GPU; returns CPU tensors
    (snr_max [H, W], argmax [H, W], candidate records [k_top] uint8 or None,
    n_candidates [1] int32 or None), valid after the stream is synchronised.
    `out` may pass those four tensors (pinned) to reuse them.  copy_stream
    (torch.cuda.Stream) runs the upload apart from the kernels; ws_free
    (torch.cuda.Event) orders calls that reuse one workspace."""
    if stack.device.type != "cpu":
        raise ValueError("search_host takes a CPU stack; use search for device stacks")
    st = make_stack(stack, frame_scale)
    T, H, W = stack.shape
    _device_arg("sigma", sigma, optional=False)
    dev = sigma.device
    _check_search_inputs(stack, sigma, mask, frame_scale, device=dev)
    _device_arg("workspace", workspace, dev)
    if out is None:
        pin = stack.is_pinned()
        smax = torch.empty((H, W), dtype=torch.float32, pin_memory=pin)
        amax = torch.empty((H, W), dtype=torch.int32, pin_memory=pin)
        cand = torch.zeros((k_top, CANDIDATE_BYTES), dtype=torch.uint8, pin_memory=pin) if k_top else None
        ncand = torch.zeros(1, dtype=torch.int32, pin_memory=pin) if k_top else None
    else:
        smax, amax, cand, ncand = out
    ws = _workspace(search_host_workspace_size(stack, table, k_top), dev, workspace)
    if ws_free is not None and not ws_free.cuda_event:
        # torch creates the CUDA event on its first record: make it exist
        ws_free.record(stream if stream is not None else torch.cuda.current_stream())
    _check(load().mf_search_host(ctypes.byref(st), _ptr(sigma), _ptr(mask), table.handle, _ptr(smax), _ptr(amax),
                                 int(k_top), _ptr(cand), _ptr(ncand), _ptr(ws), ws.numel() * ws.element_size(),
                                 _stream_ptr(stream),
                                 None if copy_stream is None else ctypes.c_void_p(copy_stream.cuda_stream),
                                 None if ws_free is None else ctypes.c_void_p(ws_free.cuda_event)))
    return smax, amax, cand, ncand


def rescore_workspace_size(H, W, k_top) -> int:
    n = ctypes.c_size_t()
    _check(load().mf_rescore_workspace_size(int(H), int(W), int(k_top), ctypes.byref(n)))
    return n.value


def rescore_topk(master: torch.Tensor, sigma: torch.Tensor, table: PrfTable, snr_max: torch.Tensor,
                 argmax: torch.Tensor, k_top: int, mask: torch.Tensor | None = None,
                 frame_scale: torch.Tensor | None = None, workspace=None, stream=None):
    """mf_rescore_topk: returns (candidates as a uint8 tensor of k_top records, n_out int32 [1])."""
    st = make_stack(master, frame_scale)
    T, H, W = master.shape
    dev = master.device
    _check_search_inputs(master, sigma, mask, frame_scale)
    _device_arg("snr_max", snr_max, dev, torch.float32, (H, W), optional=False)
    _device_arg("argmax", argmax, dev, torch.int32, (H, W), optional=False)
    _device_arg("workspace", workspace, dev)
    out = torch.zeros((k_top, CANDIDATE_BYTES), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    nbytes = rescore_workspace_size(H, W, k_top)
    ws = _workspace(nbytes, dev, workspace)
    _check(load().mf_rescore_topk(ctypes.byref(st), _ptr(sigma), _ptr(mask), table.handle, _ptr(snr_max),
                                  _ptr(argmax), int(k_top), _ptr(out), _ptr(n_out), _ptr(ws),
                                  ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return out, n_out


def decode_candidates(raw: torch.Tensor, n: int):
    """Candidate records (uint8 tensor from rescore_topk) -> list of dicts."""
    import numpy as np
    buf = raw[:n].cpu().numpy().tobytes()
    dt = np.dtype([("y", "<i4"), ("x", "<i4"), ("k", "<i4"), ("r", "<i4"), ("snr", "<f8"),
                   ("flux", "<f8"), ("snr_search", "<f4"), ("r2", "<f4")])
    return np.frombuffer(buf, dtype=dt, count=n)


def refit_workspace_size(T: int) -> int:
    n = ctypes.c_size_t()
    _check(load().mf_refit_workspace_size(int(T), ctypes.byref(n)))
    return n.value


def background_refit(data: torch.Tensor, jitter, delta: float, iterations: int = 10,
                     scatter: torch.Tensor | None = None, resid: torch.Tensor | None = None, want_coef: bool = True,
                     workspace=None, stream=None):
    """mf_background_refit: data [T, H, W] float32 (device, contiguous),
    jitter [T, 2] (x, y) host array, scatter [T, n, n] float32 or None.
    Returns (residual [T, H, W], coefficients [H, W, 6] or None); pass
    resid=data to work in place."""
    import numpy as np
    if data.dim() != 3:
        raise ValueError("data must be [T, H, W]")
    T, H, W = data.shape
    _device_arg("data", data, dtype=torch.float32, optional=False)
    dev = data.device
    if scatter is not None:
        n_s = scatter.shape[-1] if scatter.dim() == 3 else 0
        _device_arg("scatter", scatter, dev, torch.float32, (T, n_s, n_s))
    _device_arg("resid", resid, dev, torch.float32, (T, H, W))
    _device_arg("workspace", workspace, dev)
    jt = np.ascontiguousarray(jitter, np.float64)
    if jt.shape != (T, 2):
        raise ValueError("jitter must have shape (T, 2)")
    if resid is None:
        resid = torch.empty_like(data)
    coef = torch.empty((H, W, 6), dtype=torch.float32, device=dev) if want_coef else None
    n = 0 if scatter is None else int(scatter.shape[-1])
    ws = _workspace(refit_workspace_size(T), dev, workspace)
    opts = RefitOpts(int(iterations), 0, float(delta))
    _check(load().mf_background_refit(_ptr(data), int(T), int(H), int(W), _ptr(scatter), n,
                                      jt.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts), _ptr(resid),
                                      _ptr(coef), _ptr(ws), ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return resid, coef


def detect_workspace_size(H: int, W: int, max_out: int) -> int:
    n = ctypes.c_size_t()
    _check(load().mf_detect_workspace_size(int(H), int(W), int(max_out), ctypes.byref(n)))
    return n.value


def detect(snr_max: torch.Tensor, argmax: torch.Tensor, window: int = 255, threshold: float = 3.0,
           subtract_mean: bool = True, max_out: int = 4096, z_out: torch.Tensor | None = None, workspace=None,
           stream=None):
    """mf_detect: returns (detections as a uint8 tensor of max_out records,
    n_out int32 [2] = (found, written)), both on the device."""
    if snr_max.dim() != 2:
        raise ValueError("snr_max must be [H, W]")
    H, W = snr_max.shape
    _device_arg("snr_max", snr_max, dtype=torch.float32, optional=False)
    dev = snr_max.device
    _device_arg("argmax", argmax, dev, torch.int32, (H, W), optional=False)
    _device_arg("z_out", z_out, dev, torch.float32, (H, W))
    _device_arg("workspace", workspace, dev)
    out = torch.zeros((max(max_out, 1), DETECTION_BYTES), dtype=torch.uint8, device=dev)
    n_out = torch.zeros(2, dtype=torch.int32, device=dev)
    ws = _workspace(detect_workspace_size(H, W, max_out), dev, workspace)
    opts = DetectOpts(int(window), 1 if subtract_mean else 0, float(threshold))
    _check(load().mf_detect(_ptr(snr_max), _ptr(argmax), int(H), int(W), ctypes.byref(opts), _ptr(z_out),
                            _ptr(out), int(max_out), _ptr(n_out), _ptr(ws), ws.numel() * ws.element_size(),
                            _stream_ptr(stream)))
    return out, n_out


def decode_detections(raw: torch.Tensor, n: int):
    """Detection records (uint8 tensor from detect) -> numpy structured array."""
    import numpy as np
    buf = raw[:n].cpu().numpy().tobytes()
    dt = np.dtype([("y", "<i4"), ("x", "<i4"), ("k", "<i4"), ("npix", "<i4"), ("z", "<f8"), ("mean", "<f8"),
                   ("sigma", "<f8"), ("snr", "<f4"), ("reserved", "<i4")])
    return np.frombuffer(buf, dtype=dt, count=n)


def profile_enable(on: bool = True):
    _check(load().mf_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    """{kernel name: (launches, summed device ms)} plus '_launches' total."""
    p = Profile()
    _check(load().mf_profile_read(ctypes.byref(p), 1 if reset else 0))
    out = {p.k[i].name.decode(): (int(p.k[i].launches), float(p.k[i].ms)) for i in range(p.n)}
    out["_launches"] = int(p.launches)
    return out


class Batch:
    """mf_batch: many searches captured into one CUDA graph with a persistent
    numerator launch.  Keeps every tensor it was given alive."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().mf_batch_create(ctypes.byref(h)))
        self._h = h
        self._keep = []
        self.outputs = []
        self._ws = None

    def add(self, stack, sigma, table, mask=None, frame_scale=None, want_all=False):
        st = make_stack(stack, frame_scale)
        T, H, W = stack.shape
        dev = stack.device
        _check_search_inputs(stack, sigma, mask, frame_scale)
        snr_max = torch.empty((H, W), dtype=torch.float32, device=dev)
        argmax = torch.empty((H, W), dtype=torch.int32, device=dev)
        snr_all = torch.empty((table.K, H, W), dtype=torch.float32, device=dev) if want_all else None
        idx = ctypes.c_int32()
        _check(load().mf_batch_add(self._h, ctypes.byref(st), _ptr(sigma), _ptr(mask), table.handle,
                                   _ptr(snr_max), _ptr(argmax), _ptr(snr_all), ctypes.byref(idx)))
        self._keep += [stack, sigma, mask, frame_scale, table]
        self.outputs.append((snr_max, argmax, snr_all))
        return idx.value

    def workspace_size(self) -> int:
        n = ctypes.c_size_t()
        _check(load().mf_batch_workspace_size(self._h, ctypes.byref(n)))
        return n.value

    def prepare(self, workspace=None, device="cuda"):
        n = self.workspace_size()
        _device_arg("workspace", workspace)
        self._ws = workspace if workspace is not None else torch.empty(max(n, 1), dtype=torch.uint8, device=device)
        _check(load().mf_batch_prepare(self._h, _ptr(self._ws), self._ws.numel() * self._ws.element_size()))

    def run(self, stream=None):
        _check(load().mf_batch_run(self._h, _stream_ptr(stream)))

    def poll(self) -> bool:
        """True once the latest run has finished on the device (mf_batch_poll)."""
        d = ctypes.c_int32()
        _check(load().mf_batch_poll(self._h, ctypes.byref(d)))
        return bool(d.value)

    def info(self) -> dict:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().mf_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"items": a.value, "shape_groups": b.value, "graph_ready": bool(c.value)}

    def destroy(self):
        if self._h:
            load().mf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def device_status() -> int:
    """mf_device_status: synchronise, then read and clear the device status
    word (0, or MF_ETIMEOUT with the wait's code in last_error())."""
    return load().mf_device_status()


def wait_probe(stream=None):
    """mf_wait_probe: one CTA whose bounded wait runs out (about a second);
    the next device_status() returns MF_ETIMEOUT and clears the word."""
    _check(load().mf_wait_probe(_stream_ptr(stream)))


def wait_probe_search(workspace: torch.Tensor, stream=None):
    """mf_wait_probe_search: a bounded wait that runs out and records its code
    (4) in the status slot of this search workspace (and the device word)."""
    _device_arg("workspace", workspace, optional=False)
    _check(load().mf_wait_probe_search(_ptr(workspace), _stream_ptr(stream)))


def search_status(workspace: torch.Tensor, out: torch.Tensor, stream=None):
    """mf_search_status: enqueue a copy of the search's status slot (at the
    start of `workspace`) into `out`, an int32 tensor of one element (pinned
    host memory or device memory).  Nonzero once the copy has run: a bounded
    wait of that search gave up (MF_ETIMEOUT)."""
    _device_arg("workspace", workspace, optional=False)
    if out.dtype != torch.int32 or out.numel() < 1 or not out.is_contiguous():
        raise ValueError("out must be a contiguous int32 tensor with at least one element")
    if not out.is_cuda and not out.is_pinned():
        raise ValueError("a host `out` must be pinned memory")
    _check(load().mf_search_status(_ptr(workspace), _ptr(out), _stream_ptr(stream)))
