"""Thin ctypes binding of libconvtune.so (C ABI in include/convtune.h).

Argument marshalling only: every step of the compute path runs in the
library's CUDA kernels.  Device buffers are anything with ``data_ptr()``
(torch tensors), streams are ``torch.cuda.Stream`` objects or raw handles.
If the library has not been built, every call raises -- there is no CPU or
PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

c_int, c_long, c_double, c_void_p = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p

# status codes (include/convtune.h)
CT_OK, CT_EINVAL, CT_ENOTSUP, CT_EPERM, CT_ECUDA, CT_ENOMEM, CT_ETIMEOUT, CT_ECONFIG, CT_EIO = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STAGE_DIRECT, STAGE_SMEM, STAGE_TMA = 0, 1, 2
FILTER_SHARED, FILTER_CONST = 0, 1


class CtConfig(ctypes.Structure):
    _fields_ = [("block_x", c_int), ("block_y", c_int), ("tile_x", c_int), ("tile_y", c_int),
                ("staging", c_int), ("filter_mem", c_int), ("vec_width", c_int)]


class CtProblem(ctypes.Structure):
    _fields_ = [("in_", c_void_p), ("in_pitch", c_long), ("filt", c_void_p), ("fh", c_int),
                ("fw", c_int), ("out", c_void_p), ("out_pitch", c_long), ("out_h", c_int),
                ("out_w", c_int)]


class CtDeviceInfo(ctypes.Structure):
    _fields_ = [("sm_count", c_int), ("cc_major", c_int), ("cc_minor", c_int),
                ("max_smem_optin_bytes", c_int), ("l2_bytes", c_int),
                ("sm_clock_max_mhz", c_double), ("name", ctypes.c_char * 96)]


class ConvTuneError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


@dataclasses.dataclass(frozen=True)
class Config:
    """One point of the tuning space (see ct_config)."""
    block_x: int = 32
    block_y: int = 8
    tile_x: int = 4
    tile_y: int = 4
    staging: int = STAGE_SMEM
    filter_mem: int = FILTER_CONST
    vec_width: int = 4

    def to_c(self) -> CtConfig:
        return CtConfig(*dataclasses.astuple(self))

    @classmethod
    def from_c(cls, c: CtConfig) -> "Config":
        return cls(c.block_x, c.block_y, c.tile_x, c.tile_y, c.staging, c.filter_mem, c.vec_width)

    def as_tuple(self):
        return dataclasses.astuple(self)


_lock = threading.Lock()
_lib = None

_SIGS = {
    "ct_strerror": (ctypes.c_char_p, [c_int]),
    "ct_version": (ctypes.c_char_p, []),
    "ct_conv2d_check": (c_int, [c_void_p, c_void_p, ctypes.c_char_p, c_int]),
    "ct_conv2d_run": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ct_conv2d_run_host": (c_int, [c_void_p, c_long, c_void_p, c_int, c_int, c_void_p, c_long,
                                   c_int, c_int, c_void_p, c_void_p]),
    "ct_status_read": (c_int, [ctypes.POINTER(ctypes.c_uint), c_int]),
    "ct_device_info_get": (c_int, [c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(
                    "libconvtune.so is not built (python -m paper_2211_07260_gb300.build); "
                    "there is no fallback implementation")
            h = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().ct_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def version() -> str:
    return lib().ct_version().decode()


def _check(rc: int, what: str):
    if rc != CT_OK:
        raise ConvTuneError(rc, what)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def stream_handle(stream) -> int:
    """cudaStream_t of a torch stream (or the value itself if it is an int)."""
    if stream is None:
        try:
            import torch
            return int(torch.cuda.current_stream().cuda_stream)
        except Exception:  # no torch / no CUDA: legacy default stream
            return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _taps(filt) -> np.ndarray:
    if hasattr(filt, "detach"):
        filt = filt.detach().cpu().numpy()
    f = np.ascontiguousarray(filt, dtype=np.float32)
    if f.ndim != 2:
        raise ValueError("filter must be 2-D")
    return f


def make_problem(inp, filt, out, out_h: int, out_w: int, in_pitch: int | None = None,
                 out_pitch: int | None = None):
    """CtProblem for device buffers ``inp`` / ``out`` and a host filter.

    Pitches default to the tensors' row strides.  Returns (problem, taps);
    keep ``taps`` alive until the call that uses the problem returns.
    """
    f = _taps(filt)
    if in_pitch is None:
        in_pitch = int(inp.stride(0))
    if out_pitch is None:
        out_pitch = int(out.stride(0))
    p = CtProblem(_ptr(inp), int(in_pitch), f.ctypes.data, f.shape[0], f.shape[1], _ptr(out),
                  int(out_pitch), int(out_h), int(out_w))
    return p, f


def conv2d_check(inp, filt, out, out_h, out_w, cfg: Config, in_pitch=None, out_pitch=None):
    """(status, reason) of ct_conv2d_check."""
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    c = cfg.to_c()
    why = ctypes.create_string_buffer(256)
    rc = lib().ct_conv2d_check(ctypes.byref(p), ctypes.byref(c), why, 256)
    return rc, why.value.decode()


def conv2d_run(inp, filt, out, out_h, out_w, cfg: Config, stream=None, in_pitch=None,
               out_pitch=None):
    """Launch the correlation on device buffers (asynchronous)."""
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    c = cfg.to_c()
    _check(lib().ct_conv2d_run(ctypes.byref(p), ctypes.byref(c), c_void_p(stream_handle(stream))),
           "ct_conv2d_run")


def conv2d_run_host(inp: np.ndarray, filt, out: np.ndarray, out_h: int, out_w: int, cfg: Config,
                    stream=None):
    """The correlation on host arrays (copies in and out inside the call)."""
    if inp.dtype != np.float32 or out.dtype != np.float32:
        raise TypeError("float32 arrays required")
    if not (inp.flags.c_contiguous and out.flags.c_contiguous):
        raise ValueError("contiguous arrays required")
    f = _taps(filt)
    c = cfg.to_c()
    _check(lib().ct_conv2d_run_host(inp.ctypes.data, inp.shape[1], f.ctypes.data, f.shape[0],
                                    f.shape[1], out.ctypes.data, out.shape[1], int(out_h),
                                    int(out_w), ctypes.byref(c), c_void_p(stream_handle(stream))),
           "ct_conv2d_run_host")


def status_read(clear: bool = False) -> int:
    bits = ctypes.c_uint(0)
    _check(lib().ct_status_read(ctypes.byref(bits), int(bool(clear))), "ct_status_read")
    return int(bits.value)


def device_info() -> dict:
    d = CtDeviceInfo()
    _check(lib().ct_device_info_get(ctypes.byref(d)), "ct_device_info_get")
    return dict(sm_count=d.sm_count, cc=(d.cc_major, d.cc_minor),
                max_smem_optin_bytes=d.max_smem_optin_bytes, l2_bytes=d.l2_bytes,
                sm_clock_max_mhz=d.sm_clock_max_mhz, name=d.name.decode())
