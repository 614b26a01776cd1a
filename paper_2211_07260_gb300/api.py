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


CT_UNIT_CONV, CT_UNIT_FMA, CT_UNIT_COPY = 0, 1, 2
CT_THR_SW_POWER_CAP, CT_THR_HW_SLOWDOWN, CT_THR_SW_THERMAL, CT_THR_HW_THERMAL = 0x4, 0x8, 0x20, 0x40
CT_STEER_UNION = 3
CT_OBJ_TIME, CT_OBJ_ENERGY, CT_OBJ_GFLOPS_PER_W = 0, 1, 2
CT_SPACE_BASIC, CT_SPACE_FULL = 0, 1
REC_THROTTLED, REC_COTENANT, REC_DEFAULT_CLOCKS, REC_INVALID, REC_CACHED, REC_NO_ENERGY, \
    REC_IDLE_GAPS = 1, 2, 4, 8, 16, 32, 64
OBJECTIVES = {"time": CT_OBJ_TIME, "energy": CT_OBJ_ENERGY, "gflops_per_w": CT_OBJ_GFLOPS_PER_W}

c_uint, c_ulonglong = ctypes.c_uint, ctypes.c_ulonglong
_FN_ULL = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_ulonglong))
_FN_UINT = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_uint))
_FN_INTP = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_int))
_FN_CLOCKS = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int))
_FN_LOCK = ctypes.CFUNCTYPE(c_int, c_void_p, c_int)
_FN_RESET = ctypes.CFUNCTYPE(c_int, c_void_p)
_FN_NOW = ctypes.CFUNCTYPE(c_double, c_void_p)
_FN_PLRANGE = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                               ctypes.POINTER(c_int))
_FN_RUN = ctypes.CFUNCTYPE(c_int, c_void_p, c_int, ctypes.POINTER(CtConfig), c_int,
                           ctypes.POINTER(c_double))


class CtPlatformOps(ctypes.Structure):
    _fields_ = [("ctx", c_void_p), ("energy_mj", _FN_ULL), ("power_mw", _FN_UINT),
                ("sm_clock_mhz", _FN_UINT), ("throttle_reasons", _FN_ULL),
                ("temperature_c", _FN_UINT), ("other_processes", _FN_INTP),
                ("supported_sm_clocks", _FN_CLOCKS), ("lock_sm_clock", _FN_LOCK),
                ("reset_sm_clock", _FN_RESET), ("now_s", _FN_NOW), ("run_launches", _FN_RUN),
                ("set_power_limit", _FN_LOCK), ("reset_power_limit", _FN_RESET),
                ("power_limit_range", _FN_PLRANGE)]


class CtMeasureOptions(ctypes.Structure):
    _fields_ = [("window_s", c_double), ("warmup_s", c_double), ("graph_ms", c_double),
                ("time_only", c_int), ("time_reps", c_int)]


class CtRecord(ctypes.Structure):
    _fields_ = [("cfg", CtConfig), ("clock_mhz_req", c_int), ("clock_mhz_meas", c_double),
                ("t_s", c_double), ("energy_j", c_double), ("power_w_mean", c_double),
                ("power_w_median", c_double), ("energy_j_median_power", c_double),
                ("gflops", c_double), ("gflops_per_j", c_double), ("temp_c", c_double),
                ("wall_s", c_double), ("n_launches", c_int), ("flags", c_int),
                ("power_limit_w", c_double)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "cfg"}
        d["cfg"] = Config.from_c(self.cfg).as_tuple()
        return d


class CtPowerModel(ctypes.Structure):
    _fields_ = [("p_idle_w", c_double), ("alpha", c_double), ("beta", c_double),
                ("tau_mhz", c_double), ("p_max_w", c_double), ("has_voltage", c_int),
                ("sse", c_double), ("n_used", c_int), ("f_lo_mhz", c_double),
                ("f_thr_mhz", c_double), ("f_opt_mhz", c_double)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "CtPowerModel":
        m = cls()
        for k, _ in cls._fields_:
            if k in d:
                setattr(m, k, d[k])
        return m


class CtTuneOptions(ctypes.Structure):
    _fields_ = [("objective", c_int), ("measure", CtMeasureOptions), ("cache_path", ctypes.c_char_p),
                ("settle_s", c_double), ("fallback_default_clocks", c_int)]


class CtTimeModel(ctypes.Structure):
    _fields_ = [("t_mem_s", c_double), ("c_core_s_ghz", c_double), ("sse", c_double),
                ("n_used", c_int), ("f_lo_mhz", c_double), ("f_thr_mhz", c_double)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "CtTimeModel":
        m = cls()
        for k, _ in cls._fields_:
            setattr(m, k, d[k])
        return m


class CtSteerResult(ctypes.Structure):
    _fields_ = [("model", CtPowerModel), ("center_mhz", c_double), ("n_range", c_int),
                ("fit_wall_s", c_double), ("tune_wall_s", c_double),
                ("model_mem", CtPowerModel), ("time_mem", CtTimeModel),
                ("center_mem_mhz", c_double), ("n_range_compute", c_int),
                ("n_range_memory", c_int)]


class ConvTuneError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = ""
        if status == CT_ECUDA:
            try:
                detail = " [" + lib().ct_last_error().decode() + "]"
            except RuntimeError:
                pass
        super().__init__(f"{what}: {strerror(status)} ({status}){detail}")


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
    "ct_last_error": (ctypes.c_char_p, []),
    "ct_conv2d_check": (c_int, [c_void_p, c_void_p, ctypes.c_char_p, c_int]),
    "ct_conv2d_run": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ct_conv2d_run_host": (c_int, [c_void_p, c_long, c_void_p, c_int, c_int, c_void_p, c_long,
                                   c_int, c_int, c_void_p, c_void_p]),
    "ct_conv2d_run_host_async": (c_int, [c_void_p, c_long, c_void_p, c_int, c_int, c_void_p,
                                         c_long, c_int, c_int, c_void_p]),
    "ct_conv2d_host_wait": (c_int, []),
    "ct_conv2d_run_host_bands": (c_int, [c_void_p, c_long, c_void_p, c_int, c_int, c_void_p, c_long,
                                         c_int, c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "ct_conv2d_host_bands_default": (c_int, [c_int, c_void_p, c_int, c_void_p]),
    "ct_status_read": (c_int, [ctypes.POINTER(ctypes.c_uint), c_int]),
    "ct_device_info_get": (c_int, [c_void_p]),
    "ct_set_platform_ops": (c_int, [c_void_p]),
    "ct_nvml_status": (c_int, []),
    "ct_supported_sm_clocks": (c_int, [c_void_p, c_int, c_void_p]),
    "ct_lock_sm_clock": (c_int, [c_int]),
    "ct_reset_sm_clock": (c_int, []),
    "ct_measure_conv": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ct_fit_power_model": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double,
                                   c_void_p]),
    "ct_model_power": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "ct_optimal_clock": (c_int, [c_void_p, c_void_p]),
    "ct_fit_time_model": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "ct_model_time": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "ct_memory_aware_optimum": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ct_clock_range": (c_int, [c_double, c_void_p, c_int, c_double, c_void_p, c_int, c_void_p]),
    "ct_pick_clock_range": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_int,
                                    c_void_p, c_void_p]),
    "ct_space": (c_int, [c_int, c_void_p, c_int, c_void_p]),
    "ct_tune": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                        c_int, c_void_p, c_void_p]),
    "ct_tune_power_limits": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p,
                                     c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "ct_power_limit_range": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ct_select_best": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_void_p]),
    "ct_microbench_launch": (c_int, [c_int, c_void_p, c_void_p]),
    "ct_measure_microbench": (c_int, [c_int, c_void_p, c_void_p, c_void_p]),
    "ct_measure_power_samples": (c_int, [c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p]),
    "ct_microbench_release": (c_int, []),
    "ct_batch_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "ct_batch_run": (c_int, [c_void_p, c_void_p]),
    "ct_batch_run_plain": (c_int, [c_void_p, c_void_p]),
    "ct_batch_run_mode": (c_int, [c_void_p, c_int, c_void_p]),
    "ct_batch_info": (c_int, [c_void_p, c_void_p]),
    "ct_batch_destroy": (c_int, [c_void_p]),
    "ct_measure_batch": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ct_batch_tune": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_int, c_void_p]),
    "ct_batch_tune_launches": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_int, c_void_p]),
    "ct_batch_run_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "ct_batch_noalloc_status": (c_int, [c_void_p, c_int, c_void_p]),
    "ct_server_create": (c_int, [c_void_p, c_void_p]),
    "ct_server_submit": (c_int, [c_void_p, c_void_p, c_long, c_void_p, c_int, c_void_p, c_long,
                                 c_int, c_int, c_void_p]),
    "ct_server_wait": (c_int, [c_void_p, ctypes.c_longlong, c_double, c_void_p]),
    "ct_server_drain": (c_int, [c_void_p, c_double]),
    "ct_server_stats_get": (c_int, [c_void_p, c_int, c_void_p]),
    "ct_server_destroy": (c_int, [c_void_p]),
    "ct_server_trace_get": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "ct_read_sensors": (c_int, [c_void_p]),
    "ct_tuning_methods": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "ct_pareto_front": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p]),
    "ct_centrality": (c_int, [c_void_p, c_int, c_int, c_double, c_void_p, c_int, c_void_p]),
    "ct_selftest_wait_timeout": (c_int, [ctypes.c_uint, c_void_p]),
    "ct_tune_steered": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                                c_double, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                c_void_p, c_int, c_void_p, c_void_p]),
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
                    stream=None, bands=None):
    """The correlation on host arrays (copies in and out inside the call).

    ``bands``: optional output-row counts of the pipelined row bands (their
    sum is out_h); None takes the library's default split."""
    if inp.dtype != np.float32 or out.dtype != np.float32:
        raise TypeError("float32 arrays required")
    if not (inp.flags.c_contiguous and out.flags.c_contiguous):
        raise ValueError("contiguous arrays required")
    f = _taps(filt)
    c = cfg.to_c()
    args = (inp.ctypes.data, inp.shape[1], f.ctypes.data, f.shape[0], f.shape[1],
            out.ctypes.data, out.shape[1], int(out_h), int(out_w), ctypes.byref(c))
    if bands is None:
        _check(lib().ct_conv2d_run_host(*args, c_void_p(stream_handle(stream))),
               "ct_conv2d_run_host")
        return
    rows = np.ascontiguousarray(bands, dtype=np.int32)
    _check(lib().ct_conv2d_run_host_bands(*args, rows.ctypes.data, int(rows.size),
                                          c_void_p(stream_handle(stream))),
           "ct_conv2d_run_host_bands")


def conv2d_run_host_async(inp: np.ndarray, filt, out: np.ndarray, out_h: int, out_w: int,
                          cfg: Config):
    """ct_conv2d_run_host_async: enqueue the host-buffer correlation (after
    the earlier host-buffer calls) and return.  Keep `inp` and `out` alive,
    `inp` unmodified and `out` unread, until host_wait() returns."""
    if inp.dtype != np.float32 or out.dtype != np.float32:
        raise TypeError("float32 arrays required")
    if not (inp.flags.c_contiguous and out.flags.c_contiguous):
        raise ValueError("contiguous arrays required")
    f = _taps(filt)
    c = cfg.to_c()
    _check(lib().ct_conv2d_run_host_async(inp.ctypes.data, inp.shape[1], f.ctypes.data,
                                          f.shape[0], f.shape[1], out.ctypes.data, out.shape[1],
                                          int(out_h), int(out_w), ctypes.byref(c)),
           "ct_conv2d_run_host_async")


def host_wait():
    """ct_conv2d_host_wait: every earlier conv2d_run_host_async output is on
    the host when this returns."""
    _check(lib().ct_conv2d_host_wait(), "ct_conv2d_host_wait")


def host_bands_default(out_h: int) -> list:
    """The library's default row-band split for out_h output rows."""
    buf = np.zeros(64, np.int32)
    n = c_int(0)
    _check(lib().ct_conv2d_host_bands_default(int(out_h), buf.ctypes.data, 64, ctypes.byref(n)),
           "ct_conv2d_host_bands_default")
    return buf[:n.value].tolist()


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


# ---- platform ---------------------------------------------------------------
_platform_keepalive = None


def set_platform_ops(ops: "CtPlatformOps | None"):
    """Install a platform table (None restores NVML).  The Python callbacks
    are kept alive until the next call."""
    global _platform_keepalive
    _check(lib().ct_set_platform_ops(ctypes.byref(ops) if ops is not None else None),
           "ct_set_platform_ops")
    _platform_keepalive = ops


class CtSensors(ctypes.Structure):
    _fields_ = [("energy_j", c_double), ("power_w", c_double), ("sm_clock_mhz", c_double),
                ("temp_c", c_double), ("throttle_reasons", ctypes.c_ulonglong),
                ("other_processes", c_int)]


def read_sensors() -> dict:
    s = CtSensors()
    _check(lib().ct_read_sensors(ctypes.byref(s)), "ct_read_sensors")
    return {k: getattr(s, k) for k, _ in CtSensors._fields_}


def nvml_status() -> int:
    return int(lib().ct_nvml_status())


def supported_sm_clocks() -> list:
    buf = (c_int * 1024)()
    n = c_int(0)
    _check(lib().ct_supported_sm_clocks(buf, 1024, ctypes.byref(n)), "ct_supported_sm_clocks")
    return [buf[i] for i in range(n.value)]


def measure_options(window_s=1.0, warmup_s=0.2, graph_ms=2.0, time_only=False, time_reps=5):
    return CtMeasureOptions(window_s, warmup_s, graph_ms, int(bool(time_only)), time_reps)


def measure_conv(inp, filt, out, out_h, out_w, cfg: Config, opts=None, stream=None,
                 in_pitch=None, out_pitch=None):
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    c = cfg.to_c()
    r = CtRecord()
    o = opts or measure_options()
    _check(lib().ct_measure_conv(ctypes.byref(p), ctypes.byref(c), ctypes.byref(o),
                                 c_void_p(stream_handle(stream)), ctypes.byref(r)),
           "ct_measure_conv")
    return r.to_dict()


# ---- power model ------------------------------------------------------------
def _darr(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data


def fit_power_model(f_mhz, p_w, v=None, throttled=None, p_max_w=0.0) -> dict:
    f, fp = _darr(f_mhz)
    p, pp = _darr(p_w)
    vv, vp = _darr(v) if v is not None else (None, None)
    t = np.ascontiguousarray(throttled, dtype=np.int32) if throttled is not None else None
    m = CtPowerModel()
    _check(lib().ct_fit_power_model(fp, pp, vp, t.ctypes.data if t is not None else None, f.size,
                                    float(p_max_w or 0.0), ctypes.byref(m)), "ct_fit_power_model")
    return m.to_dict()


def model_power(model: dict, f_mhz):
    f, fp = _darr(f_mhz)
    out = np.empty_like(f)
    m = CtPowerModel.from_dict(model)
    _check(lib().ct_model_power(ctypes.byref(m), fp, f.size, out.ctypes.data), "ct_model_power")
    return out


def optimal_clock(model: dict) -> float:
    m = CtPowerModel.from_dict(model)
    v = c_double(0)
    _check(lib().ct_optimal_clock(ctypes.byref(m), ctypes.byref(v)), "ct_optimal_clock")
    return v.value


def pick_clock_range(model: dict, supported_mhz, rel_halfwidth=0.10, center="optimum"):
    sup = np.ascontiguousarray(supported_mhz, dtype=np.int32)
    out = np.zeros(max(1, sup.size), dtype=np.int32)
    n = c_int(0)
    c0 = c_double(0)
    m = CtPowerModel.from_dict(model)
    _check(lib().ct_pick_clock_range(ctypes.byref(m), sup.ctypes.data, sup.size,
                                     float(rel_halfwidth), 1 if center == "ridge" else 0,
                                     out.ctypes.data, out.size, ctypes.byref(n),
                                     ctypes.byref(c0)), "ct_pick_clock_range")
    return [int(x) for x in out[:n.value]], c0.value


# ---- memory-aware energy model ----------------------------------------------
def fit_time_model(f_mhz, t_s, throttled=None) -> dict:
    """t(f) = t_mem + c_core / f by non-negative least squares (ct_fit_time_model)."""
    f, fp = _darr(f_mhz)
    t, tp = _darr(t_s)
    if f.shape != t.shape:
        raise ValueError("f and t differ in length")
    th = np.ascontiguousarray(throttled, dtype=np.int32) if throttled is not None else None
    m = CtTimeModel()
    _check(lib().ct_fit_time_model(fp, tp, th.ctypes.data if th is not None else None, f.size,
                                   ctypes.byref(m)), "ct_fit_time_model")
    return m.to_dict()


def model_time(tm: dict, f_mhz):
    f, fp = _darr(f_mhz)
    out = np.empty_like(f)
    m = CtTimeModel.from_dict(tm)
    _check(lib().ct_model_time(ctypes.byref(m), fp, f.size, out.ctypes.data), "ct_model_time")
    return out


def memory_aware_optimum(pm: dict, tm: dict):
    """(f_opt_mhz, E there) of P*(f) t(f) (ct_memory_aware_optimum)."""
    p = CtPowerModel.from_dict(pm)
    t = CtTimeModel.from_dict(tm)
    f, e = c_double(0), c_double(0)
    _check(lib().ct_memory_aware_optimum(ctypes.byref(p), ctypes.byref(t), ctypes.byref(f),
                                         ctypes.byref(e)), "ct_memory_aware_optimum")
    return f.value, e.value


def clock_range(center_mhz, supported_mhz, rel_halfwidth=0.10):
    sup = np.ascontiguousarray(supported_mhz, dtype=np.int32)
    out = np.zeros(max(1, sup.size), dtype=np.int32)
    n = c_int(0)
    _check(lib().ct_clock_range(float(center_mhz), sup.ctypes.data, sup.size,
                                float(rel_halfwidth), out.ctypes.data, out.size, ctypes.byref(n)),
           "ct_clock_range")
    return [int(x) for x in out[:n.value]]


# ---- tuning -----------------------------------------------------------------
def space(which=CT_SPACE_BASIC) -> list:
    n = c_int(0)
    lib().ct_space(which, None, 0, ctypes.byref(n))
    buf = (CtConfig * n.value)()
    _check(lib().ct_space(which, buf, n.value, ctypes.byref(n)), "ct_space")
    return [Config.from_c(buf[i]) for i in range(n.value)]


def tune_options(objective="energy", window_s=1.0, warmup_s=0.2, graph_ms=2.0, time_only=False,
                 cache_path=None, settle_s=0.0, fallback_default_clocks=True):
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    return CtTuneOptions(obj, measure_options(window_s, warmup_s, graph_ms, time_only),
                         cache_path.encode() if cache_path else None, settle_s,
                         int(bool(fallback_default_clocks)))


def _space_array(cfgs):
    if cfgs is None:
        return None, 0
    arr = (CtConfig * len(cfgs))(*[c.to_c() for c in cfgs])
    return arr, len(cfgs)


def tune(inp, filt, out, out_h, out_w, cfgs=None, clocks=None, opts=None, stream=None,
         in_pitch=None, out_pitch=None):
    """Exhaustive search (ct_tune).  Returns (records, best_index)."""
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    sp, ns = _space_array(cfgs)
    ck = np.ascontiguousarray(clocks if clocks is not None else [], dtype=np.int32)
    o = opts or tune_options()
    n_space = ns if sp is not None else len(space(CT_SPACE_BASIC))
    cap = n_space * max(1, ck.size)
    recs = (CtRecord * cap)()
    n = c_int(0)
    best = c_int(-1)
    _check(lib().ct_tune(ctypes.byref(p), sp, ns, ck.ctypes.data if ck.size else None, ck.size,
                         ctypes.byref(o), c_void_p(stream_handle(stream)), recs, cap,
                         ctypes.byref(n), ctypes.byref(best)), "ct_tune")
    return [recs[i].to_dict() for i in range(n.value)], best.value


def tune_power_limits(inp, filt, out, out_h, out_w, limits_w, cfgs=None, opts=None, stream=None,
                      in_pitch=None, out_pitch=None):
    """Exhaustive search over configurations x board power limits in watts
    (ct_tune_power_limits).  Returns (records, best_index)."""
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    sp, ns = _space_array(cfgs)
    lim = np.ascontiguousarray([int(round(w * 1000)) for w in limits_w], dtype=np.int32)
    o = opts or tune_options()
    n_space = ns if sp is not None else len(space(CT_SPACE_BASIC))
    cap = n_space * max(1, lim.size)
    recs = (CtRecord * cap)()
    n = c_int(0)
    best = c_int(-1)
    _check(lib().ct_tune_power_limits(ctypes.byref(p), sp, ns,
                                      lim.ctypes.data if lim.size else None, lim.size,
                                      ctypes.byref(o), c_void_p(stream_handle(stream)), recs, cap,
                                      ctypes.byref(n), ctypes.byref(best)), "ct_tune_power_limits")
    return [recs[i].to_dict() for i in range(n.value)], best.value


def power_limit_range():
    """(min, max, default) board power limit in watts."""
    lo, hi, de = c_int(0), c_int(0), c_int(0)
    _check(lib().ct_power_limit_range(ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(de)),
           "ct_power_limit_range")
    return lo.value / 1000.0, hi.value / 1000.0, de.value / 1000.0


def select_best(records, objective="energy", clocks=None) -> int:
    arr = (CtRecord * len(records))()
    for i, r in enumerate(records):
        for k, _ in CtRecord._fields_:
            if k == "cfg":
                arr[i].cfg = Config(*r["cfg"]).to_c()
            else:
                setattr(arr[i], k, r.get(k, 0))
    ck = np.ascontiguousarray(clocks if clocks is not None else [], dtype=np.int32)
    best = c_int(-1)
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    _check(lib().ct_select_best(arr, len(records), obj, ck.ctypes.data if ck.size else None,
                                ck.size, ctypes.byref(best)), "ct_select_best")
    return best.value


def microbench_launch(which: int, stream=None) -> float:
    w = c_double(0)
    _check(lib().ct_microbench_launch(which, c_void_p(stream_handle(stream)), ctypes.byref(w)),
           "ct_microbench_launch")
    return w.value


def measure_microbench(which: int, opts=None, stream=None) -> dict:
    r = CtRecord()
    o = opts or measure_options()
    _check(lib().ct_measure_microbench(which, ctypes.byref(o), c_void_p(stream_handle(stream)),
                                       ctypes.byref(r)), "ct_measure_microbench")
    return r.to_dict()


def measure_power_samples(which: int, clocks=None, opts=None, stream=None):
    ck = np.ascontiguousarray(clocks if clocks is not None else [], dtype=np.int32)
    n = max(1, ck.size)
    f = np.zeros(n)
    p = np.zeros(n)
    t = np.zeros(n, dtype=np.int32)
    recs = (CtRecord * n)()
    o = opts or measure_options()
    _check(lib().ct_measure_power_samples(which, ck.ctypes.data if ck.size else None, ck.size,
                                          ctypes.byref(o), c_void_p(stream_handle(stream)),
                                          f.ctypes.data, p.ctypes.data, t.ctypes.data, recs),
           "ct_measure_power_samples")
    return f, p, t.astype(bool), [r.to_dict() for r in recs]


def tune_steered(inp, filt, out, out_h, out_w, fit_clocks, cfgs=None, supported=None,
                 rel_halfwidth=0.10, which_bench=CT_UNIT_FMA, opts=None, stream=None,
                 in_pitch=None, out_pitch=None):
    """Model-steered search (ct_tune_steered).  Returns (result, range,
    records, best_index)."""
    p, f = make_problem(inp, filt, out, out_h, out_w, in_pitch, out_pitch)
    sp, ns = _space_array(cfgs)
    fc = np.ascontiguousarray(fit_clocks, dtype=np.int32)
    su = np.ascontiguousarray(supported if supported is not None else [], dtype=np.int32)
    n_space = ns if sp is not None else len(space(CT_SPACE_BASIC))
    rng = np.zeros(1024, dtype=np.int32)
    cap = n_space * 1024
    recs = (CtRecord * cap)()
    res = CtSteerResult()
    n = c_int(0)
    best = c_int(-1)
    o = opts or tune_options()
    _check(lib().ct_tune_steered(ctypes.byref(p), sp, ns, fc.ctypes.data, fc.size,
                                 su.ctypes.data if su.size else None, su.size,
                                 float(rel_halfwidth), which_bench, ctypes.byref(o),
                                 c_void_p(stream_handle(stream)), ctypes.byref(res),
                                 rng.ctypes.data, rng.size, recs, cap, ctypes.byref(n),
                                 ctypes.byref(best)), "ct_tune_steered")
    result = dict(model=res.model.to_dict(), center_mhz=res.center_mhz, n_range=res.n_range,
                  fit_wall_s=res.fit_wall_s, tune_wall_s=res.tune_wall_s,
                  model_mem=res.model_mem.to_dict(), time_mem=res.time_mem.to_dict(),
                  center_mem_mhz=res.center_mem_mhz, n_range_compute=res.n_range_compute,
                  n_range_memory=res.n_range_memory)
    return result, [int(x) for x in rng[:res.n_range]], \
        [recs[i].to_dict() for i in range(n.value)], best.value


# ---- persistent batched correlation ----------------------------------------
class CtBatchItem(ctypes.Structure):
    _fields_ = [("in_", c_void_p), ("in_pitch", c_long), ("filt", c_void_p), ("k", c_int),
                ("out", c_void_p), ("out_pitch", c_long), ("out_h", c_int), ("out_w", c_int)]


BATCH_MODES = {"auto": 0, "persistent": 1, "launches": 2}
BATCH_RUNS = {"default": 0, "plain": 1, "persistent": 2, "launches": 3}


class CtBatchTiles(ctypes.Structure):
    _fields_ = [("block_x", (c_int * 18) * 2), ("tile_y", (c_int * 18) * 2),
                ("class_threads", c_int * 3), ("claim_items", c_int * 3),
                ("launch_block_x", (c_int * 18) * 2), ("launch_block_y", (c_int * 18) * 2),
                ("launch_tile_y", (c_int * 18) * 2), ("mode", c_int)]

    def to_dict(self) -> dict:
        """{(size class, k): (block_x, tile_y)} of the persistent kernels,
        {("threads", filter-side class): CTA size}, {("claim", filter-side
        class): items per claim}, {("L<size class>", k): (block_x, block_y,
        tile_y)} of the launches graph and {("mode", 0): mode}, where set."""
        out = {}
        for cls in (0, 1):
            for k in range(18):
                if self.block_x[cls][k]:
                    out[(cls, k)] = (self.block_x[cls][k], self.tile_y[cls][k])
                if self.launch_block_x[cls][k]:
                    out[(f"L{cls}", k)] = (self.launch_block_x[cls][k],
                                           self.launch_block_y[cls][k],
                                           self.launch_tile_y[cls][k])
        for c in range(3):
            if self.class_threads[c]:
                out[("threads", c)] = self.class_threads[c]
            if self.claim_items[c]:
                out[("claim", c)] = self.claim_items[c]
        if self.mode:
            out[("mode", 0)] = self.mode
        return out

    @classmethod
    def from_dict(cls, d: dict) -> "CtBatchTiles":
        t = cls()
        for key, val in d.items():
            if key[0] == "threads":
                t.class_threads[int(key[1])] = int(val)
            elif key[0] == "claim":
                t.claim_items[int(key[1])] = int(val)
            elif key[0] == "mode":
                t.mode = int(val)
            elif isinstance(key[0], str) and key[0] in ("L0", "L1"):
                c, k = int(key[0][1]), int(key[1])
                (t.launch_block_x[c][k], t.launch_block_y[c][k],
                 t.launch_tile_y[c][k]) = (int(v) for v in val)
            else:
                c, k = key
                t.block_x[c][k], t.tile_y[c][k] = val
        return t


def tiles_from_json(raw: dict) -> dict:
    """Tiles dict from its JSON form ({"c,k": [bx, ty], "threads,c": n,
    "claim,c": n, "Lc,k": [bx, by, ty], "mode,0": n})."""
    out = {}
    for key, val in raw.items():
        a, b = key.split(",")
        if a in ("threads", "claim", "mode"):
            out[(a, int(b))] = int(val)
        elif a in ("L0", "L1"):
            out[(a, int(b))] = tuple(val)
        else:
            out[(int(a), int(b))] = tuple(val)
    return out


def tiles_to_json(tiles: dict) -> dict:
    return {f"{a},{b}": (val if a in ("threads", "claim", "mode") else list(val))
            for (a, b), val in tiles.items()}


class CtBatchStats(ctypes.Structure):
    _fields_ = [("n_images", c_int), ("n_items", ctypes.c_longlong), ("grid", c_int),
                ("smem_bytes", c_long), ("flop", c_double), ("bytes", c_double),
                ("launches", c_int), ("mode", c_int), ("has_launch_graph", c_int)]


def batch_items(entries):
    """CtBatchItem array from (d_in, taps (host 2-D), d_out, out_h, out_w)
    tuples; returns (array, kept taps)."""
    arr = (CtBatchItem * len(entries))()
    keep = []
    for i, (d_in, filt, d_out, oh, ow) in enumerate(entries):
        f = _taps(filt)
        keep.append(f)
        arr[i] = CtBatchItem(_ptr(d_in), int(d_in.stride(0)) if hasattr(d_in, "stride") else 0,
                             f.ctypes.data, f.shape[0], _ptr(d_out),
                             int(d_out.stride(0)) if hasattr(d_out, "stride") else 0,
                             int(oh), int(ow))
    return arr, keep


def _batch_run_code(which) -> int:
    if isinstance(which, bool):  # measure(True): the plain comparison
        return BATCH_RUNS["plain"] if which else BATCH_RUNS["default"]
    return BATCH_RUNS[which] if isinstance(which, str) else int(which)


class Batch:
    """A batched plan (ct_batch_create); destroy() or use as a context
    manager.  mode: "auto", "persistent" or "launches" (overrides the tiles'
    mode)."""

    def __init__(self, entries, tiles: dict | None = None, mode: str | None = None):
        self._items, self._keep = batch_items(entries)
        self._h = c_void_p(0)
        t = CtBatchTiles.from_dict(tiles) if tiles else None
        if mode is not None:
            t = t if t is not None else CtBatchTiles()
            t.mode = BATCH_MODES[mode]
        _check(lib().ct_batch_create(self._items, len(entries),
                                     ctypes.byref(t) if t is not None else None,
                                     ctypes.byref(self._h)), "ct_batch_create")

    def run(self, stream=None, which="default"):
        _check(lib().ct_batch_run_mode(self._h, _batch_run_code(which),
                                       c_void_p(stream_handle(stream))), "ct_batch_run_mode")

    def run_plain(self, stream=None):
        _check(lib().ct_batch_run_plain(self._h, c_void_p(stream_handle(stream))),
               "ct_batch_run_plain")

    def info(self) -> dict:
        st = CtBatchStats()
        _check(lib().ct_batch_info(self._h, ctypes.byref(st)), "ct_batch_info")
        d = {k: getattr(st, k) for k, _ in CtBatchStats._fields_}
        d["mode_name"] = {1: "persistent", 2: "launches"}.get(d["mode"], "?")
        return d

    def measure(self, which="default", opts=None, stream=None) -> dict:
        """which: "default" (the batch's mode), "plain", "persistent",
        "launches" (True / False: plain / default)."""
        r = CtRecord()
        o = opts or measure_options()
        _check(lib().ct_measure_batch(self._h, _batch_run_code(which), ctypes.byref(o),
                                      c_void_p(stream_handle(stream)), ctypes.byref(r)),
               "ct_measure_batch")
        return r.to_dict()

    def destroy(self):
        if self._h:
            lib().ct_batch_destroy(self._h)
            self._h = c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def batch_tune(entries, objective="energy", opts=None, stream=None, class_threads=None,
               start: dict | None = None):
    """Per-bucket tiles by the tuner (ct_batch_tune): (tiles dict, records).
    class_threads: optional CTA size per filter-side class to tune with;
    start: optional tiles dict to start the search from."""
    items, keep = batch_items(entries)
    t = CtBatchTiles.from_dict(start) if start else CtBatchTiles()
    for c, n in enumerate(class_threads or ()):
        t.class_threads[c] = int(n)
    cap = 12 * 2 * 18
    recs = (CtRecord * cap)()
    n = c_int(0)
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    o = opts or measure_options()
    _check(lib().ct_batch_tune(items, len(entries), obj, ctypes.byref(o),
                               c_void_p(stream_handle(stream)), ctypes.byref(t), recs, cap,
                               ctypes.byref(n)), "ct_batch_tune")
    return t.to_dict(), [recs[i].to_dict() for i in range(n.value)]


def batch_tune_launches(entries, objective="energy", opts=None, stream=None,
                        start: dict | None = None):
    """Per-bucket single-image configurations of the launches graph
    (ct_batch_tune_launches): (tiles dict, records); start: optional tiles
    dict whose other entries are kept."""
    items, keep = batch_items(entries)
    t = CtBatchTiles.from_dict(start) if start else CtBatchTiles()
    cap = 9 * 2 * 18
    recs = (CtRecord * cap)()
    n = c_int(0)
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    o = opts or measure_options()
    _check(lib().ct_batch_tune_launches(items, len(entries), obj, ctypes.byref(o),
                                        c_void_p(stream_handle(stream)), ctypes.byref(t), recs,
                                        cap, ctypes.byref(n)), "ct_batch_tune_launches")
    return t.to_dict(), [recs[i].to_dict() for i in range(n.value)]


# ---- request server ---------------------------------------------------------
class CtServerOptions(ctypes.Structure):
    _fields_ = [("n_streams", c_int), ("max_batch", c_int), ("pool_bytes", ctypes.c_longlong),
                ("max_wait_s", c_double), ("plain", c_int), ("use_tiles", c_int),
                ("tiles", CtBatchTiles), ("trace_cap", c_int)]


class CtServerTraceEntry(ctypes.Structure):
    _fields_ = [("t_dispatch", c_double), ("dispatch_s", c_double), ("plan_s", c_double),
                ("t_done", c_double), ("oldest_wait_s", c_double), ("loop_gap_s", c_double),
                ("n_requests", c_int), ("slot", c_int), ("queued", c_int),
                ("busy_slots", c_int), ("h2d_ms", c_double), ("kernels_ms", c_double),
                ("d2h_ms", c_double), ("bytes_in", c_double), ("bytes_out", c_double)]


class CtServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("p50_s", c_double), ("p99_s", c_double),
                ("mean_s", c_double), ("max_s", c_double), ("wall_s", c_double),
                ("flop", c_double), ("energy_j", c_double), ("batches", ctypes.c_longlong),
                ("mean_batch", c_double), ("pool_used_bytes", ctypes.c_longlong)]


class Server:
    """Continuous-batching request server (ct_server_*).  Host buffers passed
    to submit() must stay alive until the request completes."""

    def __init__(self, n_streams=4, max_batch=64, pool_bytes=8 << 30, max_wait_s=200e-6,
                 plain=False, tiles: dict | None = None, trace_cap=0):
        o = CtServerOptions(n_streams, max_batch, pool_bytes, max_wait_s, int(bool(plain)),
                            1 if tiles else 0, CtBatchTiles.from_dict(tiles) if tiles
                            else CtBatchTiles(), int(trace_cap))
        self._h = c_void_p(0)
        _check(lib().ct_server_create(ctypes.byref(o), ctypes.byref(self._h)), "ct_server_create")
        self._keep = {}

    def submit(self, inp: np.ndarray, filt, out: np.ndarray, out_h: int, out_w: int) -> int:
        f = _taps(filt)
        rid = ctypes.c_longlong(0)
        _check(lib().ct_server_submit(self._h, inp.ctypes.data, inp.shape[1], f.ctypes.data,
                                      f.shape[0], out.ctypes.data, out.shape[1], int(out_h),
                                      int(out_w), ctypes.byref(rid)), "ct_server_submit")
        return rid.value

    def wait(self, rid: int, timeout_s=60.0) -> float:
        lat = c_double(0)
        _check(lib().ct_server_wait(self._h, rid, timeout_s, ctypes.byref(lat)), "ct_server_wait")
        return lat.value

    def drain(self, timeout_s=120.0):
        _check(lib().ct_server_drain(self._h, timeout_s), "ct_server_drain")

    def stats(self, reset=False) -> dict:
        st = CtServerStats()
        _check(lib().ct_server_stats_get(self._h, int(bool(reset)), ctypes.byref(st)),
               "ct_server_stats_get")
        return {k: getattr(st, k) for k, _ in CtServerStats._fields_}

    def trace(self) -> list:
        """The timeline of the last completed batches (ct_server_trace_get)."""
        n = c_int(0)
        rc = lib().ct_server_trace_get(self._h, None, 0, ctypes.byref(n))
        if rc not in (CT_OK, CT_ENOMEM):
            _check(rc, "ct_server_trace_get")
        buf = (CtServerTraceEntry * max(1, n.value))()
        _check(lib().ct_server_trace_get(self._h, buf, n.value, ctypes.byref(n)),
               "ct_server_trace_get")
        return [{k: getattr(buf[i], k) for k, _ in CtServerTraceEntry._fields_}
                for i in range(n.value)]

    def close(self):
        if self._h:
            lib().ct_server_destroy(self._h)
            self._h = c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- analyses of tuning records ---------------------------------------------
METHODS = ("race_to_idle", "energy_maxclock", "race_to_idle_clocks", "energy_clocks",
           "global_energy")


def _record_array(records):
    arr = (CtRecord * len(records))()
    for i, r in enumerate(records):
        for k, _ in CtRecord._fields_:
            if k == "cfg":
                arr[i].cfg = Config(*r["cfg"]).to_c()
            else:
                setattr(arr[i], k, r.get(k, 0))
    return arr


def tuning_methods(records, base_clock_mhz: int) -> dict:
    """The five tuning methods of Section IV-A (ct_tuning_methods)."""
    out = (c_int * 5)()
    _check(lib().ct_tuning_methods(_record_array(records), len(records), int(base_clock_mhz),
                                   out), "ct_tuning_methods")
    return {m: out[i] for i, m in enumerate(METHODS)}


def pareto_front(records) -> list:
    idx = (c_int * max(1, len(records)))()
    n = c_int(0)
    _check(lib().ct_pareto_front(_record_array(records), len(records), idx, len(idx),
                                 ctypes.byref(n)), "ct_pareto_front")
    return [idx[i] for i in range(n.value)]


def centrality(records, objective="energy", ps=(1.0, 1.05, 1.1, 1.25, 1.5, 2.0),
               damping=0.85) -> dict:
    p = np.ascontiguousarray(ps, dtype=np.float64)
    out = np.zeros_like(p)
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    _check(lib().ct_centrality(_record_array(records), len(records), obj, float(damping),
                               p.ctypes.data, p.size, out.ctypes.data), "ct_centrality")
    return dict(zip(ps, out.tolist()))
