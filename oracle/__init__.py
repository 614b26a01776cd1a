"""Independent CPU oracle for the convolution / energy-tuning hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import anything from
this package.  The product library (``paper_2211_07260_gb300``) never imports
it, and this package imports nothing from the product: the two share no code,
headers, tables or helpers.  Only the seeded input generators
(``paper_2211_07260_gb300.synth``, which holds none of the method's
arithmetic) feed both.

Contents
--------
``conv2d`` / ``conv2d_points``  FP64 direct 2-D cross-correlation (C, OpenMP)
                                 -- ``conv2d_ref.c``.
``power_model``                  FP64 fit of the power curve (Section IV-E,
                                 Eq. powercurve, voltage estimate), its
                                 energy-optimal clock and the +-10 % clock
                                 range.
``selection``                    energy / metric bookkeeping (Section III-A,
                                 III-C) and exhaustive-vs-steered selection
                                 over a results table.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_conv2d.so")
_SRC = os.path.join(_HERE, "conv2d_ref.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``conv2d_ref.c`` with gcc (-O2, OpenMP) into ``_build/``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c_long, c_int, vp = ctypes.c_long, ctypes.c_int, ctypes.c_void_p
            lib.oracle_conv2d_f64.argtypes = [vp, c_long, c_long, c_long, vp, c_long, c_long,
                                              vp, c_long, c_long, c_long, c_int]
            lib.oracle_conv2d_f64.restype = c_int
            lib.oracle_conv2d_points_f64.argtypes = [vp, c_long, c_long, c_long, vp, c_long,
                                                     c_long, vp, vp, c_long, vp, c_int]
            lib.oracle_conv2d_points_f64.restype = c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _as_padded(in_buf, in_w):
    a = np.ascontiguousarray(in_buf, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("padded input must be 2-D (rows x pitch)")
    in_h, pitch = a.shape
    in_w = pitch if in_w is None else int(in_w)
    if in_w > pitch:
        raise ValueError("logical width exceeds the row pitch")
    return a, in_h, pitch, in_w


def conv2d(in_buf, filt, in_w=None, nthreads=None) -> np.ndarray:
    """FP64 cross-correlation of the padded input with the filter.

    ``in_buf`` is the padded input, shape (in_h, pitch) float32, whose first
    ``in_w`` columns are valid; ``filt`` is (fh, fw) float32.  Returns the
    (in_h-fh+1, in_w-fw+1) float64 result of
    ``ref[y][x] = sum_j sum_i in[y+j][x+i] * filt[j][i]``.
    """
    a, in_h, pitch, in_w = _as_padded(in_buf, in_w)
    f = np.ascontiguousarray(filt, dtype=np.float32)
    fh, fw = f.shape
    oh, ow = in_h - fh + 1, in_w - fw + 1
    if oh < 1 or ow < 1:
        raise ValueError("filter larger than the input")
    out = np.empty((oh, ow), dtype=np.float64)
    nt = max_threads() if nthreads is None else int(nthreads)
    rc = _load().oracle_conv2d_f64(a.ctypes.data, pitch, in_h, in_w, f.ctypes.data, fh, fw,
                                   out.ctypes.data, ow, oh, ow, nt)
    if rc != 0:
        raise ValueError("oracle_conv2d_f64 rejected its arguments")
    return out


def conv2d_points(in_buf, filt, ys, xs, in_w=None, nthreads=None) -> np.ndarray:
    """The FP64 sum at selected output coordinates only."""
    a, in_h, pitch, in_w = _as_padded(in_buf, in_w)
    f = np.ascontiguousarray(filt, dtype=np.float32)
    fh, fw = f.shape
    ys = np.ascontiguousarray(ys, dtype=np.int64)
    xs = np.ascontiguousarray(xs, dtype=np.int64)
    if ys.shape != xs.shape:
        raise ValueError("ys and xs differ in shape")
    out = np.empty(ys.shape, dtype=np.float64)
    nt = max_threads() if nthreads is None else int(nthreads)
    rc = _load().oracle_conv2d_points_f64(a.ctypes.data, pitch, in_h, in_w, f.ctypes.data,
                                          fh, fw, ys.ctypes.data, xs.ctypes.data, ys.size,
                                          out.ctypes.data, nt)
    if rc != 0:
        raise ValueError("oracle_conv2d_points_f64 rejected its arguments")
    return out
