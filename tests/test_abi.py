"""The C ABI library loads on a CPU-only host and exports every function that
include/*.h declares; host-side argument checks answer without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ct_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return api.lib()


def test_header_declares_functions():
    names = declared_functions()
    assert "ct_conv2d_run" in names and "ct_strerror" in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    assert api.strerror(api.CT_OK) == "ok"
    assert "configuration" in api.strerror(api.CT_ECONFIG)
    assert api.strerror(12345) == "unknown status"
    assert api.version().startswith("convtune")


def test_host_side_argument_checks_need_no_gpu(lib):
    assert lib.ct_conv2d_run(None, None, None) == api.CT_EINVAL
    c = api.Config().to_c()
    p = api.CtProblem(0, 0, 0, 3, 3, 0, 0, 4, 4)  # null filter
    assert lib.ct_conv2d_check(ctypes.byref(p), ctypes.byref(c), None, 0) == api.CT_EINVAL
    taps = (ctypes.c_float * 9)()
    p = api.CtProblem(0, 0, ctypes.addressof(taps), 3, 3, 0, 0, 0, 4)  # empty: nothing to do
    assert lib.ct_conv2d_run(ctypes.byref(p), ctypes.byref(c), None) == api.CT_OK
    p = api.CtProblem(16, 9, ctypes.addressof(taps), 3, 3, 32, 8, 4, 8)  # pitch too small
    why = ctypes.create_string_buffer(128)
    assert lib.ct_conv2d_check(ctypes.byref(p), ctypes.byref(c), why, 128) == api.CT_EINVAL
    assert b"in_pitch" in why.value
    bad = api.Config(block_x=48).to_c()
    p = api.CtProblem(16, 12, ctypes.addressof(taps), 3, 3, 32, 8, 4, 8)
    assert lib.ct_conv2d_check(ctypes.byref(p), ctypes.byref(bad), None, 0) == api.CT_ECONFIG


def test_default_host_band_split(lib):
    # host logic of the pipelined host-buffer entry point: an even split into
    # max(min(h // 256, 8), ceil(h / 512)) bands, 1..64 of them, covering
    # every row once
    assert api.host_bands_default(1) == [1]
    assert api.host_bands_default(511) == [511]
    assert api.host_bands_default(512) == [256, 256]
    assert api.host_bands_default(1024) == [256] * 4
    assert api.host_bands_default(4096) == [512] * 8
    assert api.host_bands_default(8192) == [512] * 16
    assert api.host_bands_default(1000) == [334, 333, 333]
    for h in (513, 4097, 32767, 70000, 2**31 - 1):
        b = api.host_bands_default(h)
        n = max(min(h // 256, 8), -(-h // 512))
        assert len(b) == min(n, 64) and sum(b) == h and max(b) - min(b) <= 1, h
    n = ctypes.c_int(0)
    assert lib.ct_conv2d_host_bands_default(0, None, 0, ctypes.byref(n)) == api.CT_EINVAL
    assert lib.ct_conv2d_host_bands_default(4096, None, 0, ctypes.byref(n)) == api.CT_ENOMEM
    assert n.value == 8


def test_explicit_band_split_is_checked_on_the_host(lib):
    taps = (ctypes.c_float * 9)()
    buf_in = (ctypes.c_float * (10 * 10))()
    buf_out = (ctypes.c_float * (8 * 8))()
    c = api.Config().to_c()

    def run(rows):
        arr = (ctypes.c_int * len(rows))(*rows)
        return lib.ct_conv2d_run_host_bands(buf_in, 10, taps, 3, 3, buf_out, 8, 8, 8,
                                            ctypes.byref(c), arr, len(rows), None)
    for bad in ([8, 0], [4, 3], [4, 5], [1] * 65, [-1, 9]):
        assert run(bad) == api.CT_EINVAL, bad


def test_async_host_entry_checks_arguments_on_the_host(lib):
    taps = (ctypes.c_float * 9)()
    buf_in = (ctypes.c_float * (10 * 10))()
    buf_out = (ctypes.c_float * (8 * 8))()
    c = api.Config().to_c()
    run = lib.ct_conv2d_run_host_async
    assert run(buf_in, 10, None, 3, 3, buf_out, 8, 8, 8, ctypes.byref(c)) == api.CT_EINVAL
    assert run(None, 10, taps, 3, 3, buf_out, 8, 8, 8, ctypes.byref(c)) == api.CT_EINVAL
    assert run(buf_in, 9, taps, 3, 3, buf_out, 8, 8, 8, ctypes.byref(c)) == api.CT_EINVAL  # pitch
    assert run(buf_in, 10, taps, 3, 3, buf_out, 8, 8, 8, None) == api.CT_EINVAL
    # nothing to do: no device work, no error
    assert run(buf_in, 10, taps, 3, 3, buf_out, 8, 0, 8, ctypes.byref(c)) == api.CT_OK


def test_batch_modes_host_checks_and_tiles_round_trip(lib):
    # null handles are refused before any device work
    assert lib.ct_batch_run_mode(None, api.BATCH_RUNS["launches"], None) == api.CT_EINVAL
    assert lib.ct_batch_run(None, None) == api.CT_EINVAL
    assert lib.ct_measure_batch(None, 0, None, None, None) == api.CT_EINVAL
    n = ctypes.c_int(0)
    assert lib.ct_batch_tune_launches(None, 0, 0, None, None, None, None, 0,
                                      ctypes.byref(n)) == api.CT_EINVAL
    # every kind of tiles entry survives the struct and the JSON form
    tiles = {(0, 3): (16, 8), (1, 17): (32, 4), ("threads", 1): 128, ("claim", 0): 2,
             ("L0", 5): (32, 4, 2), ("L1", 17): (16, 8, 4), ("mode", 0): api.BATCH_MODES["launches"]}
    assert api.CtBatchTiles.from_dict(tiles).to_dict() == tiles
    assert api.tiles_from_json(api.tiles_to_json(tiles)) == tiles
    assert ctypes.sizeof(api.CtBatchTiles) == 4 * (2 * 18 * 5 + 3 + 3 + 1)
