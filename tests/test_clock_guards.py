"""A clock lock never outlives the process: the library undoes it at normal
exit, on SIGTERM and on SIGINT (host-side failure handling, tested with a
C fake of the platform table in child processes; no GPU involved)."""
import os
import signal
import subprocess
import sys
import textwrap

import pytest

from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fake_so(tmp_path_factory):
    pkg_build.build()
    out = str(tmp_path_factory.mktemp("fake") / "libfake_platform.so")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-o", out, os.path.join(ROOT, "tests", "fakes", "fake_platform.c"),
                    api.lib_path()], check=True)
    return out


def _child(fake, log, tail):
    code = textwrap.dedent(f"""
        import ctypes, os, signal, sys, time
        lib = ctypes.CDLL({api.lib_path()!r})
        fake = ctypes.CDLL({fake!r})
        assert fake.fake_install({log!r}.encode()) == 0
        assert lib.ct_lock_sm_clock(1500) == 0
        sys.stdout.write("locked\\n"); sys.stdout.flush()
    """) + textwrap.dedent(tail)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                          timeout=60)


def _log(path):
    return open(path).read().split("\n")[:-1] if os.path.exists(path) else []


def test_lock_is_reset_at_normal_exit(fake_so, tmp_path):
    log = str(tmp_path / "exit.log")
    r = _child(fake_so, log, "sys.exit(0)\n")
    assert r.returncode == 0 and "locked" in r.stdout
    assert _log(log) == ["lock 1500", "reset 0"]


def test_lock_is_reset_on_sigterm(fake_so, tmp_path):
    log = str(tmp_path / "term.log")
    r = _child(fake_so, log, "os.kill(os.getpid(), signal.SIGTERM)\ntime.sleep(10)\n")
    assert r.returncode == -signal.SIGTERM
    assert _log(log) == ["lock 1500", "reset 0"]


def test_lock_is_reset_on_sigint(fake_so, tmp_path):
    log = str(tmp_path / "int.log")
    r = _child(fake_so, log, "os.kill(os.getpid(), signal.SIGINT)\ntime.sleep(10)\n")
    assert r.returncode != 0  # KeyboardInterrupt after the library's handler ran
    assert _log(log)[:2] == ["lock 1500", "reset 0"]
    assert _log(log).count("reset 0") == 1


def test_explicit_reset_leaves_nothing_for_exit(fake_so, tmp_path):
    log = str(tmp_path / "explicit.log")
    r = _child(fake_so, log, "assert lib.ct_reset_sm_clock() == 0\nsys.exit(0)\n")
    assert r.returncode == 0
    assert _log(log) == ["lock 1500", "reset 0"]
