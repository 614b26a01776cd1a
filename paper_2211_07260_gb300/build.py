"""Build libconvtune.so in-tree with nvcc for sm_103a.

Translation units are compiled in parallel (one per specialised filter side,
plus the runtime, tuner, measurement, microbenchmark and batched units) and
linked into ``_build/libconvtune.so``.  An object is rebuilt only when a
source or header under ``csrc/`` or ``include/`` is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libconvtune.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SPECIALISED_K = (1, 3, 5, 7, 9, 11, 13, 15, 17)


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libconvtune")
    return cand


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


def _units():
    """(object name, source, extra flags) of every translation unit."""
    units = [(f"conv2d_k{k}.o", "conv2d_inst.cu", [f"-DCT_K={k}"]) for k in SPECIALISED_K]
    for src in sorted(os.listdir(CSRC)):
        if src == "conv2d_inst.cu" or not src.endswith((".cu", ".cpp")):
            continue
        units.append((os.path.splitext(src)[0] + ".o", src, []))
    return units


def _newest_dep() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    newest = _newest_dep()
    # host code: no contraction of a*b+c into FMA (aarch64 hosts would
    # otherwise round the FP64 model arithmetic differently from x86-64)
    common = ["-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]

    def compile_one(unit):
        obj, src, extra = unit
        out = os.path.join(BUILD, obj)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            return obj, None
        tmp = out + ".tmp"
        cmd = [nvcc, *common, *extra, "-c", os.path.join(CSRC, src), "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return obj, r.stderr + r.stdout
        os.replace(tmp, out)
        if verbose:
            sys.stderr.write(f"built {obj}\n")
        return obj, None

    units = _units()
    jobs = jobs or max(1, min(len(units), os.cpu_count() or 4))
    errors = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, err in ex.map(compile_one, units):
            if err:
                errors.append(f"--- {obj}\n{err}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))

    objs = [os.path.join(BUILD, u[0]) for u in units]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, objs)):
        libdir = _cuda_lib_dir(nvcc)
        tmp = LIB + ".tmp"
        cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-L", libdir, "-lcudart", "-ldl",
               "-lpthread", "-Xlinker", f"-rpath,{libdir}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr + r.stdout)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
