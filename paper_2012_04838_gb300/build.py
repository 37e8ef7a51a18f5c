"""Build ``libpsc.so`` in-tree with nvcc for sm_103a.

One object file per (precision, grid size) instantiation of the FFT passes is
compiled in parallel, plus the host API; objects are reused when their
sources and flags are unchanged.  ``PSC_CHECKED=1`` in the environment builds
the variant whose kernels check every global index (a separate library,
``libpsc_checked.so``).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")

SIZES = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 520, 1024)
PRECISIONS = ("float", "double")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpsc")


def lib_path(checked: bool = False) -> str:
    return os.path.join(HERE, "libpsc_checked.so" if checked else "libpsc.so")


def _sources_digest(extra: list[str]) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "psc.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()[:16]


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout)


def build(checked: bool | None = None, jobs: int | None = None, verbose: bool = True) -> str:
    """Compile every translation unit and link the shared library; returns its path."""
    if checked is None:
        checked = os.environ.get("PSC_CHECKED", "0") == "1"
    cc = nvcc()
    flags = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC] + ARCH
    if checked:
        flags.append("-DPSC_CHECKED=1")
    # developer knob for kernel-variant experiments, e.g. PSC_NVCC_FLAGS="-DPSC_X2_MIN_N=2048"
    flags += os.environ.get("PSC_NVCC_FLAGS", "").split()
    tag = ("chk_" if checked else "") + _sources_digest(flags)
    odir = os.path.join(BUILD, tag)
    os.makedirs(odir, exist_ok=True)
    units = []
    for t in PRECISIONS:
        for n in SIZES:
            obj = os.path.join(odir, f"inst_{t}_{n}.o")
            units.append((obj, [cc] + flags + [f"-DPSC_INST_T={t}", f"-DPSC_INST_N={n}", "-c",
                                               os.path.join(CSRC, "psc_inst.cu"), "-o", obj]))
    for src in ("psc_capi", "psc_noalloc", "psc_batch"):
        obj = os.path.join(odir, src + ".o")
        units.append((obj, [cc] + flags + ["-c", os.path.join(CSRC, src + ".cu"), "-o", obj]))
    # the persistent ensemble kernel, one unit per RK stage
    for stage in (1, 2, 3, 4):
        obj = os.path.join(odir, f"batch_stage_{stage}.o")
        # global loads cached in L2 only: CTAs of one launch read what others wrote
        units.append((obj, [cc] + flags + [f"-DPSCB_STAGE={stage}", "-Xptxas", "-dlcm=cg", "-c",
                                           os.path.join(CSRC, "psc_batch_stage.cu"), "-o", obj]))
    todo = [(o, c) for o, c in units if not os.path.exists(o)]
    if todo:
        jobs = jobs or max(1, os.cpu_count() or 1)
        if verbose:
            print(f"[psc build] compiling {len(todo)} units with {jobs} jobs", file=sys.stderr, flush=True)
        with cf.ThreadPoolExecutor(jobs) as ex:
            list(ex.map(lambda oc: _run(oc[1]), todo))
    out = lib_path(checked)
    tmp = out + ".tmp"
    _run([cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in units])
    os.replace(tmp, out)
    if verbose:
        print(f"[psc build] {out}", file=sys.stderr, flush=True)
    return out


if __name__ == "__main__":
    build(checked="--checked" in sys.argv)
