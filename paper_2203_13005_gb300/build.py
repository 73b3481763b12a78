"""Compile the native parts of the package in-tree.

* ``libgxp.so``: the C-ABI superstep engine (CUDA for sm_103a + C++ host
  runtime), declared in ``include/gxp.h``.
* ``libgxp_synth.so``: the seeded input generators (plain C, OpenMP).

Both land in ``paper_2203_13005_gb300/_build/``. A library is rebuilt when any
of its sources is newer than it. Translation units compile in parallel, one
``-gencode`` (sm_103a), no cmake.
"""
from __future__ import annotations

import concurrent.futures as _fut
import os
import shutil
import subprocess
import tempfile

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(REPO_DIR, "include")
BUILD_DIR = os.path.join(PKG_DIR, "_build")

GXP_LIB = os.path.join(BUILD_DIR, "libgxp.so")
SYNTH_LIB = os.path.join(BUILD_DIR, "libgxp_synth.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgxp")
    return cand


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)


def _atomic_link(objs: list[str], out: str, linker: list[str]) -> None:
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD_DIR)
    os.close(fd)
    try:
        _run(linker + objs + ["-o", tmp])
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)


def gxp_sources() -> tuple[list[str], list[str], list[str]]:
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                 if f.endswith(".cpp"))
    hdr = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                 if f.endswith((".cuh", ".h", ".hpp")))
    hdr.append(os.path.join(INCLUDE, "gxp.h"))
    return cu, cpp, hdr


def build_synth(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(CSRC, "synth.c")
    if force or _stale(SYNTH_LIB, [src, __file__]):
        cc = shutil.which("gcc") or "cc"
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD_DIR)
        os.close(fd)
        try:
            _run([cc, "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp])
            os.replace(tmp, SYNTH_LIB)
        finally:
            if os.path.exists(tmp):
                os.unlink(tmp)
    return SYNTH_LIB


def build_gxp(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile every ``.cu``/``.cpp`` under csrc/ (except synth.c) into libgxp.so."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    cu, cpp, hdr = gxp_sources()
    if not (force or _stale(GXP_LIB, cu + cpp + hdr + [__file__])):
        return GXP_LIB
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for s in cu:
        o = os.path.join(BUILD_DIR, os.path.basename(s) + ".o")
        cmd = [nvcc, *ARCH_FLAGS, "-lineinfo", *common, "--expt-relaxed-constexpr",
               "-Xcompiler", "-fPIC,-fvisibility=hidden", "-c", s, "-o", o]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, o))
    for s in cpp:
        o = os.path.join(BUILD_DIR, os.path.basename(s) + ".o")
        cmd = [nvcc, *common, "-x", "c++", "-Xcompiler", "-fPIC,-fvisibility=hidden,-fopenmp",
               "-c", s, "-o", o]
        jobs.append((cmd, o))
    outputs: list[str] = []
    with _fut.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_run, cmd) for cmd, _ in jobs]
        for f in futs:
            f.result()
    outputs = [o for _, o in jobs]
    linker = [nvcc, *ARCH_FLAGS, "-shared", "-Xcompiler", "-fopenmp",
              "-L", os.path.join(_cuda_home(), "lib64"), "-lcudart", "-lgomp"]
    _atomic_link(outputs, GXP_LIB, linker)
    return GXP_LIB


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_gxp(force)
