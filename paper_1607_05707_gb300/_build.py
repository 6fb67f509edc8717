"""In-tree build of the native parts of the package.

* ``libirglgen.so``  -- seeded CSR generator (plain C++, host only).
* ``libirgl.so``     -- the C-ABI library: host runtime plus the sm_103a kernels.

Everything is compiled in place next to the sources (no pip install), with one
``-gencode`` for sm_103a, and the translation units of ``libirgl.so`` are
compiled in parallel so a fresh build takes about a minute.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
ROOT = PKG.parent
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"

GEN_LIB = PKG / "libirglgen.so"
IRGL_LIB = PKG / "libirgl.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# CUDA translation units of libirgl.so (kernels are split so they compile in parallel).
CUDA_UNITS = [
    "irgl_api.cu",
    "irgl_k_single.cu",
    "irgl_k_launch.cu",
    "irgl_k_smem.cu",
    "irgl_k_batch.cu",
    "irgl_batch.cu",
    "irgl_server.cu",
    "irgl_tune.cu",
    "irgl_noalloc.cu",
    "irgl_msf.cu",
]
HOST_UNITS: list[str] = []


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libirgl.so")


def _cuda_home() -> Path:
    return Path(_nvcc()).resolve().parent.parent


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    if os.environ.get("IRGL_BUILD_VERBOSE"):
        sys.stderr.write(r.stdout)


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps if d.exists())


def build_gen(force: bool = False) -> Path:
    src = CSRC / "graphgen.cpp"
    if force or _stale(GEN_LIB, [src, INCLUDE / "irgl_gen.h"]):
        tmp = GEN_LIB.with_suffix(f".so.tmp{os.getpid()}")
        _run(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", str(tmp), str(src)])
        os.replace(tmp, GEN_LIB)
    return GEN_LIB


def build_irgl(force: bool = False, extra_flags: list[str] | None = None) -> Path:
    deps = [CSRC / u for u in CUDA_UNITS + HOST_UNITS] + list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + [
        INCLUDE / "irgl.h"
    ]
    if not force and not _stale(IRGL_LIB, deps):
        return IRGL_LIB
    BUILD.mkdir(exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + [
        "-O3",
        "-lineinfo",
        "-std=c++17",
        "-Xcompiler",
        "-fPIC",
        "-I",
        str(INCLUDE),
        "-I",
        str(CSRC),
        "--expt-relaxed-constexpr",
    ] + (extra_flags or []) + os.environ.get("IRGL_EXTRA_NVCC_FLAGS", "").split()
    if os.environ.get("IRGL_PTXAS_VERBOSE"):
        flags += ["-Xptxas", "-v"]
    objs: list[Path] = []
    cmds: list[list[str]] = []
    for u in CUDA_UNITS:
        o = BUILD / (u + ".o")
        objs.append(o)
        cmds.append([nvcc, *flags, "-c", str(CSRC / u), "-o", str(o)])
    for u in HOST_UNITS:
        o = BUILD / (u + ".o")
        objs.append(o)
        cmds.append([
            "g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", str(INCLUDE), "-I", str(CSRC),
            "-I", str(_cuda_home() / "include"), "-c", str(CSRC / u), "-o", str(o),
        ])
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        list(ex.map(_run, cmds))
    tmp = IRGL_LIB.with_suffix(f".so.tmp{os.getpid()}")
    _run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", str(tmp), *map(str, objs), "-lpthread"])
    os.replace(tmp, IRGL_LIB)
    return IRGL_LIB


def build_all(force: bool = False) -> None:
    build_gen(force)
    build_irgl(force)
