"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain serial CPU implementations of the fixed points that the GPU worklist
kernels must reach: FIFO-queue BFS levels, binary-heap Dijkstra distances,
union-find minimum-id component labels and the Kruskal minimum spanning forest
(``oracle.c``; each function there cites the definition it follows).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package. The library under
``paper_1607_05707_gb300`` never imports it, and it shares no code with the
CUDA path: the two meet only in the seeded CSR arrays the input generator
writes and in the uint32 arrays they return.

Status: every function is pinned by ``tests/test_oracle_pins.py`` (brute force on
tiny graphs, closed forms, invariants, special shapes, hand-worked golden files);
nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

INF = 0xFFFFFFFF

_lib = None


def build(force: bool = False) -> Path:
    """Compile oracle.c with gcc into liboracle.so (in place)."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", str(tmp), str(SRC)], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_bfs.restype = ctypes.c_int
        lib.oracle_bfs.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint32, u32p, u32p]
        lib.oracle_sssp.restype = ctypes.c_int
        lib.oracle_sssp.argtypes = [ctypes.c_uint32, u32p, u32p, i32p, ctypes.c_uint32, u32p, u32p]
        lib.oracle_cc.restype = ctypes.c_int
        lib.oracle_cc.argtypes = [ctypes.c_uint32, u32p, u32p, u32p]
        lib.oracle_msf.restype = ctypes.c_int
        lib.oracle_msf.argtypes = [ctypes.c_uint32, u32p, u32p, i32p, u32p, u32p, i32p, u32p,
                                   ctypes.POINTER(ctypes.c_uint64)]
        _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a: np.ndarray, ct=ctypes.c_uint32):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


def bfs(n: int, row_ptr, col, srcs) -> np.ndarray:
    """Levels from the sources (multi-source: min over sources); INF if unreachable."""
    rp, c, s = _u32(row_ptr), _u32(col), _u32(np.atleast_1d(srcs))
    out = np.empty(n, dtype=np.uint32)
    _check(_load().oracle_bfs(n, _ptr(rp), _ptr(c), s.size, _ptr(s), _ptr(out)), "oracle_bfs")
    return out


def sssp(n: int, row_ptr, col, w, srcs) -> np.ndarray:
    """Shortest-path distances (non-negative int32 weights); INF if unreachable."""
    rp, c, s = _u32(row_ptr), _u32(col), _u32(np.atleast_1d(srcs))
    ww = np.ascontiguousarray(w, dtype=np.int32)
    out = np.empty(n, dtype=np.uint32)
    _check(_load().oracle_sssp(n, _ptr(rp), _ptr(c), _ptr(ww, ctypes.c_int32), s.size, _ptr(s), _ptr(out)),
           "oracle_sssp")
    return out


def cc(n: int, row_ptr, col) -> np.ndarray:
    """Minimum vertex id of each vertex's connected component (edges undirected)."""
    rp, c = _u32(row_ptr), _u32(col)
    out = np.empty(n, dtype=np.uint32)
    _check(_load().oracle_cc(n, _ptr(rp), _ptr(c), _ptr(out)), "oracle_cc")
    return out


def msf(n: int, row_ptr, col, w) -> tuple[np.ndarray, int]:
    """Minimum spanning forest under the key (w, min(u,v), max(u,v)): its edges as
    rows (u, v, w) with u < v, in key order, and their total weight."""
    rp, c = _u32(row_ptr), _u32(col)
    ww = np.ascontiguousarray(w, dtype=np.int32)
    cap = max(n - 1, 1)
    ou, ov = np.empty(cap, dtype=np.uint32), np.empty(cap, dtype=np.uint32)
    ow = np.empty(cap, dtype=np.int32)
    cnt = ctypes.c_uint32(0)
    tot = ctypes.c_uint64(0)
    _check(_load().oracle_msf(n, _ptr(rp), _ptr(c), _ptr(ww, ctypes.c_int32), _ptr(ou), _ptr(ov),
                              _ptr(ow, ctypes.c_int32), ctypes.byref(cnt), ctypes.byref(tot)), "oracle_msf")
    k = cnt.value
    edges = np.stack([ou[:k].astype(np.int64), ov[:k].astype(np.int64), ow[:k].astype(np.int64)], axis=1)
    return edges.reshape(k, 3), int(tot.value)


def run(kind: str, g, srcs=None) -> np.ndarray:
    """Dispatch on 'bfs' | 'sssp' | 'cc' for a CSR object with n, row_ptr, col, w."""
    if kind == "bfs":
        return bfs(g.n, g.row_ptr, g.col, srcs)
    if kind == "sssp":
        return sssp(g.n, g.row_ptr, g.col, g.w, srcs)
    if kind == "cc":
        return cc(g.n, g.row_ptr, g.col)
    raise ValueError(kind)
