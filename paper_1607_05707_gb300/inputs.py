"""Seeded synthetic inputs: CSR meshes, R-MAT graphs, sources and arrivals.

This module only *makes inputs*; it holds none of the traversal arithmetic.
Both the CUDA path and the CPU oracle consume the arrays it returns.

Workloads (sizes as used by the tests and the benchmark):

* ``grid64``        64 x 64 4-neighbour grid, V = 4096, m = 16,128, source 0
* ``rmat20``        R-MAT scale 20, edge factor 16, (a,b,c) = (.57,.19,.19),
                    weights uniform [1,100], seeded sources of out-degree > 0
* ``mesh4096``      4096 x 4096 mesh, 1% of grid edges deleted, 0.1% of
                    vertices with one extra edge within Manhattan radius 8
* ``batch256``      256 R-MAT instances, scale uniform in 10..18, edge factor 8,
                    1-4 sources each, weights uniform [1,100]
* ``serve``         R-MAT scale 24 (edge factor 16) plus 32 grids of side
                    uniform in [256, 2048], Poisson arrivals

Seeds: graph seed = 1000 + workload number, source seed = 2000 + workload number.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _build

INF = 0xFFFFFFFF

_lib = None


def _gen():
    global _lib
    if _lib is None:
        path = _build.build_gen()
        lib = ctypes.CDLL(str(path))
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.irglgen_draw.restype = ctypes.c_uint64
        lib.irglgen_draw.argtypes = [ctypes.c_uint64] * 3
        lib.irglgen_mesh.restype = ctypes.c_int64
        lib.irglgen_mesh.argtypes = [
            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
            ctypes.c_uint32, u32p, u32p, i32p, ctypes.c_uint64,
        ]
        lib.irglgen_rmat.restype = ctypes.c_int64
        lib.irglgen_rmat.argtypes = [
            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_uint64, ctypes.c_int, u32p, u32p, i32p, ctypes.c_uint64,
        ]
        _lib = lib
    return _lib


def _p32(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32 if a.dtype == np.uint32 else ctypes.c_int32))


@dataclass
class CSR:
    """Host CSR graph: ``row_ptr`` u32[n+1], ``col`` u32[m], optional ``w`` i32[m]."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray | None = None
    symmetric: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def draw(seed: int, stream: int, index: int) -> int:
    """One counter-based SplitMix64 draw keyed by (seed, stream, index)."""
    return int(_gen().irglgen_draw(seed, stream, index))


def mesh(rows: int, cols: int | None = None, seed: int = 0, del_frac: float = 0.0,
         extra_frac: float = 0.0, radius: int = 8, weights: bool = False) -> CSR:
    """4-neighbour mesh, optionally perturbed (deleted grid edges, extra short-range edges)."""
    cols = rows if cols is None else cols
    n = rows * cols
    extra = int(round(extra_frac * n))
    cap = 4 * n + 2 * extra + 8
    row_ptr = np.empty(n + 1, dtype=np.uint32)
    col = np.empty(cap, dtype=np.uint32)
    w = np.empty(cap, dtype=np.int32) if weights else None
    m = _gen().irglgen_mesh(rows, cols, seed, del_frac, extra_frac, radius, _p32(row_ptr), _p32(col), _p32(w), cap)
    if m < 0:
        raise RuntimeError(f"irglgen_mesh failed with code {m}")
    return CSR(n, row_ptr, col[:m].copy(), None if w is None else w[:m].copy(), symmetric=True,
               meta=dict(kind="mesh", rows=rows, cols=cols, seed=seed, del_frac=del_frac,
                         extra_frac=extra_frac, radius=radius))


def grid(rows: int, cols: int | None = None, seed: int = 0, weights: bool = False) -> CSR:
    return mesh(rows, cols, seed=seed, weights=weights)


def rmat(scale: int, ef: int, a: float = 0.57, b: float = 0.19, c: float = 0.19, seed: int = 0,
         weights: bool = True, nthreads: int = 0) -> CSR:
    """R-MAT graph with self-loops dropped, duplicates merged and rows sorted."""
    n = 1 << scale
    cap = ef * n
    row_ptr = np.empty(n + 1, dtype=np.uint32)
    col = np.empty(cap, dtype=np.uint32)
    w = np.empty(cap, dtype=np.int32) if weights else None
    m = _gen().irglgen_rmat(scale, ef, a, b, c, seed, nthreads, _p32(row_ptr), _p32(col), _p32(w), cap)
    if m < 0:
        raise RuntimeError(f"irglgen_rmat failed with code {m}")
    return CSR(n, row_ptr, col[:m].copy(), None if w is None else w[:m].copy(), symmetric=False,
               meta=dict(kind="rmat", scale=scale, ef=ef, a=a, b=b, c=c, seed=seed))


def csr_from_edges(n: int, src, dst, w=None, symmetric: bool = False) -> CSR:
    """CSR from an explicit edge list, kept as given (multi-edges and self-loops allowed).

    Edges are ordered by (src, dst, position) so the result is deterministic."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    order = np.lexsort((np.arange(src.size), dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.uint32)
    ww = None
    if w is not None:
        ww = np.asarray(w, dtype=np.int32)[order]
    return CSR(n, row_ptr, dst.astype(np.uint32), ww, symmetric=symmetric, meta=dict(kind="edges"))


def sources(g: CSR, k: int, seed: int) -> np.ndarray:
    """k seeded uniform source draws, each redrawn until its out-degree is > 0."""
    deg = g.out_degree()
    if not (deg > 0).any():
        raise ValueError("graph has no vertex with out-degree > 0")
    out = []
    i = 0
    while len(out) < k:
        v = draw(seed, 7, i) % g.n
        i += 1
        if deg[v] > 0:
            out.append(v)
    return np.asarray(out, dtype=np.uint32)


# ----------------------------------------------------------------------------- named workloads

def workload_grid64() -> tuple[CSR, np.ndarray]:
    """64 x 64 4-neighbour grid, source 0 (one query per launch)."""
    g = grid(64, 64, seed=1001)
    return g, np.array([0], dtype=np.uint32)


def workload_rmat20(nsrc: int = 64, scale: int = 20) -> tuple[CSR, np.ndarray]:
    """R-MAT scale 20, edge factor 16, weights [1,100]; seeded sources of out-degree > 0."""
    g = rmat(scale, 16, seed=1002, weights=True)
    return g, sources(g, nsrc, seed=2002)


def workload_mesh(side: int = 4096, weights: bool = False) -> tuple[CSR, np.ndarray]:
    """High-diameter mesh: 1% grid edges deleted, 0.1% vertices with an extra edge (radius 8); source 0."""
    g = mesh(side, side, seed=1003, del_frac=0.01, extra_frac=0.001, radius=8, weights=weights)
    return g, np.array([0], dtype=np.uint32)


def workload_batch(count: int = 256, lo: int = 10, hi: int = 18, ef: int = 8):
    """Batched SSSP instances: R-MAT scale ~U{lo..hi}, edge factor 8, 1-4 seeded sources each."""
    rng = np.random.default_rng(2004)
    scales = rng.integers(lo, hi + 1, size=count)
    nsrcs = rng.integers(1, 5, size=count)
    out = []
    for i in range(count):
        g = rmat(int(scales[i]), ef, seed=1004 * 1000 + i, weights=True)
        out.append((g, sources(g, int(nsrcs[i]), seed=2004 * 1000 + i)))
    return out


def workload_grid_batch(count: int = 32, graphs: int = 16, lo: int = 256, hi: int = 1024):
    """Serving-like batch of high-diameter queries: `graphs` weighted 4-neighbour grids of side U[lo, hi]
    and `count` single-source queries on them, 70% BFS / 30% SSSP, uniform sources.
    Returns [(graph, sources, kind)]; queries on one mesh share its CSR object."""
    rng = np.random.default_rng(2005)
    sides = rng.integers(lo, hi + 1, size=graphs)
    meshes = [mesh(int(sd), int(sd), seed=1005000 + i, weights=True) for i, sd in enumerate(sides)]
    gi = rng.integers(0, graphs, size=count)
    kinds = np.where(rng.random(count) < 0.7, "bfs", "sssp")
    out = []
    for i in range(count):
        g = meshes[gi[i]]
        out.append((g, np.array([int(rng.integers(0, g.n))], np.uint32), str(kinds[i])))
    return out


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 2005) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate over [0, duration)."""
    rng = np.random.default_rng(seed)
    n_est = int(rate_hz * duration_s * 1.2 + 100)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_est))
    while t[-1] < duration_s:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate_hz, size=n_est))])
    return t[t < duration_s]
