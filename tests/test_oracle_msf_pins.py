"""Pins for the oracle's minimum spanning forest (Kruskal under the key
(w, min(u,v), max(u,v))), independent of the oracle's own code (CPU only):

  * brute force over every edge subset of tiny graphs: the forest that spans
    every component and minimises sum(2**rank(key)) is the unique minimum
    spanning forest under the key order; its plain weight is the minimum;
  * independent libraries: scipy.sparse.csgraph.minimum_spanning_tree (weight)
    and networkx's Prim (edge set, on graphs with distinct weights);
  * closed forms: path, star, K_n with w(i, j) = i + j (the star at 0), two
    disjoint copies, unit-weight grid, empty and one-vertex graphs;
  * the cycle property on every non-forest edge of medium graphs;
  * planted mistakes in a copy of oracle.c fail at least one of these pins.
"""
from __future__ import annotations

import ctypes
import itertools
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

nx = pytest.importorskip("networkx")


def _sym_graph(n, us, vs, ws):
    """Symmetric CSR with each undirected edge in both directions (weights shared)."""
    us, vs, ws = np.asarray(us, np.int64), np.asarray(vs, np.int64), np.asarray(ws, np.int64)
    return inputs.csr_from_edges(n, np.concatenate([us, vs]), np.concatenate([vs, us]), np.concatenate([ws, ws]),
                                 symmetric=True)


def _triples(g):
    """Distinct undirected keys (w, lo, hi) of a CSR graph, self-loops dropped."""
    out = set()
    for u in range(g.n):
        for e in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            v = int(g.col[e])
            if v != u:
                out.add((int(g.w[e]), min(u, v), max(u, v)))
    return sorted(out)


def _components(n, triples):
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((a, b) for _, a, b in triples)
    return nx.number_connected_components(G)


def _as_keys(edges):
    return [(int(w), int(u), int(v)) for u, v, w in edges]


def brute_force_msf(g):
    T = _triples(g)
    rank = {t: i for i, t in enumerate(T)}
    k = g.n - _components(g.n, T)
    best, best_cost, best_w = None, None, None
    for sub in itertools.combinations(T, k):
        F = nx.Graph()
        F.add_nodes_from(range(g.n))
        F.add_edges_from((a, b) for _, a, b in sub)
        if F.number_of_edges() != k or not nx.is_forest(F):
            continue
        cost = sum(1 << rank[t] for t in sub)
        wsum = sum(t[0] for t in sub)
        if best_cost is None or cost < best_cost:
            best, best_cost = sorted(sub), cost
        best_w = wsum if best_w is None else min(best_w, wsum)
    return best, best_w


def test_msf_brute_force_tiny():
    rng = np.random.default_rng(81)
    done = 0
    while done < 120:
        n = int(rng.integers(1, 7))
        p = float(rng.choice([0.3, 0.6]))
        a, b = np.nonzero(np.triu(rng.random((n, n)) < p, 1))
        w = rng.integers(0, 4, size=a.size)  # small weights: many ties between different edges
        # parallel copies (same or heavier weight) and self-loops
        if a.size:
            k = int(rng.integers(0, 3))
            pick = rng.integers(0, a.size, size=k)
            a, b = np.concatenate([a, a[pick]]), np.concatenate([b, b[pick]])
            w = np.concatenate([w, w[pick] + rng.integers(0, 2, size=k)])
        a, b, w = np.concatenate([a, [0]]), np.concatenate([b, [0]]), np.concatenate([w, [1]])
        g = _sym_graph(n, a, b, w)
        if len(_triples(g)) > 12:
            continue
        edges, total = oracle.msf(g.n, g.row_ptr, g.col, g.w)
        want, want_w = brute_force_msf(g)
        assert _as_keys(edges) == want
        assert total == (want_w or 0)
        done += 1


def test_msf_vs_scipy_and_networkx():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    graphs = [inputs.mesh(60, 50, seed=82, del_frac=0.05, extra_frac=0.01, weights=True)]
    r = inputs.rmat(11, 8, seed=83, weights=True)
    u = np.repeat(np.arange(r.n), np.diff(r.row_ptr.astype(np.int64)))
    graphs.append(_sym_graph(r.n, u, r.col, r.w))
    for g in graphs:
        edges, total = oracle.msf(g.n, g.row_ptr, g.col, g.w)
        T = _triples(g)
        # scipy: weight of a minimum spanning forest (weights >= 1, min over parallel copies)
        best = {}
        for w, a, b in T:
            best[(a, b)] = min(best.get((a, b), w), w)
        rows = np.array([a for a, _ in best], np.int64)
        cols = np.array([b for _, b in best], np.int64)
        vals = np.array(list(best.values()), np.float64)
        M = sp.csr_matrix((vals, (rows, cols)), shape=(g.n, g.n))
        assert total == int(round(csgraph.minimum_spanning_tree(M).sum()))
        assert len(edges) == g.n - _components(g.n, T)
    # distinct weights: the forest is unique by weight alone, so networkx's Prim must give the same edges
    rng = np.random.default_rng(84)
    n = 400
    a, b = np.nonzero(np.triu(rng.random((n, n)) < 0.01, 1))
    w = rng.permutation(a.size) + 1
    g = _sym_graph(n, a, b, w)
    edges, _ = oracle.msf(g.n, g.row_ptr, g.col, g.w)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_weighted_edges_from(zip(a.tolist(), b.tolist(), w.tolist()))
    F = nx.minimum_spanning_edges(G, algorithm="prim", data=True)
    want = sorted((int(d["weight"]), min(x, y), max(x, y)) for x, y, d in F)
    assert _as_keys(edges) == want


def test_msf_closed_forms():
    n = 50
    path = _sym_graph(n, np.arange(n - 1), np.arange(1, n), np.arange(n - 1) % 5 + 1)
    e, t = oracle.msf(path.n, path.row_ptr, path.col, path.w)
    assert len(e) == n - 1 and t == int((np.arange(n - 1) % 5 + 1).sum())
    star = _sym_graph(n, np.zeros(n - 1, int), np.arange(1, n), np.full(n - 1, 7))
    e, t = oracle.msf(star.n, star.row_ptr, star.col, star.w)
    assert len(e) == n - 1 and t == 7 * (n - 1) and set(e[:, 0].tolist()) == {0}
    k = 12
    a, b = np.nonzero(np.triu(np.ones((k, k)), 1))
    kn = _sym_graph(k, a, b, a + b)
    e, t = oracle.msf(kn.n, kn.row_ptr, kn.col, kn.w)
    assert _as_keys(e) == [(j, 0, j) for j in range(1, k)] and t == k * (k - 1) // 2
    two = _sym_graph(2 * n, np.concatenate([np.arange(n - 1), n + np.arange(n - 1)]),
                     np.concatenate([np.arange(1, n), n + np.arange(1, n)]), np.ones(2 * (n - 1), int))
    e, t = oracle.msf(two.n, two.row_ptr, two.col, two.w)
    assert len(e) == 2 * (n - 1) and t == 2 * (n - 1)
    grid = inputs.grid(20)
    e, t = oracle.msf(grid.n, grid.row_ptr, grid.col, np.ones(grid.m, np.int32))
    assert len(e) == grid.n - 1 and t == grid.n - 1
    for g in (inputs.csr_from_edges(5, [], [], []), inputs.csr_from_edges(1, [], [], []),
              inputs.csr_from_edges(3, [0, 2], [0, 2], [4, 4])):
        e, t = oracle.msf(g.n, g.row_ptr, g.col, np.zeros(g.m, np.int32) if g.w is None else g.w)
        assert len(e) == 0 and t == 0


def test_msf_cycle_property():
    g = inputs.mesh(25, 21, seed=85, del_frac=0.1, extra_frac=0.05, weights=True)
    edges, _ = oracle.msf(g.n, g.row_ptr, g.col, g.w)
    F = nx.Graph()
    F.add_nodes_from(range(g.n))
    for u, v, w in edges:
        F.add_edge(int(u), int(v), key=(int(w), int(u), int(v)))
    assert nx.is_forest(F)
    chosen = set(_as_keys(edges))
    for key in _triples(g):
        if key in chosen:
            continue
        w, a, b = key
        # every other edge closes a cycle of strictly lighter keys (it spans no new pair)
        path = nx.shortest_path(F, a, b)
        assert all(F.edges[x, y]["key"] < key for x, y in zip(path, path[1:]))


MSF_MUTANTS = {
    "msf_weight_order_reversed": ("if (a->w != b->w) return a->w < b->w ? -1 : 1;",
                                  "if (a->w != b->w) return a->w > b->w ? -1 : 1;"),
    "msf_tie_break_dropped": ("if (a->u != b->u) return a->u < b->u ? -1 : 1;", "if (0) return 0;"),
    "msf_cycle_edge_kept": ("if (a == b) continue; /* closes a cycle", "if (0) continue; /* closes a cycle"),
    "msf_union_skipped": ("parent[a > b ? a : b] = a < b ? a : b;", "parent[a] = a;"),
    "msf_endpoints_swapped": ("edges[k].u = u < v ? u : v;", "edges[k].u = u < v ? v : u;"),
}


@pytest.mark.parametrize("name", sorted(MSF_MUTANTS))
def test_msf_planted_mistakes_are_caught(tmp_path, name, monkeypatch):
    old, new = MSF_MUTANTS[name]
    text = (Path(oracle.__file__).parent / "oracle.c").read_text()
    assert text.count(old) == 1, name
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(src)], check=True)
    lib = ctypes.CDLL(str(so))
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_msf.restype = ctypes.c_int
    lib.oracle_msf.argtypes = [ctypes.c_uint32, u32p, u32p, i32p, u32p, u32p, i32p, u32p,
                               ctypes.POINTER(ctypes.c_uint64)]
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = False
    for test in (test_msf_closed_forms, test_msf_brute_force_tiny, test_msf_cycle_property):
        try:
            test()
        except (AssertionError, ValueError, KeyError, nx.NetworkXException):
            caught = True
            break
    assert caught, f"mutant {name} survived every pin"
