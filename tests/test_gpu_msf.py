"""Minimum spanning forest (Boruvka as an outlined multi-kernel Pipe with
Atomic component locks and a Retry worklist) against the Kruskal oracle.

The forest is unique under the key (w, min(u,v), max(u,v)), so the GPU's edge
set, mapped to keys, must equal the oracle's exactly (parallel copies of an
edge have the same key), under every lock form, both modes and every CTA size.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu

LOCKS = ("blocking", "ticket", "retry")
MODES = ("persistent", "per_launch")


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300.api import Context

    c = Context(0)
    yield c
    c.close()


def sym(n, us, vs, ws):
    us, vs, ws = np.asarray(us, np.int64), np.asarray(vs, np.int64), np.asarray(ws, np.int64)
    return inputs.csr_from_edges(n, np.concatenate([us, vs]), np.concatenate([vs, us]), np.concatenate([ws, ws]),
                                 symmetric=True)


def keys_of(g, idx):
    """CSR edge indices -> sorted keys (w, lo, hi)."""
    idx = np.asarray(idx, np.int64)
    u = np.searchsorted(g.row_ptr.astype(np.int64), idx, side="right") - 1
    v = g.col.astype(np.int64)[idx]
    w = g.w.astype(np.int64)[idx]
    return sorted(zip(w.tolist(), np.minimum(u, v).tolist(), np.maximum(u, v).tolist()))


def check(ctx, g, dg, mode="persistent", lock="blocking", tuning=None):
    got, st = ctx.msf(dg, mode=mode, lock=lock, tuning=tuning)
    edges, total = oracle.msf(g.n, g.row_ptr, g.col, g.w)
    want = sorted((int(w), int(u), int(v)) for u, v, w in edges)
    have = keys_of(g, got)
    assert have == want, f"{mode}/{lock}/{tuning}: {len(have)} edges vs {len(want)}"
    assert st["weight"] == total and st["edges"] == len(want)
    assert len(set(got.tolist())) == len(got)  # no edge recorded twice
    return st


def rmat_sym(scale, ef, seed):
    r = inputs.rmat(scale, ef, seed=seed, weights=True)
    u = np.repeat(np.arange(r.n), np.diff(r.row_ptr.astype(np.int64)))
    return sym(r.n, u, r.col, r.w)


def test_tiny_graphs_every_lock_and_mode(ctx):
    rng = np.random.default_rng(91)
    for trial in range(24):
        n = int(rng.integers(1, 90))
        a, b = np.nonzero(np.triu(rng.random((n, n)) < float(rng.choice([0.02, 0.1, 0.4])), 1))
        w = rng.integers(0, 6, size=a.size)  # ties between different edges, zero weights
        if a.size:  # parallel copies and self-loops
            pick = rng.integers(0, a.size, size=int(rng.integers(0, 4)))
            a, b = np.concatenate([a, a[pick]]), np.concatenate([b, b[pick]])
            w = np.concatenate([w, w[pick] + rng.integers(0, 2, size=pick.size)])
        a, b, w = np.concatenate([a, [n - 1]]), np.concatenate([b, [n - 1]]), np.concatenate([w, [2]])
        g = sym(n, a, b, w)
        dg = ctx.load(g)
        for mode in MODES:
            for lock in LOCKS:
                check(ctx, g, dg, mode, lock)
        dg.close()


def test_special_shapes(ctx):
    n = 300
    path = sym(n, np.arange(n - 1), np.arange(1, n), np.arange(n - 1) % 7)
    star = sym(2001, np.zeros(2000, int), np.arange(1, 2001), np.full(2000, 3))  # one hub: every lock on it
    k = 40
    a, b = np.nonzero(np.triu(np.ones((k, k)), 1))
    kn = sym(k, a, b, a + b)
    two = sym(2 * n, np.concatenate([np.arange(n - 1), n + np.arange(n - 1)]),
              np.concatenate([np.arange(1, n), n + np.arange(1, n)]), np.ones(2 * (n - 1), int))
    iso = sym(10, [0, 8], [1, 9], [5, 5])
    empty = inputs.csr_from_edges(7, [], [], [], symmetric=True)
    one = inputs.csr_from_edges(1, [], [], [], symmetric=True)
    for g in (path, star, kn, two, iso, empty, one):
        if g.w is None:
            g.w = np.zeros(g.m, np.int32)
        dg = ctx.load(g)
        for lock in LOCKS:
            for tuning in (None, dict(cta_size=128, max_blocks=3), dict(cta_size=1024)):
                check(ctx, g, dg, "persistent", lock, tuning)
        check(ctx, g, dg, "per_launch", "retry")
        dg.close()


@pytest.mark.parametrize("lock", LOCKS)
def test_meshes_and_power_law(ctx, lock):
    m = inputs.mesh(300, 257, seed=92, del_frac=0.02, extra_frac=0.002, weights=True)
    dm = ctx.load(m)
    for tuning in (None, dict(cta_size=256), dict(cta_size=512, max_blocks=40)):
        check(ctx, m, dm, "persistent", lock, tuning)
    check(ctx, m, dm, "per_launch", lock)
    dm.close()
    r = rmat_sym(15, 8, 93)  # hubs: a giant component whose vertices all contend for one record
    dr = ctx.load(r)
    st = check(ctx, r, dr, "persistent", lock)
    assert st["iterations"] <= 32
    if lock == "retry":
        assert st["locks"] > 0
    check(ctx, r, dr, "per_launch", lock)
    dr.close()


def test_mesh2048_full(ctx):
    g = inputs.mesh(2048, 2048, seed=94, del_frac=0.01, extra_frac=0.001, weights=True)
    dg = ctx.load(g, validate=False)
    for lock in LOCKS:
        st = check(ctx, g, dg, "persistent", lock)
        assert st["launches"] == 1
    dg.close()


def test_errors_and_lock_timeout(ctx):
    from paper_1607_05707_gb300 import irgl as C

    g = rmat_sym(10, 8, 95)
    dg = ctx.load(g)
    # a component lock that starts held and is never released: every wait on it
    # ends at the 20 ms limit with a status (blocking and ticket forms) and the
    # retry form stops retrying at the same limit
    hub = int(np.argmax(np.diff(g.row_ptr.astype(np.int64))))
    ctx.debug_set(1, 20000)
    ctx.debug_set(6, hub)
    try:
        for mode in MODES:
            for lock in LOCKS:
                with pytest.raises(C.IrglError) as ei:
                    ctx.msf(dg, mode=mode, lock=lock)
                assert ei.value.status == C.IRGL_ERR_LOCK_TIMEOUT, (mode, lock)
    finally:
        ctx.debug_set(6, -1)
        ctx.debug_set(1, 0)
    for lock in LOCKS:
        check(ctx, g, dg, "persistent", lock)  # the context is usable afterwards
    # a graph not loaded as symmetric, a graph without weights
    d = inputs.rmat(8, 4, seed=96, weights=True)
    dd = ctx.load(d, symmetric=False)
    with pytest.raises(C.IrglError) as ei:
        ctx.msf(dd)
    assert ei.value.status == C.IRGL_ERR_NOT_SYMMETRIC
    dd.close()
    gu = inputs.grid(8)
    dgu = ctx.load(gu)
    with pytest.raises(C.IrglError) as ei:
        ctx.msf(dgu)
    assert ei.value.status == C.IRGL_ERR_INVALID_ARG
    dgu.close()
    dg.close()
