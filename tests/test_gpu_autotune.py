"""Autotuning (block-level choices, CTA-local sub-rounds, near-far delta): the
search returns a valid tuning whose runs stay bit-exact against the oracle, for
one graph and for a batch. Results never depend on the tuning; only time does."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300.api import Context

    c = Context(0, torch.cuda.Stream())
    yield c
    c.close()


def _valid(t: dict) -> None:
    assert t["cta_size"] in (128, 256, 512, 1024)
    assert t["warp_thresh"] <= t["cta_thresh"]
    assert t["flags"] in (0, 4 << 8, 15 << 8, 2)  # sub-rounds, or direction-optimising BFS
    assert t["max_blocks"] in (0, 1, 2, 8, 32) or t["max_blocks"] >= 100  # or one CTA per SM


@pytest.mark.parametrize("kind,make,srcs", [
    ("bfs", lambda: inputs.grid(64, 64), [0]),
    ("sssp", lambda: inputs.mesh(96, 80, seed=4, del_frac=0.02, extra_frac=0.002, weights=True), [5, 4000]),
    ("sssp", lambda: inputs.rmat(12, 8, seed=9, weights=True), None),
    ("cc", lambda: inputs.mesh(70, 50, seed=6, del_frac=0.05), None),
])
def test_autotune_single_graph(ctx, kind, make, srcs):
    g = make()
    if srcs is None and kind != "cc":
        srcs = inputs.sources(g, 3, seed=11)
    s = None if srcs is None else np.asarray(srcs, np.uint32)
    d = ctx.load(g, symmetric=kind == "cc" or None)
    t, ms = ctx.autotune(kind, d, s, reps=2)
    _valid(t)
    assert ms > 0
    if kind != "sssp":
        assert t["delta"] == 0
    if kind == "cc":
        assert t["flags"] == 0  # the sub-round axis is searched for BFS and SSSP only
    out, st = ctx.run_host(kind, d, s, tuning=t)
    np.testing.assert_array_equal(out, oracle.run(kind, g, s), err_msg=str(t))
    d.close()


def test_autotune_batch(ctx):
    from paper_1607_05707_gb300.api import Batch

    graphs = [inputs.rmat(10, 8, seed=40 + i, weights=True) for i in range(6)] + [inputs.grid(40, 30, weights=True)]
    b = Batch(ctx)
    dgs, qs = [], []
    for i, g in enumerate(graphs):
        dg = ctx.load(g)
        dgs.append(dg)
        kind = "bfs" if i % 2 else "sssp"
        s = inputs.sources(g, 2, seed=70 + i)
        qs.append((b.add(kind, dg, s), kind, g, s))
    b.prepare()
    t, ms = b.autotune(reps=2)
    _valid(t)
    assert ms > 0
    from paper_1607_05707_gb300 import irgl as C

    assert C.irgl_batch_info(b.handle)["waves"] >= 1  # left prepared with the chosen wave budget
    b.run()
    for q, kind, g, s in qs:
        got, _ = b.result(q)
        np.testing.assert_array_equal(got, oracle.run(kind, g, s), err_msg=f"{q} {kind} {t}")
    b.close()
    for dg in dgs:
        dg.close()
