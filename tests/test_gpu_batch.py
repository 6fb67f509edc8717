"""Batched multi-instance launches vs the oracle (bit-exact), with and without
CUDA-graph replay, under several schedules; per-instance termination rounds."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300.api import Context

    c = Context(0, torch.cuda.Stream())
    yield c
    c.close()


def _instances():
    rng = np.random.default_rng(17)
    out = []
    for i in range(24):
        g = inputs.rmat(int(rng.integers(8, 14)), 8, seed=500 + i, weights=True)
        srcs = inputs.sources(g, int(rng.integers(1, 5)), seed=600 + i)
        out.append(("sssp" if i % 3 else "bfs", g, srcs))
    m = inputs.mesh(60, 45, seed=3, del_frac=0.05, extra_frac=0.01, weights=True)
    out.append(("cc", m, None))
    out.append(("bfs", m, np.array([0], np.uint32)))
    out.append(("sssp", m, np.array([17, 2000], np.uint32)))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("tuning", [None, dict(cta_size=128, warp_thresh=4, cta_thresh=64, chunk=2),
                                    dict(cta_size=512, warp_thresh=1 << 30, cta_thresh=1 << 30, max_blocks=5),
                                    dict(cta_size=256, flags=8)])  # two-array arena (IRGL_TUNE_NO_PACKED)
def test_batch_matches_oracle(ctx, use_graph, tuning):
    from paper_1607_05707_gb300.api import Batch

    inst = _instances()
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 64)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    info = b.prepare(tuning, use_cuda_graph=use_graph)
    if use_graph:
        assert info["graph_captured"], "cooperative launch was not captured in a CUDA graph"
    for rep in range(2):  # replays recompute everything from the sources
        st = b.run()
        assert st["rounds"] >= 1 and st["device_ms"] > 0
        for q, (k, g, s) in enumerate(inst):
            got, rounds = b.result(q)
            want = oracle.run(k, g, s)
            np.testing.assert_array_equal(got, want, err_msg=f"query {q} ({k}) rep {rep}")
            if k == "bfs":
                assert rounds == int(want[want != INF].max()) + 1
    b.close()
    for dg in graphs:
        dg.close()


def _waves(sizes, budget):
    # consecutive queries while their 8-byte packed words fit the budget
    w, acc = 0, None
    for n in sizes:
        if acc is None or acc + 8 * n > budget:
            w, acc = w + 1, 0
        acc += 8 * n
    return w


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("wave_bytes", [1, 8 * 3000, 8 * 20000, 0, (1 << 64) - 1])
def test_batch_waves_match_oracle(ctx, use_graph, wave_bytes):
    """Queries split into consecutive waves (one persistent launch each) give the
    same results, and each query's rounds still count its own rounds."""
    from paper_1607_05707_gb300.api import Batch

    inst = _instances()
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 64)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    info = b.prepare(None, use_cuda_graph=use_graph, wave_bytes=wave_bytes)
    waves = _waves([g.n for _, g, _ in inst], wave_bytes or (1 << 64) - 1)  # 0: one wave
    assert info["waves"] == waves
    if wave_bytes == 1:
        assert waves == len(inst)
    for rep in range(2):
        st = b.run()
        assert st["launches"] == 3 * waves + 1
        total = 0
        for q, (k, g, s) in enumerate(inst):
            got, rounds = b.result(q)
            want = oracle.run(k, g, s)
            np.testing.assert_array_equal(got, want, err_msg=f"query {q} ({k}) rep {rep} waves {waves}")
            if k == "bfs":
                assert rounds == int(want[want != INF].max()) + 1
            total = max(total, rounds)
        assert st["rounds"] >= total
    b.close()
    for dg in graphs:
        dg.close()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("delta,wave_bytes", [(1, 0), (8, 0), (100, 0), (1000, 0), (64, 8 * 20000)])
def test_batch_near_far_matches_oracle(ctx, use_graph, delta, wave_bytes):
    """Per-query near-far for the SSSP queries of a mixed batch: same results, and
    BFS queries keep their round counts."""
    from paper_1607_05707_gb300.api import Batch

    inst = _instances()
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 64)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    b.prepare(dict(delta=delta), use_cuda_graph=use_graph, wave_bytes=wave_bytes)
    for rep in range(2):
        b.run()
        for q, (k, g, s) in enumerate(inst):
            got, rounds = b.result(q)
            want = oracle.run(k, g, s)
            np.testing.assert_array_equal(got, want, err_msg=f"query {q} ({k}) delta {delta} rep {rep}")
            if k == "bfs":
                assert rounds == int(want[want != INF].max()) + 1
    b.close()
    for dg in graphs:
        dg.close()


def test_batch_near_far_scans_fewer_edges(ctx):
    """SSSP on a weighted mesh: label-correcting rounds re-relax most edges many
    times; with per-query near-far the same 8 queries scan far fewer."""
    from paper_1607_05707_gb300.api import Batch

    g = inputs.mesh(160, 150, seed=11, del_frac=0.01, extra_frac=0.001, weights=True)
    dg = ctx.load(g)
    srcs = inputs.sources(g, 8, seed=12)
    scanned = {}
    for delta in (0, 128):
        b = Batch(ctx, 8)
        for s in srcs:
            b.add("sssp", dg, [int(s)])
        b.prepare(dict(delta=delta))
        st = b.run()
        scanned[delta] = st["edges_scanned"]
        for q, s in enumerate(srcs):
            np.testing.assert_array_equal(b.result(q)[0], oracle.run("sssp", g, np.array([s], np.uint32)))
        b.close()
    assert scanned[128] * 4 < scanned[0], scanned
    dg.close()


def test_batch_results_one_copy(ctx):
    from paper_1607_05707_gb300.api import Batch

    inst = _instances()[:10]
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 16)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    b.prepare(wave_bytes=8 * 4000)
    b.run()
    res = b.results()
    assert len(res) == len(inst)
    for q, (k, g, s) in enumerate(inst):
        np.testing.assert_array_equal(res[q], oracle.run(k, g, s), err_msg=f"query {q}")
        np.testing.assert_array_equal(res[q], b.result(q)[0])
    with pytest.raises(ValueError):
        b.results(np.empty(3, dtype=np.uint32))
    b.close()
    for dg in graphs:
        dg.close()


def test_batch_alone_equals_mix(ctx):
    from paper_1607_05707_gb300.api import Batch, as_u32

    inst = _instances()[:8]
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 16)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    b.prepare()
    b.run()
    for q, ((k, g, s), dg) in enumerate(zip(inst, graphs)):
        alone, _ = ctx.run(k, dg, s)
        got, _ = b.result(q)
        np.testing.assert_array_equal(got, as_u32(alone)[: g.n])
    b.close()


def test_batch_config_sample(ctx):
    # a sample of the 256-instance workload (R-MAT scale 10..18, edge factor 8, 1-4 sources, SSSP)
    from paper_1607_05707_gb300.api import Batch

    inst = inputs.workload_batch(count=20)
    graphs = [ctx.load(g, validate=False) for g, _ in inst]
    b = Batch(ctx, 32)
    for (g, s), dg in zip(inst, graphs):
        b.add("sssp", dg, s)
    b.prepare()
    b.run()
    for q, (g, s) in enumerate(inst):
        got, _ = b.result(q)
        np.testing.assert_array_equal(got, oracle.sssp(g.n, g.row_ptr, g.col, g.w, s))
    b.close()


@pytest.mark.parametrize("wave_mb", [0, 16])
def test_batch256_full_matches_oracle(ctx, wave_mb):
    """The whole 256-instance batched SSSP workload (R-MAT scale 10..18, edge factor 8,
    1-4 sources), one CUDA-graph replay, every instance equal to the oracle's Dijkstra:
    in one wave, and in waves of 16 MB of packed state each (many launches)."""
    from paper_1607_05707_gb300.api import Batch

    inst = inputs.workload_batch(count=256)
    graphs = [ctx.load(g, validate=False) for g, _ in inst]
    b = Batch(ctx, 256)
    for (g, s), dg in zip(inst, graphs):
        b.add("sssp", dg, s)
    b.prepare(use_cuda_graph=True, wave_bytes=(wave_mb << 20) if wave_mb else None)
    b.run()
    for q, (g, s) in enumerate(inst):
        got, _ = b.result(q)
        np.testing.assert_array_equal(got, oracle.sssp(g.n, g.row_ptr, g.col, g.w, s), err_msg=f"instance {q}")
    b.close()
    for dg in graphs:
        dg.close()


def test_trace_records_rounds(ctx):
    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import as_u32, trace

    g, srcs = inputs.workload_grid64()
    dg = ctx.load(g)
    C.irgl_trace_enable(ctx.handle, 1024)
    out, st = ctx.run("bfs", dg, srcs)
    t, a, o = trace(ctx)
    C.irgl_trace_enable(ctx.handle, 0)
    # prologue record, one record per round, epilogue record
    assert len(t) == st["rounds"] + 2 == 129
    assert (np.diff(t.astype(np.int64)) >= 0).all()
    assert 0 < int(o[0]) < 10**9  # prologue duration (ns)
    # round r pops the r-th anti-diagonal of the 64x64 grid (from the corner): min(r+1, 127-r) vertices
    r = np.arange(0, 127)
    np.testing.assert_array_equal(a[1:-1], np.minimum(r + 1, 127 - r))
    assert o[-2] == 0
    assert a[-1] == 0xFFFFFFFF and o[-1] == 0xFFFFFFFF
    dg.close()


def test_trace_phase_records(ctx):
    """Phase records of a grid-wide persistent SSSP: per round the first phase
    ends (earliest <= latest CTA) before CTA 0 leaves the first barrier, the big
    phase (when a big list was published) after it, all within the round; the
    big lists' edges are at most the edges the launch scanned, and two launches
    in a row each leave their own records."""
    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import as_u32, trace

    g = inputs.rmat(16, 16, seed=71, weights=True)
    dg = ctx.load(g)
    src = inputs.sources(g, 2, seed=72)
    C.irgl_trace_enable(ctx.handle, 256)
    mask = (1 << 64) - 1
    for s in src:
        out, st = ctx.run("sssp", dg, np.array([s], np.uint32), tuning=dict(flags=0x40))
        np.testing.assert_array_equal(as_u32(out)[: g.n], oracle.run("sssp", g, np.array([s], np.uint32)))
        t, a, o = trace(ctx)
        ph = C.irgl_trace_phases(ctx.handle)
        assert len(ph) == st["rounds"] > 1
        big_edges = 0
        for r in range(st["rounds"]):
            w = [int(x) for x in ph[r]]
            start, end = int(t[r]), int(t[r + 1])
            if r == 0 and (~w[0] & mask) < start:
                start -= int(o[0])  # round 0 ran inside the prologue: from the kernel's start
            first, last = ~w[0] & mask, w[1]
            assert start <= first <= last <= w[2] <= end, (r, start, first, last, w[2], end)
            if w[3]:
                big_edges += w[3] & ((1 << 40) - 1)
                assert w[2] <= (~w[4] & mask) <= w[5] <= w[6] <= end, (r, w)
            else:
                assert w[4] == w[5] == w[6] == 0
        assert big_edges <= st["edges_scanned"]
    C.irgl_trace_enable(ctx.handle, 0)
    dg.close()


@pytest.mark.parametrize("delta", [0, 32])
def test_batch_config_sample_near_far(ctx, delta):
    """A sample of the 256-instance R-MAT workload batched with and without per-query near-far."""
    from paper_1607_05707_gb300.api import Batch

    inst = inputs.workload_batch(count=16)
    graphs = [ctx.load(g, validate=False) for g, _ in inst]
    b = Batch(ctx, 16)
    for (g, s), dg in zip(inst, graphs):
        b.add("sssp", dg, s)
    b.prepare(dict(delta=delta))
    b.run()
    for q, (g, s) in enumerate(inst):
        np.testing.assert_array_equal(b.result(q)[0], oracle.sssp(g.n, g.row_ptr, g.col, g.w, s), err_msg=f"{q}")
    b.close()
    for dg in graphs:
        dg.close()


@pytest.mark.parametrize("delta", [0, 512])
def test_grid_batch_matches_oracle(ctx, delta):
    """The serving-like grid batch (BFS and SSSP queries sharing a few weighted grids), smaller sides."""
    from paper_1607_05707_gb300.api import Batch

    inst = inputs.workload_grid_batch(count=12, graphs=4, lo=64, hi=220)
    loaded = {}
    for g, _, _ in inst:
        if id(g) not in loaded:
            loaded[id(g)] = ctx.load(g)
    b = Batch(ctx, 16)
    for g, s, k in inst:
        b.add(k, loaded[id(g)], s)
    b.prepare(dict(delta=delta))
    for rep in range(2):
        b.run()
        for q, (g, s, k) in enumerate(inst):
            got, rounds = b.result(q)
            want = oracle.run(k, g, s)
            np.testing.assert_array_equal(got, want, err_msg=f"query {q} ({k}) delta {delta} rep {rep}")
            if k == "bfs":
                assert rounds == int(want[want != INF].max()) + 1
    b.close()
    for dg in loaded.values():
        dg.close()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("tuning", [dict(flags=15 << 8), dict(flags=4 << 8, delta=512),
                                    dict(flags=(15 << 8) | 0x20, cta_size=256, delta=64),
                                    dict(flags=2 << 8, cta_size=1024, warp_thresh=2, cta_thresh=8)])
def test_batch_sub_rounds_match_oracle(ctx, use_graph, tuning):
    """CTA-local sub-rounds in the batched kernel (BFS as unit-weight relaxation,
    a local pop clearing its round stamp): grids, meshes and R-MAT instances
    mixed, with and without per-query near-far; every result equals the
    oracle's and a grid BFS needs fewer global rounds than levels."""
    from paper_1607_05707_gb300.api import Batch

    inst = [(g, s, k) for g, s, k in inputs.workload_grid_batch(count=10, graphs=3, lo=64, hi=200)]
    inst += [(g, s, k) for k, g, s in _instances()[:9] if k != "cc"]
    m = inputs.mesh(90, 70, seed=5, del_frac=0.02, extra_frac=0.01, weights=True)
    inst += [(m, np.array([0], np.uint32), "bfs"), (m, np.array([11], np.uint32), "sssp")]
    loaded = {}
    for g, _, _ in inst:
        if id(g) not in loaded:
            loaded[id(g)] = ctx.load(g)
    b = Batch(ctx, 32)
    for g, s, k in inst:
        b.add(k, loaded[id(g)], s)
    b.prepare(tuning, use_cuda_graph=use_graph)
    for rep in range(2):
        b.run()
        for q, (g, s, k) in enumerate(inst):
            got, rounds = b.result(q)
            want = oracle.run(k, g, s)
            np.testing.assert_array_equal(got, want, err_msg=f"query {q} ({k}) {tuning} rep {rep}")
            if k == "bfs":
                levels = int(want[want != INF].max()) + 1
                assert 1 <= rounds <= levels
                if g is m and (tuning["flags"] >> 8) >= 4:
                    assert rounds < levels
    b.close()
    for dg in loaded.values():
        dg.close()


@pytest.mark.parametrize("tuning", [dict(max_blocks=2, warp_thresh=4, cta_thresh=1024),
                                    dict(max_blocks=2, warp_thresh=4, cta_thresh=1024, delta=64),
                                    dict(max_blocks=3, cta_size=256, warp_thresh=8, cta_thresh=4096, flags=4 << 8)])
def test_batch_warp_bin_matches_oracle(ctx, tuning):
    """The warp bin of the batched kernel (lists of warp_thresh..cta_thresh edges,
    used when a round's frontier is larger than the grid: a grid of two or three
    CTAs makes every round that large) lowers each query's own packed words: all
    results equal the oracle's, with and without near-far and sub-rounds."""
    from paper_1607_05707_gb300.api import Batch

    inst = [(k, g, s) for k, g, s in _instances() if k != "cc"]
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 64)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    b.prepare(tuning)
    for rep in range(2):
        b.run()
        for q, (k, g, s) in enumerate(inst):
            got, _ = b.result(q)
            np.testing.assert_array_equal(got, oracle.run(k, g, s), err_msg=f"query {q} ({k}) {tuning} rep {rep}")
    b.close()
    for dg in graphs:
        dg.close()


@pytest.mark.parametrize("tuning", [dict(defer_deg=1, defer_delta=1), dict(cta_size=256, defer_deg=8, defer_delta=4),
                                    dict(max_blocks=3, warp_thresh=4, cta_thresh=64, defer_deg=4, defer_delta=1),
                                    dict(flags=0x1000)])
def test_batch_deferred_expansion_matches_oracle(ctx, tuning):
    """SSSP queries of a batch defer long lists whose vertex is above the query's
    smallest pushed distance of the last round + defer_delta (every list of at
    least one edge with defer_deg = 1); with BFS and CC queries in the same
    batch, every result equals the oracle's, over two runs."""
    from paper_1607_05707_gb300.api import Batch

    inst = _instances()
    graphs = [ctx.load(g) for _, g, _ in inst]
    b = Batch(ctx, 64)
    for (k, g, s), dg in zip(inst, graphs):
        b.add(k, dg, s)
    b.prepare(tuning)
    for rep in range(2):
        b.run()
        for q, (k, g, s) in enumerate(inst):
            got, _ = b.result(q)
            np.testing.assert_array_equal(got, oracle.run(k, g, s), err_msg=f"query {q} ({k}) {tuning} rep {rep}")
    b.close()
    for dg in graphs:
        dg.close()
