"""GPU parity: the CUDA path through the C-ABI vs the CPU oracle, bit-exact.

Levels, distances and labels are uint32 fixed points, so the comparison is
element-by-element equality (tolerance 0) under every schedule: thread/warp/CTA
thresholds, CTA sizes, chunk sizes, grid sizes and both Iterate modes.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF

MODES = ("persistent", "per_launch")
SCHEDULES = [
    None,
    dict(cta_size=128, warp_thresh=1, cta_thresh=1),          # every list to the whole CTA
    dict(cta_size=256, warp_thresh=1, cta_thresh=1 << 30),    # every list to a warp
    dict(cta_size=512, warp_thresh=1 << 30, cta_thresh=1 << 30),  # every list through the scan bin
    dict(cta_size=1024, warp_thresh=4, cta_thresh=64, chunk=3),
    dict(cta_size=256, warp_thresh=8, cta_thresh=128, chunk=2, max_blocks=3),
    dict(cta_size=128, warp_thresh=16, cta_thresh=512, max_blocks=1),
    dict(cta_size=256, warp_thresh=32, cta_thresh=256, flags=1),  # long lists kept in the CTA bin (no split)
    dict(cta_size=1024, warp_thresh=2, cta_thresh=8),             # most lists split over the grid
    dict(cta_size=128, delta=16),                                 # SSSP near-far schedule
    dict(cta_size=256, warp_thresh=4, cta_thresh=16, delta=1),    # near-far, one distance per bucket
    dict(cta_size=512, delta=100000),                             # near-far bucket wider than any distance
    dict(cta_size=256, flags=4 | 8),      # BFS visited bitmap, SSSP distances and stamps in two arrays
    dict(cta_size=1024, warp_thresh=1 << 30, cta_thresh=1 << 30, flags=8),  # two-array SSSP through the scan bin
    dict(cta_size=512, warp_thresh=4, cta_thresh=32, delta=8),    # near-far through small bins
    dict(cta_size=128, flags=0x10),       # small frontiers through the bins and the big list as well
    dict(cta_size=256, warp_thresh=4, cta_thresh=16, flags=0x10 | 8),  # the same, two-array SSSP
    dict(cta_size=128, flags=0x20),       # lists of 1..4 edges walked by their own lane (thread bin)
    dict(cta_size=128, flags=0x80),       # large frontiers popped in vertex order (dense rounds)
    dict(cta_size=512, warp_thresh=4, cta_thresh=16, flags=0x80 | 0x10),  # dense, no broadcast rounds
    dict(cta_size=512, warp_thresh=8, cta_thresh=64, flags=0x30, delta=16),  # thread bin, no broadcast, near-far
    dict(cta_size=256, defer_deg=1, defer_delta=1),   # SSSP: any vertex above the round's smallest + 1 waits
    dict(cta_size=128, warp_thresh=4, cta_thresh=16, defer_deg=16, defer_delta=8),  # deferred lists, small bins
    dict(cta_size=512, flags=0x1000),     # SSSP expands every pop (no deferred long lists)
]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300.api import Context

    c = Context(0)
    yield c
    c.close()


def run(ctx, kernel, g, dg, srcs, mode="persistent", tuning=None):
    from paper_1607_05707_gb300.api import as_u32

    out, st = ctx.run(kernel, dg, None if kernel.startswith("cc") else srcs, mode=mode, tuning=tuning)
    return as_u32(out)[: g.n], st


NO_SMEM = 0x40  # IRGL_TUNE_NO_SMEM: grid-wide kernels even for graphs that fit in shared memory


def check(ctx, kernel, g, dg, srcs, mode="persistent", tuning=None):
    want = oracle.run("cc" if kernel == "cc_jump" else kernel, g, srcs)
    tunings = [tuning]
    if mode == "persistent" and kernel != "cc_jump" and g.n <= 20000:
        # small graphs run in one CTA with the graph in shared memory by default:
        # check the grid-wide kernels on them as well
        t2 = dict(tuning or {})
        t2["flags"] = int(t2.get("flags", 0)) | NO_SMEM
        tunings.append(t2)
    st0 = None
    for t in tunings:
        got, st = run(ctx, kernel, g, dg, srcs, mode, t)
        if not np.array_equal(got, want):
            bad = np.flatnonzero(got != want)
            raise AssertionError(f"{kernel}/{mode}/{t}: {bad.size} of {g.n} differ; first {bad[:8]} "
                                 f"got {got[bad[:8]]} want {want[bad[:8]]}")
        st0 = st if st0 is None else st0
    return st0


def tiny_graph(rng, n, p, symmetric):
    src, dst = np.nonzero(rng.random((n, n)) < p)
    w = rng.integers(0, 101, size=src.size)
    if src.size:
        k = int(rng.integers(0, 3))
        src = np.concatenate([src, src[:k], [0]])
        dst = np.concatenate([dst, dst[:k], [0]])
        w = np.concatenate([w, w[:k] + 1, [5]])
    if symmetric:
        src, dst, w = np.concatenate([src, dst]), np.concatenate([dst, src]), np.concatenate([w, w])
    return inputs.csr_from_edges(n, src, dst, w, symmetric=symmetric)


# ----------------------------------------------------------------------------- small cases

def test_tiny_random_graphs(ctx):
    rng = np.random.default_rng(3)
    for trial in range(40):
        n = int(rng.integers(1, 200))
        sym = bool(trial % 2)
        g = tiny_graph(rng, n, float(rng.choice([0.01, 0.05, 0.2])), sym)
        dg = ctx.load(g)
        srcs = rng.integers(0, n, size=int(rng.integers(1, 5))).astype(np.uint32)
        for mode in MODES:
            check(ctx, "bfs", g, dg, srcs, mode)
            check(ctx, "sssp", g, dg, srcs, mode)
            if sym:
                check(ctx, "cc", g, dg, srcs, mode)
        if sym:
            check(ctx, "cc_jump", g, dg, srcs, "persistent")
        dg.close()


def test_special_shapes(ctx):
    n = 300
    path = inputs.csr_from_edges(n, np.arange(n - 1), np.arange(1, n), np.arange(1, n) % 7)
    star = inputs.csr_from_edges(2001, np.zeros(2000, int), np.arange(1, 2001), np.full(2000, 3))
    iso = inputs.csr_from_edges(10, [0, 9], [1, 8], [1, 1])
    e = [(0, 1), (1, 2), (2, 0), (2, 3)]
    s = [a for a, b in e] + [b for a, b in e]
    d = [b for a, b in e] + [a for a, b in e]
    two = inputs.csr_from_edges(8, s + [x + 4 for x in s], d + [x + 4 for x in d], np.ones(16), symmetric=True)
    multi = inputs.csr_from_edges(3, [0, 0, 0, 1, 1, 2], [1, 1, 0, 1, 2, 2], [9, 2, 0, 1, 5, 4])
    empty = inputs.csr_from_edges(5, [], [], [])
    one = inputs.csr_from_edges(1, [], [], [])
    for g, srcs in [(path, [0]), (path, [150]), (star, [0]), (star, [7]), (iso, [1]), (iso, [0, 9]),
                    (two, [1]), (multi, [0]), (empty, [3]), (one, [0])]:
        dg = ctx.load(g)
        srcs = np.array(srcs, dtype=np.uint32)
        for mode in MODES:
            for tuning in (None, SCHEDULES[1], SCHEDULES[3]):
                check(ctx, "bfs", g, dg, srcs, mode, tuning)
                check(ctx, "sssp", g, dg, srcs, mode, tuning)
        dg.close()
    for g in (two, empty, one, inputs.csr_from_edges(4, [1, 2], [2, 1], [1, 1], symmetric=True)):
        dg = ctx.load(g, symmetric=True)
        for mode in MODES:
            check(ctx, "cc", g, dg, None, mode)
        check(ctx, "cc_jump", g, dg, None, "persistent")
        dg.close()


def test_grid64_closed_form(ctx):
    g, srcs = inputs.workload_grid64()
    dg = ctx.load(g)
    r, c = np.divmod(np.arange(g.n), 64)
    for mode in MODES:
        got, st = run(ctx, "bfs", g, dg, srcs, mode)
        np.testing.assert_array_equal(got, (r + c).astype(np.uint32))
        assert st["rounds"] == 127
        check(ctx, "cc", g, dg, srcs, mode)
    dg.close()


@pytest.mark.parametrize("tuning", SCHEDULES)
def test_schedule_independence_rmat(ctx, tuning):
    g = inputs.rmat(15, 16, seed=41, weights=True)
    dg = ctx.load(g)
    srcs = inputs.sources(g, 2, seed=42)
    for s in srcs:
        for mode in MODES:
            check(ctx, "bfs", g, dg, np.array([s], np.uint32), mode, tuning)
            check(ctx, "sssp", g, dg, np.array([s], np.uint32), mode, tuning)
    check(ctx, "bfs", g, dg, srcs, "persistent", tuning)
    check(ctx, "sssp", g, dg, srcs, "persistent", tuning)
    dg.close()


@pytest.mark.parametrize("tuning", SCHEDULES[:4])
def test_mesh_bfs_cc(ctx, tuning):
    g = inputs.mesh(300, 257, seed=9, del_frac=0.01, extra_frac=0.001, radius=8, weights=True)
    dg = ctx.load(g)
    for mode in MODES:
        check(ctx, "bfs", g, dg, np.array([0], np.uint32), mode, tuning)
        check(ctx, "cc", g, dg, None, mode, tuning)
    check(ctx, "sssp", g, dg, np.array([1234], np.uint32), "persistent", tuning)
    check(ctx, "cc_jump", g, dg, None, "persistent", tuning)
    dg.close()


@pytest.mark.parametrize("tuning", SCHEDULES[:5])
def test_cc_jump_many_components(ctx, tuning):
    # heavily cut mesh (many components) and a symmetric R-MAT graph (hubs, isolated vertices)
    g = inputs.mesh(200, 170, seed=13, del_frac=0.45, extra_frac=0.01, radius=8)
    dg = ctx.load(g)
    st = check(ctx, "cc_jump", g, dg, None, "persistent", tuning)
    assert st["rounds"] < 64
    dg.close()
    r = inputs.rmat(14, 8, seed=14, weights=False)
    u = np.repeat(np.arange(r.n), np.diff(r.row_ptr.astype(np.int64)))
    sym = inputs.csr_from_edges(r.n, np.concatenate([u, r.col]), np.concatenate([r.col, u]), symmetric=True)
    ds = ctx.load(sym)
    check(ctx, "cc_jump", sym, ds, None, "persistent", tuning)
    check(ctx, "cc", sym, ds, None, "persistent", tuning)
    ds.close()


@pytest.mark.parametrize("delta", [1, 7, 1000, 1 << 30])
def test_cc_near_far(ctx, delta):
    """Min-label CC under the near-far schedule (labels below the limit first):
    same labels on many-component meshes, hub graphs and tiny graphs; with
    delta = 1 the smallest label floods first, so a mostly connected mesh is
    scanned about twice (round 0 plus the flood), not once per label change."""
    tn = dict(delta=delta)
    g = inputs.mesh(200, 170, seed=13, del_frac=0.45, extra_frac=0.01, radius=8)
    dg = ctx.load(g)
    check(ctx, "cc", g, dg, None, "persistent", tn)
    check(ctx, "cc", g, dg, None, "persistent", dict(tn, cta_size=1024, warp_thresh=2, cta_thresh=8))
    dg.close()
    r = inputs.rmat(13, 8, seed=15, weights=False)
    u = np.repeat(np.arange(r.n), np.diff(r.row_ptr.astype(np.int64)))
    sym = inputs.csr_from_edges(r.n, np.concatenate([u, r.col]), np.concatenate([r.col, u]), symmetric=True)
    ds = ctx.load(sym)
    check(ctx, "cc", sym, ds, None, "persistent", dict(tn, cta_size=256))
    ds.close()
    rng = np.random.default_rng(16 + delta % 97)
    for trial in range(6):
        n = int(rng.integers(1, 120))
        t = tiny_graph(rng, n, float(rng.choice([0.01, 0.05])), True)
        dt = ctx.load(t)
        check(ctx, "cc", t, dt, None, "persistent", tn)
        dt.close()
    m = inputs.mesh(300, 257, seed=9, del_frac=0.01, extra_frac=0.001, radius=8)
    dm = ctx.load(m)
    st = check(ctx, "cc", m, dm, None, "persistent", tn)
    if delta == 1:
        assert st["edges_scanned"] <= 3 * m.m
    dm.close()


def test_cc_jump_mesh4096_full(ctx):
    g, _ = inputs.workload_mesh(4096)
    dg = ctx.load(g, validate=False)
    st = check(ctx, "cc_jump", g, dg, None, "persistent")
    assert st["rounds"] < 64
    dg.close()


def test_many_sources_init_path(ctx):
    # more than eight initial items exercises the two-pass state initialisation
    g = inputs.rmat(12, 8, seed=5, weights=True)
    dg = ctx.load(g)
    srcs = inputs.sources(g, 37, seed=6)
    for mode in MODES:
        check(ctx, "bfs", g, dg, srcs, mode)
        check(ctx, "sssp", g, dg, srcs, mode)
    dg.close()


@pytest.mark.parametrize("nsrc", [1, 992, 993, 3000])
def test_run_source_block_sizes(ctx, nsrc):
    """irgl_run passes up to 992 sources in one copy of its source block and more
    through a worklist push: both sides of the bound, with device and host
    result buffers and repeated calls, equal the oracle (repeated sources included)."""
    g = inputs.rmat(13, 8, seed=7, weights=True)
    dg = ctx.load(g)
    rng = np.random.default_rng(nsrc)
    srcs = rng.integers(0, g.n, size=nsrc).astype(np.uint32)
    for kernel in ("bfs", "sssp"):
        want = oracle.run(kernel, g, srcs)
        for rep in range(2):
            got, _ = run(ctx, kernel, g, dg, srcs)
            np.testing.assert_array_equal(got, want, err_msg=f"{kernel} device rep {rep}")
            host, _ = ctx.run_host(kernel, dg, srcs)
            np.testing.assert_array_equal(host, want, err_msg=f"{kernel} host rep {rep}")
    dg.close()


def fused_round0_graph(rng):
    """Uniform random graph (n = 700,003: n mod 4 = 3, and vertices past four per thread of the
    widest grid) whose first vertices are sources with chosen out-degrees around 256."""
    n = 700_003
    m = 3_000_000
    src = rng.integers(16, n, size=m)
    dst = rng.integers(0, n, size=m)

    def targets(k, extra=()):
        t = list(extra) + rng.integers(0, n, size=k - len(extra)).tolist()
        return t[:k]

    edges = []
    # 0: 256 out-edges with the last three vertices, far vertices, a repeated target and a self-loop
    edges += [(0, v) for v in targets(256, (n - 1, n - 2, n - 3, 4 * 155_648 + 5, 99, 99, 0))]
    edges += [(1, v) for v in targets(257, (n - 1,))]   # 1: 257 out-edges
    edges += [(2, v) for v in targets(255, (n - 2,))]   # 2: 255 out-edges
    # 3: no out-edges; 4: a self-loop only
    edges += [(4, 4)]
    for u in range(5, 14):                              # 5..13: 32 out-edges each
        edges += [(u, v) for v in targets(32)]
    edges += [(14, v) for v in targets(33)]             # 14: 33 out-edges
    es, ed = zip(*edges)
    src = np.concatenate([src, np.array(es)])
    dst = np.concatenate([dst, np.array(ed)])
    w = rng.integers(1, 101, size=src.size)
    return inputs.csr_from_edges(n, src, dst, w)


def test_bfs_round0_in_prologue(ctx):
    """BFS from one to eight sources with at most 256 out-edges together runs its first round in
    the persistent kernel's prologue; both sides of each bound (255/256/257 edges, 8/9 sources),
    sources with no out-edge or only a self-loop, repeated sources, the direction-optimising
    form and the visited bitmap (never fused) equal the oracle."""
    g = fused_round0_graph(np.random.default_rng(1607))
    dg = ctx.load(g)
    sets = [[0], [1], [2], [3], [4], [0, 0], [3, 4], [0, 3], list(range(5, 13)), list(range(5, 14)),
            list(range(7, 15)), [12, 13, 3, 4, 2], [3, 4, 2], [4, 4, 3]]
    for srcs in sets:
        srcs = np.array(srcs, dtype=np.uint32)
        want = oracle.run("bfs", g, srcs)
        for t in (None, dict(flags=2), dict(flags=4), dict(cta_size=1024), dict(cta_size=128, max_blocks=1)):
            got, st = run(ctx, "bfs", g, dg, srcs, tuning=t)
            np.testing.assert_array_equal(got, want, err_msg=f"sources {srcs.tolist()} tuning {t}")
            if t is None or not t.get("flags"):
                # top-down: one round per level plus the last round that pushes nothing
                assert st["rounds"] == int(want[want != INF].max()) + 1, (srcs.tolist(), t)
    dg.close()


# ----------------------------------------------------------------------------- Invoke, reductions, worklists

def test_invoke_bulk_synchronous_and_reductions(ctx):
    from paper_1607_05707_gb300.api import as_u32

    # 0 -> {1,2}, 1 -> {3}, 2 -> {}, 3 -> {0}
    g = inputs.csr_from_edges(4, [0, 0, 1, 3], [1, 2, 3, 0], [1, 1, 1, 1])
    dg = ctx.load(g)
    a, b = ctx.worklist(16), ctx.worklist(16)
    state = ctx.state(4)
    a.push([0])
    ctx.init_state("bfs", dg, a, state)
    assert list(as_u32(state)) == [0, INF, INF, INF]
    res = ctx.invoke("bfs", dg, a, b, state, level=0, reduce="any")
    assert res == 1
    assert a.size() == 0                      # in-worklist popped
    assert sorted(b.read()) == [1, 2]         # pushes land in out only
    assert list(as_u32(state)) == [0, 1, 1, INF]
    # All: item 2 has no out-edges, so "every item pushed" is false
    res = ctx.invoke("bfs", dg, b, a, state, level=1, reduce="all")
    assert res == 0
    assert sorted(a.read()) == [3]
    # next round: 3 -> 0 (already visited) pushes nothing: Any = 0, All = 0
    res = ctx.invoke("bfs", dg, a, b, state, level=2, reduce="any")
    assert res == 0 and b.size() == 0
    # reductions over an empty worklist: Any = false, All = true
    assert ctx.invoke("bfs", dg, a, b, state, level=3, reduce="any") == 0
    assert ctx.invoke("bfs", dg, a, b, state, level=3, reduce="all") == 1
    # All = true when every popped item pushes
    state2 = ctx.state(4)
    a.clear(); b.clear()
    a.push([0])
    ctx.init_state("bfs", dg, a, state2)
    assert ctx.invoke("bfs", dg, a, b, state2, level=0, reduce="all") == 1
    for h in (a, b):
        h.close()
    dg.close()


def test_iterate_with_worklist_object(ctx):
    from paper_1607_05707_gb300.api import as_u32

    g = inputs.rmat(13, 8, seed=11, weights=True)
    dg = ctx.load(g)
    srcs = inputs.sources(g, 3, seed=12)
    wl = ctx.worklist(8)
    wl.push(srcs)
    for mode in MODES:
        out, st = ctx.iterate("sssp", dg, wl, mode=mode)
        np.testing.assert_array_equal(as_u32(out)[: g.n], oracle.sssp(g.n, g.row_ptr, g.col, g.w, srcs))
        assert wl.size() == 3  # the initial worklist is read, not consumed
    gs = inputs.mesh(40, 30, seed=3, del_frac=0.1)
    dgs = ctx.load(gs)
    allv = ctx.worklist(gs.n)
    allv.push_range(gs.n)
    out, _ = ctx.iterate("cc", dgs, allv)
    np.testing.assert_array_equal(as_u32(out)[: gs.n], oracle.cc(gs.n, gs.row_ptr, gs.col))
    wl.close(); allv.close(); dg.close(); dgs.close()


def test_run_host_buffers(ctx):
    g = inputs.rmat(14, 16, seed=21, weights=True)
    dg = ctx.load(g)
    s = inputs.sources(g, 1, seed=22)
    for mode in MODES:
        out, st = ctx.run_host("bfs", dg, s, mode=mode)
        np.testing.assert_array_equal(out, oracle.bfs(g.n, g.row_ptr, g.col, s))
        out, st = ctx.run_host("sssp", dg, s, mode=mode)
        np.testing.assert_array_equal(out, oracle.sssp(g.n, g.row_ptr, g.col, g.w, s))
        assert st["rounds"] > 1
    dg.close()


# ----------------------------------------------------------------------------- errors (host-made, no GPU fault)

def test_errors_and_recovery(ctx):
    from paper_1607_05707_gb300 import irgl as C

    g = inputs.rmat(12, 16, seed=31, weights=True)
    dg = ctx.load(g)
    s = inputs.sources(g, 1, seed=32)
    # worklist overflow: scratch worklists far too small
    ctx.debug_set(3, 4)
    for mode in MODES:
        for kernel in ("bfs", "sssp"):
            with pytest.raises(C.IrglError) as ei:
                ctx.run(kernel, dg, s, mode=mode)
            assert ei.value.status == C.IRGL_ERR_WL_OVERFLOW
    ctx.debug_set(3, 0)
    check(ctx, "bfs", g, dg, s)
    # barrier timeout: one CTA never arrives, the others give up after 20 ms
    ctx.debug_set(1, 20000)
    ctx.debug_set(2, 1)
    for kernel in ("bfs", "sssp"):
        with pytest.raises(C.IrglError) as ei:
            ctx.run(kernel, dg, s, mode="persistent")
        assert ei.value.status == C.IRGL_ERR_BARRIER_TIMEOUT
    ctx.debug_set(2, -1)
    ctx.debug_set(1, 0)
    check(ctx, "bfs", g, dg, s)
    check(ctx, "sssp", g, dg, s)
    # max_rounds (extra_cond): stops with a status, never a silent wrong answer
    for mode in MODES:
        with pytest.raises(C.IrglError) as ei:
            ctx.run("bfs", dg, s, mode=mode, max_rounds=2)
        assert ei.value.status == C.IRGL_ERR_MAX_ROUNDS
    check(ctx, "sssp", g, dg, s, "per_launch")
    # pointer-jumping CC is a persistent-only Iterate
    gs = inputs.grid(8)
    dgs = ctx.load(gs)
    with pytest.raises(C.IrglError) as ei:
        ctx.run("cc_jump", dgs, None, mode="per_launch")
    assert ei.value.status == C.IRGL_ERR_UNSUPPORTED
    dgs.close()
    # CC on a graph not loaded as symmetric
    with pytest.raises(C.IrglError) as ei:
        ctx.run("cc", dg, None)
    assert ei.value.status == C.IRGL_ERR_NOT_SYMMETRIC
    # SSSP without weights; source out of range
    gu = inputs.grid(8)
    dgu = ctx.load(gu)
    with pytest.raises(C.IrglError) as ei:
        ctx.run("sssp", dgu, [0])
    assert ei.value.status == C.IRGL_ERR_INVALID_ARG
    with pytest.raises(C.IrglError):
        ctx.run("bfs", dgu, [64])
    dgu.close()
    dg.close()


def test_big_list_overflow_falls_back(ctx):
    # a big list of 3 entries: further long lists take the warp-bin path in the same round
    g = inputs.rmat(14, 16, seed=61, weights=True)
    dg = ctx.load(g)
    s = inputs.sources(g, 1, seed=62)
    ctx.debug_set(4, 3)
    try:
        for k in ("bfs", "sssp"):
            check(ctx, k, g, dg, s, "persistent", dict(cta_size=256, warp_thresh=4, cta_thresh=16))
    finally:
        ctx.debug_set(4, 0)
    dg.close()


DIROPT = [dict(flags=2), dict(flags=2, cta_size=256, warp_thresh=8, cta_thresh=64), dict(flags=3, cta_size=512)]


@pytest.mark.parametrize("tuning", DIROPT)
def test_direction_optimising_bfs(ctx, tuning):
    g = inputs.rmat(16, 16, seed=51, weights=True)
    dg = ctx.load(g, in_edges=True)
    for s in inputs.sources(g, 3, seed=52):
        check(ctx, "bfs", g, dg, np.array([s], np.uint32), "persistent", tuning)
    check(ctx, "bfs", g, dg, inputs.sources(g, 5, seed=53), "persistent", tuning)
    dg.close()
    m = inputs.mesh(300, 300, seed=54, del_frac=0.01, extra_frac=0.001)  # symmetric: in-edges = out-edges
    dm = ctx.load(m)
    check(ctx, "bfs", m, dm, np.array([0], np.uint32), "persistent", tuning)
    dm.close()


def test_bottom_up_every_round(ctx):
    # test hook: every round bottom-up, on tiny random, special and directed graphs
    rng = np.random.default_rng(57)
    ctx.debug_set(5, 1)
    try:
        for trial in range(16):
            n = int(rng.integers(1, 150))
            g = tiny_graph(rng, n, float(rng.choice([0.02, 0.08])), bool(trial % 2))
            dg = ctx.load(g, in_edges=True)
            check(ctx, "bfs", g, dg, rng.integers(0, n, size=2).astype(np.uint32), "persistent", dict(flags=2))
            dg.close()
        g = inputs.rmat(13, 8, seed=58, weights=False)
        dg = ctx.load(g, in_edges=True)
        check(ctx, "bfs", g, dg, inputs.sources(g, 1, seed=59), "persistent", dict(flags=2))
        dg.close()
    finally:
        ctx.debug_set(5, 0)


LOCAL = [dict(flags=1 << 8), dict(flags=4 << 8), dict(flags=15 << 8), dict(cta_size=1024, flags=8 << 8),
         dict(cta_size=128, warp_thresh=1 << 30, cta_thresh=1 << 30, flags=3 << 8),
         dict(cta_size=256, warp_thresh=2, cta_thresh=8, flags=4 << 8)]


@pytest.mark.parametrize("tuning", LOCAL)
def test_cta_local_sub_rounds(ctx, tuning):
    """CTA-local sub-rounds (IRGL_TUNE_LOCAL(k)): BFS runs as unit-weight
    label-correcting relaxation, SSSP keeps its operator; a CTA expands its own
    fresh pushes k more times between grid barriers. Same levels and distances
    on tiny, high-diameter and power-law graphs, single and multiple sources."""
    rng = np.random.default_rng(71)
    for trial in range(10):
        n = int(rng.integers(1, 160))
        g = tiny_graph(rng, n, float(rng.choice([0.02, 0.08])), bool(trial % 2))
        dg = ctx.load(g)
        srcs = rng.integers(0, n, size=int(rng.integers(1, 4))).astype(np.uint32)
        check(ctx, "bfs", g, dg, srcs, "persistent", tuning)
        check(ctx, "sssp", g, dg, srcs, "persistent", tuning)
        dg.close()
    m = inputs.mesh(300, 257, seed=72, del_frac=0.02, extra_frac=0.002, weights=True)
    dm = ctx.load(m)
    for srcs in ([0], [40000, 7]):
        s = np.array(srcs, np.uint32)
        st = check(ctx, "bfs", m, dm, s, "persistent", tuning)
        check(ctx, "sssp", m, dm, s, "persistent", tuning)
    dm.close()
    r = inputs.rmat(15, 16, seed=73, weights=True)
    dr = ctx.load(r)
    for s in inputs.sources(r, 2, seed=74):
        check(ctx, "bfs", r, dr, np.array([s], np.uint32), "persistent", tuning)
        check(ctx, "sssp", r, dr, np.array([s], np.uint32), "persistent", tuning)
    dr.close()
    g, srcs = inputs.workload_grid64()
    dg = ctx.load(g)
    got, st = run(ctx, "bfs", g, dg, srcs, "persistent", tuning)
    rr, cc = np.divmod(np.arange(g.n), 64)
    np.testing.assert_array_equal(got, (rr + cc).astype(np.uint32))
    assert st["rounds"] <= 127  # never more grid rounds than levels
    dg.close()


def test_bfs_visited_bitmap(ctx):
    """The persistent BFS visited bitmap (IRGL_TUNE_BITMAP = 4) gives the same
    levels; it is cleared per launch, so a graph run after a larger one (whose
    bits were all set) is not filtered by stale bits; vertex counts that are
    not multiples of 32 end in a partial word."""
    rng = np.random.default_rng(61)
    big = inputs.rmat(15, 16, seed=62)
    dbig = ctx.load(big)
    for tuning in (dict(flags=4), None, dict(cta_size=1024, warp_thresh=2, cta_thresh=8, flags=4),
                   dict(cta_size=128, warp_thresh=1 << 30, cta_thresh=1 << 30, flags=1 | 4), dict(flags=2 | 4)):
        check(ctx, "bfs", big, dbig, inputs.sources(big, 1, seed=63), "persistent", tuning)
        for n in (1, 31, 33, 1000 + 7):
            g = tiny_graph(rng, n, min(1.0, 4.0 / n), bool(n % 2))
            dg = ctx.load(g)
            check(ctx, "bfs", g, dg, np.array([int(rng.integers(0, n))], np.uint32), "persistent", tuning)
            dg.close()
    dbig.close()


# ----------------------------------------------------------------------------- configuration sizes

def test_rmat20_bfs_direction_optimising_full(ctx):
    g, srcs = inputs.workload_rmat20(nsrc=3)
    dg = ctx.load(g, validate=False, in_edges=True)
    for s in srcs:
        check(ctx, "bfs", g, dg, np.array([s], np.uint32), "persistent", dict(flags=2))
    dg.close()


def test_time_limit_stops_and_recovers(ctx):
    """A persistent launch past its wall-time limit (test hook key 7, here 1 ms)
    stops at its next round with IRGL_ERR_TIME_LIMIT instead of running on, and
    the context is exact afterwards; the same for a batch."""
    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import Batch

    g = inputs.mesh(300, 257, seed=9, del_frac=0.01, extra_frac=0.001, radius=8)  # min-label CC: ~500 rounds
    dg = ctx.load(g)
    ctx.debug_set(7, 1)
    try:
        with pytest.raises(C.IrglError) as ei:
            ctx.run("cc", dg, None, tuning=dict(flags=NO_SMEM))
        assert ei.value.status == C.IRGL_ERR_TIME_LIMIT
        b = Batch(ctx, 4)
        b.add("cc", dg)
        b.prepare()
        with pytest.raises(C.IrglError) as ei:
            b.run()
        assert ei.value.status == C.IRGL_ERR_TIME_LIMIT
        b.close()
    finally:
        ctx.debug_set(7, 0)
    check(ctx, "cc", g, dg, None, "persistent")
    b = Batch(ctx, 4)
    b.add("cc", dg)
    b.prepare()
    b.run()
    np.testing.assert_array_equal(b.result(0)[0], oracle.cc(g.n, g.row_ptr, g.col))
    b.close()
    dg.close()


@pytest.mark.parametrize("mode", MODES)
def test_rmat20_bfs_sssp_full(ctx, mode):
    g, srcs = inputs.workload_rmat20(nsrc=3)
    dg = ctx.load(g, validate=False)
    for s in srcs[:2]:
        one = np.array([s], np.uint32)
        check(ctx, "bfs", g, dg, one, mode)
        check(ctx, "sssp", g, dg, one, mode)
    dg.close()


def test_mesh4096_cc_near_far_full(ctx):
    g, _ = inputs.workload_mesh(4096)
    dg = ctx.load(g, validate=False)
    st = check(ctx, "cc", g, dg, None, "persistent", dict(delta=1))
    assert st["edges_scanned"] <= 3 * g.m
    dg.close()


def test_mesh4096_local_sub_rounds_full(ctx):
    g, srcs = inputs.workload_mesh(4096)
    dg = ctx.load(g, validate=False)
    st = check(ctx, "bfs", g, dg, srcs, "persistent", dict(flags=8 << 8))
    assert st["rounds"] < 7211  # fewer grid barriers than BFS levels
    dg.close()
    r, rs = inputs.workload_rmat20(nsrc=1)
    dr = ctx.load(r, validate=False)
    one = np.array([rs[0]], np.uint32)
    check(ctx, "bfs", r, dr, one, "persistent", dict(flags=4 << 8))
    check(ctx, "sssp", r, dr, one, "persistent", dict(flags=4 << 8))
    dr.close()


def test_mesh4096_bfs_full(ctx):
    g, srcs = inputs.workload_mesh(4096)
    dg = ctx.load(g, validate=False)
    st = check(ctx, "bfs", g, dg, srcs, "persistent")
    lv = oracle.bfs(g.n, g.row_ptr, g.col, srcs)
    # one round per BFS level, plus the last round that pushes nothing
    assert st["rounds"] == int(lv[lv != INF].max()) + 1
    assert st["rounds"] > 4000
    dg.close()


def test_batch_config_instances_sssp(ctx):
    # the per-instance (one query per launch) form of the batched workload, on a sample
    for g, srcs in inputs.workload_batch(count=12):
        dg = ctx.load(g, validate=False)
        check(ctx, "sssp", g, dg, srcs, "persistent")
        dg.close()
