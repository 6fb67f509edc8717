"""irgl_bfs_noalloc: the BFS entry point for callers that cannot allocate device memory.

Checked through the C-ABI, exactly (levels are integers), against the CPU oracle's
FIFO BFS and against the regular entry point (irgl_run), on two calls in a row: the
second call reuses the shared scratch array that the first call left behind. Two
graph sizes: R-MAT scale 16, and R-MAT scale 20 at the entry point's vertex limit
(2^20), whose heavy round has more long adjacency lists than the entry point's
65,536-entry big list holds, so the overflow into the warp bin runs too. The
oversize and wrong-stream checks need no GPU work. This file is collected last,
so a failure here leaves every other test already run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF


def _noalloc(lib, n, m, rp, col, src, level, stream, device=0):
    rounds = ctypes.c_uint32()
    fn = lib.irgl_bfs_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]
    fn.restype = ctypes.c_int
    rc = fn(device, stream, n, m, rp, col, src, level, ctypes.byref(rounds))
    return rc, int(rounds.value)


@pytest.mark.parametrize("scale", [16, 20])
def test_noalloc_bfs_matches_oracle_and_regular_entry_point(scale):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import Context, as_u32

    lib = C.lib()
    stream = torch.cuda.Stream()
    ctx = Context(0, stream)
    g = inputs.rmat(scale, 16, seed=91 + scale, weights=False)
    assert g.n <= 1 << 20
    dg = ctx.load(g, validate=False)
    # the caller owns inputs and outputs: torch allocates them, the entry point allocates nothing
    rp = torch.from_numpy(g.row_ptr.view(np.int32)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srcs = inputs.sources(g, 2, seed=92 + scale)
    for s in srcs:  # two calls in a row share the scratch array
        rc, rounds = _noalloc(lib, g.n, g.m, rp.data_ptr(), col.data_ptr(), int(s), level.data_ptr(),
                              stream.cuda_stream)
        assert rc == 0, C.irgl_last_error()
        got = as_u32(level)
        want = oracle.bfs(g.n, g.row_ptr, g.col, [int(s)])
        np.testing.assert_array_equal(got, want)
        assert rounds == int(want[want != INF].max()) + 1
        regular, st = ctx.run("bfs", dg, np.array([s], np.uint32))
        np.testing.assert_array_equal(got, as_u32(regular)[: g.n])
        assert rounds == st["rounds"]
    # beyond the stated maximum: rejected before any GPU work
    rc, _ = _noalloc(lib, (1 << 20) + 1, g.m, rp.data_ptr(), col.data_ptr(), 0, level.data_ptr(), stream.cuda_stream)
    assert rc == C.IRGL_ERR_INVALID_ARG
    assert "vertices" in C.irgl_last_error()
    # a stream is checked against the device it is named with
    if torch.cuda.device_count() > 1:
        other = torch.cuda.Stream(device=1)
        rc, _ = _noalloc(lib, g.n, g.m, rp.data_ptr(), col.data_ptr(), 0, level.data_ptr(), other.cuda_stream)
        assert rc == C.IRGL_ERR_INVALID_ARG
    dg.close()
    ctx.close()
