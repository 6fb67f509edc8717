"""irgl_bfs_noalloc: the BFS entry point that allocates no device memory.

Checked through the C-ABI against the regular entry point (irgl_run), exactly
(levels are integers), on two calls in a row: the second call reuses the
shared scratch array that the first call left behind. The oversize check needs
no GPU work. This file is collected last so that a failure here leaves every
other test already run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1607_05707_gb300 import inputs

pytestmark = pytest.mark.gpu


def _noalloc(lib, n, m, rp, col, src, level, stream):
    rounds = ctypes.c_uint32()
    fn = lib.irgl_bfs_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]
    fn.restype = ctypes.c_int
    rc = fn(0, stream, n, m, rp, col, src, level, ctypes.byref(rounds))
    return rc, int(rounds.value)


def test_noalloc_bfs_matches_regular_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_05707_gb300 import irgl as C
    from paper_1607_05707_gb300.api import Context, as_u32

    lib = C.lib()
    stream = torch.cuda.Stream()
    ctx = Context(0, stream)
    g = inputs.rmat(16, 16, seed=91, weights=False)
    dg = ctx.load(g, validate=False)
    # the caller owns inputs and outputs: torch allocates them, the entry point allocates nothing
    rp = torch.from_numpy(g.row_ptr.view(np.int32)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srcs = inputs.sources(g, 2, seed=92)
    for s in srcs:  # two calls in a row share the scratch array
        rc, rounds = _noalloc(lib, g.n, g.m, rp.data_ptr(), col.data_ptr(), int(s), level.data_ptr(), stream.cuda_stream)
        assert rc == 0, C.irgl_last_error()
        want, st = ctx.run("bfs", dg, np.array([s], np.uint32))
        np.testing.assert_array_equal(as_u32(level), as_u32(want)[: g.n])
        assert rounds == st["rounds"]
    # beyond the stated maximum: rejected before any GPU work
    rc, _ = _noalloc(lib, (1 << 20) + 1, g.m, rp.data_ptr(), col.data_ptr(), 0, level.data_ptr(), stream.cuda_stream)
    assert rc == C.IRGL_ERR_INVALID_ARG
    assert "vertices" in C.irgl_last_error()
    dg.close()
    ctx.close()
