"""ctypes binding of libirgl.so (the C-ABI declared in include/irgl.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name and raises :class:`IrglError` on a non-zero status. Every step
of the traversal runs in the library's CUDA kernels; there is no Python or CPU
fallback, and loading fails loudly when libirgl.so has not been built.

Pointers are passed as integers (``tensor.data_ptr()``, ``numpy.ctypes.data``);
streams as ``torch.cuda.Stream.cuda_stream`` integers.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_char_p, c_int, c_int64, c_uint32, c_uint64, c_void_p

from . import _build

IRGL_OK = 0
IRGL_ERR_INVALID_ARG = -1
IRGL_ERR_OOM = -2
IRGL_ERR_WL_OVERFLOW = -3
IRGL_ERR_BARRIER_TIMEOUT = -4
IRGL_ERR_CUDA = -5
IRGL_ERR_NOT_SYMMETRIC = -6
IRGL_ERR_ADMISSION = -7
IRGL_ERR_MAX_ROUNDS = -8
IRGL_ERR_NOT_READY = -9
IRGL_ERR_UNSUPPORTED = -10
IRGL_ERR_LOCK_TIMEOUT = -11
IRGL_ERR_TIME_LIMIT = -12

IRGL_INF = 0xFFFFFFFF

IRGL_BFS, IRGL_SSSP, IRGL_CC, IRGL_CC_JUMP = 0, 1, 2, 3
IRGL_PER_LAUNCH, IRGL_PERSISTENT = 0, 1
IRGL_REDUCE_ANY, IRGL_REDUCE_ALL = 0, 1
IRGL_LOCK_BLOCKING, IRGL_LOCK_TICKET, IRGL_LOCK_RETRY = 0, 1, 2
LOCKS = {"blocking": IRGL_LOCK_BLOCKING, "ticket": IRGL_LOCK_TICKET, "retry": IRGL_LOCK_RETRY}

IRGL_HOST_PTRS = 0x0
IRGL_DEVICE_PTRS = 0x1
IRGL_SYMMETRIC = 0x2
IRGL_VALIDATE = 0x4
IRGL_IN_EDGES = 0x8
IRGL_TUNE_NO_SPLIT = 0x1
IRGL_TUNE_DIROPT = 0x2
IRGL_TUNE_BITMAP = 0x4
IRGL_TUNE_NO_PACKED = 0x8
IRGL_TUNE_NO_BCAST = 0x10
IRGL_TUNE_THREAD_BIN = 0x20
IRGL_TUNE_NO_SMEM = 0x40
IRGL_TUNE_DENSE = 0x80
IRGL_TUNE_NO_DEFER = 0x1000


def IRGL_TUNE_LOCAL(k: int) -> int:
    """Flag bits of k CTA-local sub-rounds (0..15)."""
    return (int(k) & 15) << 8

KERNELS = {"bfs": IRGL_BFS, "sssp": IRGL_SSSP, "cc": IRGL_CC, "cc_jump": IRGL_CC_JUMP}
MODES = {"per_launch": IRGL_PER_LAUNCH, "persistent": IRGL_PERSISTENT}


class irgl_tuning(ctypes.Structure):
    _fields_ = [
        ("cta_size", c_uint32),
        ("warp_thresh", c_uint32),
        ("cta_thresh", c_uint32),
        ("chunk", c_uint32),
        ("blocks_per_sm", c_uint32),
        ("max_blocks", c_uint32),
        ("flags", c_uint32),
        ("delta", c_uint32),
        ("defer_deg", c_uint32),
        ("defer_delta", c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class irgl_stats(ctypes.Structure):
    _fields_ = [
        ("rounds", c_uint32),
        ("grid", c_uint32),
        ("cta_size", c_uint32),
        ("launches", c_uint32),
        ("edges_scanned", c_uint64),
        ("last_out", c_uint32),
        ("device_ms", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "device_ms"}
        d["device_ms"] = float(self.device_ms)
        return d


class irgl_msf_stats(ctypes.Structure):
    _fields_ = [
        ("edges", c_uint32),
        ("iterations", c_uint32),
        ("weight", c_uint64),
        ("invocations", c_uint32),
        ("retries", c_uint32),
        ("locks", c_uint32),
        ("launches", c_uint32),
        ("grid", c_uint32),
        ("cta_size", c_uint32),
        ("device_ms", ctypes.c_float),
        ("reserved", c_uint32),
    ]

    def as_dict(self) -> dict:
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k not in ("device_ms", "reserved")}
        d["device_ms"] = float(self.device_ms)
        return d


class irgl_server_config(ctypes.Structure):
    _fields_ = [
        ("arena_bytes", c_uint64),
        ("max_slots", c_uint32),
        ("epoch_rounds", c_uint32),
        ("count_edges", c_uint32),
        ("solo_min_n", c_uint32),
        ("tuning", irgl_tuning),
    ]


class irgl_query_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("rounds", c_uint32),
        ("latency_s", ctypes.c_double),
        ("t_submit_s", ctypes.c_double),
        ("t_done_s", ctypes.c_double),
        ("edges", c_uint64),
    ]


class irgl_server_counters(ctypes.Structure):
    _fields_ = [
        ("submitted", c_uint64), ("completed", c_uint64), ("rejected", c_uint64), ("epochs", c_uint64),
        ("rounds", c_uint64), ("edges", c_uint64), ("busy_s", ctypes.c_double), ("kernel_s", ctypes.c_double),
        ("active", c_uint32),
        ("queued", c_uint32), ("arena_entries", c_uint64), ("grid", c_uint32), ("cta_size", c_uint32),
        ("solo", c_uint64),
    ]

    def as_dict(self) -> dict:
        return {k: (float(getattr(self, k)) if k in ("busy_s", "kernel_s") else int(getattr(self, k)))
                for k, _ in self._fields_}


class IrglError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"irgl status {status}: {message}")
        self.status = status


_P = c_void_p  # opaque handles and raw pointers

# name -> argtypes (every function returns int status unless listed in _RESTYPE)
_SIGS = {
    "irgl_last_error": [],
    "irgl_status_string": [c_int],
    "irgl_ctx_create": [c_int, _P, POINTER(_P)],
    "irgl_ctx_destroy": [_P],
    "irgl_ctx_set_stream": [_P, _P],
    "irgl_ctx_info": [_P, POINTER(c_uint32), POINTER(irgl_tuning)],
    "irgl_csr_validate": [c_uint32, c_uint64, _P, _P, _P, c_int],
    "irgl_csr_load": [_P, c_uint32, c_uint64, _P, _P, _P, c_int, POINTER(_P)],
    "irgl_graph_destroy": [_P],
    "irgl_graph_info": [_P, POINTER(c_uint32), POINTER(c_uint64), POINTER(c_int)],
    "irgl_worklist_create": [_P, c_uint32, POINTER(_P)],
    "irgl_worklist_destroy": [_P],
    "irgl_worklist_push": [_P, _P, c_uint32],
    "irgl_worklist_push_range": [_P, c_uint32],
    "irgl_worklist_clear": [_P],
    "irgl_worklist_size": [_P, POINTER(c_uint32)],
    "irgl_worklist_read": [_P, _P, c_uint32, POINTER(c_uint32)],
    "irgl_init_state": [_P, c_int, _P, _P, _P],
    "irgl_invoke": [_P, c_int, _P, _P, _P, _P, c_uint32, c_int, POINTER(irgl_tuning), POINTER(c_int)],
    "irgl_iterate": [_P, c_int, _P, _P, _P, c_int, POINTER(irgl_tuning), c_uint32, POINTER(irgl_stats)],
    "irgl_iterate_async": [_P, c_int, _P, _P, _P, POINTER(irgl_tuning), c_uint32],
    "irgl_ctx_sync": [_P, POINTER(irgl_stats)],
    "irgl_run": [_P, c_int, _P, _P, c_uint32, _P, c_int, c_int, POINTER(irgl_tuning), c_uint32, POINTER(irgl_stats)],
    "irgl_debug_set": [_P, c_int, c_int64],
    "irgl_trace_enable": [_P, c_uint32],
    "irgl_trace_read": [_P, _P, _P, _P, c_uint32, POINTER(c_uint32)],
    "irgl_trace_phases": [_P, _P, c_uint32, POINTER(c_uint32)],
    "irgl_server_create": [_P, POINTER(irgl_server_config), POINTER(_P)],
    "irgl_server_submit": [_P, _P, c_int, c_uint32, _P, POINTER(c_uint64)],
    "irgl_server_poll": [_P, c_uint64, POINTER(irgl_query_info)],
    "irgl_server_drain": [_P, c_uint32],
    "irgl_server_stats": [_P, POINTER(irgl_server_counters)],
    "irgl_server_destroy": [_P],
    "irgl_autotune": [_P, c_int, _P, _P, c_uint32, c_uint32, POINTER(irgl_tuning), POINTER(ctypes.c_float)],
    "irgl_batch_autotune": [_P, c_uint32, POINTER(irgl_tuning), POINTER(ctypes.c_float)],
    "irgl_bfs_noalloc": [c_int, _P, c_uint32, c_uint64, _P, _P, c_uint32, _P, POINTER(c_uint32)],
    "irgl_control_cta": [POINTER(c_uint32), c_uint32, c_uint32, POINTER(c_uint32)],
    "irgl_batch_create": [_P, c_uint32, POINTER(_P)],
    "irgl_batch_destroy": [_P],
    "irgl_batch_add": [_P, _P, c_int, _P, c_uint32, POINTER(c_uint32)],
    "irgl_batch_prepare": [_P, POINTER(irgl_tuning), c_int],
    "irgl_batch_set_wave_bytes": [_P, c_uint64],
    "irgl_batch_waves": [_P, POINTER(c_uint32)],
    "irgl_batch_launch": [_P],
    "irgl_batch_sync": [_P, POINTER(irgl_stats)],
    "irgl_batch_run": [_P, POINTER(irgl_stats)],
    "irgl_batch_info": [_P, POINTER(c_uint32), POINTER(c_uint32), POINTER(c_uint32), POINTER(c_int), POINTER(c_uint64)],
    "irgl_batch_result": [_P, c_uint32, POINTER(_P), POINTER(c_uint32), POINTER(c_uint32)],
    "irgl_batch_copy_result": [_P, c_uint32, _P],
    "irgl_batch_copy_results": [_P, _P],
    "irgl_msf": [_P, _P, c_int, c_int, _P, c_uint32, c_int, POINTER(irgl_tuning), POINTER(irgl_msf_stats)],
}
_RESTYPE = {"irgl_last_error": c_char_p, "irgl_status_string": c_char_p}

_lib = None


def lib():
    """Load libirgl.so (built in place by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        path = _build.IRGL_LIB
        if not path.exists():
            raise ImportError(f"{path.name} is not built: run __graft_entry__.build() (no CPU fallback exists)")
        L = ctypes.CDLL(str(path))
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, c_int)
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def _check(rc: int) -> None:
    if rc != IRGL_OK:
        raise IrglError(rc, lib().irgl_last_error().decode(errors="replace"))


def _tuning(t) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if isinstance(t, irgl_tuning):
        return ctypes.byref(t)
    tt = irgl_tuning()
    for k, v in dict(t).items():
        setattr(tt, k, int(v))
    return ctypes.byref(tt)


# ----------------------------------------------------------------------------- same-name wrappers

def irgl_last_error() -> str:
    return lib().irgl_last_error().decode(errors="replace")


def irgl_status_string(status: int) -> str:
    return lib().irgl_status_string(status).decode()


def irgl_ctx_create(device: int = 0, cuda_stream: int | None = None) -> int:
    h = _P()
    _check(lib().irgl_ctx_create(device, cuda_stream, ctypes.byref(h)))
    return h.value


def irgl_ctx_destroy(ctx: int) -> None:
    _check(lib().irgl_ctx_destroy(ctx))


def irgl_ctx_set_stream(ctx: int, cuda_stream: int | None) -> None:
    _check(lib().irgl_ctx_set_stream(ctx, cuda_stream))


def irgl_ctx_info(ctx: int) -> tuple[int, dict]:
    sm = c_uint32()
    t = irgl_tuning()
    _check(lib().irgl_ctx_info(ctx, ctypes.byref(sm), ctypes.byref(t)))
    return int(sm.value), t.as_dict()


def irgl_csr_validate(n: int, m: int, row_ptr: int, col: int, w: int | None, flags: int) -> None:
    _check(lib().irgl_csr_validate(n, m, row_ptr, col, w, flags))


def irgl_csr_load(ctx: int, n: int, m: int, row_ptr: int, col: int, w: int | None, flags: int) -> int:
    h = _P()
    _check(lib().irgl_csr_load(ctx, n, m, row_ptr, col, w, flags, ctypes.byref(h)))
    return h.value


def irgl_graph_destroy(g: int) -> None:
    _check(lib().irgl_graph_destroy(g))


def irgl_graph_info(g: int) -> tuple[int, int, int]:
    n, m, f = c_uint32(), c_uint64(), c_int()
    _check(lib().irgl_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(f)))
    return int(n.value), int(m.value), int(f.value)


def irgl_worklist_create(ctx: int, capacity: int) -> int:
    h = _P()
    _check(lib().irgl_worklist_create(ctx, capacity, ctypes.byref(h)))
    return h.value


def irgl_worklist_destroy(wl: int) -> None:
    _check(lib().irgl_worklist_destroy(wl))


def irgl_worklist_push(wl: int, items_host: int, k: int) -> None:
    _check(lib().irgl_worklist_push(wl, items_host, k))


def irgl_worklist_push_range(wl: int, k: int) -> None:
    _check(lib().irgl_worklist_push_range(wl, k))


def irgl_worklist_clear(wl: int) -> None:
    _check(lib().irgl_worklist_clear(wl))


def irgl_worklist_size(wl: int) -> int:
    n = c_uint32()
    _check(lib().irgl_worklist_size(wl, ctypes.byref(n)))
    return int(n.value)


def irgl_worklist_read(wl: int, items_host: int, cap: int) -> int:
    n = c_uint32()
    _check(lib().irgl_worklist_read(wl, items_host, cap, ctypes.byref(n)))
    return int(n.value)


def irgl_init_state(ctx: int, kernel: int, g: int, initial: int | None, state_dev: int) -> None:
    _check(lib().irgl_init_state(ctx, kernel, g, initial, state_dev))


def irgl_invoke(ctx: int, kernel: int, g: int, wl_in: int, wl_out: int, state_dev: int, level: int,
                reduce: int = IRGL_REDUCE_ANY, tuning=None) -> int:
    res = c_int()
    _check(lib().irgl_invoke(ctx, kernel, g, wl_in, wl_out, state_dev, level, reduce, _tuning(tuning),
                             ctypes.byref(res)))
    return int(res.value)


def irgl_iterate(ctx: int, kernel: int, g: int, initial: int | None, state_dev: int, mode: int = IRGL_PERSISTENT,
                 tuning=None, max_rounds: int = 0) -> dict:
    st = irgl_stats()
    _check(lib().irgl_iterate(ctx, kernel, g, initial, state_dev, mode, _tuning(tuning), max_rounds,
                              ctypes.byref(st)))
    return st.as_dict()


def irgl_iterate_async(ctx: int, kernel: int, g: int, initial: int | None, state_dev: int, tuning=None,
                       max_rounds: int = 0) -> None:
    _check(lib().irgl_iterate_async(ctx, kernel, g, initial, state_dev, _tuning(tuning), max_rounds))


def irgl_ctx_sync(ctx: int) -> dict:
    st = irgl_stats()
    _check(lib().irgl_ctx_sync(ctx, ctypes.byref(st)))
    return st.as_dict()


def irgl_run(ctx: int, kernel: int, g: int, srcs_host: int | None, nsrc: int, state: int, state_on_host: int,
             mode: int = IRGL_PERSISTENT, tuning=None, max_rounds: int = 0) -> dict:
    st = irgl_stats()
    _check(lib().irgl_run(ctx, kernel, g, srcs_host, nsrc, state, state_on_host, mode, _tuning(tuning), max_rounds,
                          ctypes.byref(st)))
    return st.as_dict()


def irgl_debug_set(ctx: int, key: int, value: int) -> None:
    _check(lib().irgl_debug_set(ctx, key, value))


def irgl_control_cta(masks, preferred: int = 0) -> int:
    arr = (c_uint32 * max(len(masks), 1))(*masks)
    out = c_uint32()
    _check(lib().irgl_control_cta(arr, len(masks), preferred, ctypes.byref(out)))
    return int(out.value)


def irgl_batch_create(ctx: int, max_queries: int) -> int:
    h = _P()
    _check(lib().irgl_batch_create(ctx, max_queries, ctypes.byref(h)))
    return h.value


def irgl_batch_destroy(b: int) -> None:
    _check(lib().irgl_batch_destroy(b))


def irgl_batch_add(b: int, g: int, kernel: int, srcs_host: int | None, nsrc: int) -> int:
    q = c_uint32()
    _check(lib().irgl_batch_add(b, g, kernel, srcs_host, nsrc, ctypes.byref(q)))
    return int(q.value)


def irgl_batch_prepare(b: int, tuning=None, use_cuda_graph: int = 1) -> None:
    _check(lib().irgl_batch_prepare(b, _tuning(tuning), use_cuda_graph))


def irgl_batch_set_wave_bytes(b: int, nbytes: int) -> None:
    _check(lib().irgl_batch_set_wave_bytes(b, nbytes))


def irgl_batch_waves(b: int) -> int:
    w = c_uint32()
    _check(lib().irgl_batch_waves(b, ctypes.byref(w)))
    return int(w.value)


def irgl_batch_launch(b: int) -> None:
    _check(lib().irgl_batch_launch(b))


def irgl_batch_sync(b: int) -> dict:
    st = irgl_stats()
    _check(lib().irgl_batch_sync(b, ctypes.byref(st)))
    return st.as_dict()


def irgl_batch_run(b: int) -> dict:
    st = irgl_stats()
    _check(lib().irgl_batch_run(b, ctypes.byref(st)))
    return st.as_dict()


def irgl_batch_info(b: int) -> dict:
    nq, grid, cta, arena = c_uint32(), c_uint32(), c_uint32(), c_uint64()
    cap = c_int()
    _check(lib().irgl_batch_info(b, ctypes.byref(nq), ctypes.byref(grid), ctypes.byref(cta), ctypes.byref(cap),
                                 ctypes.byref(arena)))
    return dict(nqueries=int(nq.value), grid=int(grid.value), cta_size=int(cta.value),
                graph_captured=bool(cap.value), arena_entries=int(arena.value), waves=irgl_batch_waves(b))


def irgl_batch_result(b: int, query_id: int) -> tuple[int, int, int]:
    p, n, r = _P(), c_uint32(), c_uint32()
    _check(lib().irgl_batch_result(b, query_id, ctypes.byref(p), ctypes.byref(n), ctypes.byref(r)))
    return int(p.value or 0), int(n.value), int(r.value)


def irgl_batch_copy_result(b: int, query_id: int, host_out: int) -> None:
    _check(lib().irgl_batch_copy_result(b, query_id, host_out))


def irgl_batch_copy_results(b: int, host_out: int) -> None:
    _check(lib().irgl_batch_copy_results(b, host_out))


def irgl_trace_enable(ctx: int, max_rounds: int) -> None:
    _check(lib().irgl_trace_enable(ctx, max_rounds))


def irgl_trace_phases(ctx: int, cap: int = 1 << 16):
    """Phase records of the last single-query persistent Iterate: uint64 array (rounds, 8)."""
    import numpy as np

    w = np.zeros((cap, 8), dtype=np.uint64)
    n = c_uint32()
    _check(lib().irgl_trace_phases(ctx, w.ctypes.data, cap, ctypes.byref(n)))
    return w[: int(n.value)]


def irgl_trace_read(ctx: int, cap: int = 1 << 16):
    """Per-round trace of the last persistent launch: (t_ns, in_n, out_n) numpy arrays."""
    import numpy as np

    t = np.zeros(cap, dtype=np.uint64)
    a = np.zeros(cap, dtype=np.uint32)
    b = np.zeros(cap, dtype=np.uint32)
    n = c_uint32()
    _check(lib().irgl_trace_read(ctx, t.ctypes.data, a.ctypes.data, b.ctypes.data, cap, ctypes.byref(n)))
    k = int(n.value)
    return t[:k], a[:k], b[:k]


def irgl_server_create(ctx: int, arena_bytes: int = 0, max_slots: int = 256, epoch_rounds: int = 64,
                       count_edges: int = 1, tuning=None, solo_min_n: int = 0) -> int:
    cfg = irgl_server_config()
    cfg.arena_bytes = arena_bytes
    cfg.max_slots = max_slots
    cfg.epoch_rounds = epoch_rounds
    cfg.count_edges = count_edges
    cfg.solo_min_n = solo_min_n
    if tuning is not None:
        for k, v in dict(tuning).items():
            setattr(cfg.tuning, k, int(v))
    h = _P()
    _check(lib().irgl_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def irgl_server_submit(srv: int, g: int, kernel: int, src: int, host_out: int | None = None) -> int:
    t = c_uint64()
    _check(lib().irgl_server_submit(srv, g, kernel, src, host_out, ctypes.byref(t)))
    return int(t.value)


def irgl_server_poll(srv: int, ticket: int) -> dict | None:
    info = irgl_query_info()
    rc = lib().irgl_server_poll(srv, ticket, ctypes.byref(info))
    if rc == IRGL_ERR_NOT_READY:
        return None
    _check(rc)
    return dict(status=int(info.status), rounds=int(info.rounds), latency_s=float(info.latency_s),
                t_submit_s=float(info.t_submit_s), t_done_s=float(info.t_done_s), edges=int(info.edges))


def irgl_server_drain(srv: int, timeout_ms: int = 600000) -> None:
    _check(lib().irgl_server_drain(srv, timeout_ms))


def irgl_server_stats(srv: int) -> dict:
    c = irgl_server_counters()
    _check(lib().irgl_server_stats(srv, ctypes.byref(c)))
    return c.as_dict()


def irgl_server_destroy(srv: int) -> None:
    _check(lib().irgl_server_destroy(srv))


def irgl_autotune(ctx: int, kernel: int, g: int, srcs_host: int | None, nsrc: int, reps: int = 3) -> tuple[dict, float]:
    t = irgl_tuning()
    ms = ctypes.c_float()
    _check(lib().irgl_autotune(ctx, kernel, g, srcs_host, nsrc, reps, ctypes.byref(t), ctypes.byref(ms)))
    return t.as_dict(), float(ms.value)


def irgl_batch_autotune(b: int, reps: int = 3) -> tuple[dict, float]:
    t = irgl_tuning()
    ms = ctypes.c_float()
    _check(lib().irgl_batch_autotune(b, reps, ctypes.byref(t), ctypes.byref(ms)))
    return t.as_dict(), float(ms.value)


def irgl_bfs_noalloc(device: int, cuda_stream: int | None, n: int, m: int, row_ptr: int, col: int, src: int,
                     level: int) -> int:
    rounds = c_uint32()
    _check(lib().irgl_bfs_noalloc(device, cuda_stream, n, m, row_ptr, col, src, level, ctypes.byref(rounds)))
    return int(rounds.value)


def irgl_msf(ctx: int, g: int, mode: int, lock: int, out_edges: int, cap: int, out_on_host: int,
             tuning=None) -> dict:
    st = irgl_msf_stats()
    _check(lib().irgl_msf(ctx, g, mode, lock, out_edges, cap, out_on_host, _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()
