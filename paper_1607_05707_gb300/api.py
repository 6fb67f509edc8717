"""Torch-facing convenience layer over the C-ABI binding (marshalling only).

PyTorch supplies device memory and the CUDA stream; every traversal step runs in
libirgl.so's kernels through the same-name functions of :mod:`.irgl`.
"""
from __future__ import annotations

import weakref

import numpy as np
import torch

from . import irgl as C
from .inputs import CSR


def _np_ptr(a: np.ndarray | None) -> int | None:
    return None if a is None else int(a.ctypes.data)


class Graph:
    """A CSR graph resident on the device (owned by the library)."""

    def __init__(self, ctx: "Context", g: CSR, symmetric: bool | None = None, validate: bool = True,
                 in_edges: bool = False):
        self.ctx = ctx
        self.n, self.m = g.n, g.m
        self.symmetric = g.symmetric if symmetric is None else symmetric
        flags = C.IRGL_HOST_PTRS | (C.IRGL_SYMMETRIC if self.symmetric else 0) | (C.IRGL_VALIDATE if validate else 0)
        if in_edges:
            flags |= C.IRGL_IN_EDGES
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint32)
        col = np.ascontiguousarray(g.col, dtype=np.uint32)
        w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
        self.weighted = w is not None
        self.handle = C.irgl_csr_load(ctx.handle, g.n, g.m, _np_ptr(rp), _np_ptr(col), _np_ptr(w), flags)
        ctx._adopt(self)

    def close(self) -> None:
        if self.handle:
            C.irgl_graph_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Worklist:
    def __init__(self, ctx: "Context", capacity: int):
        self.ctx = ctx
        self.capacity = capacity
        self.handle = C.irgl_worklist_create(ctx.handle, capacity)
        ctx._adopt(self)

    def push(self, items) -> None:
        a = np.ascontiguousarray(np.atleast_1d(items), dtype=np.uint32)
        C.irgl_worklist_push(self.handle, _np_ptr(a), a.size)

    def push_range(self, k: int) -> None:
        C.irgl_worklist_push_range(self.handle, k)

    def clear(self) -> None:
        C.irgl_worklist_clear(self.handle)

    def size(self) -> int:
        return C.irgl_worklist_size(self.handle)

    def read(self) -> np.ndarray:
        buf = np.empty(self.capacity, dtype=np.uint32)
        n = C.irgl_worklist_read(self.handle, _np_ptr(buf), self.capacity)
        return buf[: min(n, self.capacity)].copy()

    def close(self) -> None:
        if self.handle:
            C.irgl_worklist_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Device + stream binding (defaults to torch's current stream on ``device``)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.handle = C.irgl_ctx_create(device, self.stream.cuda_stream)
        self.sm_count, self.default_tuning = C.irgl_ctx_info(self.handle)
        # objects made on this context: the library frees them before the context
        self._children: weakref.WeakSet = weakref.WeakSet()

    def _adopt(self, obj) -> None:
        self._children.add(obj)

    def load(self, g: CSR, symmetric: bool | None = None, validate: bool = True, in_edges: bool = False) -> Graph:
        return Graph(self, g, symmetric, validate, in_edges)

    def worklist(self, capacity: int) -> Worklist:
        return Worklist(self, capacity)

    def state(self, n: int) -> torch.Tensor:
        return torch.empty(max(n, 1), dtype=torch.int32, device=f"cuda:{self.device}")

    def iterate(self, kernel: str, g: Graph, initial: Worklist | None, out: torch.Tensor | None = None,
                mode: str = "persistent", tuning=None, max_rounds: int = 0) -> tuple[torch.Tensor, dict]:
        out = self.state(g.n) if out is None else out
        st = C.irgl_iterate(self.handle, C.KERNELS[kernel], g.handle, None if initial is None else initial.handle,
                            out.data_ptr(), C.MODES[mode], tuning, max_rounds)
        return out, st

    def iterate_async(self, kernel: str, g: Graph, initial: Worklist | None, out: torch.Tensor,
                      tuning=None, max_rounds: int = 0) -> None:
        C.irgl_iterate_async(self.handle, C.KERNELS[kernel], g.handle, None if initial is None else initial.handle,
                             out.data_ptr(), tuning, max_rounds)

    def sync(self) -> dict:
        return C.irgl_ctx_sync(self.handle)

    def run(self, kernel: str, g: Graph, srcs=None, out: torch.Tensor | None = None, mode: str = "persistent",
            tuning=None, max_rounds: int = 0) -> tuple[torch.Tensor, dict]:
        """One query; result stays on the device (int32 view of the uint32 values)."""
        out = self.state(g.n) if out is None else out
        s = None if srcs is None else np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.uint32)
        st = C.irgl_run(self.handle, C.KERNELS[kernel], g.handle, _np_ptr(s), 0 if s is None else s.size,
                        out.data_ptr(), 0, C.MODES[mode], tuning, max_rounds)
        return out, st

    def run_host(self, kernel: str, g: Graph, srcs=None, out: np.ndarray | None = None, mode: str = "persistent",
                 tuning=None, max_rounds: int = 0) -> tuple[np.ndarray, dict]:
        """One query with host buffers: sources in, uint32 result out (copies inside the call)."""
        out = np.empty(g.n, dtype=np.uint32) if out is None else out
        s = None if srcs is None else np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.uint32)
        st = C.irgl_run(self.handle, C.KERNELS[kernel], g.handle, _np_ptr(s), 0 if s is None else s.size,
                        _np_ptr(out), 1, C.MODES[mode], tuning, max_rounds)
        return out, st

    def invoke(self, kernel: str, g: Graph, wl_in: Worklist, wl_out: Worklist, state: torch.Tensor, level: int = 0,
               reduce: str = "any", tuning=None) -> int:
        return C.irgl_invoke(self.handle, C.KERNELS[kernel], g.handle, wl_in.handle, wl_out.handle, state.data_ptr(),
                             level, C.IRGL_REDUCE_ANY if reduce == "any" else C.IRGL_REDUCE_ALL, tuning)

    def msf(self, g: Graph, mode: str = "persistent", lock: str = "blocking", tuning=None,
            out: np.ndarray | None = None) -> tuple[np.ndarray, dict]:
        """Minimum spanning forest (Boruvka): CSR indices of its edges (one direction each, any order)."""
        cap = max(g.n - 1, 1)
        buf = np.empty(cap, dtype=np.uint32) if out is None else out
        st = C.irgl_msf(self.handle, g.handle, C.MODES[mode], C.LOCKS[lock], _np_ptr(buf), buf.size, 1, tuning)
        return buf[: st["edges"]].copy(), st

    def autotune(self, kernel: str, g: Graph, srcs=None, reps: int = 3) -> tuple[dict, float]:
        """Fastest tuning for persistent runs of `kernel` from `srcs` on g, and its median ms."""
        s = None if srcs is None else np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.uint32)
        return C.irgl_autotune(self.handle, C.KERNELS[kernel], g.handle, _np_ptr(s), 0 if s is None else s.size, reps)

    def init_state(self, kernel: str, g: Graph, initial: Worklist | None, state: torch.Tensor) -> None:
        C.irgl_init_state(self.handle, C.KERNELS[kernel], g.handle, None if initial is None else initial.handle,
                          state.data_ptr())

    def debug_set(self, key: int, value: int) -> None:
        C.irgl_debug_set(self.handle, key, value)

    def close(self) -> None:
        if self.handle:
            # servers and batches hold graphs; graphs and worklists hold the context
            live = list(self._children)
            for kind in (Server, Batch, Worklist, Graph):
                for obj in live:
                    if isinstance(obj, kind):
                        obj.close()
            C.irgl_ctx_destroy(self.handle)
            self.handle = 0


def as_u32(t: torch.Tensor) -> np.ndarray:
    """Device int32 tensor holding uint32 values -> host uint32 array."""
    return t.detach().cpu().numpy().view(np.uint32)


class Batch:
    """Many queries in one persistent launch (optionally replayed from a CUDA graph)."""

    def __init__(self, ctx: Context, max_queries: int = 1024):
        self.ctx = ctx
        self.handle = C.irgl_batch_create(ctx.handle, max_queries)
        ctx._adopt(self)
        self.sizes: list[int] = []

    def add(self, kernel: str, g: Graph, srcs=None) -> int:
        s = None if srcs is None else np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.uint32)
        q = C.irgl_batch_add(self.handle, g.handle, C.KERNELS[kernel], _np_ptr(s), 0 if s is None else s.size)
        self.sizes.append(g.n)
        return q

    def prepare(self, tuning=None, use_cuda_graph: bool = True, wave_bytes: int | None = None) -> dict:
        """wave_bytes: packed-state budget of one wave (0 or 2**64 - 1 = one wave, the default)."""
        if wave_bytes is not None:
            C.irgl_batch_set_wave_bytes(self.handle, wave_bytes)
        C.irgl_batch_prepare(self.handle, tuning, 1 if use_cuda_graph else 0)
        return C.irgl_batch_info(self.handle)

    def autotune(self, reps: int = 3) -> tuple[dict, float]:
        """Fastest tuning for this batch (prepared with it afterwards) and its median ms."""
        return C.irgl_batch_autotune(self.handle, reps)

    def launch(self) -> None:
        C.irgl_batch_launch(self.handle)

    def sync(self) -> dict:
        return C.irgl_batch_sync(self.handle)

    def run(self) -> dict:
        return C.irgl_batch_run(self.handle)

    def result(self, q: int) -> tuple[np.ndarray, int]:
        """Host copy of query q's result and the rounds it was active."""
        _, n, rounds = C.irgl_batch_result(self.handle, q)
        out = np.empty(max(n, 1), dtype=np.uint32)
        C.irgl_batch_copy_result(self.handle, q, _np_ptr(out))
        return out[:n], rounds

    def results(self, out: np.ndarray | None = None) -> list[np.ndarray]:
        """Every query's result from one device-to-host copy (views into `out`, add order)."""
        total = sum(self.sizes)
        out = np.empty(max(total, 1), dtype=np.uint32) if out is None else out
        if out.dtype != np.uint32 or out.size < total or not out.flags.c_contiguous:
            raise ValueError(f"out must be a contiguous uint32 array of at least {total} entries")
        C.irgl_batch_copy_results(self.handle, _np_ptr(out))
        offs = np.cumsum([0] + self.sizes)
        return [out[offs[i]:offs[i + 1]] for i in range(len(self.sizes))]

    def close(self) -> None:
        if self.handle:
            C.irgl_batch_destroy(self.handle)
            self.handle = 0


def trace(ctx: Context):
    """(t_ns, in_n, out_n) per round of the context's last persistent launch (tracing must be enabled)."""
    return C.irgl_trace_read(ctx.handle)


class Server:
    """Continuous-batching query server over device-resident graphs."""

    def __init__(self, ctx: Context, arena_bytes: int = 0, max_slots: int = 256, epoch_rounds: int = 64,
                 count_edges: bool = True, tuning=None, solo_min_n: int = 0):
        self.ctx = ctx
        self.handle = C.irgl_server_create(ctx.handle, arena_bytes, max_slots, epoch_rounds, int(count_edges), tuning,
                                           solo_min_n)
        ctx._adopt(self)

    def submit(self, kernel: str, g: Graph, src: int, out: np.ndarray | None = None) -> int:
        return C.irgl_server_submit(self.handle, g.handle, C.KERNELS[kernel], int(src), _np_ptr(out))

    def poll(self, ticket: int) -> dict | None:
        return C.irgl_server_poll(self.handle, ticket)

    def drain(self, timeout_s: float = 600.0) -> None:
        C.irgl_server_drain(self.handle, int(timeout_s * 1000))

    def stats(self) -> dict:
        return C.irgl_server_stats(self.handle)

    def close(self) -> None:
        if self.handle:
            C.irgl_server_destroy(self.handle)
            self.handle = 0
