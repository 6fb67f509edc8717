"""Context.close() frees the objects made on it first (graphs, worklists, batches
and servers keep a pointer to their context in the library), so a graph left
open by a failed test or a forgotten close() is never destroyed after its
context. Host-only check of the ordering with a stub library."""
from __future__ import annotations

import pytest


def test_context_closes_children_first(monkeypatch):
    pytest.importorskip("torch")
    from paper_1607_05707_gb300 import api
    from paper_1607_05707_gb300 import irgl as C

    calls = []
    monkeypatch.setattr(C, "irgl_graph_destroy", lambda h: calls.append(("graph", h)))
    monkeypatch.setattr(C, "irgl_worklist_destroy", lambda h: calls.append(("worklist", h)))
    monkeypatch.setattr(C, "irgl_batch_destroy", lambda h: calls.append(("batch", h)))
    monkeypatch.setattr(C, "irgl_server_destroy", lambda h: calls.append(("server", h)))
    monkeypatch.setattr(C, "irgl_ctx_destroy", lambda h: calls.append(("ctx", h)))

    ctx = object.__new__(api.Context)
    ctx.handle = 1
    ctx._children = api.weakref.WeakSet()
    objs = []
    for cls, h in ((api.Graph, 10), (api.Worklist, 11), (api.Server, 12), (api.Batch, 13), (api.Graph, 14)):
        o = object.__new__(cls)
        o.ctx, o.handle = ctx, h
        ctx._adopt(o)
        objs.append(o)
    objs[4].close()  # closed early by the user: not destroyed twice
    ctx.close()
    kinds = [k for k, _ in calls]
    assert kinds[0] == "graph" and calls[0][1] == 14
    assert kinds[1:] == ["server", "batch", "worklist", "graph", "ctx"]
    assert all(o.handle == 0 for o in objs) and ctx.handle == 0
    ctx.close()  # idempotent
    assert len(calls) == 6
