"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every symbol declared in include/irgl.h, and its host-side CSR
validation rejects malformed input (no compute call needs a GPU here)."""
from __future__ import annotations

import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_1607_05707_gb300 import _build, irgl

    _build.build_irgl()
    return irgl.lib()


def declared(header: str) -> list[str]:
    text = (ROOT / "include" / header).read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(irgl\w*)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_1607_05707_gb300 import irgl

    names = declared("irgl.h")
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), f"libirgl.so does not export {name}"
    # and the Python binding wraps exactly what the header declares
    assert sorted(irgl.exported_symbols()) == names


def test_generator_exports():
    import ctypes

    from paper_1607_05707_gb300 import _build

    g = ctypes.CDLL(str(_build.build_gen()))
    for name in declared("irgl_gen.h"):
        assert hasattr(g, name)


def _validate(n, row_ptr, col, w=None, flags=0):
    from paper_1607_05707_gb300 import irgl

    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    c = np.ascontiguousarray(col, dtype=np.uint32)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
    irgl.irgl_csr_validate(n, c.size, rp.ctypes.data, c.ctypes.data, None if ww is None else ww.ctypes.data, flags)


def test_host_validation(lib):
    from paper_1607_05707_gb300 import irgl

    _validate(3, [0, 1, 2, 2], [1, 2], [5, 0])
    _validate(3, [0, 1, 2, 2], [1, 0], None)
    cases = [
        (3, [1, 1, 2, 2], [1, 2], None, 0, irgl.IRGL_ERR_INVALID_ARG),      # row_ptr[0] != 0
        (3, [0, 2, 1, 2], [1, 2], None, 0, irgl.IRGL_ERR_INVALID_ARG),      # not monotone
        (3, [0, 1, 2, 3], [1, 2], None, 0, irgl.IRGL_ERR_INVALID_ARG),      # row_ptr[n] != m
        (3, [0, 1, 2, 2], [1, 3], None, 0, irgl.IRGL_ERR_INVALID_ARG),      # col >= n
        (3, [0, 1, 2, 2], [1, 2], [1, -1], 0, irgl.IRGL_ERR_INVALID_ARG),   # negative weight
        (3, [0, 1, 2, 2], [1, 2], None, irgl.IRGL_SYMMETRIC, irgl.IRGL_ERR_NOT_SYMMETRIC),
    ]
    for n, rp, col, w, flags, code in cases:
        with pytest.raises(irgl.IrglError) as ei:
            _validate(n, rp, col, w, flags)
        assert ei.value.status == code
    _validate(3, [0, 1, 3, 4], [1, 0, 2, 1], None, irgl.IRGL_SYMMETRIC)


def test_status_strings(lib):
    from paper_1607_05707_gb300 import irgl

    assert irgl.irgl_status_string(irgl.IRGL_ERR_WL_OVERFLOW) == "worklist overflow"
    assert irgl.irgl_status_string(0) == "ok"


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_1607_05707_gb300 import _build, irgl

    monkeypatch.setattr(_build, "IRGL_LIB", tmp_path / "libirgl.so")
    monkeypatch.setattr(irgl, "_lib", None)
    with pytest.raises(ImportError):
        irgl.lib()
