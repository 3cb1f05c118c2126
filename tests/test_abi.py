"""The C interface library loads and exports every symbol the header
declares; argument checks that need no GPU (no compute call here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "osmodi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi.lib()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"OSMODI_API\s+[\w\s\*]+?\b(osmodi_\w+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = _declared()
    for must in ("osmodi_create", "osmodi_solve", "osmodi_solve_batched", "osmodi_destroy", "osmodi_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2311_16935_gb300 import osmodi

    for name in _declared():
        assert hasattr(lib, name), name
        assert name in osmodi.exported_symbols(), name


def test_status_strings(lib):
    from paper_2311_16935_gb300 import osmodi

    assert osmodi.status_string(0) == "ok"
    assert "valid" in osmodi.status_string(-7)
    assert osmodi.status_string(12345) == "unknown status"


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_2311_16935_gb300 import osmodi

    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 1)
    sp = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.osmodi_create(4, dims, sp, None, None, None, ctypes.byref(h)) == osmodi.E_INVALID
    bad = (ctypes.c_double * 3)(1.0, -1.0, 1.0)
    assert lib.osmodi_create(2, dims, bad, None, None, None, ctypes.byref(h)) == osmodi.E_INVALID
    zero = (ctypes.c_int64 * 3)(0, 4, 1)
    assert lib.osmodi_create(2, zero, sp, None, None, None, ctypes.byref(h)) == osmodi.E_INVALID
    assert lib.osmodi_create(2, dims, sp, None, None, None, None) == osmodi.E_INVALID
    o = osmodi.osmodi_options()
    lib.osmodi_default_options(ctypes.byref(o))
    o.precision = 7
    assert lib.osmodi_create(2, dims, sp, None, ctypes.byref(o), None, ctypes.byref(h)) == osmodi.E_INVALID
    # multigrid smoothing sweeps 1..8 and coarse scale (0, 4] (0 = default)
    for field, value in (("mg_sweeps", 9), ("mg_sweeps", -1), ("mg_scale", -0.5), ("mg_scale", 4.5),
                         ("mg_scale", float("nan")), ("refine_ff", 2)):
        lib.osmodi_default_options(ctypes.byref(o))
        setattr(o, field, value)
        assert lib.osmodi_create(2, dims, sp, None, ctypes.byref(o), None, ctypes.byref(h)) == osmodi.E_INVALID


def test_solve_rejects_null_plan(lib):
    from paper_2311_16935_gb300 import osmodi

    assert lib.osmodi_solve(None, None, 0, None, 0, 1e-8, 10, None, None, None) == osmodi.E_INVALID
    assert lib.osmodi_workspace_bytes(None) == 0
    assert lib.osmodi_history(None, None, 0) == 0


def test_default_options(lib):
    from paper_2311_16935_gb300 import osmodi

    o = osmodi.default_options()
    assert o.precision == osmodi.FP32_REFINE and o.scheme == osmodi.FPCG
    assert o.check_every >= 0 and o.max_refine >= 1
    assert o.mg_sweeps == 0 and o.mg_scale == 0.0 and o.zero_start == 0 and o.precond == 0
    assert o.refine_ff == 0  # FP64 refinement unless asked


def test_product_does_not_import_oracle():
    """The CUDA path never routes through the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2311_16935_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), fn
                assert "liboracle" not in txt, fn


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: a missing libosmodi.so is an ImportError at the first
    call, not a silent substitute."""
    from paper_2311_16935_gb300 import osmodi

    monkeypatch.setattr(osmodi, "LIB_PATH", str(tmp_path / "libosmodi_missing.so"))
    monkeypatch.setattr(osmodi, "_lib", None)
    with pytest.raises(ImportError):
        osmodi.default_options()


def test_binding_argument_checks(lib):
    """Host-side checks of the binding, before any device work."""
    import torch
    from paper_2311_16935_gb300 import osmodi

    with pytest.raises(TypeError):
        osmodi.default_options(no_such_option=1)
    o = osmodi.default_options(precond=1, mg_sweeps=3, mg_scale=1.5, refine_ff=1, zero_start=1)
    assert (o.precond, o.mg_sweeps, o.mg_scale, o.refine_ff, o.zero_start) == (1, 3, 1.5, 1, 1)
    with pytest.raises(ValueError):
        osmodi._check_cuda(torch.zeros(4), "grad")  # a host tensor is not a device buffer
    with pytest.raises(ValueError):
        osmodi._check_solve_buffer(torch.zeros(4), "grad")  # nor is unpinned host memory
    with pytest.raises(ValueError):
        osmodi._check_solve_buffer(torch.zeros(4, 4).t(), "grad")  # nor a strided view
