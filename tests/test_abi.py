"""The C-ABI library loads and exports every entry point include/ect.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ect.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ect_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_03207_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = header_symbols()
    for s in ("ect_create", "ect_set_mesh", "ect_set_physics", "ect_assemble", "ect_coil_rhs", "ect_solve",
              "ect_impedance", "ect_last_error", "ect_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1602_03207_gb300 import ect
    missing = [s for s in header_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(ect.EXPORTS) == header_symbols()


def test_default_options_without_gpu(lib):
    from paper_1602_03207_gb300 import ect
    o = ect.default_options()
    assert o.tol == 1e-10 and o.restart == 30 and o.mode == ect.ECT_MODE_F64 and o.use_graph == 1
    # staged FP32 SpMM with automatic rows, selective reorthogonalisation, zero initial guess
    assert o.spmm_rows == 0 and o.reorth == 1 and o.x0 == 0


def test_options_layout_matches_header():
    """The binding's ect_options fields are the header's, in the header's order."""
    from paper_1602_03207_gb300 import ect
    src = open(os.path.join(ROOT, "include", "ect.h")).read()
    body = src[src.index("typedef struct {\n    double tol;"):]
    body = body[:body.index("} ect_options;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(?:double|int)\s+([a-z_0-9]+)\s*;", body)
    assert names == [f for f, _ in ect.Options._fields_]


def test_null_context_rejected(lib):
    from paper_1602_03207_gb300 import ect
    L = ect.load_library()
    assert L.ect_set_physics(None, 1e5, 1.0, 1.0) == ect.ECT_ERR_ARG
    assert L.ect_assemble(None, 0, 1) == ect.ECT_ERR_ARG
    assert L.ect_last_error(None) is not None


def test_stats_layout_matches_header():
    """The binding's ect_stats fields are the header's, in the header's order."""
    from paper_1602_03207_gb300 import ect
    src = open(os.path.join(ROOT, "include", "ect.h")).read()
    body = src[src.index("typedef struct {\n    int iters;"):]
    body = body[:body.index("} ect_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(?:double|int|int64_t)\s+([a-z_0-9]+)\s*;", body)
    assert names == [f for f, _ in ect.Stats._fields_]
