"""CPU checks of the C ABI library and of the product/oracle separation.

No compute call is made here: the library is built (nvcc cross-compiles
sm_103a), loaded, and checked to export every entry point include/gw.h
declares.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|long long)\s*\*?\s*(gw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_05798_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gw_assemble", "gw_amg_setup", "gw_pcg_solve", "gw_hierarchy_info", "gw_matrix_free",
                     "gw_hierarchy_free", "gw_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2001_05798_gb300 import gw

    assert sorted(gw.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(lib):
    from paper_2001_05798_gb300 import gw

    L = gw.load()
    assert L.gw_status_str(0) == b"GW_OK"
    assert L.gw_status_str(5) == b"GW_ERR_NOT_CONVERGED"
    o = gw.amg_opts()
    assert abs(o.theta - 0.04) < 1e-15 and o.n_coarse == 1024 and o.seed == 0x5EED and o.smoother == 1


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2001_05798_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gw_oracle" not in text and "liboracle" not in text, f


def test_null_arguments_are_rejected_without_a_device(lib):
    """Every entry point checks its handles and pointers before it touches the
    GPU: a null argument returns GW_ERR_ARG with a message, and nothing aborts."""
    from paper_2001_05798_gb300 import gw

    L = gw.load()
    it, rel, rb = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    calls = {
        "gw_pcg_solve": lambda: L.gw_pcg_solve(None, None, None, 1e-8, 10, ctypes.byref(it), ctypes.byref(rel), None),
        "gw_pcg_solve_many": lambda: L.gw_pcg_solve_many(None, 2, None, None, 1e-8, 10, None, None, None),
        "gw_hierarchy_prepare": lambda: L.gw_hierarchy_prepare(None),
        "gw_hierarchy_shift": lambda: L.gw_hierarchy_shift(None, None, 0.01, ctypes.byref(rb), None),
        "gw_vcycle": lambda: L.gw_vcycle(None, None, None, None),
        "gw_amg_setup": lambda: L.gw_amg_setup(None, None, None, None),
        "gw_darcy_flux": lambda: L.gw_darcy_flux(None, None, None, None, None, None, None, None, None, None),
        "gw_adjoint_gradient": lambda: L.gw_adjoint_gradient(None, None, None, None, None, None, None, None, None),
        "gw_matrix_size": lambda: L.gw_matrix_size(None, None, None),
        "gw_hierarchy_info": lambda: L.gw_hierarchy_info(None, None, 0, None),
    }
    for name, call in calls.items():
        assert call() == gw.GW_ERR_ARG, name
        assert L.gw_last_error(), name
