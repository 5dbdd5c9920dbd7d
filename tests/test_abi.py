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
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(gw_\w+)\s*\(", src, flags=re.M)
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
