"""Failure paths of the C ABI, driven from the host.

Every failure here is made on the host side (an option that caps the MIS-2
rounds, a right-hand side with a non-finite entry); none of them faults or
hangs the GPU.  Each case checks the status code, that the call returned
instead of waiting, and that the same hierarchy or matrix still solves
correctly afterwards (the context stays usable).
"""
import time

import numpy as np
import pytest

from paper_2001_05798_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05798_gb300 import build, gw as gwm

    build.build()
    gwm.load()
    return gwm


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def system(gw):
    p = wl.problem(24, 20, 16, var=3.0, corr=4.0, seed=21, wells_count=3, wells_seed=2)
    n = p["nx"] * p["ny"] * p["nz"]
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(p["nx"], p["ny"], p["nz"], dev(p["Kx"]), dev(p["Ky"]), dev(p["Kz"]), p["bct"], p["bcv"],
                          dev(p["q"]), b_out=b)
    torch.cuda.synchronize()
    return A, b


def test_mis2_round_cap_reports_a_setup_failure(gw, system):
    A, b = system
    # one round cannot finish the distance-2 independent set of a 3D grid
    with pytest.raises(gw.GwError) as e:
        gw.Hierarchy(A, n_coarse=64, mis_max_rounds=1)
    assert e.value.status == gw.GW_ERR_SETUP
    assert "MIS-2" in str(e.value)
    with pytest.raises(gw.GwError) as e:
        gw.Hierarchy(A, n_coarse=64, mis_max_rounds=-1)
    assert e.value.status == gw.GW_ERR_ARG
    with pytest.raises(gw.GwError) as e:  # bit 1 (FP16 transfer operators) no longer exists
        gw.Hierarchy(A, n_coarse=64, half_storage=1)
    assert e.value.status == gw.GW_ERR_ARG
    # the matrix and the device are still usable: the default cap sets up and solves
    H = gw.Hierarchy(A, n_coarse=64)
    h, it, rel, st = H.solve(b, tol=1e-8)
    assert st == gw.GW_OK and rel <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed32"])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_right_hand_side_is_rejected(gw, system, prec, bad):
    A, b = system
    H = gw.Hierarchy(A, n_coarse=64, prec=gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED32)
    bb = b.clone()
    bb[17] = bad
    t0 = time.perf_counter()
    with pytest.raises(gw.GwError) as e:
        H.solve(bb, tol=1e-8)
    assert time.perf_counter() - t0 < 30.0
    assert e.value.status == gw.GW_ERR_ARG and "non-finite" in str(e.value)
    # the hierarchy solves a good right-hand side afterwards, bit for bit as a fresh one
    h, it, rel, st = H.solve(b, tol=1e-8)
    H2 = gw.Hierarchy(A, n_coarse=64, prec=gw.GW_PREC_FP64 if prec == "fp64" else gw.GW_PREC_MIXED32)
    h2, it2, rel2, st2 = H2.solve(b, tol=1e-8)
    assert st == st2 == gw.GW_OK and it == it2 and torch.equal(h, h2)


def test_non_finite_column_of_a_block_solve(gw, system):
    A, b = system
    H = gw.Hierarchy(A, n_coarse=64)
    B = torch.stack([b, 0.5 * b, b.clone(), 2.0 * b])
    B[2, 5] = np.nan
    with pytest.raises(gw.GwError) as e:
        H.solve_many(B.contiguous(), tol=1e-8)
    assert e.value.status == gw.GW_ERR_ARG
    # the good columns alone still solve to the tolerance afterwards
    X, its, rels, st = H.solve_many(torch.stack([b, 0.5 * b]).contiguous(), tol=1e-8)
    assert st == gw.GW_OK and max(rels) <= 1e-8


def test_index_validation_of_every_level(gw):
    """GW_VALIDATE=1 checks every index array the cycle kernels gather through
    (all levels' CSR row pointers and columns, sliced-ELL columns and row
    permutations, the implicit level-0 transfer's lists) after the setup; the
    variable is read once per process, so the check runs in a child process."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import torch\n"
            "from paper_2001_05798_gb300 import gw, workload as wl\n"
            "for shape, prec in (((33, 31, 29), 1), ((20, 18, 16), 0), ((64, 64, 32), 1)):\n"
            "    p = wl.problem(*shape, var=3.0, corr=4.0, seed=2)\n"
            "    n = shape[0] * shape[1] * shape[2]\n"
            "    K = torch.from_numpy(p['Kx']).cuda()\n"
            "    b = torch.empty(n, dtype=torch.float64, device='cuda')\n"
            "    A, _ = gw.gw_assemble(*shape, K, K, K, p['bct'], p['bcv'], None, b_out=b)\n"
            "    H = gw.Hierarchy(A, n_coarse=64, prec=prec)\n"
            "    h, it, rel, st = H.solve(b, tol=1e-8)\n"
            "    assert st == 0 and rel <= 1e-8, (st, rel)\n"
            "print('validated')\n") % root
    env = dict(os.environ, GW_VALIDATE="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "validated" in r.stdout, r.stdout + r.stderr
