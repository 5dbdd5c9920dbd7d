"""Transient form (Eq. 2): (C + S/dt) h = Q with a cached hierarchy.

gw_hierarchy_shift keeps the aggregates and prolongators while
|s_i - s_built_i| < delta C_ii in every row, forming every coarse operator
again as P^T A P of the shifted level above, and rebuilds the hierarchy
otherwise.  A reused hierarchy is compared bit for bit, level by level, with
the oracle's numerically refreshed one, a rebuilt one with a fresh oracle
setup of C + diag(s), and every solve with the oracle's solution.
"""
import numpy as np
import pytest

import oracle
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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [0, 1])
def test_shift_reuse_and_rebuild(gw, prec):
    nx = ny = nz = 16
    p = wl.heterogeneous_3d(side=nx, var=3.0, corr=4.0, seed=9)
    K = dev(p["Kx"])
    b = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(nx, ny, nz, K, K, K, p["bct"], p["bcv"], None, b_out=b)
    H = gw.Hierarchy(A, prec=prec, n_coarse=100)
    C, bo = oracle.assemble(nx, ny, nz, p["Kx"])
    Cd = C.dense()
    d = np.diag(Cd)
    rng = np.random.default_rng(3)
    h_prev = rng.normal(size=C.nr)

    def same_levels(Href):
        for l in range(Href.nlevels):
            agg, root, (arp, aci, av), _ = H.export_level(l)
            orp, oci, ov = Href.A(l).arrays()
            assert np.array_equal(aci, oci) and np.array_equal(av.view(np.uint64), ov.view(np.uint64)), l

    def step(s, expect_rebuild, Href):
        rb = H.shift(dev(s), delta=0.01)
        assert rb == expect_rebuild
        if Href is not None:
            same_levels(Href)
        rhs = bo + s * h_prev
        h, it, rel, st = H.solve(dev(rhs), tol=1e-10)
        assert st == gw.GW_OK and rel <= 1e-10
        As = oracle.shift(C, s)
        ref = np.linalg.solve(As.dense(), rhs)
        assert np.linalg.norm(h.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
        if prec == 0 and Href is not None:
            _, it_ref, _, _ = Href.pcg(rhs, tol=1e-10)
            assert abs(it - it_ref) <= 1
        return As

    # small storage term: the aggregates of C are kept, the coarse operators formed again
    s1 = 0.005 * d * (0.5 + rng.random(C.nr))
    Ho = oracle.Hierarchy(C, n_coarse=100)
    Ho.refresh_numeric(oracle.shift(C, s1))
    step(s1, 2, Ho)
    # within a quarter of that shift: the coarse operators are kept, level 0 refreshed
    s1b = s1 * (1.0 + 0.2 * (rng.random(C.nr) - 0.5))
    Ho.refresh_level0(oracle.shift(C, s1b))
    step(s1b, 0, Ho)
    # large storage term (short time step): rebuilt for C + diag(s2), bit-exact setup
    s2 = 0.5 * d
    As2 = step(s2, 1, oracle.Hierarchy(oracle.shift(C, s2), n_coarse=100))
    # a small change relative to the rebuilt shift reuses it again
    s3 = s2 + 0.004 * d
    Ho3 = oracle.Hierarchy(As2, n_coarse=100)
    Ho3.refresh_level0(oracle.shift(C, s3))
    step(s3, 0, Ho3)
    # back to the steady operator: far from the built shift, rebuilt
    assert H.shift(None, delta=0.01) == 1
    h, it, rel, st = H.solve(dev(bo), tol=1e-10)
    ref = np.linalg.solve(Cd, bo)
    assert st == gw.GW_OK and np.linalg.norm(h.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_shift_rejects_bad_delta(gw):
    p = wl.problem(10, 10, 10)
    A, b = gw.gw_assemble(10, 10, 10, p["Kx"])
    H = gw.Hierarchy(A, n_coarse=100)
    with pytest.raises(gw.GwError):
        H.shift(np.zeros(1000), delta=0.0)
