"""Darcy face velocities and several right-hand sides on one hierarchy.

gw_darcy_flux is compared face by face with the oracle's staggered-grid
fluxes (anisotropic spacing, both boundary kinds, three conductivity
fields); gw_pcg_solve_many with column-by-column single solves and with the
oracle's solutions of the same systems.
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


@pytest.mark.parametrize("bct,bcv", [((1, 1, 0, 0, 0, 0), (1.0, 0.0, 0, 0, 0, 0)),
                                     ((0, 1, 1, 0, 0, 1), (0, 0.3, -0.7, 0, 0, 2.0))])
@pytest.mark.parametrize("shape", [(23, 17, 9), (1, 40, 3), (64, 1, 1)])
def test_darcy_flux_matches_oracle(gw, shape, bct, bcv):
    nx, ny, nz = shape
    p = wl.problem(nx, ny, nz, var=3.0, corr=3.0, seed=4, kz_ratio=5.0, bct=bct, bcv=bcv)
    rng = np.random.default_rng(8)
    h = rng.normal(size=nx * ny * nz)
    sp = (2.0, 1.0, 0.5)
    ref = oracle.darcy_flux(nx, ny, nz, p["Kx"], h, p["Ky"], p["Kz"], bct, bcv, spacing=sp)
    v = [torch.full((r.size,), np.nan, dtype=torch.float64, device="cuda") for r in ref]
    gw.gw_darcy_flux(nx, ny, nz, dev(p["Kx"]), dev(h), *v, Ky=dev(p["Ky"]), Kz=dev(p["Kz"]), bct=bct, bcv=bcv,
                     spacing=sp)
    for a, r in zip(v, ref):
        np.testing.assert_allclose(a.cpu().numpy(), r, rtol=1e-14, atol=1e-15 * np.abs(r).max())


def test_darcy_flux_of_a_solve_balances_sources(gw):
    """Heads solved by the GPU path: the net outflow of every cell's faces is its source."""
    nx, ny, nz = 32, 24, 16
    p = wl.problem(nx, ny, nz, var=2.0, corr=4.0, seed=3, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0))
    q = np.zeros(nx * ny * nz)
    q[wl.cells(q.size, 5, 1)] = [0.4, -0.3, 0.2, -0.1, 0.05]
    K = dev(p["Kx"])
    b = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(nx, ny, nz, K, K, K, p["bct"], p["bcv"], dev(q), b_out=b)
    h, it, rel, st = gw.Hierarchy(A).solve(b, tol=1e-12)
    assert st == gw.GW_OK
    v = [torch.empty(n, dtype=torch.float64, device="cuda") for n in
         ((nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1))]
    gw.gw_darcy_flux(nx, ny, nz, K, h, *v, bct=p["bct"], bcv=p["bcv"])
    vx = v[0].cpu().numpy().reshape(nz, ny, nx + 1)
    vy = v[1].cpu().numpy().reshape(nz, ny + 1, nx)
    vz = v[2].cpu().numpy().reshape(nz + 1, ny, nx)
    out = (vx[:, :, 1:] - vx[:, :, :-1]) + (vy[:, 1:, :] - vy[:, :-1, :]) + (vz[1:] - vz[:-1])
    np.testing.assert_allclose(out.ravel(), q, atol=1e-9)


def test_darcy_flux_rejects_host_arrays(gw):
    a = np.zeros(8)
    with pytest.raises(gw.GwError):
        gw.gw_darcy_flux(2, 2, 2, a, a, np.zeros(12), np.zeros(12), np.zeros(12))


def test_solve_many_fp64_equals_single_solves_bitwise(gw):
    """The FP64 form solves the columns one after another: bit-identical to gw_pcg_solve."""
    side, k = 20, 3
    p = wl.heterogeneous_3d(side=side, var=3.0, corr=4.0, seed=2)
    A, b = gw.gw_assemble(side, side, side, p["Kx"])
    H = gw.Hierarchy(A, prec=0, n_coarse=200)
    B = np.random.default_rng(4).normal(size=(k, side ** 3))
    Ao, _ = oracle.assemble(side, side, side, p["Kx"])
    Ho = oracle.Hierarchy(Ao, n_coarse=200)
    X, its, rels, st = H.solve_many(dev(B), tol=1e-10)
    assert st == gw.GW_OK
    X = X.cpu().numpy()
    for c in range(k):
        h, it, _, _ = H.solve(dev(B[c]), tol=1e-10)
        assert it == its[c]
        np.testing.assert_array_equal(h.cpu().numpy(), X[c])
        ref, it_ref, _, _ = Ho.pcg(B[c], tol=1e-10)
        assert abs(its[c] - it_ref) <= 1
        assert np.linalg.norm(X[c] - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [2, 4, 5, 8, 11])
@pytest.mark.parametrize("smoother", [1, 0])
def test_interleaved_block_solve_matches_oracle(gw, k, smoother):
    """The mixed form solves k >= 2 columns in interleaved blocks of 4 or 8
    (k = 11: a block of 8 and one of 3 padded to 4).  Every column meets the
    FP64 residual test, agrees with the oracle's solve of the same system and
    needs within two iterations of the single-vector solver; a zero column
    stops at once with a zero solution."""
    side = 24
    p = wl.heterogeneous_3d(side=side, var=3.0, corr=4.0, seed=5)
    K = dev(p["Kx"])
    A, b = gw.gw_assemble(side, side, side, K, K, K, p["bct"], p["bcv"], None)
    H = gw.Hierarchy(A, n_coarse=200, smoother=smoother)
    rng = np.random.default_rng(10 + k)
    B = rng.normal(size=(k, side ** 3))
    B[0] = b
    if k > 2:
        B[2] = 0.0
        B[1] *= 1e-6
    Ao, _ = oracle.assemble(side, side, side, p["Kx"])
    Ho = oracle.Hierarchy(Ao, n_coarse=200, smoother=smoother)
    for src in (dev(B), B):
        X, its, rels, st = H.solve_many(src, tol=1e-9)
        X = X.cpu().numpy() if hasattr(X, "cpu") else X
        assert st == gw.GW_OK, (its, rels)
        for c in range(k):
            if not B[c].any():
                assert its[c] == 0 and rels[c] == 0.0 and not X[c].any()
                continue
            assert rels[c] <= 1e-9
            r = B[c] - Ao.matvec(X[c])
            assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(B[c]) * (1 + 1e-6)
            ref, _, _, _ = Ho.pcg(B[c], tol=1e-12)
            assert np.linalg.norm(X[c] - ref) <= 1e-7 * np.linalg.norm(ref)
            _, it1, _, _ = H.solve(dev(B[c]), tol=1e-9)
            assert abs(its[c] - it1) <= 2, (c, its[c], it1)


def test_interleaved_graphs_follow_a_refreshed_level0(gw):
    """gw_hierarchy_shift refreshes level 0 in place: the interleaved graphs are recaptured."""
    side = 16
    p = wl.heterogeneous_3d(side=side, var=2.0, corr=4.0, seed=3)
    A, b = gw.gw_assemble(side, side, side, p["Kx"])
    H = gw.Hierarchy(A, n_coarse=100)
    B = np.stack([b, 0.5 * b, b[::-1].copy()])
    H.solve_many(dev(B), tol=1e-9)
    C, _ = oracle.assemble(side, side, side, p["Kx"])
    s = 0.004 * np.diag(C.dense())
    assert H.shift(dev(s), delta=0.01) == 2  # aggregates kept, coarse operators formed again
    X, its, rels, st = H.solve_many(dev(B), tol=1e-9)
    As = oracle.shift(C, s)
    for c in range(3):
        ref = np.linalg.solve(As.dense(), B[c])
        assert np.linalg.norm(X[c].cpu().numpy() - ref) <= 1e-7 * np.linalg.norm(ref)


def test_solve_many_reports_non_convergence(gw):
    side = 16
    p = wl.heterogeneous_3d(side=side, var=3.0, corr=4.0, seed=2)
    A, b = gw.gw_assemble(side, side, side, p["Kx"])
    H = gw.Hierarchy(A, n_coarse=100)
    B = np.stack([b, 2 * b])
    X, its, rels, st = H.solve_many(B, tol=1e-14, maxit=2)
    assert st == gw.GW_ERR_NOT_CONVERGED and its == [2, 2]


@pytest.mark.parametrize("degree,nu", [(3, 1), (2, 2)])
def test_interleaved_block_other_cycles(gw, degree, nu):
    """Interleaved blocks with Chebyshev(3) and with V(2,2): every column meets the
    FP64 residual test and agrees with the oracle's solve."""
    side = 20
    p = wl.heterogeneous_3d(side=side, var=3.0, corr=4.0, seed=6)
    A, b = gw.gw_assemble(side, side, side, p["Kx"])
    H = gw.Hierarchy(A, n_coarse=200, degree=degree, nu=nu)
    B = np.random.default_rng(3).normal(size=(3, side ** 3))
    X, its, rels, st = H.solve_many(dev(B), tol=1e-9)
    assert st == gw.GW_OK and max(rels) <= 1e-9
    Ao, _ = oracle.assemble(side, side, side, p["Kx"])
    Ho = oracle.Hierarchy(Ao, n_coarse=200, degree=degree, nu=nu)
    X = X.cpu().numpy()
    for c in range(3):
        ref, _, _, _ = Ho.pcg(B[c], tol=1e-12)
        assert np.linalg.norm(X[c] - ref) <= 1e-7 * np.linalg.norm(ref)
