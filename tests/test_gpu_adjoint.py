"""Adjoint sensitivity d(head misfit)/d(ln K) on the GPU against the oracle and
against central finite differences.

The objective is J = sum_k (h[o_k] - hobs_k)^2 over observation cells; the
gradient comes from one extra AMG-PCG solve C lambda = dJ/dh on the forward
hierarchy and the face-flux product kernel (gw_adjoint_gradient).
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


def dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype))).cuda()


@pytest.mark.parametrize("bct,bcv,kz", [((1, 1, 0, 0, 0, 0), (1.0, 0.0, 0, 0, 0, 0), 1.0),
                                        ((0, 0, 0, 1, 0, 1), (0, 0, 0, 0.4, 0, -0.2), 10.0)])
def test_gradient_kernel_matches_oracle(gw, bct, bcv, kz):
    nx, ny, nz = 21, 17, 9
    p = wl.problem(nx, ny, nz, var=3.0, corr=3.0, seed=4, kz_ratio=kz, bct=bct, bcv=bcv)
    rng = np.random.default_rng(2)
    h, lam = rng.normal(size=nx * ny * nz), rng.normal(size=nx * ny * nz)
    ref = oracle.adjoint_grad(nx, ny, nz, p["Kx"], h, lam, p["Ky"], p["Kz"], bct, bcv, spacing=(2.0, 1.0, 0.5))
    g = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    gw.gw_adjoint_gradient(nx, ny, nz, dev(p["Kx"]), dev(h), dev(lam), g, Ky=dev(p["Ky"]), Kz=dev(p["Kz"]), bct=bct,
                           bcv=bcv, spacing=(2.0, 1.0, 0.5))
    np.testing.assert_allclose(g.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_misfit_kernel_matches_oracle(gw):
    rng = np.random.default_rng(5)
    h = rng.normal(size=1000)
    obs = np.array([3, 17, 17, 999, 0], np.int32)
    hobs = rng.normal(size=5)
    J_ref, d_ref = oracle.misfit(h, obs, hobs)
    d = torch.empty(1000, dtype=torch.float64, device="cuda")
    J = gw.gw_misfit(dev(h), dev(obs), dev(hobs), d)
    assert J == pytest.approx(J_ref, rel=1e-14)
    np.testing.assert_array_equal(d.cpu().numpy(), d_ref)


def adjoint_problem(side, var, corr, seed, truth_seed, nobs, obs_seed):
    p = wl.heterogeneous_3d(side=side, var=var, corr=corr, seed=seed)
    truth = wl.heterogeneous_3d(side=side, var=var, corr=corr, seed=truth_seed)
    obs = wl.cells(side ** 3, nobs, obs_seed).astype(np.int32)
    return p, truth, obs


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_gradient_small_against_oracle(gw, prec):
    from paper_2001_05798_gb300.adjoint import heads

    side = 14
    p, truth, obs = adjoint_problem(side, 2.0, 3.0, 5, 6, 12, 7)
    At, bt = oracle.assemble(side, side, side, truth["Kx"])
    hobs = np.linalg.solve(At.dense(), bt)[obs]
    lnK = dev(np.log(p["Kx"])).requires_grad_(True)
    h = heads(lnK, side, side, side, tol=1e-12, prec=prec, n_coarse=100)
    J = ((h[dev(obs, np.int64)] - dev(hobs)) ** 2).sum()
    J.backward()
    A, b = oracle.assemble(side, side, side, p["Kx"])
    href = np.linalg.solve(A.dense(), b)
    Jref, dJdh = oracle.misfit(href, obs, hobs)
    lam = np.linalg.solve(A.dense(), dJdh)
    gref = oracle.adjoint_grad(side, side, side, p["Kx"], href, lam)
    assert float(J.detach()) == pytest.approx(Jref, rel=1e-8)
    g = lnK.grad.cpu().numpy()
    assert np.linalg.norm(g - gref) <= 1e-7 * np.linalg.norm(gref)


def test_adjoint_96_cubed_against_finite_differences_and_oracle(gw):
    """96^3 cells, lnK variance 2, correlation length 6 cells; 64 observation
    cells observe the heads of a second field; central differences
    (eps = 1e-4 in ln K, solves to 1e-12) on 20 cells and the oracle's adjoint."""
    from paper_2001_05798_gb300.adjoint import heads

    side = 96
    p, truth, obs = adjoint_problem(side, 2.0, 6.0, 5, 6, 64, 7)
    tK = dev(truth["Kx"])
    bt = torch.empty(side ** 3, dtype=torch.float64, device="cuda")
    At, _ = gw.gw_assemble(side, side, side, tK, tK, tK, truth["bct"], truth["bcv"], None, b_out=bt)
    ht, _, _, st = gw.Hierarchy(At).solve(bt, tol=1e-12)
    assert st == gw.GW_OK
    obs_t = dev(obs)
    hobs = ht[obs_t.long()].contiguous()
    lnK0 = dev(np.log(p["Kx"]))

    def J_of(lnK):
        h = heads(lnK, side, side, side, tol=1e-12)
        return gw.gw_misfit(h, obs_t, hobs)

    lnK = lnK0.clone().requires_grad_(True)
    h = heads(lnK, side, side, side, tol=1e-12)
    J = ((h[obs_t.long()] - hobs) ** 2).sum()
    J.backward()
    g = lnK.grad.cpu().numpy()

    def J64(lnK):  # FP64 form solved to 1e-13: the misfit to about 1e-12
        return gw.gw_misfit(heads(lnK, side, side, side, tol=1e-13, prec=gw.GW_PREC_FP64), obs_t, hobs)

    def fd(i, eps):
        lp, lm = lnK0.clone(), lnK0.clone()
        lp[i] += eps
        lm[i] -= eps
        return (J64(lp) - J64(lm)) / (2 * eps)

    # the 20 seeded cells, the cells of largest sensitivity and the most
    # sensitive cells on the Dirichlet faces (x = 0, x = side - 1), where the
    # boundary transmissibility term enters; Richardson-extrapolated central
    # differences (truncation O(eps^4)) with eps = 2e-3 and 1e-3
    gmax = np.abs(g).max()
    xs = np.arange(side ** 3) % side
    face = np.flatnonzero((xs == 0) | (xs == side - 1))
    cells = list(wl.cells(side ** 3, 20, 8)) + list(np.argsort(-np.abs(g))[:6])
    cells += list(face[np.argsort(-np.abs(g[face]))[:4]])
    for i in cells:
        i = int(i)
        rich = (4.0 * fd(i, 1e-3) - fd(i, 2e-3)) / 3.0
        assert abs(rich - g[i]) <= 1e-5 * abs(g[i]) + 1e-6 * gmax, (i, rich, g[i])
    # the oracle's adjoint on the oracle's own solves
    A, b = oracle.assemble(side, side, side, p["Kx"])
    Ho = oracle.Hierarchy(A)
    href, _, _, _ = Ho.pcg(b, tol=1e-12)
    _, dJdh = oracle.misfit(href, obs, hobs.cpu().numpy())
    lam, _, _, _ = Ho.pcg(dJdh, tol=1e-12)
    gref = oracle.adjoint_grad(side, side, side, p["Kx"], href, lam)
    assert np.linalg.norm(g - gref) <= 1e-6 * np.linalg.norm(gref)
