"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here runs on a GPU.  Each test checks the oracle against something
other than itself: the paper's Table 1, closed-form heads, series
resistances, published hash outputs, dense linear algebra from numpy,
characterisations of the MIS-2 and aggregation definitions, and Chebyshev
polynomials evaluated in closed form.
"""
import os
from collections import deque

import numpy as np
import pytest

import oracle
from paper_2001_05798_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def asm(p):
    return oracle.assemble(p["nx"], p["ny"], p["nz"], p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"])


def read_table1():
    levels, summary = [], {}
    with open(os.path.join(GOLDEN, "table1_amgcl.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].isdigit():
                levels.append((int(parts[1]), int(parts[2]), float(parts[3])))
            else:
                summary[parts[0]] = float(parts[1])
    return levels, summary


# ---------------------------------------------------------------- constants --
def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014) starts 0xe220a8397b1dcdaf,
    # 0x6e789e6aa1b965f4; key(s, 0, 0) = mix(s + gamma) is that sequence's step.
    assert oracle.key(0, 0, 0) == 0xE220A8397B1DCDAF
    assert oracle.key(0x9E3779B97F4A7C15, 0, 0) == 0x6E789E6AA1B965F4


def test_table1_level0_size_pins_the_stencil():
    levels, summary = read_table1()
    n0, nnz0, _ = levels[0]
    # 550 x 500 x 10 is the only grid with 10 layers and 2.75M cells whose
    # 7-point operator has the printed number of nonzeros
    assert 550 * 500 * 10 == n0
    assert oracle.nnz7(550, 500, 10) == nnz0
    assert oracle.nnz7(550, 500, 1) == 5 * 275000 - 2 * (550 + 500)
    K = np.ones(n0)
    A, _ = oracle.assemble(550, 500, 10, K)
    assert A.nnz == nnz0 and A.nr == n0
    assert summary["levels"] == len(levels)
    # CG memory: four FP64 vectors of n0 in MiB
    assert round(4 * 8 * n0 / 2 ** 20, 2) == summary["cg_memory_MiB"]


def test_table1_complexity_definitions():
    levels, summary = read_table1()
    st = oracle.complexities([l[0] for l in levels], [l[1] for l in levels])
    assert round(st["op_complexity"], 2) == summary["operator_complexity"]
    assert round(st["grid_complexity"], 2) == summary["grid_complexity"]
    assert [round(p, 2) for p in st["nnz_percent"]] == [l[2] for l in levels]


# ----------------------------------------------------------------- assembly --
@pytest.mark.parametrize("dims", [(16, 12, 1), (8, 6, 5), (5, 1, 1)])
def test_homogeneous_head_is_linear(dims):
    nx, ny, nz = dims
    p = wl.problem(nx, ny, nz)
    A, b = asm(p)
    h = np.linalg.solve(A.dense(), b)
    x = np.tile(np.arange(nx), ny * nz)
    np.testing.assert_allclose(h, 1.0 - (x + 0.5) / nx, rtol=0, atol=1e-13)


def test_series_heterogeneity_pins_harmonic_mean():
    # K varies along x only; the flux through the column is (h_L - h_R) / sum of
    # series resistances, each face resistance 1/(2K_i) + 1/(2K_j), the two
    # boundary faces 1/(2K) (half-cell distance to the Dirichlet face).
    nx, ny, nz = 9, 3, 2
    rng = np.random.default_rng(11)
    kx = np.exp(rng.normal(0, 2, nx))
    K = np.tile(kx, ny * nz)
    A, b = oracle.assemble(nx, ny, nz, K, bct=(1, 1, 0, 0, 0, 0), bcv=(2.0, -1.0, 0, 0, 0, 0))
    h = np.linalg.solve(A.dense(), b)
    res = [1 / (2 * kx[0])] + [1 / (2 * kx[i]) + 1 / (2 * kx[i + 1]) for i in range(nx - 1)] + [1 / (2 * kx[-1])]
    Q = (2.0 - (-1.0)) / sum(res)
    href = np.empty(nx)
    href[0] = 2.0 - Q * res[0]
    for i in range(1, nx):
        href[i] = href[i - 1] - Q * res[i]
    np.testing.assert_allclose(h, np.tile(href, ny * nz), rtol=0, atol=1e-12)


def test_layered_in_z_flow_in_x_is_linear_per_layer():
    nx, ny, nz = 7, 4, 6
    kz_layers = np.exp(np.linspace(-3, 3, nz))
    K = np.repeat(kz_layers, nx * ny)
    A, b = oracle.assemble(nx, ny, nz, K, Kz=K / 10.0)
    h = np.linalg.solve(A.dense(), b)
    x = np.tile(np.arange(nx), ny * nz)
    np.testing.assert_allclose(h, 1.0 - (x + 0.5) / nx, rtol=0, atol=1e-12)


def test_anisotropic_spacing_uses_face_area_over_distance():
    # flow in x on cells dx*dy*dz: the head stays linear whatever the spacing,
    # and the flux per unit head drop is K*ny*dy*nz*dz/(nx*dx)
    nx, ny, nz = 6, 3, 2
    A, b = oracle.assemble(nx, ny, nz, np.full(nx * ny * nz, 3.0), spacing=(2.0, 0.5, 4.0))
    h = np.linalg.solve(A.dense(), b)
    x = np.tile(np.arange(nx), ny * nz)
    np.testing.assert_allclose(h, 1.0 - (x + 0.5) / nx, atol=1e-13)
    left = np.arange(0, nx * ny * nz, nx)
    flux = np.sum(A.dense()[left].sum(axis=1) * (1.0 - h[left]))
    np.testing.assert_allclose(flux, 3.0 * (ny * 0.5) * (nz * 4.0) / (nx * 2.0), rtol=1e-13)


def test_m_matrix_invariants():
    p = wl.problem(10, 9, 8, var=4.0, corr=3.0, seed=5, bct=(1, 1, 0, 1, 0, 0), bcv=(1.0, 0.0, 0, 0.25, 0, 0),
                   wells_count=3, wells_seed=9)
    A, b = asm(p)
    D = A.dense()
    assert np.array_equal(D, D.T), "not bitwise symmetric"
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0.0)
    assert np.all(np.diag(D) > 0.0)
    rp, ci, v = A.arrays()
    assert np.all(np.diff(rp) >= 1)
    for i in range(A.nr):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
    nx, ny, nz = 10, 9, 8
    x = np.tile(np.arange(nx), ny * nz)
    y = np.tile(np.repeat(np.arange(ny), nx), nz)
    rs = D.sum(axis=1)
    q = p["q"]
    on_left, on_right, on_top_y = x == 0, x == nx - 1, y == ny - 1
    interior = ~(on_left | on_right | on_top_y)
    assert np.all(np.abs(rs[interior]) <= 1e-14 * np.diag(D)[interior])
    assert np.all(rs[~interior] > 0)
    # b - q only on Dirichlet faces: h = 1 on -x, 0 on +x, 0.25 on +y
    only_left = on_left & ~on_top_y
    dg = np.diag(D)
    assert np.all(np.abs(rs[only_left] - (b - q)[only_left]) <= 1e-14 * dg[only_left])
    assert np.all((b - q)[on_right & ~on_top_y] == 0)
    assert np.all(b[interior] == q[interior])
    assert A.nnz == oracle.nnz7(nx, ny, nz)


def test_pumping_wells_draw_the_head_down():
    p = wl.layered_wells_3d(nx=12, ny=10, nz=6, corr=(4.0, 4.0, 2.0), wells_count=2, wells_seed=4)
    A, b = asm(p)
    h = np.linalg.solve(A.dense(), b)
    assert np.all(h < 0.0)
    assert np.argmin(h) in set(p["wells"].tolist())


@pytest.mark.parametrize("bad", ["kzero", "knan", "noflow", "qnan"])
def test_assembly_rejects_bad_input(bad):
    n = 4 * 3 * 2
    K = np.ones(n)
    bct, q = (1, 1, 0, 0, 0, 0), None
    if bad == "kzero":
        K[5] = 0.0
    elif bad == "knan":
        K[5] = np.nan
    elif bad == "noflow":
        bct = (0,) * 6
    else:
        q = np.zeros(n)
        q[3] = np.inf
    with pytest.raises(ValueError):
        oracle.assemble(4, 3, 2, K, bct=bct, q=q)


# ----------------------------------------------------------------- dense LU --
def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 40):
        M = rng.normal(size=(n, n)) + n * np.eye(n)
        if n > 1:
            M[0, 0] = 0.0  # forces a row exchange
        lu, piv = oracle.lu_factor(M)
        bvec = rng.normal(size=n)
        np.testing.assert_allclose(oracle.lu_solve(lu, piv, bvec), np.linalg.solve(M, bvec), rtol=1e-11, atol=1e-12)
    p = wl.problem(6, 5, 4, var=2.0, corr=2.0, seed=2)
    A, b = asm(p)
    lu, piv = oracle.lu_factor(A.dense())
    np.testing.assert_allclose(oracle.lu_solve(lu, piv, b), np.linalg.solve(A.dense(), b), rtol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_factor(np.zeros((3, 3)))


# ----------------------------------------------------------------- strength --
def test_strength_on_chain():
    A, _ = oracle.assemble(6, 1, 1, np.ones(6))
    # interior a_ii = 2, end cells a_ii = 3 (Dirichlet half-cell), a_ij = -1
    S = oracle.strength(A, 0.0064)
    rp, ci, v = A.arrays()
    offd = ci != np.repeat(np.arange(6), np.diff(rp))
    assert np.all(S[offd] == 1) and np.all(S[~offd] == 0)
    S = oracle.strength(A, 0.2)  # 1 > 0.8 between interior cells, 1 > 1.2 fails at the ends
    rows = np.repeat(np.arange(6), np.diff(rp))
    for e in range(A.nnz):
        i, j = rows[e], ci[e]
        want = i != j and i not in (0, 5) and j not in (0, 5)
        assert S[e] == want


def test_strength_is_symmetrised():
    rp = np.array([0, 2, 4])
    ci = np.array([0, 1, 0, 1])
    v = np.array([1.0, -1.0, -0.01, 1.0])
    A = oracle.CSR.from_arrays(rp, ci, v)
    S = oracle.strength(A, 0.0064)
    assert list(S) == [0, 1, 1, 0]


# --------------------------------------------------------- MIS-2, aggregates --
def strength_graph(A, S):
    rp, ci, _ = A.arrays()
    adj = [[] for _ in range(A.nr)]
    for i in range(A.nr):
        for e in range(rp[i], rp[i + 1]):
            if S[e] and ci[e] != i:
                adj[i].append(int(ci[e]))
    return adj


def within2(adj, r):
    out = {r}
    for j in adj[r]:
        out.add(j)
        out.update(adj[j])
    return out


def small_graphs():
    out = []
    p = wl.problem(9, 8, 1, var=4.0, corr=2.0, seed=3)
    out.append(asm(p)[0])
    p = wl.problem(6, 5, 4, var=3.0, corr=1.5, seed=4)
    out.append(asm(p)[0])
    rng = np.random.default_rng(7)
    n = 60
    M = (rng.random((n, n)) < 0.06).astype(float)
    M = np.triu(M, 1)
    M = -(M + M.T)
    M += np.diag(-M.sum(axis=1) + 1.0)
    rows, cols = np.nonzero(M)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    out.append(oracle.CSR.from_arrays(np.cumsum(rp), cols, M[rows, cols]))
    return out


@pytest.mark.parametrize("gi", [0, 1, 2])
@pytest.mark.parametrize("seed,level", [(0x5EED, 0), (17, 2)])
def test_mis2_is_the_lexicographically_first_distance2_mis(gi, seed, level):
    A = small_graphs()[gi]
    S = oracle.strength(A, 0.0064)
    adj = strength_graph(A, S)
    root = oracle.mis2(A, S, seed, level)
    pri = {i: (oracle.key(seed, level, i), i) for i in range(A.nr)}
    roots = [i for i in range(A.nr) if root[i]]
    for r in roots:  # independence in S^2
        assert not (within2(adj, r) - {r}) & set(roots)
    for v in range(A.nr):  # every non-root is blocked by a higher-priority root
        if root[v]:
            continue
        assert any(root[u] and pri[u] > pri[v] for u in within2(adj, v))


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_aggregation_rules(gi):
    A = small_graphs()[gi]
    seed, level = 0x5EED, 1
    S = oracle.strength(A, 0.0064)
    adj = strength_graph(A, S)
    root = oracle.mis2(A, S, seed, level)
    agg, m = oracle.aggregate(A, S, root, seed, level)
    roots = [i for i in range(A.nr) if root[i]]
    assert m == len(roots)
    assert [agg[r] for r in roots] == list(range(m))  # ascending numbering
    assert set(agg.tolist()) == set(range(m))
    for r in roots:
        for j in adj[r]:
            assert agg[j] == agg[r]
    step2 = {r: r for r in roots}
    for r in roots:
        for j in adj[r]:
            step2[j] = r
    for v in range(A.nr):
        if v in step2:
            continue
        cands = {step2[j] for j in adj[v] if j in step2}
        assert cands, "node not within distance 2 of a root"
        best = max(cands, key=lambda r: (oracle.key(seed, level, r), r))
        assert agg[v] == agg[best]
    for c in range(m):  # each aggregate connected in S
        members = set(np.nonzero(agg == c)[0].tolist())
        start = next(iter(members))
        seen, dq = {start}, deque([start])
        while dq:
            u = dq.popleft()
            for w in adj[u]:
                if w in members and w not in seen:
                    seen.add(w)
                    dq.append(w)
        assert seen == members


# ----------------------------------------------------------- smoothed P, RAP --
def filtered_dense(A, S):
    D = A.dense()
    rp, ci, v = A.arrays()
    rows = np.repeat(np.arange(A.nr), np.diff(rp))
    F = np.zeros_like(D)
    keep = (S == 1) | (rows == ci)
    F[rows[keep], ci[keep]] = v[keep]
    F[np.arange(A.nr), np.arange(A.nr)] = D.sum(axis=1) - F.sum(axis=1) + np.diag(F)
    return F


def test_smoothed_prolongator_against_dense_definition():
    p = wl.problem(10, 9, 8, var=4.0, corr=3.0, seed=8)
    A, _ = asm(p)
    S = oracle.strength(A, 0.0064)
    root = oracle.mis2(A, S, 0x5EED, 0)
    agg, m = oracle.aggregate(A, S, root, 0x5EED, 0)
    P, omega, rho = oracle.smooth_p(A, S, agg, m)
    F = filtered_dense(A, S)
    hs = (np.abs(F - np.diag(np.diag(F))) > 0).any(axis=1)
    rho_ref = max((np.abs(F[i]).sum() / F[i, i]) for i in range(A.nr) if hs[i])
    np.testing.assert_allclose(rho, rho_ref, rtol=1e-14)
    np.testing.assert_allclose(omega * rho, 4.0 / 3.0, rtol=1e-15)
    T = np.zeros((A.nr, m))
    T[np.arange(A.nr), agg] = 1.0
    Pref = T - omega * (F / np.diag(F)[:, None]) @ T
    Pref[~hs] = T[~hs]
    np.testing.assert_allclose(P.dense(), Pref, rtol=0, atol=1e-14)
    # row sums are 1 where the filtered row sums to zero (no Dirichlet face)
    zero_rows = np.abs(F.sum(axis=1)) <= 1e-14 * np.diag(F)
    np.testing.assert_allclose(P.dense().sum(axis=1)[zero_rows], 1.0, atol=1e-13)
    # pattern: aggregates of {i} U S(i), nothing dropped
    rp, ci, _ = P.arrays()
    patt = (np.abs(F) > 0).astype(int) @ T > 0
    patt[~hs] = T[~hs] > 0
    got = np.zeros_like(patt)
    got[np.repeat(np.arange(A.nr), np.diff(rp)), ci] = True
    assert np.array_equal(got, patt)


def test_transpose_and_spgemm_against_dense():
    rng = np.random.default_rng(5)

    def rand_csr(nr, nc, dens):
        M = (rng.random((nr, nc)) < dens) * rng.normal(size=(nr, nc))
        rows, cols = np.nonzero(M)
        rp = np.zeros(nr + 1, np.int64)
        np.add.at(rp, rows + 1, 1)
        return oracle.CSR.from_arrays(np.cumsum(rp), cols, M[rows, cols], nc=nc), M

    Lm, Ld = rand_csr(30, 20, 0.2)
    Rm, Rd = rand_csr(20, 25, 0.2)
    C = oracle.spgemm(Lm, Rm)
    np.testing.assert_allclose(C.dense(), Ld @ Rd, rtol=1e-14, atol=1e-14)
    T = oracle.transpose(Lm)
    assert np.array_equal(T.dense(), Ld.T)
    rp, ci, _ = T.arrays()
    for i in range(T.nr):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def test_galerkin_coarse_operators_against_dense():
    p = wl.problem(14, 13, 12, var=4.0, corr=4.0, seed=6)
    A, _ = asm(p)
    H = oracle.Hierarchy(A, n_coarse=50)
    assert H.status == 0 and H.nlevels >= 3
    for l in range(H.nlevels - 1):
        Al, Pl = H.A(l).dense(), H.P(l).dense()
        ref = Pl.T @ Al @ Pl
        Ac = H.A(l + 1).dense()
        scale = np.abs(ref).max()
        assert np.abs(Ac - ref).max() <= 1e-13 * scale
        assert np.abs(Ac - Ac.T).max() <= 1e-14 * scale
        np.linalg.cholesky(Ac)
        assert np.array_equal(H.R(l).dense(), Pl.T)
        assert H.A(l + 1).nr == H.nagg(l)


# ---------------------------------------------------------------- smoothers --
def chain_laplacian(n):
    """tridiag(-1, 2, -1): D^-1 A has eigenpairs 1 - cos(k pi/(n+1)), sin(i k pi/(n+1))."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(v)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, np.array(rows) + 1, 1)
    return oracle.CSR.from_arrays(np.cumsum(rp), np.array(cols), np.array(vals))


def cheb_T(m, t):
    return np.cosh(m * np.arccosh(t)) if abs(t) >= 1 else np.cos(m * np.arccos(t))


@pytest.mark.parametrize("k", [1, 20, 50, 63])
def test_jacobi_and_chebyshev_error_polynomials(k):
    n = 64
    A = chain_laplacian(n)
    lam_k = 1.0 - np.cos(k * np.pi / (n + 1))
    v = np.sin(np.arange(1, n + 1) * k * np.pi / (n + 1))
    Hj = oracle.Hierarchy(A, smoother=0, nu=1, n_coarse=16)
    assert Hj.scalars(0)["jacobi_w"] == (4.0 / 3.0) / 2.0
    xj = Hj.smooth(0, np.zeros(n), v)
    np.testing.assert_allclose(xj, (1 - (2.0 / 3.0) * lam_k) * v, atol=1e-13)
    for m in (2, 3):
        Hc = oracle.Hierarchy(A, smoother=1, degree=m, nu=1, n_coarse=16)
        lam = Hc.scalars(0)["lam"]
        assert 1.0 < lam <= 2.0
        a, b = lam / 30.0, 1.1 * lam
        th, de = (a + b) / 2, (b - a) / 2
        pk = cheb_T(m, (th - lam_k) / de) / cheb_T(m, th / de)
        xc = Hc.smooth(0, np.zeros(n), v)
        np.testing.assert_allclose(xc, pk * v, atol=1e-12)


# ------------------------------------------------------------ V-cycle, PCG --
@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycle_is_symmetric_positive_and_contracts(smoother):
    p = wl.problem(16, 16, 16, var=4.0, corr=4.0, seed=3)
    A, b = asm(p)
    H = oracle.Hierarchy(A, smoother=smoother, n_coarse=64)
    assert H.status == 0 and H.nlevels >= 3
    rng = np.random.default_rng(1)
    u, w = rng.normal(size=A.nr), rng.normal(size=A.nr)
    Mu, Mw = H.vcycle(u), H.vcycle(w)
    assert abs(Mu @ w - u @ Mw) <= 1e-12 * abs(Mu @ w)
    assert Mu @ u > 0
    # stationary iteration x <- x + M(b - A x): error contracts
    href = np.linalg.solve(A.dense(), b)
    x = np.zeros(A.nr)
    errs = []
    for _ in range(6):
        x = x + H.vcycle(b - A.matvec(x))
        errs.append(np.linalg.norm(x - href))
    factor = (errs[-1] / errs[1]) ** (1 / 4)
    assert factor < 0.8


@pytest.mark.parametrize("smoother,nu", [(0, 1), (0, 2), (1, 1)])
def test_pcg_matches_dense_solution(smoother, nu):
    p = wl.problem(8, 8, 8, var=4.0, corr=2.0, seed=4, bct=(1, 1, 0, 0, 1, 0), bcv=(1.0, 0.0, 0, 0, 0.5, 0),
                   wells_count=3, wells_seed=2)
    A, b = asm(p)
    H = oracle.Hierarchy(A, smoother=smoother, nu=nu, n_coarse=40)
    x, it, rel, st = H.pcg(b, tol=1e-12)
    assert st == 0 and rel <= 1e-12
    ref = np.linalg.solve(A.dense(), b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(b - A.matvec(x)) / np.linalg.norm(b) == pytest.approx(rel, rel=1e-6)


def test_pcg_config0_closed_form():
    p = wl.homogeneous_2d_128()
    A, b = asm(p)
    H = oracle.Hierarchy(A)
    x, it, rel, st = H.pcg(b, tol=1e-8)
    assert st == 0 and rel <= 1e-8
    xx = np.tile(np.arange(128), 128)
    href = 1.0 - (xx + 0.5) / 128
    assert np.linalg.norm(x - href) / np.linalg.norm(href) <= 1e-6
    x, it12, rel, st = H.pcg(b, tol=1e-12)
    assert st == 0 and np.abs(x - href).max() <= 1e-10


def test_pcg_flux_balance_and_speedup_over_cg():
    p = wl.heterogeneous_3d(side=24, var=4.0, corr=4.0, seed=1)
    A, b = asm(p)
    H = oracle.Hierarchy(A)
    x, it, rel, st = H.pcg(b, tol=1e-12)
    assert st == 0
    r = b - A.matvec(x)
    rp, ci, v = A.arrays()
    diag = v[rp[:-1] + np.array([np.searchsorted(ci[rp[i]:rp[i + 1]], i) for i in range(A.nr)])]
    assert np.all(np.abs(r) <= 1e-10 * (diag * np.abs(x).max()))
    # AMG preconditioning cuts the CG iteration count by an order of magnitude
    _, it_cg, _, _ = oracle.cg_plain(A, b, tol=1e-8)
    _, it_amg, _, _ = H.pcg(b, tol=1e-8)
    assert it_amg * 8 < it_cg


def test_pcg_status_codes():
    p = wl.heterogeneous_3d(side=12, var=4.0, corr=3.0, seed=2)
    A, b = asm(p)
    H = oracle.Hierarchy(A, n_coarse=30)
    x, it, rel, st = H.pcg(b, tol=1e-14, maxit=2)
    assert st == oracle.ERR_NOT_CONVERGED and it == 2 and rel > 1e-14
    x, it, rel, st = H.pcg(np.zeros(A.nr))
    assert st == 0 and it == 0 and not x.any()


# ----------------------------------------------------------------- workload --
def test_lnk_field_statistics():
    f1, clipped = wl.lnk_field(64, 64, 64, 4.0, 4.0, 1)
    f2, _ = wl.lnk_field(64, 64, 64, 4.0, 4.0, 1)
    assert np.array_equal(f1, f2)
    assert clipped < 0.01
    assert abs(f1.mean()) < 0.3
    assert 3.0 < f1.var() < 5.0
    # covariance at a lag of one correlation length along x is about var / e
    c = np.mean((f1[:, :, :-4] - f1.mean()) * (f1[:, :, 4:] - f1.mean()))
    assert 0.8 < c / (4.0 / np.e) < 1.25


# ----------------------------------------------------------------- adjoint --
def _adjoint_case(nx, ny, nz, seed, kz_ratio=1.0, bct=(1, 1, 0, 0, 0, 0), bcv=(1.0, 0.0, 0, 0, 0, 0)):
    p = wl.problem(nx, ny, nz, var=2.0, corr=2.0, seed=seed, kz_ratio=kz_ratio, bct=bct, bcv=bcv,
                   wells_count=2, wells_seed=seed + 1)
    lnk = np.log(p["Kx"])
    obs = wl.cells(nx * ny * nz, 6, seed + 2)
    hobs = np.random.default_rng(seed + 3).normal(0.5, 0.1, len(obs))
    return p, lnk, obs, hobs


def _J_of(lnk, p, obs, hobs, kz_ratio):
    K = np.exp(lnk)
    A, b = oracle.assemble(p["nx"], p["ny"], p["nz"], K, K, K / kz_ratio, p["bct"], p["bcv"], p["q"])
    h = np.linalg.solve(A.dense(), b)
    return oracle.misfit(h, obs, hobs)[0], h, A


@pytest.mark.parametrize("kz_ratio,bct,bcv", [(1.0, (1, 1, 0, 0, 0, 0), (1.0, 0.0, 0, 0, 0, 0)),
                                              (10.0, (0, 0, 0, 0, 0, 1), (0, 0, 0, 0, 0, 0.3))])
def test_adjoint_gradient_matches_central_differences(kz_ratio, bct, bcv):
    nx, ny, nz = 7, 6, 5
    p, lnk, obs, hobs = _adjoint_case(nx, ny, nz, 3, kz_ratio, bct, bcv)
    J, h, A = _J_of(lnk, p, obs, hobs, kz_ratio)
    _, dJdh = oracle.misfit(h, obs, hobs)
    lam = np.linalg.solve(A.dense(), dJdh)
    K = np.exp(lnk)
    g = oracle.adjoint_grad(nx, ny, nz, K, h, lam, K, K / kz_ratio, p["bct"], p["bcv"])
    eps = 1e-5
    for i in np.random.default_rng(1).choice(nx * ny * nz, 25, replace=False):
        lp, lm = lnk.copy(), lnk.copy()
        lp[i] += eps
        lm[i] -= eps
        fd = (_J_of(lp, p, obs, hobs, kz_ratio)[0] - _J_of(lm, p, obs, hobs, kz_ratio)[0]) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9 * max(1.0, abs(J)))


def test_misfit_definition():
    h = np.array([1.0, 2.0, 3.0, 4.0])
    J, d = oracle.misfit(h, [1, 3], [1.5, 3.0])
    assert J == pytest.approx(0.25 + 1.0)
    assert list(d) == [0.0, 1.0, 0.0, 2.0]


# --------------------------------------------------------- transient shift --
def test_shift_and_reuse_criterion():
    p = wl.problem(6, 5, 4, var=2.0, corr=2.0, seed=3)
    C, b = asm(p)
    s = np.linspace(0.0, 0.3, C.nr)
    np.testing.assert_array_equal(oracle.shift(C, s).dense(), C.dense() + np.diag(s))
    d = np.diag(C.dense())
    assert oracle.reuse_ok(C, 0.009 * d, delta=0.01)
    assert not oracle.reuse_ok(C, 0.011 * d, delta=0.01)
    bad = 0.005 * d
    bad[7] = 0.02 * d[7]
    assert not oracle.reuse_ok(C, bad, delta=0.01)
    assert oracle.reuse_ok(C, bad, s_built=bad - 0.001 * d, delta=0.01)


@pytest.mark.parametrize("frac", [0.005, 0.5])
def test_transient_step_with_reused_hierarchy_solves_the_shifted_system(frac):
    # implicit step (C + S/dt) h1 = Q + (S/dt) h0 on a cached hierarchy of C
    p = wl.problem(12, 11, 10, var=3.0, corr=3.0, seed=8)
    C, b = asm(p)
    d = np.diag(C.dense())
    s = frac * d * np.random.default_rng(4).random(C.nr)
    h0 = np.random.default_rng(5).normal(size=C.nr)
    A = oracle.shift(C, s)
    rhs = b + s * h0
    H = oracle.Hierarchy(C, n_coarse=60)
    H.refresh_level0(A)
    x, it, rel, st = H.pcg(rhs, tol=1e-12)
    assert st == 0 and rel <= 1e-12
    ref = np.linalg.solve(A.dense(), rhs)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


# ------------------------------------------------------------ face fluxes --
def test_darcy_flux_uniform_for_linear_head():
    nx, ny, nz = 8, 5, 3
    K = 2.5
    A, b = oracle.assemble(nx, ny, nz, np.full(nx * ny * nz, K), spacing=(2.0, 1.0, 0.5))
    h = np.linalg.solve(A.dense(), b)
    vx, vy, vz = oracle.darcy_flux(nx, ny, nz, np.full(nx * ny * nz, K), h, spacing=(2.0, 1.0, 0.5))
    # Darcy: v = -K dh/dx with h falling from 1 to 0 over nx * dx
    np.testing.assert_allclose(vx, K / (nx * 2.0), rtol=1e-12)
    np.testing.assert_allclose(vy, 0.0, atol=1e-14)
    np.testing.assert_allclose(vz, 0.0, atol=1e-14)


def test_darcy_flux_balances_sources_per_cell():
    p = wl.problem(9, 7, 6, var=3.0, corr=2.0, seed=6, bct=(1, 0, 0, 1, 0, 1), bcv=(1.0, 0, 0, 0.2, 0, -0.4),
                   wells_count=3, wells_seed=4)
    nx, ny, nz = 9, 7, 6
    A, b = asm(p)
    h = np.linalg.solve(A.dense(), b)
    vx, vy, vz = oracle.darcy_flux(nx, ny, nz, p["Kx"], h, p["Ky"], p["Kz"], p["bct"], p["bcv"])
    vx = vx.reshape(nz, ny, nx + 1)
    vy = vy.reshape(nz, ny + 1, nx)
    vz = vz.reshape(nz + 1, ny, nx)
    out = (vx[:, :, 1:] - vx[:, :, :-1]) + (vy[:, 1:, :] - vy[:, :-1, :]) + (vz[1:] - vz[:-1])
    np.testing.assert_allclose(out.ravel(), p["q"], atol=1e-10)


def test_numeric_refresh_is_the_galerkin_product_on_kept_prolongators():
    # the refreshed coarse operators are P^T A P of the shifted level above,
    # with the prolongators of the original setup (dense products by numpy)
    p = wl.problem(12, 11, 10, var=3.0, corr=3.0, seed=8)
    C, b = asm(p)
    d = np.diag(C.dense())
    s = 0.02 * d * np.random.default_rng(6).random(C.nr)
    H = oracle.Hierarchy(C, n_coarse=60)
    L = H.nlevels
    assert L >= 3
    P = [H.P(l).dense() for l in range(L - 1)]
    old = [H.A(l).dense() for l in range(L)]
    pats = [tuple(a.copy() for a in H.A(l).arrays()[:2]) for l in range(L)]
    A = oracle.shift(C, s)
    H.refresh_numeric(A)
    assert H.nlevels == L
    new = [H.A(l).dense() for l in range(L)]
    np.testing.assert_array_equal(new[0], C.dense() + np.diag(s))
    for l in range(L - 1):
        np.testing.assert_array_equal(H.P(l).dense(), P[l])
        ref = P[l].T @ new[l] @ P[l]
        assert np.abs(new[l + 1] - ref).max() <= 1e-13 * np.abs(ref).max()
        rp, ci, _ = H.A(l + 1).arrays()
        assert np.array_equal(rp, pats[l + 1][0]) and np.array_equal(ci, pats[l + 1][1])
    # the change of level 1 is the Galerkin product of the storage diagonal
    assert np.abs((new[1] - old[1]) - P[0].T @ np.diag(s) @ P[0]).max() <= 1e-12 * np.abs(old[1]).max()
    # with no shift the refresh reproduces the original operators bit for bit
    H2 = oracle.Hierarchy(C, n_coarse=60)
    H2.refresh_numeric(C)
    for l in range(L):
        np.testing.assert_array_equal(H2.A(l).dense(), old[l])
    # and the refreshed hierarchy solves the shifted system
    rhs = b + s
    x, it, rel, st = H.pcg(rhs, tol=1e-12)
    assert st == 0 and rel <= 1e-12
    ref = np.linalg.solve(A.dense(), rhs)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def _smoother_propagator(H, l, smoother, degree, nu):
    """Error propagator of one smoothing application on level l from the
    smoothers' closed forms: (I - w D^-1 A)^nu for damped Jacobi with the
    Gershgorin weight, and p_m(D^-1 A)^nu for Chebyshev of degree m on
    [lam/30, 1.1 lam], p_m(t) = T_m((b + a - 2t)/(b - a)) / T_m((b + a)/(b - a)),
    evaluated by an eigendecomposition of D^-1/2 A D^-1/2."""
    A = H.A(l).dense()
    n = A.shape[0]
    d = np.diag(A)
    sc = H.scalars(l)
    if smoother == 0:
        E1 = np.eye(n) - sc["jacobi_w"] * (A / d[:, None])
    else:
        lam = sc["lam"]
        a, b = lam / 30.0, 1.1 * lam
        s = 1.0 / np.sqrt(d)
        w, V = np.linalg.eigh(s[:, None] * A * s[None, :])
        Tm = [0.0] * degree + [1.0]  # T_m in the Chebyshev basis (numpy's chebval)
        p = np.polynomial.chebyshev.chebval((b + a - 2 * w) / (b - a), Tm)
        p = p / np.polynomial.chebyshev.chebval((b + a) / (b - a), Tm)
        E1 = (s[:, None] * (V * p) @ V.T) / s[None, :]  # D^-1/2 f(S) D^1/2
    return np.linalg.matrix_power(E1, nu)


def _vcycle_matrix(H, l, smoother, degree, nu):
    """The V-cycle from level l down as a matrix B_l: on the coarsest level the
    exact inverse, above it I - B_l A_l = E (I - P_l B_{l+1} P_l^T A_l) E."""
    A = H.A(l).dense()
    if l == H.nlevels - 1:
        return np.linalg.inv(A)
    P = H.P(l).dense()
    Bc = _vcycle_matrix(H, l + 1, smoother, degree, nu)
    E = _smoother_propagator(H, l, smoother, degree, nu)
    n = A.shape[0]
    Mid = np.eye(n) - P @ Bc @ P.T @ A
    return (np.eye(n) - E @ Mid @ E) @ np.linalg.inv(A)


@pytest.mark.parametrize("smoother,degree,nu", [(0, 1, 1), (0, 1, 2), (1, 2, 1), (1, 3, 2)])
def test_vcycle_is_the_multigrid_error_propagator(smoother, degree, nu):
    # the oracle's V-cycle, applied to unit vectors, equals the dense product
    # of smoother, coarse-correction and smoother error propagators on every level
    p = wl.problem(9, 8, 7, var=3.0, corr=3.0, seed=6, wells_count=2, wells_seed=1)
    A, b = asm(p)
    H = oracle.Hierarchy(A, smoother=smoother, degree=degree, nu=nu, n_coarse=20)
    assert H.status == 0 and H.nlevels >= 3
    n = A.nr
    Bo = np.column_stack([H.vcycle(e) for e in np.eye(n)])
    Bref = _vcycle_matrix(H, 0, smoother, degree, nu)
    assert np.abs(Bo - Bref).max() <= 1e-10 * np.abs(Bref).max()
