"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Assembly and the whole setup (aggregates, MIS-2 roots, P and A_l patterns
and values on every level) must be bit-exact: both sides follow the same
summation order with no fused multiply-add.  Solutions must satisfy
||h_gpu - h_ref|| / ||h_ref|| <= 1e-6 and a true relative residual <= 1e-8,
h_ref being the oracle's solve to 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05798_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_ERR = 1e-6
TOL = 1e-8


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


def gpu_assemble(gw, p, spacing=(1.0, 1.0, 1.0)):
    n = p["nx"] * p["ny"] * p["nz"]
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(p["nx"], p["ny"], p["nz"], dev(p["Kx"]), dev(p["Ky"]), dev(p["Kz"]), p["bct"], p["bcv"],
                          dev(p["q"]), b_out=b, spacing=spacing)
    torch.cuda.synchronize()
    return A, b


def ora_assemble(p, spacing=(1.0, 1.0, 1.0)):
    return oracle.assemble(p["nx"], p["ny"], p["nz"], p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"],
                           spacing=spacing)


PROBLEMS = {
    "2d_homog_128": lambda: wl.homogeneous_2d_128(),
    "3d_het_20": lambda: wl.problem(20, 17, 13, var=4.0, corr=3.0, seed=5, wells_count=3, wells_seed=1,
                                    bct=(1, 1, 0, 1, 0, 0), bcv=(1.0, 0.0, 0, 0.3, 0, 0)),
    "3d_layered_24": lambda: wl.layered_wells_3d(nx=24, ny=22, nz=12, corr=(6.0, 6.0, 2.0), wells_count=4),
    "3d_het_33_sigma4": lambda: wl.heterogeneous_3d(side=33, var=4.0, corr=8.0, seed=1),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_assembly_bit_exact(gw, name):
    p = PROBLEMS[name]()
    for spacing in ((1.0, 1.0, 1.0), (2.0, 0.5, 3.0)):
        A, b = gpu_assemble(gw, p, spacing)
        Ao, bo = ora_assemble(p, spacing)
        rp, ci, v = A.export()
        orp, oci, ov = Ao.arrays()
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
        assert np.array_equal(v.view(np.uint64), ov.view(np.uint64))
        assert np.array_equal(b.cpu().numpy().view(np.uint64), bo.view(np.uint64))


def test_assembly_host_pointers(gw):
    p = PROBLEMS["3d_het_20"]()
    A, b = gw.gw_assemble(p["nx"], p["ny"], p["nz"], p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"])
    Ao, bo = ora_assemble(p)
    assert np.array_equal(b, bo)
    assert np.array_equal(A.export()[2], Ao.arrays()[2])


@pytest.mark.parametrize("bad", ["kneg", "knan", "noflow", "qinf", "zero_size"])
def test_assembly_rejects_bad_input(gw, bad):
    n = 6 * 5 * 4
    K = np.ones(n)
    bct, q, nx = (1, 1, 0, 0, 0, 0), None, 6
    if bad == "kneg":
        K[7] = -1.0
    elif bad == "knan":
        K[7] = np.nan
    elif bad == "noflow":
        bct = (0,) * 6
    elif bad == "qinf":
        q = np.zeros(n)
        q[2] = np.inf
    else:
        nx = 0
    with pytest.raises(gw.GwError) as e:
        gw.gw_assemble(nx, 5, 4, dev(K), q=dev(q), bct=bct)
    assert e.value.status == gw.GW_ERR_ARG


def compare_setup(gw, p, **opts):
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, **opts)
    Ao, bo = ora_assemble(p)
    Ho = oracle.Hierarchy(Ao, n_coarse=opts.get("n_coarse", 1024), seed=opts.get("seed", 0x5EED))
    info = H.info()
    assert len(info) == Ho.nlevels
    for l in range(Ho.nlevels):
        agg, root, (arp, aci, av), P = H.export_level(l)
        Al = Ho.A(l)
        orp, oci, ov = Al.arrays()
        assert np.array_equal(arp, orp) and np.array_equal(aci, oci), "A_%d pattern" % l
        assert np.array_equal(av.view(np.uint64), ov.view(np.uint64)), "A_%d values" % l
        if l < Ho.nlevels - 1:
            oagg, oroot, _ = Ho.level(l)
            assert np.array_equal(root, oroot), "MIS-2 roots on level %d" % l
            assert np.array_equal(agg, oagg), "aggregates on level %d" % l
            prp, pci, pv = P
            Pl = Ho.P(l)
            qrp, qci, qv = Pl.arrays()
            assert np.array_equal(prp, qrp) and np.array_equal(pci, qci), "P_%d pattern" % l
            assert np.array_equal(pv.view(np.uint64), qv.view(np.uint64)), "P_%d values" % l
            assert info[l]["omega_p"] == Ho.scalars(l)["omegaP"]
    return H, Ho, A, b, Ao, bo


@pytest.mark.parametrize("name,nc", [("2d_homog_128", 1024), ("3d_het_20", 64), ("3d_layered_24", 100),
                                     ("3d_het_33_sigma4", 200)])
def test_setup_bit_exact(gw, name, nc):
    compare_setup(gw, PROBLEMS[name](), n_coarse=nc)


def test_setup_bit_exact_other_seed(gw):
    compare_setup(gw, PROBLEMS["3d_het_20"](), n_coarse=64, seed=12345)


@pytest.mark.parametrize("form", ["thread", "warp"])
def test_setup_bit_exact_in_each_row_form(gw, form):
    """The SpGEMM and the smoothed-prolongator passes have a thread-per-row and
    a warp-per-row form (the library picks one per product from the row
    counts and lengths, so small problems would only see one of them);
    GW_SETUP_FORMS forces either on every product, including the thread
    form's hand-over of rows with more than 64 distinct columns to the warp
    form.  Every level stays bit-exact with the oracle.  The variable is read
    once per process, so the setup tests run again in a child process."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GW_SETUP_FORMS=form)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        "-k", "setup_bit_exact and not each_row_form", os.path.join(root, "tests", "test_gpu_parity.py")],
                       env=env, cwd=root, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and " passed" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("smoother,nu", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_solve_parity(gw, prec, smoother, nu):
    p = PROBLEMS["3d_het_33_sigma4"]()
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, n_coarse=200, prec=prec, smoother=smoother, nu=nu)
    h, it, rel, st = H.solve(b, tol=TOL)
    assert st == gw.GW_OK and rel <= TOL
    Ao, bo = ora_assemble(p)
    Ho = oracle.Hierarchy(Ao, n_coarse=200, smoother=smoother, nu=nu)
    href, it_ref, _, _ = Ho.pcg(bo, tol=1e-12)
    hh = h.cpu().numpy()
    assert np.linalg.norm(hh - href) / np.linalg.norm(href) <= REL_ERR
    true_rel = np.linalg.norm(bo - Ao.matvec(hh)) / np.linalg.norm(bo)
    assert true_rel <= TOL * 1.0001
    assert rel == pytest.approx(true_rel, rel=1e-6)
    if prec == 0:
        _, it_o8, _, _ = Ho.pcg(bo, tol=TOL)
        assert abs(it - it_o8) <= 1


def test_vcycle_matches_oracle_fp64(gw):
    p = PROBLEMS["3d_het_20"]()
    A, b = gpu_assemble(gw, p)
    Ao, bo = ora_assemble(p)
    for smoother, tol in ((0, 1e-12), (1, 1e-9)):
        H = gw.Hierarchy(A, n_coarse=64, prec=0, smoother=smoother)
        Ho = oracle.Hierarchy(Ao, n_coarse=64, smoother=smoother)
        z = torch.empty_like(b)
        H.vcycle(b, z)
        zo = Ho.vcycle(bo)
        assert np.linalg.norm(z.cpu().numpy() - zo) <= tol * np.linalg.norm(zo)
        H32 = gw.Hierarchy(A, n_coarse=64, prec=1, smoother=smoother)
        H32.vcycle(b, z)
        assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-5 * np.linalg.norm(zo)


def test_config0_closed_form(gw):
    p = wl.homogeneous_2d_128()
    A, b = gpu_assemble(gw, p)
    for prec in (0, 1):
        H = gw.Hierarchy(A, prec=prec)
        h, it, rel, st = H.solve(b, tol=TOL)
        assert st == gw.GW_OK and rel <= TOL
        x = np.tile(np.arange(128), 128)
        href = 1.0 - (x + 0.5) / 128
        assert np.linalg.norm(h.cpu().numpy() - href) / np.linalg.norm(href) <= REL_ERR


def test_status_codes_and_edge_cases(gw):
    p = PROBLEMS["3d_het_20"]()
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, n_coarse=64)
    h, it, rel, st = H.solve(b, tol=1e-14, maxit=2)
    assert st == gw.GW_ERR_NOT_CONVERGED and it == 2 and rel > 1e-14
    true_rel = np.linalg.norm(b.cpu().numpy() - A_mat(A) @ h.cpu().numpy()) / np.linalg.norm(b.cpu().numpy())
    assert rel == pytest.approx(true_rel, rel=1e-6)
    z = torch.zeros_like(b)
    h, it, rel, st = H.solve(z, tol=1e-8)
    assert st == gw.GW_OK and it == 0 and not h.any()
    with pytest.raises(gw.GwError):
        H.solve(b, tol=-1.0)
    # host buffers in and out
    hb, it2, rel2, st2 = H.solve(b.cpu().numpy(), tol=1e-8)
    hd, it3, rel3, st3 = H.solve(b, tol=1e-8)
    assert st2 == st3 == gw.GW_OK and it2 == it3
    assert np.array_equal(hb, hd.cpu().numpy())


def A_mat(A):
    import scipy.sparse as sp

    rp, ci, v = A.export()
    return sp.csr_matrix((v, ci, rp), shape=(A.n, A.n))


def test_bitwise_reproducible(gw):
    p = PROBLEMS["3d_het_33_sigma4"]()
    A, b = gpu_assemble(gw, p)
    outs = []
    for _ in range(2):
        H = gw.Hierarchy(A, n_coarse=200)
        h, it, rel, st = H.solve(b, tol=TOL)
        h2, it2, _, _ = H.solve(b, tol=TOL)
        assert torch.equal(h, h2) and it == it2
        outs.append((h.cpu().numpy(), it))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_hierarchy_info_matches_oracle_statistics(gw):
    p = PROBLEMS["3d_het_33_sigma4"]()
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, n_coarse=200)
    Ao, _ = ora_assemble(p)
    st = oracle.Hierarchy(Ao, n_coarse=200).stats()
    info = H.info()
    assert [l["n"] for l in info] == st["n"]
    assert [l["nnz"] for l in info] == st["nnz"]
    assert all(l["bytes"] > 0 for l in info)


@pytest.mark.parametrize("prec", [1, 0])
def test_full_size_128_cubed_sigma4(gw, prec):
    """The 128^3 sigma^2 = 4 workload at full size, in the bench's configuration."""
    p = wl.heterogeneous_3d(side=128, var=4.0, corr=8.0, seed=1)
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, prec=prec)
    h, it, rel, st = H.solve(b, tol=TOL)
    assert st == gw.GW_OK and rel <= TOL
    Ao, bo = ora_assemble(p)
    Ho = oracle.Hierarchy(Ao)
    info = H.info()
    assert [l["n"] for l in info] == Ho.stats()["n"]
    # every level bit for bit: aggregates, roots, P_l and A_l
    for l in range(len(info)):
        agg, root, (arp, aci, av), P = H.export_level(l)
        orp, oci, ov = Ho.A(l).arrays()
        assert np.array_equal(arp, orp) and np.array_equal(aci, oci), l
        assert np.array_equal(av.view(np.uint64), ov.view(np.uint64)), l
        if P is not None:
            oagg, oroot, _ = Ho.level(l)
            assert np.array_equal(agg, oagg) and np.array_equal(root, oroot), l
            prp, pci, pv = P
            qrp, qci, qv = Ho.P(l).arrays()
            assert np.array_equal(prp, qrp) and np.array_equal(pci, qci), l
            assert np.array_equal(pv.view(np.uint64), qv.view(np.uint64)), l
    href, _, _, _ = Ho.pcg(bo, tol=1e-12)
    assert np.linalg.norm(h.cpu().numpy() - href) / np.linalg.norm(href) <= REL_ERR


@pytest.mark.parametrize("half", ["bf16", "fp16"])
@pytest.mark.parametrize("name", ["3d_het_33_sigma4", "3d_layered_24", "2d_homog_128"])
def test_half_fine_stencil_solves_to_parity(gw, name, half):
    """GW_HALF_FINE (BF16 couplings, corrected FP32 diagonal) and GW_HALF_FINE16
    (FP16 couplings of the diagonally scaled stencil): the solve still stops
    on the FP64 residual, agrees with the oracle, and the preconditioner stays
    close to the FP32 one (a few iterations more at most)."""
    bits, alias = ((gw.GW_HALF_FINE, gw.GW_PREC_MIXEDBF16) if half == "bf16"
                   else (gw.GW_HALF_FINE16, gw.GW_PREC_MIXED16))
    p = PROBLEMS[name]()
    A, b = gpu_assemble(gw, p)
    H32 = gw.Hierarchy(A, n_coarse=64)
    Hb = gw.Hierarchy(A, n_coarse=64, half_storage=bits)
    h32, it32, _, _ = H32.solve(b, tol=TOL)
    hb, itb, relb, st = Hb.solve(b, tol=TOL)
    assert st == gw.GW_OK and relb <= TOL
    assert itb <= it32 + 3
    Ao, bo = ora_assemble(p)
    href, _, _, _ = oracle.Hierarchy(Ao, n_coarse=64).pcg(bo, tol=1e-12)
    assert np.linalg.norm(hb.cpu().numpy() - href) / np.linalg.norm(href) <= REL_ERR
    # the precision name of the same configuration
    hp, itp, _, _ = gw.Hierarchy(A, n_coarse=64, prec=alias).solve(b, tol=TOL)
    assert itp == itb and torch.equal(hp, hb)
    with pytest.raises(gw.GwError):
        gw.Hierarchy(A, prec=gw.GW_PREC_FP64, half_storage=bits)
    with pytest.raises(gw.GwError):
        gw.Hierarchy(A, half_storage=gw.GW_HALF_FINE | gw.GW_HALF_FINE16)
    # the interleaved block path runs the same stored operator
    B = torch.stack([b, 2.0 * b])
    X, its, rels, st = Hb.solve_many(B, tol=TOL)
    assert st == gw.GW_OK and max(rels) <= TOL
    assert np.linalg.norm(X[1].cpu().numpy() - 2 * href) / np.linalg.norm(2 * href) <= REL_ERR


@pytest.mark.parametrize("half", [0, 2, 4])
@pytest.mark.parametrize("prec", [1, 0])
def test_full_size_layered_256x256x128(gw, prec, half):
    """The 256x256x128 layered case (lnK variance 1, correlation 32/32/4 cells,
    Kh/Kv = 10, 16 wells, fixed head on top) at full size: level-0 aggregates,
    roots and the level-1 operator bit-exact, the solution within 1e-6 of the
    oracle's, in the FP64 form, the mixed form and the mixed form with the
    BF16- or FP16-stored fine stencil."""
    if prec == 0 and half:
        pytest.skip("BF16 storage belongs to the mixed form")
    p = wl.layered_wells_3d()
    assert (p["nx"], p["ny"], p["nz"]) == (256, 256, 128)
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, prec=prec, half_storage=half)
    h, it, rel, st = H.solve(b, tol=TOL)
    assert st == gw.GW_OK and rel <= TOL
    ref = _layered_reference()
    info = H.info()
    assert [l["n"] for l in info] == ref["n"]
    agg, root, _, _ = H.export_level(0)
    assert np.array_equal(agg, ref["agg"]) and np.array_equal(root, ref["root"])
    _, _, (arp1, aci1, av1), _ = H.export_level(1)
    assert np.array_equal(arp1, ref["A1"][0]) and np.array_equal(aci1, ref["A1"][1])
    assert np.array_equal(av1.view(np.uint64), ref["A1"][2].view(np.uint64))
    err = np.linalg.norm(h.cpu().numpy() - ref["h"]) / np.linalg.norm(ref["h"])
    assert err <= REL_ERR, err


_LAYERED = {}


def _layered_reference():
    """The oracle's hierarchy statistics, level-0/1 data and solve to 1e-12 of the layered case (computed once)."""
    if not _LAYERED:
        p = wl.layered_wells_3d()
        Ao, bo = ora_assemble(p)
        Ho = oracle.Hierarchy(Ao)
        agg, root, _ = Ho.level(0)
        _LAYERED.update(n=Ho.stats()["n"], agg=agg.copy(), root=root.copy(),
                        A1=[a.copy() for a in Ho.A(1).arrays()])
        _LAYERED["h"] = Ho.pcg(bo, tol=1e-12)[0]
    return _LAYERED


@pytest.mark.parametrize("prec", [1, 0])
def test_chebyshev_degree3_solve_parity(gw, prec):
    """Chebyshev of degree 3 (the steps after the first two keep r and d)."""
    p = PROBLEMS["3d_het_33_sigma4"]()
    A, b = gpu_assemble(gw, p)
    H = gw.Hierarchy(A, n_coarse=200, prec=prec, degree=3)
    h, it, rel, st = H.solve(b, tol=TOL)
    assert st == gw.GW_OK and rel <= TOL
    Ao, bo = ora_assemble(p)
    href, _, _, _ = oracle.Hierarchy(Ao, n_coarse=200, degree=3).pcg(bo, tol=1e-12)
    assert np.linalg.norm(h.cpu().numpy() - href) / np.linalg.norm(href) <= REL_ERR
