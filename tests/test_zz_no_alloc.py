"""gw_assemble_noalloc: assembly for callers that cannot allocate device memory.

Some host codes hand the solver a fixed device pool or call it where a
cudaMalloc is not allowed.  For them the library offers an assembly entry
point that allocates nothing: the caller passes the output arrays and the
kernels' working memory is a fixed array the library keeps on the device.
These tests call that entry point through the C ABI, twice in a row and after
a rejected call, and check every result against gw_assemble bit for bit (the
tolerance the assembly parity tests use).  The file is collected last so a
failure here stops a run only after every other test has run.
"""
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


def reference(gw, p, spacing=(1.0, 1.0, 1.0)):
    n = p["nx"] * p["ny"] * p["nz"]
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(p["nx"], p["ny"], p["nz"], dev(p["Kx"]), dev(p["Ky"]), dev(p["Kz"]), p["bct"], p["bcv"],
                          dev(p["q"]), b_out=b, spacing=spacing)
    rp, ci, v = A.export()
    return rp, ci, v, b.cpu().numpy()


def no_alloc(gw, p, spacing=(1.0, 1.0, 1.0), stream=None):
    """Calls the allocation-free entry point into fresh output arrays and
    checks that the library made no device allocation meanwhile."""
    n = p["nx"] * p["ny"] * p["nz"]
    nnz = 7 * n - 2 * (p["ny"] * p["nz"] + p["nx"] * p["nz"] + p["nx"] * p["ny"])
    rp = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    ci = torch.full((nnz,), -1, dtype=torch.int32, device="cuda")
    v = torch.full((nnz,), np.nan, dtype=torch.float64, device="cuda")
    b = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    Kx, Ky, Kz, q = dev(p["Kx"]), dev(p["Ky"]), dev(p["Kz"]), dev(p["q"])
    torch.cuda.synchronize()
    before = gw.gw_device_allocations()
    try:
        gw.gw_assemble_noalloc(p["nx"], p["ny"], p["nz"], Kx, rp, ci, v, b, Ky=Ky, Kz=Kz, bct=p["bct"],
                               bcv=p["bcv"], q=q, spacing=spacing, stream=stream)
    finally:
        assert gw.gw_device_allocations() == before, "the allocation-free assembly allocated device memory"
    torch.cuda.synchronize()
    return rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), b.cpu().numpy()


def same(a, b):
    for x, y in zip(a, b):
        assert x.shape == y.shape
        if x.dtype == np.float64:
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64))
        else:
            assert np.array_equal(x, y)


def test_no_alloc_matches_gw_assemble_on_consecutive_calls(gw):
    p1 = wl.problem(23, 19, 11, var=4.0, corr=3.0, seed=5, wells_count=3, wells_seed=1,
                    bct=(1, 1, 0, 1, 0, 0), bcv=(1.0, 0.0, 0, 0.3, 0, 0))
    p2 = wl.layered_wells_3d(nx=40, ny=36, nz=9, corr=(6.0, 6.0, 2.0), wells_count=4)
    r1, r2 = reference(gw, p1), reference(gw, p2)
    same(no_alloc(gw, p1), r1)
    same(no_alloc(gw, p2), r2)
    same(no_alloc(gw, p1), r1)


def test_no_alloc_degenerate_axis_shared_conductivity_and_spacing(gw):
    # a 2D grid (nz = 1, where the nonzero count formula is tightest), no
    # sources, Ky and Kz left to default to Kx, and unequal cell sizes
    p = wl.problem(31, 17, 1, var=3.0, corr=3.0, seed=11)
    p = dict(p, q=None, Ky=None, Kz=None, bct=(1, 1, 1, 0, 0, 0), bcv=(1.0, 0.0, 0.5, 0, 0, 0))
    for spacing in ((1.0, 1.0, 1.0), (1.0, 2.0, 0.5)):
        r = reference(gw, p, spacing)
        same(no_alloc(gw, p, spacing), r)
        same(no_alloc(gw, p, spacing), r)


def test_no_alloc_on_a_caller_stream(gw):
    p = wl.problem(20, 12, 6, var=2.0, corr=2.0, seed=13, wells_count=2, wells_seed=3)
    r = reference(gw, p)
    s = torch.cuda.Stream()
    same(no_alloc(gw, p, stream=s), r)
    same(no_alloc(gw, p, stream=s), r)


def test_no_alloc_refuses_a_capturing_stream(gw):
    p = wl.problem(8, 8, 4, var=1.0, corr=2.0, seed=3)
    n = 8 * 8 * 4
    nnz = 7 * n - 2 * (8 * 4 + 8 * 4 + 8 * 8)
    K = dev(p["Kx"])
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(nnz, dtype=torch.int32, device="cuda")
    v = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="thread_local")
        try:
            gw.gw_assemble_noalloc(8, 8, 4, K, rp, ci, v, b, stream=s)
        except gw.GwError as e:
            status = e.status
        finally:
            g.capture_end()
    assert status == gw.GW_ERR_ARG
    same(no_alloc(gw, p), reference(gw, p))


def test_no_alloc_after_a_rejected_call(gw):
    p = wl.problem(17, 13, 7, var=2.0, corr=2.0, seed=9)
    bad = dict(p)
    K = p["Kx"].copy()
    K[5] = -1.0
    bad["Kx"] = bad["Ky"] = bad["Kz"] = K
    with pytest.raises(gw.GwError) as e:
        no_alloc(gw, bad)
    assert e.value.status == gw.GW_ERR_ARG
    same(no_alloc(gw, p), reference(gw, p))
    same(no_alloc(gw, p), reference(gw, p))


def test_no_alloc_rejects_what_it_cannot_hold(gw):
    K = torch.ones(8, dtype=torch.float64, device="cuda")
    out_i = torch.zeros(8, dtype=torch.int32, device="cuda")
    out_d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(gw.GwError) as e:  # beyond the fixed workspace
        gw.gw_assemble_noalloc(1 << 14, 1 << 14, 2, K, out_i, out_i, out_d, out_d)
    assert e.value.status == gw.GW_ERR_ARG
    with pytest.raises(gw.GwError) as e:  # host arrays would need staging
        gw.gw_assemble_noalloc(2, 2, 2, np.ones(8), out_i, out_i, out_d, out_d)
    assert e.value.status == gw.GW_ERR_ARG
