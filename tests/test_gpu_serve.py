"""Continuous batching: each result is the same alone and in the mix.

Requests of different sizes and fields are solved one at a time, then all at
once on four slots (their kernels overlapping on the device); heads and
iteration counts must agree bit for bit, and every result must match the
oracle.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05798_gb300 import build, gw, serve as srv

    build.build()
    gw.load()
    return srv


def test_alone_and_in_the_mix_agree(serve):
    from paper_2001_05798_gb300 import workload as wl

    reqs = wl.serving_requests(count=8, seed=11, side_range=(16, 40))
    alone = {}
    s1 = serve.Server(slots=1, n_coarse=200)
    try:
        for r in reqs:
            out = s1.submit(r).result(timeout=300)
            alone[r["id"]] = out
    finally:
        s1.close()
    s4 = serve.Server(slots=4, n_coarse=200)
    try:
        futs = [s4.submit(r) for r in reqs]
        mixed = {f.result(timeout=300)["id"]: f.result() for f in futs}
    finally:
        s4.close()
    assert s4.peak_inflight >= 2
    for r in reqs:
        a, m = alone[r["id"]], mixed[r["id"]]
        assert a["iters"] == m["iters"]
        assert torch.equal(a["h"], m["h"])
        assert a["relres"] <= 1e-8
    # one result against the oracle (the field is regenerated identically)
    r = reqs[0]
    s = r["side"]
    K = torch.exp(wl.lnk_field_device(s, s, s, r["var"], r["corr"], r["seed"], pad=serve.FIELD_PAD)).cpu().numpy()
    A, b = oracle.assemble(s, s, s, K)
    href, _, _, _ = oracle.Hierarchy(A, n_coarse=200).pcg(b, tol=1e-12)
    h = alone[r["id"]]["h"].cpu().numpy()
    assert np.linalg.norm(h - href) <= 1e-6 * np.linalg.norm(href)


def test_budget_admission_and_rejection(serve):
    from paper_2001_05798_gb300 import workload as wl

    reqs = wl.serving_requests(count=6, seed=12, side_range=(20, 30))
    srv = serve.Server(slots=4, hbm_budget=1500.0 * 30 ** 3 * 1.01, n_coarse=200)
    try:
        futs = [srv.submit(r) for r in reqs]
        for f in futs:
            try:
                assert f.result(timeout=300)["relres"] <= 1e-8
            except MemoryError:
                pass  # the per-cell estimate grew past this tiny budget: rejected, not hung
    finally:
        srv.close()
    assert srv.peak_in_use <= srv.budget
    big = serve.Server(slots=1, hbm_budget=1e6)
    try:
        with pytest.raises(MemoryError):
            big.submit(dict(id=0, side=64, var=1.0, corr=4.0, seed=1)).result(timeout=60)
    finally:
        big.close()


def test_prepare_then_solve_equals_plain_solve(serve):
    """gw_hierarchy_prepare captures the solver's graphs up front; the solves
    that follow replay them and give the same heads, bit for bit, as a
    hierarchy whose first solve captures them itself."""
    from paper_2001_05798_gb300 import gw, workload as wl

    p = wl.heterogeneous_3d(side=24, var=2.0, corr=4.0, seed=8)
    A, b = gw.gw_assemble(24, 24, 24, p["Kx"])
    H1 = gw.Hierarchy(A, n_coarse=200)
    H1.prepare()
    H1.prepare()  # a second call keeps the captured graphs
    H2 = gw.Hierarchy(A, n_coarse=200)
    bd = torch.from_numpy(b).cuda()
    h1, it1, rel1, st1 = H1.solve(bd, tol=1e-9)
    h2, it2, rel2, st2 = H2.solve(bd, tol=1e-9)
    assert st1 == st2 == gw.GW_OK and it1 == it2 and rel1 == rel2
    assert torch.equal(h1, h2)


def test_batched_server_alone_and_in_the_mix_agree(serve):
    """The batched server: every launch of the iteration covers all solves in
    flight; each result is the same bit for bit served alone or in the mix."""
    from paper_2001_05798_gb300 import workload as wl

    reqs = wl.serving_requests(count=8, seed=12, side_range=(16, 40))
    s1 = serve.BatchedServer(slots=1, setup_workers=1, n_coarse=200)
    try:
        alone = {r["id"]: s1.submit(r).result(timeout=300) for r in reqs}
    finally:
        s1.close()
    s4 = serve.BatchedServer(slots=4, setup_workers=3, n_coarse=200)
    try:
        futs = [s4.submit(r) for r in reqs]
        mixed = {f.result(timeout=300)["id"]: f.result() for f in futs}
    finally:
        s4.close()
    assert s4.peak_inflight >= 2
    for r in reqs:
        a, m = alone[r["id"]], mixed[r["id"]]
        assert a["iters"] == m["iters"] and a["relres"] <= 1e-8
        assert torch.equal(a["h"], m["h"])
    r = reqs[1]
    s = r["side"]
    K = torch.exp(wl.lnk_field_device(s, s, s, r["var"], r["corr"], r["seed"], pad=serve.FIELD_PAD)).cpu().numpy()
    A, b = oracle.assemble(s, s, s, K)
    href, _, _, _ = oracle.Hierarchy(A, n_coarse=200).pcg(b, tol=1e-12)
    h = mixed[r["id"]]["h"].cpu().numpy()
    assert np.linalg.norm(h - href) <= 1e-6 * np.linalg.norm(href)
