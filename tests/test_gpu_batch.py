"""Batched solves (gw_batch_*): one launch per pass for every solve in flight.

Each solve of a batch keeps its own hierarchy and runs every pass on a
virtual grid fixed by its own size, so its result must be the same bit for
bit whether it runs alone or next to other solves of other sizes, depths and
fields, and whenever it joins.  Results are checked against the oracle's
solve to 1e-12 (relative error <= 1e-6, true relative residual <= 1e-8), and
the refusal paths (unsupported hierarchies, a hierarchy already in flight,
a slot that has not finished) against their status codes.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05798_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


# grids whose x extent makes the level-0 stencil take 4, 2 and 1 rows a thread,
# and depths from 3 to 4 levels
SHAPES = [(24, 20, 16, 3.0, 4.0, 11), (30, 14, 12, 2.0, 3.0, 12), (17, 19, 21, 4.0, 5.0, 13),
          (32, 32, 32, 1.0, 6.0, 14), (20, 18, 10, 0.5, 2.0, 15)]


def system(gw, nx, ny, nz, var, corr, seed):
    p = wl.problem(nx, ny, nz, var=var, corr=corr, seed=seed, wells_count=2, wells_seed=seed + 1)
    n = nx * ny * nz
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(nx, ny, nz, dev(p["Kx"]), dev(p["Ky"]), dev(p["Kz"]), p["bct"], p["bcv"], dev(p["q"]),
                          b_out=b)
    torch.cuda.synchronize()
    return p, A, b


def run_to_end(gw, B, limit=2000):
    for _ in range(limit):
        if not [s for s in B.held if B.state(s) == 1]:
            return
        B.run(4)
    raise AssertionError("batched solves did not finish")


def take(B, slot, n):
    h = torch.empty(n, dtype=torch.float64, device="cuda")
    _, it, rel, st = B.take(slot, h)
    torch.cuda.synchronize()
    return h.cpu().numpy(), it, rel, st


def test_alone_and_in_the_mix_bit_identical_and_match_the_oracle(gw):
    systems = [system(gw, *s) for s in SHAPES]
    alone = []
    for p, A, b in systems:
        H = gw.Hierarchy(A, n_coarse=64)
        B = gw.Batch(4)
        s = B.add(H, b, tol=TOL)
        run_to_end(gw, B)
        alone.append(take(B, s, b.numel()))
        B.close()
    for (h, it, rel, st) in alone:
        assert st == gw.GW_OK and rel <= TOL
    # all at once (the last one joins after the others have run a while), in a
    # batch with fewer slots than solves so that a freed slot is reused
    B = gw.Batch(4)
    Hs = [gw.Hierarchy(A, n_coarse=64) for _, A, _ in systems]
    slots = {}
    for k in range(4):
        slots[B.add(Hs[k], systems[k][2], tol=TOL)] = k
    B.run(3)
    mixed = {}
    pending = [4]
    for _ in range(2000):
        for s in [s for s in list(B.held) if B.state(s) == 2]:
            k = slots.pop(s)
            mixed[k] = take(B, s, systems[k][2].numel())
            if pending:
                j = pending.pop()
                slots[B.add(Hs[j], systems[j][2], tol=TOL)] = j
        if len(mixed) == len(systems):
            break
        B.run(2)
    B.close()
    assert len(mixed) == len(systems)
    for k, (p, A, b) in enumerate(systems):
        h0, it0, rel0, st0 = alone[k]
        h1, it1, rel1, st1 = mixed[k]
        assert st1 == gw.GW_OK and it1 == it0 and rel1 == rel0
        assert np.array_equal(h0.view(np.uint64), h1.view(np.uint64)), "solve %d differs alone and in the mix" % k
        Ao, bo = oracle.assemble(p["nx"], p["ny"], p["nz"], p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"])
        Ho = oracle.Hierarchy(Ao, n_coarse=64)
        ho, _, _, _ = Ho.pcg(bo, tol=1e-12)
        assert np.linalg.norm(h1 - ho) / np.linalg.norm(ho) <= 1e-6
        # the batched iteration follows gw_pcg_solve up to the rounding of its reductions
        H = gw.Hierarchy(A, n_coarse=64)
        _, its, _, sts = H.solve(b, tol=TOL)
        assert sts == gw.GW_OK and abs(its - it1) <= 1


def test_chebyshev_degree_three_batch(gw):
    systems = [system(gw, *s) for s in SHAPES[:3]]
    B = gw.Batch(3)
    slots = {B.add(gw.Hierarchy(A, n_coarse=64, degree=3), b, tol=TOL): k for k, (_, A, b) in enumerate(systems)}
    run_to_end(gw, B)
    for s, k in slots.items():
        p, A, b = systems[k]
        h, it, rel, st = take(B, s, b.numel())
        assert st == gw.GW_OK and rel <= TOL
        Ao, bo = oracle.assemble(p["nx"], p["ny"], p["nz"], p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"])
        ho, _, _, _ = oracle.Hierarchy(Ao, n_coarse=64, degree=3).pcg(bo, tol=1e-12)
        assert np.linalg.norm(h - ho) / np.linalg.norm(ho) <= 1e-6
    B.close()


def test_batch_refusals(gw):
    p, A, b = system(gw, *SHAPES[0])
    B = gw.Batch(2)
    for bad in (dict(prec=gw.GW_PREC_FP64), dict(smoother=gw.GW_SMOOTH_JACOBI), dict(nu=2),
                dict(half_storage=gw.GW_HALF_FINE)):
        with pytest.raises(gw.GwError) as e:
            B.add(gw.Hierarchy(A, n_coarse=64, **bad), b)
        assert e.value.status == gw.GW_ERR_ARG
    H = gw.Hierarchy(A, n_coarse=64)
    s = B.add(H, b, tol=TOL)
    with pytest.raises(gw.GwError) as e:  # its solve is in flight
        H.solve(b)
    assert e.value.status == gw.GW_ERR_ARG
    with pytest.raises(gw.GwError) as e:
        B.add(H, b)
    assert e.value.status == gw.GW_ERR_ARG
    with pytest.raises(gw.GwError) as e:  # another degree in the same batch
        B.add(gw.Hierarchy(A, n_coarse=64, degree=3), b)
    assert e.value.status == gw.GW_ERR_ARG
    if B.state(s) == 1:
        with pytest.raises(gw.GwError) as e:
            B.take(s, torch.empty_like(b))
        assert e.value.status == gw.GW_ERR_ARG
    run_to_end(gw, B)
    h, it, rel, st = take(B, s, b.numel())
    assert st == gw.GW_OK and rel <= TOL
    h2, it2, rel2, st2 = H.solve(b, tol=TOL)  # usable on its own again
    assert st2 == gw.GW_OK
    # a non-finite right-hand side fails alone; the others of the batch go on
    bb = b.clone()
    bb[3] = float("nan")
    H1, H2 = gw.Hierarchy(A, n_coarse=64), gw.Hierarchy(A, n_coarse=64)
    s1 = B.add(H1, bb, tol=TOL)
    s2 = B.add(H2, b, tol=TOL)
    run_to_end(gw, B)
    with pytest.raises(gw.GwError) as e:
        take(B, s1, b.numel())
    assert e.value.status == gw.GW_ERR_ARG
    h3, it3, rel3, st3 = take(B, s2, b.numel())
    assert st3 == gw.GW_OK and it3 == it and np.array_equal(h3, h)
    # a hierarchy freed while in flight leaves the batch
    H4 = gw.Hierarchy(A, n_coarse=64)
    s4 = B.add(H4, b, tol=TOL)
    B.held.pop(s4)
    del H4
    assert B.state(s4) == 0
    B.close()
