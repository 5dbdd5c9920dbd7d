"""Benchmark: AMG-PCG solve time and fine-level V-cycle HBM bandwidth.

Workload: 3D heterogeneous steady flow on 128^3 cells (2,097,152 unknowns),
7-point finite volumes with harmonic-mean transmissibilities, lnK Gaussian
(mean 0, variance 4, exponential covariance, correlation length 8 cells,
seed 1), h = 1 / h = 0 on the x faces, no-flow elsewhere; solved to a true
relative residual of 1e-8 from h0 = 0.  One step = one gw_pcg_solve with the
hierarchy resident (setup excluded and reported separately).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The primary arm runs the mixed-precision form (FP32 V-cycle inside FP64 CG);
the all-FP64 form is timed beside it.  --impl reference times the FP64 CPU
oracle on the same workload.  Under torchrun (N > 1) every rank solves its own
copy of the workload on its own GPU (replicas, no collective on the data
path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AMG-PCG solve ms & V-cycle HBM GB/s @128³ to 1e-8 (mixed vs FP64); p50/p99"
WORKLOAD = ("3D heterogeneous steady flow 128^3 cells (2,097,152 unknowns), 7-point FV harmonic-mean "
            "transmissibilities, lnK N(0, 4) exponential covariance corr 8 cells seed 1, h=1/h=0 on x faces, "
            "tol 1e-8 (true relative residual), x0 = 0")
SIDE, VAR, CORR, SEED, TOL = 128, 4.0, 8.0, 1, 1e-8
# --side changes the grid for profiling captures only (the benchmark is 128^3)
L2_FLUSH_BYTES = 256 << 20
# level-0 kernels timed one by one in the profiled pass (kind -> kernel at 128^3)
# with the arrays each touches once per row (stencil: diagonal and the +x, +y,
# +z couplings, 16 bytes); the profiled bytes are these times 2,097,152 rows
SINGLE_KERNELS = {
    "spmv": "k_cg_dir_spmv<MSten<float,4>> (stencil 16 B; z, p_old read, p_new, q written: 32 B/row)",
    "update": "k_cg_update<float,4> (xs, r read and written, p, q read: 24 B/row)",
    "pre1": "k_cheb_zero2<MSten<float,4>,float,0> (stencil, dw, b read, x written: 28 B/row)",
    "resid": "k_residual<MSten<float,4>,float> (stencil, b, x read, r written: 28 B/row)",
    "prolong": "k_prolong_imp<4> (s, fx, fy, fz, agg, x read, x written: 28 B/row + coarse vector)",
    "post1": "k_cheb0<MSten<float,4>,float,float,0> (stencil, dw, b, x read, r, d written: 36 B/row)",
    "post2": "k_chebk<MSten<float,4>,float,1> (stencil, d, r, dw, x, b, q read, r, d2, z written: 52 B/row)",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:  # sampling runs before timing starts
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_problem():
    from paper_2001_05798_gb300 import workload as wl

    return wl.heterogeneous_3d(side=SIDE, var=VAR, corr=CORR, seed=SEED)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity on one
    rank).  Replicas exchange only these timing scalars; no data-path collective."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(world_size, p50_ms):
    """Whole-job solves per second of N replicas each solving one problem per step."""
    return world_size * 1e3 / p50_ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


REFERENCE_BUDGET_S = 120.0  # whole --impl reference run, timed and warm-up steps together


def run_reference(args):
    """FP64 CPU oracle on the same workload.  One step is one oracle solve when
    K + W full solves fit REFERENCE_BUDGET_S; otherwise a bounded sample: the
    first m CG iterations of the solve (m chosen to fit), scaled to the full
    solve's iteration count.  Setup excluded."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    p = make_problem()
    A, b = oracle.assemble(SIDE, SIDE, SIDE, p["Kx"], bct=p["bct"], bcv=p["bcv"])
    t0 = time.perf_counter()
    H = oracle.Hierarchy(A)
    setup_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    x, its_full, rel, st = H.pcg(b, tol=TOL)  # first warm-up step: iteration count and cost
    full_s = time.perf_counter() - t0
    allowance = REFERENCE_BUDGET_S / max(1, args.steps + args.warmup)
    m = its_full if full_s <= allowance else max(1, int(its_full * allowance / full_s))
    for _ in range(max(0, args.warmup - 1)):
        H.pcg(b, tol=TOL, maxit=m)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        H.pcg(b, tol=TOL, maxit=m)
        times.append((time.perf_counter() - t0) * 1e3 * its_full / m)
    p50 = float(np.median(times))
    sample = ("one full oracle solve of the 128^3 workload per step (%d iterations, setup excluded)" % its_full
              if m == its_full else
              "the first %d of the %d CG iterations of the 128^3 oracle solve per step, scaled by %d/%d "
              "(setup excluded)" % (m, its_full, its_full, m))
    out = {"metric": METRIC, "value": p50, "unit": "ms", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(times)),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "tol": TOL, "smoother": "chebyshev", "implementation":
                      "FP64 CPU oracle (plain C, single thread)"},
           "p50_ms": p50, "p99_ms": float(np.percentile(times, 99)), "iters": its_full, "relres": rel,
           "setup_ms": setup_ms,
           "cpu_baseline": {"value": p50, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": p50, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline_sample():
    """The oracle as it stands, one solve of the same workload on one host core."""
    import oracle

    p = make_problem()
    A, b = oracle.assemble(SIDE, SIDE, SIDE, p["Kx"], bct=p["bct"], bcv=p["bcv"])
    t0 = time.perf_counter()
    H = oracle.Hierarchy(A)
    setup_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    x, its, rel, st = H.pcg(b, tol=TOL)
    ms = (time.perf_counter() - t0) * 1e3
    return {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": "one full FP64 oracle solve of the 128^3 workload to 1e-8 (setup %.0f ms excluded), "
                      "%d iterations; host has %d cores" % (setup_ms, its, os.cpu_count() or 0)}, x


def timed_solves(torch, H, b, h, steps, flush, stream):
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, it, rel, st = H.solve(b, h, tol=TOL, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, it, rel, st


TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "ncu_traffic_bench_128cubed.json")


def traffic_of(roof, n):
    """DRAM bytes per launch of the roofline kernel from the committed ncu capture
    of the same workload (read + write, caches flushed by ncu), when it covers
    this kernel at this size."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return
    k = t.get("kinds", {}).get(roof.get("kind"))
    if k and t.get("n") == n:
        roof["traffic"] = k["dram_bytes_per_launch"]
        roof["traffic_source"] = "profiles/ncu_traffic_bench_128cubed.json (%s)" % ", ".join(k["kernels"])


def run_ours(args):
    import torch

    from paper_2001_05798_gb300 import build, gw

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    build.build()
    gw.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    p = make_problem()
    n = SIDE ** 3
    K = torch.from_numpy(p["Kx"]).to(dev)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    A, _ = gw.gw_assemble(SIDE, SIDE, SIDE, K, K, K, p["bct"], p["bcv"], None, b_out=b)
    smoother = gw.GW_SMOOTH_CHEBYSHEV if args.smoother == "chebyshev" else gw.GW_SMOOTH_JACOBI
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hm = gw.Hierarchy(A, prec=gw.GW_PREC_MIXED32, smoother=smoother, delta=args.delta,
                      half_storage=args.half_storage)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    Hd = None if args.no_fp64 else gw.Hierarchy(A, prec=gw.GW_PREC_FP64, smoother=smoother)
    info = Hm.info()
    h = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        Hm.solve(b, h, tol=TOL, stream=stream)
        if Hd is not None:
            Hd.solve(b, h, tol=TOL, stream=stream)
    Hm.profile_read(reset=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # timed region: the headline solves, instrumentation off
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall = time.perf_counter()
        tm, it_m, rel_m, st_m = timed_solves(torch, Hm, b, h, args.steps, flush, stream)
        t_wall = time.perf_counter() - t_wall
    _, launches, solves = Hm.profile_read(reset=True)
    # second timed pass with CUDA events captured around the level-0 kernels
    Hm.profile(True)
    for _ in range(2):
        Hm.solve(b, h, tol=TOL, stream=stream)
    Hm.profile_read(reset=True)
    tp, _, _, _ = timed_solves(torch, Hm, b, h, args.steps, flush, stream)
    kinds, _, _ = Hm.profile_read(reset=True)
    Hm.profile(False)
    h_mixed = h.clone()
    if args.no_fp64:
        td, it_d, rel_d, st_d = [float("nan")], 0, float("nan"), -1
    else:
        td, it_d, rel_d, st_d = timed_solves(torch, Hd, b, h, args.steps, flush, stream)
    # end to end through the C ABI with host buffers: the H2D copy of b and the
    # D2H copy of h happen inside gw_pcg_solve, inside the timed region
    b_host = b.cpu().pin_memory()
    h_host = torch.empty(n, dtype=torch.float64).pin_memory()
    te = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hm.solve(b_host, h_host, tol=TOL, stream=stream)
        te.append((time.perf_counter() - t0) * 1e3)
    p50m, p50d = float(np.median(tm)), float(np.median(td))
    p50m, p50d, mean_m, p50e = max_over_ranks([p50m, p50d, float(np.mean(tm)), float(np.median(te))], device=dev)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    peak, peak_src = peaks()
    kern = {}
    for name, (ms, cnt, byts) in kinds.items():
        if cnt:
            per = ms / cnt
            kern[name] = {"ms_per_launch": per, "launches": cnt, "bytes_per_launch": byts, "ms_total": ms,
                          "gbs": byts / (per * 1e-3) / 1e9 if per > 0 and byts > 0 else None}
    # fine-level V-cycle: every level-0 kernel of the cycle, bytes over time
    fine = [k for k in ("pre1", "pre2", "resid", "restrict", "prolong", "post1", "post2") if k in kern]
    fb = sum(kern[k]["bytes_per_launch"] * kern[k]["launches"] for k in fine)
    ft = sum(kern[k]["ms_total"] for k in fine)
    fine_gbs = fb / (ft * 1e-3) / 1e9 if ft > 0 else None
    # the roofline line names one kernel: the single level-0 kernel with the
    # largest total time (the restriction is two launches and the coarse
    # groups are many, so they are reported in "kernels" only)
    timed = [k for k in kern if kern[k]["gbs"] and k in SINGLE_KERNELS]
    if timed:
        dom = max(timed, key=lambda k: kern[k]["ms_per_launch"] * kern[k]["launches"])
        roof = {"bound": "hbm", "kernel": SINGLE_KERNELS[dom], "kind": dom, "achieved": kern[dom]["gbs"],
                "peak": peak, "unit": "GB/s", "frac": kern[dom]["gbs"] / peak, "peak_source": peak_src,
                "traffic": None, "bytes_per_launch": kern[dom]["bytes_per_launch"],
                "bytes_per_row": kern[dom]["bytes_per_launch"] / n, "ms_per_launch": kern[dom]["ms_per_launch"]}
    else:
        roof = {"bound": "hbm", "kernel": None, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "peak_source": peak_src, "traffic": None, "note": "kernel timing unavailable"}
    out = {"metric": METRIC, "value": p50m, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean_m, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 V-cycle + f64 CG", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "tol": TOL, "prec": "mixed32", "delta": args.delta, "half_storage": args.half_storage,
                      "smoother": args.smoother, "levels": [l["n"] for l in info],
                      "l2": "flushed before every timed solve (256 MiB write)",
                      "parallelism": "replicas" if ws > 1 else "single GPU"},
           "p50_ms": p50m, "p99_ms": float(np.percentile(tm, 99)), "iters": it_m, "relres": rel_m,
           "status": st_m, "solves_per_s": replica_throughput(ws, p50m), "profiled_p50_ms": float(np.median(tp)),
           "fp64": {"p50_ms": p50d, "p99_ms": float(np.percentile(td, 99)), "iters": it_d, "relres": rel_d,
                    "status": st_d},
           "mixed_speedup_vs_fp64": p50d / p50m,
           "vcycle_fine_gbs": fine_gbs, "vcycle_fine_frac": (fine_gbs / peak) if fine_gbs else None,
           "kernels": kern, "setup_ms": setup_ms,
           "e2e": {"value": p50e, "unit": "ms", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
           "roofline": roof, "gpu_launches": int(launches), "timed_wall_s": t_wall,
           "clocks": clk.summary()}
    traffic_of(roof, n)
    if ws == 1 and not args.no_cpu_baseline:
        cb, x_or = cpu_baseline_sample()
        out["cpu_baseline"] = cb
        href = x_or
        out["rel_err_vs_oracle_at_1e-8"] = float(np.linalg.norm(h_mixed.cpu().numpy() - href) / np.linalg.norm(href))
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_adjoint(args):
    """Secondary workload: adjoint sensitivity at 96^3 (lnK variance 2, correlation
    6 cells, seeds 5/6/7): one step = forward solve (setup included) + backward
    (adjoint solve on the same hierarchy + face-flux gradient kernel)."""
    import torch

    from paper_2001_05798_gb300 import build, gw, workload as wl
    from paper_2001_05798_gb300.adjoint import heads

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    side = 96
    p = wl.heterogeneous_3d(side=side, var=2.0, corr=6.0, seed=5)
    t = wl.heterogeneous_3d(side=side, var=2.0, corr=6.0, seed=6)
    obs = torch.from_numpy(wl.cells(side ** 3, 64, 7).astype(np.int64)).cuda()
    tK = torch.from_numpy(t["Kx"]).cuda()
    bt = torch.empty(side ** 3, dtype=torch.float64, device="cuda")
    At, _ = gw.gw_assemble(side, side, side, tK, tK, tK, t["bct"], t["bcv"], None, b_out=bt)
    ht, _, _, _ = gw.Hierarchy(At).solve(bt, tol=1e-10)
    hobs = ht[obs].contiguous()
    lnK0 = torch.from_numpy(np.log(p["Kx"])).cuda()

    def step():
        lnK = lnK0.clone().requires_grad_(True)
        h = heads(lnK, side, side, side, tol=1e-8)
        J = ((h[obs] - hobs) ** 2).sum()
        J.backward()
        return J, lnK.grad

    for _ in range(max(args.warmup, 3)):
        step()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        J, g = step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    out = {"metric": "adjoint d(head misfit)/d(lnK) per cell, forward + backward ms", "value": float(np.median(times)),
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": float(np.mean(times)), "higher_is_better": False, "dtype": "f32 V-cycle + f64 CG",
           "data": "synthetic", "config": {"workload": "adjoint sensitivity 96^3, lnK var 2 corr 6 seed 5, truth seed 6, "
                                                       "64 observation cells seed 7, tol 1e-8, setup included"},
           "J": float(J.detach()), "grad_norm": float(g.norm())}
    print(json.dumps(out), flush=True)


def run_transient(args):
    """Secondary workload: implicit transient steps (Eq. 2) on the 128^3 field.
    One step = gw_hierarchy_shift + solve.  Small storage terms
    (s = 0.005 C_ii, alternating +-10%) keep the cached aggregates: the first
    step forms the coarse operators for the shift, the later ones keep them and
    refresh level 0; large ones (s = 0.5 C_ii) are far from the built shift and
    rebuild the hierarchy every step.  Reports both step times and outcomes."""
    import torch

    from paper_2001_05798_gb300 import build, gw

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    p = make_problem()
    n = SIDE ** 3
    K = torch.from_numpy(p["Kx"]).cuda()
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(SIDE, SIDE, SIDE, K, K, K, p["bct"], p["bcv"], None, b_out=b)
    rp, ci, v = A.export()
    rows = np.repeat(np.arange(n), np.diff(rp))
    diag = torch.from_numpy(v[rows == ci].copy()).cuda()
    H = gw.Hierarchy(A)
    h = torch.zeros_like(b)
    res = {}
    for name, frac in (("reuse", 0.005), ("rebuild", 0.5)):
        times, rebuilt, outcome = [], [], []
        for k in range(max(args.warmup, 3) + args.steps):
            s = diag * (frac * (1.0 + 0.1 * (k % 2)))
            rhs = b + s * h
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rb = H.shift(s, delta=0.01)
            h, it, rel, st = H.solve(rhs, tol=TOL)
            torch.cuda.synchronize()
            outcome.append(rb)
            if k >= max(args.warmup, 3):
                times.append((time.perf_counter() - t0) * 1e3)
                rebuilt.append(rb == 1)
        res[name] = {"p50_ms": float(np.median(times)), "rebuilt": int(sum(rebuilt)), "steps": len(times),
                     "iters": it, "outcomes": outcome}
    out = {"metric": "implicit transient step (shift + solve) ms, cached vs rebuilt hierarchy",
           "value": res["reuse"]["p50_ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": False, "dtype": "f32 V-cycle + f64 CG", "data": "synthetic",
           "config": {"workload": "128^3 lnK var 4 corr 8 seed 1; s = 0.005 C_ii (reuse, delta 0.01) or 0.5 C_ii "
                                  "(rebuild), alternating +-10%, tol 1e-8"}, "transient": res}
    print(json.dumps(out), flush=True)


def run_setup(args):
    """Secondary workload: the AMG setup alone (strength, MIS-2 aggregation,
    smoothed prolongators, Galerkin products, coarse inverse, cycle storage)
    on the heterogeneous field (lnK var 4, corr 8) for cubes of side 32 to 160,
    the sizes of the serving stream.  One step = gw_amg_setup of the resident
    matrix; the hierarchy is freed after each step (its free is timed apart)."""
    import torch

    from paper_2001_05798_gb300 import build, gw, workload as wl

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    sides = [int(x) for x in args.setup_sides.split(",")]
    res = {}
    for side in sides:
        p = wl.heterogeneous_3d(side=side, var=4.0, corr=8.0, seed=1)
        n = side ** 3
        K = torch.from_numpy(p["Kx"]).cuda()
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        A, _ = gw.gw_assemble(side, side, side, K, K, K, p["bct"], p["bcv"], None, b_out=b)
        torch.cuda.synchronize()
        times, frees = [], []
        for k in range(max(args.warmup, 3) + args.steps):
            t0 = time.perf_counter()
            H = gw.Hierarchy(A)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            levels = [l["n"] for l in H.info()]
            del H
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if k >= max(args.warmup, 3):
                times.append((t1 - t0) * 1e3)
                frees.append((t2 - t1) * 1e3)
        res[str(side)] = {"p50_ms": float(np.median(times)), "min_ms": float(np.min(times)),
                          "free_ms": float(np.median(frees)), "levels": levels}
    big = str(max(sides))
    out = {"metric": "AMG setup ms (gw_amg_setup, mixed form) per cube side", "value": res[big]["p50_ms"],
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "f64 setup", "data": "synthetic",
           "config": {"workload": "cubes of side %s, lnK var 4 corr 8 seed 1, x faces 1/0; value = side %s"
                                  % (args.setup_sides, big)}, "setup": res}
    print(json.dumps(out), flush=True)


def run_many(args):
    """Secondary workload: k = 8 right-hand sides (the benchmark's b and seven
    well scenarios of 6 random wells each, rate U[-1e-3, 1e-3]) on one 128^3
    hierarchy: gw_pcg_solve_many (interleaved block of 8) from device and from
    pinned host buffers, the same columns by k calls of gw_pcg_solve, and
    gw_darcy_flux on the solved heads.  Setup excluded."""
    import torch

    from paper_2001_05798_gb300 import build, gw, workload as wl

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    p = make_problem()
    n, k = SIDE ** 3, 8
    K = torch.from_numpy(p["Kx"]).cuda()
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(SIDE, SIDE, SIDE, K, K, K, p["bct"], p["bcv"], None, b_out=b)
    H = gw.Hierarchy(A)
    rng = np.random.default_rng(11)
    B = b.repeat(k, 1)
    for c in range(1, k):
        B[c, torch.from_numpy(wl.cells(n, 6, 20 + c)).cuda()] += torch.from_numpy(rng.uniform(-1e-3, 1e-3, 6)).cuda()
    X = torch.empty_like(B)
    Bh, Xh = B.cpu().pin_memory(), torch.empty(B.shape, dtype=torch.float64).pin_memory()
    v = [torch.empty(m, dtype=torch.float64, device="cuda") for m in
         ((SIDE + 1) * SIDE * SIDE, SIDE * (SIDE + 1) * SIDE, SIDE * SIDE * (SIDE + 1))]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    res = {}
    for name, (src, dst) in (("device", (B, X)), ("host", (Bh, Xh))):
        times = []
        for s in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, its, rels, st = H.solve_many(src, dst, tol=TOL)
            torch.cuda.synchronize()
            if s >= args.warmup:
                times.append((time.perf_counter() - t0) * 1e3)
        assert st == gw.GW_OK and max(rels) <= TOL
        res[name] = {"p50_ms": float(np.median(times)), "iters": its, "max_relres": max(rels)}
    times = []
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in range(k):
            _, it1, rel1, st1 = H.solve(B[c], X[c], tol=TOL)
        torch.cuda.synchronize()
        if s >= args.warmup:
            times.append((time.perf_counter() - t0) * 1e3)
    res["one_by_one"] = {"p50_ms": float(np.median(times))}
    ftimes = []
    for s in range(args.warmup + args.steps):
        ev[0].record()
        gw.gw_darcy_flux(SIDE, SIDE, SIDE, K, X[0], *v, bct=p["bct"], bcv=p["bcv"])
        ev[1].record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            ftimes.append(ev[0].elapsed_time(ev[1]))
    fms = float(np.median(ftimes))
    fbytes = 8.0 * (2 * n + sum(x.numel() for x in v))  # K and h read once, three face arrays written
    out = {"metric": "right-hand sides per second on one resident hierarchy (gw_pcg_solve_many)",
           "value": k / (res["device"]["p50_ms"] * 1e-3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "dtype": "f32 V-cycle + f64 CG", "data": "synthetic",
           "config": {"workload": "128^3 lnK var 4 corr 8 seed 1; k = 8 right-hand sides (b and 7 six-well "
                                  "scenarios), tol 1e-8, setup excluded, interleaved block of 8"},
           "many": res, "host_solves_per_s": k / (res["host"]["p50_ms"] * 1e-3),
           "one_by_one_solves_per_s": k / (res["one_by_one"]["p50_ms"] * 1e-3),
           "darcy_flux": {"ms": fms, "algorithmic_GBps": fbytes / (fms * 1e-3) / 1e9}}
    print(json.dumps(out), flush=True)


def run_layered(args):
    """Secondary workload: the 256x256x128 layered case (lnK variance 1,
    correlation 32/32/4 cells, Kh/Kv = 10, 16 wells of -1e-3, fixed head on
    top): solve time of the mixed form with the FP32 fine stencil, the mixed
    form with the BF16- and with the FP16-stored fine stencil, and the FP64
    form, each with its
    error against the FP64 form solved to 1e-12 (the oracle comparison of the
    same case is a GPU test).  L2 flushed before every timed solve."""
    import torch

    from paper_2001_05798_gb300 import build, gw, workload as wl

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    stream = torch.cuda.current_stream()
    p = wl.layered_wells_3d()
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    n = nx * ny * nz
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    A, _ = gw.gw_assemble(nx, ny, nz, dv(p["Kx"]), dv(p["Ky"]), dv(p["Kz"]), p["bct"], p["bcv"], dv(p["q"]), b_out=b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    h = torch.empty_like(b)
    forms = {"mixed_fp32_fine": dict(prec=gw.GW_PREC_MIXED32),
             "mixed_bf16_fine": dict(prec=gw.GW_PREC_MIXED32, half_storage=gw.GW_HALF_FINE),
             "mixed_fp16_fine": dict(prec=gw.GW_PREC_MIXED32, half_storage=gw.GW_HALF_FINE16),
             "fp64": dict(prec=gw.GW_PREC_FP64)}
    Href = gw.Hierarchy(A, prec=gw.GW_PREC_FP64)
    href, _, _, _ = Href.solve(b, tol=1e-12)
    del Href
    res = {}
    for name, o in forms.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = gw.Hierarchy(A, **o)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        for _ in range(max(args.warmup, 3)):
            H.solve(b, h, tol=TOL, stream=stream)
        tm, it, rel, st = timed_solves(torch, H, b, h, args.steps, flush, stream)
        err = float(torch.linalg.norm(h - href) / torch.linalg.norm(href))
        res[name] = {"p50_ms": float(np.median(tm)), "p99_ms": float(np.percentile(tm, 99)), "iters": it,
                     "relres": rel, "status": st, "rel_err_vs_fp64_1e-12": err, "setup_ms": setup_ms,
                     "levels": [l["n"] for l in H.info()]}
        del H
    out = {"metric": "AMG-PCG solve ms, 256x256x128 layered anisotropic case with wells, to 1e-8",
           "value": res["mixed_bf16_fine"]["p50_ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": False, "dtype": "bf16-stored fine A, f32 V-cycle + f64 CG",
           "data": "synthetic",
           "config": {"workload": "256x256x128 layered: lnK var 1 corr 32/32/4 seed 2, Kh/Kv 10, 16 wells "
                                  "-1e-3 seed 3, h = 0 on top; tol 1e-8; L2 flushed before every timed solve"},
           "forms": res}
    print(json.dumps(out), flush=True)


def run_baseline(args):
    """Secondary workload: the CPU baseline plan.  For the 128^2 homogeneous,
    the 128^3 sigma^2 = 4 and the 256x256x128 layered cases, the FP64 oracle on
    one host core (assembly, setup and solve timed separately, at tol 1e-8 and
    at the paper's 1e-12) beside the GPU FP64 and mixed forms (p50 of the solve
    with the hierarchy resident, setup timed separately), the iterations, true
    residuals and each GPU form's error against the oracle's 1e-12 solution."""
    import torch

    import oracle
    from paper_2001_05798_gb300 import build, gw, workload as wl

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    oracle.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    cases = {"128x128 homogeneous (2D)": wl.homogeneous_2d_128(),
             "128^3 lnK var 4": wl.heterogeneous_3d(),
             "256x256x128 layered, wells": wl.layered_wells_3d()}
    res = {}
    for name, p in cases.items():
        nx, ny, nz = p["nx"], p["ny"], p["nz"]
        n = nx * ny * nz
        row = {"n": n}
        t0 = time.perf_counter()
        Ao, bo = oracle.assemble(nx, ny, nz, p["Kx"], p["Ky"], p["Kz"], p["bct"], p["bcv"], p["q"])
        row["oracle_assemble_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        Ho = oracle.Hierarchy(Ao)
        row["oracle_setup_ms"] = (time.perf_counter() - t0) * 1e3
        for tol in (1e-8, 1e-12):
            t0 = time.perf_counter()
            ho, it, rel, st = Ho.pcg(bo, tol=tol)
            row["oracle_solve_ms_%g" % tol] = (time.perf_counter() - t0) * 1e3
            row["oracle_iters_%g" % tol] = it
            if tol == 1e-12:
                href = ho
        del Ho, Ao
        dv = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A, _ = gw.gw_assemble(nx, ny, nz, dv(p["Kx"]), dv(p["Ky"]), dv(p["Kz"]), p["bct"], p["bcv"], dv(p["q"]),
                              b_out=b)
        torch.cuda.synchronize()
        row["gpu_assemble_ms"] = (time.perf_counter() - t0) * 1e3
        h = torch.empty_like(b)
        hr = torch.from_numpy(href).cuda()
        forms = (("fp64", gw.GW_PREC_FP64),) if nz == 1 else (("fp64", gw.GW_PREC_FP64), ("mixed", gw.GW_PREC_MIXED32))
        for fname, prec in forms:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = gw.Hierarchy(A, prec=prec)
            torch.cuda.synchronize()
            row["gpu_%s_setup_ms" % fname] = (time.perf_counter() - t0) * 1e3
            for _ in range(max(args.warmup, 3)):
                H.solve(b, h, tol=TOL, stream=stream)
            tm, it, rel, st = timed_solves(torch, H, b, h, args.steps, flush, stream)
            row["gpu_%s_p50_ms" % fname] = float(np.median(tm))
            row["gpu_%s_p99_ms" % fname] = float(np.percentile(tm, 99))
            row["gpu_%s_iters" % fname] = it
            row["gpu_%s_relres" % fname] = rel
            row["gpu_%s_rel_err_vs_oracle_1e-12" % fname] = float(torch.linalg.norm(h - hr) / torch.linalg.norm(hr))
            del H
        res[name] = row
        del A, b, h, hr
    out = {"metric": "CPU baseline plan: FP64 oracle (1 host core) at 1e-8 and 1e-12 beside the GPU FP64 and mixed "
                     "solves", "value": res["128^3 lnK var 4"]["gpu_mixed_p50_ms"], "unit": "ms", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "data": "synthetic",
           "host_cores": os.cpu_count(), "cases": res}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Secondary workload: the serving stream.  Requests with cubic grids of side
    round(exp(U[ln 32, ln 160])), lnK variance U[0.5, 4], correlation length
    U[4, 16] cells, field seed 1000 + r, tol 1e-8, admitted by a 120 GB HBM
    budget.  A closed-loop pass measures the saturated throughput; requests
    then arrive as a Poisson process at 0.7 of it.  Latency = arrival to result."""
    import torch

    from paper_2001_05798_gb300 import build, gw, serve, workload as wl

    torch.cuda.set_device(0)
    build.build()
    gw.load()
    reqs = wl.serving_requests(count=args.requests, seed=4)
    warm = wl.serving_requests(count=8, seed=99)
    if args.serve_mode == "batched":
        srv = serve.BatchedServer(slots=args.slots, setup_workers=args.setup_workers, hbm_budget=120e9)
    else:
        srv = serve.Server(slots=args.slots, hbm_budget=120e9)
    for f in [srv.submit(r) for r in warm]:
        f.result()
    # closed loop: everything queued at once
    nclosed = min(len(reqs), max(16, args.requests // 10))
    t0 = time.perf_counter()
    for f in [srv.submit(r) for r in reqs[:nclosed]]:
        f.result()
    sat = nclosed / (time.perf_counter() - t0)
    rate = 0.7 * sat
    arrivals = wl.poisson_arrivals(len(reqs), rate, seed=4)
    start = time.perf_counter()
    futs = []
    for r, a in zip(reqs, arrivals):
        delay = start + a - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(srv.submit(r, arrival=start + a))
    outs = [f.result() for f in futs]
    wall = max(o["done"] for o in outs) - start
    srv.close()
    lat = np.array([o["latency_s"] for o in outs]) * 1e3
    out = {"metric": "serving stream of flow solves: solves/s and p50/p99 latency", "value": len(outs) / wall,
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32 V-cycle + f64 CG",
           "data": "synthetic", "requests": len(outs), "slots": args.slots, "mode": args.serve_mode,
           "setup_workers": args.setup_workers if args.serve_mode == "batched" else None,
           "config": {"workload": "cubic grids side log-uniform [32,160], lnK var U[0.5,4], corr U[4,16], seed 4, "
                                  "field seed 1000+r, tol 1e-8, Poisson arrivals at 0.7 x closed-loop throughput, "
                                  "HBM budget 120 GB"},
           "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
           "closed_loop_solves_per_s": sat, "arrival_rate": rate, "peak_inflight": srv.peak_inflight,
           "peak_budget_in_use_gb": srv.peak_in_use / 1e9, "mean_iters": float(np.mean([o["iters"] for o in outs])),
           "max_relres": float(max(o["relres"] for o in outs))}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--smoother", choices=("jacobi", "chebyshev"), default="chebyshev")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 arm (profiling runs)")
    ap.add_argument("--delta", type=float, default=0.1, help="reliable-update factor of the mixed form")
    ap.add_argument("--half-storage", type=int, default=0,
                    help="half-precision fine stencil of the mixed form: 2 = BF16 couplings, 4 = scaled FP16")
    ap.add_argument("--side", type=int, default=SIDE, help="grid side for profiling captures (default 128)")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: number of requests")
    ap.add_argument("--slots", type=int, default=16, help="serving workload: solves in flight")
    ap.add_argument("--serve-mode", choices=("batched", "streams"), default="batched",
                    help="serving workload: batched launches over a slot table, or one stream and graph per slot")
    ap.add_argument("--setup-workers", type=int, default=6, help="serving workload, batched: concurrent setups")
    ap.add_argument("--setup-sides", default="32,64,96,128,160", help="setup workload: cube sides")
    ap.add_argument("--workload", choices=("solve", "adjoint", "transient", "serve", "many", "layered", "baseline",
                                           "setup"),
                    default="solve",
                    help="solve: the 128^3 benchmark (default); adjoint: the 96^3 sensitivity case; "
                         "transient: implicit steps with a cached hierarchy; serve: the request stream; "
                         "many: several right-hand sides on one hierarchy, and face fluxes; "
                         "layered: the 256x256x128 case with FP32 and BF16 fine stencils and FP64")
    args = ap.parse_args()
    if args.side != SIDE:
        globals()["SIDE"] = args.side
        args.no_cpu_baseline = True
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "transient":
        run_transient(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "setup":
        run_setup(args)
    elif args.workload == "many":
        run_many(args)
    elif args.workload == "layered":
        run_layered(args)
    elif args.workload == "baseline":
        run_baseline(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
