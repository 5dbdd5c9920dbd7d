"""Continuous batching of flow solves on one GPU.

Requests (a grid and a conductivity field) arrive at any time.  The server
keeps `slots` solves in flight, each on its own CUDA stream and host thread
(the C ABI releases the Python lock, so their kernels overlap on the
device), and admits the oldest waiting request as soon as a slot is free and
its estimated device memory fits the HBM budget; a request that does not fit
waits, and nothing behind it overtakes it.  Each request assembles its
system, sets up its own hierarchy (resident for the request's lifetime),
solves with the captured iteration graphs, and releases its memory.  The
graph capture of a request runs while no other slot is inside its torch,
cuFFT or set-up work (a shared/exclusive gate): their allocations and first
kernel launches would invalidate it.  Solves themselves only replay graphs.  All of
it runs in libgw's kernels; results do not depend on what else is running,
because solves share no device state and every reduction has a fixed order.
"""
import collections
import concurrent.futures
import os
import threading
import time

import torch

# Slots capture their CUDA graphs while other slots launch torch and libgw
# kernels.  Under lazy module loading a kernel whose code is loaded during a
# capture on another thread invalidates that capture (libgw loads its own
# kernels outside captures, but torch and cuFFT load theirs on first use), so
# a process that starts serving before it touches CUDA loads modules eagerly.
if not torch.cuda.is_initialized():
    os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")

from . import gw
from . import workload as wl


# the request fields' padded FFT grids are multiples of this many cells per
# axis, so that a stream of many grid sizes reuses a few cuFFT plans (a new
# plan costs tens of milliseconds)
FIELD_PAD = 32


class _SharedExclusive:
    """Many holders of the shared side or one of the exclusive side; a waiting
    exclusive holder keeps new shared holders out."""

    def __init__(self):
        self._cv = threading.Condition()
        self._shared = 0
        self._exclusive = False
        self._waiting = 0

    def acquire_shared(self):
        with self._cv:
            self._cv.wait_for(lambda: not self._exclusive and self._waiting == 0)
            self._shared += 1

    def release_shared(self):
        with self._cv:
            self._shared -= 1
            self._cv.notify_all()

    def acquire_exclusive(self):
        with self._cv:
            self._waiting += 1
            self._cv.wait_for(lambda: not self._exclusive and self._shared == 0)
            self._waiting -= 1
            self._exclusive = True

    def release_exclusive(self):
        with self._cv:
            self._exclusive = False
            self._cv.notify_all()


class Server:
    def __init__(self, slots=4, hbm_budget=120e9, device=0, tol=1e-8, maxit=500, bytes_per_cell=1500.0, **opts):
        self.slots = slots
        self.budget = float(hbm_budget)
        self.device = device
        self.tol, self.maxit, self.opts = tol, maxit, opts
        self.bytes_per_cell = float(bytes_per_cell)
        self.in_use = 0.0
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.closed = False
        self.peak_in_use = 0.0
        self.peak_inflight = 0
        self.inflight = 0
        # graph captures (exclusive) never overlap the slots' torch, cuFFT and
        # set-up work (shared), whose allocations and first kernel launches
        # would invalidate them
        self.capture_gate = _SharedExclusive()
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for t in self.threads:
            t.start()

    def estimate(self, req):
        return self.bytes_per_cell * req["side"] ** 3

    def submit(self, req, arrival=None):
        fut = concurrent.futures.Future()
        with self.cv:
            if self.estimate(req) > self.budget:
                fut.set_exception(MemoryError("request %s needs more than the HBM budget" % req.get("id")))
                return fut
            self.pending.append((req, fut, time.perf_counter() if arrival is None else arrival))
            self.cv.notify_all()
        return fut

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()

    def _admit(self):
        # called with the lock held: the oldest request, if it fits
        while True:
            while self.pending and self.pending[0][1].cancelled():  # cancelled while waiting: dropped
                self.pending.popleft()
            if self.pending:
                req, fut, arr = self.pending[0]
                need = self.estimate(req)
                if need > self.budget:  # the estimate grew past the budget: fail it, do not wait forever
                    self.pending.popleft()
                    fut.set_exception(MemoryError("request %s needs more than the HBM budget" % req.get("id")))
                    continue
                if self.in_use + need <= self.budget:
                    self.pending.popleft()
                    if not fut.set_running_or_notify_cancel():
                        continue
                    self.in_use += need
                    self.inflight += 1
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.peak_inflight = max(self.peak_inflight, self.inflight)
                    return req, fut, arr, need
            elif self.closed:
                return None
            self.cv.wait()

    def _worker(self):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        while True:
            with self.cv:
                item = self._admit()
            if item is None:
                return
            req, fut, arrival, need = item
            try:
                with torch.cuda.stream(stream):
                    out = self._solve(req, stream)
                out["arrival"] = arrival
                out["done"] = time.perf_counter()
                out["latency_s"] = out["done"] - arrival
                fut.set_result(out)
            except Exception as e:  # the request fails alone; the server keeps going
                fut.set_exception(e)
            finally:
                with self.cv:
                    self.in_use -= need
                    self.inflight -= 1
                    self.cv.notify_all()

    def _solve(self, req, stream):
        s = req["side"]
        n = s ** 3
        t0 = time.perf_counter()
        gate = self.capture_gate
        gate.acquire_shared()
        try:
            if "K" in req:
                K = req["K"]
            else:
                K = torch.exp(wl.lnk_field_device(s, s, s, req["var"], req["corr"], req["seed"], pad=FIELD_PAD))
            b = torch.empty(n, dtype=torch.float64, device=K.device)
            A, _ = gw.gw_assemble(s, s, s, K, K, K, (1, 1, 0, 0, 0, 0), (1.0, 0.0, 0, 0, 0, 0), None, b_out=b,
                                  stream=stream)
            H = gw.Hierarchy(A, stream=stream, **self.opts)
            h = torch.empty_like(b)
            stream.synchronize()
        finally:
            gate.release_shared()
        used = sum(l["bytes"] for l in H.info()) + 16 * n
        with self.cv:
            self.bytes_per_cell = max(self.bytes_per_cell, 1.25 * used / n)
        gate.acquire_exclusive()
        try:
            H.prepare()
        finally:
            gate.release_exclusive()
        t1 = time.perf_counter()
        _, it, rel, st = H.solve(b, h, tol=self.tol, maxit=self.maxit, stream=stream)
        t2 = time.perf_counter()
        if st != gw.GW_OK:
            raise gw.GwError(st, "request %s: relres %.3e after %d iterations" % (req.get("id"), rel, it))
        gate.acquire_shared()
        try:
            del H, A
        finally:
            gate.release_shared()
        return dict(id=req.get("id"), n=n, h=h, iters=it, relres=rel, setup_s=t1 - t0, solve_s=t2 - t1)


class BatchedServer:
    """Continuous batching with batched launches.

    Setup workers (each on its own stream) draw a request's field, assemble
    it and set up its hierarchy; a finished setup waits in a ready queue.  One
    batch thread admits ready solves into free slots of a gw_batch, replays
    the batched CG iteration (one launch per pass for every solve in flight)
    and hands finished solves back, so requests of different sizes share
    every launch of the iteration.  Admission to setup is FIFO by the HBM
    budget, as in Server; a request holds its budget from the start of its
    setup to the end of its solve.  A request whose future is cancelled while
    it still waits is dropped at admission (a running one can no longer be
    cancelled).  Results are the same bit for bit as the request's solve alone
    in a batch."""

    def __init__(self, slots=8, setup_workers=4, hbm_budget=120e9, device=0, tol=1e-8, maxit=500,
                 bytes_per_cell=1500.0, iterations_per_step=2, **opts):
        self.slots = slots
        self.budget = float(hbm_budget)
        self.device = device
        self.tol, self.maxit, self.opts = tol, maxit, opts
        self.bytes_per_cell = float(bytes_per_cell)
        self.k = iterations_per_step
        self.in_use = 0.0
        self.pending = collections.deque()
        self.ready = collections.deque()
        self.cv = threading.Condition()
        self.closed = False
        self.peak_in_use = 0.0
        self.peak_inflight = 0
        self.inflight = 0
        self.capture_gate = _SharedExclusive()
        self.graph_levels = 0  # depth of the batched graph captured so far
        torch.cuda.set_device(device)
        self.batch = gw.Batch(slots)
        self.setups = [threading.Thread(target=self._setup_worker, daemon=True) for _ in range(setup_workers)]
        self.runner = threading.Thread(target=self._batch_loop, daemon=True)
        for t in self.setups:
            t.start()
        self.runner.start()

    def estimate(self, req):
        return self.bytes_per_cell * req["side"] ** 3

    def submit(self, req, arrival=None):
        fut = concurrent.futures.Future()
        with self.cv:
            if self.estimate(req) > self.budget:
                fut.set_exception(MemoryError("request %s needs more than the HBM budget" % req.get("id")))
                return fut
            self.pending.append((req, fut, time.perf_counter() if arrival is None else arrival))
            self.cv.notify_all()
        return fut

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.setups:
            t.join()
        self.runner.join()
        self.batch.close()

    def _release(self, need):
        with self.cv:
            self.in_use -= need
            self.inflight -= 1
            self.cv.notify_all()

    def _admit_setup(self):
        # with the lock held: the oldest request, if it fits the budget
        while True:
            while self.pending and self.pending[0][1].cancelled():
                self.pending.popleft()
            if self.pending:
                req, fut, arr = self.pending[0]
                need = self.estimate(req)
                if need > self.budget:
                    self.pending.popleft()
                    fut.set_exception(MemoryError("request %s needs more than the HBM budget" % req.get("id")))
                    continue
                if self.in_use + need <= self.budget:
                    self.pending.popleft()
                    if not fut.set_running_or_notify_cancel():
                        continue
                    self.in_use += need
                    self.inflight += 1
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.peak_inflight = max(self.peak_inflight, self.inflight)
                    return req, fut, arr, need
            elif self.closed:
                return None
            self.cv.wait()

    def _setup_worker(self):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        while True:
            with self.cv:
                item = self._admit_setup()
            if item is None:
                return
            req, fut, arrival, need = item
            try:
                s = req["side"]
                n = s ** 3
                t0 = time.perf_counter()
                self.capture_gate.acquire_shared()
                try:
                    with torch.cuda.stream(stream):
                        if "K" in req:
                            K = req["K"]
                        else:
                            K = torch.exp(wl.lnk_field_device(s, s, s, req["var"], req["corr"], req["seed"],
                                                              pad=FIELD_PAD))
                        b = torch.empty(n, dtype=torch.float64, device=K.device)
                        A, _ = gw.gw_assemble(s, s, s, K, K, K, (1, 1, 0, 0, 0, 0), (1.0, 0.0, 0, 0, 0, 0), None,
                                              b_out=b, stream=stream)
                        H = gw.Hierarchy(A, stream=stream, **self.opts)
                        h = torch.empty_like(b)
                    stream.synchronize()
                finally:
                    self.capture_gate.release_shared()
                info = H.info()
                used = sum(l["bytes"] for l in info) + 16 * n
                with self.cv:
                    self.bytes_per_cell = max(self.bytes_per_cell, 1.25 * used / n)
                    self.ready.append(dict(req=req, fut=fut, arrival=arrival, need=need, H=H, A=A, b=b, h=h, n=n,
                                           L=len(info), setup_s=time.perf_counter() - t0))
                    self.cv.notify_all()
            except Exception as e:  # the request fails alone
                fut.set_exception(e)
                self._release(need)

    def _finish(self, job, slot):
        _, it, rel, st = self.batch.take(slot, job["h"])  # returns with the batch's stream synchronised
        done = time.perf_counter()
        self.capture_gate.acquire_shared()
        try:
            del job["H"], job["A"]
        finally:
            self.capture_gate.release_shared()
        if st != gw.GW_OK:
            job["fut"].set_exception(gw.GwError(st, "request %s: relres %.3e after %d iterations"
                                                % (job["req"].get("id"), rel, it)))
        else:
            job["fut"].set_result(dict(id=job["req"].get("id"), n=job["n"], h=job["h"], iters=it, relres=rel,
                                       setup_s=job["setup_s"], solve_s=done - job["start"], arrival=job["arrival"],
                                       done=done, latency_s=done - job["arrival"]))
        self._release(job["need"])

    def _batch_loop(self):
        torch.cuda.set_device(self.device)
        running = {}  # slot -> job
        while True:
            with self.cv:
                while not self.ready and not running and not (self.closed and not self.inflight):
                    self.cv.wait()
                if self.closed and not self.inflight and not self.ready and not running:
                    return
                joining = []
                while self.ready and len(running) + len(joining) < self.slots:
                    joining.append(self.ready.popleft())
            for job in joining:
                # an add captures the batched graph again only for a hierarchy deeper
                # than every one before it: only then must the setup workers pause
                capture = job["L"] > self.graph_levels
                if capture:
                    self.capture_gate.acquire_exclusive()
                try:
                    slot = self.batch.add(job["H"], job["b"], tol=self.tol, maxit=self.maxit)
                    self.graph_levels = max(self.graph_levels, job["L"])
                except Exception as e:
                    job["fut"].set_exception(e)
                    self._release(job["need"])
                    continue
                finally:
                    if capture:
                        self.capture_gate.release_exclusive()
                job["start"] = time.perf_counter()
                running[slot] = job
            if running:
                self.batch.run(self.k)
                for slot in [s for s in list(running) if self.batch.state(s) == 2]:
                    self._finish(running.pop(slot), slot)
