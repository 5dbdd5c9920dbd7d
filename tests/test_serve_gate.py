"""Host logic of the serving loop's capture gate, on the CPU.

A graph capture must not overlap another slot's torch, cuFFT or set-up work:
the server holds a shared side for that work and an exclusive side for the
capture.  These tests drive the gate with plain threads: shared holders run
together, an exclusive holder runs alone, and a waiting exclusive holder is
not starved by a stream of new shared holders.
"""
import threading
import time

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gate_cls():
    from paper_2001_05798_gb300 import serve

    return serve._SharedExclusive


def test_shared_holders_overlap(gate_cls):
    g = gate_cls()
    inside, peak, lock = [0], [0], threading.Lock()

    def work():
        g.acquire_shared()
        with lock:
            inside[0] += 1
            peak[0] = max(peak[0], inside[0])
        time.sleep(0.05)
        with lock:
            inside[0] -= 1
        g.release_shared()

    ts = [threading.Thread(target=work) for _ in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert peak[0] >= 2


def test_exclusive_holder_runs_alone(gate_cls):
    g = gate_cls()
    log, lock = [], threading.Lock()

    def shared(i):
        g.acquire_shared()
        with lock:
            log.append(("s+", i))
        time.sleep(0.02)
        with lock:
            log.append(("s-", i))
        g.release_shared()

    def exclusive(i):
        g.acquire_exclusive()
        with lock:
            log.append(("x+", i))
        time.sleep(0.02)
        with lock:
            log.append(("x-", i))
        g.release_exclusive()

    ts = [threading.Thread(target=shared if k % 3 else exclusive, args=(k,)) for k in range(12)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    active_shared, active_x = 0, 0
    for kind, _ in log:
        if kind == "s+":
            assert active_x == 0
            active_shared += 1
        elif kind == "s-":
            active_shared -= 1
        elif kind == "x+":
            assert active_x == 0 and active_shared == 0
            active_x += 1
        else:
            active_x -= 1
    assert active_shared == 0 and active_x == 0


def test_waiting_exclusive_is_not_starved(gate_cls):
    g = gate_cls()
    stop = threading.Event()
    got = threading.Event()

    def churn():
        while not stop.is_set():
            g.acquire_shared()
            time.sleep(0.005)
            g.release_shared()

    ts = [threading.Thread(target=churn) for _ in range(4)]
    for t in ts:
        t.start()
    time.sleep(0.02)

    def capture():
        g.acquire_exclusive()
        got.set()
        g.release_exclusive()

    c = threading.Thread(target=capture)
    c.start()
    ok = got.wait(timeout=5.0)
    stop.set()
    for t in ts + [c]:
        t.join()
    assert ok


@pytest.mark.parametrize("cls_name", ["Server", "BatchedServer"])
def test_cancelled_requests_are_dropped_at_admission(cls_name):
    """A request whose future is cancelled while it waits never takes budget
    or a slot; the requests around it are admitted in order."""
    import collections
    import concurrent.futures

    from paper_2001_05798_gb300 import serve

    cls = getattr(serve, cls_name)
    s = cls.__new__(cls)  # the admission logic only, without devices or threads
    s.cv = threading.Condition()
    s.pending = collections.deque()
    s.budget, s.in_use, s.bytes_per_cell = 1e12, 0.0, 1.0
    s.inflight = s.peak_inflight = 0
    s.peak_in_use = 0.0
    s.closed = False
    futs = [concurrent.futures.Future() for _ in range(4)]
    for k, f in enumerate(futs):
        s.pending.append(({"id": k, "side": 4}, f, 0.0))
    assert futs[1].cancel() and futs[2].cancel()
    admit = s._admit if cls_name == "Server" else s._admit_setup
    with s.cv:
        a = admit()
        b = admit()
    assert [a[0]["id"], b[0]["id"]] == [0, 3]
    assert futs[0].running() and futs[3].running()
    assert s.inflight == 2 and s.in_use == 2 * 64.0 and not s.pending
    s.closed = True
    with s.cv:
        assert admit() is None


def test_batched_admission_takes_the_exclusive_side_only_to_recapture(monkeypatch):
    """The batch thread makes the setup workers pause (the exclusive side of
    the gate) only for an admission whose hierarchy is deeper than any the
    batched graph was captured for: only such an add captures again.  A
    failed add fails its request alone and leaves the captured depth as it
    was.  Driven on the CPU with a stand-in batch."""
    import collections
    import concurrent.futures

    from paper_2001_05798_gb300 import serve

    monkeypatch.setattr(serve.torch.cuda, "set_device", lambda d: None)

    class Gate:
        def __init__(self):
            self.log = []

        def acquire_exclusive(self):
            self.log.append("x+")

        def release_exclusive(self):
            self.log.append("x-")

        def acquire_shared(self):
            pass

        def release_shared(self):
            pass

    class Batch:
        def __init__(self):
            self.state_of, self.next, self.order = {}, 0, []

        def add(self, H, b, tol, maxit):
            if H == "bad":
                raise RuntimeError("refused")
            s = self.next
            self.next += 1
            self.state_of[s] = 2  # finished at the next look
            self.order.append(H)
            return s

        def run(self, k):
            pass

        def state(self, s):
            return self.state_of.get(s, 0)

        def take(self, s, h):
            del self.state_of[s]
            return h, 7, 1e-9, 0

    s = serve.BatchedServer.__new__(serve.BatchedServer)
    s.cv = threading.Condition()
    s.ready = collections.deque()
    s.closed = True
    s.slots, s.k, s.tol, s.maxit, s.device = 2, 1, 1e-8, 100, 0
    s.capture_gate = Gate()
    s.graph_levels = 0
    s.batch = Batch()
    depths = [3, 3, 4, 2, 4, 6, 5]
    names = ["h%d" % k for k in range(len(depths))]
    names[5] = "bad"
    futs = []
    for k, (L, H) in enumerate(zip(depths, names)):
        f = concurrent.futures.Future()
        f.set_running_or_notify_cancel()
        futs.append(f)
        s.ready.append(dict(req={"id": k}, fut=f, arrival=0.0, need=1.0, H=H, A=None, b=None, h=None, n=8, L=L,
                            setup_s=0.0))
    s.in_use, s.inflight = float(len(depths)), len(depths)
    s._batch_loop()
    # exclusive only for depths 3 (first capture), 4 and 6 (refused: its try still held the side), then 5
    assert s.capture_gate.log == ["x+", "x-"] * 4
    assert s.batch.order == ["h0", "h1", "h2", "h3", "h4", "h6"]
    assert s.graph_levels == 5 and s.inflight == 0 and s.in_use == 0.0
    assert isinstance(futs[5].exception(), RuntimeError)
    assert all(f.result()["iters"] == 7 for k, f in enumerate(futs) if k != 5)
