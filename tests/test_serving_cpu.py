"""Host logic of the serving loop, on the CPU: admission by HBM budget and free slots (first fit
in arrival order), the budget and slot accounting across completions and failures, cancellation
of queued requests, refusal of a request larger than the budget, and the latency statistics.

The server's device work is replaced by host fakes (library calls that block until the test
releases them, or raise); the scheduler and the request runner are the server's own code.
"""
import contextlib
import itertools
import threading
import time
import types

import numpy as np
import pytest

from paper_1807_04180_gb300 import ddm as D
from paper_1807_04180_gb300 import serving as S


class FakeWorkload:
    def __init__(self, nbytes, nrhs=1, fail=False, n=4):
        self.nbytes = nbytes
        self.nrhs = nrhs
        self.fail = fail
        self.omega = 1.0
        self.c = np.zeros((n, n))
        self.f = np.zeros((nrhs, n, n), dtype=complex)


def fake_torch():
    cuda = types.SimpleNamespace(
        set_device=lambda dev: None,
        Stream=lambda dev: types.SimpleNamespace(synchronize=lambda: None),
        stream=lambda s: contextlib.nullcontext())
    return types.SimpleNamespace(cuda=cuda, float64=np.float64, complex128=np.complex128,
                                 as_tensor=lambda a, dtype=None, device=None: np.asarray(a),
                                 zeros=lambda shape, dtype=None, device=None: FakeTensor(np.zeros(shape, dtype=complex)))


class FakeTensor:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class Harness:
    """A DDMServer with host fakes for the device: each request's factorisation blocks on a
    per-request event; `running` records the admitted workloads in admission order."""

    def __init__(self, monkeypatch, budget, max_active, policy="fifo"):
        self.release = {}
        self.running = []
        self.lock = threading.Lock()
        self.peak_used = 0
        srv = object.__new__(S.DDMServer)
        srv.torch = fake_torch()
        srv.device = "cpu"
        srv.budget = budget
        srv.max_active = max_active
        srv.precision = D.DDM_MIXED
        srv.K, srv.restart, srv.max_it = 16, 20, 10
        srv.keep_results = True
        srv.collect_timing = False
        srv.policy = policy
        srv._rate = 3e-8
        srv._cv = threading.Condition()
        srv._queue = []
        srv._reqs = {}
        srv._ids = itertools.count(1)
        srv._used = 0
        srv._active = 0
        srv._peak_active = 0
        srv._stop = False
        srv._threads = []
        srv.footprint = lambda wl, K=None, restart=None: wl.nbytes
        self.srv = srv

        def setup(params, omega, c, stream):
            return params

        def factor(ctx):
            wl = ctx
            with self.lock:
                self.running.append(wl)
                self.peak_used = max(self.peak_used, srv._used)
            assert self.release[id(wl)].wait(10.0), "test did not release the request"
            if wl.fail:
                raise D.DDMError(D.DDM_E_SINGULAR, "planted failure")

        monkeypatch.setattr(S.D, "params_from", lambda wl, prec, max_rhs=1: (wl, None))
        monkeypatch.setattr(S.D, "ddm_setup", setup)
        monkeypatch.setattr(S.D, "ddm_factor", factor)
        monkeypatch.setattr(S.D, "ddm_solve", lambda ctx, f, u, **kw: {"iters": 1, "rel_residual": 0.0})
        monkeypatch.setattr(S.D, "ddm_destroy", lambda ctx: None)
        srv._sched = threading.Thread(target=srv._scheduler, daemon=True)
        srv._sched.start()

    def submit(self, wl):
        self.release[id(wl)] = threading.Event()
        return self.srv.submit(wl)

    def wait_running(self, n, timeout=5.0):
        end = time.perf_counter() + timeout
        while time.perf_counter() < end:
            with self.lock:
                if len(self.running) >= n:
                    return True
            time.sleep(0.005)
        return False


def test_admission_first_fit_budget_and_slots(monkeypatch):
    h = Harness(monkeypatch, budget=100, max_active=2)
    big, mid, small, tail = FakeWorkload(70), FakeWorkload(60), FakeWorkload(30), FakeWorkload(20)
    ids = [h.submit(w) for w in (big, mid, small, tail)]
    # big (70) is admitted; mid (60) does not fit beside it, small (30) does (first fit);
    # then the slot limit (2) holds tail back although it fits the budget
    assert h.wait_running(2)
    time.sleep(0.1)
    assert h.running == [big, small]
    assert h.srv._used == 100 and h.srv._active == 2
    assert h.srv.poll(ids[1]).status == "queued" and h.srv.poll(ids[3]).status == "queued"
    # big finishes: mid (60) fits beside small (30) and arrived before tail
    h.release[id(big)].set()
    assert h.wait_running(3)
    time.sleep(0.1)
    assert h.running[2] is mid and h.srv.poll(ids[3]).status == "queued"
    for w in (small, mid, tail):
        h.release[id(w)].set()
    assert h.srv.wait(timeout=5.0)
    assert [h.srv.poll(i).status for i in ids] == ["done"] * 4
    assert h.srv._used == 0 and h.srv._active == 0
    assert h.peak_used <= 100 and h.srv._peak_active == 2
    st = h.srv.stats()
    assert st["completed"] == 4 and st["failed"] == 0
    assert 0 <= st["p50_ms"] <= st["p99_ms"]
    h.srv.shutdown()


def test_failed_request_releases_its_budget_and_slot(monkeypatch):
    h = Harness(monkeypatch, budget=100, max_active=1)
    bad, good = FakeWorkload(80, fail=True), FakeWorkload(80)
    i_bad, i_good = h.submit(bad), h.submit(good)
    assert h.wait_running(1)
    h.release[id(bad)].set()           # the factorisation raises inside the request's thread
    assert h.wait_running(2)           # the server keeps running and admits the next request
    assert h.srv.poll(i_bad).status == "failed" and "planted failure" in h.srv.poll(i_bad).error
    h.release[id(good)].set()
    assert h.srv.wait(timeout=5.0)
    assert h.srv.poll(i_good).status == "done" and h.srv.poll(i_good).result is not None
    assert h.srv._used == 0 and h.srv._active == 0
    st = h.srv.stats()
    assert st["completed"] == 1 and st["failed"] == 1
    h.srv.shutdown()


def test_cancel_queued_and_refuse_oversized(monkeypatch):
    h = Harness(monkeypatch, budget=100, max_active=1)
    first, queued = FakeWorkload(50), FakeWorkload(50)
    i1, i2 = h.submit(first), h.submit(queued)
    assert h.wait_running(1)
    assert h.srv.cancel(i2) is True            # still queued: cancelled
    assert h.srv.cancel(i1) is False           # running: not cancellable
    assert h.srv.poll(i2).status == "cancelled"
    with pytest.raises(D.DDMError) as exc:
        h.submit(FakeWorkload(101))            # larger than the whole budget
    assert exc.value.status == D.DDM_E_BUDGET
    h.release[id(first)].set()
    assert h.srv.wait(timeout=5.0)
    time.sleep(0.05)
    assert h.running == [first]                # the cancelled request never ran
    assert h.srv._used == 0
    h.srv.shutdown()


def _policy_server(policy, rate=1e-6, budget=100):
    srv = object.__new__(S.DDMServer)
    srv.policy, srv._rate, srv.budget, srv._used, srv._queue = policy, rate, budget, 0, []
    return srv


def _queued(srv, wl, waited_s, now):
    r = S.Request(len(srv._queue) + 1, wl, 1e-6, 16, 20, wl.nbytes)
    r.t_submit = now - waited_s
    srv._queue.append(r)
    return r


def test_hrrn_admits_short_requests_first_and_ages_long_ones():
    now = 1000.0
    # work = nodes x rhs: big 400^2 x 16 = 2.56e6 (est 2.56 s at 1e-6 s per unit), small 16 (est 16 us)
    srv = _policy_server("hrrn")
    big = _queued(srv, FakeWorkload(10, nrhs=16, n=400), waited_s=1.0, now=now)
    small = _queued(srv, FakeWorkload(10, n=4), waited_s=0.5, now=now)
    assert srv._pick(now) is small              # arrived later, but its ratio is far higher
    fifo = _policy_server("fifo")
    fifo._queue = list(srv._queue)
    assert fifo._pick(now) is big               # arrival order
    # aging: once the long request has waited many times its expected service, it goes first
    srv2 = _policy_server("hrrn")
    old = _queued(srv2, FakeWorkload(10, nrhs=16, n=400), waited_s=60.0, now=now)   # ratio ~24
    new = _queued(srv2, FakeWorkload(10, nrhs=1, n=100), waited_s=0.0, now=now)      # ratio 1
    assert srv2._pick(now) is old
    # the budget still applies: a request that does not fit is skipped
    srv3 = _policy_server("hrrn", budget=50)
    _queued(srv3, FakeWorkload(60, n=4), waited_s=5.0, now=now)
    fit = _queued(srv3, FakeWorkload(40, n=400), waited_s=0.0, now=now)
    assert srv3._pick(now) is fit
    srv3._queue = srv3._queue[:1]
    assert srv3._pick(now) is None


def test_hrrn_server_runs_every_request_and_learns_its_rate(monkeypatch):
    h = Harness(monkeypatch, budget=100, max_active=1, policy="hrrn")
    first = FakeWorkload(10, n=4)
    big, small = FakeWorkload(10, nrhs=16, n=400), FakeWorkload(10, n=4)
    i1 = h.submit(first)
    assert h.wait_running(1)
    ib, i_s = h.submit(big), h.submit(small)
    rate0 = h.srv._rate
    h.release[id(first)].set()
    assert h.wait_running(2)
    assert h.running[1] is small                # the short request passes the long one
    h.release[id(small)].set()
    h.release[id(big)].set()
    assert h.srv.wait(timeout=5.0)
    assert [h.srv.poll(i).status for i in (i1, ib, i_s)] == ["done"] * 3
    assert h.srv._rate != rate0                 # updated from the completed requests
    h.srv.shutdown()
