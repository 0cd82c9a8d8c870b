"""Serving loop for DDM Helmholtz solves on one GPU: continuous batching with HBM-budget admission.

Requests (a workloads.Workload: grid, partition, medium c, sources f with 1..R right-hand
sides) are queued on submit().  A scheduler thread admits queued requests whenever the free
slots and the HBM budget allow: a request's device footprint is the library's own upper bound
(ddm_workspace_bytes) plus its input/output buffers.  Among the queued requests that fit, the
default policy ("hrrn", highest response ratio next) admits the one with the largest
(waiting time + expected service) / expected service, the expected service being the request's
work (grid nodes x right-hand sides) times the seconds per unit of work measured on the
requests completed so far: short requests pass long ones, and a long request's ratio grows
while it waits, so none starves.  Policy "fifo" admits the first that fits in arrival order.  Each
admitted request runs on its own CUDA stream and library context -- set-up, factorisation and
the batched FGMRES solve stay resident on the device until it finishes -- so requests that
arrive while others are running join them and their kernels overlap on the device.  Every
computation is in libddm; this module only schedules.

Latency = completion - submission; p50/p99 latency, queueing time, service time, solves/s and
the peak concurrency come from stats().
"""
from __future__ import annotations

import itertools
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import ddm as D


class Request:
    def __init__(self, rid, wl, tol, K, restart, nbytes):
        self.id = rid
        self.wl = wl
        self.tol = tol
        self.K = K
        self.restart = restart
        self.nbytes = nbytes
        self.t_submit = time.perf_counter()
        self.t_admit: Optional[float] = None
        self.t_done: Optional[float] = None
        self.status = "queued"      # queued | running | done | failed | cancelled
        self.result: Optional[np.ndarray] = None
        self.info: Optional[dict] = None
        self.error: Optional[str] = None


class DDMServer:
    """Continuous-batching server of DDM-FGMRES solves on one device.

    hbm_budget: bytes the admitted requests may hold (default budget_fraction of the free
    device memory at start); max_active: concurrent requests; precision: DDM_MIXED or DDM_FP64.
    """

    def __init__(self, device: int = 0, hbm_budget: Optional[int] = None, budget_fraction: float = 0.8,
                 max_active: int = 8, precision: int = D.DDM_MIXED, K: int = 16, restart: int = 20,
                 max_it: int = 400, keep_results: bool = True, policy: str = "hrrn",
                 collect_timing: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget) if hbm_budget is not None else int(free * budget_fraction)
        self.max_active = int(max_active)
        self.precision = precision
        self.K, self.restart, self.max_it = K, restart, max_it
        self.keep_results = keep_results
        if policy not in ("hrrn", "fifo"):
            raise ValueError("policy must be 'hrrn' or 'fifo'")
        self.policy = policy
        # collect_timing: record each request's kernel times (the library's per-launch CUDA
        # events) and the algorithmic bytes of its local solves in its info dict
        self.collect_timing = collect_timing
        self._rate = 3e-8           # seconds per grid node and right-hand side, updated online
        self._cv = threading.Condition()
        self._queue: List[Request] = []
        self._reqs: Dict[int, Request] = {}
        self._ids = itertools.count(1)
        self._used = 0
        self._active = 0
        self._peak_active = 0
        self._stop = False
        self._threads: List[threading.Thread] = []
        self._sched = threading.Thread(target=self._scheduler, name="ddm-scheduler", daemon=True)
        self._sched.start()

    # ------------------------------------------------------------------ API
    def footprint(self, wl, K=None, restart=None) -> int:
        """Device bytes a request holds while it runs: the library's upper bound for its
        context plus the wave speed, sources and solutions."""
        p, keep = D.params_from(wl, self.precision, max_rhs=wl.nrhs)
        lib_bytes = D.ddm_workspace_bytes(p, self.restart if restart is None else restart)
        io = wl.c.size * 8 + 2 * wl.f.size * 16
        return int(lib_bytes + io)

    def submit(self, wl, tol: float = 1e-6, K: Optional[int] = None, restart: Optional[int] = None) -> int:
        nbytes = self.footprint(wl, K, restart)
        if nbytes > self.budget:
            raise D.DDMError(D.DDM_E_BUDGET, f"request needs {nbytes} bytes, budget is {self.budget}")
        with self._cv:
            rid = next(self._ids)
            req = Request(rid, wl, tol, self.K if K is None else K, self.restart if restart is None else restart,
                          nbytes)
            self._reqs[rid] = req
            self._queue.append(req)
            self._cv.notify_all()
        return rid

    def poll(self, rid: int) -> Request:
        return self._reqs[rid]

    def cancel(self, rid: int) -> bool:
        with self._cv:
            req = self._reqs.get(rid)
            if req is None or req.status != "queued":
                return False
            self._queue.remove(req)
            req.status = "cancelled"
            req.t_done = time.perf_counter()
            self._cv.notify_all()
            return True

    def wait(self, ids=None, timeout: Optional[float] = None) -> bool:
        end = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while True:
                pending = [r for r in (self._reqs.values() if ids is None else (self._reqs[i] for i in ids))
                           if r.status in ("queued", "running")]
                if not pending:
                    return True
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    return False
                self._cv.wait(left)

    def shutdown(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()
        for t in self._threads:
            t.join()

    def stats(self) -> dict:
        done = [r for r in self._reqs.values() if r.status == "done"]
        failed = [r for r in self._reqs.values() if r.status == "failed"]
        if not done:
            return {"completed": 0, "failed": len(failed)}
        lat = np.array([r.t_done - r.t_submit for r in done]) * 1e3
        wait = np.array([r.t_admit - r.t_submit for r in done]) * 1e3
        serv = np.array([r.t_done - r.t_admit for r in done]) * 1e3
        t0 = min(r.t_submit for r in done)
        t1 = max(r.t_done for r in done)
        rhs = sum(r.wl.nrhs for r in done)
        return {"completed": len(done), "failed": len(failed),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_queue_ms": float(wait.mean()), "p99_queue_ms": float(np.percentile(wait, 99)),
                "mean_service_ms": float(serv.mean()),
                "requests_per_s": len(done) / (t1 - t0), "rhs_solves_per_s": rhs / (t1 - t0),
                "peak_active": self._peak_active, "budget_bytes": self.budget}

    # ------------------------------------------------------------------ internals
    @staticmethod
    def work(wl) -> float:
        """A request's work in grid nodes x right-hand sides (its service time is about
        proportional to it at a fixed number of points per wavelength)."""
        return float(np.prod(wl.c.shape)) * max(1, int(wl.nrhs))

    def _pick(self, now: float) -> Optional[Request]:
        """The queued request to admit now (caller holds the lock), or None."""
        fits = [r for r in self._queue if self._used + r.nbytes <= self.budget]
        if not fits:
            return None
        if self.policy == "fifo":
            return fits[0]                   # first fit, in arrival order
        best, best_ratio = None, -1.0
        for r in fits:                       # highest response ratio; ties to the earliest
            est = max(self.work(r.wl) * self._rate, 1e-6)
            ratio = (now - r.t_submit + est) / est
            if ratio > best_ratio:
                best, best_ratio = r, ratio
        return best

    def _scheduler(self):
        with self._cv:
            while not self._stop:
                admitted = None
                if self._active < self.max_active:
                    admitted = self._pick(time.perf_counter())
                if admitted is None:
                    self._cv.wait(0.05)
                    continue
                self._queue.remove(admitted)
                self._used += admitted.nbytes
                self._active += 1
                self._peak_active = max(self._peak_active, self._active)
                admitted.status = "running"
                admitted.t_admit = time.perf_counter()
                t = threading.Thread(target=self._run, args=(admitted,), name=f"ddm-req-{admitted.id}", daemon=True)
                self._threads.append(t)
                t.start()

    def _run(self, req: Request):
        torch = self.torch
        ctx = None
        status, info, error, result = "failed", None, None, None
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
            wl = req.wl
            with torch.cuda.stream(stream):
                c_dev = torch.as_tensor(np.ascontiguousarray(wl.c), dtype=torch.float64, device=self.device)
                f_dev = torch.as_tensor(np.ascontiguousarray(wl.f), dtype=torch.complex128, device=self.device)
                u_dev = torch.zeros(wl.f.shape, dtype=torch.complex128, device=self.device)
                params, keep = D.params_from(wl, self.precision, max_rhs=wl.nrhs)
                ctx = D.ddm_setup(params, wl.omega, c_dev, stream)
                if self.collect_timing:
                    D.ddm_timing(ctx, enable=True, reset=True)
                D.ddm_factor(ctx)
                info = D.ddm_solve(ctx, f_dev, u_dev, nrhs=wl.nrhs, tol=req.tol, max_it=self.max_it,
                                   mode=D.DDM_FGMRES, K=req.K, restart=req.restart, check=True)
                if self.collect_timing:
                    info["kernel_ms"] = D.ddm_timing(ctx, enable=False)
                    per_solve, _ = D.ddm_factor_bytes(ctx)
                    el = 8 if self.precision == D.DDM_MIXED else 16
                    # factor once per sweep pair, source read, t written and read, x written
                    info["local_solve_bytes"] = per_solve + 4 * el * D.ddm_local_layout(ctx)["total"] * wl.nrhs
                if self.keep_results:
                    result = u_dev.cpu().numpy()
                stream.synchronize()
            status = "done"
        except Exception as exc:   # the request fails; the server keeps running
            error = str(exc)
        finally:
            if ctx is not None:
                D.ddm_destroy(ctx)
            with self._cv:          # outcome, completion time and accounting change together
                req.result, req.info, req.error = result, info, error
                req.t_done = time.perf_counter()
                req.status = status
                if status == "done":         # seconds per unit of work, smoothed
                    obs = (req.t_done - req.t_admit) / max(self.work(req.wl), 1.0)
                    self._rate = 0.7 * self._rate + 0.3 * obs
                self._used -= req.nbytes
                self._active -= 1
                self._cv.notify_all()


def request_workload(n: int, nrhs: int, seed: int, sub: int = 64, ppw: float = 10.0):
    """A served request: 2D heterogeneous medium on n^2 (the Gaussian-sum recipe, per-request
    seed), subdomains of `sub` own nodes, omega for `ppw` points per wavelength at c_min,
    nrhs seeded single-node sources."""
    from . import workloads as W
    import math
    ov, npml = 2, 10
    h = 1.0 / n
    e = ov + npml
    c = W.gaussian_sum_medium((n, n), h, e, seed)
    omega = 2 * math.pi * 1.5 / (ppw * h)
    parts = max(1, n // sub)
    f = W.random_point_sources((n, n), h, e, nrhs, seed + 7)
    return W.Workload(f"served-{n}-{nrhs}-{seed}", (n, n), h, (W.uniform_cuts(n, parts),) * 2, ov, npml, 50.0, 2.0,
                      omega, c, f)
