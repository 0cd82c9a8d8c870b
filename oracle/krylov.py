"""Flexible GMRES right-preconditioned by K DDM steps (oracle, FP64).

Test infrastructure: see the package docstring.

Section 4.2.2 uses Algorithm 3.1 as a preconditioner of flexible GMRES with K
DDM steps per application and reports the GMRES iteration count.  The paper
gives no further detail; the readings used here:
x_0 = 0, restart length m, classical Gram-Schmidt applied twice (CGS2) for the
Arnoldi step, Givens rotations for the least-squares problem, and the stop
test |g_{j+1}| / ||b|| <= tol on the least-squares residual estimate.
"""
from __future__ import annotations

from typing import Callable, Dict, List

import numpy as np


def fgmres(apply_A: Callable[[np.ndarray], np.ndarray], apply_M: Callable[[np.ndarray], np.ndarray],
           b: np.ndarray, tol: float, restart: int, max_it: int) -> Dict:
    """Solve A x = b with right-preconditioned flexible GMRES(restart).

    apply_M may change from one call to the next (flexible: the preconditioned
    vectors z_j are stored).  Returns x, the iteration count, the history of
    residual estimates |g_{j+1}| / ||b|| and whether tol was met.
    """
    shape = b.shape
    bv = b.ravel().astype(np.complex128)
    N = bv.size
    bnorm = np.linalg.norm(bv)
    x = np.zeros(N, dtype=np.complex128)
    hist: List[float] = []
    it = 0
    if bnorm == 0.0:
        return {"x": x.reshape(shape), "iters": 0, "history": hist, "converged": True}
    converged = False
    while it < max_it and not converged:
        r = bv - apply_A(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            converged = True
            break
        m = restart
        V = np.zeros((m + 1, N), dtype=np.complex128)
        Z = np.zeros((m, N), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)     # Givens cosines (real-valued, kept complex)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = apply_M(V[j].reshape(shape)).ravel()
            w = apply_A(Z[j].reshape(shape)).ravel()
            # classical Gram-Schmidt, twice
            h = np.zeros(j + 1, dtype=np.complex128)
            for _ in range(2):
                c = V[: j + 1].conj() @ w
                w = w - V[: j + 1].T @ c
                h += c
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            # apply earlier rotations, then build the new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(a) == 0:
                cs[j], sn[j] = 0.0, np.conj(bb) / abs(bb)
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(bb) / den
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hist[-1] <= tol or it >= max_it:
                break
        # least squares: H[:j,:j] y = g[:j] (upper triangular)
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: j_done] @ y[i + 1: j_done]) / H[i, i]
        x = x + Z[:j_done].T @ y
        if hist and hist[-1] <= tol:
            converged = True
    return {"x": x.reshape(shape), "iters": it, "history": hist, "converged": converged}


def ddm_fgmres(oracle, b: np.ndarray, K: int, tol: float, restart: int, max_it: int) -> Dict:
    """FGMRES on the global truncated system preconditioned by M_K (Section 4.2.2)."""
    return fgmres(oracle.apply_global, lambda v: oracle.precondition(v, K), b, tol, restart, max_it)


def ddm_stepping(oracle, b: np.ndarray, tol: float, max_steps: int) -> Dict:
    """Algorithm 3.1 as an iterative solver (Section 4.2.1): keep stepping until the
    relative residual ||b - A w_s|| / ||b|| of the assembled solution is <= tol.

    The residual is taken on the own regions from the last steps' transfers
    (DDMOracle.strip_residual), which equals b - A w_s exactly."""
    bnorm = np.linalg.norm(b)
    hist: List[float] = []

    def cb(s, h, U):
        r2 = sum(np.linalg.norm(oracle.strip_residual(R, s, h)) ** 2 for R in oracle.subs)
        hist.append(float(np.sqrt(r2)) / bnorm)
        return hist[-1] <= tol

    res = oracle.run(b, max_steps, callback=cb)
    return {"w": res["w"], "steps": res["steps"], "history": hist,
            "converged": bool(hist and hist[-1] <= tol)}
