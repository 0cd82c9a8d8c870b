"""Additive overlapping DDM, Algorithm 3.1 of Leng & Ju (2018) (oracle, FP64).

Test infrastructure: see the package docstring.

Indexing.  Arrays are C ordered; "axis a" is an array axis (the physical x is
the last one).  Global node p along an axis runs over -e .. n+e-1 and sits at
array index p + e of the global extended grid.  A subdomain R has index tuple
(i_0, .., i_{d-1}), own nodes [lo_a, hi_a) = [cuts_a[i_a], cuts_a[i_a+1]) and
the extended node range [lo_a - e, hi_a + e), i.e. the global array window
[lo_a, hi_a + 2e).

Readings of the paper taken here (where it is silent, ambiguous or garbled):
  * cut-offs: beta_0(t) = 1 - (10 t^3 - 15 t^4 + 6 t^5) on [0, 1], clamped
    (C^2, monotone, 1 for t <= 0, 0 for t >= 1, as Section 2.2 requires); a
    node q = 0, 1, .. nodes beyond a face (q = 0: first node outside) gets
    beta_0(q / ov), so beta = 1 on the own box plus one stencil layer;
  * transfer receivers: the characteristic function is always the receiver's
    side of the shared interface(s) (the printed indices of chi for the
    left/down/corner directions are off by one relative to the right/up ones);
  * lags: a direction with m non-zero components uses u^{s-m} (faces 1,
    corners/edges 2, 3D vertices 3), Eq. (38) in 2D;
  * the iteration continues past N1+N2(+N3) steps with the same recurrence;
  * a subdomain's source f_ij is the global right-hand side on its "own
    region": its own box, continued through the global extension band on the
    sides where it touches the global boundary (these regions partition the
    global extended grid).
"""
from __future__ import annotations

import itertools
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse.linalg as spla

from .pml_operator import box_alpha, jacobian, pml_operator


def beta0(t) -> np.ndarray:
    """The cut-off profile beta_0 of Section 2.2: C^2, monotone, 1 (t<=0) -> 0 (t>=1)."""
    t = np.clip(np.asarray(t, dtype=np.float64), 0.0, 1.0)
    return 1.0 - (10 * t ** 3 - 15 * t ** 4 + 6 * t ** 5)


def directions(dim: int) -> List[Tuple[int, ...]]:
    """The 3^d - 1 transfer directions (8 in 2D, 26 in 3D; Section 2.2, Remark after Alg. 3.1)."""
    return [d for d in itertools.product((-1, 0, 1), repeat=dim) if any(d)]


def lag(d: Sequence[int]) -> int:
    """Step lag of direction d: number of non-zero components (Eq. (38))."""
    return sum(1 for x in d if x != 0)


class DDMOracle:
    """The truncated PML problem on a structured overlapping partition.

    Parameters mirror Section 3.1 / 4: n interior nodes per axis, spacing h,
    partition cuts per axis, overlap ov cells (d~ = ov h), npml PML cells,
    profile sigma0 ((t-ov)/npml)^power, angular frequency omega and the wave
    speed c on the global extended grid (k = omega / c, Section 1).
    """

    def __init__(self, n: Sequence[int], h: float, cuts: Sequence[Sequence[int]], ov: int, npml: int,
                 sigma0: float, power: float, omega: float, c: np.ndarray, workers: int = 1):
        self.n = tuple(int(x) for x in n)
        self.dim = len(self.n)
        self.h = float(h)
        self.cuts = [np.asarray(cu, dtype=np.int64) for cu in cuts]
        self.parts = tuple(len(cu) - 1 for cu in self.cuts)
        self.ov, self.npml = int(ov), int(npml)
        self.e = self.ov + self.npml
        self.sigma0, self.power, self.omega = float(sigma0), float(power), float(omega)
        self.gshape = tuple(m + 2 * self.e for m in self.n)
        c = np.asarray(c, dtype=np.float64)
        assert c.shape == self.gshape, (c.shape, self.gshape)
        self.k2 = (self.omega / c) ** 2
        self.workers = int(workers)
        for a in range(self.dim):
            cu = self.cuts[a]
            assert cu[0] == 0 and cu[-1] == self.n[a] and np.all(np.diff(cu) >= 1)
        # the global truncated problem (Section 3.1)
        ga = [box_alpha(0, self.n[a], self.e, self.ov, self.npml, self.sigma0, self.power)
              for a in range(self.dim)]
        self.A_global = pml_operator([g[0] for g in ga], [g[1] for g in ga], self.k2, self.h)
        self.J_global = jacobian([g[0] for g in ga], self.gshape)
        self._glu = None
        # subdomain problems P^_{Omega_ij} (Algorithm 3.1)
        self.subs = list(itertools.product(*[range(p) for p in self.parts]))
        self.sub_A, self.sub_lu, self.sub_win, self.sub_shape = {}, {}, {}, {}
        for R in self.subs:
            lo = [int(self.cuts[a][R[a]]) for a in range(self.dim)]
            hi = [int(self.cuts[a][R[a] + 1]) for a in range(self.dim)]
            win = tuple(slice(lo[a], hi[a] + 2 * self.e) for a in range(self.dim))
            al = [box_alpha(lo[a], hi[a], self.e, self.ov, self.npml, self.sigma0, self.power)
                  for a in range(self.dim)]
            self.sub_win[R] = win
            self.sub_shape[R] = tuple(hi[a] - lo[a] + 2 * self.e for a in range(self.dim))
            self.sub_A[R] = pml_operator([x[0] for x in al], [x[1] for x in al], self.k2[win], self.h)

    # ------------------------------------------------------------------ basics
    def lo_hi(self, R, a) -> Tuple[int, int]:
        return int(self.cuts[a][R[a]]), int(self.cuts[a][R[a] + 1])

    def rhs(self, f: np.ndarray) -> np.ndarray:
        """b = h^2 J f: right-hand side of the J-scaled system (weak form, Eq. (32))."""
        return (self.h * self.h) * self.J_global * f

    def apply_global(self, w: np.ndarray) -> np.ndarray:
        return (self.A_global @ w.ravel()).reshape(self.gshape)

    def global_solve(self, b: np.ndarray) -> np.ndarray:
        """Direct solve of the global truncated PML problem (sparse LU, a library routine)."""
        if self._glu is None:
            self._glu = spla.splu(self.A_global.tocsc())
        return self._glu.solve(b.ravel()).reshape(self.gshape)

    def factor(self):
        """Factor every subdomain operator once (the paper uses MUMPS; here SuperLU)."""
        def one(R):
            return R, spla.splu(self.sub_A[R].tocsc())
        todo = [R for R in self.subs if R not in self.sub_lu]
        if self.workers > 1:
            with ThreadPoolExecutor(self.workers) as ex:
                for R, lu in ex.map(one, todo):
                    self.sub_lu[R] = lu
        else:
            for R in todo:
                self.sub_lu[R] = one(R)[1]

    def local_solve(self, R, src: np.ndarray) -> np.ndarray:
        """u = L^_{ij}^{-1} src on the subdomain's extended grid (Eqs. (37)/(38))."""
        if R not in self.sub_lu:
            self.sub_lu[R] = spla.splu(self.sub_A[R].tocsc())
        return self.sub_lu[R].solve(src.ravel()).reshape(self.sub_shape[R])

    # ----------------------------------------------------- cut-offs and masks
    def cutoff_1d(self, R, a: int, side: int) -> np.ndarray:
        """One-sided cut-off of subdomain R along axis a on its extended range.

        side = -1: beta_{<-;i} (decays below the low face, Section 2.2),
        side = +1: beta_{->;i+1} (decays above the high face).  A side on the
        global boundary has beta = 1 (i = 1 and i = N+1 cases in the paper).
        """
        lo, hi = self.lo_hi(R, a)
        p = np.arange(lo - self.e, hi + self.e)
        if side < 0:
            if R[a] == 0:
                return np.ones(p.shape)
            return beta0((lo - 1 - p) / self.ov)
        if R[a] == self.parts[a] - 1:
            return np.ones(p.shape)
        return beta0((p - hi) / self.ov)

    def _outer(self, vecs: Sequence[np.ndarray]) -> np.ndarray:
        out = np.ones([len(v) for v in vecs])
        for a, v in enumerate(vecs):
            shape = [1] * len(vecs)
            shape[a] = len(v)
            out = out * v.reshape(shape)
        return out

    def beta_own(self, R) -> np.ndarray:
        """beta_{0;ij}: product of the subdomain's one-sided cut-offs (Section 2.2)."""
        return self._outer([self.cutoff_1d(R, a, -1) * self.cutoff_1d(R, a, +1) for a in range(self.dim)])

    def beta_dir(self, S, d) -> np.ndarray:
        """beta_d of sender S for direction d: product over the non-zero components of d of
        the sender's cut-off on the side facing the receiver (e.g. beta_-> * beta_^ for the
        upper-right corner)."""
        vecs = []
        for a in range(self.dim):
            vecs.append(np.ones(self.sub_shape[S][a]) if d[a] == 0 else self.cutoff_1d(S, a, d[a]))
        return self._outer(vecs)

    def chi_dir(self, R, d) -> np.ndarray:
        """chi_d on receiver R's grid: the receiver's side of each shared interface."""
        vecs = []
        for a in range(self.dim):
            lo, hi = self.lo_hi(R, a)
            p = np.arange(lo - self.e, hi + self.e)
            if d[a] > 0:
                vecs.append((p >= lo).astype(np.float64))
            elif d[a] < 0:
                vecs.append((p < hi).astype(np.float64))
            else:
                vecs.append(np.ones(p.shape))
        return self._outer(vecs)

    def own_mask(self, R) -> np.ndarray:
        """Indicator of R's own region on its extended grid (own box, continued through the
        global extension band on sides at the global boundary)."""
        vecs = []
        for a in range(self.dim):
            lo, hi = self.lo_hi(R, a)
            p = np.arange(lo - self.e, hi + self.e)
            m = (p >= lo) & (p < hi)
            if R[a] == 0:
                m |= p < lo
            if R[a] == self.parts[a] - 1:
                m |= p >= hi
            vecs.append(m.astype(np.float64))
        return self._outer(vecs)

    # --------------------------------------------------------------- transfer
    def sender(self, R, d):
        S = tuple(R[a] - d[a] for a in range(self.dim))
        if all(0 <= S[a] < self.parts[a] for a in range(self.dim)):
            return S
        return None

    def transfer(self, R, d, v_sender: np.ndarray) -> np.ndarray:
        """Psi_d(v) = -L^_R(beta_d v) chi_d on the receiver's grid (Section 2.2, transfer
        operators; Eq. (38) uses them with the receiver's truncated operator).

        beta_d v lives on the sender's grid; it is carried onto the receiver's grid
        through the global node positions (zero where the grids do not overlap; chi_d
        keeps only receiver nodes whose stencil stays inside the overlap).
        """
        S = self.sender(R, d)
        bv = self.beta_dir(S, d) * v_sender
        moved = np.zeros(self.sub_shape[R], dtype=np.complex128)
        wr, ws = self.sub_win[R], self.sub_win[S]
        dst, srcs = [], []
        for a in range(self.dim):
            g0 = max(wr[a].start, ws[a].start)
            g1 = min(wr[a].stop, ws[a].stop)
            dst.append(slice(g0 - wr[a].start, g1 - wr[a].start))
            srcs.append(slice(g0 - ws[a].start, g1 - ws[a].start))
        moved[tuple(dst)] = bv[tuple(srcs)]
        Lbv = (self.sub_A[R] @ moved.ravel()).reshape(self.sub_shape[R])
        return -Lbv * self.chi_dir(R, d)

    def restrict_own(self, R, b: np.ndarray) -> np.ndarray:
        """f_ij = f chi_{Omega_ij} (Section 2.2) on R's grid, for the J-scaled b."""
        return b[self.sub_win[R]] * self.own_mask(R)

    # -------------------------------------------------------------- Algorithm
    def step_source(self, R, s: int, hist: Dict[int, Dict]) -> np.ndarray:
        """Right-hand side of Eq. (38) for subdomain R at step s >= 2."""
        src = np.zeros(self.sub_shape[R], dtype=np.complex128)
        for d in directions(self.dim):
            S = self.sender(R, d)
            t = s - lag(d)
            if S is None or t < 1:
                continue
            src += self.transfer(R, d, hist[t][S])
        return src

    def run(self, b: np.ndarray, nsteps: int, callback=None, keep_all: bool = False):
        """Algorithm 3.1 for ``nsteps`` steps (continued past N1+N2 as an iteration).

        ``callback(s, hist, U)`` runs after every step; returning True stops the
        iteration there.  Returns a dict with U (per-subdomain sums of u^s), the
        assembled solution w (Eq. (39)), the last ``dim`` per-step solutions
        ``u`` (step -> {R: u^s_R}), the number of steps taken and, if keep_all,
        every step's sources and solutions.
        """
        self.factor()
        hist: Dict[int, Dict] = {}
        U = {R: np.zeros(self.sub_shape[R], dtype=np.complex128) for R in self.subs}
        srcs_all, u_all = {}, {}
        maxlag = self.dim
        for s in range(1, nsteps + 1):
            def one(R):
                src = self.restrict_own(R, b) if s == 1 else self.step_source(R, s, hist)
                return R, src, self.local_solve(R, src)
            if self.workers > 1:
                with ThreadPoolExecutor(self.workers) as ex:
                    res = list(ex.map(one, self.subs))
            else:
                res = [one(R) for R in self.subs]
            hist[s] = {}
            for R, src, u in res:
                hist[s][R] = u
                U[R] += u
                if keep_all:
                    srcs_all[(s, R)] = src
                    u_all[(s, R)] = u
            for old in [t for t in hist if t <= s - maxlag]:
                del hist[old]
            if callback is not None and callback(s, hist, U):
                break
        out = {"U": U, "w": self.assemble(U), "u": hist, "steps": s}
        if keep_all:
            out["src"] = srcs_all
            out["u_all"] = u_all
        return out

    def assemble(self, U: Dict) -> np.ndarray:
        """u^_DDM = sum_ij beta_{0;ij} U_ij on the global grid (Eq. (39))."""
        w = np.zeros(self.gshape, dtype=np.complex128)
        for R in self.subs:
            w[self.sub_win[R]] += self.beta_own(R) * U[R]
        return w

    def strip_residual(self, R, s: int, hist: Dict[int, Dict]) -> np.ndarray:
        """Residual b - A w_s on R's own region, from transfers of the last steps only.

        With U^(s) = sum_{t<=s} u^t, summing Eq. (38) over the steps gives
        L^_R U_R^(s) = f_R + sum_d Psi_d(U_S^(s - lag d)), while at an own node the
        neighbours' terms of A w equal -Psi_d(U_S^(s)) (beta_{0;S} and beta_d agree on
        the stencil there).  Hence r = sum_d Psi_d(u^s + .. + u^{s-lag(d)+1}) on own(R).
        """
        r = np.zeros(self.sub_shape[R], dtype=np.complex128)
        for d in directions(self.dim):
            S = self.sender(R, d)
            if S is None:
                continue
            v = np.zeros(self.sub_shape[S], dtype=np.complex128)
            for t in range(s - lag(d) + 1, s + 1):
                if t >= 1:
                    v = v + hist[t][S]
            r += self.transfer(R, d, v)
        return r * self.own_mask(R)

    def global_from_own(self, per_sub: Dict) -> np.ndarray:
        """Scatter per-subdomain values on own regions into one global array."""
        g = np.zeros(self.gshape, dtype=np.complex128)
        for R in self.subs:
            g[self.sub_win[R]] += per_sub[R] * self.own_mask(R)
        return g

    def precondition(self, r: np.ndarray, K: int) -> np.ndarray:
        """M_K(r): K steps of Algorithm 3.1 with right-hand side r, returning u^_DDM
        (Section 4.2.2, the DDM as a preconditioner)."""
        return self.run(r, K)["w"]
