"""Pins of the oracle's DDM (oracle/ddm.py) and FGMRES (oracle/krylov.py).

What each check is tied to:
  * Lemma 2.1 (source transfer) holds exactly for the discrete operator: the
    oracle's transfer Psi reproduces u0 = beta u0 + L^{-1}(-(L beta u0) chi).
  * The box-replacement remark after Lemma 2.1: the receiver's own truncated
    problem gives the same u2 as the big box.
  * N1 = N2 = 1: one step of Algorithm 3.1 is the global direct solve.
  * Structural zeros (Section 3.2): with the source in one subdomain, u^s_ij = 0
    for s < |i-i0| + |j-j0| + 1.
  * Theorem 2.4 (exactness in R^2) survives discretely as a remnant that
    shrinks when the PML gets stronger.
  * Fixed point: continued stepping converges to the global direct solution, and
    the residual taken from the last steps' transfers equals b - A w exactly; a
    planted lag mistake breaks that identity.
  * FGMRES: on a random dense system it matches a dense solve, its residual
    estimate equals the true residual, and it is monotone.
"""
import math

import numpy as np
import pytest

import oracle.ddm as ddm_mod
from oracle.ddm import DDMOracle, beta0, directions, lag
from oracle.krylov import ddm_fgmres, ddm_stepping, fgmres
from paper_1807_04180_gb300 import workloads as W


def make(wl, **kw):
    return DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c, **kw)


def test_beta0_properties():
    """beta_0 in C^2, monotone, 1 for t <= 0 and 0 for t >= 1 (Section 2.2)."""
    t = np.linspace(-0.5, 1.5, 4001)
    b = beta0(t)
    assert np.all(b[t <= 0] == 1) and np.all(b[t >= 1] == 0)
    assert np.all(np.diff(b) <= 1e-15)
    eps = 1e-4
    for t0 in (0.0, 1.0):   # first and second derivatives vanish at the joins
        d1 = (beta0(t0 + eps) - beta0(t0 - eps)) / (2 * eps)
        d2 = (beta0(t0 + eps) - 2 * beta0(t0) + beta0(t0 - eps)) / eps ** 2
        assert abs(d1) < 1e-6 and abs(d2) < 1e-3


def test_direction_count_and_lags():
    assert len(directions(2)) == 8 and len(directions(3)) == 26
    assert sorted(lag(d) for d in directions(2)) == [1] * 4 + [2] * 4
    assert sorted(lag(d) for d in directions(3)) == [1] * 6 + [2] * 12 + [3] * 8


@pytest.mark.parametrize("corner", [False, True])
def test_lemma_2_1_discrete(corner):
    """Lemma 2.1 on the global box: f in Omega_1, u0 = L^{-1} f, u1 = beta u0,
    u2 = L^{-1}(-(L u1) chi_2)  =>  u1 + u2 = u0 and u2 = 0 where beta = 1.
    The oracle's transfer operator must produce -(L u1) chi_2 on the receiver, and
    the receiver's own truncated problem must return u2 (box replacement)."""
    n, ov, npml = 16, 2, 6
    # the face case uses one part across the interface's tangential axis, so that the
    # receiver's tangential PML is the global one (its rows on the strip equal L's)
    wl = W.tiny_2d(seed=5, n=n, parts=(2, 2) if corner else (1, 2), ov=ov, npml=npml)
    o = make(wl)
    e = o.e
    S = (0, 0)
    f = np.zeros(o.gshape, dtype=complex)
    f[e + 2: e + 6, e + 1: e + 5] = np.random.default_rng(1).standard_normal((4, 4))
    u0 = o.global_solve(o.rhs(f))
    d = (1, 1) if corner else (0, 1)            # corner: towards (1,1); face: x-direction
    R = (1, 1) if corner else (0, 1)
    # beta on the global grid: the sender's cut-off(s) facing the receiver
    beta = np.ones(o.gshape)
    chi = np.ones(o.gshape)
    for a in range(2):
        if d[a]:
            lo, hi = o.lo_hi(S, a)
            cut = o.cutoff_1d(S, a, +1)                         # on S's range lo-e..hi+e-1
            full = np.ones(o.gshape[a])
            full[lo: hi + 2 * e] = cut
            full[hi + 2 * e:] = 0.0
            shape = [1, 1]; shape[a] = -1
            beta = beta * full.reshape(shape)
            m = np.zeros(o.gshape[a]); m[hi + e:] = 1.0          # receiver side of the face
            chi = chi * m.reshape(shape)
    if corner:
        # Lemma 2.1 needs beta = 1 on Omega_1; for the quarter-plane cut that is
        # beta_-> + beta_^ - beta_-> beta_^ (Section 2.2, corner construction).
        bx = np.ones(o.gshape[1]); lo, hi = o.lo_hi(S, 1)
        bx[lo: hi + 2 * e] = o.cutoff_1d(S, 1, +1); bx[hi + 2 * e:] = 0
        by = np.ones(o.gshape[0]); lo, hi = o.lo_hi(S, 0)
        by[lo: hi + 2 * e] = o.cutoff_1d(S, 0, +1); by[hi + 2 * e:] = 0
        beta_full = 1 - (1 - bx[None, :]) * (1 - by[:, None])
    else:
        beta_full = beta
    u1 = beta_full * u0
    src = -(o.apply_global(u1)) * chi
    u2 = o.global_solve(src)
    assert np.linalg.norm(u1 + u2 - u0) < 1e-10 * np.linalg.norm(u0)
    assert np.abs(u2[beta_full == 1.0]).max() < 1e-12 * np.abs(u0).max()
    # the oracle's Psi_d on the receiver equals -(L beta_d u0) chi_d there
    psi = o.transfer(R, d, u0[o.sub_win[S]])
    ref = (-(o.apply_global(beta * u0)) * chi)[o.sub_win[R]]
    assert np.linalg.norm(psi - ref) < 1e-12 * np.linalg.norm(ref)
    if not corner:
        # box replacement: the receiver's truncated problem reproduces u2 on its grid
        u2_R = o.local_solve(R, src[o.sub_win[R]])
        assert np.linalg.norm(u2_R - u2[o.sub_win[R]]) < 1e-10 * np.linalg.norm(u2)


def test_single_subdomain_is_global_solve():
    wl = W.tiny_2d(seed=2, parts=(1, 1))
    o = make(wl)
    b = o.rhs(wl.f[0])
    w = o.run(b, 1)["w"]
    u = o.global_solve(b)
    assert np.linalg.norm(w - u) < 1e-12 * np.linalg.norm(u)


def test_structural_zeros():
    """Section 3.2: with the source only in Omega_{i0,j0}, u^s_ij = 0 for s < |i-i0|+|j-j0|+1."""
    wl = W.tiny_2d(seed=4, n=20, parts=(4, 4), ov=1, npml=3)
    o = make(wl)
    e = o.e
    f = np.zeros(o.gshape, dtype=complex)
    i0, j0 = 1, 2
    y0, x0 = o.cuts[0][i0] + e + 2, o.cuts[1][j0] + e + 2
    f[y0, x0] = 1.0
    res = o.run(o.rhs(f), 8, keep_all=True)
    for (s, R), u in res["u_all"].items():
        dist = abs(R[0] - i0) + abs(R[1] - j0)
        if s < dist + 1:
            assert np.all(u == 0), (s, R)
        elif s == dist + 1:
            assert np.abs(u).max() > 0, (s, R)


def _const(n, parts, ov, npml, sigma0, k=2 * math.pi * 3, seed=0):
    h = 1.0 / n
    e = ov + npml
    c = W.constant_medium((n, n), e)
    f = W.gaussian_source((n, n), h, e, (0.37, 0.58), 2 * h)[None]
    cuts = (W.uniform_cuts(n, parts),) * 2
    return W.Workload("c", (n, n), h, cuts, ov, npml, sigma0, 2.0, k, c, f)


def test_theorem_2_4_remnant_shrinks_with_pml():
    """Theorem 2.4: in R^2 with a constant medium u_DDM = u after N1+N2 steps.  Truncated and
    discretised, the remnant error shrinks as the PML absorbs better (Eq. (34))."""
    errs = []
    for npml, s0 in ((3, 2.0), (6, 8.0), (12, 20.0)):
        wl = _const(48, 3, 2, npml, s0)
        o = make(wl)
        b = o.rhs(wl.f[0])
        w = o.run(b, 6)["w"]
        u = o.global_solve(b)
        errs.append(np.linalg.norm(w - u) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-2, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_fixed_point_and_strip_residual(dim):
    """Continued stepping converges to the global direct solution, and the residual from the
    last steps' transfers equals b - A w_s (to rounding) at every step."""
    if dim == 2:
        wl = W.tiny_2d(seed=7, n=18, parts=(3, 2), ov=2, npml=3)
    else:
        n, ov, npml = 8, 1, 3
        h = 1.0 / n
        e = ov + npml
        c = W.gaussian_sum_medium((n, n, n), h, e, 3, n_bumps=3, cmin=1.0, cmax=2.0)
        f = W.gaussian_source((n, n, n), h, e, (0.3, 0.6, 0.45), 2 * h)[None]
        wl = W.Workload("t3", (n, n, n), h, (np.array([0, 4, 8]),) * 3, ov, npml, 10.0, 2.0,
                        2 * math.pi * 1.5, c, f)
    o = make(wl)
    b = o.rhs(wl.f[0])
    bn = np.linalg.norm(b)
    checks = []

    def cb(s, hist, U):
        w = o.assemble(U)
        r_explicit = b - o.apply_global(w)
        r_strips = o.global_from_own({R: o.strip_residual(R, s, hist) for R in o.subs})
        checks.append(np.linalg.norm(r_strips - r_explicit) / bn)
        return False

    res = o.run(b, 30, callback=cb)
    assert max(checks) < 1e-12, checks
    u = o.global_solve(b)
    assert np.linalg.norm(res["w"] - u) / np.linalg.norm(u) < 1e-8


def test_planted_lag_mistake_breaks_residual_identity(monkeypatch):
    """A plausible mistake (corners lagged by one step instead of two) must be caught."""
    wl = W.tiny_2d(seed=7, n=18, parts=(3, 3), ov=2, npml=3)
    monkeypatch.setattr(ddm_mod, "lag", lambda d: 1)
    o = make(wl)
    b = o.rhs(wl.f[0])
    out = {}

    def cb(s, hist, U):
        if s == 4:
            w = o.assemble(U)
            # the identity as derived for the paper's lags
            r = np.zeros(o.gshape, dtype=complex)
            per = {}
            for R in o.subs:
                acc = np.zeros(o.sub_shape[R], dtype=complex)
                for d in directions(2):
                    S = o.sender(R, d)
                    if S is None:
                        continue
                    v = hist[s][S] + (hist[s - 1][S] if sum(map(abs, d)) == 2 else 0)
                    acc += o.transfer(R, d, v)
                per[R] = acc * o.own_mask(R)
            r = o.global_from_own(per)
            out["gap"] = np.linalg.norm(r - (b - o.apply_global(w))) / np.linalg.norm(b)
        return False

    o.run(b, 4, callback=cb)
    assert out["gap"] > 1e-6


def test_uneven_partition_converges():
    wl = W.tiny_2d(seed=8, n=21, parts=(3, 2), ov=1, npml=4)
    wl.cuts = (np.array([0, 6, 13, 21]), np.array([0, 12, 21]))
    o = make(wl)
    b = o.rhs(wl.f[0])
    st = ddm_stepping(o, b, 1e-10, 80)
    u = o.global_solve(b)
    assert st["converged"] and np.linalg.norm(st["w"] - u) / np.linalg.norm(u) < 1e-8


def test_fgmres_dense_random():
    rng = np.random.default_rng(0)
    N = 40
    A = np.eye(N) * 3 + rng.standard_normal((N, N)) * 0.3 + 1j * rng.standard_normal((N, N)) * 0.3
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ests = []
    res = fgmres(lambda x: A @ x, lambda v: v, b, 1e-12, 15, 200)
    assert res["converged"]
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(res["x"] - x) / np.linalg.norm(x) < 1e-10
    h = res["history"]
    assert all(h[i + 1] <= h[i] * (1 + 1e-12) for i in range(min(len(h), 15) - 1))
    # the least-squares estimate equals the true residual within one cycle
    for m in (3, 7):
        r = fgmres(lambda x: A @ x, lambda v: v, b, 0.0, 30, m)
        true = np.linalg.norm(b - A @ r["x"]) / np.linalg.norm(b)
        assert abs(true - r["history"][-1]) < 1e-10


def test_ddm_fgmres_converges_to_direct():
    wl = W.tiny_2d(seed=9, n=16, parts=(2, 2), ov=1, npml=4)
    o = make(wl)
    b = o.rhs(wl.f[0])
    u = o.global_solve(b)
    res = ddm_fgmres(o, b, K=2, tol=1e-10, restart=20, max_it=60)
    assert res["converged"]
    assert np.linalg.norm(res["x"] - u) / np.linalg.norm(u) < 1e-8
    # an exact preconditioner (one subdomain) needs one iteration
    wl1 = W.tiny_2d(seed=9, n=16, parts=(1, 1), ov=1, npml=4)
    o1 = make(wl1)
    r1 = ddm_fgmres(o1, o1.rhs(wl1.f[0]), K=1, tol=1e-10, restart=5, max_it=5)
    assert r1["iters"] == 1 and r1["converged"]
