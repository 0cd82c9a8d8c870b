"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 mode agrees with the oracle to a relative L2 error of 1e-10 per iterate
(global operator, local solves, every DDM step, the preconditioner and FGMRES); mixed mode
(complex64 local solves inside FP64 Krylov) must reach an explicit FP64 relative residual of
1e-6, and its error against the FP64 oracle solution is checked to the level that residual
allows.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import from_local, from_local_batch, oracle_of, rel, to_local, to_local_batch  # noqa: E402
from oracle.krylov import ddm_fgmres  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402

DEV = "cuda"


def cases():
    """Small problems spanning several 16-row solve chunks with ragged tails, uneven cuts,
    one-subdomain and strip-heavy partitions."""
    out = {}
    out["tiny-2x2"] = W.tiny_2d(seed=1, n=20, parts=(2, 2), ov=1, npml=3)
    out["3x2-ov2"] = W.tiny_2d(seed=2, n=30, parts=(3, 2), ov=2, npml=4)
    wl = W.tiny_2d(seed=3, n=37, parts=(3, 4), ov=2, npml=5)
    wl.cuts = (np.array([0, 11, 25, 37]), np.array([0, 9, 17, 28, 37]))   # uneven, ragged
    out["uneven-3x4"] = wl
    out["1x1"] = W.tiny_2d(seed=4, n=24, parts=(1, 1), ov=1, npml=4)
    out["wide-1x3"] = W.tiny_2d(seed=5, n=48, parts=(1, 3), ov=2, npml=6)
    return out


CASES = cases()


def make(wl, prec=D.DDM_FP64, max_rhs=1):
    return D.Solver(wl, precision=prec, max_rhs=max_rhs).factor()


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_and_global_operator(name):
    wl = CASES[name]
    o = oracle_of(wl)
    s = D.Solver(wl)
    rng = np.random.default_rng(0)
    x = cplx(rng, o.gshape)
    y = torch.empty(o.gshape, dtype=torch.complex128, device=DEV)
    D.ddm_global_apply(s.ctx, s.to_dev(x), y)
    assert rel(y.cpu().numpy(), o.apply_global(x)) < 1e-13
    b = torch.empty_like(y)
    D.ddm_rhs(s.ctx, s.to_dev(wl.f[0]), b)
    assert rel(b.cpu().numpy(), o.rhs(wl.f[0])) < 1e-14
    s.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [D.DDM_FP64, D.DDM_MIXED])
def test_local_solves(name, prec):
    wl = CASES[name]
    o = oracle_of(wl)
    s = make(wl, prec, max_rhs=3)
    rng = np.random.default_rng(1)
    nrhs = 3
    srcs = [{R: cplx(rng, o.sub_shape[R]) for R in o.subs} for _ in range(nrhs)]
    dt = np.complex128 if prec == D.DDM_FP64 else np.complex64
    tdt = torch.complex128 if prec == D.DDM_FP64 else torch.complex64
    src = to_local_batch(o, srcs, dt)
    u = torch.zeros(src.shape, dtype=tdt, device=DEV)
    D.ddm_local_solve(s.ctx, s.to_dev(src), u, nrhs)
    gots = from_local_batch(o, u.cpu().numpy(), nrhs)
    tol = 1e-10 if prec == D.DDM_FP64 else 2e-4
    for r in range(nrhs):
        got = gots[r]
        for R in o.subs:
            assert rel(got[R], o.local_solve(R, srcs[r][R])) < tol, (R, r)
    s.close()


@pytest.mark.parametrize("name", ["tiny-2x2", "3x2-ov2", "uneven-3x4", "wide-1x3"])
def test_every_step_matches_oracle(name):
    """Per iterate: the assembled w_s, the last step's local solutions and the own-region
    residual after every step s = 1..N1+N2+3 match Algorithm 3.1 in the oracle."""
    wl = CASES[name]
    o = oracle_of(wl)
    s = make(wl)
    b = o.rhs(wl.f[0])
    bd = s.to_dev(b)
    nmax = sum(o.parts) + 3
    hist_or = {}

    def cb(step, hist, U):
        hist_or[step] = {"w": o.assemble(U), "u": {R: hist[step][R].copy() for R in o.subs},
                         "res": math.sqrt(sum(np.linalg.norm(o.strip_residual(R, step, hist)) ** 2 for R in o.subs))}
        return False

    o.run(b, nmax, callback=cb)
    L = D.ddm_local_layout(s.ctx)["total"]
    for K in range(1, nmax + 1):
        w = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
        ul = torch.zeros(L, dtype=torch.complex128, device=DEV)
        res = D.ddm_steps(s.ctx, bd, K, w, ul)
        assert rel(w.cpu().numpy(), hist_or[K]["w"]) < 1e-10, K
        got = from_local(o, ul.cpu().numpy())
        ref = hist_or[K]["u"]
        assert rel(to_local(o, got), to_local(o, ref)) < 1e-10, K
        for st in range(1, K + 1):
            assert abs(res[st - 1] - hist_or[st]["res"]) <= 1e-9 * np.linalg.norm(b) + 1e-10 * hist_or[st]["res"], (K, st)
    s.close()


def test_structural_zeros_exact():
    """Section 3.2: with the source in one subdomain, u^s vanishes (exactly) in subdomains farther
    than s-1 Manhattan steps."""
    wl = W.tiny_2d(seed=4, n=40, parts=(4, 4), ov=1, npml=3)
    o = oracle_of(wl)
    s = make(wl)
    e = o.e
    f = np.zeros(o.gshape, dtype=complex)
    f[o.cuts[0][1] + e + 3, o.cuts[1][2] + e + 4] = 1.0
    b = o.rhs(f)
    L = D.ddm_local_layout(s.ctx)["total"]
    for K in range(1, 6):
        ul = torch.zeros(L, dtype=torch.complex128, device=DEV)
        D.ddm_steps(s.ctx, s.to_dev(b), K, None, ul, want_res=False)
        got = from_local(o, ul.cpu().numpy())
        for R in o.subs:
            dist = abs(R[0] - 1) + abs(R[1] - 2)
            if K < dist + 1:
                assert np.all(got[R] == 0), (K, R)
            elif K == dist + 1:
                assert np.abs(got[R]).max() > 0
    s.close()


def test_single_subdomain_step_is_direct_solve():
    wl = CASES["1x1"]
    o = oracle_of(wl)
    s = make(wl)
    b = o.rhs(wl.f[0])
    w = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
    D.ddm_steps(s.ctx, s.to_dev(b), 1, w, None)
    assert rel(w.cpu().numpy(), o.global_solve(b)) < 1e-10
    s.close()


@pytest.mark.parametrize("name", ["3x2-ov2", "uneven-3x4"])
def test_apply_matches_preconditioner(name):
    wl = CASES[name]
    o = oracle_of(wl)
    s = make(wl, max_rhs=2)
    rng = np.random.default_rng(3)
    v = cplx(rng, (2,) + o.gshape)
    out = torch.zeros(v.shape, dtype=torch.complex128, device=DEV)
    D.ddm_apply(s.ctx, 2, s.to_dev(v), out, 2)
    out = out.cpu().numpy()
    for r in range(2):
        assert rel(out[r], o.precondition(v[r], 2)) < 1e-10
    # a batch of right-hand sides gives what each gives alone
    one = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
    D.ddm_apply(s.ctx, 2, s.to_dev(v[1]), one, 1)
    assert rel(one.cpu().numpy(), out[1]) < 1e-14
    s.close()


@pytest.mark.parametrize("name", ["3x2-ov2", "uneven-3x4"])
def test_fgmres_fp64_matches_oracle(name):
    wl = CASES[name]
    o = oracle_of(wl)
    s = make(wl)
    b = o.rhs(wl.f[0])
    u = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-10, max_it=200, mode=D.DDM_FGMRES, K=2, restart=30)
    ref = ddm_fgmres(o, b, K=2, tol=1e-10, restart=30, max_it=200)
    assert info["converged"] and info["rel_residual"] <= 1e-10
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    assert rel(u.cpu().numpy(), o.global_solve(b)) < 1e-8
    s.close()


@pytest.mark.parametrize("mode", [D.DDM_FGMRES, D.DDM_STEPPING])
@pytest.mark.parametrize("name", ["3x2-ov2", "uneven-3x4", "wide-1x3"])
def test_mixed_precision_reaches_1e6(name, mode):
    wl = CASES[name]
    o = oracle_of(wl)
    s = make(wl, D.DDM_MIXED)
    b = o.rhs(wl.f[0])
    u = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-6, max_it=400, mode=mode, K=2, restart=40)
    x = u.cpu().numpy()
    r = np.linalg.norm(b - o.apply_global(x)) / np.linalg.norm(b)
    assert info["converged"] and r <= 1e-6 and abs(r - info["rel_residual"]) < 1e-9
    # error against the FP64 oracle solution, bounded by the residual through the conditioning
    err = rel(x, o.global_solve(b))
    assert err < 1e-3, err
    s.close()


def test_stepping_fp64_matches_direct():
    wl = CASES["3x2-ov2"]
    o = oracle_of(wl)
    s = make(wl)
    b = o.rhs(wl.f[0])
    u = torch.zeros(o.gshape, dtype=torch.complex128, device=DEV)
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-10, max_it=300, mode=D.DDM_STEPPING)
    assert info["converged"]
    assert rel(u.cpu().numpy(), o.global_solve(b)) < 1e-8
    s.close()


def test_identical_subdomains_share_one_factor():
    wl = W.constant_2d_160()
    s = make(wl)
    u = torch.zeros(wl.c.shape, dtype=torch.complex128, device=DEV)
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-6, max_it=100, K=2, restart=30)
    assert info["n_unique_factors"] == 1 and info["converged"]
    s.close()


def test_solve_host_buffers_match_device_path():
    wl = CASES["3x2-ov2"]
    s = make(wl, D.DDM_MIXED)
    f = np.ascontiguousarray(wl.f[0])
    uh = np.zeros_like(f)
    ih = D.ddm_solve_host(s.ctx, f, uh, tol=1e-8, max_it=200)
    ud = torch.zeros(f.shape, dtype=torch.complex128, device=DEV)
    idv = D.ddm_solve(s.ctx, s.to_dev(f), ud, tol=1e-8, max_it=200)
    assert ih["iters"] == idv["iters"]
    assert rel(uh, ud.cpu().numpy()) < 1e-12
    s.close()


def test_error_statuses():
    wl = CASES["tiny-2x2"]
    s = D.Solver(wl)
    u = torch.zeros(wl.c.shape, dtype=torch.complex128, device=DEV)
    with pytest.raises(D.DDMError) as ei:
        D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u)
    assert ei.value.status == D.DDM_E_STATE
    s.factor()
    with pytest.raises(D.DDMError) as ei:
        D.ddm_apply(s.ctx, 0, s.to_dev(wl.f[0]), u)
    assert ei.value.status == D.DDM_E_INVAL
    with pytest.raises(D.DDMError) as ei:
        D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-14, max_it=2)
    assert ei.value.status == D.DDM_E_NOCONV
    s.close()


@pytest.mark.parametrize("prec", [D.DDM_FP64, D.DDM_MIXED])
def test_batched_fgmres_matches_single_rhs(prec):
    """nrhs right-hand sides solved together (one nrhs-wide preconditioner per iteration)
    give what each gives alone."""
    wl = W.tiny_2d(seed=13, n=30, parts=(3, 2), ov=2, npml=4, nrhs=5)
    o = oracle_of(wl)
    s = make(wl, prec, max_rhs=5)
    f = s.to_dev(np.ascontiguousarray(wl.f))
    U = torch.zeros(wl.f.shape, dtype=torch.complex128, device=DEV)
    info = D.ddm_solve(s.ctx, f, U, nrhs=5, tol=1e-8, max_it=200, K=2, restart=20)
    assert info["converged"]
    for r in range(5):
        u1 = torch.zeros(wl.c.shape, dtype=torch.complex128, device=DEV)
        D.ddm_solve(s.ctx, s.to_dev(wl.f[r]), u1, nrhs=1, tol=1e-8, max_it=200, K=2, restart=20)
        assert rel(U[r].cpu().numpy(), u1.cpu().numpy()) < 1e-12, r
        b = o.rhs(wl.f[r])
        assert rel(U[r].cpu().numpy(), o.global_solve(b)) < (1e-6 if prec == D.DDM_FP64 else 1e-4)
    s.close()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_graph_replay_matches_direct_launches(nrhs):
    """One DDM preconditioner application replayed from a captured CUDA graph gives the same
    result as the launched kernels, in ddm_apply and inside FGMRES."""
    wl = W.tiny_2d(seed=17, n=30, parts=(3, 2), ov=2, npml=4, nrhs=nrhs)
    s = make(wl, D.DDM_MIXED, max_rhs=nrhs)
    rng = np.random.default_rng(9)
    v = s.to_dev(cplx(rng, (nrhs,) + wl.c.shape))
    plain = torch.zeros_like(v)
    D.ddm_apply(s.ctx, 3, v, plain, nrhs)
    D.ddm_set_graph(s.ctx, True)
    for _ in range(2):                       # capture, then replay
        g = torch.zeros_like(v)
        D.ddm_apply(s.ctx, 3, v, g, nrhs)
        assert torch.equal(g, plain)
    f = s.to_dev(np.ascontiguousarray(wl.f))
    u_g = torch.zeros_like(f)
    ig = D.ddm_solve(s.ctx, f, u_g, nrhs=nrhs, tol=1e-7, max_it=200, K=4, restart=20)
    D.ddm_set_graph(s.ctx, False)
    u_p = torch.zeros_like(f)
    ip = D.ddm_solve(s.ctx, f, u_p, nrhs=nrhs, tol=1e-7, max_it=200, K=4, restart=20)
    assert ig["iters"] == ip["iters"] and torch.equal(u_g, u_p)
    assert D.ddm_timing(s.ctx)["graph"][1] >= 0
    s.close()
