"""3D GPU parity: the 7-point operator, 26 transfer directions with lags 1/2/3, z-plane block
factors and the plane-GEMM solves against the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import from_local, from_local_batch, oracle_of, rel, to_local, to_local_batch  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def cases():
    out = {"gauss-2x2x2": W.tiny_3d(seed=1, n=12, parts=(2, 2, 2), ov=1, npml=3)}
    wl = W.tiny_3d(seed=2, n=14, parts=(2, 2, 2), ov=2, npml=3)
    wl.cuts = (np.array([0, 6, 14]), np.array([0, 8, 14]), np.array([0, 7, 14]))   # uneven
    out["uneven-ov2"] = wl
    out["3x1x2"] = W.tiny_3d(seed=3, n=12, parts=(3, 1, 2), ov=1, npml=2)
    return out


CASES = cases()


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("name", list(CASES))
def test_3d_global_operator(name):
    wl = CASES[name]
    o = oracle_of(wl)
    s = D.Solver(wl)
    x = cplx(np.random.default_rng(0), o.gshape)
    y = torch.empty(o.gshape, dtype=torch.complex128, device="cuda")
    D.ddm_global_apply(s.ctx, s.to_dev(x), y)
    assert rel(y.cpu().numpy(), o.apply_global(x)) < 1e-13
    s.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [D.DDM_FP64, D.DDM_MIXED])
def test_3d_local_solves(name, prec):
    wl = CASES[name]
    o = oracle_of(wl)
    s = D.Solver(wl, precision=prec, max_rhs=2).factor()
    rng = np.random.default_rng(1)
    srcs = [{R: cplx(rng, o.sub_shape[R]) for R in o.subs} for _ in range(2)]
    dt = np.complex128 if prec == D.DDM_FP64 else np.complex64
    tdt = torch.complex128 if prec == D.DDM_FP64 else torch.complex64
    src = to_local_batch(o, srcs, dt)
    u = torch.zeros(src.shape, dtype=tdt, device="cuda")
    D.ddm_local_solve(s.ctx, s.to_dev(src), u, 2)
    gots = from_local_batch(o, u.cpu().numpy(), 2)
    tol = 1e-10 if prec == D.DDM_FP64 else 2e-4
    for r in range(2):
        got = gots[r]
        for R in o.subs:
            assert rel(got[R], o.local_solve(R, srcs[r][R])) < tol, (R, r)
    s.close()


@pytest.mark.parametrize("name", ["gauss-2x2x2", "uneven-ov2"])
def test_3d_every_step_matches_oracle(name):
    wl = CASES[name]
    o = oracle_of(wl)
    s = D.Solver(wl).factor()
    b = o.rhs(wl.f[0])
    nmax = sum(o.parts) + 3
    ref = {}

    def cb(step, hist, U):
        ref[step] = (o.assemble(U), math.sqrt(sum(np.linalg.norm(o.strip_residual(R, step, hist)) ** 2
                                                   for R in o.subs)))
        return False

    o.run(b, nmax, callback=cb)
    for K in range(1, nmax + 1):
        w = torch.zeros(o.gshape, dtype=torch.complex128, device="cuda")
        res = D.ddm_steps(s.ctx, s.to_dev(b), K, w, None)
        assert rel(w.cpu().numpy(), ref[K][0]) < 1e-10, K
        assert abs(res[K - 1] - ref[K][1]) <= 1e-9 * np.linalg.norm(b) + 1e-10 * ref[K][1], K
    s.close()


@pytest.mark.parametrize("mode", [D.DDM_FGMRES, D.DDM_STEPPING])
def test_3d_mixed_reaches_1e6(mode):
    wl = CASES["gauss-2x2x2"]
    o = oracle_of(wl)
    s = D.Solver(wl, precision=D.DDM_MIXED).factor()
    u = torch.zeros(o.gshape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-6, max_it=300, mode=mode, K=4, restart=40)
    b = o.rhs(wl.f[0])
    x = u.cpu().numpy()
    assert info["converged"] and np.linalg.norm(b - o.apply_global(x)) / np.linalg.norm(b) <= 1e-6
    assert rel(x, o.global_solve(b)) < 1e-3
    s.close()


def test_3d_constant_medium_shares_one_factor():
    wl = W.tiny_3d(seed=4, n=12, parts=(2, 2, 2), ov=1, npml=3, medium="const")
    o = oracle_of(wl)
    s = D.Solver(wl).factor()
    u = torch.zeros(o.gshape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-9, max_it=100, K=3, restart=30)
    assert info["n_unique_factors"] == 1 and info["converged"]
    b = o.rhs(wl.f[0])
    assert rel(u.cpu().numpy(), o.global_solve(b)) < 1e-6
    s.close()
