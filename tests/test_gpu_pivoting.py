"""Pivoting of the dense-block factorisation (ddm_set_pivoting): 3D partitions and wide 2D
subdomains.

The Schur blocks D_k = T_k - L_k G_(k-1) U_(k-1) are inverted by Gauss-Jordan with partial
pivoting (the local solves of Algorithm 3.1, Eqs. (37)/(38)).  By default each panel's pivots are
searched among its own diagonal rows, and a threshold check sends the whole factorisation back to
the cluster search over all rows when the restricted choice is weak.

* The restricted search and the search over all rows give local solves equal to rounding, and
  both match the oracle: 3D (a small heterogeneous partition, FP64 and complex64) and the
  paper-scale 2D subdomains (b = 360).
* A threshold that every factorisation fails (tau = 1e-3) is redone with the full search, the
  redo is counted, and its results are the full search's bits.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import from_local, oracle_of, rel, single_box_oracle, to_local  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def _solve(wl, prec, src_np, tau):
    s = D.Solver(wl, precision=prec)
    D.ddm_set_pivoting(s.ctx, tau)
    s.factor()
    dt = torch.complex128 if prec == D.DDM_FP64 else torch.complex64
    src = torch.as_tensor(src_np, device="cuda").to(dt)
    u = torch.zeros_like(src)
    D.ddm_local_solve(s.ctx, src, u, 1)
    info = D.ddm_pivoting_info(s.ctx)
    s.close()
    return u.cpu().numpy(), info


@pytest.mark.parametrize("prec", [D.DDM_FP64, D.DDM_MIXED])
def test_3d_restricted_search_equals_full_search_and_oracle(prec):
    wl = W.tiny_3d(seed=2, n=20, parts=(2, 2, 2))
    o = oracle_of(wl)
    rng = np.random.default_rng(3)
    srcs = {R: rng.standard_normal(o.sub_shape[R]) + 1j * rng.standard_normal(o.sub_shape[R]) for R in o.subs}
    src = to_local(o, srcs)
    u_r, (tau, redone) = _solve(wl, prec, src, 4.0)
    assert tau == 4.0 and redone == 0
    u_f, (_, redone_f) = _solve(wl, prec, src, 0.0)
    assert redone_f == 0
    u_x, (_, redone_x) = _solve(wl, prec, src, 1e-3)
    assert redone_x == 1 and np.array_equal(u_x, u_f)
    eps = 1e-12 if prec == D.DDM_FP64 else 1e-5
    assert rel(u_r, u_f) < eps, rel(u_r, u_f)
    tol = 1e-10 if prec == D.DDM_FP64 else 5e-4
    got = from_local(o, u_r)
    for R in o.subs:
        assert rel(got[R], o.local_solve(R, srcs[R])) < tol, R


def test_paper_scale_2d_restricted_search_equals_full_search():
    wl = W.paper_table3(2)
    ob, R0 = single_box_oracle(wl, (0, 0))
    shape = ob.sub_shape[R0]
    rng = np.random.default_rng(5)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = ob.local_solve(R0, a)
    s = D.Solver(wl, precision=D.DDM_MIXED)
    total = D.ddm_local_layout(s.ctx)["total"]
    s.close()
    src = np.zeros(total, complex)
    src[: a.size] = a.ravel()                  # subdomain (0, 0) first in the local layout
    u_r, (_, redone) = _solve(wl, D.DDM_MIXED, src, 4.0)
    u_f, _ = _solve(wl, D.DDM_MIXED, src, 0.0)
    assert redone == 0
    assert rel(u_r, u_f) < 1e-5, rel(u_r, u_f)
    assert rel(u_r[: a.size].reshape(shape), ref) < 5e-4


def test_pivoting_argument_checks():
    wl = W.tiny_3d(seed=1, n=8, parts=(2, 2, 2))
    s = D.Solver(wl, precision=D.DDM_MIXED)
    for bad in (-1.0, float("nan"), 1e7):
        with pytest.raises(D.DDMError) as ei:
            D.ddm_set_pivoting(s.ctx, bad)
        assert ei.value.status == D.DDM_E_INVAL
    s.close()
