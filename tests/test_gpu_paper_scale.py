"""Paper-scale 2D subdomains (Section 4.2.1): 300^2 own nodes plus a 30-node overlap + PML band,
i.e. x-lines of b = 360 nodes, wider than the 2D register and shared-memory kernels take.  Such
partitions run on the dense-block path (the Schur blocks inverted by the cluster-panel
Gauss-Jordan, each block step of the local solves a contraction over all subdomains sharing the
factor).

* Local solves (Algorithm 3.1's subdomain problems, Eqs. (37)/(38)) on sampled subdomains of the
  2 x 2 Table 3 problem against the oracle's sparse direct solve of the same subdomain: FP64 to
  1e-10, complex64 to the FP32 bound on the tensor cores and on the CUDA cores.
* Algorithm 3.1 as an iterative solver in FP64: the number of DDM steps to a relative residual
  of 1e-8 equals the oracle's (tests/golden/oracle_table3.json, written by the oracle only), and
  the explicit FP64 residual is at or below 1e-8.  Mixed precision reaches 1e-8 as well.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import rel, single_box_oracle  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_table3.json")


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_b360_local_solves_match_oracle():
    wl = W.paper_table3(2)
    sample = [(0, 0), (1, 1)]
    rng = np.random.default_rng(41)
    ob, R0 = single_box_oracle(wl, sample[0])          # constant medium: every subdomain's operator
    shape = ob.sub_shape[R0]
    assert shape == (360, 360)
    srcs = {R: cplx(rng, shape) for R in sample}
    ref = {R: ob.local_solve(R0, srcs[R]) for R in sample}
    for prec, tc, tol in ((D.DDM_FP64, False, 1e-10), (D.DDM_MIXED, True, 5e-4), (D.DDM_MIXED, False, 5e-4)):
        s = D.Solver(wl, precision=prec).factor()
        D.ddm_set_tensor_cores(s.ctx, tc)
        lay = D.ddm_local_layout(s.ctx)
        dt = torch.complex128 if prec == D.DDM_FP64 else torch.complex64
        src = torch.zeros(lay["total"], dtype=dt, device="cuda")
        n = shape[0] * shape[1]
        for R in sample:
            o = lay["offsets"][R[0] * 2 + R[1]]
            src[o: o + n] = torch.as_tensor(srcs[R].ravel(), device="cuda").to(dt)
        u = torch.zeros_like(src)
        D.ddm_local_solve(s.ctx, src, u, 1)
        got = u.cpu().numpy()
        for R in sample:
            o = lay["offsets"][R[0] * 2 + R[1]]
            err = rel(got[o: o + n].reshape(shape), ref[R])
            assert err < tol, (prec, tc, R, err)
        s.close()


@pytest.mark.parametrize("N", [2, 4])
def test_table3_fp64_stepping_counts_match_oracle(N):
    with open(GOLD) as fh:
        gold = json.load(fh)[str(N)]
    wl = W.paper_table3(N)
    s = D.Solver(wl, precision=D.DDM_FP64).factor()
    u = torch.zeros(wl.c.shape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-8, max_it=40 * N, mode=D.DDM_STEPPING)
    assert info["converged"] and info["rel_residual"] <= 1e-8
    assert info["n_unique_factors"] == 1                # the constant medium shares one factor
    assert info["ddm_steps"] == gold["ddm_steps"], (info["ddm_steps"], gold["ddm_steps"])
    s.close()


def test_table3_mixed_stepping_reaches_1e8():
    wl = W.paper_table3(4)
    s = D.Solver(wl, precision=D.DDM_MIXED).factor()
    u = torch.zeros(wl.c.shape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-8, max_it=400, mode=D.DDM_STEPPING)
    assert info["converged"] and info["rel_residual"] <= 1e-8
    s.close()
