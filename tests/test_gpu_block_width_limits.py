"""Local solves at the block widths where the 2D kernels switch (Algorithm 3.1's subdomain
problems, Eqs. (37)/(38)), against the oracle's sparse direct solve.

The 2D factorisation keeps a subdomain's Schur blocks in registers (complex64, x-lines of at most
128 nodes) or shared memory (complex128, at most 96); wider x-lines go to the dense-block path.
Partitions here are two subdomains along x whose extended x-lines are exactly at and one past each
limit: 128 / 129 (complex64) and 96 / 97 (complex128), 16 own nodes along y, a heterogeneous
medium.  The complex64 case at 128 also runs 16 right-hand sides on the tensor cores (blocks of
at most 128 rows) and on the CUDA cores.  Each case then solves to 1e-6 with FGMRES.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import from_local_batch, oracle_of, rel, to_local_batch  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402

OV, NPML = 2, 6
E = OV + NPML


def _workload(ext_x):
    own = ext_x - 2 * E
    nx, ny = 2 * own, 16
    h = 1.0 / nx
    c = W.gaussian_sum_medium((ny, nx), h, E, seed=7, n_bumps=4, cmin=1.0, cmax=2.0)
    f = W.point_source((ny, nx), h, E, (0.5 * ny * h, 0.3 * nx * h))[None]
    cuts = (np.array([0, ny]), np.array([0, own, nx]))
    omega = 2 * math.pi * 1.5 / (10 * h)
    return W.Workload(f"width-{ext_x}", (ny, nx), h, cuts, OV, NPML, 50.0, 2.0, omega, c, f)


@pytest.mark.parametrize("prec,ext_x", [(D.DDM_MIXED, 128), (D.DDM_MIXED, 129), (D.DDM_FP64, 96), (D.DDM_FP64, 97)])
def test_local_solves_at_the_kernel_width_limits(prec, ext_x):
    wl = _workload(ext_x)
    o = oracle_of(wl)
    assert all(o.sub_shape[R][1] == ext_x for R in o.subs)
    nrhs = 16 if prec == D.DDM_MIXED and ext_x == 128 else 2
    rng = np.random.default_rng(ext_x)
    per = [{R: rng.standard_normal(o.sub_shape[R]) + 1j * rng.standard_normal(o.sub_shape[R]) for R in o.subs}
           for _ in range(nrhs)]
    dt = np.complex128 if prec == D.DDM_FP64 else np.complex64
    tdt = torch.complex128 if prec == D.DDM_FP64 else torch.complex64
    tol = 1e-10 if prec == D.DDM_FP64 else 5e-4
    s = D.Solver(wl, precision=prec, max_rhs=nrhs).factor()
    src = to_local_batch(o, per, dt)
    modes = [64, 4] if nrhs == 16 else [0]       # tensor cores, then CUDA cores; 0: the default choice
    for nr in modes:
        if nr:
            D.ddm_set_rhs_per_cta(s.ctx, nr)
        u = torch.zeros(src.shape, dtype=tdt, device="cuda")
        D.ddm_local_solve(s.ctx, s.to_dev(src), u, nrhs)
        got = from_local_batch(o, u.cpu().numpy(), nrhs)
        for r in (0, nrhs - 1):
            for R in o.subs:
                err = rel(got[r][R], o.local_solve(R, per[r][R]))
                assert err < tol, (prec, ext_x, nr, r, R, err)
    uu = torch.zeros(wl.c.shape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), uu, tol=1e-6, max_it=100, mode=D.DDM_FGMRES, K=4, restart=30)
    assert info["converged"] and info["rel_residual"] <= 1e-6
    s.close()
