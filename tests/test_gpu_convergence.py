"""Scaled convergence studies of Tables 1 and 2 (Section 4.1) through the GPU path.

The paper measures the DDM solution of Algorithm 3.1 (N1 + N2 (+ N3) steps, no Krylov
acceleration) against the exact solution on a sequence of meshes and reports rate 2.0 (2D,
5 x 5 subdomains) and about 2 (3D, 3 x 3 x 3 subdomains).  Here the same is done through the
library: ddm_steps with the paper's number of steps on a constant medium with a unit-mass
Gaussian source, compared on an annulus around the source with the closed-form free-space
solutions of Section 2.1 (2D: -(i/4) H0(k r) exp(-k^2 s^2 / 2); 3D: -exp(i k r) / (4 pi r)
exp(-k^2 s^2 / 2), the factor being the Gaussian's Fourier transform at k).  The sizes are scaled
down from the paper's (k / 2pi = 25 and 10 on 560^2..6720^2 and 80^3..160^3) so that every
subdomain stays within the 2D kernels' 128-node block width: 2D k / 2pi = 5 on [0, 1]^2 with
80^2, 160^2, 320^2 interiors; 3D k / 2pi = 1.5 with 24^3 and 48^3.  The PML keeps its physical
thickness (cells scale with n) and the overlap is 2 cells (1 in 3D).  At the coarsest size
every iterate is also checked against the oracle's Algorithm 3.1.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
scipy_special = pytest.importorskip("scipy.special")

from gpu_helpers import oracle_of, rel  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402

TABLE_RATE = 2.0      # Tables 1-2: second-order convergence of the DDM solutions


def _workload(dim, n, parts, k, width, ov, npml):
    h = 1.0 / n
    e = ov + npml
    shape = (n,) * dim
    c = W.constant_medium(shape, e, 1.0)
    f = W.gaussian_source(shape, h, e, (0.5,) * dim, width)[None]
    cuts = (W.uniform_cuts(n, parts),) * dim
    return W.Workload(f"conv-{dim}d-{n}", shape, h, cuts, ov, npml, 50.0, 2.0, k, c, f)


def _ddm_error(wl, dim, nsteps, width, r_lo, r_hi):
    s = D.Solver(wl, precision=D.DDM_FP64).factor()
    b = torch.zeros(wl.c.shape, dtype=torch.complex128, device="cuda")
    D.ddm_rhs(s.ctx, s.to_dev(wl.f[0]), b, 1)
    w = torch.zeros_like(b)
    D.ddm_steps(s.ctx, b, nsteps, w, None, want_res=False)
    u = w.cpu().numpy()
    s.close()
    e = wl.ov + wl.npml
    x = (np.arange(-e, wl.n[0] + e) + 0.5) * wl.h
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    r = np.sqrt(sum((g - 0.5) ** 2 for g in grids))
    ring = (r > r_lo) & (r < r_hi)
    k = wl.omega
    damp = math.exp(-(k * width) ** 2 / 2)
    if dim == 2:
        exact = -(0.25j) * scipy_special.hankel1(0, k * r[ring]) * damp
    else:
        exact = -np.exp(1j * k * r[ring]) / (4 * math.pi * r[ring]) * damp
    return float(np.linalg.norm(u[ring] - exact) / np.linalg.norm(exact)), u


def test_table1_scaled_2d_rate_two_through_the_gpu_ddm():
    k, width, parts = 2 * math.pi * 5.0, 0.03, 5
    errs = []
    for n in (80, 160, 320):
        wl = _workload(2, n, parts, k, width, ov=2, npml=n // 16)
        err, u = _ddm_error(wl, 2, 2 * parts, width, 0.15, 0.35)
        errs.append(err)
        if n == 80:          # the GPU iterates are Algorithm 3.1's (the oracle, to rounding)
            o = oracle_of(wl)
            ref = o.run(o.rhs(wl.f[0]), 2 * parts)["w"]
            assert rel(u, ref) < 1e-10
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print(f"\n2D scaled Table 1: errors {errs}, rates {rates}")
    assert errs[-1] < 1e-2, errs
    for r in rates:
        assert abs(r - TABLE_RATE) < 0.35, (errs, rates)


def test_table2_scaled_3d_rate_about_two_through_the_gpu_ddm():
    k, width, parts = 2 * math.pi * 1.5, 0.06, 3
    errs = []
    for n in (24, 48):
        wl = _workload(3, n, parts, k, width, ov=1, npml=n // 8)
        err, u = _ddm_error(wl, 3, 3 * parts, width, 0.3, 0.45)
        errs.append(err)
    rate = math.log2(errs[0] / errs[1])
    print(f"\n3D scaled Table 2: errors {errs}, rate {rate}")
    assert errs[1] < errs[0] and errs[1] < 0.06, errs
    assert rate > 1.5, (errs, rate)
