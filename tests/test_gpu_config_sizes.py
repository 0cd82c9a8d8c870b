"""Local-solve parity at the full sizes of the two multi-right-hand-side workloads, in the launch
configuration bench.py times (Algorithm 3.1's batched local solves, Eqs. (37)/(38)).

* 3D constant 192^3, 8x8x8 subdomains of 24^3 + 1 overlap + 6 PML: one shared factor of 38
  plane blocks 1444 wide, every plane step a contraction over all 512 subdomain columns (the
  tensor-core kernels tile it in 12 row tiles with split K; the CUDA-core kernels too).
* 2D layered 2048^2, 32x32 subdomains of uneven widths (extended 80..97 nodes per axis), 64
  right-hand sides per subdomain on the tensor cores (64 per CTA) and on the CUDA cores.

The oracle cannot build these problems whole on the host, so it solves the sampled subdomains
one at a time with the single-box oracle (its operator equals the subdomain's in the partition,
pinned on the CPU in test_oracle_single_box.py).  Sources are random on the sampled subdomains
and zero elsewhere; the comparison is element by element on each sampled subdomain.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import rel, single_box_oracle  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402

# FP32 local solves: the bound the 2D full-size test uses (complex64 factors and sweeps)
TOL_FP32 = 5e-4


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _run(s, lay, srcs, nrhs):
    """Local solve of nrhs right-hand sides with srcs {(sub, r): array} (zero elsewhere);
    returns {(sub, r): solution}."""
    total = lay["total"]
    src = torch.zeros(total * nrhs, dtype=torch.complex64, device="cuda")
    for (sid, r), a in srcs.items():
        n = a.size
        o = lay["offsets"][sid] * nrhs + r * n
        src[o: o + n] = torch.as_tensor(a.ravel().astype(np.complex64), device="cuda")
    u = torch.zeros_like(src)
    D.ddm_local_solve(s.ctx, src, u, nrhs)
    torch.cuda.synchronize()
    out = {}
    for (sid, r), a in srcs.items():
        n = a.size
        o = lay["offsets"][sid] * nrhs + r * n
        out[(sid, r)] = u[o: o + n].cpu().numpy().reshape(a.shape)
    return out


def _sid(wl, R):
    """Library subdomain index of oracle index R (C order, x fastest = last array axis)."""
    parts = [len(c) - 1 for c in wl.cuts]
    sid = 0
    for a in range(len(R)):
        sid = sid * parts[a] + R[a]
    return sid


def test_constant_3d_192_sampled_local_solves_tc_and_cuda_cores():
    wl = W.constant_3d()
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=1).factor()
    lay = D.ddm_local_layout(s.ctx)
    assert lay["n_sub"] == 512
    sample = [(0, 0, 0), (0, 3, 7), (4, 5, 2), (7, 7, 7)]
    rng = np.random.default_rng(31)
    ob, R0 = single_box_oracle(wl, sample[0])     # every subdomain has this operator (constant c)
    shape = ob.sub_shape[R0]
    assert shape == (38, 38, 38)
    srcs = {(_sid(wl, R), 0): cplx(rng, shape) for R in sample}
    ref = {k: ob.local_solve(R0, a) for k, a in srcs.items()}
    errs = {}
    for tc in (True, False):
        D.ddm_set_tensor_cores(s.ctx, tc)
        got = _run(s, lay, srcs, 1)
        errs[tc] = max(rel(got[k], ref[k]) for k in srcs)
    assert errs[True] < TOL_FP32 and errs[False] < TOL_FP32, errs
    # split TF32 carries about 21 bits against FP32's 24: within a small factor of the CUDA cores
    assert errs[True] < 10 * errs[False] + 1e-6, errs
    s.close()


def test_layered_2048_batched_sampled_local_solves_tc_and_cuda_cores():
    wl = W.layered_2d_batched()
    nrhs = wl.nrhs
    assert nrhs == 64
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=nrhs).factor()
    lay = D.ddm_local_layout(s.ctx)
    ext = np.array([e[:2] for e in lay["ext"]])            # (x, y) extents per subdomain
    parts = [len(c) - 1 for c in wl.cuts]                  # array axes (y, x)
    # the widest and the narrowest blocks (x extent = the factor's block width b), the largest
    # and smallest subdomains, a corner and an interior one
    picks = {int(np.argmax(ext[:, 0])), int(np.argmin(ext[:, 0])), int(np.argmax(ext[:, 0] * ext[:, 1])),
             int(np.argmin(ext[:, 0] * ext[:, 1])), 0, (parts[0] // 2) * parts[1] + parts[1] // 3}
    sample = sorted(picks)
    rhs_cmp = (0, 17, 63)
    rng = np.random.default_rng(32)
    srcs, ref = {}, {}
    for sid in sample:
        R = (sid // parts[1], sid % parts[1])
        ob, R0 = single_box_oracle(wl, R)
        shape = ob.sub_shape[R0]
        assert shape == (ext[sid, 1], ext[sid, 0])
        for r in range(nrhs):
            srcs[(sid, r)] = cplx(rng, shape)
        for r in rhs_cmp:
            ref[(sid, r)] = ob.local_solve(R0, srcs[(sid, r)])
    errs = {}
    for nr in (64, 4):                                      # tensor cores, CUDA cores
        D.ddm_set_rhs_per_cta(s.ctx, nr)
        got = _run(s, lay, srcs, nrhs)
        errs[nr] = max(rel(got[k], ref[k]) for k in ref)
    assert errs[64] < TOL_FP32 and errs[4] < TOL_FP32, errs
    assert errs[64] < 10 * errs[4] + 1e-6, errs
    s.close()
