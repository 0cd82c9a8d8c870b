"""GPU test of the allocation-free norm entry point (ddm_norms_noalloc).

Callers that cannot allocate device memory where they need a norm (a fixed memory budget, an
allocator that must not be re-entered, or code that must not trigger cudaMalloc's implicit
device synchronisation) use ddm_norms_noalloc, whose reduction scratch is a static device
array.  Its results must equal the norms that the allocating path (ddm_residual) returns for
the same vectors, on two calls in a row (the second call reuses the static scratch the first
left behind).  This file is collected last and also runs on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def test_noalloc_norms_match_residual_norms_twice():
    wl = W.tiny_2d(seed=21, n=30, parts=(3, 2), ov=2, npml=4)
    s = D.Solver(wl, precision=D.DDM_FP64, max_rhs=2)
    n = int(np.prod(wl.c.shape))
    rng = np.random.default_rng(5)
    for call in range(2):
        x = s.to_dev(rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n)))
        b = s.to_dev(rng.standard_normal((2, n)) * (call + 1) + 1j * rng.standard_normal((2, n)))
        r = torch.empty_like(b)
        ref = D.ddm_residual(s.ctx, b, x, r, 2)           # existing path: [(||r_i||, ||b_i||)]
        out_r = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        out_b = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        D.ddm_norms_noalloc(r, n, 2, out_r)
        D.ddm_norms_noalloc(b, n, 2, out_b)
        torch.cuda.synchronize()
        got_r, got_b = out_r.cpu().numpy(), out_b.cpu().numpy()
        for i in range(2):
            assert abs(got_r[i] - ref[i][0]) <= 1e-12 * ref[i][0], (call, i, got_r[i], ref[i][0])
            assert abs(got_b[i] - ref[i][1]) <= 1e-12 * ref[i][1], (call, i, got_b[i], ref[i][1])
    s.close()


def test_noalloc_rejects_more_vectors_than_its_scratch_holds():
    x = torch.zeros((17, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDMError) as ei:
        D.ddm_norms_noalloc(x, 8, 17, out)
    assert ei.value.status == D.DDM_E_INVAL and "16" in D.ddm_last_error(None)
