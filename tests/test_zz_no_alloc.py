"""GPU tests of the allocation-free norm entry point (ddm_norms_noalloc).

Some callers cannot allocate device memory where they need a vector norm: code under a fixed
device-memory budget, code running inside a caching allocator that must not be re-entered, or a
section where cudaMalloc's implicit device synchronisation would stall other streams.  They call
ddm_norms_noalloc, whose reduction scratch is a static device array of the library.

The results are compared with numpy.linalg.norm of host copies of the same vectors, within the
1e-12 relative tolerance the FP64 tests use, on two calls in a row (the second call reuses the
scratch the first left behind).  One case runs the entry point as the first library call of a
fresh process, so that its once-per-device address lookup is exercised on its own.  This file
is collected last, so that a run stopping at the first failure has run every other test.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1807_04180_gb300 import ddm as D  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_twice(n, nvec, stream=None):
    rng = np.random.default_rng(5 + n + nvec)
    for call in range(2):
        x = rng.standard_normal((nvec, n)) * (call + 1) + 1j * rng.standard_normal((nvec, n))
        xd = torch.as_tensor(x, dtype=torch.complex128, device="cuda")
        out = torch.full((nvec,), -1.0, dtype=torch.float64, device="cuda")
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                D.ddm_norms_noalloc(xd, n, nvec, out, stream=stream)
            stream.synchronize()
        else:
            D.ddm_norms_noalloc(xd, n, nvec, out)
            torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = np.linalg.norm(x, axis=1)
        assert np.all(np.abs(got - ref) <= 1e-12 * ref), (call, n, nvec, got, ref)


def test_noalloc_norms_match_numpy_twice():
    _check_twice(n=3 * 1000 + 17, nvec=2)


def test_noalloc_sixteen_vectors_wrapping_grid_stride_on_a_side_stream():
    # n above 304 blocks x 256 threads: every thread of the reduction takes several elements
    _check_twice(n=304 * 256 * 3 + 101, nvec=16, stream=torch.cuda.Stream())


def test_noalloc_first_call_in_a_fresh_process():
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_1807_04180_gb300 import ddm as D\n"
        "rng = np.random.default_rng(9)\n"
        "x = rng.standard_normal((3, 5000)) + 1j * rng.standard_normal((3, 5000))\n"
        "xd = torch.as_tensor(x, device='cuda')\n"
        "for call in range(2):\n"
        "    out = torch.zeros(3, dtype=torch.float64, device='cuda')\n"
        "    D.ddm_norms_noalloc(xd, 5000, 3, out)\n"
        "    torch.cuda.synchronize()\n"
        "    ref = np.linalg.norm(x, axis=1)\n"
        "    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-12 * ref), (out, ref)\n"
        "print('fresh-process ok')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "fresh-process ok" in r.stdout, r.stdout + r.stderr


def test_noalloc_rejects_more_vectors_than_its_scratch_holds():
    x = torch.zeros((17, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDMError) as ei:
        D.ddm_norms_noalloc(x, 8, 17, out)
    assert ei.value.status == D.DDM_E_INVAL and "16" in D.ddm_last_error(None)
