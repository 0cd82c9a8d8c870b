"""Write full-size golden records from the FP64 oracle only (no CUDA path involved).

    python tests/golden/make_golden.py heterogeneous-1024 [K]

For the 2D heterogeneous workload (1024^2 interior, 16x16 subdomains, K DDM steps per
preconditioner application (default 2), restart 60) it
runs the oracle's DDM-preconditioned FGMRES to a relative residual of 1e-10 and stores: the
residual-estimate history (so the iteration count to 1e-6 is the first entry <= 1e-6), and the
solution at 512 seeded interior nodes plus the 64 nodes around the source.  The GPU tests
compare the CUDA solution there; bench.py's reference arm reads the iteration count.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.ddm import DDMOracle  # noqa: E402
from oracle.krylov import ddm_fgmres  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def sample_indices(gshape, e, f, seed=7, count=512):
    rng = np.random.default_rng(seed)
    ny, nx = gshape
    ys = rng.integers(e, ny - e, count)
    xs = rng.integers(e, nx - e, count)
    idx = list(ys * nx + xs)
    sy, sx = np.unravel_index(np.argmax(np.abs(f)), gshape)
    for dy in range(-4, 4):
        for dx in range(-4, 4):
            idx.append((sy + dy) * nx + (sx + dx))
    return np.array(idx, dtype=np.int64)


def heterogeneous_1024(workers, K):
    wl = W.heterogeneous_2d()
    wl.K = K
    t0 = time.time()
    o = DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c, workers=workers)
    o.factor()
    b = o.rhs(wl.f[0])
    res = ddm_fgmres(o, b, K=wl.K, tol=1e-10, restart=wl.restart, max_it=600)
    x = res["x"]
    r = np.linalg.norm(b - o.apply_global(x)) / np.linalg.norm(b)
    idx = sample_indices(o.gshape, o.e, wl.f[0])
    hist = [float(v) for v in res["history"]]
    it6 = next(i + 1 for i, v in enumerate(hist) if v <= 1e-6)
    return {
        "workload": wl.name, "K": wl.K, "restart": wl.restart,
        "source": "tests/golden/make_golden.py: oracle/ (FP64 numpy/scipy) only",
        "fgmres_history": hist, "fgmres_iters_to_1e-6": it6, "fgmres_iters_to_1e-10": res["iters"],
        "explicit_rel_residual": float(r), "sample_index": idx.tolist(),
        "sample_re": x.ravel()[idx].real.tolist(), "sample_im": x.ravel()[idx].imag.tolist(),
        "oracle_seconds": time.time() - t0, "workers": workers,
    }


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "heterogeneous-1024"
    K = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    workers = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    out = {"heterogeneous-1024": heterogeneous_1024}[which](workers, K)
    path = os.path.join(HERE, f"oracle_{which}.json" if K == 2 else f"oracle_{which}_K{K}.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(path, out["fgmres_iters_to_1e-6"], out["fgmres_iters_to_1e-10"], out["explicit_rel_residual"],
          f"{out['oracle_seconds']:.0f}s")
