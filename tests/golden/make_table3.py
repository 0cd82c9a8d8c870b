"""Write the oracle's Table 3 records (the FP64 oracle only, no CUDA path involved).

    python tests/golden/make_table3.py [N ...]        (default: 2 4)

For the paper's iterative-solver experiment (Section 4.2.1, Table 3: N x N subdomains of 300^2
own nodes plus a 30-node overlap + PML band, constant medium, omega / 2 pi = 5 + 25 N, single
shot in the first subdomain, tolerance 1e-8) it runs Algorithm 3.1 as an iterative solver in the
oracle and stores, per N, the number of DDM steps to 1e-8 and the relative-residual history
(oracle_table3.json).  The GPU tests compare the library's FP64 stepping solver with it.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.ddm import DDMOracle  # noqa: E402
from oracle.krylov import ddm_stepping  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def record(N, workers):
    wl = W.paper_table3(N)
    t0 = time.time()
    o = DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c, workers=workers)
    res = ddm_stepping(o, o.rhs(wl.f[0]), tol=1e-8, max_steps=40 * N)
    return {"workload": wl.name, "parts": N, "omega_over_2pi": W.TABLE3_FREQ[N], "tol": 1e-8,
            "ddm_steps": res["steps"], "converged": res["converged"],
            "history": [float(v) for v in res["history"]], "oracle_seconds": time.time() - t0,
            "source": "tests/golden/make_table3.py: oracle/ (FP64 numpy/scipy) only"}


if __name__ == "__main__":
    Ns = [int(a) for a in sys.argv[1:]] or [2, 4]
    workers = int(os.environ.get("ORACLE_WORKERS", os.cpu_count() or 1))
    path = os.path.join(HERE, "oracle_table3.json")
    out = {}
    if os.path.exists(path):
        with open(path) as fh:
            out = json.load(fh)
    for N in Ns:
        out[str(N)] = record(N, workers)
        print(N, out[str(N)]["ddm_steps"], f"{out[str(N)]['oracle_seconds']:.0f}s", flush=True)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
