"""Serving: continuous batching with HBM-budget admission.  Each request's result is the same
when it runs alone and when it runs in the mix with others (within 1e-12: the kernels are
deterministic and each request has its own context and stream)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300.serving import DDMServer, request_workload  # noqa: E402


def reqs():
    return [request_workload(64, 1, 11, sub=32), request_workload(96, 3, 12, sub=32),
            request_workload(128, 2, 13, sub=32), request_workload(64, 4, 14, sub=16)]


def test_results_same_alone_and_in_the_mix():
    wls = reqs()
    alone = DDMServer(max_active=1, K=8, restart=20)
    ids = [alone.submit(w, tol=1e-8) for w in wls]
    assert alone.wait(ids, timeout=300)
    ref = [alone.poll(i).result for i in ids]
    st1 = alone.stats()
    alone.shutdown()
    assert st1["completed"] == 4 and st1["peak_active"] == 1
    mix = DDMServer(max_active=4, K=8, restart=20)
    ids = [mix.submit(w, tol=1e-8) for w in wls]
    assert mix.wait(ids, timeout=300)
    st = mix.stats()
    mix.shutdown()
    assert st["completed"] == 4 and st["failed"] == 0, [mix.poll(i).error for i in ids]
    for i, r in zip(ids, ref):
        got = mix.poll(i)
        assert got.info["converged"] and got.info["rel_residual"] <= 1e-8
        assert np.linalg.norm(got.result - r) <= 1e-12 * np.linalg.norm(r)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # the mix really ran together: several requests were admitted at once and their
    # admission-to-completion intervals overlap in time
    assert st["peak_active"] > 1, st
    spans = sorted((mix.poll(i).t_admit, mix.poll(i).t_done) for i in ids)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1)), spans


def test_budget_admission_serialises_and_rejects():
    wls = reqs()[:3]
    probe = DDMServer(max_active=4)
    need = max(probe.footprint(w) for w in wls)
    probe.shutdown()
    srv = DDMServer(max_active=4, hbm_budget=int(need * 1.2), K=8, restart=20)
    ids = [srv.submit(w, tol=1e-7) for w in wls]
    assert srv.wait(ids, timeout=300)
    st = srv.stats()
    assert st["completed"] == 3 and st["peak_active"] == 1      # only one fits at a time
    big = request_workload(256, 4, 15)
    with pytest.raises(D.DDMError) as ei:
        srv.submit(big)
    assert ei.value.status == D.DDM_E_BUDGET
    srv.shutdown()


def test_cancel_queued_request():
    srv = DDMServer(max_active=1, K=8, restart=20)
    ids = [srv.submit(w, tol=1e-7) for w in reqs()]
    cancelled = srv.cancel(ids[-1])
    assert srv.wait(ids, timeout=300)
    assert cancelled and srv.poll(ids[-1]).status == "cancelled"
    assert all(srv.poll(i).status == "done" for i in ids[:-1])
    srv.shutdown()
