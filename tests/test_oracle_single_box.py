"""CPU pin of the single-box oracle the full-size GPU tests use: a subdomain's operator in a
partition equals the operator of the one-subdomain problem built on its own box and medium
window, exactly (same sparse entries), in 2D over uneven cuts and a heterogeneous medium and
in 3D over a constant one."""
import numpy as np

from gpu_helpers import oracle_of, single_box_oracle
from paper_1807_04180_gb300 import workloads as W


def _same(a, b):
    d = (a - b).tocoo()
    return d.nnz == 0 or np.max(np.abs(d.data)) == 0.0


def test_single_box_operator_equals_partition_subdomain_2d():
    wl = W.tiny_2d(seed=4, n=40, parts=(3, 3), ov=2, npml=4)
    wl.cuts = (np.array([0, 11, 27, 40]), np.array([0, 15, 24, 40]))
    o = oracle_of(wl)
    for R in [(0, 0), (1, 2), (2, 1), (1, 1)]:
        ob, R0 = single_box_oracle(wl, R)
        assert ob.sub_shape[R0] == o.sub_shape[R]
        assert _same(ob.sub_A[R0], o.sub_A[R]), R


def test_single_box_operator_equals_partition_subdomain_3d():
    wl = W.tiny_3d(seed=5, n=16, parts=(2, 2, 2), ov=1, npml=3, medium="const")
    o = oracle_of(wl)
    for R in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        ob, R0 = single_box_oracle(wl, R)
        assert _same(ob.sub_A[R0], o.sub_A[R]), R
