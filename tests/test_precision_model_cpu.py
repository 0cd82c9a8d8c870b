"""A CPU model of the split-TF32 products of the tensor-core local solves.

Each FP32 operand is split as x = hi + lo with hi = x with its low 13 mantissa bits cleared (a
TF32 value) and lo = x - hi (exact in FP32); the tensor core reads every operand as TF32, so lo
also loses its low 13 bits.  The product is hi*hi' + hi*lo' + lo*hi', each term exact in FP32
(two 11-bit significands), accumulated in FP32.  The model checks the accuracy claim behind the
mixed-precision local solves: the split product stays within a small factor of a plain FP32
product's error against the exact one, while a single TF32 product is about 2^10 worse.
(The accumulation order of the hardware is not modelled; any order gives FP32-level rounding.)
"""
import numpy as np


def tf32(x):
    """Round toward zero to TF32: clear the low 13 of the 23 FP32 mantissa bits."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = tf32(x)
    lo = (x - hi).astype(np.float32)                 # exact in FP32
    return hi, lo


def matvec_fp32_accumulate(terms):
    """sum_j a_j b_j over the last axis, each product exact, accumulated in FP32 in j order."""
    acc = np.zeros(terms[0][0].shape[0], dtype=np.float32)
    for a, b in terms:
        for j in range(a.shape[1]):
            acc = (acc + (a[:, j].astype(np.float64) * b[j]).astype(np.float32)).astype(np.float32)
    return acc


def split_tf32_matvec(G, y):
    gh, gl = split(G)
    yh, yl = split(y)
    return matvec_fp32_accumulate([(gh, yh), (gh, tf32(yl)), (tf32(gl), yh)])


def test_split_tf32_is_fp32_level():
    rng = np.random.default_rng(7)
    b = 88
    errs_split, errs_fp32, errs_tf32 = [], [], []
    for _ in range(20):
        G = rng.standard_normal((b, b)).astype(np.float32)
        y = rng.standard_normal(b).astype(np.float32)
        exact = G.astype(np.float64) @ y.astype(np.float64)
        ref = np.linalg.norm(exact)
        s = split_tf32_matvec(G, y)
        p = matvec_fp32_accumulate([(G, y)])
        t = matvec_fp32_accumulate([(tf32(G), tf32(y))])
        errs_split.append(np.linalg.norm(s - exact) / ref)
        errs_fp32.append(np.linalg.norm(p - exact) / ref)
        errs_tf32.append(np.linalg.norm(t - exact) / ref)
    e_s, e_p, e_t = np.median(errs_split), np.median(errs_fp32), np.median(errs_tf32)
    assert e_s < 5 * e_p, (e_s, e_p)                  # FP32 level (the GPU tests allow 10x)
    assert e_s < 1e-6
    assert e_t > 100 * e_s, (e_t, e_s)                # one TF32 product alone is far coarser


def test_split_is_exact_and_hi_is_tf32():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(10000) * 10.0 ** rng.integers(-20, 20, 10000)).astype(np.float32)
    hi, lo = split(x)
    assert np.array_equal((hi.astype(np.float64) + lo.astype(np.float64)).astype(np.float32), x)
    assert np.all(hi.view(np.uint32) & np.uint32(0x1FFF) == 0)
    # |lo| < one TF32 unit in the last place of hi: below 2^-10 |x|
    nz = x != 0
    assert np.all(np.abs(lo[nz]) <= np.abs(x[nz]) * 2.0 ** -10)
