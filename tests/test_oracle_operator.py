"""Pins of the oracle's PML stretching and finite-difference operator.

Each check ties oracle/pml_operator.py to something other than itself:
a textbook Kronecker-sum Laplacian, complex symmetry, a dense library solve,
the free-space Green's functions of Section 2.1 (2D Hankel, 3D e^{ikr}/(4 pi r))
with the second-order convergence the paper reports in Tables 1-2, and the
exponential decay of the PML truncation error in sigma-bar (Eq. (34)).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import hankel1

from oracle.ddm import DDMOracle
from oracle.pml_operator import box_alpha, pml_operator, sigma_profile
from paper_1807_04180_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kron_laplacian(shape):
    """Textbook h^2-scaled Dirichlet Laplacian as a Kronecker sum of 1D tridiag(1,-2,1)."""
    mats = [sp.diags([np.ones(m - 1), -2 * np.ones(m), np.ones(m - 1)], [-1, 0, 1]) for m in shape]
    L = None
    for a, m in enumerate(shape):
        left = sp.identity(int(np.prod(shape[:a]))) if a else None
        right = sp.identity(int(np.prod(shape[a + 1:]))) if a < len(shape) - 1 else None
        term = mats[a]
        if left is not None:
            term = sp.kron(left, term)
        if right is not None:
            term = sp.kron(term, right)
        L = term if L is None else L + term
    return L.tocsr()


@pytest.mark.parametrize("shape", [(7, 9), (4, 5, 6)])
def test_no_pml_is_textbook_laplacian(shape):
    """With sigma = 0 the operator is h^2 (Laplacian + k^2) with Dirichlet ghosts."""
    rng = np.random.default_rng(0)
    h = 0.1
    k2 = rng.uniform(1.0, 4.0, shape)
    an = [np.ones(m, dtype=complex) for m in shape]
    ah = [np.ones(m + 1, dtype=complex) for m in shape]
    A = pml_operator(an, ah, k2, h)
    ref = _kron_laplacian(shape) + sp.diags(h * h * k2.ravel())
    assert abs(A - ref).max() < 1e-14


def test_operator_complex_symmetric_and_dense_solve():
    wl = W.tiny_2d(seed=3)
    o = DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c)
    A = o.A_global.toarray()
    assert np.abs(A - A.T).max() == 0.0
    assert np.abs(A - A.conj().T).max() > 1e-3          # PML makes it non-Hermitian
    b = o.rhs(wl.f[0])
    x_dense = np.linalg.solve(A, b.ravel())
    x = o.global_solve(b).ravel()
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-12


def test_pml_profile_shape():
    """Shifted profile: zero on the overlap band, non-decreasing, sigma0 at the outer edge."""
    ov, npml, s0 = 2, 10, 50.0
    t = np.linspace(0, ov + npml, 241)
    s = sigma_profile(t, ov, npml, s0, 2.0)
    assert np.all(s[t <= ov] == 0) and np.all(np.diff(s) >= 0)
    assert abs(s[-1] - s0) < 1e-12
    a_node, a_half = box_alpha(5, 9, ov + npml, ov, npml, s0, 2.0)
    # inside the box and its overlap band alpha = 1
    assert np.all(a_node[npml: npml + 2 * ov + 4] == 1.0)
    # the profile is symmetric about the box centre
    assert np.allclose(a_node, a_node[::-1]) and np.allclose(a_half, a_half[::-1])


def _green_error_2d(n, k, width, sigma0=8.0):
    h = 1.0 / n
    ov, npml = 2, n // 4
    e = ov + npml
    shape = (n, n)
    c = W.constant_medium(shape, e, 1.0)
    f = W.gaussian_source(shape, h, e, (0.5, 0.5), width)
    o = DDMOracle(shape, h, [[0, n], [0, n]], ov, npml, sigma0, 2.0, k, c)
    u = o.global_solve(o.rhs(f))
    y = (np.arange(-e, n + e) + 0.5) * h
    Y, X = np.meshgrid(y, y, indexing="ij")
    r = np.hypot(Y - 0.5, X - 0.5)
    ring = (r > 0.2) & (r < 0.4)
    exact = -(0.25j) * hankel1(0, k * r[ring]) * math.exp(-(k * width) ** 2 / 2)
    return np.linalg.norm(u[ring] - exact) / np.linalg.norm(exact)


@pytest.mark.slow
def test_green_function_2d_second_order():
    """Section 2.1: Delta u + k^2 u = f has u = -(i/4) H0(k r) * FT[f](k); the 5-point scheme
    converges at rate 2 (Table 1 reports rate 2.0)."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as fh:
        gold = json.load(fh)
    k = 2 * math.pi * 4.0
    errs = [_green_error_2d(n, k, 0.03) for n in (64, 128, 256)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 5e-3, errs
    for r in rates:
        assert abs(r - gold["table1_2d_rate"]["value"]) < 0.35, (errs, rates)


def test_pml_truncation_error_decays_with_sigma():
    """Eq. (34): ||u - u^|| <= C k^2 (1+kL)^2 exp(-k gamma0 sigma_bar / 2), sigma_bar = int sigma.
    At fixed fine mesh the error against the closed form drops as sigma0 grows (until the
    discretisation error takes over)."""
    k = 2 * math.pi * 3.0
    errs = [_green_error_2d(160, k, 0.03, sigma0=s0) for s0 in (0.25, 1.0, 4.0)]
    assert errs[0] > 3 * errs[1] > 0 and errs[1] > errs[2], errs


@pytest.mark.slow
def test_green_function_3d():
    """3D: u = -exp(ikr)/(4 pi r) * FT[f](k) up to O(h^2) (Table 2 reports rate ~2)."""
    k = 2 * math.pi * 1.5
    width = 0.06
    errs = []
    for n in (16, 24):
        h = 1.0 / n
        ov, npml = 1, n // 4
        e = ov + npml
        shape = (n, n, n)
        c = W.constant_medium(shape, e, 1.0)
        f = W.gaussian_source(shape, h, e, (0.5, 0.5, 0.5), width)
        o = DDMOracle(shape, h, [[0, n]] * 3, ov, npml, 6.0, 2.0, k, c)
        u = o.global_solve(o.rhs(f))
        x = (np.arange(-e, n + e) + 0.5) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt((Z - 0.5) ** 2 + (Y - 0.5) ** 2 + (X - 0.5) ** 2)
        ring = (r > 0.3) & (r < 0.45)
        exact = -np.exp(1j * k * r[ring]) / (4 * math.pi * r[ring]) * math.exp(-(k * width) ** 2 / 2)
        errs.append(np.linalg.norm(u[ring] - exact) / np.linalg.norm(exact))
    assert errs[1] < errs[0] and errs[1] < 0.06, errs
    assert math.log(errs[0] / errs[1]) / math.log(24 / 16) > 1.5, errs
