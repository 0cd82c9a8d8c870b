"""PML stretching and the finite-difference PML operator (oracle, FP64).

Test infrastructure: see the package docstring.

Geometry (a reading; the paper only says "uniform rectangular meshes",
Section 4): along every axis the nodes sit at (p + 1/2) h.  A box with own
nodes [lo, hi) (global node indices) has faces at lo*h and hi*h and is
extended by e = ov + npml nodes on each side; homogeneous Dirichlet "ghost"
values sit just beyond the extension.  The global box is the interior [0, n)
extended the same way, so a boundary subdomain's outer PML is the global PML.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import scipy.sparse as sp


def sigma_profile(t: np.ndarray, ov: int, npml: int, sigma0: float, power: float) -> np.ndarray:
    """Shifted PML profile, Eq. (11) of Section 2.1.

    ``t`` is the distance beyond the box face in cells.  sigma = 0 on the
    overlap band t <= d~ (d~ = ov cells); beyond it the medium profile
    sigma~(t - d~) = sigma0 ((t - ov) / npml)^power (the paper leaves sigma~
    open beyond "smooth"; this polynomial is the reading used throughout).
    """
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    m = t > ov
    out[m] = sigma0 * ((t[m] - ov) / npml) ** power
    return out


def box_alpha(lo: int, hi: int, e: int, ov: int, npml: int, sigma0: float, power: float):
    """Stretching factors alpha = 1 + i sigma (Section 2.1) along one axis of a box.

    Returns (alpha_node, alpha_half) on the box's extended node range
    p = lo-e .. hi+e-1: alpha_node[j] at node p = lo-e+j (position (p+1/2)h),
    alpha_half[j] at the half node between ext nodes j-1 and j (position
    (lo-e+j) h), j = 0..m, where j = 0 and j = m are the half nodes next to the
    Dirichlet ghosts.
    """
    p = np.arange(lo - e, hi + e, dtype=np.float64)
    pos_node = p + 0.5
    pos_half = np.arange(lo - e, hi + e + 1, dtype=np.float64)

    def dist(pos):
        return np.maximum(np.maximum(lo - pos, pos - hi), 0.0)

    a_node = 1.0 + 1j * sigma_profile(dist(pos_node), ov, npml, sigma0, power)
    a_half = 1.0 + 1j * sigma_profile(dist(pos_half), ov, npml, sigma0, power)
    return a_node, a_half


def _bcast(v: np.ndarray, axis: int, ndim: int) -> np.ndarray:
    shape = [1] * ndim
    shape[axis] = v.shape[0]
    return v.reshape(shape)


def pml_operator(alpha_node: Sequence[np.ndarray], alpha_half: Sequence[np.ndarray],
                 k2: np.ndarray, h: float) -> sp.csr_matrix:
    """h^2 J L_B: the J-scaled 5-point (2D) / 7-point (3D) PML operator on a box.

    Eq. (9) with A = diag(J / alpha_a^2) and J = prod_a alpha_a reads
    J L u = sum_a d/dx_a( (prod_{b != a} alpha_b) / alpha_a du/dx_a ) + k^2 J u;
    since prod_{b != a} alpha_b does not depend on x_a it stays outside the
    derivative.  Central differences on the node grid give, at node x,

      (A u)(x) = sum_a (prod_{b!=a} alpha_b(x_b)) *
                   [ (u(x+e_a) - u(x)) / alpha_a(x_a + 1/2)
                   - (u(x) - u(x-e_a)) / alpha_a(x_a - 1/2) ]
                 + h^2 k^2(x) prod_a alpha_a(x_a) u(x),

    with u = 0 beyond the box's extended grid (homogeneous Dirichlet, the
    truncated problem of Section 3.1).  The matrix is complex symmetric and is
    the discrete weak form (Eq. (10)) up to sign.  Rows/cols follow the C
    order of ``k2`` (last axis fastest).
    """
    shape = k2.shape
    d = len(shape)
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    a_node = [_bcast(np.asarray(alpha_node[a]), a, d) for a in range(d)]
    J = np.ones(shape, dtype=np.complex128)
    for a in range(d):
        J = J * a_node[a]
    diag = (h * h) * k2 * J
    rows, cols, vals = [], [], []
    for a in range(d):
        others = np.ones(shape, dtype=np.complex128)
        for b in range(d):
            if b != a:
                others = others * a_node[b]
        ah = np.asarray(alpha_half[a])
        c_plus = others / _bcast(ah[1:], a, d)     # coupling to x + e_a
        c_minus = others / _bcast(ah[:-1], a, d)   # coupling to x - e_a
        diag = diag - c_plus - c_minus
        m = shape[a]
        lo_sl = [slice(None)] * d
        hi_sl = [slice(None)] * d
        lo_sl[a] = slice(0, m - 1)
        hi_sl[a] = slice(1, m)
        lo_sl, hi_sl = tuple(lo_sl), tuple(hi_sl)
        rows.append(idx[lo_sl].ravel()); cols.append(idx[hi_sl].ravel()); vals.append(c_plus[lo_sl].ravel())
        rows.append(idx[hi_sl].ravel()); cols.append(idx[lo_sl].ravel()); vals.append(c_minus[hi_sl].ravel())
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()


def jacobian(alpha_node: Sequence[np.ndarray], shape) -> np.ndarray:
    """J = prod_a alpha_a at the nodes of a box (Section 2.1)."""
    d = len(shape)
    J = np.ones(shape, dtype=np.complex128)
    for a in range(d):
        J = J * _bcast(np.asarray(alpha_node[a]), a, d)
    return J
