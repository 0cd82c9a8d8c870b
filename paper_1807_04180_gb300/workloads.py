"""Seeded synthetic inputs for the overlapping-DDM Helmholtz solver.

This module only *draws* inputs: wave-speed fields c(x), source fields f(x)
and partition cut positions.  It holds none of the method's arithmetic (no
PML, no operator, no transfer, no solve), so that both the CUDA path and the
FP64 CPU oracle can be fed the very same arrays without sharing any code that
computes the method.

Conventions shared by every array produced here
-----------------------------------------------
* Arrays are C-ordered with the physical x axis LAST: 2D fields have shape
  (ny, nx), 3D fields (nz, ny, nx).  Partition cuts are given per array axis.
* The interior (physical) grid has ``n`` nodes per axis, spacing ``h`` and
  node p at coordinate (p + 1/2) h (cell-centred nodes on [0, n h]).
* Fields that the solver needs beyond the interior (the wave speed) are given
  on the *extended* grid, which adds ``e`` nodes on every side; the wave speed
  is continued outward by the nearest interior value (constant along the
  normal).  Sources are zero outside the interior.

Workload recipes follow the experiments of Leng & Ju (2018), Section 4: a
Gaussian or single-shot point source, about 10 points per wavelength, fixed
subdomain size as the subdomain count grows, and synthetic media standing in
for the paper's layered model (which is only shown as a figure there).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------
# coordinates
# ----------------------------------------------------------------------------
def node_coords(n: int, h: float) -> np.ndarray:
    """Coordinates (p + 1/2) h of the interior nodes p = 0..n-1 along one axis."""
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _mesh(shape: Sequence[int], h: float):
    axes = [node_coords(m, h) for m in shape]
    return np.meshgrid(*axes, indexing="ij")


def extend_edge(field: np.ndarray, e: int) -> np.ndarray:
    """Continue an interior field by ``e`` nodes per side with its nearest value."""
    return np.pad(field, e, mode="edge")


# ----------------------------------------------------------------------------
# media
# ----------------------------------------------------------------------------
def constant_medium(shape: Sequence[int], e: int, c0: float = 1.0) -> np.ndarray:
    return np.full([m + 2 * e for m in shape], float(c0), dtype=np.float64)


def gaussian_sum_medium(shape: Sequence[int], h: float, e: int, seed: int,
                        n_bumps: int = 20, cmin: float = 1.5, cmax: float = 4.5) -> np.ndarray:
    """c(x) = cmin + (cmax-cmin) * normalise(sum_m a_m exp(-|x-x_m|^2 / (2 w_m^2))).

    a_m ~ U[-1,1], x_m ~ U[0,L]^d, w_m ~ U[0.03,0.15] L with L = n h (per axis
    the largest extent).  normalise maps the field's min/max to 0/1.
    """
    rng = np.random.default_rng(seed)
    L = max(shape) * h
    d = len(shape)
    a = rng.uniform(-1.0, 1.0, n_bumps)
    xm = rng.uniform(0.0, L, (n_bumps, d))
    wm = rng.uniform(0.03, 0.15, n_bumps) * L
    X = _mesh(shape, h)
    g = np.zeros(tuple(shape), dtype=np.float64)
    for m in range(n_bumps):
        r2 = sum((X[ax] - xm[m, ax]) ** 2 for ax in range(d))
        g += a[m] * np.exp(-r2 / (2.0 * wm[m] ** 2))
    g = (g - g.min()) / max(g.max() - g.min(), 1e-300)
    return extend_edge(cmin + (cmax - cmin) * g, e)


def layered_medium(shape: Sequence[int], h: float, e: int, seed: int,
                   n_layers: int = 6, cmin: float = 1.5, cmax: float = 4.5) -> np.ndarray:
    """Seeded layered medium with gently curved interfaces.

    Layer l (l = 0..n_layers-1, from the first array axis' low end) has speed
    c_l ~ U[cmin, cmax]; interface l sits at depth z_l(x) = l L / n_layers +
    0.05 L sin(2 pi x k_l / L + phi_l), k_l ~ U[1,3], phi_l ~ U[0, 2 pi).
    Depth runs along the first array axis, x along the last.
    """
    rng = np.random.default_rng(seed)
    d = len(shape)
    L = max(shape) * h
    speeds = rng.uniform(cmin, cmax, n_layers)
    kk = rng.uniform(1.0, 3.0, n_layers)
    ph = rng.uniform(0.0, 2 * math.pi, n_layers)
    X = _mesh(shape, h)
    depth, xx = X[0], X[d - 1]
    layer = np.zeros(tuple(shape), dtype=np.int64)
    for l in range(1, n_layers):
        z_l = l * L / n_layers + 0.05 * L * np.sin(2 * math.pi * xx * kk[l] / L + ph[l])
        layer += (depth >= z_l).astype(np.int64)
    return extend_edge(speeds[layer], e)


# ----------------------------------------------------------------------------
# sources (values of f at interior nodes, zero in the extension band)
# ----------------------------------------------------------------------------
def gaussian_source(shape: Sequence[int], h: float, e: int, center: Sequence[float],
                    width: float) -> np.ndarray:
    """Unit-mass Gaussian f = (2 pi s^2)^(-d/2) exp(-|x-x0|^2 / (2 s^2)), s = width."""
    d = len(shape)
    X = _mesh(shape, h)
    r2 = sum((X[ax] - center[ax]) ** 2 for ax in range(d))
    f = (2 * math.pi * width ** 2) ** (-d / 2) * np.exp(-r2 / (2 * width ** 2))
    return np.pad(f.astype(np.complex128), e)


def point_source(shape: Sequence[int], h: float, e: int, position: Sequence[float]) -> np.ndarray:
    """Discrete delta of unit mass, 1/h^d, at the interior node nearest ``position``."""
    d = len(shape)
    f = np.zeros([m + 2 * e for m in shape], dtype=np.complex128)
    idx = tuple(int(min(max(round(position[ax] / h - 0.5), 0), shape[ax] - 1)) + e for ax in range(d))
    f[idx] = 1.0 / h ** d
    return f


def random_point_sources(shape: Sequence[int], h: float, e: int, count: int, seed: int) -> np.ndarray:
    """``count`` single-node unit-mass sources at seeded uniform interior positions."""
    rng = np.random.default_rng(seed)
    L = np.array(shape, dtype=np.float64) * h
    out = np.zeros([count] + [m + 2 * e for m in shape], dtype=np.complex128)
    for r in range(count):
        out[r] = point_source(shape, h, e, rng.uniform(0.05, 0.95, len(shape)) * L)
    return out


# ----------------------------------------------------------------------------
# partitions
# ----------------------------------------------------------------------------
def uniform_cuts(n: int, parts: int) -> np.ndarray:
    if n % parts:
        raise ValueError(f"{n} nodes do not split into {parts} equal parts")
    return np.arange(parts + 1, dtype=np.int64) * (n // parts)


def uneven_cuts(n: int, parts: int, seed: int, jitter: int) -> np.ndarray:
    """Seeded uneven cuts: widths n/parts + U{-jitter..jitter}, then the sum corrected to n by
    +-1 steps on randomly chosen parts, every width staying within n//parts - jitter ..
    n//parts + jitter + 1."""
    rng = np.random.default_rng(seed)
    base = n // parts
    w = base + rng.integers(-jitter, jitter + 1, parts)
    lo, hi = max(1, base - jitter), base + jitter + 1
    while w.sum() != n:
        step = 1 if w.sum() < n else -1
        i = int(rng.integers(parts))
        if lo <= w[i] + step <= hi:
            w[i] += step
    return np.concatenate([[0], np.cumsum(w)]).astype(np.int64)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """One synthetic problem: geometry, PML/overlap widths, medium and sources.

    ``c`` is on the extended grid (shape n+2e per axis); ``f`` has a leading
    right-hand-side axis and the same extended shape (zero outside the interior).
    """
    name: str
    n: Tuple[int, ...]             # interior nodes per array axis (x last)
    h: float
    cuts: Tuple[np.ndarray, ...]   # per array axis, parts+1 node offsets
    ov: int                        # overlap cells (d~ = ov h)
    npml: int                      # PML cells
    sigma0: float
    power: float
    omega: float
    c: np.ndarray
    f: np.ndarray
    tol: float = 1e-6
    K: int = 2
    restart: int = 60
    note: str = ""

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def e(self) -> int:
        return self.ov + self.npml

    @property
    def parts(self) -> Tuple[int, ...]:
        return tuple(len(c) - 1 for c in self.cuts)

    @property
    def nrhs(self) -> int:
        return self.f.shape[0]


def tiny_2d(seed: int = 0, n: int = 12, parts=(2, 2), ov: int = 1, npml: int = 3,
            medium: str = "gauss", k_over_2pi: float = 2.0, nrhs: int = 1) -> Workload:
    """Small 2D case that a dense solve handles: n^2 interior, parts subdomains."""
    h = 1.0 / n
    e = ov + npml
    shape = (n, n)
    if medium == "const":
        c = constant_medium(shape, e)
    else:
        c = gaussian_sum_medium(shape, h, e, seed, n_bumps=4, cmin=1.0, cmax=2.0)
    rng = np.random.default_rng(seed + 1000)
    f = np.stack([gaussian_source(shape, h, e, rng.uniform(0.2, 0.8, 2), 2 * h) for _ in range(nrhs)])
    cuts = tuple(uniform_cuts(n, p) if n % p == 0 else uneven_cuts(n, p, seed, 0) for p in parts)
    return Workload("tiny2d", shape, h, cuts, ov, npml, 10.0, 2.0, 2 * math.pi * k_over_2pi, c, f)


def tiny_3d(seed: int = 0, n: int = 12, parts=(2, 2, 2), ov: int = 1, npml: int = 3,
            medium: str = "gauss", k_over_2pi: float = 1.5) -> Workload:
    """Small 3D case the oracle solves directly: n^3 interior, parts subdomains."""
    h = 1.0 / n
    e = ov + npml
    shape = (n, n, n)
    if medium == "const":
        c = constant_medium(shape, e)
    else:
        c = gaussian_sum_medium(shape, h, e, seed, n_bumps=4, cmin=1.0, cmax=2.0)
    rng = np.random.default_rng(seed + 2000)
    f = gaussian_source(shape, h, e, rng.uniform(0.25, 0.75, 3), 2 * h)[None]
    cuts = tuple(uniform_cuts(n, p) for p in parts)
    return Workload("tiny3d", shape, h, cuts, ov, npml, 10.0, 2.0, 2 * math.pi * k_over_2pi, c, f)


def constant_2d_160(seed: int = 1) -> Workload:
    """2D constant medium, k = 2 pi 10 on [0,1]^2, 160^2 interior, 4x4 subdomains of 40^2,
    2-cell overlap, 10-cell PML (sigma0 = 50, quadratic), Gaussian source of width 2h at a
    seeded location, plain FP64 DDM."""
    n, parts, ov, npml = 160, 4, 2, 10
    h = 1.0 / n
    e = ov + npml
    rng = np.random.default_rng(seed)
    f = gaussian_source((n, n), h, e, rng.uniform(0.1, 0.9, 2), 2 * h)[None]
    return Workload("2d-constant-160", (n, n), h, (uniform_cuts(n, parts),) * 2, ov, npml, 50.0, 2.0,
                    2 * math.pi * 10.0, constant_medium((n, n), e), f, tol=1e-6, K=2)


def heterogeneous_2d(n: int = 1024, parts: int = 16, seed: int = 2, ov: int = 2, npml: int = 10,
                     nrhs: int = 1, ppw: float = 10.0) -> Workload:
    """2D heterogeneous medium: c in [1.5, 4.5] as a seeded sum of 20 Gaussians,
    omega chosen for ``ppw`` points per wavelength at c_min, ``parts``^2 subdomains,
    single-shot source in the first subdomain at (x0 + dxi/4, y0 + deta/3)."""
    h = 1.0 / n
    e = ov + npml
    c = gaussian_sum_medium((n, n), h, e, seed)
    omega = 2 * math.pi * 1.5 / (ppw * h)
    sub = n // parts
    pos = ((sub / 3.0) * h, (sub / 4.0) * h)       # (y, x): y0 + deta/3, x0 + dxi/4
    if nrhs == 1:
        f = point_source((n, n), h, e, pos)[None]
    else:
        f = random_point_sources((n, n), h, e, nrhs, seed)
    return Workload(f"2d-heterogeneous-{n}", (n, n), h, (uniform_cuts(n, parts),) * 2, ov, npml, 50.0, 2.0,
                    omega, c, f, tol=1e-6, K=2, restart=60)


def layered_2d_batched(n: int = 2048, parts: int = 32, seed: int = 3, nrhs: int = 64,
                       jitter: int = 8) -> Workload:
    """2D seeded layered medium, parts^2 subdomains of uneven widths, ``nrhs`` point sources."""
    ov, npml = 2, 10
    h = 1.0 / n
    e = ov + npml
    c = layered_medium((n, n), h, e, seed)
    omega = 2 * math.pi * 1.5 / (10.0 * h)
    cuts = (uneven_cuts(n, parts, seed, jitter), uneven_cuts(n, parts, seed + 1, jitter))
    f = random_point_sources((n, n), h, e, nrhs, seed)
    return Workload(f"2d-layered-{n}-batched", (n, n), h, cuts, ov, npml, 50.0, 2.0, omega, c, f,
                    tol=1e-6, K=2)


def constant_3d(n: int = 192, parts: int = 8, ov: int = 1, npml: int = 6, k_over_2pi: float = 16.0,
                seed: int = 4) -> Workload:
    """3D constant medium, n^3 interior on [0,1]^3, parts^3 subdomains, Gaussian source."""
    h = 1.0 / n
    e = ov + npml
    shape = (n, n, n)
    k = 2 * math.pi * k_over_2pi
    center = (0.5 + 0.125, 0.5 + 0.133, 0.5 + 0.12)     # (z, y, x)
    f = gaussian_source(shape, h, e, center, 2 * h)[None]
    return Workload(f"3d-constant-{n}", shape, h, (uniform_cuts(n, parts),) * 3, ov, npml, 50.0, 2.0, k,
                    constant_medium(shape, e), f, tol=1e-6, K=2)


# Table 3: omega / 2 pi for N x N subdomains of 300^2 (5 + 25 N: 55, 105, 205, 405, 805, 1605)
TABLE3_FREQ = {2: 55.0, 4: 105.0, 8: 205.0, 16: 405.0, 32: 805.0, 64: 1605.0}
# Table 4 (layered medium): 27.5, 52.5, 102.5, ...
TABLE4_FREQ = {2: 27.5, 4: 52.5, 8: 102.5, 16: 202.5, 32: 402.5, 64: 802.5}


def paper_table3(N: int, medium: str = "constant", seed: int = 6, ov: int = 2, npml: int = 28) -> Workload:
    """The paper's iterative-solver experiments (Section 4.2.1, Tables 3-4): N x N subdomains of
    300^2 own nodes on [0, 1]^2 (h = 1 / (300 N)), each extended by overlap + PML = 30 nodes per
    side (b = 360 nodes per x-line), omega / 2 pi from the tables (about 11 points per
    wavelength at c = 1), a single-shot source at (x0 + dxi / 4, y0 + deta / 3) of the first
    subdomain, tolerance 1e-8.  medium "constant": c = 1 (Table 3); "layered": the seeded
    6-layer stand-in for the paper's 5-layer model (Table 4's frequencies, c in [1, 3] so that the
    slowest layer keeps the table's points per wavelength; the model itself exists only as a
    figure)."""
    n = 300 * N
    h = 1.0 / n
    e = ov + npml
    if medium == "constant":
        c = constant_medium((n, n), e, 1.0)
        omega = 2 * math.pi * TABLE3_FREQ[N]
    elif medium == "layered":
        c = layered_medium((n, n), h, e, seed, cmin=1.0, cmax=3.0)
        omega = 2 * math.pi * TABLE4_FREQ[N]
    else:
        raise ValueError("medium must be 'constant' or 'layered'")
    pos = ((300 / 3.0) * h, (300 / 4.0) * h)       # (y, x): y0 + deta/3, x0 + dxi/4
    f = point_source((n, n), h, e, pos)[None]
    return Workload(f"2d-table3-{medium}-{N}x{N}", (n, n), h, (uniform_cuts(n, N),) * 2, ov, npml, 50.0, 2.0,
                    omega, c, f, tol=1e-8, K=2)
