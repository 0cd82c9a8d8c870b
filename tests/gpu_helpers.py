"""Helpers shared by the GPU tests: oracle construction and local-layout conversion."""
import numpy as np

from oracle.ddm import DDMOracle


def oracle_of(wl, workers=1):
    return DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c, workers=workers)


def to_local(o, per_sub, dtype=np.complex128):
    """Concatenate per-subdomain arrays in the library's local layout (subdomains in C order of
    their index, each x-fastest), which is the oracle's subdomain order and array order."""
    return np.concatenate([np.asarray(per_sub[R], dtype=dtype).ravel() for R in o.subs])


def from_local(o, flat):
    out, ofs = {}, 0
    for R in o.subs:
        n = int(np.prod(o.sub_shape[R]))
        out[R] = np.asarray(flat[ofs: ofs + n]).reshape(o.sub_shape[R])
        ofs += n
    return out


def to_local_batch(o, per_rhs, dtype=np.complex128):
    """Local vectors of several right-hand sides (a list of per-subdomain dicts) in the library's
    multi-right-hand-side layout: subdomain-major, the vectors of one subdomain adjacent."""
    return np.concatenate([np.asarray(sr[R], dtype=dtype).ravel() for R in o.subs for sr in per_rhs])


def from_local_batch(o, flat, nrhs):
    """Inverse of to_local_batch: a list of nrhs per-subdomain dicts."""
    out, ofs = [dict() for _ in range(nrhs)], 0
    for R in o.subs:
        n = int(np.prod(o.sub_shape[R]))
        for r in range(nrhs):
            out[r][R] = np.asarray(flat[ofs: ofs + n]).reshape(o.sub_shape[R])
            ofs += n
    return out


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def single_box_oracle(wl, R):
    """An oracle whose whole problem is subdomain R of ``wl``: its interior is R's own box and
    its medium R's window of the global wave speed, so its one subdomain operator is R's
    operator in the full partition (box-relative PML tables, the same h, omega and k^2).  Lets
    a test solve one subdomain of a workload too large to build whole on the host."""
    d = len(wl.n)
    e = wl.ov + wl.npml
    lo = [int(wl.cuts[a][R[a]]) for a in range(d)]
    hi = [int(wl.cuts[a][R[a] + 1]) for a in range(d)]
    win = tuple(slice(lo[a], hi[a] + 2 * e) for a in range(d))
    n = [hi[a] - lo[a] for a in range(d)]
    cuts = [np.array([0, n[a]], dtype=np.int64) for a in range(d)]
    return DDMOracle(n, wl.h, cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega,
                     np.ascontiguousarray(wl.c[win])), (0,) * d
