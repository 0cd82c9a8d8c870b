"""Host logic of the nested-dissection local solver: the plan (ddm_nd_plan, pure host code).

The paper solves each subdomain problem of Algorithm 3.1 with a sparse direct (multifrontal)
solver (Section 4).  The library's DDM_LOCAL_ND solver orders each subdomain grid by nested
dissection and factors it front by front.  Its plan is checked here without a GPU, against what
the method fixes:

* structure: every node is the pivot of exactly one front; children come before their parents
  and have lower heights; a front's boundary nodes are pivots of its ancestors; each child's
  boundary positions point at the same nodes in the parent's front;
* assembly: the entries cover every nonzero of the subdomain operator exactly once, each with
  the operator plane that holds it;
* a multifrontal factorisation and solve driven by the plan's arrays, written here in numpy
  (a dense inverse of each front's pivot block, Schur complements passed to the parent, update
  vectors up the tree and back-substitution down it), equals the oracle's sparse direct local
  solve (Eqs. (37)/(38)) on the subdomains of a heterogeneous 2D partition with uneven widths,
  for several leaf sizes including one front per subdomain.
"""
import numpy as np
import pytest

from oracle.ddm import DDMOracle
from paper_1807_04180_gb300 import ddm as D
from paper_1807_04180_gb300 import workloads as W


def _nodes(plan, j):
    s, d, _, po, bo = plan["fronts"][j][:5]
    return np.concatenate([plan["piv"][po: po + s], plan["bnd"][bo: bo + d]])


def _neighbour(node, plane, nx):
    return node + {0: 0, 1: -1, 2: 1, 3: -nx, 4: nx}[int(plane)]


def _ancestors(fronts):
    parent = {}
    for j, fr in enumerate(fronts):
        for c in fr[5:7]:
            if c >= 0:
                parent[int(c)] = j
    def anc(j):
        out = []
        while j in parent:
            j = parent[j]
            out.append(j)
        return out
    return anc


@pytest.mark.parametrize("nx,ny,leaf", [(13, 11, 8), (25, 21, 1), (40, 17, 32), (7, 5, 1000), (88, 88, 32)])
def test_plan_structure(nx, ny, leaf):
    p = D.ddm_nd_plan(nx, ny, leaf)
    fr = p["fronts"]
    assert p["nfront"] == len(fr) and fr[-1][2] == p["height"]
    assert np.array_equal(np.sort(p["piv"]), np.arange(nx * ny))          # each node pivots once
    anc = _ancestors(fr)
    owner = np.empty(nx * ny, int)
    for j, f in enumerate(fr):
        owner[p["piv"][f[3]: f[3] + f[0]]] = j
    total_m_s = 0
    for j, f in enumerate(fr):
        s, d, h = int(f[0]), int(f[1]), int(f[2])
        total_m_s += (s + d) * s
        kids = [int(c) for c in f[5:7] if c >= 0]
        assert all(c < j and fr[c][2] < h for c in kids)
        assert h == (max(fr[c][2] for c in kids) + 1 if kids else 0)
        bnd = p["bnd"][f[4]: f[4] + d]
        assert np.all(np.diff(bnd) > 0)
        assert set(owner[bnd].tolist()) <= set(anc(j))                    # boundary = ancestors' pivots
        nodes = _nodes(p, j)
        for c in kids:
            slot = 7 if c == f[5] else 8
            cpos = p["cmap"][f[slot]: f[slot] + fr[c][1]]
            cbnd = p["bnd"][fr[c][4]: fr[c][4] + fr[c][1]]
            assert np.array_equal(nodes[cpos], cbnd)
    assert fr[-1][1] == 0                                                  # the root has no boundary
    assert p["factor_entries"] == total_m_s


@pytest.mark.parametrize("nx,ny,leaf", [(13, 11, 8), (25, 21, 1), (40, 17, 32)])
def test_plan_entries_cover_the_operator_once(nx, ny, leaf):
    p = D.ddm_nd_plan(nx, ny, leaf)
    seen = set()
    for j, f in enumerate(p["fronts"]):
        nodes = _nodes(p, j)
        for row, col, node, plane in p["ent"][f[9]: f[9] + f[10]]:
            a, b = int(nodes[row]), int(nodes[col])
            assert a == node and b == _neighbour(node, plane, nx)
            assert (a, b) not in seen
            seen.add((a, b))
    expect = set()
    for n in range(nx * ny):
        x, y = n % nx, n // nx
        expect.add((n, n))
        for ok, m in ((x > 0, n - 1), (x + 1 < nx, n + 1), (y > 0, n - nx), (y + 1 < ny, n + nx)):
            if ok:
                expect.add((n, m))
    assert seen == expect


def _plan_solve(p, A, src):
    """Multifrontal factorisation and solve of A (CSR, natural x-fastest order) with the plan's
    fronts, maps and entries; dense numpy linear algebra for each front."""
    A = A.tocsr()
    fr = p["fronts"]
    Ms, Ss = [], []
    for j, f in enumerate(fr):
        s, d = int(f[0]), int(f[1])
        m = s + d
        F = np.zeros((m, m), complex)
        nodes = _nodes(p, j)
        for row, col, node, plane in p["ent"][f[9]: f[9] + f[10]]:
            F[row, col] += A[int(nodes[row]), int(nodes[col])]
        for c, slot in ((int(f[5]), 7), (int(f[6]), 8)):
            if c >= 0:
                cpos = p["cmap"][f[slot]: f[slot] + fr[c][1]]
                F[np.ix_(cpos, cpos)] += Ss[c]
        Pinv = np.linalg.inv(F[:s, :s])
        Ms.append(np.vstack([Pinv, -F[s:, :s] @ Pinv]))
        Ss.append(F[s:, s:] - F[s:, :s] @ Pinv @ F[:s, s:])
    x = np.zeros(src.size, complex)
    ups = []
    for j, f in enumerate(fr):                      # forward, children first
        s, d = int(f[0]), int(f[1])
        r = np.zeros(s + d, complex)
        r[:s] = src[p["piv"][f[3]: f[3] + s]]
        for c, slot in ((int(f[5]), 7), (int(f[6]), 8)):
            if c >= 0:
                r[p["cmap"][f[slot]: f[slot] + fr[c][1]]] += ups[c]
        y = Ms[j] @ r[:s]
        x[p["piv"][f[3]: f[3] + s]] = y[:s]
        ups.append(r[s:] + y[s:])
    for j in range(len(fr) - 1, -1, -1):            # backward, parents first
        f = fr[j]
        s, d = int(f[0]), int(f[1])
        pv = p["piv"][f[3]: f[3] + s]
        xb = x[p["bnd"][f[4]: f[4] + d]]
        x[pv] = x[pv] + Ms[j][s:].T @ xb
    return x


@pytest.mark.parametrize("leaf", [1, 8, 32, 4096])
def test_plan_driven_multifrontal_solve_equals_the_oracle_local_solve(leaf):
    wl = W.tiny_2d(seed=3, n=26, parts=(2, 3), ov=2, npml=4)
    o = DDMOracle(wl.n, wl.h, wl.cuts, wl.ov, wl.npml, wl.sigma0, wl.power, wl.omega, wl.c)
    rng = np.random.default_rng(17)
    for R in [(0, 0), (1, 2), (0, 1)]:
        ny, nx = o.sub_shape[R]
        p = D.ddm_nd_plan(nx, ny, leaf)
        src = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
        ref = o.local_solve(R, src).ravel()
        got = _plan_solve(p, o.sub_A[R], src.ravel())
        assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref), (R, leaf)


def test_plan_rejects_bad_arguments():
    for args in ((0, 5, 8), (5, 0, 8), (4097, 5, 8), (5, 5, -1), (5, 5, 4097)):
        with pytest.raises(D.DDMError) as ei:
            D.ddm_nd_plan(*args)
        assert ei.value.status == D.DDM_E_INVAL


def test_set_local_solver_rejects_a_null_context():
    assert D.lib().ddm_set_local_solver(None, D.DDM_LOCAL_ND, 0) == D.DDM_E_INVAL
