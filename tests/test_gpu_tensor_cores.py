"""Tensor-core (tcgen05, split TF32) block solves against the FP64 oracle and against the
CUDA-core FP32 kernels, on cases that span several 128-row tiles of the factor blocks and
several 128-column tiles of the right-hand-side operand, each with a ragged tail."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import from_local, from_local_batch, oracle_of, rel, to_local, to_local_batch  # noqa: E402
from paper_1807_04180_gb300 import ddm as D  # noqa: E402
from paper_1807_04180_gb300 import workloads as W  # noqa: E402


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _uneven(wl, cuts):
    wl.cuts = tuple(np.array(c) for c in cuts)
    return wl


def cases3d():
    return {
        # b = 20 x 20 = 400 rows per plane block: 4 row tiles, the last 16 rows; 8 x 17 = 136 columns
        "gauss-b400": (W.tiny_3d(seed=11, n=24, parts=(2, 2, 2), ov=1, npml=3), 17),
        # uneven parts (plane blocks of 19x22, 23x20, ... rows), ov = 2
        "uneven-ov2": (_uneven(W.tiny_3d(seed=12, n=22, parts=(2, 2, 2), ov=2, npml=3),
                               ([0, 9, 22], [0, 12, 22], [0, 10, 22])), 3),
        # constant medium: one shared factor, all 8 x 20 columns in one contraction
        "const-shared": (W.tiny_3d(seed=13, n=20, parts=(2, 2, 2), ov=1, npml=3, medium="const"), 20),
    }


CASES3D = cases3d()


def _local_solves(wl, nrhs, tc):
    o = oracle_of(wl)
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=nrhs).factor()
    D.ddm_set_tensor_cores(s.ctx, tc)
    rng = np.random.default_rng(5)
    srcs = [{R: cplx(rng, o.sub_shape[R]) for R in o.subs} for _ in range(nrhs)]
    src = to_local_batch(o, srcs, np.complex64)
    u = torch.zeros(src.shape, dtype=torch.complex64, device="cuda")
    D.ddm_local_solve(s.ctx, s.to_dev(src), u, nrhs)
    # one row per right-hand side, each in the one-right-hand-side layout
    out = np.stack([to_local(o, d, np.complex64) for d in from_local_batch(o, u.cpu().numpy(), nrhs)])
    s.close()
    return o, srcs, out


@pytest.mark.parametrize("name", list(CASES3D))
def test_3d_tensor_core_local_solves_match_oracle(name):
    wl, nrhs = CASES3D[name]
    o, srcs, tc = _local_solves(wl, nrhs, True)
    _, _, cc = _local_solves(wl, nrhs, False)
    err_tc = err_cc = 0.0
    for r in range(nrhs):
        got_tc, got_cc = from_local(o, tc[r]), from_local(o, cc[r])
        for R in o.subs:
            if r < 3 or R == o.subs[-1]:          # the oracle's sparse solves: a sample of them
                ref = o.local_solve(R, srcs[r][R])
                err_tc = max(err_tc, rel(got_tc[R], ref))
                err_cc = max(err_cc, rel(got_cc[R], ref))
    # FP32-level accuracy: the bound of the FP32 local solves, and no worse than the CUDA-core
    # FP32 kernels on the same inputs (split TF32 carries about 21 bits against FP32's 24)
    assert err_tc < 2e-4, (err_tc, err_cc)
    assert err_tc < 4 * err_cc + 1e-6, (err_tc, err_cc)


def test_3d_tensor_core_fgmres_reaches_1e6():
    wl, _ = CASES3D["gauss-b400"]
    o = oracle_of(wl)
    s = D.Solver(wl, precision=D.DDM_MIXED).factor()
    u = torch.zeros(o.gshape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f[0]), u, tol=1e-6, max_it=300, mode=D.DDM_FGMRES, K=4, restart=40)
    b = o.rhs(wl.f[0])
    x = u.cpu().numpy()
    assert info["converged"] and np.linalg.norm(b - o.apply_global(x)) / np.linalg.norm(b) <= 1e-6
    s.close()


# ------------------------------------------------------------------------------------------- 2D
def _uneven2(wl, cuts):
    wl.cuts = tuple(np.array(c) for c in cuts)
    return wl


def cases2d():
    return {
        # blocks of b = 12 + 2 * 12 = 36 rows (3 K chunks, the last ragged), 2 x 2 subdomains
        "b36": W.tiny_2d(seed=21, n=24, parts=(2, 2), ov=2, npml=10),
        # b = 124: near the 128-row limit, 8 K chunks, the last ragged; uneven y widths
        "b124": _uneven2(W.tiny_2d(seed=22, n=200, parts=(2, 3), ov=2, npml=10),
                         ([0, 100, 200], [0, 50, 130, 200])),
        # b = 13 (< one 16-column chunk), ov = 1, 3 x 2 subdomains of uneven widths
        "b13-uneven": _uneven2(W.tiny_2d(seed=23, n=18, parts=(3, 2), ov=1, npml=3),
                               ([0, 5, 11, 18], [0, 10, 18])),
    }


CASES2D = cases2d()


def _local2d(wl, nrhs, nr, seed=7):
    o = oracle_of(wl)
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=max(nrhs, 16)).factor()
    D.ddm_set_rhs_per_cta(s.ctx, nr)
    rng = np.random.default_rng(seed)
    srcs = [{R: cplx(rng, o.sub_shape[R]) for R in o.subs} for _ in range(nrhs)]
    src = to_local_batch(o, srcs, np.complex64)
    u = torch.zeros(src.shape, dtype=torch.complex64, device="cuda")
    D.ddm_local_solve(s.ctx, s.to_dev(src), u, nrhs)
    # one row per right-hand side, each in the one-right-hand-side layout
    out = np.stack([to_local(o, d, np.complex64) for d in from_local_batch(o, u.cpu().numpy(), nrhs)])
    s.close()
    return o, srcs, out


@pytest.mark.parametrize("name", list(CASES2D))
@pytest.mark.parametrize("nr,nrhs", [(64, 16), (64, 21), (64, 64), (64, 37), (64, 70)])
def test_2d_tensor_core_local_solves_match_oracle(name, nr, nrhs):
    wl = CASES2D[name]
    o, srcs, tc = _local2d(wl, nrhs, nr)
    _, _, cc = _local2d(wl, nrhs, 4)              # CUDA-core FP32 kernel on the same inputs
    err_tc = err_cc = 0.0
    for r in sorted({0, 1, nrhs // 2, nrhs - 1}):
        got_tc, got_cc = from_local(o, tc[r]), from_local(o, cc[r])
        for R in o.subs:
            ref = o.local_solve(R, srcs[r][R])
            err_tc = max(err_tc, rel(got_tc[R], ref))
            err_cc = max(err_cc, rel(got_cc[R], ref))
    # FP32 local solves lose digits with the subdomain size (about 1e-3 at 124 x 130 nodes for
    # both kernels).  Split TF32 keeps about 21 significant bits per product against FP32's 24,
    # so its rounding error may reach 8x that of the FP32 CUDA cores, never more
    assert err_tc < 5e-3, (err_tc, err_cc)
    assert err_tc < 10 * err_cc + 1e-5, (err_tc, err_cc)
    # every right-hand side is solved (the ragged last group included)
    assert rel(tc, cc) < 10 * err_cc + 1e-5


def test_2d_tensor_core_accumulates_U_like_cuda_cores():
    """The DDM steps accumulate U = sum_s u^s inside the solve kernel: M_K (5 steps, 16
    right-hand sides) through the tensor-core kernel and the CUDA-core kernel agree."""
    wl = W.tiny_2d(seed=24, n=32, parts=(2, 2), ov=2, npml=6, nrhs=16)
    o = oracle_of(wl)
    b = np.stack([o.rhs(wl.f[r]) for r in range(16)])
    res = {}
    for nr in (64, 2):
        s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=16).factor()
        D.ddm_set_rhs_per_cta(s.ctx, nr)
        w = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        D.ddm_apply(s.ctx, 5, s.to_dev(b), w, 16)
        res[nr] = w.cpu().numpy()
        s.close()
    assert rel(res[64], res[2]) < 1e-4


def test_2d_tensor_core_fgmres_batched_reaches_1e6():
    wl = W.tiny_2d(seed=25, n=40, parts=(2, 2), ov=2, npml=8, nrhs=20)
    o = oracle_of(wl)
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=20).factor()
    D.ddm_set_rhs_per_cta(s.ctx, 64)
    u = torch.zeros(wl.f.shape, dtype=torch.complex128, device="cuda")
    info = D.ddm_solve(s.ctx, s.to_dev(wl.f), u, nrhs=20, tol=1e-6, max_it=200, mode=D.DDM_FGMRES, K=4,
                       restart=30)
    x = u.cpu().numpy()
    for r in (0, 7, 19):
        b = o.rhs(wl.f[r])
        assert np.linalg.norm(b - o.apply_global(x[r])) / np.linalg.norm(b) <= 1e-6
    assert info["converged"]
    s.close()


def test_rhs_per_cta_validation():
    wl = W.tiny_2d(seed=26, n=16, parts=(2, 2), ov=1, npml=3)
    s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=4).factor()     # max_rhs < 16: nothing packed
    with pytest.raises(D.DDMError):
        D.ddm_set_rhs_per_cta(s.ctx, 64)
    with pytest.raises(D.DDMError):
        D.ddm_set_rhs_per_cta(s.ctx, 16)
    D.ddm_set_rhs_per_cta(s.ctx, 4)
    D.ddm_set_rhs_per_cta(s.ctx, 0)
    s.close()


def test_2d_graph_replay_survives_refactorisation():
    """A graph of M_K captured before ddm_set_medium + ddm_factor keeps addressing valid factor
    buffers: replays after a new medium give what a context without graphs gives."""
    wl = W.tiny_2d(seed=27, n=32, parts=(2, 2), ov=2, npml=6, nrhs=16)
    o = oracle_of(wl)
    b = np.stack([o.rhs(wl.f[r]) for r in range(16)])
    c2 = np.asarray(wl.c) * 1.1                       # a second medium
    outs = {}
    for graph in (True, False):
        s = D.Solver(wl, precision=D.DDM_MIXED, max_rhs=16).factor()
        D.ddm_set_rhs_per_cta(s.ctx, 64)                 # the same kernel in both contexts
        D.ddm_set_graph(s.ctx, graph)
        w = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        D.ddm_apply(s.ctx, 3, s.to_dev(b), w, 16)       # captures the graph (first medium)
        D.ddm_set_medium(s.ctx, wl.omega, s.to_dev(c2, torch.float64))
        D.ddm_factor(s.ctx)
        D.ddm_apply(s.ctx, 3, s.to_dev(b), w, 16)       # replays it on the second medium's factors
        outs[graph] = w.cpu().numpy()
        s.close()
    assert rel(outs[True], outs[False]) < 1e-12
