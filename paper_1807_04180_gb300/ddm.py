"""ctypes binding of libddm (include/ddm.h): the same entry points, argument marshalling only.

Device buffers are torch CUDA tensors (complex128 for global vectors, float64 for the wave
speed, complex64/complex128 for local vectors); the binding passes their data pointers and
the current CUDA stream.  Every computation runs in the library's kernels; there is no CPU
fallback, and importing this module without the built library raises an error.

Array conventions: fields are C ordered with the physical x axis last (2D shape (ny, nx)),
so their flat order is the library's x-fastest order.  ``params_from`` turns a
``workloads.Workload`` into a ``ddm_params`` (physical axis order x, y, z).
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ddm.h")

DDM_OK, DDM_E_INVAL, DDM_E_NOMEM, DDM_E_CUDA, DDM_E_STATE, DDM_E_SINGULAR, DDM_E_NOCONV, DDM_E_TIMEOUT, \
    DDM_E_BUDGET = range(9)
DDM_FP64, DDM_MIXED = 0, 1
DDM_STEPPING, DDM_FGMRES = 0, 1
DDM_LOCAL_BLOCK, DDM_LOCAL_ND = 0, 1
DDM_ND_LEAF_DEFAULT = 32
STATUS_NAMES = ["DDM_OK", "DDM_E_INVAL", "DDM_E_NOMEM", "DDM_E_CUDA", "DDM_E_STATE", "DDM_E_SINGULAR",
                "DDM_E_NOCONV", "DDM_E_TIMEOUT", "DDM_E_BUDGET"]
TIMING_SLOTS = ["solve", "transfer", "assemble", "global", "krylov", "factor", "graph"]


class ddm_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double),
                ("parts", ctypes.c_int * 3), ("cuts", ctypes.POINTER(ctypes.c_int64) * 3),
                ("overlap", ctypes.c_int), ("pml", ctypes.c_int), ("sigma0", ctypes.c_double),
                ("pml_power", ctypes.c_double), ("precision", ctypes.c_int), ("max_rhs", ctypes.c_int)]


class ddm_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("ddm_steps", ctypes.c_int), ("converged", ctypes.c_int),
                ("n_unique_factors", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_est", ctypes.c_double), ("factor_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddm_nd_plan_info(ctypes.Structure):
    _fields_ = [("nfront", ctypes.c_int), ("height", ctypes.c_int), ("n_piv", ctypes.c_int64),
                ("n_bnd", ctypes.c_int64), ("n_cmap", ctypes.c_int64), ("n_ent", ctypes.c_int64),
                ("factor_entries", ctypes.c_int64), ("scratch_entries", ctypes.c_int64),
                ("update_entries", ctypes.c_int64)]


class DDMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libddm.so (built by paper_1807_04180_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1807_04180_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "ddm_setup": [ctypes.POINTER(ddm_params), ctypes.c_double, _P, _P, ctypes.POINTER(_P)],
        "ddm_factor": [_P],
        "ddm_set_medium": [_P, ctypes.c_double, _P],
        "ddm_set_medium_host": [_P, ctypes.c_double, _P],
        "ddm_kernel_launches": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
        "ddm_apply": [_P, ctypes.c_int, _P, _P, ctypes.c_int],
        "ddm_solve": [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_int, ctypes.POINTER(ddm_info)],
        "ddm_solve_host": [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.POINTER(ddm_info)],
        "ddm_destroy": [_P],
        "ddm_rhs": [_P, _P, _P, ctypes.c_int],
        "ddm_global_apply": [_P, _P, _P, ctypes.c_int],
        "ddm_residual": [_P, _P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
        "ddm_local_layout": [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "ddm_local_solve": [_P, _P, _P, ctypes.c_int],
        "ddm_steps": [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double)],
        "ddm_timing": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int64)],
        "ddm_factor_bytes": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "ddm_norms_noalloc": [_P, ctypes.c_int64, ctypes.c_int, _P, _P],
        "ddm_workspace_bytes": [ctypes.POINTER(ddm_params), ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
        "ddm_set_graph": [_P, ctypes.c_int],
        "ddm_set_tensor_cores": [_P, ctypes.c_int],
        "ddm_set_rhs_per_cta": [_P, ctypes.c_int],
        "ddm_set_local_solver": [_P, ctypes.c_int, ctypes.c_int],
        "ddm_set_pivoting": [_P, ctypes.c_double],
        "ddm_pivoting_info": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
        "ddm_nd_plan": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ddm_nd_plan_info), _P, _P, _P, _P,
                        _P],
        "ddm_autotune_log": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.ddm_last_error.argtypes = [_P]
    L.ddm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def header_symbols(path: str = HEADER):
    """Names of the functions include/ddm.h declares."""
    with open(path) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^(?:ddm_status|const char \*)\s*(ddm_\w+)\s*\(", txt, re.M)))


def _check(status: int, ctx) -> None:
    if status != DDM_OK:
        msg = lib().ddm_last_error(ctx)
        raise DDMError(status, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device buffers must be CUDA torch tensors")
    if not t.is_contiguous():
        raise ValueError("device buffers must be contiguous")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


# ----------------------------------------------------------------------------- params
def params_from(wl, precision: int = DDM_FP64, max_rhs: int = 1):
    """ddm_params for a workloads.Workload (array axes reversed into physical x, y, z).
    Returns (params, keepalive) where keepalive holds the cut arrays."""
    p = ddm_params()
    d = wl.dim
    p.dim = d
    keep = []
    for a in range(3):
        if a < d:
            arr_axis = d - 1 - a
            p.n[a] = int(wl.n[arr_axis])
            p.parts[a] = len(wl.cuts[arr_axis]) - 1
            cu = np.ascontiguousarray(np.asarray(wl.cuts[arr_axis], dtype=np.int64))
            keep.append(cu)
            p.cuts[a] = cu.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        else:
            p.n[a] = 1
            p.parts[a] = 1
            p.cuts[a] = ctypes.POINTER(ctypes.c_int64)()
    p.h = wl.h
    p.overlap = wl.ov
    p.pml = wl.npml
    p.sigma0 = wl.sigma0
    p.pml_power = wl.power
    p.precision = precision
    p.max_rhs = max_rhs
    return p, keep


# ----------------------------------------------------------------------------- entry points
def ddm_setup(params: ddm_params, omega: float, c_dev, stream=None):
    out = _P()
    st = lib().ddm_setup(ctypes.byref(params), float(omega), _ptr(c_dev), _stream(stream), ctypes.byref(out))
    _check(st, None)
    return out


def ddm_set_graph(ctx, enable: bool = True) -> None:
    _check(lib().ddm_set_graph(ctx, int(bool(enable))), ctx)


def ddm_set_tensor_cores(ctx, enable: bool = True) -> None:
    _check(lib().ddm_set_tensor_cores(ctx, int(bool(enable))), ctx)


def ddm_set_rhs_per_cta(ctx, nr: int = 0) -> None:
    _check(lib().ddm_set_rhs_per_cta(ctx, int(nr)), ctx)


def ddm_set_local_solver(ctx, solver: int = DDM_LOCAL_BLOCK, leaf: int = 0) -> None:
    _check(lib().ddm_set_local_solver(ctx, int(solver), int(leaf)), ctx)


def ddm_set_pivoting(ctx, tau: float = 4.0) -> None:
    _check(lib().ddm_set_pivoting(ctx, float(tau)), ctx)


def ddm_pivoting_info(ctx):
    """(tau, number of factorisations redone with the search over all rows)"""
    t = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().ddm_pivoting_info(ctx, ctypes.byref(t), ctypes.byref(n)), ctx)
    return t.value, n.value


def ddm_nd_plan(nx: int, ny: int, leaf: int = 0) -> dict:
    """Nested-dissection plan of an nx x ny grid (host only): the info fields plus the arrays
    fronts (nfront x 12), piv, bnd, cmap and ent (n_ent x 4) as numpy int32 arrays."""
    info = ddm_nd_plan_info()
    L = lib()
    _check(L.ddm_nd_plan(int(nx), int(ny), int(leaf), ctypes.byref(info), None, None, None, None, None), None)
    arrs = {"fronts": np.zeros((max(info.nfront, 1), 12), np.int32), "piv": np.zeros(max(info.n_piv, 1), np.int32),
            "bnd": np.zeros(max(info.n_bnd, 1), np.int32), "cmap": np.zeros(max(info.n_cmap, 1), np.int32),
            "ent": np.zeros((max(info.n_ent, 1), 4), np.int32)}
    _check(L.ddm_nd_plan(int(nx), int(ny), int(leaf), ctypes.byref(info),
                         *(a.ctypes.data_as(_P) for a in arrs.values())), None)
    out = {k: getattr(info, k) for k, _ in info._fields_}
    out.update({"fronts": arrs["fronts"][:info.nfront], "piv": arrs["piv"][:info.n_piv],
                "bnd": arrs["bnd"][:info.n_bnd], "cmap": arrs["cmap"][:info.n_cmap], "ent": arrs["ent"][:info.n_ent]})
    return out


def ddm_workspace_bytes(params: ddm_params, restart: int) -> int:
    """Upper bound of a context's device bytes (set-up, factors, FGMRES workspace)."""
    out = ctypes.c_int64()
    _check(lib().ddm_workspace_bytes(ctypes.byref(params), int(restart), ctypes.byref(out)), None)
    return out.value


def ddm_set_medium(ctx, omega: float, c_dev) -> None:
    _check(lib().ddm_set_medium(ctx, float(omega), _ptr(c_dev)), ctx)


def ddm_set_medium_host(ctx, omega: float, c_host) -> None:
    """c_host: float64 host array (numpy, or a pinned torch CPU tensor) on the global grid."""
    ptr = c_host.data_ptr() if hasattr(c_host, "data_ptr") else np.ascontiguousarray(c_host, np.float64).ctypes.data
    _check(lib().ddm_set_medium_host(ctx, float(omega), ptr), ctx)


def ddm_kernel_launches(ctx, reset: bool = False) -> int:
    n = ctypes.c_int64()
    _check(lib().ddm_kernel_launches(ctx, ctypes.byref(n), int(bool(reset))), ctx)
    return n.value


def ddm_factor(ctx) -> None:
    _check(lib().ddm_factor(ctx), ctx)


def ddm_apply(ctx, K: int, src_dev, dst_dev, nrhs: int = 1) -> None:
    _check(lib().ddm_apply(ctx, int(K), _ptr(src_dev), _ptr(dst_dev), int(nrhs)), ctx)


def ddm_solve(ctx, f_dev, u_dev, nrhs: int = 1, tol: float = 1e-6, max_it: int = 500, mode: int = DDM_FGMRES,
              K: int = 2, restart: int = 60, check: bool = True) -> dict:
    info = ddm_info()
    st = lib().ddm_solve(ctx, _ptr(f_dev), _ptr(u_dev), int(nrhs), float(tol), int(max_it), int(mode), int(K),
                         int(restart), ctypes.byref(info))
    if check:
        _check(st, ctx)
    d = info.as_dict()
    d["status"] = st
    return d


def ddm_solve_host(ctx, f_host: np.ndarray, u_host: np.ndarray, nrhs: int = 1, tol: float = 1e-6,
                   max_it: int = 500, mode: int = DDM_FGMRES, K: int = 2, restart: int = 60,
                   check: bool = True) -> dict:
    """Host-buffer solve: f_host / u_host are complex128 host arrays (numpy or pinned torch CPU
    tensors); the library copies them to and from the device inside the call."""
    def hp(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        assert a.dtype == np.complex128 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    info = ddm_info()
    st = lib().ddm_solve_host(ctx, hp(f_host), hp(u_host), int(nrhs), float(tol), int(max_it), int(mode), int(K),
                              int(restart), ctypes.byref(info))
    if check:
        _check(st, ctx)
    d = info.as_dict()
    d["status"] = st
    return d


def ddm_destroy(ctx) -> None:
    if ctx:
        lib().ddm_destroy(ctx)


def ddm_last_error(ctx=None) -> str:
    m = lib().ddm_last_error(ctx)
    return m.decode() if m else ""


def ddm_rhs(ctx, f_dev, b_dev, nrhs: int = 1) -> None:
    _check(lib().ddm_rhs(ctx, _ptr(f_dev), _ptr(b_dev), int(nrhs)), ctx)


def ddm_global_apply(ctx, x_dev, y_dev, nrhs: int = 1) -> None:
    _check(lib().ddm_global_apply(ctx, _ptr(x_dev), _ptr(y_dev), int(nrhs)), ctx)


def ddm_residual(ctx, b_dev, x_dev, r_dev, nrhs: int = 1):
    norms = (ctypes.c_double * (2 * nrhs))()
    _check(lib().ddm_residual(ctx, _ptr(b_dev), _ptr(x_dev), _ptr(r_dev), int(nrhs), norms), ctx)
    return [(norms[2 * i], norms[2 * i + 1]) for i in range(nrhs)]


def ddm_local_layout(ctx):
    n = ctypes.c_int()
    tot = ctypes.c_int64()
    _check(lib().ddm_local_layout(ctx, ctypes.byref(n), ctypes.byref(tot), None, None, None, None), ctx)
    offs = (ctypes.c_int64 * n.value)()
    ex = [(ctypes.c_int * n.value)() for _ in range(3)]
    _check(lib().ddm_local_layout(ctx, None, None, offs, ex[0], ex[1], ex[2]), ctx)
    return {"n_sub": n.value, "total": tot.value, "offsets": list(offs),
            "ext": [(ex[0][i], ex[1][i], ex[2][i]) for i in range(n.value)]}


def ddm_local_solve(ctx, src_dev, u_dev, nrhs: int = 1) -> None:
    _check(lib().ddm_local_solve(ctx, _ptr(src_dev), _ptr(u_dev), int(nrhs)), ctx)


def ddm_steps(ctx, b_dev, nsteps: int, w_dev=None, u_last_dev=None, want_res: bool = True):
    res = (ctypes.c_double * nsteps)() if want_res else None
    _check(lib().ddm_steps(ctx, _ptr(b_dev), int(nsteps), _ptr(w_dev), _ptr(u_last_dev), res), ctx)
    return list(res) if want_res else None


def ddm_timing(ctx, enable: bool = True, reset: bool = False) -> dict:
    ms = (ctypes.c_double * 7)()
    n = (ctypes.c_int64 * 7)()
    _check(lib().ddm_timing(ctx, int(bool(enable)), int(bool(reset)), ms, n), ctx)
    return {TIMING_SLOTS[i]: (ms[i], n[i]) for i in range(7)}


def ddm_autotune_log(ctx):
    """[(nrhs, right-hand sides per CTA, device ms)] measured by the local-solve autotuner."""
    n = ctypes.c_int()
    _check(lib().ddm_autotune_log(ctx, 0, None, None, None, ctypes.byref(n)), ctx)
    a = (ctypes.c_int * max(n.value, 1))()
    b = (ctypes.c_int * max(n.value, 1))()
    m = (ctypes.c_float * max(n.value, 1))()
    _check(lib().ddm_autotune_log(ctx, n.value, a, b, m, None), ctx)
    return [(a[i], b[i], m[i]) for i in range(n.value)]


def ddm_factor_bytes(ctx):
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(lib().ddm_factor_bytes(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def _noalloc_args_error(x_dev, n: int, nvec: int, norms_dev) -> Optional[str]:
    """Why (x_dev, n, nvec, norms_dev) cannot go to ddm_norms_noalloc, or None.  The C entry
    point has no context to bound n, so the binding checks the buffers it would read and write:
    x_dev complex128 with at least n * nvec elements, norms_dev float64 with at least nvec, both
    contiguous CUDA tensors on the current device."""
    import torch
    if not isinstance(x_dev, torch.Tensor) or not isinstance(norms_dev, torch.Tensor):
        return "x_dev and norms_dev must be torch tensors"
    if x_dev.dtype != torch.complex128:
        return f"x_dev must be complex128, not {x_dev.dtype}"
    if norms_dev.dtype != torch.float64:
        return f"norms_dev must be float64, not {norms_dev.dtype}"
    if n < 1 or nvec < 1:
        return "n and nvec must be >= 1"
    if x_dev.numel() < n * nvec:
        return f"x_dev holds {x_dev.numel()} elements, fewer than n * nvec = {n * nvec}"
    if norms_dev.numel() < nvec:
        return f"norms_dev holds {norms_dev.numel()} elements, fewer than nvec = {nvec}"
    if not (x_dev.is_cuda and norms_dev.is_cuda):
        return "x_dev and norms_dev must be CUDA tensors"
    if not (x_dev.is_contiguous() and norms_dev.is_contiguous()):
        return "x_dev and norms_dev must be contiguous"
    cur = torch.cuda.current_device()
    if x_dev.device.index != cur or norms_dev.device.index != cur:
        return f"x_dev and norms_dev must be on the current device (cuda:{cur})"
    return None


def ddm_norms_noalloc(x_dev, n: int, nvec: int, norms_dev, stream=None) -> None:
    """Allocation-free norms: norms_dev[i] = ||x_i|| for nvec complex128 vectors of length n
    (x_dev and norms_dev are CUDA tensors; enqueued on the current stream, not synchronised).
    Raises DDMError(DDM_E_INVAL) before any CUDA call when the buffers do not fit the call."""
    why = _noalloc_args_error(x_dev, int(n), int(nvec), norms_dev)
    if why is not None:
        raise DDMError(DDM_E_INVAL, "ddm_norms_noalloc: " + why)
    _check(lib().ddm_norms_noalloc(_ptr(x_dev), int(n), int(nvec), _stream(stream), _ptr(norms_dev)), None)


# ----------------------------------------------------------------------------- convenience
class Solver:
    """Owns one context: set-up from a Workload, factor, apply, solve."""

    def __init__(self, wl, precision: int = DDM_FP64, max_rhs: int = 1, device: str = "cuda", stream=None,
                 local_solver: int = DDM_LOCAL_BLOCK, leaf: int = 0):
        import torch
        self.wl = wl
        self.precision = precision
        self.device = torch.device(device)
        self._params, self._keep = params_from(wl, precision, max_rhs)
        self.c = torch.as_tensor(np.ascontiguousarray(wl.c), dtype=torch.float64, device=self.device)
        self.stream = stream
        self.ctx = ddm_setup(self._params, wl.omega, self.c, stream)
        self.gshape = tuple(wl.c.shape)
        if local_solver != DDM_LOCAL_BLOCK or leaf:
            ddm_set_local_solver(self.ctx, local_solver, leaf)

    def factor(self):
        ddm_factor(self.ctx)
        return self

    def to_dev(self, a, dtype=None):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a), device=self.device, dtype=dtype)

    def close(self):
        if getattr(self, "ctx", None):
            ddm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
