"""CPU-side checks of the C-ABI library: it builds, loads and exports every declared symbol.
No compute call runs here (there is no GPU in this environment)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def built():
    from paper_1807_04180_gb300 import build
    return build.build()


def test_library_exports_every_header_symbol(built):
    from paper_1807_04180_gb300 import ddm
    names = ddm.header_symbols()
    assert {"ddm_setup", "ddm_factor", "ddm_apply", "ddm_solve", "ddm_destroy", "ddm_last_error"} <= set(names)
    L = ctypes.CDLL(built)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert all(hasattr(ddm, n) for n in names)


def test_setup_rejects_bad_params_before_touching_the_gpu(built):
    """Parameter validation happens before any CUDA call, so it can be exercised here."""
    from paper_1807_04180_gb300 import ddm, workloads as W
    wl = W.tiny_2d()
    p, keep = ddm.params_from(wl)
    p.dim = 4
    out = ctypes.c_void_p()
    L = ddm.lib()
    st = L.ddm_setup(ctypes.byref(p), 1.0, ctypes.c_void_p(16), None, ctypes.byref(out))
    assert st == ddm.DDM_E_INVAL and b"dim" in L.ddm_last_error(None)
    p, keep = ddm.params_from(wl)
    p.overlap = 0
    st = L.ddm_setup(ctypes.byref(p), 1.0, ctypes.c_void_p(16), None, ctypes.byref(out))
    assert st == ddm.DDM_E_INVAL
    p, keep = ddm.params_from(wl)
    st = L.ddm_setup(ctypes.byref(p), -1.0, ctypes.c_void_p(16), None, ctypes.byref(out))
    assert st == ddm.DDM_E_INVAL
    # a part narrower than twice the overlap is refused
    wl2 = W.tiny_2d(n=12, parts=(4, 4), ov=2)
    p, keep = ddm.params_from(wl2)
    st = L.ddm_setup(ctypes.byref(p), 1.0, ctypes.c_void_p(16), None, ctypes.byref(out))
    assert st == ddm.DDM_E_INVAL


def test_binding_refuses_cpu_tensors(built):
    torch = pytest.importorskip("torch")
    from paper_1807_04180_gb300 import ddm
    with pytest.raises(TypeError):
        ddm._ptr(torch.zeros(4, dtype=torch.complex128))


def test_workspace_estimate_is_pure_arithmetic_and_monotone(built):
    """ddm_workspace_bytes needs no GPU; it grows with the grid, the right-hand sides and the
    Krylov restart."""
    from paper_1807_04180_gb300 import ddm, workloads as W
    small = W.tiny_2d(n=24, parts=(2, 2))
    big = W.tiny_2d(n=48, parts=(4, 4))
    b = []
    for wl, R, m in [(small, 1, 0), (small, 1, 20), (small, 4, 20), (big, 4, 20)]:
        p, keep = ddm.params_from(wl, ddm.DDM_MIXED, R)
        b.append(ddm.ddm_workspace_bytes(p, m))
    assert b[0] < b[1] < b[2] < b[3]
    p, keep = ddm.params_from(small, ddm.DDM_FP64, 1)
    assert ddm.ddm_workspace_bytes(p, 0) > b[0]       # complex128 local storage


@pytest.mark.parametrize("case", ["x_dtype", "norms_dtype", "x_short", "norms_short", "bad_n", "not_cuda"])
def test_noalloc_binding_rejects_buffers_that_do_not_fit(built, case):
    """ddm_norms_noalloc has no context to bound n, so the binding refuses, before any CUDA
    call, buffers the kernels would read or write past: a wrong dtype, too few elements, a bad
    size, or tensors not on the GPU (the order of the checks lets each case reach its own)."""
    torch = pytest.importorskip("torch")
    from paper_1807_04180_gb300 import ddm
    n, nvec = 100, 3
    x = torch.zeros(n * nvec, dtype=torch.complex128)
    out = torch.zeros(nvec, dtype=torch.float64)
    if case == "x_dtype":
        x = torch.zeros(n * nvec, dtype=torch.complex64)
    elif case == "norms_dtype":
        out = torch.zeros(nvec, dtype=torch.float32)
    elif case == "x_short":
        x = torch.zeros(n * nvec - 1, dtype=torch.complex128)
    elif case == "norms_short":
        out = torch.zeros(nvec - 1, dtype=torch.float64)
    elif case == "bad_n":
        n = 0
    with pytest.raises(ddm.DDMError) as ei:
        ddm.ddm_norms_noalloc(x, n, nvec, out)
    assert ei.value.status == ddm.DDM_E_INVAL
    expect = {"x_dtype": "complex128", "norms_dtype": "float64", "x_short": "fewer than n * nvec",
              "norms_short": "fewer than nvec", "bad_n": ">= 1", "not_cuda": "CUDA tensors"}[case]
    assert expect in str(ei.value)
