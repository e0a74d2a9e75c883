"""The C-ABI library builds, loads and exports every declared entry point
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmadj.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2501_02161_gb300 import build as B
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return B.build()


def test_header_declares_the_solver_calls():
    names = declared_symbols()
    for must in ["lbm_create", "lbm_destroy", "lbm_set_flags", "lbm_set_gamma",
                 "lbm_set_bc_values", "lbm_set_params", "lbm_set_objective", "lbm_forward",
                 "lbm_adjoint", "lbm_sensitivity", "lbm_get_fields"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(lbm_[a-z0-9_]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2501_02161_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == declared_symbols()
    L = _capi.lib()
    for name in declared_symbols():
        assert hasattr(L, name)
    assert b"sm_103a" in L.lbm_version()


def test_argument_errors_without_gpu(libpath):
    """Argument checks happen before any device call."""
    import ctypes
    from paper_2501_02161_gb300 import _capi as C
    L = C.lib()
    ctx = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(ctx), 0, 8, 8, 2, 1, 0) == C.LBM_ERR_ARG  # D2Q9, nz=2
    assert L.lbm_create(ctypes.byref(ctx), 0, 8, 8, 1, 1, 1) == C.LBM_ERR_UNSUPPORTED
    assert L.lbm_create(ctypes.byref(ctx), 1, 0, 8, 8, 1, 0) == C.LBM_ERR_ARG
    assert L.lbm_create(ctypes.byref(ctx), 7, 8, 8, 8, 1, 0) == C.LBM_ERR_ARG
    assert L.lbm_create(None, 1, 8, 8, 8, 1, 0) == C.LBM_ERR_ARG
    assert L.lbm_forward(None, None, None) == C.LBM_ERR_ARG
    assert b"null" in L.lbm_last_error()


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2501_02161_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "lbm_oracle" not in text, fn


def test_no_gpu_means_a_loud_failure_not_a_cpu_path(libpath):
    """On a machine without a usable GPU the library refuses to create a
    context (LBM_ERR_CUDA with a message) and the Python face raises: there is
    no CPU fallback for any step of the solve."""
    import ctypes

    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2501_02161_gb300 import _capi as C
    L = C.lib()
    ctx = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(ctx), C.LBM_D3Q19, 16, 16, 16, C.LBM_FP32, 0) == C.LBM_ERR_CUDA
    assert not ctx.value and L.lbm_last_error()
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.solver import Solver
    with pytest.raises(Exception):
        Solver.from_lattice(I.pipe_bend_3d(n=16, width=4, re=20.0), storage="fp32")
