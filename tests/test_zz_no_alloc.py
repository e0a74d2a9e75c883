"""lbm_flow_step_noalloc against the context-based solver.

The allocation-free entry point exists for callers that may not allocate
device memory themselves: code embedded in a framework that owns every device
allocation through its own pool, or code running where cudaMalloc is not
allowed.  It takes every buffer from the caller and keeps its reduction
scratch in a static device array of the library.

Two calls in a row (rest state -> step 1 -> step 2) must reproduce what the
existing entry point (lbm_forward on a context) reports after one and two
steps: the fields rho and u and the residual / objective sums, within the
FP32 parity tolerance the other tests use (1e-12 for FP64 storage).  Every
storage the call accepts is covered: D3Q19 with FP32, FP16 and BF16 offset
populations, D2Q9 with FP64 and FP32.  This file is collected last so
that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    # (lattice, storage name, storage code, population dtype, aux dtype, tolerance)
    ("d3q19", "fp32", 1, torch.float32, torch.float32, TOL),
    ("d2q9", "fp64", 0, torch.float64, torch.float64, 1e-12),
    ("d2q9", "fp32", 1, torch.float32, torch.float32, TOL),
    ("d3q19", "fp16", 2, torch.float16, torch.float32, TOL),
    ("d3q19", "bf16", 3, torch.bfloat16, torch.float32, TOL),
]


def tau_of(lat):
    """The lattice's relaxation time: as given, or the library's conversion
    of its Reynolds number (the same one the context-based path uses)."""
    from paper_2501_02161_gb300 import _capi as C
    if lat.tau is not None:
        return lat.tau
    ph = C.lbm_physics(lat.re, lat.u_ref, lat.l_ref, lat.dp, lat.pr or 0.0, lat.rho0,
                       lat.gamma_model, lat.k_ratio, lat.q_flux, lat.T0, lat.beta_max)
    prm = C.lbm_params()
    C.check(C.lib().lbm_physics_to_params(ctypes.byref(ph), ctypes.byref(prm)), "lbm_physics_to_params")
    return prm.tau


def lattice_of(kind):
    if kind == "d2q9":
        return I.pipe_bend_2d(nx=37, ny=29, width=7, tau=0.7, gamma_value=0.8)
    return I.pipe_bend_3d(n=24, width=6, re=30.0, seed=2)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def test_noalloc_step_matches_context_solver_twice(case):
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver

    kind, storage, code, pdt, adt, tol = case
    lat = lattice_of(kind)
    Q = 9 if lat.stencil == I.D2Q9 else 19
    N = lat.n
    nonwall = int(((lat.flags & 7) != I.WALL).sum())
    n_in = int(((lat.flags & 7) == I.VEL).sum())

    # the existing entry point: one step, then two steps from rest
    ref = []
    s = Solver.from_lattice(lat, storage=storage)
    for k in (1, 2):
        r = s.forward(tol=0, max_steps=k, check_every=k, reset=True)
        rho, u, _ = s.fields(torch.float64)
        ref.append((r, rho.cpu().numpy(), u.cpu().numpy()))
    s.close()

    # caller-owned buffers for the allocation-free call (rest state: h = 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stride = (N + 63) // 64 * 64
    f = [torch.zeros(Q * stride, dtype=pdt, device=dev) for _ in range(3)]
    flags = torch.as_tensor(lat.flags, dtype=torch.uint8, device=dev)
    gamma = torch.as_tensor(lat.gamma, dtype=adt, device=dev)
    bc = torch.as_tensor(lat.bcval, dtype=adt, device=dev)
    rho = torch.empty(N, dtype=adt, device=dev)
    u = torch.empty(3 * stride, dtype=adt, device=dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    L = C.lib()
    stream = torch.cuda.current_stream(dev).cuda_stream

    for k in (1, 2):
        d = C.lbm_step_desc(lat.stencil, code, lat.nx, lat.ny, lat.nz, stride,
                            f[k - 1].data_ptr(), f[k].data_ptr(), flags.data_ptr(),
                            gamma.data_ptr(), bc.data_ptr(), rho.data_ptr(), u.data_ptr(),
                            sums.data_ptr(), tau_of(lat), lat.rho0, lat.gamma_model)
        C.check(L.lbm_flow_step_noalloc(ctypes.byref(d), ctypes.c_void_p(stream)),
                "lbm_flow_step_noalloc")
        torch.cuda.synchronize()
        r, rho_ref, u_ref = ref[k - 1]
        got_u = u.view(3, stride)[:, :N].double().cpu().numpy()
        assert rel(rho.double().cpu().numpy(), rho_ref) <= tol
        assert rel(got_u, u_ref) <= tol
        sm = sums.cpu().numpy()
        assert abs(sm[0] / nonwall - r.I) <= tol * abs(r.I)
        J = lat.w_pin * sm[1] / (3.0 * n_in)
        assert abs(J - r.J) <= tol * abs(r.J)


def test_noalloc_rejects_oversized_lattice():
    from paper_2501_02161_gb300 import _capi as C
    d = C.lbm_step_desc(C.LBM_D3Q19, C.LBM_FP32, 512, 512, 128, 512 * 512 * 128,
                        1, 2, 3, 4, 5, 6, 7, 8, 0.6, 1.0, 0)
    code = C.lib().lbm_flow_step_noalloc(ctypes.byref(d), None)
    assert code == C.LBM_ERR_ARG
    assert b"reduction blocks" in C.lib().lbm_last_error()
