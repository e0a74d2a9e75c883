"""lbm_flow_step_noalloc against the context-based solver.

The allocation-free entry point exists for callers that may not allocate
device memory themselves: code embedded in a framework that owns every device
allocation through its own pool, or code running where cudaMalloc is not
allowed.  It takes every buffer from the caller and keeps its reduction
scratch in a static device array of the library.

Two calls in a row (rest state -> step 1 -> step 2) must reproduce what the
existing entry point (lbm_forward on a context) reports after one and two
steps: the fields rho and u and the residual / objective sums, within the
FP32 parity tolerance the other tests use.  This file is collected last so
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


def test_noalloc_step_matches_context_solver_twice():
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver

    lat = I.pipe_bend_3d(n=24, width=6, re=30.0, seed=2)
    N = lat.n
    nonwall = int(((lat.flags & 7) != I.WALL).sum())
    n_in = int(((lat.flags & 7) == I.VEL).sum())

    # the existing entry point: one step, then two steps from rest
    ref = []
    s = Solver.from_lattice(lat, storage="fp32")
    for k in (1, 2):
        r = s.forward(tol=0, max_steps=k, check_every=k, reset=True)
        rho, u, _ = s.fields(torch.float64)
        ref.append((r, rho.cpu().numpy(), u.cpu().numpy()))
    s.close()

    # caller-owned buffers for the allocation-free call
    dev = torch.device("cuda", torch.cuda.current_device())
    stride = (N + 63) // 64 * 64
    f = [torch.zeros(19 * stride, dtype=torch.float32, device=dev) for _ in range(3)]
    flags = torch.as_tensor(lat.flags, dtype=torch.uint8, device=dev)
    gamma = torch.as_tensor(lat.gamma, dtype=torch.float32, device=dev)
    bc = torch.as_tensor(lat.bcval, dtype=torch.float32, device=dev)
    rho = torch.empty(N, dtype=torch.float32, device=dev)
    u = torch.empty(3 * stride, dtype=torch.float32, device=dev)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    L = C.lib()
    stream = torch.cuda.current_stream(dev).cuda_stream

    for k in (1, 2):
        d = C.lbm_step_desc(C.LBM_D3Q19, C.LBM_FP32, lat.nx, lat.ny, lat.nz, stride,
                            f[k - 1].data_ptr(), f[k].data_ptr(), flags.data_ptr(),
                            gamma.data_ptr(), bc.data_ptr(), rho.data_ptr(), u.data_ptr(),
                            sums.data_ptr(), lat.tau, lat.rho0, lat.gamma_model)
        C.check(L.lbm_flow_step_noalloc(ctypes.byref(d), ctypes.c_void_p(stream)),
                "lbm_flow_step_noalloc")
        torch.cuda.synchronize()
        r, rho_ref, u_ref = ref[k - 1]
        got_u = u.view(3, stride)[:, :N].double().cpu().numpy()
        assert rel(rho.double().cpu().numpy(), rho_ref) <= TOL
        assert rel(got_u, u_ref) <= TOL
        sm = sums.cpu().numpy()
        assert abs(sm[0] / nonwall - r.I) <= TOL * abs(r.I)
        J = lat.w_pin * sm[1] / (3.0 * n_in)
        assert abs(J - r.J) <= TOL * abs(r.J)


def test_noalloc_rejects_oversized_lattice():
    from paper_2501_02161_gb300 import _capi as C
    d = C.lbm_step_desc(C.LBM_D3Q19, C.LBM_FP32, 512, 512, 128, 512 * 512 * 128,
                        1, 2, 3, 4, 5, 6, 7, 8, 0.6, 1.0, 0)
    code = C.lib().lbm_flow_step_noalloc(ctypes.byref(d), None)
    assert code == C.LBM_ERR_ARG
    assert b"reduction blocks" in C.lib().lbm_last_error()
