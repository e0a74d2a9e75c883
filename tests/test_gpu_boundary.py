"""The boundary's problem-statement calls on the GPU: parameters from Re and
Pr (lbm_set_physics), boundary values per face (lbm_set_bc) and the batch's
memory budget (lbm_batch_create / admit / release)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()


def _solve(s, thermal):
    rf = s.forward(tol=0, max_steps=120, check_every=40)
    ra = s.adjoint(tol=0, max_steps=80, check_every=40)
    rho, u, T = s.fields(torch.float64)
    return [rf.J, ra.I, rho.cpu(), u.cpu(), s.sensitivity(dtype=torch.float64).cpu()] + \
        ([T.cpu()] if thermal else [])


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, torch.Tensor):
            assert torch.equal(x, y)
        else:
            assert x == y


@pytest.mark.parametrize("lat", [I.pipe_bend_3d(n=24, width=6, re=30.0, seed=5),
                                 I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=5e-3, seed=4)],
                         ids=lambda l: l.name)
def test_physics_gives_the_same_solve_as_the_converted_params(lat):
    """lbm_set_physics(Re, U, L, Pr) and lbm_set_params with the tau and kappa_f
    that lbm_physics_to_params gives are the same problem, bit for bit."""
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver
    a = Solver.from_lattice(lat, storage="fp32")          # through lbm_set_physics
    ra = _solve(a, lat.thermal)
    a.close()
    ph = C.lbm_physics(lat.re, lat.u_ref, lat.l_ref, lat.dp, lat.pr or 0.0, lat.rho0,
                       lat.gamma_model, lat.k_ratio, lat.q_flux, lat.T0, lat.beta_max)
    p = C.lbm_params()
    C.check(C.lib().lbm_physics_to_params(ctypes.byref(ph), ctypes.byref(p)), "convert")
    b = Solver.from_lattice(lat, storage="fp32")
    b.set_params(tau=p.tau, rho0=p.rho0, gamma_model=p.gamma_model, kappa_f=p.kappa_f,
                 k_ratio=p.k_ratio, q_flux=p.q_flux, T0=p.T0)
    rb = _solve(b, lat.thermal)
    b.close()
    _same(ra, rb)


FACE_OF_NORMAL = {(1, 0, 0): 0, (-1, 0, 0): 1, (0, 1, 0): 2, (0, -1, 0): 3, (0, 0, 1): 4, (0, 0, -1): 5}


@pytest.mark.parametrize("swap", [False, True])
def test_face_values_equal_node_values(swap):
    """Every opening of the six-port box given per face (lbm_set_bc) instead of
    per node (lbm_set_bc_values): bit-identical solves, both kinds on all six
    faces."""
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver
    lat = I.six_port_box(swap=swap, thermal=True)
    ref = Solver.from_lattice(lat, storage="fp32")
    want = _solve(ref, True)
    ref.close()
    s = Solver(lat.stencil, lat.nx, lat.ny, lat.nz, "fp32", True)
    s.set_flags(torch.as_tensor(lat.flags))
    s.set_gamma(torch.as_tensor(lat.gamma, dtype=torch.float32))
    kind = lat.flags & 7
    code = (lat.flags >> 3) & 7
    bc = lat.bcval.reshape(-1, 4)
    for face in range(6):
        for k in (C.LBM_VEL, C.LBM_PRES):
            sel = np.where((kind == k) & (code == face))[0]
            if len(sel) == 0:
                continue
            vals = bc[sel]
            if k == C.LBM_PRES and np.all(vals == vals[0]):
                s.set_bc(face, k, np.ascontiguousarray(vals[0]))            # one value for the face
            else:
                s.set_bc(face, k, torch.as_tensor(vals.ravel(), device="cuda"))  # per node, on device
    s.set_lattice_params(lat)
    got = _solve(s, True)
    s.close()
    _same(got, want)


def test_face_values_reject_bad_calls():
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver
    lat = I.six_port_box()
    s = Solver.from_lattice(lat, storage="fp32")
    for face, kind, vals in [(6, C.LBM_VEL, np.zeros(4)), (0, 1, np.zeros(4)),
                             (0, C.LBM_PRES, np.zeros(4)),      # face 0 holds inlets only
                             (0, C.LBM_VEL, np.zeros(8))]:      # neither 4 nor 4 x count
        with pytest.raises(C.LBMError) as e:
            s.set_bc(face, kind, vals)
        assert e.value.code == C.LBM_ERR_ARG
    s.close()


def test_batch_budget_admits_releases_and_counts_kept_contexts():
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.serve import Batch, footprint
    from paper_2501_02161_gb300.solver import Solver
    a_lat = I.pipe_bend_3d(n=24, width=6, re=30.0, seed=5)
    b_lat = I.pipe_bend_3d(n=20, width=5, re=20.0, seed=2)
    fa, fb = footprint(a_lat, "fp32"), footprint(b_lat, "fp32")
    batch = Batch("fp32", 20, 4, None, budget_bytes=fa + fb - 1)
    a = Solver.from_lattice(a_lat, storage="fp32")
    b = Solver.from_lattice(b_lat, storage="fp32")
    assert batch.try_admit(a, 0.0, 40, True) is not None
    assert batch.memory() == (fa + fb - 1, fa)
    assert batch.try_admit(b, 0.0, 40, True) is None            # over the budget: not admitted
    with pytest.raises(C.LBMError) as e:
        batch.release(a)                                         # still running
    assert e.value.code == C.LBM_ERR_ORDER
    while batch.step():
        pass
    assert len(batch.poll()) == 1
    assert batch.memory()[1] == fa                               # kept contexts still count
    assert batch.try_admit(a, 0.0, 40, False) is not None        # counted already: admitted
    while batch.step():
        pass
    batch.poll()
    batch.release(a)
    assert batch.memory()[1] == 0
    assert batch.try_admit(b, 0.0, 40, True) is not None
    while batch.step():
        pass
    batch.poll()
    b.close()                                                     # destroying releases it
    assert batch.memory()[1] == 0
    a.close()
    batch.close()
