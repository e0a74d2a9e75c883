"""The adjoint as a torch.autograd backward: gradient of J(gamma) against
central finite differences (FP64 storage) and against the FP64 oracle."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


def _grad(solver, gamma, opts):
    from paper_2501_02161_gb300.autograd import lbm_objective
    g = gamma.clone().requires_grad_(True)
    J = lbm_objective(g, solver, opts)
    J.backward()
    return float(J.item()), g.grad.detach().clone()


def _fd(lat, storage, cells, h, tol, base_gamma):
    from paper_2501_02161_gb300.autograd import SolveOpts, lbm_objective
    from paper_2501_02161_gb300.solver import Solver
    s = Solver.from_lattice(lat, storage=storage)
    opts = SolveOpts(tol=tol, max_steps=2000000, check_every=500, warm=False)
    lbm_objective(base_gamma, s, opts)
    warm = SolveOpts(tol=tol, max_steps=2000000, check_every=500, warm=True)
    out = []
    for c in cells:
        gp = base_gamma.clone()
        gp[c] += h
        Jp = float(lbm_objective(gp, s, warm).item())
        gm = base_gamma.clone()
        gm[c] -= h
        Jm = float(lbm_objective(gm, s, warm).item())
        out.append((Jp - Jm) / (2 * h))
    s.close()
    return np.array(out)


def _cells(lat, k, seed):
    design = np.where((lat.flags & 7) == I.FLUID)[0]
    rng = np.random.default_rng(seed)
    return sorted(int(c) for c in rng.choice(design, size=k, replace=False))


def test_gradient_vs_central_differences_small_heat_sink_fp64():
    from paper_2501_02161_gb300.autograd import SolveOpts
    from paper_2501_02161_gb300.solver import Solver
    lat = I.heat_sink(nx=20, ny=12, nz=10, re=8.0, q_flux=5e-3, seed=11)
    gam = torch.as_tensor(lat.gamma, dtype=torch.float64, device="cuda")
    s = Solver.from_lattice(lat, storage="fp64")
    J, g = _grad(s, gam, SolveOpts(tol=1e-13, max_steps=2000000, check_every=500))
    cells = _cells(lat, 8, 3)
    fd = _fd(lat, "fp64", cells, 1e-5, 1e-13, gam)
    gc = g.cpu().numpy()[cells]
    scale = np.abs(gc).max()
    assert np.abs(fd - gc).max() <= 1e-5 * scale, (fd, gc)


def test_gradient_vs_oracle_heat_sink_32cubed():
    """FP32 autograd gradient after fixed step counts vs the oracle's."""
    from paper_2501_02161_gb300.autograd import SolveOpts
    from paper_2501_02161_gb300.solver import Solver
    lat = I.heat_sink(nx=32, ny=32, nz=32, re=20.0, q_flux=2e-3, seed=12)
    gam = torch.as_tensor(lat.gamma, dtype=torch.float32, device="cuda")
    s = Solver.from_lattice(lat, storage="fp32")
    J, g = _grad(s, gam, SolveOpts(tol=0, max_steps=300, check_every=100))
    orc = O.Oracle(lat)
    orc.flow_run(300)
    orc.thermal_run(300)
    orc.thermal_adjoint_run(300)
    orc.finish_thermal_adjoint()
    orc.adjoint_run(300)
    so = orc.sensitivity()
    gg = g.double().cpu().numpy()
    assert np.linalg.norm(gg - so) / np.linalg.norm(so) <= 1e-4
    assert abs(J - orc.objective()) <= 1e-5 * abs(orc.objective())


def test_gradient_vs_central_differences_96x48x24_fp64_32_cells():
    """The 96 x 48 x 24 heat sink: 32 seeded cells, central differences with
    step 1e-3 (FP64 storage: an FP32 J resolves only ~1e-7, below the
    per-cell change h * dJ/dgamma)."""
    from paper_2501_02161_gb300.autograd import SolveOpts
    from paper_2501_02161_gb300.solver import Solver
    lat = I.heat_sink(nx=96, ny=48, nz=24, re=50.0, seed=4)
    gam = torch.as_tensor(lat.gamma, dtype=torch.float64, device="cuda")
    s = Solver.from_lattice(lat, storage="fp64")
    J, g = _grad(s, gam, SolveOpts(tol=1e-11, max_steps=2000000, check_every=1000))
    cells = _cells(lat, 32, 5)
    fd = _fd(lat, "fp64", cells, 1e-3, 1e-11, gam)
    gc = g.cpu().numpy()[cells]
    err = np.abs(fd - gc)
    rec = {"cells": cells, "fd": fd.tolist(), "adjoint": gc.tolist()}
    out = os.environ.get("LBM_TEST_RECORDS")  # optional folder for the measured values
    if out and os.path.isdir(out):
        json.dump(rec, open(os.path.join(out, "fd_96x48x24.json"), "w"))
    assert err.max() <= 1e-2 * np.abs(gc).max(), rec


def test_projected_gradient_loop_decreases_objective():
    from paper_2501_02161_gb300.autograd import SolveOpts, projected_gradient_loop
    from paper_2501_02161_gb300.solver import Solver
    lat = I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=5e-3, seed=4)
    s = Solver.from_lattice(lat, storage="fp32")
    rho, hist = projected_gradient_loop(s, lat, iters=6, step=0.05,
                                        opts=SolveOpts(tol=1e-6, max_steps=200000,
                                                       check_every=500, warm=True))
    Js = [h["J"] for h in hist]
    assert all(np.isfinite(Js))
    assert Js[-1] < Js[0]
