"""The level-set optimiser (Eq. 13-15, 66-67) driven through the CUDA solver
against the same loop run entirely on the FP64 oracles: the lattice oracle
for the converged forward / adjoint / sensitivity (Eq. 35, 53-56, 66) and
the level-set oracle for the update.  2D D2Q9 pipe bend, FP64 storage,
warm-started solves to 1e-9, a seeded random initial level set so that nodes
change phase (alpha = 0 / 1, Eq. 15) during the run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import levelset_oracle as LO
from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ITERS, K, SIGMA, VMAX, TOL, CHECK = 4, 0.2, 5e-3, 0.5, 1e-9, 500


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


def test_level_set_loop_on_gpu_matches_the_oracles():
    from paper_2501_02161_gb300.levelset import level_set_loop
    from paper_2501_02161_gb300.solver import Solver
    lat = I.pipe_bend_2d(nx=32, ny=32, width=8, tau=0.8, gamma_value=1.0)
    shape = (lat.ny, lat.nx)
    mask = (lat.flags & 7).reshape(shape) == I.FLUID
    rng = np.random.default_rng(21)
    phi0 = np.where(mask, rng.uniform(-0.3, 1.0, shape), 1.0)

    s = Solver.from_lattice(lat, storage="fp64")
    phi_g, hist = level_set_loop(s, lat, iters=ITERS, K=K, sigma=SIGMA, vmax=VMAX,
                                 phi0=torch.as_tensor(phi0, device="cuda"), tol=TOL,
                                 max_steps=400000, check_every=CHECK)
    s.close()
    phi_g = phi_g.cpu().numpy()

    orc = O.Oracle(lat)
    fixed = lat.gamma.reshape(shape)
    phi = phi0.copy()
    flips = 0
    for it in range(ITERS):
        alpha = LO.alpha_of(phi)
        orc.gamma[:] = np.where(mask, alpha, fixed).ravel()
        orc.flow_solve(TOL, 400000, CHECK)
        orc.adjoint_solve(TOL, 400000, CHECK)
        J = orc.objective()
        jw = orc.sensitivity().reshape(shape)
        jw = jw / np.abs(jw[mask]).max()
        new, alpha_new, lam, G = LO.step(phi, jw, K, SIGMA, VMAX, mask)
        flips += int((alpha_new != alpha).sum())
        h = hist[it]
        assert h["J"] == pytest.approx(J, rel=1e-10)
        assert h["G"] == pytest.approx(G, rel=1e-12, abs=1e-15)
        assert h["lambda"] == pytest.approx(lam, rel=1e-9)
        assert h["fluid_fraction"] == pytest.approx(float(alpha_new[mask].mean()), abs=0)
        phi = new
    assert flips > 0                       # the design did change phase
    assert np.array_equal(LO.alpha_of(phi_g), LO.alpha_of(phi))
    assert np.abs(phi_g - phi).max() < 1e-9
