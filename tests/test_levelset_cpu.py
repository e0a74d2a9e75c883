"""Level-set design update (Eq. 13-15, 66-67): the FP64 oracle pinned to closed
forms, the package's tensor implementation against the oracle, and the
optimisation loop's mechanics with a stand-in solver.  All on CPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import levelset_oracle as LO
from paper_2501_02161_gb300 import levelset as LS


# ---------------------------------------------------------------- oracle pins

@pytest.mark.parametrize("n,k", [(8, 1), (8, 3), (13, 5)])
def test_oracle_laplacian_eigenfunctions_of_the_mirrored_grid(n, k):
    """cos(pi k (x + 1/2) / n) is an eigenvector of the second difference with
    mirrored ends, eigenvalue -4 sin^2(pi k / (2n)): edges included."""
    x = np.arange(n)
    f = np.cos(math.pi * k * (x + 0.5) / n)
    ev = -4.0 * math.sin(math.pi * k / (2 * n)) ** 2
    lap = LO.sigma_laplacian(f[None, :], 0.7)     # (ny=1, nx)
    assert np.allclose(lap[0], 0.7 * ev * f, atol=1e-13)
    # 3D: the product of such modes, anisotropic weights add the eigenvalues
    g = np.cos(math.pi * 2 * (np.arange(5) + 0.5) / 5)
    field = g[:, None, None] * f[None, None, :] * np.ones((1, 4, 1))
    lap3 = LO.sigma_laplacian(field, (0.5, 2.0, 3.0))
    ev_z = -4.0 * math.sin(math.pi * 2 / 10) ** 2
    assert np.allclose(lap3, (0.5 * ev + 3.0 * ev_z) * field, atol=1e-12)


def test_oracle_laplacian_of_a_quadratic_is_its_second_derivative():
    ny, nx = 6, 9
    x = np.arange(nx, dtype=float)
    f = np.tile(x * x, (ny, 1))
    lap = LO.sigma_laplacian(f, 1.0)
    assert np.allclose(lap[:, 1:-1], 2.0)  # interior: the exact second difference
    assert np.allclose(LO.sigma_laplacian(np.full((3, 4, 5), 0.3), 2.0), 0.0)


def test_oracle_multiplier_and_step_for_constant_inputs():
    """sigma = 0, J_W' = c everywhere, all fluid: G = 1 - V_max,
    lambda = exp(G) |c|, phi <- clip(phi - K (c + lambda))."""
    phi = np.full((4, 5), 0.25)
    c, K, vmax = -0.3, 0.2, 0.6
    new, alpha, lam, G = LO.step(phi, np.full_like(phi, c), K, 0.0, vmax)
    assert G == pytest.approx(1 - vmax, abs=1e-15)
    assert lam == pytest.approx(math.exp(1 - vmax) * abs(c), rel=1e-15)
    assert np.allclose(new, np.clip(0.25 - K * (c + lam), -1, 1))
    # a large step clips at the ends of the range Eq. 13 allows
    new2, alpha2, _, _ = LO.step(phi, np.full_like(phi, 50.0), 1.0, 0.0, vmax)
    assert np.all(new2 == -1.0) and np.all(alpha2 == 0.0)


def test_oracle_alpha_map_threshold():
    phi = np.array([[-1.0, -1e-300, 0.0, 1e-300, 1.0]])
    assert LO.alpha_of(phi).tolist() == [[0.0, 0.0, 1.0, 1.0, 1.0]]


def test_oracle_step_leaves_non_design_nodes_alone():
    rng = np.random.default_rng(2)
    phi = rng.uniform(-1, 1, (3, 4, 5))
    mask = rng.random((3, 4, 5)) > 0.4
    new, _, _, _ = LO.step(phi, rng.normal(size=phi.shape), 0.5, 0.1, 0.5, mask)
    assert np.array_equal(new[~mask], phi[~mask])


# ------------------------------------------------- package against the oracle

@pytest.mark.parametrize("shape,sigma", [((7, 9), 0.01), ((4, 5, 6), 5e-3), ((3, 6, 5), (5e-3, 5e-3, 5e-2)),
                                         ((1, 4, 7), 0.2), ((2, 1, 1), 1.0)])
def test_level_set_step_matches_the_oracle(shape, sigma):
    rng = np.random.default_rng(7)
    phi = rng.uniform(-1, 1, shape)
    mask = rng.random(shape) > 0.25
    tphi = torch.tensor(phi)
    tmask = torch.tensor(mask)
    for it in range(3):  # chained steps
        jw = rng.normal(scale=0.5, size=shape)
        o_new, o_alpha, o_lam, o_G = LO.step(phi, jw, 0.15, sigma, 0.45, mask)
        t_new, t_alpha, t_lam, t_G = LS.level_set_step(tphi, torch.tensor(jw), 0.15, sigma, 0.45, tmask)
        assert t_G == pytest.approx(o_G, abs=1e-15)
        assert t_lam == pytest.approx(o_lam, rel=1e-13)
        assert np.allclose(t_new.numpy(), o_new, rtol=0, atol=1e-13)
        assert np.array_equal(t_alpha.numpy(), o_alpha)
        phi, tphi = o_new, t_new


def test_laplacian_matches_the_oracle():
    rng = np.random.default_rng(9)
    f = rng.normal(size=(5, 6, 7))
    for sigma in (1.0, (0.5, 2.0, 3.0)):
        assert np.allclose(LS.laplacian(torch.tensor(f), sigma).numpy(), LO.sigma_laplacian(f, sigma),
                           rtol=0, atol=1e-13)


# ------------------------------------------------------------- the loop

class StandInSolver:
    """Returns a fixed sensitivity field (positive: solid lowers J there)."""

    def __init__(self, sens):
        self.device = torch.device("cpu")
        self.rdtype = torch.float32
        self.sens = sens
        self.gammas = []

    def set_gamma(self, g):
        self.gammas.append(g.clone())

    def forward(self, **kw):
        class R:
            J = 1.0
        return R()

    def adjoint(self, **kw):
        return None

    def sensitivity(self, dtype=torch.float64):
        return self.sens.to(dtype)


def test_level_set_loop_moves_the_design_towards_the_volume_bound():
    from paper_2501_02161_gb300 import inputs as I
    lat = I.pipe_bend_2d(nx=24, ny=20, width=6)
    shape = (lat.ny, lat.nx)
    # a smooth positive sensitivity: everywhere, solid lowers J
    yy, xx = torch.meshgrid(torch.arange(shape[0]), torch.arange(shape[1]), indexing="ij")
    sens = (1.0 + 0.5 * torch.cos(xx / 4.0) * torch.sin(yy / 3.0)).reshape(-1).double()
    s = StandInSolver(sens)
    phi, hist = LS.level_set_loop(s, lat, iters=30, K=0.05, sigma=5e-3, vmax=0.4)
    kind = torch.as_tensor(lat.flags & 7).reshape(shape)
    assert phi.min() >= -1 and phi.max() <= 1
    assert torch.all(phi[kind != 0] == 1.0)          # non-design nodes untouched
    fr = [h["fluid_fraction"] for h in hist]
    assert fr[0] == 1.0 and fr[-1] < fr[0]           # solid appears where it lowers J
    # the solver saw gamma = alpha(phi) on design nodes, its own gamma elsewhere
    g = s.gammas[-1].double().reshape(shape)
    fixed = torch.as_tensor(lat.gamma).reshape(shape)
    assert torch.equal(g[kind != 0], fixed[kind != 0].to(g.dtype))
    assert set(g[kind == 0].unique().tolist()) <= {0.0, 1.0}
