"""The paper's heat-generation variant on the GPU against the FP64 oracle:
source Q = beta_max (1 - gamma)(1 - T) in the temperature collision (Eq. 69,
71), objective J_Q = -sum Q (Eq. 72), their adjoint terms in the temperature
adjoint, the coupling and dJ/dgamma.  Same steps on both sides, every node
compared; FP64 rel-L2 <= 1e-11, FP32 <= 1e-5 on fields and J and <= 1e-4 on
adjoints and dJ/dgamma."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I
from test_gpu_parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


def with_source(lat, beta, w_qgen, w_tmean, seed):
    """Seeded gamma in (0.3, 0.9) on the design (fluid) nodes, so the source is
    active on all of them, plus the source and objective weights."""
    rng = np.random.default_rng(seed)
    fluid = (lat.flags & 7) == I.FLUID
    lat.gamma = np.where(fluid, 0.3 + 0.6 * rng.random(lat.n), lat.gamma)
    lat.beta_max, lat.w_qgen, lat.w_tmean = beta, w_qgen, w_tmean
    return lat


def lattices():
    return [with_source(I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=0.0, seed=4), 0.05, 1.0, 0.0, 1),
            with_source(I.heat_sink(nx=19, ny=11, nz=9, re=10.0, q_flux=5e-3, seed=6,
                                    gamma_model=I.GAMMA_LINEAR), 0.02, 0.5, 1.0, 2),
            with_source(I.six_port_box(thermal=True), 0.03, 1.0, 1.0, 3)]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("lat", lattices(), ids=lambda l: l.name)
def test_heat_generation_parity_fixed_steps(lat, storage):
    g = run_gpu(lat, storage, 200, 150, K=50)
    o = run_oracle(lat, 200, 150)
    assert np.abs(o["T"]).max() > 1e-3  # the source heats the lattice
    compare(g, o, storage)


def test_heat_generation_full_size_heat_sink():
    """The 128 x 64 x 32 heat sink with the source (beta_max 1e-3), FP32."""
    lat = with_source(I.heat_sink(re=50.0, seed=4, q_flux=0.0), 1e-3, 1.0, 0.0, 5)
    g = run_gpu(lat, "fp32", 30, 20, K=10)
    o = run_oracle(lat, 30, 20)
    compare(g, o, "fp32")


def test_heat_generation_objective_value():
    """J_Q on the GPU equals -w_qgen sum beta_max (1 - gamma)(1 - T) over
    non-wall nodes of the GPU's own temperature field (Eq. 72)."""
    from paper_2501_02161_gb300.solver import Solver
    lat = with_source(I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=0.0, seed=4), 0.05, 0.7, 0.0, 1)
    lat.w_pin = 0.0
    s = Solver.from_lattice(lat, storage="fp64")
    r = s.forward(tol=0, max_steps=300, check_every=100)
    _, _, T = s.fields(torch.float64)
    T = T.cpu().numpy()
    nw = (lat.flags & 7) != I.WALL
    want = -0.7 * np.sum(0.05 * (1 - lat.gamma[nw]) * (1 - T[nw]))
    assert r.J == pytest.approx(want, rel=1e-12)
    s.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_nonzero_initial_temperature(storage):
    """The temperature lattice starts from g = w T0; with T0 != 0 that state
    is not a fixed point of the collision (the advection term moves it), so
    the first step must collide it like every later state."""
    lat = I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=5e-3, seed=4)
    lat.T0 = 0.3
    g = run_gpu(lat, storage, 60, 40, K=20)
    o = run_oracle(lat, 60, 40)
    compare(g, o, storage)
