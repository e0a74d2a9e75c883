"""Symmetry planes and the pressure-driven temperature inlet on the GPU
against the FP64 oracle (whose symmetry planes are pinned against the
unfolded full domain): the quarter-domain heat sink of Sec. 3.3 with heat
generation (Eq. 69-72), and planes on every axis of lattices whose faces
carry walls and open boundaries of both kinds.  Same steps on both sides,
every node compared."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I
from test_gpu_parity import compare, rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


def quarter(nx=24, ny=9, nz=7, **kw):
    lat = I.heat_sink_quarter(nx=nx, ny=ny, nz=nz, re=20.0, beta_max=0.02, plenum=3, seed=3, **kw)
    rng = np.random.default_rng(5)
    fluid = (lat.flags & 7) == I.FLUID
    lat.gamma = np.where(fluid, 0.3 + 0.7 * rng.random(lat.n), lat.gamma)
    return lat


def boxes():
    a = I.six_port_box(nx=12, ny=10, nz=9, thermal=True)
    a.mirror = 7
    b = I.six_port_box(nx=11, ny=13, nz=9, swap=True, thermal=True)
    b.mirror = 5
    c = I.pipe_bend_3d(n=16, width=4, re=20.0, seed=3)
    c.mirror = 2
    return [a, b, c]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_quarter_heat_sink_parity(storage):
    lat = quarter()
    g = run_gpu(lat, storage, 200, 150, K=50)
    o = run_oracle(lat, 200, 150)
    assert np.abs(o["T"]).max() > 1e-3
    compare(g, o, storage)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("lat", boxes(), ids=lambda l: f"{l.name}_m{l.mirror}")
def test_symmetry_planes_on_every_axis_parity(lat, storage):
    g = run_gpu(lat, storage, 160, 120, K=40)
    o = run_oracle(lat, 160, 120)
    compare(g, o, storage)


def test_symmetry_planes_in_2d():
    lat = I.pipe_bend_2d(nx=20, ny=18, width=5, tau=0.7, gamma_value=0.8)
    lat.mirror = 3
    g = run_gpu(lat, "fp64", 200, 150, K=50)
    o = run_oracle(lat, 200, 150)
    compare(g, o, "fp64")


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_quarter_heat_sink_sixteen_bit(storage):
    """16-bit flow populations on a lattice with symmetry planes (the one-node
    kernels: the paired step needs periodic x); bounds of the 16-bit tests."""
    from test_gpu_precision import BOUND
    lat = quarter()
    g = run_gpu(lat, storage, 300, 200, K=100)
    o = run_oracle(lat, 300, 200)
    for k in ("rho", "u", "T", "sens", "fs"):
        assert rel(g[k], o[k]) <= BOUND[storage][k], (k, rel(g[k], o[k]))
