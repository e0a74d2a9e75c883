"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Both sides take the same seeded inputs and run the same number of steps of
the same discrete maps (forward Eq. 35, adjoint Eq. 53-56), so every field can
be compared node by node.  Tolerances: FP64 storage rel-L2 <= 1e-11;
FP32 storage rel-L2 <= 1e-5 on rho, u, T and <= 1e-4 on f*, g* and dJ/dgamma.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-11, 1e-11), "fp32": (1e-5, 1e-4)}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run_gpu(lat, storage, fsteps, asteps, K=None):
    from paper_2501_02161_gb300.solver import Solver
    K = K or max(1, min(fsteps, asteps, 50))
    s = Solver.from_lattice(lat, storage=storage)
    rf = s.forward(tol=0, max_steps=fsteps, check_every=K)
    ra = s.adjoint(tol=0, max_steps=asteps, check_every=K)
    rho, u, T = s.fields(torch.float64)
    fs, gs = s.adjoint_fields(torch.float64)
    out = dict(rho=rho.cpu().numpy(), u=u.cpu().numpy().T, J=rf.J,
               sens=s.sensitivity(dtype=torch.float64).cpu().numpy(),
               fs=fs.cpu().numpy().T, rf=rf, ra=ra)
    if T is not None:
        out["T"] = T.cpu().numpy()
        out["gs"] = gs.cpu().numpy().T
    s.close()
    return out


def run_oracle(lat, fsteps, asteps):
    orc = O.Oracle(lat)
    orc.flow_run(fsteps)
    out = {}
    if lat.thermal:
        orc.thermal_run(fsteps)
        out["T"] = orc.temperature()
        orc.thermal_adjoint_run(asteps)
        orc.finish_thermal_adjoint()
        out["gs"] = orc.thermal_adjoint_post_bc().reshape(orc.N, 7)
    orc.adjoint_run(asteps)
    rho, u = orc.macro()
    out.update(rho=rho, u=u, J=orc.objective(), sens=orc.sensitivity(),
               fs=orc.adjoint_post_bc().reshape(orc.N, orc.Q))
    return out


def compare(g, o, storage):
    tf, ta = TOL[storage]
    errs = {k: rel(g[k], o[k]) for k in ("rho", "u", "sens", "fs") + (("T", "gs") if "T" in o else ())}
    errs["J"] = abs(g["J"] - o["J"]) / abs(o["J"])
    for k in ("rho", "u", "T", "J"):
        if k in errs:
            assert errs[k] <= tf, errs
    for k in ("sens", "fs", "gs"):
        if k in errs:
            assert errs[k] <= ta, errs
    return errs


def lattices_small():
    return [
        I.pipe_bend_2d(),  # the 64 x 64 D2Q9 pipe bend at full size
        I.pipe_bend_2d(nx=37, ny=29, width=7, tau=0.7, gamma_value=0.8,
                       gamma_model=I.GAMMA_LINEAR),
        I.pipe_bend_3d(n=20, width=5, re=20.0, seed=2, ny=18, nz=13),
        I.pipe_bend_3d(n=16, width=4, re=20.0, seed=3, gamma_model=I.GAMMA_LINEAR),
        I.six_port_box(),
        I.six_port_box(nx=11, ny=13, nz=9, swap=True),
    ]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("lat", lattices_small(), ids=lambda l: l.name)
def test_flow_parity_fixed_steps(lat, storage):
    if lat.stencil == I.D2Q9 and storage not in ("fp64", "fp32"):
        pytest.skip()
    g = run_gpu(lat, storage, 240, 160, K=40)
    o = run_oracle(lat, 240, 160)
    compare(g, o, storage)


def thermal_lattices():
    return [I.heat_sink(nx=24, ny=14, nz=10, re=10.0, q_flux=5e-3, seed=4),
            I.heat_sink(nx=19, ny=11, nz=9, re=10.0, q_flux=5e-3, seed=6,
                        gamma_model=I.GAMMA_LINEAR),
            I.six_port_box(thermal=True),
            I.six_port_box(nx=11, ny=13, nz=9, swap=True, thermal=True)]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("lat", thermal_lattices(), ids=lambda l: l.name)
def test_thermal_parity_fixed_steps(lat, storage):
    g = run_gpu(lat, storage, 200, 150, K=50)
    o = run_oracle(lat, 200, 150)
    compare(g, o, storage)


def test_pipe_bend_64cubed_full_size():
    """The 64^3 D3Q19 FP32 pipe bend at full size, every node compared."""
    lat = I.pipe_bend_3d(n=64, re=100.0, seed=1)
    g = run_gpu(lat, "fp32", 60, 40, K=20)
    o = run_oracle(lat, 60, 40)
    compare(g, o, "fp32")


def test_heat_sink_full_size():
    """The 128 x 64 x 32 heat sink (D3Q19 + D3Q7) at full size."""
    lat = I.heat_sink(re=50.0, seed=4)
    g = run_gpu(lat, "fp32", 30, 20, K=10)
    o = run_oracle(lat, 30, 20)
    compare(g, o, "fp32")


def test_converged_config_2d_matches_oracle():
    """D2Q9 FP64 64x64, forward and adjoint iterated to 1e-8 on both sides."""
    from paper_2501_02161_gb300.solver import Solver
    lat = I.pipe_bend_2d()
    s = Solver.from_lattice(lat, storage="fp64")
    rf = s.forward(tol=1e-8, max_steps=20000, check_every=1000)
    ra = s.adjoint(tol=1e-8, max_steps=20000, check_every=1000)
    orc = O.Oracle(lat)
    fo = orc.flow_solve(1e-8, 20000, 1000)
    ao = orc.adjoint_solve(1e-8, 20000, 1000)
    assert rf.steps == fo[0] and ra.steps == ao[0]
    sens = s.sensitivity(dtype=torch.float64).cpu().numpy()
    assert rel(sens, orc.sensitivity()) < 1e-10
    assert abs(rf.J - orc.objective()) < 1e-12 * abs(orc.objective())


def test_repeatable_and_warm_start_bitwise():
    from paper_2501_02161_gb300.solver import Solver
    lat = I.pipe_bend_3d(n=24, width=6, re=30.0, seed=5)
    s = Solver.from_lattice(lat, storage="fp32")
    s.forward(tol=0, max_steps=200, check_every=50)
    a = s.fields()[1].clone()
    s.forward(tol=0, max_steps=200, check_every=50)
    b = s.fields()[1].clone()
    s.forward(tol=0, max_steps=100, check_every=50)
    s.forward(tol=0, max_steps=100, check_every=50, reset=False)
    c = s.fields()[1].clone()
    assert torch.equal(a, b) and torch.equal(a, c)


def test_new_inputs_on_a_used_context_match_a_fresh_context():
    """Re-setting the same inputs keeps the captured step graphs and gives
    bit-identical results; inputs with other inlet / non-wall node counts (and
    other parameters) must behave exactly like a fresh context."""
    from paper_2501_02161_gb300.solver import Solver

    def solve(s):
        rf = s.forward(tol=0, max_steps=200, check_every=100)
        ra = s.adjoint(tol=0, max_steps=100, check_every=100)
        return rf.J, ra.I, s.sensitivity(dtype=torch.float64).cpu()

    a = I.pipe_bend_3d(n=24, width=6, re=30.0, seed=5)
    b = I.pipe_bend_3d(n=24, width=4, re=15.0, seed=6)   # other N_in, N_nonwall, tau
    s = Solver.from_lattice(a, storage="fp32")
    first = solve(s)
    for lat in (a, b, a):
        s.set_flags(torch.as_tensor(lat.flags))
        s.set_gamma(torch.as_tensor(lat.gamma, dtype=torch.float32))
        s.set_bc_values(torch.as_tensor(lat.bcval, dtype=torch.float32))
        s.set_lattice_params(lat)
        got = solve(s)
        fresh = Solver.from_lattice(lat, storage="fp32")
        ref = solve(fresh)
        fresh.close()
        assert got[0] == ref[0] and got[1] == ref[1] and torch.equal(got[2], ref[2]), lat.name
    assert first[0] == got[0] and torch.equal(first[2], got[2])
    s.close()


def test_degenerate_periodic_box_stays_at_rest():
    """All-fluid periodic lattice with no boundaries: the rest state is a fixed point."""
    from paper_2501_02161_gb300.solver import Solver
    for (nx, ny, nz) in [(3, 2, 2), (1, 1, 1), (33, 1, 2)]:
        N = nx * ny * nz
        lat = I.Lattice("box", I.D3Q19, nx, ny, nz, np.zeros(N, np.uint8),
                        np.full(N, 0.5), np.zeros(4 * N), tau=0.7, w_pin=0.0)
        s = Solver.from_lattice(lat, storage="fp64")
        s.forward(tol=0, max_steps=10, check_every=5)
        rho, u, _ = s.fields()
        assert torch.allclose(rho, torch.ones_like(rho)) and u.abs().max() == 0


def test_error_paths():
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver
    lat = I.pipe_bend_3d(n=12, width=3, re=10.0)
    s = Solver.from_lattice(lat, storage="fp32")
    with pytest.raises(C.LBMError) as e:
        s.adjoint(tol=0, max_steps=10)
    assert e.value.code == C.LBM_ERR_ORDER
    with pytest.raises(C.LBMError) as e:
        s.sensitivity()
    assert e.value.code == C.LBM_ERR_ORDER
    bad = torch.as_tensor(lat.flags, device="cuda").clone()
    bad[5] = 0x80
    with pytest.raises(C.LBMError) as e:
        s.set_flags(bad)
    assert e.value.code == C.LBM_ERR_ARG
    with pytest.raises(C.LBMError) as e:
        s.set_params(tau=0.5)
    assert e.value.code == C.LBM_ERR_ARG
    r = s.forward(tol=1e-14, max_steps=100, check_every=50)
    assert r.status == C.LBM_NOT_CONVERGED and r.steps == 100
    g = torch.as_tensor(lat.gamma, dtype=torch.float32, device="cuda").clone()
    g[700] = float("nan")
    s.set_gamma(g)
    with pytest.raises(C.LBMError) as e:
        s.forward(tol=1e-6, max_steps=200, check_every=50)
    assert e.value.code == C.LBM_ERR_DIVERGED
