"""The paper's heat-generation variant in the FP64 oracle: a source
Q = beta_max (1 - gamma)(1 - T) in the temperature collision (Eq. 69, 71)
and the objective J_Q = -sum Q (Eq. 72).  Pinned to a closed form, to the
tangent/transposition identities of the thermal step, and to central finite
differences of the converged objective.  (The CUDA path's parity with it is
in test_gpu_heatgen.py.)"""
import ctypes

import numpy as np
import pytest

from paper_2501_02161_gb300 import inputs as I

from test_oracle_pins import _fd_check, _sample_cells


def test_uniform_source_relaxes_temperature_geometrically(oracle_mod):
    """All-solid periodic box at rest: streaming moves nothing and the source
    gives T(t+1) = T(t) + beta (1 - T(t)), so T(t) = 1 - (1 - T0)(1 - beta)^t."""
    O = oracle_mod
    nx, ny, nz = 3, 4, 2
    N = nx * ny * nz
    beta, T0 = 0.08, 0.2
    lat = I.Lattice("box", I.D3Q19, nx, ny, nz, np.zeros(N, np.uint8), np.zeros(N), np.zeros(4 * N),
                    tau=0.8, w_pin=0.0, thermal=True, kappa_f=0.05, k_ratio=2.0, T0=T0,
                    beta_max=beta)
    orc = O.Oracle(lat)
    for t in (1, 5, 17):
        orc.reset()
        orc.thermal_run(t)
        assert np.allclose(orc.temperature(), 1 - (1 - T0) * (1 - beta) ** t, rtol=0, atol=1e-14)


def _heat_sink_with_source():
    """A small heat sink whose fluid nodes carry a seeded gamma in (0.3, 0.9),
    so that the source heats every one of them (at this size the generator's
    design field leaves them all at gamma = 1, where Q vanishes)."""
    lat = I.heat_sink(nx=8, ny=6, nz=6, re=5.0, pr=1.0, k_ratio=3.0, q_flux=0.0, seed=7)
    rng = np.random.default_rng(11)
    fluid = (lat.flags & 7) == I.FLUID
    lat.gamma = np.where(fluid, 0.3 + 0.6 * rng.random(lat.n), lat.gamma)
    lat.beta_max, lat.w_qgen, lat.w_tmean = 0.05, 1.0, 0.0
    return lat


def test_thermal_tangent_and_transposition_with_the_source(oracle_mod):
    O = oracle_mod
    orc = O.Oracle(_heat_sink_with_source())
    orc.flow_run(60)
    orc.thermal_run(60)
    assert orc.temperature().max() > 1e-3  # the source is active
    rng = np.random.default_rng(4)
    dg = rng.standard_normal(orc.g.size)
    df = rng.standard_normal(orc.f.size)

    def step(g, f):
        out = np.zeros_like(g)
        work = np.zeros_like(g)
        O.lib().orc_thermal_step(ctypes.byref(orc.P), O._p(orc.flags, ctypes.c_uint8), O._p(orc.gamma),
                                 O._p(orc.bcval), O._p(f), O._p(g), O._p(out), O._p(work))
        return out
    h = 1e-6
    fd = (step(orc.g + h * dg, orc.f + h * df) - step(orc.g - h * dg, orc.f - h * df)) / (2 * h)
    tl = orc.thermal_tangent_of(dg, df)
    assert np.abs(fd - tl).max() <= 1e-7 * np.abs(tl).max()
    v = rng.standard_normal(orc.g.size)
    cpl, _ = orc.thermal_coupling_of(v)
    rhs = orc.thermal_adjoint_step_of(v, with_source=False) @ dg + cpl @ df
    assert abs(v @ tl - rhs) <= 1e-12 * (abs(v @ tl) + np.abs(v).sum())


def test_objective_is_minus_the_generated_heat(oracle_mod):
    O = oracle_mod
    lat = _heat_sink_with_source()
    lat.w_pin = 0.0
    orc = O.Oracle(lat)
    orc.flow_run(30)
    orc.thermal_run(30)
    T = orc.temperature()
    nw = (lat.flags & 7) != I.WALL
    want = -np.sum(lat.beta_max * (1 - lat.gamma[nw]) * (1 - T[nw]))
    assert orc.objective() == pytest.approx(want, rel=1e-13)


def test_sensitivity_with_heat_generation_vs_finite_difference(oracle_mod):
    lat = _heat_sink_with_source()
    _fd_check(oracle_mod, lat, _sample_cells(lat, 5, 3))
