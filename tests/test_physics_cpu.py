"""The problem's physical parameters through the C-ABI (host-only calls, no
GPU): tau from Re, U and L (Eq. 3), U from a pressure drop (Eq. 70) and the
fluid diffusivity from Pr.  The library's conversion is compared with the
oracle driver's own (written separately) and with the closed forms."""
import ctypes
import math

import numpy as np
import pytest

from paper_2501_02161_gb300 import inputs as I


@pytest.fixture(scope="module")
def C():
    from paper_2501_02161_gb300 import build as B
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    B.build()
    from paper_2501_02161_gb300 import _capi
    return _capi


def convert(C, **kw):
    base = dict(re=1.0, u_ref=0.0, l_ref=1.0, dp=0.0, pr=0.0, rho0=1.0, gamma_model=0,
                k_ratio=1.0, q_flux=0.0, T0=0.0, beta_max=0.0)
    base.update(kw)
    ph = C.lbm_physics(*[base[f] for f, _ in C.lbm_physics._fields_])
    out = C.lbm_params()
    code = C.lib().lbm_physics_to_params(ctypes.byref(ph), ctypes.byref(out))
    return code, out


def test_tau_from_reynolds_number(C):
    # Re = U L / nu, nu = (tau - 1/2)/3: U = 0.05, L = 16, Re = 100 gives
    # nu = 0.008 and tau = 0.524
    code, p = convert(C, re=100.0, u_ref=0.05, l_ref=16.0)
    assert code == C.LBM_OK
    assert p.tau == pytest.approx(0.524, rel=1e-15)
    # the 2D workload's tau = 0.6 with U = 0.05 and L = 16 is Re = 24
    code, p = convert(C, re=24.0, u_ref=0.05, l_ref=16.0)
    assert p.tau == pytest.approx(0.6, rel=1e-15)


def test_pressure_drop_velocity_scale_and_prandtl_number(C):
    # Eq. 70: U = sqrt(dp / rho0); with dp = 1e-4, rho0 = 1: U = 0.01
    code, p = convert(C, re=2.0, u_ref=0.0, dp=1e-4, l_ref=10.0, pr=7.1, rho0=1.0)
    assert code == C.LBM_OK
    nu = 0.01 * 10.0 / 2.0
    assert p.tau == pytest.approx(0.5 + 3 * nu, rel=1e-14)
    assert p.kappa_f == pytest.approx(nu / 7.1, rel=1e-14)
    code, p2 = convert(C, re=2.0, u_ref=0.0, dp=4e-4, l_ref=10.0, rho0=4.0)
    assert p2.tau == pytest.approx(p.tau, rel=1e-14)   # dp / rho0 is what counts


def test_other_fields_are_copied(C):
    code, p = convert(C, re=50.0, u_ref=0.05, l_ref=14.0, pr=7.0, rho0=1.3, gamma_model=1,
                      k_ratio=100.0, q_flux=1e-3, T0=0.25, beta_max=1e-5)
    assert code == C.LBM_OK
    assert (p.rho0, p.gamma_model, p.k_ratio, p.q_flux, p.T0, p.beta_max) == (1.3, 1, 100.0, 1e-3, 0.25, 1e-5)


@pytest.mark.parametrize("kw", [dict(re=0.0, u_ref=0.05), dict(re=-1.0, u_ref=0.05),
                                dict(re=10.0, u_ref=0.0, dp=0.0), dict(re=10.0, u_ref=0.05, l_ref=0.0),
                                dict(re=10.0, u_ref=0.05, rho0=0.0), dict(re=10.0, u_ref=0.05, pr=-1.0),
                                dict(re=float("nan"), u_ref=0.05)])
def test_bad_physics_is_rejected(C, kw):
    code, _ = convert(C, **kw)
    assert code == C.LBM_ERR_ARG


def test_library_and_oracle_conversions_agree_on_the_workloads(C):
    from oracle import oracle as O
    for lat in [I.pipe_bend_3d(n=16, width=4, re=50.0), I.pipe_bend_3d(n=32, re=500.0),
                I.heat_sink(nx=24, ny=14, nz=10, re=10.0), I.heat_sink(re=400.0)]:
        code, p = convert(C, re=lat.re, u_ref=lat.u_ref, l_ref=lat.l_ref, dp=lat.dp,
                          pr=lat.pr or 0.0, rho0=lat.rho0)
        tau, kappa = O.relaxation_of(lat)
        assert code == C.LBM_OK
        assert p.tau == pytest.approx(tau, rel=1e-15, abs=0)
        assert p.kappa_f == pytest.approx(kappa, rel=1e-14, abs=0)
