"""Symmetry planes and the pressure-driven heat sink in the FP64 oracle.

A face of the lattice box can be a symmetry plane instead of a periodic seam
(the quarter domain of the paper's Sec. 3.3): streaming across it reads the
mirror-image node with the population reflected.  Pinned by (a) the exact
equality of a quarter lattice and the full symmetric lattice it unfolds to
(periodic streaming only), field by field through the whole solve sequence;
(b) mirrored geometries giving mirrored fields (no symmetry plane involved);
(c) the dot-product test of the flow and thermal steps with symmetry planes,
a pressure-driven inlet that holds the temperature (Eq. 70) and the heat
source of Eq. 69/71; (d) central finite differences of the converged J_Q of
Eq. 72 on the quarter lattice."""
import ctypes

import numpy as np
import pytest

from paper_2501_02161_gb300 import inputs as I

from test_oracle_pins import _fd_check, _sample_cells

D3Q19_E = None


def _solve_sequence(O, lat, fwd=150, therm=150, tadj=100, adj=100):
    orc = O.Oracle(lat)
    orc.flow_run(fwd)
    if lat.thermal:
        orc.thermal_run(therm)
        orc.thermal_adjoint_run(tadj)
        orc.finish_thermal_adjoint()
    orc.adjoint_run(adj)
    out = {"f": orc.f.copy(), "fs": orc.adjoint_post_bc(), "sens": orc.sensitivity(),
           "J": orc.objective()}
    if lat.thermal:
        out["g"] = orc.g.copy()
        out["gs"] = orc.thermal_adjoint_post_bc()
    return out


def _block(a, lat_full, q, nz, ny):
    """the part of a full-lattice array (nodes x q values) beyond both planes"""
    return a.reshape(lat_full.nz, lat_full.ny, lat_full.nx, q)[nz:, ny:]


def tiny_quarter(**kw):
    base = dict(nx=14, ny=5, nz=4, re=20.0, beta_max=0.02, plenum=2, seed=3)
    base.update(kw)
    lat = I.heat_sink_quarter(**base)
    rng = np.random.default_rng(5)
    fluid = (lat.flags & 7) == I.FLUID
    lat.gamma = np.where(fluid, 0.3 + 0.7 * rng.random(lat.n), lat.gamma)
    return lat


@pytest.mark.parametrize("objective", ["qgen", "mean_T"])
def test_quarter_equals_the_unfolded_full_domain(oracle_mod, objective):
    O = oracle_mod
    q = tiny_quarter()
    if objective == "mean_T":
        q.w_qgen, q.w_tmean = 0.0, 1.0
    full = I.unfold(I.unfold(q, 1), 2)
    assert full.mirror == 0 and (full.ny, full.nz) == (2 * q.ny, 2 * q.nz)
    a = _solve_sequence(O, q)
    b = _solve_sequence(O, full)
    assert np.abs(a["g"]).max() > 1e-4
    # wall nodes hold populations that no other node reads (bounce-back
    # leftovers that arrive through the periodic seam): compare the others
    live = (q.flags & 7) != I.WALL
    for key, Q in (("f", 19), ("fs", 19), ("g", 7), ("gs", 7)):
        blk = _block(b[key], full, Q, q.nz, q.ny).reshape(-1, Q)[live]
        # the whole's J_Q sums four quarters; its mean-T objective averages them
        scale = 1.0 if key in ("f", "g") or objective == "qgen" else 4.0
        got = a[key].reshape(-1, Q)[live]
        assert np.allclose(got, blk * scale, rtol=0, atol=1e-12 * np.abs(blk * scale).max()), key
    sb = _block(b["sens"], full, 1, q.nz, q.ny).reshape(-1)
    want = sb if objective == "qgen" else 4.0 * sb
    assert np.allclose(a["sens"], want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert a["J"] == pytest.approx(b["J"] / (4.0 if objective == "qgen" else 1.0), rel=1e-12)


def _reflect(lat, axis):
    """the same problem reflected in axis (0 x, 1 y, 2 z): node, normal,
    velocity and gamma mirrored; periodic faces stay periodic"""
    dims = [lat.nz, lat.ny, lat.nx]
    d = 2 - axis
    fl = lat.flags.reshape(dims)
    kind = fl & 7
    code = (fl >> 3) & 7
    has_normal = (kind >= I.VEL) | ((fl & I.HEAT_BIT) != 0)
    code2 = np.where((code >> 1) == axis, code ^ 1, code).astype(np.uint8)
    fl2 = np.flip(np.where(has_normal, (fl & 0xC7) | (code2 << 3), fl).astype(np.uint8), d)
    bc = lat.bcval.reshape(dims + [4]).copy()
    bc[..., axis] *= np.where(kind == I.VEL, -1.0, 1.0)
    bc = np.flip(bc, d)
    g = np.flip(lat.gamma.reshape(dims), d)
    return I.Lattice(**{**lat.__dict__, "flags": np.ascontiguousarray(fl2).ravel(),
                        "bcval": np.ascontiguousarray(bc).ravel(),
                        "gamma": np.ascontiguousarray(g).ravel(), "meta": dict(lat.meta)})


def _mirror_index(e, axis):
    want = e.copy()
    want[:, axis] *= -1
    return np.array([int(np.where((e == w).all(axis=1))[0][0]) for w in want])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reflected_geometry_gives_reflected_fields(oracle_mod, axis):
    """P6: a problem and its mirror image have mirror-image solutions (six
    openings, both kinds on every face, heated wall, temperature lattice)."""
    O = oracle_mod
    lat = I.six_port_box(nx=9, ny=8, nz=7, width=3, thermal=True)
    lat.beta_max, lat.w_qgen = 0.01, 0.5
    ref = _reflect(lat, axis)
    a = _solve_sequence(O, lat, 120, 120, 80, 80)
    b = _solve_sequence(O, ref, 120, 120, 80, 80)
    e19, _, _ = O.lattice_tables(1)
    e7, _, _ = O.lattice_tables(2)
    d = 2 - axis
    dims = [lat.nz, lat.ny, lat.nx]
    live = (ref.flags.reshape(dims) & 7) != I.WALL
    for key, e in (("f", e19), ("fs", e19), ("g", e7), ("gs", e7)):
        m = _mirror_index(e, axis)
        A = np.flip(a[key].reshape(dims + [len(e)]), d)[..., m][live]
        B = b[key].reshape(dims + [len(e)])[live]
        assert np.allclose(A, B, rtol=0, atol=1e-12 * np.abs(B).max()), key
    sa = np.flip(a["sens"].reshape(dims), d)
    assert np.allclose(sa, b["sens"].reshape(dims), rtol=0, atol=1e-12 * np.abs(sa).max())
    assert a["J"] == pytest.approx(b["J"], rel=1e-13)


def test_dot_product_with_symmetry_planes_and_pressure_inlet(oracle_mod):
    """<v, F' w> = <F'^T v, w> for the flow step and the coupled thermal step
    of the quarter lattice (symmetry planes, pressure-driven inlet holding T,
    heat source)."""
    O = oracle_mod
    orc = O.Oracle(tiny_quarter())
    orc.flow_run(60)
    orc.thermal_run(60)
    rng = np.random.default_rng(12)
    for _ in range(2):
        v = rng.standard_normal(orc.f.size)
        w = rng.standard_normal(orc.f.size)
        lhs = v @ orc.tangent_of(w)
        rhs = orc.adjoint_step_of(v, with_source=False) @ w
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.abs(v).sum())
        vg = rng.standard_normal(orc.g.size)
        dg = rng.standard_normal(orc.g.size)
        df = rng.standard_normal(orc.f.size)
        lhs = vg @ orc.thermal_tangent_of(dg, df)
        cpl, _ = orc.thermal_coupling_of(vg)
        rhs = orc.thermal_adjoint_step_of(vg, with_source=False) @ dg + cpl @ df
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(vg).sum())


def test_sensitivity_of_the_quarter_heat_sink_vs_finite_difference(oracle_mod):
    lat = tiny_quarter(nx=10, ny=4, nz=4)
    _fd_check(oracle_mod, lat, _sample_cells(lat, 5, 2))
