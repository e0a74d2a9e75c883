"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Eq. 7, 8, 58, 59, 60), moment identities of the lattices and
the equilibrium (Eq. 4-6), exactness of central differences on quadratic maps,
transposition identities (the dot-product test of Eq. 37/52-56), closed-form
flows and central finite differences of the objective (Fig. 7's check made
quantitative).
"""
from fractions import Fraction
import os

import numpy as np
import pytest

from paper_2501_02161_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_matrix(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


def tiny_problem(O, stencil=0, tau=0.8, gamma_model=0, rho0=1.0):
    return O.make_problem(stencil, 4, 4, 1 if stencil == 0 else 4, tau, rho0, gamma_model)


def node_bc(O, P, flag, bcv, fs):
    import ctypes
    out = np.zeros_like(fs)
    O.lib().orc_node_bc(ctypes.byref(P), flag, O._p(np.asarray(bcv, float)),
                        O._p(np.ascontiguousarray(fs)), O._p(out))
    return out


def node_bc_jac(O, P, flag, Q):
    import ctypes
    B = np.zeros(Q * Q)
    O.lib().orc_node_bc_jacobian(ctypes.byref(P), flag, O._p(B))
    return B.reshape(Q, Q)


def node_collide(O, P, flag, gamma, f):
    import ctypes
    out = np.zeros_like(f)
    O.lib().orc_node_collide(ctypes.byref(P), flag, gamma, O._p(np.ascontiguousarray(f)),
                             O._p(out))
    return out


def node_collide_jac(O, P, flag, gamma, f):
    import ctypes
    Q = len(f)
    C = np.zeros(Q * Q)
    O.lib().orc_node_collision_jacobian(ctypes.byref(P), flag, gamma,
                                        O._p(np.ascontiguousarray(f)), O._p(C))
    return C.reshape(Q, Q)


def node_feq(O, P, rho, u, gamma, Q):
    import ctypes
    out = np.zeros(Q)
    O.lib().orc_node_equilibrium(ctypes.byref(P), rho, O._p(np.asarray(u, float)), gamma,
                                 O._p(out))
    return out


# ---------------------------------------------------------------------------
# lattice tables (Eq. 5) and the equilibrium (Eq. 4, 6, 12)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which,cs2", [(0, 1 / 3), (1, 1 / 3), (2, 1 / 4)])
def test_lattice_moments(oracle_mod, which, cs2):
    e, w, opp = oracle_mod.lattice_tables(which)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ e).max() < 1e-15
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(m2, cs2 * np.eye(3)[: m2.shape[0]] * (np.abs(e).sum(0) > 0), atol=1e-15)
    assert (e[opp] == -e).all()
    if which in (0, 1):  # fourth-order isotropy of the flow lattices
        m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
        d = 2 if which == 0 else 3
        dd = np.eye(3)
        iso = (np.einsum("ab,cd->abcd", dd, dd) + np.einsum("ac,bd->abcd", dd, dd)
               + np.einsum("ad,bc->abcd", dd, dd)) / 9.0
        assert np.allclose(m4[:d, :d, :d, :d], iso[:d, :d, :d, :d], atol=1e-15)


def test_d2q9_order_matches_eq7(oracle_mod):
    # Eq. 7 on the left face treats 1, 5, 8 as unknown (e_x > 0), 3, 6, 7 as
    # outgoing (e_x < 0) and 2, 4 as tangential; Eq. 8 on the bottom face
    # treats 2, 5, 6 as unknown (e_y > 0).
    e, w, _ = oracle_mod.lattice_tables(0)
    assert set(np.where(e[:, 0] > 0)[0]) == {1, 5, 8}
    assert set(np.where(e[:, 0] < 0)[0]) == {3, 6, 7}
    assert set(np.where(e[:, 1] > 0)[0]) == {2, 5, 6}
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.mark.parametrize("stencil,Q", [(0, 9), (1, 19)])
@pytest.mark.parametrize("model", [0, 1])
def test_equilibrium_moments(oracle_mod, stencil, Q, model):
    O = oracle_mod
    rho0 = 1.1
    P = tiny_problem(O, stencil, gamma_model=model, rho0=rho0)
    e, _, _ = O.lattice_tables(stencil)
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        if stencil == 0:
            u[2] = 0
        gam = rng.random()
        feq = node_feq(O, P, rho, u, gam, Q)
        assert abs(feq.sum() - rho) < 1e-14
        # first moment rho0 * gamma * u for both design couplings (Brinkman drag)
        assert np.allclose(e.T @ feq, rho0 * gam * u, atol=1e-15)
        m2 = np.einsum("i,ia,ib->ab", feq, e, e)
        g2 = gam * gam if model == 0 else gam
        d = 2 if stencil == 0 else 3
        expect = rho / 3 * np.eye(3) + rho0 * g2 * np.outer(u, u)
        assert np.allclose(m2[:d, :d], expect[:d, :d], atol=1e-14)


# ---------------------------------------------------------------------------
# boundary operator: the paper's printed Zou-He (Eq. 7, 8) and Jacobians
# (Eq. 58, 59, 60)
# ---------------------------------------------------------------------------

def test_inlet_matches_eq7_values(oracle_mod):
    O = oracle_mod
    rho0 = 1.0
    P = tiny_problem(O, 0, rho0=rho0)
    rng = np.random.default_rng(11)
    fs = 1 / 9 + 0.01 * rng.standard_normal(9)
    uin = 0.037
    out = node_bc(O, P, I.make_flag(I.VEL, (1, 0, 0)), [uin, 0, 0, 0], fs)
    f = fs
    assert np.isclose(out[1], f[3] + 2 / 3 * rho0 * uin, atol=1e-15)
    assert np.isclose(out[5], f[7] + 1 / 6 * rho0 * uin + 0.5 * (f[4] - f[2]), atol=1e-15)
    assert np.isclose(out[8], f[6] + 1 / 6 * rho0 * uin - 0.5 * (f[4] - f[2]), atol=1e-15)
    # the density line of Eq. 7 holds for the completed node
    rho = f[0] + f[2] + f[4] + 2 * (f[3] + f[6] + f[7]) + rho0 * uin
    assert np.isclose(out.sum(), rho, atol=1e-15)
    keep = [0, 2, 3, 4, 6, 7]
    assert np.array_equal(out[keep], fs[keep])


def test_outlet_matches_eq8_values(oracle_mod):
    O = oracle_mod
    rho0 = 1.0
    P = tiny_problem(O, 0, rho0=rho0)
    rng = np.random.default_rng(12)
    fs = 1 / 9 + 0.01 * rng.standard_normal(9)
    out = node_bc(O, P, I.make_flag(I.PRES, (0, 1, 0)), [1.0, 0, 0, 0], fs)
    f = fs
    v = 1 - (f[0] + f[1] + f[3] + 2 * (f[4] + f[7] + f[8])) / rho0
    assert np.isclose(out[2], f[4] + 2 / 3 * rho0 * v, atol=1e-15)
    assert np.isclose(out[5], f[7] + 1 / 6 * rho0 * v + 0.5 * (f[3] - f[1]), atol=1e-15)
    assert np.isclose(out[6], f[8] + 1 / 6 * rho0 * v - 0.5 * (f[3] - f[1]), atol=1e-15)
    assert np.isclose(out.sum(), 1.0, atol=1e-15)


def test_inlet_jacobian_is_eq58(oracle_mod):
    O = oracle_mod
    P = tiny_problem(O, 0)
    B = node_bc_jac(O, P, I.make_flag(I.VEL, (1, 0, 0)), 9)
    assert np.array_equal(B, load_matrix("eq58_inlet_jacobian.txt"))


def test_adjoint_inlet_is_eq59(oracle_mod):
    O = oracle_mod
    P = tiny_problem(O, 0)
    B = node_bc_jac(O, P, I.make_flag(I.VEL, (1, 0, 0)), 9)
    assert np.array_equal(B.T, load_matrix("eq59_adjoint_inlet.txt"))


def test_adjoint_outlet_is_eq60(oracle_mod):
    O = oracle_mod
    P = tiny_problem(O, 0)
    B = node_bc_jac(O, P, I.make_flag(I.PRES, (0, 1, 0)), 9)
    assert np.allclose(B.T, load_matrix("eq60_adjoint_outlet.txt"), atol=1e-15)


NORMALS_2D = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
NORMALS_3D = NORMALS_2D + [(0, 0, 1), (0, 0, -1)]


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("kind", [I.VEL, I.PRES])
def test_zou_he_moments_every_face(oracle_mod, stencil, kind):
    """The completed node carries exactly the prescribed velocity (or density
    with zero tangential velocity), and the jacobian is exact (B is affine)."""
    O = oracle_mod
    rho0 = 1.05
    P = tiny_problem(O, stencil, rho0=rho0)
    e, w, opp = O.lattice_tables(stencil)
    Q = len(w)
    rng = np.random.default_rng(5)
    for nrm in (NORMALS_2D if stencil == 0 else NORMALS_3D):
        n = np.array(nrm)
        flag = I.make_flag(kind, nrm)
        for _ in range(3):
            fs = w * (1 + 0.05 * rng.standard_normal(Q))
            u = 0.04 * rng.standard_normal(3)
            if stencil == 0:
                u[2] = 0
            rho_out = 1 + 0.02 * rng.standard_normal()
            bcv = [*u, 0.0] if kind == I.VEL else [rho_out, 0, 0, 0]
            out = node_bc(O, P, flag, bcv, fs)
            d = e @ n
            assert np.array_equal(out[d <= 0], fs[d <= 0])
            mom = e.T @ out / rho0
            if kind == I.VEL:
                assert np.allclose(mom, u, atol=1e-14)
                K0, Km = fs[d == 0].sum(), fs[d < 0].sum()
                assert np.isclose(out.sum(), K0 + 2 * Km + rho0 * u @ n, atol=1e-14)
            else:
                assert np.isclose(out.sum(), rho_out, atol=1e-14)
                assert np.allclose(mom - (mom @ n) * n, 0, atol=1e-14)
            # non-equilibrium bounce-back along the normal
            k = int(np.where((e == n).all(1))[0][0])
            un = mom @ n
            assert np.isclose(out[k] - out[opp[k]], 6 * w[k] * rho0 * un, atol=1e-14)
            # B affine: the stored jacobian equals central differences
            B = node_bc_jac(O, P, flag, Q)
            h = 1e-3
            for j in range(Q):
                dj = np.zeros(Q)
                dj[j] = h
                col = (node_bc(O, P, flag, bcv, fs + dj) - node_bc(O, P, flag, bcv, fs - dj)) / (2 * h)
                assert np.allclose(col, B[:, j], atol=1e-12)


@pytest.mark.parametrize("stencil", [0, 1])
def test_wall_is_symmetric_permutation(oracle_mod, stencil):
    O = oracle_mod
    P = tiny_problem(O, stencil)
    Q = 9 if stencil == 0 else 19
    B = node_bc_jac(O, P, I.make_flag(I.WALL), Q)
    assert np.array_equal(B, B.T)
    assert np.array_equal(B @ B, np.eye(Q))


# ---------------------------------------------------------------------------
# collision and its jacobian (Eq. 36, 63)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("model", [0, 1])
def test_collision_jacobian_exact_central_difference(oracle_mod, stencil, model):
    """C is quadratic in f, so central differences equal its jacobian."""
    O = oracle_mod
    P = tiny_problem(O, stencil, tau=0.7, gamma_model=model, rho0=0.9)
    e, w, _ = O.lattice_tables(stencil)
    Q = len(w)
    rng = np.random.default_rng(9)
    f = w * (1 + 0.1 * rng.standard_normal(Q))
    for gam in (0.0, 0.37, 1.0):
        C = node_collide_jac(O, P, I.FLUID, gam, f)
        h = 1e-2
        for j in range(Q):
            dj = np.zeros(Q)
            dj[j] = h
            col = (node_collide(O, P, I.FLUID, gam, f + dj)
                   - node_collide(O, P, I.FLUID, gam, f - dj)) / (2 * h)
            assert np.allclose(col, C[:, j], atol=1e-13)
        out = node_collide(O, P, I.FLUID, gam, f)
        assert np.isclose(out.sum(), f.sum(), atol=1e-15)
        # momentum relaxes to gamma u at rate 1/tau (drag (1-gamma)/tau)
        m0 = e.T @ f
        assert np.allclose(e.T @ out, m0 * (1 - (1 - gam) / 0.7), atol=1e-15)


# ---------------------------------------------------------------------------
# whole-step tangent, dot-product test, conservation
# ---------------------------------------------------------------------------

def _advance(O, lat, steps):
    orc = O.Oracle(lat)
    orc.flow_run(steps)
    return orc


def small_lattices():
    yield I.pipe_bend_2d(nx=12, ny=12, width=4, tau=0.8, gamma_value=0.6)
    yield I.pipe_bend_2d(nx=12, ny=10, width=3, tau=0.7, gamma_value=0.8,
                         gamma_model=I.GAMMA_LINEAR)
    yield I.pipe_bend_3d(n=8, width=2, re=2.0, seed=3)


@pytest.mark.parametrize("lat", list(small_lattices()), ids=lambda l: l.name)
def test_tangent_equals_central_difference_of_step(oracle_mod, lat):
    """F = B S C is quadratic in f: central differences are exact."""
    O = oracle_mod
    orc = _advance(O, lat, 40)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(orc.f.size)
    h = 1e-3
    fd = (orc.flow_step_of(orc.f + h * w) - orc.flow_step_of(orc.f - h * w)) / (2 * h)
    tl = orc.tangent_of(w)
    assert np.abs(fd - tl).max() <= 1e-11 * max(1.0, np.abs(tl).max())


@pytest.mark.parametrize("lat", list(small_lattices()), ids=lambda l: l.name)
def test_dot_product_adjoint_of_step(oracle_mod, lat):
    """<v, F' w> = <F'^T v, w> for the whole step (S unitary, Eq. 37)."""
    O = oracle_mod
    orc = _advance(O, lat, 40)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(orc.f.size)
        w = rng.standard_normal(orc.f.size)
        lhs = v @ orc.tangent_of(w)
        rhs = orc.adjoint_step_of(v, with_source=False) @ w
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.abs(v).sum())


def test_closed_box_conserves_mass(oracle_mod):
    O = oracle_mod
    nx = ny = nz = 6
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[0] = flags[-1] = I.WALL
    flags[:, 0] = flags[:, -1] = I.WALL
    flags[:, :, 0] = flags[:, :, -1] = I.WALL
    lat = I.Lattice("box", I.D3Q19, nx, ny, nz, flags.ravel(), np.full(nx * ny * nz, 0.7),
                    np.zeros(nx * ny * nz * 4), tau=0.9)
    orc = O.Oracle(lat)
    rng = np.random.default_rng(0)
    orc.f *= 1 + 0.01 * rng.standard_normal(orc.f.size)
    m0 = orc.f.sum()
    orc.flow_run(50)
    assert abs(orc.f.sum() - m0) < 1e-12 * m0


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("stencil", [0, 1])
def test_uniform_momentum_decay_law(oracle_mod, model, stencil):
    """Periodic box with uniform gamma: rho0 u(t) = rho0 u0 (1-(1-gamma)/tau)^t."""
    O = oracle_mod
    nx, ny, nz = 5, 4, (1 if stencil == 0 else 3)
    N = nx * ny * nz
    tau, gam, rho0 = 0.75, 0.4, 1.0
    lat = I.Lattice("periodic", stencil, nx, ny, nz, np.zeros(N, np.uint8),
                    np.full(N, gam), np.zeros(4 * N), tau=tau, gamma_model=model)
    orc = O.Oracle(lat)
    P1 = tiny_problem(O, stencil, tau=tau, gamma_model=model, rho0=rho0)
    u0 = np.array([0.03, -0.02, 0.01 if stencil == 1 else 0.0])
    feq = node_feq(O, P1, 1.0, u0, 1.0, orc.Q)
    orc.f[:] = np.tile(feq, N)
    orc.flow_run(7)
    _, u = orc.macro()
    assert np.allclose(u, u0 * (1 - (1 - gam) / tau) ** 7, atol=1e-15)


# ---------------------------------------------------------------------------
# closed-form flows
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("stencil", [0, 1])
def test_couette_linear_profile(oracle_mod, stencil):
    """Zou-He moving and resting walls, periodic along the flow: linear u."""
    O = oracle_mod
    nx, ny, nz = 4, 9, (1 if stencil == 0 else 3)
    U = 0.04
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[:, 0, :] = I.make_flag(I.VEL, (0, 1, 0))
    flags[:, -1, :] = I.make_flag(I.VEL, (0, -1, 0))
    bc[:, -1, :, 0] = U
    N = nx * ny * nz
    lat = I.Lattice("couette", stencil, nx, ny, nz, flags.ravel(), np.ones(N), bc.ravel(),
                    tau=0.8)
    orc = O.Oracle(lat)
    orc.flow_run(6000)
    rho, u = orc.macro()
    uy = u[:, 0].reshape(nz, ny, nx)
    expect = U * np.arange(ny) / (ny - 1)
    assert np.allclose(uy, expect[None, :, None], atol=1e-12)
    assert np.allclose(rho, 1.0, atol=1e-12)
    assert np.abs(u[:, 1:]).max() < 1e-13


def test_poiseuille_curvature_matches_pressure_gradient(oracle_mod):
    """Developed channel flow between bounce-back walls: nu u'' = p'/rho0 with
    p = rho/3 and nu = (tau-1/2)/3 (Eq. 3), exactly in the discrete bulk."""
    O = oracle_mod
    nx, ny, tau, umax = 48, 11, 0.9, 0.01
    flags = np.zeros((ny, nx), np.uint8)
    bc = np.zeros((ny, nx, 4))
    flags[0, :] = flags[-1, :] = I.WALL
    for y in range(1, ny - 1):
        flags[y, 0] = I.make_flag(I.VEL, (1, 0, 0))
        bc[y, 0, 0] = umax * I.parabola(y - 1, ny - 2)
        flags[y, -1] = I.make_flag(I.PRES, (-1, 0, 0))
        bc[y, -1, 0] = 1.0
    N = nx * ny
    lat = I.Lattice("poiseuille", I.D2Q9, nx, ny, 1, flags.ravel(), np.ones(N), bc.ravel(),
                    tau=tau)
    orc = O.Oracle(lat)
    steps, res = orc.flow_solve(1e-14, 400000, 2000)
    assert res < 1e-13
    rho, u = orc.macro()
    ux = u[:, 0].reshape(ny, nx)
    rho = rho.reshape(ny, nx)
    nu = (tau - 0.5) / 3
    for x in range(18, 30):
        d2 = ux[3:ny - 2, x] - 2 * ux[2:ny - 3, x] + ux[1:ny - 4, x]
        dpdx = (rho[ny // 2, x + 1] - rho[ny // 2, x - 1]) / 2 / 3
        assert np.allclose(nu * d2, dpdx, rtol=1e-8, atol=1e-14)
        assert np.abs(u[:, 1].reshape(ny, nx)[1:ny - 1, x]).max() < 1e-10


def test_conduction_linear_profile(oracle_mod):
    """Resting fluid between a heated wall (flux q) and a T=0 boundary:
    T(z) - T(z+1) = q / kappa with kappa = (tau_g - 1/2)/4."""
    O = oracle_mod
    nx, ny, nz = 3, 3, 14
    q, kappa = 2e-3, 0.05
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[0] = I.make_flag(I.WALL, (0, 0, 1), heat=True)
    flags[-1] = I.make_flag(I.VEL, (0, 0, -1))
    N = nx * ny * nz
    lat = I.Lattice("column", I.D3Q19, nx, ny, nz, flags.ravel(), np.ones(N), bc.ravel(),
                    tau=0.8, thermal=True, kappa_f=kappa, k_ratio=1.0, q_flux=q)
    orc = O.Oracle(lat)
    orc.flow_run(10)
    steps, res = orc.thermal_solve(1e-14, 200000, 2000)
    assert res < 1e-13
    T = orc.temperature().reshape(nz, ny, nx)
    dT = T[1:nz - 2] - T[2:nz - 1]
    assert np.allclose(dT, q / kappa, rtol=1e-10)


# ---------------------------------------------------------------------------
# thermal step: tangent and transposition
# ---------------------------------------------------------------------------

def tiny_heat_sink(gamma_model=0):
    return I.heat_sink(nx=8, ny=6, nz=6, re=5.0, pr=1.0, k_ratio=3.0, q_flux=1e-2,
                       seed=7, gamma_model=gamma_model)


def test_thermal_tangent_and_dot_product(oracle_mod):
    O = oracle_mod
    lat = tiny_heat_sink()
    orc = O.Oracle(lat)
    orc.flow_run(60)
    orc.thermal_run(60)
    rng = np.random.default_rng(8)
    dg = rng.standard_normal(orc.g.size)
    df = rng.standard_normal(orc.f.size)
    h = 1e-6
    gp = orc.g.copy()
    fp = orc.f.copy()

    def step(g, f):
        import ctypes
        out = np.zeros_like(g)
        work = np.zeros_like(g)
        O.lib().orc_thermal_step(ctypes.byref(orc.P), O._p(orc.flags, ctypes.c_uint8),
                                 O._p(orc.gamma), O._p(orc.bcval), O._p(f), O._p(g),
                                 O._p(out), O._p(work))
        return out
    fd = (step(gp + h * dg, fp + h * df) - step(gp - h * dg, fp - h * df)) / (2 * h)
    tl = orc.thermal_tangent_of(dg, df)
    assert np.abs(fd - tl).max() <= 1e-7 * np.abs(tl).max()
    # transposition: <v, G_g dg + G_f df> = <G_g^T v, dg> + <G_f^T v, df>
    v = rng.standard_normal(orc.g.size)
    lhs = v @ tl
    cpl, _ = orc.thermal_coupling_of(v)
    rhs = orc.thermal_adjoint_step_of(v, with_source=False) @ dg + cpl @ df
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(v).sum())


# ---------------------------------------------------------------------------
# sensitivity against central finite differences of the converged objective
# ---------------------------------------------------------------------------

def _converged_J(O, lat, gamma, warm_f=None, warm_g=None, tol=1e-14, chunk=1000,
                 max_steps=400000):
    lat2 = I.Lattice(**{**lat.__dict__, "gamma": gamma})
    orc = O.Oracle(lat2)
    if warm_f is not None:
        orc.f[:] = warm_f
    if warm_g is not None and orc.g is not None:
        orc.g[:] = warm_g
    s, r = orc.flow_solve(tol, max_steps, chunk)
    assert r < 10 * tol, (s, r)
    if orc.g is not None:
        s, r = orc.thermal_solve(tol, max_steps, chunk)
        assert r < 10 * tol, (s, r)
    return orc.objective(), orc


def _fd_check(O, lat, cells, h=1e-5, rtol=1e-6):
    J0, base = _converged_J(O, lat, lat.gamma)
    base.solve_all(tol=1e-14, max_steps=400000, check_every=1000)
    sens = base.sensitivity()
    scale = np.abs(sens).max()
    assert scale > 0
    for c in cells:
        gp = lat.gamma.copy()
        gm = lat.gamma.copy()
        gp[c] += h
        gm[c] -= h
        Jp, _ = _converged_J(O, lat, gp, base.f, base.g)
        Jm, _ = _converged_J(O, lat, gm, base.f, base.g)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - sens[c]) <= rtol * scale + 1e-6 * abs(fd), (c, fd, sens[c])


def _sample_cells(lat, k, seed):
    nonwall = np.where((lat.flags & 7) != I.WALL)[0]
    rng = np.random.default_rng(seed)
    bc = np.where(((lat.flags & 7) == I.VEL) | ((lat.flags & 7) == I.PRES))[0]
    pick = list(rng.choice(nonwall, size=min(k, len(nonwall)), replace=False))
    pick += list(bc[:2])
    return sorted(set(int(p) for p in pick))


@pytest.mark.parametrize("model", [I.GAMMA_EQ12, I.GAMMA_LINEAR])
def test_sensitivity_vs_finite_difference_2d(oracle_mod, model):
    lat = I.pipe_bend_2d(nx=10, ny=10, width=3, tau=0.9, gamma_value=0.7, gamma_model=model)
    rng = np.random.default_rng(1)
    lat.gamma = np.where((lat.flags & 7) == I.WALL, 0.0, 0.4 + 0.5 * rng.random(lat.n))
    _fd_check(oracle_mod, lat, _sample_cells(lat, 8, 0))


def test_sensitivity_vs_finite_difference_3d(oracle_mod):
    lat = I.pipe_bend_3d(n=7, width=2, re=1.5, seed=5)
    _fd_check(oracle_mod, lat, _sample_cells(lat, 5, 1))


def test_sensitivity_vs_finite_difference_thermal(oracle_mod):
    lat = tiny_heat_sink()
    _fd_check(oracle_mod, lat, _sample_cells(lat, 5, 2))

