"""Seeded synthetic lattices: node flags, design field gamma and boundary values.

This module only builds inputs. It holds none of the method's arithmetic (no
equilibrium, collision, boundary scheme or adjoint), so both the CUDA path and
the FP64 oracle can take their inputs from it.

Flag byte per node (the layout the C-ABI documents):
  bits 0-2  node type   0 FLUID, 1 WALL (full-way bounce-back), 2 VEL (Zou-He
            velocity inlet, Eq. 7), 3 PRES (Zou-He fixed-density outlet, Eq. 8)
  bits 3-5  inward normal of an open boundary or heated wall:
            0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z
  bit 6     on a WALL node: HEAT, injects a heat flux towards its normal;
            on a PRES node: T-inlet, the temperature is held at T_in
            (a pressure-driven inlet)
  bit 7     reserved (0)

Boundary values, 4 numbers per node (only read at VEL / PRES nodes):
  VEL:  (ux, uy, uz, T_in)      PRES: (rho, 0, 0, T_in used with bit 6)

Faces of the lattice box are periodic seams unless Lattice.mirror marks an
axis (bit a) whose two faces are symmetry planes half a node beyond them.

Node linear index n = x + nx*(y + ny*z); arrays are returned flat in that order.

The paper's geometries (pipe bend, Fig. 1 and Fig. 9; microchannel heat sink,
Fig. 15) exist only as schematics, so these generators stand in for them with
the sizes of the workloads they are used for.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

FLUID, WALL, VEL, PRES = 0, 1, 2, 3
NORMAL_CODES = {(1, 0, 0): 0, (-1, 0, 0): 1, (0, 1, 0): 2, (0, -1, 0): 3,
                (0, 0, 1): 4, (0, 0, -1): 5}
HEAT_BIT = 1 << 6

D2Q9, D3Q19 = 0, 1
GAMMA_EQ12, GAMMA_LINEAR = 0, 1


def make_flag(kind: int, normal=(1, 0, 0), heat: bool = False) -> int:
    return (kind & 7) | (NORMAL_CODES[tuple(normal)] << 3) | (HEAT_BIT if heat else 0)


@dataclass
class Lattice:
    """A synthetic problem: geometry + design field + physical parameters."""
    name: str
    stencil: int
    nx: int
    ny: int
    nz: int
    flags: np.ndarray          # uint8[N]
    gamma: np.ndarray          # float64[N]
    bcval: np.ndarray          # float64[N*4]
    tau: float | None = None   # relaxation time, when the problem gives it directly
    rho0: float = 1.0
    gamma_model: int = GAMMA_EQ12
    thermal: bool = False
    kappa_f: float = 0.0       # fluid thermal diffusivity, when given directly (lattice units)
    # the problem in physical terms instead of tau / kappa_f: Reynolds number
    # Re = U L / nu with velocity scale u_ref (or a pressure drop dp) and length
    # scale l_ref, and Prandtl number pr = nu / kappa_f; the solver and the
    # oracle each turn these into tau and kappa_f
    re: float | None = None
    u_ref: float = 0.0
    l_ref: float = 0.0
    dp: float = 0.0
    pr: float | None = None
    k_ratio: float = 1.0       # solid / fluid conductivity ratio
    q_flux: float = 0.0        # heat added per step at each HEAT wall node
    T0: float = 0.0            # initial temperature
    w_pin: float = 1.0         # objective weight of mean inlet pressure
    w_tmean: float = 0.0       # objective weight of mean temperature
    beta_max: float = 0.0      # heat generation in the solid, Q = beta_max (1-gamma)(1-T) (Eq. 69)
    w_qgen: float = 0.0        # objective weight of J_Q = -sum Q (Eq. 72)
    mirror: int = 0            # axes with symmetry planes beyond both faces: bit a for axis a
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dims(self):
        return (self.nx, self.ny, self.nz)


def idx(nx, ny, x, y, z=0):
    return x + nx * (y + ny * z)


# --------------------------------------------------------------------------
# seeded random fields
# --------------------------------------------------------------------------

def uniform_noise(n: int, seed: int) -> np.ndarray:
    """U[0,1) per node from numpy's PCG64 with the given seed."""
    return np.random.default_rng(seed).random(n)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(3.0 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def gaussian_filter_nearest(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur truncated at 3 sigma, edges clamped (nearest)."""
    k = _gauss_kernel(sigma)
    r = (len(k) - 1) // 2
    out = a.astype(np.float64)
    for ax in range(out.ndim):
        if out.shape[ax] == 1:
            continue
        pad = [(0, 0)] * out.ndim
        pad[ax] = (r, r)
        p = np.pad(out, pad, mode="edge")
        acc = np.zeros_like(out)
        for j, kj in enumerate(k):
            sl = [slice(None)] * out.ndim
            sl[ax] = slice(j, j + out.shape[ax])
            acc += kj * p[tuple(sl)]
        out = acc
    return out


def filtered_design(shape_zyx, seed: int, sigma: float = 3.0,
                    fluid_fraction: float = 0.75, sharpness: float = 3.0) -> np.ndarray:
    """A near-binary random design in [0,1] from Gaussian-filtered uniform noise.

    Filtered U[0,1) noise has a standard deviation of only about 0.01 at
    sigma=3, so clipping it leaves gamma ~ 0.5 everywhere: a uniform, very
    strong Brinkman drag that no topology-optimisation design has.  The field
    is therefore standardised and passed through a smooth step
    gamma = (1 + tanh(sharpness (z - z_q))) / 2 placed at the quantile z_q that
    leaves `fluid_fraction` of the nodes fluid-like, which keeps the noise's
    spatial structure (blobs of about sigma cells) and the [0,1] range.
    """
    n = int(np.prod(shape_zyx))
    g = gaussian_filter_nearest(uniform_noise(n, seed).reshape(shape_zyx), sigma)
    s = g.std()
    z = (g - g.mean()) / (s if s > 0 else 1.0)
    zq = np.quantile(z, 1.0 - fluid_fraction)
    return np.clip(0.5 * (1.0 + np.tanh(sharpness * (z - zq))), 0.0, 1.0)


# --------------------------------------------------------------------------
# inlet profiles (prescribed boundary data)
# --------------------------------------------------------------------------

def parabola(j: int, w: int) -> float:
    s = (j + 0.5) / w
    return 4.0 * s * (1.0 - s)


# --------------------------------------------------------------------------
# geometries
# --------------------------------------------------------------------------

def pipe_bend_2d(nx: int = 64, ny: int = 64, width: int = 16, umax: float = 0.05,
                 tau: float = 0.6, gamma_value: float = 0.5,
                 gamma_model: int = GAMMA_EQ12) -> Lattice:
    """2D pipe bend (Fig. 1): inlet on the left face, outlet on the top face.

    Walls on the outer ring; inlet x=0, y in [ny/8, ny/8+W) with a parabolic
    Zou-He velocity profile; outlet y=ny-1, x in [5nx/8, 5nx/8+W) at rho=1.
    gamma is uniform on non-wall nodes.
    """
    flags = np.zeros((ny, nx), np.uint8)
    gam = np.full((ny, nx), gamma_value)
    bc = np.zeros((ny, nx, 4))
    flags[0, :] = flags[-1, :] = WALL
    flags[:, 0] = flags[:, -1] = WALL
    y0 = ny // 8
    x0 = (5 * nx) // 8
    for j in range(width):
        y = y0 + j
        flags[y, 0] = make_flag(VEL, (1, 0, 0))
        bc[y, 0, :] = (umax * parabola(j, width), 0.0, 0.0, 0.0)
        x = x0 + j
        flags[ny - 1, x] = make_flag(PRES, (0, -1, 0))
        bc[ny - 1, x, :] = (1.0, 0.0, 0.0, 0.0)
    gam[(flags & 7) == WALL] = 0.0
    lat = Lattice("pipe_bend_2d", D2Q9, nx, ny, 1, flags.ravel(), gam.ravel(),
                  bc.ravel(), tau=tau, gamma_model=gamma_model)
    lat.meta.update(width=width, umax=umax)
    return lat


def pipe_bend_3d(n: int = 64, width: int | None = None, umax: float = 0.05,
                 re: float = 100.0, seed: int = 1, sigma: float = 3.0,
                 gamma_uniform: float | None = None, ny: int | None = None,
                 nz: int | None = None, gamma_model: int = GAMMA_EQ12) -> Lattice:
    """3D pipe bend (Fig. 9): square inlet on x=0, square outlet on y=ny-1.

    Inlet x=0, y in [ny/8, ny/8+W), z centred; outlet y=ny-1, x in
    [5nx/8, 5nx/8+W), z centred; W = n/4 by default (16 at 64^3).  gamma is the
    filtered random design on interior nodes and 1 on the openings.
    """
    nx = n
    ny = ny or n
    nz = nz or n
    w = width or max(2, n // 4)
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[0, :, :] = flags[-1, :, :] = WALL
    flags[:, 0, :] = flags[:, -1, :] = WALL
    flags[:, :, 0] = flags[:, :, -1] = WALL
    y0 = ny // 8
    x0 = (5 * nx) // 8
    z0 = nz // 2 - w // 2
    for a in range(w):
        for b in range(w):
            prof = 16.0 * umax * (parabola(a, w) / 4.0) * (parabola(b, w) / 4.0)
            flags[z0 + b, y0 + a, 0] = make_flag(VEL, (1, 0, 0))
            bc[z0 + b, y0 + a, 0, :] = (prof, 0.0, 0.0, 0.0)
            flags[z0 + b, ny - 1, x0 + a] = make_flag(PRES, (0, -1, 0))
            bc[z0 + b, ny - 1, x0 + a, :] = (1.0, 0.0, 0.0, 0.0)
    if gamma_uniform is not None:
        gam = np.full((nz, ny, nx), float(gamma_uniform))
    else:
        gam = filtered_design((nz, ny, nx), seed, sigma)
    kind = flags & 7
    gam[(kind == VEL) | (kind == PRES)] = 1.0
    gam[kind == WALL] = 0.0
    lat = Lattice(f"pipe_bend_3d_{nx}x{ny}x{nz}", D3Q19, nx, ny, nz,
                  flags.ravel(), gam.ravel(), bc.ravel(), gamma_model=gamma_model,
                  re=re, u_ref=umax, l_ref=float(w))
    lat.meta.update(width=w, umax=umax, re=re, seed=seed)
    return lat


def heat_sink(nx: int = 128, ny: int = 64, nz: int = 32, umax: float = 0.05,
              re: float = 50.0, pr: float = 7.0, k_ratio: float = 100.0,
              q_flux: float = 1e-3, seed: int = 4, sigma: float = 3.0,
              w_pin: float = 1.0, w_tmean: float = 1.0,
              gamma_uniform: float | None = None, plenum: int = 4,
              gamma_model: int = GAMMA_EQ12) -> Lattice:
    """Microchannel heat sink (Fig. 15), flow along +x through a design block.

    Inlet face x=0 and outlet face x=nx-1 over the interior cross-section
    (velocity inlet with a product parabola and T=0; fixed-density outlet).
    Walls on y=0, y=ny-1, z=0, z=nz-1; the z=0 wall under the interior is
    heated with q_flux per node and step.  Re uses the inlet's peak speed and
    its smaller side; Pr sets the fluid diffusivity.
    The first and last `plenum` x-layers are fluid (gamma = 1).
    """
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[0, :, :] = flags[-1, :, :] = WALL
    flags[:, 0, :] = flags[:, -1, :] = WALL
    wy, wz = ny - 2, nz - 2
    for z in range(1, nz - 1):
        for y in range(1, ny - 1):
            prof = 16.0 * umax * (parabola(y - 1, wy) / 4.0) * (parabola(z - 1, wz) / 4.0)
            flags[z, y, 0] = make_flag(VEL, (1, 0, 0))
            bc[z, y, 0, :] = (prof, 0.0, 0.0, 0.0)
            flags[z, y, nx - 1] = make_flag(PRES, (-1, 0, 0))
            bc[z, y, nx - 1, :] = (1.0, 0.0, 0.0, 0.0)
    heat = make_flag(WALL, (0, 0, 1), heat=True)
    flags[0, 1:ny - 1, 1:nx - 1] = heat
    if gamma_uniform is not None:
        gam = np.full((nz, ny, nx), float(gamma_uniform))
    else:
        gam = filtered_design((nz, ny, nx), seed, sigma)
        # inlet and outlet plenums outside the design block (Fig. 15)
        gam[:, :, :plenum] = 1.0
        gam[:, :, nx - plenum:] = 1.0
    kind = flags & 7
    gam[(kind == VEL) | (kind == PRES)] = 1.0
    gam[kind == WALL] = 0.0
    width = min(wy, wz)
    lat = Lattice(f"heat_sink_{nx}x{ny}x{nz}", D3Q19, nx, ny, nz, flags.ravel(),
                  gam.ravel(), bc.ravel(), gamma_model=gamma_model,
                  thermal=True, k_ratio=k_ratio, q_flux=q_flux,
                  T0=0.0, w_pin=w_pin, w_tmean=w_tmean,
                  re=re, u_ref=umax, l_ref=float(width), pr=pr)
    lat.meta.update(width=width, umax=umax, re=re, pr=pr, seed=seed)
    return lat


def heat_sink_quarter(nx: int = 96, ny: int = 24, nz: int = 12, re: float = 60.0,
                      u_scale: float = 0.05, pr: float = 7.1, k_ratio: float = 100.0,
                      beta_max: float = 1e-4, seed: int = 8, sigma: float = 3.0,
                      plenum: int = 4, T_in: float = 0.0,
                      gamma_uniform: float | None = None) -> Lattice:
    """A quarter of a symmetric microchannel heat sink, the setup of the paper's
    Sec. 3.3 (Fig. 15 is a schematic only): flow along +x driven by a pressure
    drop between a fixed-density inlet at x=0 (rho_in = rho0 + 3 dp, the
    temperature held at T_in) and a fixed-density outlet at x=nx-1 (rho0);
    walls on the outer faces y=ny-1 and z=nz-1; symmetry planes beyond the low
    y and z faces (the cut planes of the full channel, whose other three
    quarters are their mirror images; the outer faces reflect too, which the
    walls there make immaterial); heat generated in the solid,
    Q = beta_max (1 - gamma)(1 - T), and the objective J = -sum Q (Eq. 72).
    Re is set through the pressure drop (Eq. 70): dp = rho0 u_scale^2, so the
    velocity scale is u_scale, with the full channel's smaller open side
    2 min(ny-1, nz-1) as the length scale."""
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[-1, :, :] = WALL
    flags[:, -1, :] = WALL
    dp = u_scale * u_scale          # rho0 = 1
    inlet = make_flag(PRES, (1, 0, 0), heat=True)   # bit 6 on a PRES node: T held at T_in
    outlet = make_flag(PRES, (-1, 0, 0))
    flags[:nz - 1, :ny - 1, 0] = inlet
    bc[:nz - 1, :ny - 1, 0, :] = (1.0 + 3.0 * dp, 0.0, 0.0, T_in)
    flags[:nz - 1, :ny - 1, nx - 1] = outlet
    bc[:nz - 1, :ny - 1, nx - 1, :] = (1.0, 0.0, 0.0, 0.0)
    if gamma_uniform is not None:
        gam = np.full((nz, ny, nx), float(gamma_uniform))
    else:
        gam = filtered_design((nz, ny, nx), seed, sigma)
        gam[:, :, :plenum] = 1.0
        gam[:, :, nx - plenum:] = 1.0
    kind = flags & 7
    gam[kind == PRES] = 1.0
    gam[kind == WALL] = 0.0
    lat = Lattice(f"heat_sink_quarter_{nx}x{ny}x{nz}", D3Q19, nx, ny, nz, flags.ravel(),
                  gam.ravel(), bc.ravel(), thermal=True, k_ratio=k_ratio, q_flux=0.0, T0=0.0,
                  w_pin=0.0, w_tmean=0.0, beta_max=beta_max, w_qgen=1.0,
                  re=re, u_ref=0.0, dp=dp, l_ref=float(2 * min(ny - 1, nz - 1)), pr=pr,
                  mirror=(1 << 1) | (1 << 2))
    lat.meta.update(seed=seed, u_scale=u_scale)
    return lat


def unfold(lat: Lattice, axis: int) -> Lattice:
    """The lattice doubled across the symmetry plane beyond its low face on
    `axis` (0 x, 1 y, 2 z): the mirror image of every node, normal and
    velocity is placed below the original, and the axis becomes periodic (its
    faces in the doubled lattice are the mirror images of the original's
    other face).  Solving the unfolded lattice solves the symmetric whole of
    which `lat` is the part beyond the plane."""
    bit = 1 << axis
    if not lat.mirror & bit:
        raise ValueError("that axis has no symmetry plane")
    dims = [lat.nz, lat.ny, lat.nx]
    d = 2 - axis                                     # array dimension of the axis
    fl = lat.flags.reshape(dims)
    kind = fl & 7
    code = (fl >> 3) & 7
    flip_code = np.where((code >> 1) == axis, code ^ 1, code).astype(np.uint8)
    has_normal = (kind >= VEL) | ((fl & HEAT_BIT) != 0)
    fl_m = np.where(has_normal, (fl & 0xC7) | (flip_code << 3), fl).astype(np.uint8)
    bc = lat.bcval.reshape(dims + [4]).copy()
    bc_m = bc.copy()
    bc_m[..., axis] *= np.where(kind == VEL, -1.0, 1.0)
    g = lat.gamma.reshape(dims)
    cat = lambda a, b: np.concatenate([np.flip(b, d), a], axis=d)
    flags2 = cat(fl, fl_m)
    bc2 = np.concatenate([np.flip(bc_m, d), bc], axis=d)
    g2 = cat(g, g)
    nd = list(dims)
    nd[d] *= 2
    out = Lattice(**{**lat.__dict__, "name": lat.name + f"_unfolded{'xyz'[axis]}",
                     "nx": nd[2], "ny": nd[1], "nz": nd[0], "flags": flags2.ravel(),
                     "gamma": g2.ravel(), "bcval": bc2.ravel(), "mirror": lat.mirror & ~bit,
                     "meta": dict(lat.meta)})
    return out


def random_fields(lat: Lattice, seed: int, scale: float = 1.0):
    """Seeded N(0,1) vectors shaped like a population field (for dot tests)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(lat.n)


# named stand-ins for the benchmark workloads (keyword overrides allowed)
WORKLOADS = {
    # 2D D2Q9 pipe bend 64 x 64, tau 0.6, gamma 0.5 (solved in FP64)
    "pipe_bend_2d_64x64": lambda **kw: pipe_bend_2d(**kw),
    # 3D D3Q19 pipe bend 64^3, filtered design field, Re 50 / 100 / 500
    "pipe_bend_3d_64cubed": lambda **kw: pipe_bend_3d(**{"n": 64, "re": 50.0, **kw}),
    # microchannel heat sink 128 x 64 x 32, D3Q19 + D3Q7, Pr 7
    "heat_sink_128x64x32": lambda **kw: heat_sink(**{"nx": 128, "ny": 64, "nz": 32, "re": 50.0, **kw}),
    # the differentiation workload: heat sink 96 x 48 x 24
    "heat_sink_96x48x24": lambda **kw: heat_sink(**{"nx": 96, "ny": 48, "nz": 24, "re": 50.0, **kw}),
}


def workload(name: str, **kw) -> "Lattice":
    """The lattice of a named workload (see WORKLOADS); served requests are
    built by serve.lattice_for from their own shape and Re."""
    if name not in WORKLOADS:
        raise ValueError(f"unknown workload {name!r}; known: {sorted(WORKLOADS)}")
    return WORKLOADS[name](**kw)


def six_port_box(nx: int = 14, ny: int = 12, nz: int = 10, width: int = 3,
                 umax: float = 0.03, tau: float = 0.8, seed: int = 9,
                 swap: bool = False, thermal: bool = False) -> Lattice:
    """A walled box with one square opening centred on each of its six faces.

    Without swap the openings on the low faces (normals +x, +y, +z) are
    velocity inlets and those on the high faces (-x, -y, -z) fixed-density
    outlets; swap exchanges the roles, so the two variants together cover both
    boundary kinds in all six orientations.  gamma is seeded U[0.3, 1).
    """
    flags = np.zeros((nz, ny, nx), np.uint8)
    bc = np.zeros((nz, ny, nx, 4))
    flags[0] = flags[-1] = WALL
    flags[:, 0] = flags[:, -1] = WALL
    flags[:, :, 0] = flags[:, :, -1] = WALL
    dims = (nx, ny, nz)
    for ax in range(3):
        for side in (0, 1):
            normal = [0, 0, 0]
            normal[ax] = 1 if side == 0 else -1
            inlet = (side == 0) != swap
            kind = VEL if inlet else PRES
            others = [a for a in range(3) if a != ax]
            c0 = [dims[a] // 2 - width // 2 for a in others]
            for i in range(width):
                for j in range(width):
                    pos = [0, 0, 0]
                    pos[ax] = 0 if side == 0 else dims[ax] - 1
                    pos[others[0]] = c0[0] + i
                    pos[others[1]] = c0[1] + j
                    x, y, z = pos
                    flags[z, y, x] = make_flag(kind, tuple(normal))
                    if inlet:
                        prof = umax * parabola(i, width) * parabola(j, width)
                        v = [0.0, 0.0, 0.0]
                        v[ax] = prof * normal[ax]
                        bc[z, y, x, :] = (*v, 0.1 * (ax + 1))
                    else:
                        bc[z, y, x, :] = (1.0 - 0.002 * ax, 0.0, 0.0, 0.0)
    rng = np.random.default_rng(seed)
    gam = 0.3 + 0.7 * rng.random((nz, ny, nx))
    kind = flags & 7
    gam[kind == WALL] = 0.0
    lat = Lattice(f"six_port_{'b' if swap else 'a'}", D3Q19, nx, ny, nz, flags.ravel(),
                  gam.ravel(), bc.ravel(), tau=tau)
    if thermal:
        lat.thermal = True
        lat.kappa_f = 0.02
        lat.k_ratio = 4.0
        lat.w_tmean = 1.0
        f3 = lat.flags.reshape(nz, ny, nx)
        f3[0, 1:ny - 1, 1:nx - 1] = np.where((f3[0, 1:ny - 1, 1:nx - 1] & 7) == WALL,
                                             make_flag(WALL, (0, 0, 1), heat=True),
                                             f3[0, 1:ny - 1, 1:nx - 1])
        lat.q_flux = 5e-3
    return lat
