"""Python driver for the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py use it.  It never imports the CUDA package; inputs come from
the seeded generators (paper_2501_02161_gb300.inputs), passed in as arrays.

The solve loops follow the paper's schedule: forward steps f -> B S C f
(Eq. 35), the residual |I(t) - I(t-K)| / |I(t)| with I the mean velocity
magnitude checked every K steps (Sec. 3.1, Fig. 8 text), then the adjoint
iteration started from f*_C = 0 (Eq. 53-56) and the sensitivity of Eq. 66.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")

T_FLUID, T_WALL, T_VEL, T_PRES = 0, 1, 2, 3


def build(force: bool = False, target: str | None = None, mutation: int = 0) -> str:
    """Compile the oracle with the host C compiler (OpenMP over nodes).
    mutation > 0 builds a copy with one planted mistake into `target`."""
    out = target or LIB
    if force or mutation or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               f"-DORC_MUTATION={int(mutation)}", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class Problem(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("gamma_model", ctypes.c_int), ("thermal", ctypes.c_int),
                ("kappa_f", ctypes.c_double), ("k_ratio", ctypes.c_double),
                ("q_flux", ctypes.c_double), ("w_pin", ctypes.c_double),
                ("w_tmean", ctypes.c_double), ("beta_max", ctypes.c_double),
                ("w_qgen", ctypes.c_double), ("mirror", ctypes.c_int)]


_lib = None


def use_library(path: str | None):
    """Load the oracle from `path` (None: the normal build) for later calls."""
    global _lib
    _lib = None
    if path is not None:
        _lib = _load(path)


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def _load(path: str):
    if True:
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Problem)
        d = ctypes.POINTER(ctypes.c_double)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        i32 = ctypes.POINTER(ctypes.c_int)
        lng = ctypes.c_long
        sig = {
            "orc_flow_init": [P, d],
            "orc_flow_step": [P, u8, d, d, d, d, d],
            "orc_flow_run": [P, u8, d, d, d, lng, d],
            "orc_flow_macro": [P, d, d, d],
            "orc_flow_tangent": [P, u8, d, d, d, d],
            "orc_adjoint_bc": [P, u8, d, d],
            "orc_flow_adjoint_step": [P, u8, d, d, d, d, ctypes.c_int, d],
            "orc_flow_adjoint_run": [P, u8, d, d, d, d, lng],
            "orc_flow_sensitivity": [P, u8, d, d, d, d],
            "orc_thermal_init": [P, ctypes.c_double, d],
            "orc_thermal_step": [P, u8, d, d, d, d, d, d],
            "orc_thermal_run": [P, u8, d, d, d, d, lng],
            "orc_thermal_macro": [P, d, d],
            "orc_thermal_tangent": [P, u8, d, d, d, d, d, d],
            "orc_thermal_adjoint_step": [P, u8, d, d, d, d, ctypes.c_int, d],
            "orc_thermal_adjoint_run": [P, u8, d, d, d, d, lng],
            "orc_thermal_coupling": [P, u8, d, d, d, d, d, d],
            "orc_thermal_adjoint_bc": [P, u8, d, d, d, d, d],
            "orc_node_bc": [P, ctypes.c_uint8, d, d, d],
            "orc_node_bc_jacobian": [P, ctypes.c_uint8, d],
            "orc_node_collide": [P, ctypes.c_uint8, ctypes.c_double, d, d],
            "orc_node_collision_jacobian": [P, ctypes.c_uint8, ctypes.c_double, d, d],
            "orc_node_equilibrium": [P, ctypes.c_double, d, ctypes.c_double, d],
            "orc_lattice": [ctypes.c_int, i32, d, i32],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = None
        L.orc_objective.argtypes = [P, u8, d, d]
        L.orc_objective.restype = ctypes.c_double
        L.orc_objective_qgen.argtypes = [P, u8, d, d]
        L.orc_objective_qgen.restype = ctypes.c_double
        L.orc_lattice.restype = ctypes.c_int
        L.orc_cont_adjoint_step.restype = ctypes.c_int
        L.orc_cont_node_bc.argtypes = [P, ctypes.c_uint8, ctypes.c_double, d, d]
        L.orc_cont_node_bc.restype = ctypes.c_int
        return L


def _p(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def lattice_tables(which: int):
    """(e[Q,3], w[Q], opp[Q]) of the oracle's D2Q9 (0), D3Q19 (1) or D3Q7 (2)."""
    e = np.zeros(19 * 3, np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    q = lib().orc_lattice(which, _p(e, ctypes.c_int), _p(w), _p(opp, ctypes.c_int))
    return e[: 3 * q].reshape(q, 3), w[:q].copy(), opp[:q].copy()


def make_problem(stencil, nx, ny, nz, tau, rho0=1.0, gamma_model=0, thermal=False,
                 kappa_f=0.0, k_ratio=1.0, q_flux=0.0, w_pin=1.0, w_tmean=0.0,
                 beta_max=0.0, w_qgen=0.0, mirror=0) -> Problem:
    return Problem(int(stencil), int(nx), int(ny), int(nz), float(tau), float(rho0),
                   int(gamma_model), int(bool(thermal)), float(kappa_f), float(k_ratio),
                   float(q_flux), float(w_pin), float(w_tmean), float(beta_max), float(w_qgen),
                   int(mirror))


def rel_change(a: float, b: float) -> float:
    """|I(t) - I(t-K)| / |I(t)| (Sec. 3.1); 0 when both are exactly zero."""
    d = abs(a - b)
    if d == 0.0:
        return 0.0
    return d / abs(a) if a != 0.0 else float("inf")


def relaxation_of(lat):
    """(tau, kappa_f) of a lattice: as given, or from its Reynolds and Prandtl
    numbers.  Sec. 2.1, Eq. 3: nu = (tau - 1/2) c_s^2 with c_s^2 = 1/3, and
    Re = U L / nu; the velocity scale U is the given one, or sqrt(dp / rho0)
    for a pressure drop dp (Eq. 70); Pr = nu / kappa_f."""
    if lat.re is None:
        return lat.tau, lat.kappa_f
    U = lat.u_ref if lat.u_ref > 0 else float(np.sqrt(lat.dp / lat.rho0))
    nu = U * lat.l_ref / lat.re
    tau = nu / (1.0 / 3.0) + 0.5
    kappa_f = nu / lat.pr if lat.pr else 0.0
    return tau, kappa_f


class Oracle:
    """FP64 forward / adjoint / sensitivity on one synthetic lattice."""

    def __init__(self, lat):
        self.lat = lat
        tau, kappa_f = relaxation_of(lat)
        self.P = make_problem(lat.stencil, lat.nx, lat.ny, lat.nz, tau, lat.rho0,
                              lat.gamma_model, lat.thermal, kappa_f, lat.k_ratio,
                              lat.q_flux, lat.w_pin, lat.w_tmean, lat.beta_max, lat.w_qgen,
                              lat.mirror)
        self.Q = 9 if lat.stencil == 0 else 19
        self.N = lat.n
        self.flags = np.ascontiguousarray(lat.flags, np.uint8)
        self.gamma = np.ascontiguousarray(lat.gamma, np.float64)
        self.bcval = np.ascontiguousarray(lat.bcval, np.float64)
        self.nonwall = (self.flags & 7) != T_WALL
        self.f = np.zeros(self.N * self.Q)
        self.work = np.zeros(self.N * self.Q)
        self.g = np.zeros(self.N * 7) if lat.thermal else None
        self.fsc = np.zeros(self.N * self.Q)
        self.gsc = np.zeros(self.N * 7) if lat.thermal else None
        self.coupling = np.zeros(self.N * self.Q) if lat.thermal else None
        self.sensT = np.zeros(self.N) if lat.thermal else None
        self.reset()

    # ---- forward ---------------------------------------------------------
    def reset(self):
        lib().orc_flow_init(ctypes.byref(self.P), _p(self.f))
        if self.g is not None:
            lib().orc_thermal_init(ctypes.byref(self.P), self.lat.T0, _p(self.g))
        self.fsc[:] = 0.0
        if self.gsc is not None:
            self.gsc[:] = 0.0
            self.coupling[:] = 0.0
            self.sensT[:] = 0.0

    def flow_run(self, nsteps: int):
        if nsteps > 0:
            lib().orc_flow_run(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                               _p(self.gamma), _p(self.bcval), _p(self.f), int(nsteps),
                               _p(self.work))

    def flow_step_of(self, f: np.ndarray) -> np.ndarray:
        out = np.zeros_like(f)
        lib().orc_flow_step(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                            _p(self.gamma), _p(self.bcval), _p(np.ascontiguousarray(f)),
                            _p(out), _p(self.work))
        return out

    def macro(self, f=None):
        f = self.f if f is None else np.ascontiguousarray(f)
        rho = np.zeros(self.N)
        u = np.zeros(self.N * 3)
        lib().orc_flow_macro(ctypes.byref(self.P), _p(f), _p(rho), _p(u))
        return rho, u.reshape(self.N, 3)

    def residual_quantity(self) -> float:
        """I = mean |u| over non-wall nodes."""
        _, u = self.macro()
        return float(np.linalg.norm(u[self.nonwall], axis=1).mean())

    def flow_solve(self, tol: float, max_steps: int, check_every: int = 1000):
        prev = self.residual_quantity()
        steps, res = 0, float("inf")
        while steps < max_steps:
            k = min(check_every, max_steps - steps)
            self.flow_run(k)
            steps += k
            cur = self.residual_quantity()
            if not np.isfinite(cur):
                return steps, float("nan")
            res = rel_change(cur, prev)
            prev = cur
            if res < tol:
                break
        return steps, res

    def objective(self) -> float:
        J = lib().orc_objective(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                _p(self.f), _p(self.g))
        if self.g is not None and self.P.w_qgen != 0.0:
            J += lib().orc_objective_qgen(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                          _p(self.gamma), _p(self.g))
        return J

    # ---- thermal forward ------------------------------------------------
    def thermal_run(self, nsteps: int):
        if nsteps > 0:
            lib().orc_thermal_run(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                  _p(self.gamma), _p(self.bcval), _p(self.f), _p(self.g),
                                  int(nsteps))

    def temperature(self, g=None) -> np.ndarray:
        g = self.g if g is None else np.ascontiguousarray(g)
        T = np.zeros(self.N)
        lib().orc_thermal_macro(ctypes.byref(self.P), _p(g), _p(T))
        return T

    def thermal_solve(self, tol: float, max_steps: int, check_every: int = 1000):
        prev = float(self.temperature()[self.nonwall].mean())
        steps, res = 0, float("inf")
        while steps < max_steps:
            k = min(check_every, max_steps - steps)
            self.thermal_run(k)
            steps += k
            cur = float(self.temperature()[self.nonwall].mean())
            if not np.isfinite(cur):
                return steps, float("nan")
            res = rel_change(cur, prev)
            prev = cur
            if res < tol:
                break
        return steps, res

    # ---- adjoint ----------------------------------------------------------
    def adjoint_post_bc(self, fsc=None) -> np.ndarray:
        """f* = B^T f*_C (the quantity the CUDA path stores)."""
        fsc = self.fsc if fsc is None else np.ascontiguousarray(fsc)
        out = np.zeros_like(fsc)
        lib().orc_adjoint_bc(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8), _p(fsc),
                             _p(out))
        return out

    def adjoint_run(self, nsteps: int):
        if nsteps > 0:
            lib().orc_flow_adjoint_run(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                       _p(self.gamma), _p(self.f), _p(self.fsc),
                                       _p(self.coupling), int(nsteps))

    def adjoint_step_of(self, fsc, with_source=True, coupling=None) -> np.ndarray:
        out = np.zeros_like(fsc)
        lib().orc_flow_adjoint_step(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                    _p(self.gamma), _p(self.f), _p(np.ascontiguousarray(fsc)),
                                    _p(coupling), int(with_source), _p(out))
        return out

    def tangent_of(self, dw: np.ndarray) -> np.ndarray:
        out = np.zeros_like(dw)
        lib().orc_flow_tangent(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                               _p(self.gamma), _p(self.f), _p(np.ascontiguousarray(dw)),
                               _p(out))
        return out

    def adjoint_quantity(self) -> float:
        fs = self.adjoint_post_bc().reshape(self.N, self.Q)
        return float(np.abs(fs[self.nonwall]).sum(axis=1).mean())

    def adjoint_solve(self, tol: float, max_steps: int, check_every: int = 1000):
        prev = self.adjoint_quantity()
        steps, res = 0, float("inf")
        while steps < max_steps:
            k = min(check_every, max_steps - steps)
            self.adjoint_run(k)
            steps += k
            cur = self.adjoint_quantity()
            if not np.isfinite(cur):
                return steps, float("nan")
            res = rel_change(cur, prev)
            prev = cur
            if res < tol:
                break
        return steps, res

    def sensitivity(self) -> np.ndarray:
        s = np.zeros(self.N)
        lib().orc_flow_sensitivity(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                   _p(self.gamma), _p(self.f), _p(self.fsc), _p(s))
        if self.sensT is not None:
            s = s + self.sensT
        return s

    # ---- thermal adjoint ------------------------------------------------
    def thermal_adjoint_run(self, nsteps: int):
        if nsteps > 0:
            lib().orc_thermal_adjoint_run(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                          _p(self.gamma), _p(self.f), _p(self.g),
                                          _p(self.gsc), int(nsteps))

    def thermal_adjoint_step_of(self, gsc, with_source=True):
        out = np.zeros_like(gsc)
        lib().orc_thermal_adjoint_step(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                       _p(self.gamma), _p(self.f), _p(self.g),
                                       _p(np.ascontiguousarray(gsc)), int(with_source),
                                       _p(out))
        return out

    def thermal_tangent_of(self, dg, df):
        out = np.zeros(self.N * 7)
        lib().orc_thermal_tangent(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                  _p(self.gamma), _p(self.f), _p(self.g),
                                  _p(np.ascontiguousarray(dg)), _p(np.ascontiguousarray(df)),
                                  _p(out))
        return out

    def thermal_coupling_of(self, gsc):
        cpl = np.zeros(self.N * self.Q)
        sT = np.zeros(self.N)
        lib().orc_thermal_coupling(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                   _p(self.gamma), _p(self.f), _p(self.g),
                                   _p(np.ascontiguousarray(gsc)), _p(cpl), _p(sT))
        return cpl, sT

    def thermal_adjoint_post_bc(self, gsc=None) -> np.ndarray:
        """g* = B_g^T g*_C (the quantity the CUDA path stores)."""
        gsc = self.gsc if gsc is None else np.ascontiguousarray(gsc)
        out = np.zeros_like(gsc)
        lib().orc_thermal_adjoint_bc(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                     _p(self.gamma), _p(self.f), _p(self.g), _p(gsc), _p(out))
        return out

    def thermal_adjoint_quantity(self) -> float:
        g = self.thermal_adjoint_post_bc().reshape(self.N, 7)
        return float(np.abs(g[self.nonwall]).sum(axis=1).mean())

    def thermal_adjoint_solve(self, tol: float, max_steps: int, check_every: int = 1000):
        prev = self.thermal_adjoint_quantity()
        steps, res = 0, float("inf")
        while steps < max_steps:
            k = min(check_every, max_steps - steps)
            self.thermal_adjoint_run(k)
            steps += k
            cur = self.thermal_adjoint_quantity()
            if not np.isfinite(cur):
                return steps, float("nan")
            res = rel_change(cur, prev)
            prev = cur
            if res < tol:
                break
        return steps, res

    def finish_thermal_adjoint(self):
        """Coupling term and thermal sensitivity from the converged g*_C."""
        self.coupling, self.sensT = self.thermal_coupling_of(self.gsc)

    # ---- continuous adjoint (the comparison of Sec. 2.3) ----------------
    def cont_adjoint_solve(self, tol: float, max_steps: int, check_every: int = 1000):
        """Iterate the continuous adjoint (Eq. 27, 29, 30) from f* = 0 to the
        residual rule on mean sum |f*|; D2Q9 lattices only."""
        fs = np.zeros(self.N * self.Q)
        tmp = np.zeros_like(fs)
        nw = self.nonwall

        def quantity(x):
            return float(np.abs(x.reshape(self.N, self.Q)[nw]).sum(axis=1).mean())
        prev, steps, res = quantity(fs), 0, float("inf")
        while steps < max_steps:
            for _ in range(min(check_every, max_steps - steps)):
                rc = lib().orc_cont_adjoint_step(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                                 _p(self.gamma), _p(self.f), _p(fs), _p(tmp))
                if rc != 0:
                    raise ValueError("the continuous adjoint is written for D2Q9 only (the 3D "
                                     "boundary forms are not printed in the paper)")
                fs, tmp = tmp, fs
                steps += 1
            cur = quantity(fs)
            if not np.isfinite(cur):
                return steps, float("nan"), fs
            res = rel_change(cur, prev)
            prev = cur
            if res < tol:
                break
        self.fs_cont = fs
        return steps, res, fs

    def cont_sensitivity(self) -> np.ndarray:
        s = np.zeros(self.N)
        lib().orc_cont_sensitivity(ctypes.byref(self.P), _p(self.flags, ctypes.c_uint8),
                                   _p(self.gamma), _p(self.f), _p(self.fs_cont), _p(s))
        return s

    # ---- whole pipeline -------------------------------------------------
    def solve_all(self, tol=1e-10, max_steps=200000, check_every=500, adj_tol=None):
        adj_tol = tol if adj_tol is None else adj_tol
        rep = {}
        rep["flow"] = self.flow_solve(tol, max_steps, check_every)
        if self.g is not None:
            rep["thermal"] = self.thermal_solve(tol, max_steps, check_every)
            rep["thermal_adjoint"] = self.thermal_adjoint_solve(adj_tol, max_steps, check_every)
            self.finish_thermal_adjoint()
        rep["adjoint"] = self.adjoint_solve(adj_tol, max_steps, check_every)
        rep["J"] = self.objective()
        rep["sens"] = self.sensitivity()
        return rep
