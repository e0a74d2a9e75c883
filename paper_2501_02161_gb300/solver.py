"""Python face of the CUDA solver: one context per lattice, torch tensors in
and out, the C-ABI underneath (paper_2501_02161_gb300._capi)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _capi as C

STORAGES = {"fp64": C.LBM_FP64, "fp32": C.LBM_FP32, "fp16": C.LBM_FP16_OFS,
            "bf16": C.LBM_BF16_OFS}


@dataclass
class Report:
    steps: int
    residual: float
    I: float
    J: float
    ms: float
    status: int

    @property
    def converged(self) -> bool:
        return self.status == C.LBM_OK


def _ptr(x):
    """(pointer, on_device, dtype code, owner) for a torch tensor or an array-like;
    keep `owner` alive until the call that uses the pointer returns."""
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if x.dtype not in (torch.float64, torch.float32):
            raise ValueError("tensor must be float64 or float32")
        dt = C.LBM_DTYPE_F64 if x.dtype == torch.float64 else C.LBM_DTYPE_F32
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), dt, x
    x = np.asarray(x)
    x = np.ascontiguousarray(x, dtype=x.dtype if x.dtype in (np.float32, np.float64) else np.float64)
    dt = C.LBM_DTYPE_F64 if x.dtype == np.float64 else C.LBM_DTYPE_F32
    return ctypes.c_void_p(x.ctypes.data), 0, dt, x


class Solver:
    """Forward / adjoint / dJ/dgamma on one lattice, resident on one GPU."""

    def __init__(self, stencil: int, nx: int, ny: int, nz: int, storage: str = "fp32",
                 thermal: bool = False, device=None):
        self.lib = C.lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stencil, self.nx, self.ny, self.nz = stencil, nx, ny, nz
        self.N = nx * ny * nz
        self.Q = 9 if stencil == C.LBM_D2Q9 else 19
        self.storage = storage
        self.thermal = thermal
        self.rdtype = torch.float64 if storage == "fp64" else torch.float32
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            C.check(self.lib.lbm_create(ctypes.byref(self._ctx), stencil, nx, ny, nz,
                                        STORAGES[storage], int(thermal)), "lbm_create")
        self._keep = []

    @classmethod
    def from_lattice(cls, lat, storage: str = "fp32", device=None) -> "Solver":
        s = cls(lat.stencil, lat.nx, lat.ny, lat.nz, storage, lat.thermal, device)
        s.set_flags(torch.as_tensor(lat.flags, dtype=torch.uint8, device=s.device))
        s.set_gamma(torch.as_tensor(lat.gamma, dtype=s.rdtype, device=s.device))
        s.set_bc_values(torch.as_tensor(lat.bcval, dtype=s.rdtype, device=s.device))
        s.set_lattice_params(lat)
        if getattr(lat, "mirror", 0):
            s.set_symmetry(lat.mirror)
        return s

    def set_adjoint_scheme(self, scheme: str):
        """'discrete' (the paper's method, default) or 'continuous' (the
        comparison of Sec. 2.3; D2Q9 flow lattices)."""
        code = {"discrete": C.LBM_ADJOINT_DISCRETE, "continuous": C.LBM_ADJOINT_CONTINUOUS}[scheme]
        C.check(self.lib.lbm_set_adjoint_scheme(self._ctx, code), "lbm_set_adjoint_scheme")

    def set_symmetry(self, axes: int):
        """Symmetry planes beyond both faces of the axes in the mask (bit 0 x,
        1 y, 2 z) instead of periodic seams."""
        C.check(self.lib.lbm_set_symmetry(self._ctx, int(axes)), "lbm_set_symmetry")

    def set_lattice_params(self, lat):
        """The lattice's physical parameters and objective weights: through
        lbm_set_physics when it is specified by Re (and Pr), else through
        lbm_set_params with its tau (and kappa_f)."""
        if lat.re is not None:
            self.set_physics(re=lat.re, u_ref=lat.u_ref, l_ref=lat.l_ref, dp=lat.dp,
                             pr=lat.pr or 0.0, rho0=lat.rho0, gamma_model=lat.gamma_model,
                             k_ratio=lat.k_ratio, q_flux=lat.q_flux, T0=lat.T0,
                             beta_max=lat.beta_max)
        else:
            self.set_params(tau=lat.tau, rho0=lat.rho0, gamma_model=lat.gamma_model,
                            kappa_f=lat.kappa_f or 0.0, k_ratio=lat.k_ratio, q_flux=lat.q_flux,
                            T0=lat.T0, beta_max=lat.beta_max)
        self.set_objective(lat.w_pin, lat.w_tmean, lat.w_qgen)

    def close(self):
        if self._ctx:
            self.lib.lbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up -------------------------------------------------------------
    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        C.check(self.lib.lbm_set_stream(self._ctx, ctypes.c_void_p(s)), "lbm_set_stream")

    def set_flags(self, flags):
        if isinstance(flags, torch.Tensor):
            assert flags.dtype == torch.uint8
            p, dev = ctypes.c_void_p(flags.data_ptr()), int(flags.is_cuda)
        else:
            flags = np.ascontiguousarray(flags, dtype=np.uint8)
            p, dev = ctypes.c_void_p(flags.ctypes.data), 0
        self._stream()
        C.check(self.lib.lbm_set_flags(self._ctx, p, self.N, dev), "lbm_set_flags")

    def set_gamma(self, gamma):
        p, dev, dt, _keep = _ptr(gamma)
        self._stream()
        C.check(self.lib.lbm_set_gamma(self._ctx, p, self.N, dt, dev), "lbm_set_gamma")

    def set_bc_values(self, values):
        p, dev, dt, _keep = _ptr(values)
        self._stream()
        C.check(self.lib.lbm_set_bc_values(self._ctx, p, 4 * self.N, dt, dev), "lbm_set_bc_values")

    def set_params(self, tau, rho0=1.0, gamma_model=0, kappa_f=0.0, k_ratio=1.0, q_flux=0.0, T0=0.0,
                   beta_max=0.0):
        prm = C.lbm_params(tau, rho0, gamma_model, kappa_f, k_ratio, q_flux, T0, beta_max)
        C.check(self.lib.lbm_set_params(self._ctx, ctypes.byref(prm)), "lbm_set_params")

    def set_physics(self, re, u_ref=0.0, l_ref=1.0, dp=0.0, pr=0.0, rho0=1.0, gamma_model=0,
                    k_ratio=1.0, q_flux=0.0, T0=0.0, beta_max=0.0):
        """Parameters from Re = U L / nu and Pr = nu / kappa_f (Eq. 3; Eq. 70 when
        the velocity scale is given by a pressure drop dp)."""
        ph = C.lbm_physics(re, u_ref, l_ref, dp, pr, rho0, gamma_model, k_ratio, q_flux, T0,
                           beta_max)
        C.check(self.lib.lbm_set_physics(self._ctx, ctypes.byref(ph)), "lbm_set_physics")

    def set_objective(self, w_pin=1.0, w_tmean=0.0, w_qgen=0.0):
        o = C.lbm_objective(w_pin, w_tmean, w_qgen)
        C.check(self.lib.lbm_set_objective(self._ctx, ctypes.byref(o)), "lbm_set_objective")

    def set_bc(self, face: int, kind: int, values):
        """Boundary values of the VEL or PRES nodes on one face of the box
        (4 numbers, or 4 per such node in node order)."""
        p, dev, dt, keep = _ptr(values)
        n = keep.numel() if isinstance(keep, torch.Tensor) else keep.size
        self._stream()
        C.check(self.lib.lbm_set_bc(self._ctx, int(face), int(kind), p, int(n), dt, dev), "lbm_set_bc")

    # ---- solves -------------------------------------------------------------
    def _solve(self, fn, name, tol, max_steps, check_every, reset, strict) -> Report:
        o = C.lbm_solve_opts(float(tol), int(max_steps), int(check_every), int(reset))
        r = C.lbm_report()
        r.status = 0
        self._stream()
        code = fn(self._ctx, ctypes.byref(o), ctypes.byref(r))
        if code == C.LBM_ERR_DIVERGED and not strict:
            return Report(r.steps, r.residual, r.I, r.J, r.ms, code)
        C.check(code, name)
        return Report(r.steps, r.residual, r.I, r.J, r.ms, r.status)

    def forward(self, tol=1e-6, max_steps=20000, check_every=1000, reset=True,
                strict=True) -> Report:
        """Forward solve; strict=False returns a LBM_ERR_DIVERGED report instead of raising."""
        return self._solve(self.lib.lbm_forward, "lbm_forward", tol, max_steps, check_every,
                           reset, strict)

    def adjoint(self, tol=1e-6, max_steps=20000, check_every=1000, reset=True,
                strict=True) -> Report:
        return self._solve(self.lib.lbm_adjoint, "lbm_adjoint", tol, max_steps, check_every,
                           reset, strict)

    def solve_phase(self, phase: int, tol=1e-6, max_steps=20000, check_every=1000, reset=True,
                    strict=True) -> Report:
        """One phase of the solve sequence (0 flow, 1 temperature, 2 flow adjoint,
        3 temperature adjoint; see lbm_solve_phase)."""
        fn = lambda ctx, o, r: self.lib.lbm_solve_phase(ctx, int(phase), o, r)
        return self._solve(fn, "lbm_solve_phase", tol, max_steps, check_every, reset, strict)

    def sensitivity(self, out: torch.Tensor | None = None, dtype=None) -> torch.Tensor:
        dtype = dtype or self.rdtype
        if out is None:
            out = torch.empty(self.N, dtype=dtype, device=self.device)
        p, dev, dt, _keep = _ptr(out)
        self._stream()
        C.check(self.lib.lbm_sensitivity(self._ctx, p, dt, dev), "lbm_sensitivity")
        return out

    def fields(self, dtype=None):
        """(rho[N], u[3, N], T[N] or None) of the converged forward state."""
        dtype = dtype or self.rdtype
        rho = torch.empty(self.N, dtype=dtype, device=self.device)
        u = torch.empty(3, self.N, dtype=dtype, device=self.device)
        T = torch.empty(self.N, dtype=dtype, device=self.device) if self.thermal else None
        dt = C.LBM_DTYPE_F64 if dtype == torch.float64 else C.LBM_DTYPE_F32
        self._stream()
        C.check(self.lib.lbm_get_fields(self._ctx, ctypes.c_void_p(rho.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(T.data_ptr()) if T is not None else None,
                                        dt, 1), "lbm_get_fields")
        return rho, u, T

    def objective(self) -> float:
        J = ctypes.c_double()
        C.check(self.lib.lbm_get_objective(self._ctx, ctypes.byref(J)), "lbm_get_objective")
        return J.value

    def adjoint_fields(self, dtype=None):
        """(f*[Q, N], g*[7, N] or None): the stored adjoint iterate f* = B^T f*_C."""
        dtype = dtype or self.rdtype
        fs = torch.empty(self.Q, self.N, dtype=dtype, device=self.device)
        gs = torch.empty(7, self.N, dtype=dtype, device=self.device) if self.thermal else None
        dt = C.LBM_DTYPE_F64 if dtype == torch.float64 else C.LBM_DTYPE_F32
        self._stream()
        C.check(self.lib.lbm_get_adjoint(self._ctx, ctypes.c_void_p(fs.data_ptr()),
                                         ctypes.c_void_p(gs.data_ptr()) if gs is not None else None,
                                         dt, 1), "lbm_get_adjoint")
        return fs, gs

    # ---- checkpoint / resume ------------------------------------------------
    def state_bytes(self) -> int:
        return int(self.lib.lbm_state_bytes(self._ctx))

    def export_state(self, out: torch.Tensor | None = None, pin: bool = True) -> torch.Tensor:
        """The solver state as a uint8 tensor (host memory, pinned by default,
        unless `out` is given: any device, at least state_bytes() long)."""
        nb = self.state_bytes()
        if out is None:
            out = torch.empty(nb, dtype=torch.uint8, pin_memory=pin)
        assert out.dtype == torch.uint8 and out.is_contiguous() and out.numel() >= nb
        self._stream()
        C.check(self.lib.lbm_export_state(self._ctx, ctypes.c_void_p(out.data_ptr()), nb),
                "lbm_export_state")
        return out

    def import_state(self, state: torch.Tensor):
        """Continue from a state written by export_state (same lattice, flags and
        parameters set; gamma may differ)."""
        assert state.dtype == torch.uint8 and state.is_contiguous()
        self._stream()
        C.check(self.lib.lbm_import_state(self._ctx, ctypes.c_void_p(state.data_ptr()),
                                          state.numel()), "lbm_import_state")

    def time_steps(self, phase: int, n: int) -> float:
        """Mean ms per plain fused step of a phase (0 flow, 1 temperature,
        2 flow adjoint, 3 temperature adjoint), CUDA events on its stream."""
        ms = ctypes.c_double()
        self._stream()
        C.check(self.lib.lbm_time_steps(self._ctx, int(phase), int(n), ctypes.byref(ms)),
                "lbm_time_steps")
        return ms.value
