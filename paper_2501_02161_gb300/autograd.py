"""Differentiation through the solver: the discrete adjoint as a backward.

`lbm_objective(gamma, solver)` returns the steady objective J(gamma) as a
0-dim tensor; its backward runs the adjoint solve (Eq. 53-56 to a fixed point)
and the sensitivity (Eq. 66), so d/dgamma of anything built on J is the exact
gradient of the discrete steady problem.  Everything here is argument
marshalling around the CUDA library; the optimiser helpers (density filter,
Heaviside projection, projected gradient) are plain tensor code on the design
side, off the solver path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch
import torch.nn.functional as F

from .solver import Solver


@dataclass
class SolveOpts:
    tol: float = 1e-6
    max_steps: int = 200000
    check_every: int = 1000
    warm: bool = False   # continue from the previous forward / adjoint state


class _LBMObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, solver: Solver, opts: SolveOpts):
        g = gamma.detach().to(solver.rdtype).contiguous()
        solver.set_gamma(g)
        rep = solver.forward(tol=opts.tol, max_steps=opts.max_steps,
                             check_every=opts.check_every, reset=not opts.warm)
        solver._token = getattr(solver, "_token", 0) + 1
        ctx.solver, ctx.opts, ctx.token = solver, opts, solver._token
        ctx.save_for_backward(gamma)
        ctx.report = rep
        return torch.tensor(rep.J, dtype=gamma.dtype, device=gamma.device)

    @staticmethod
    def backward(ctx, gJ):
        (gamma,) = ctx.saved_tensors
        s, o = ctx.solver, ctx.opts
        if getattr(s, "_token", None) != ctx.token:
            # the solver was used for another design since: redo this forward
            s.set_gamma(gamma.detach().to(s.rdtype).contiguous())
            s.forward(tol=o.tol, max_steps=o.max_steps, check_every=o.check_every, reset=True)
            s._token = ctx.token = s._token + 1
        s.adjoint(tol=o.tol, max_steps=o.max_steps, check_every=o.check_every,
                  reset=not o.warm)
        sens = s.sensitivity(dtype=gamma.dtype)
        return gJ * sens, None, None


def lbm_objective(gamma: torch.Tensor, solver: Solver, opts: SolveOpts | None = None):
    """J(gamma) of the solver's lattice; differentiable in gamma (flat, N values)."""
    return _LBMObjective.apply(gamma, solver, opts or SolveOpts())


# ---------------------------------------------------------------------------
# design parametrisation: density filter + Heaviside projection
# ---------------------------------------------------------------------------

def cone_kernel(radius: float, dims: int = 3, dtype=torch.float32, device=None) -> torch.Tensor:
    r = int(math.floor(radius))
    ax = torch.arange(-r, r + 1, dtype=dtype, device=device)
    if dims == 3:
        zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
        d = torch.sqrt(xx * xx + yy * yy + zz * zz)
    else:
        yy, xx = torch.meshgrid(ax, ax, indexing="ij")
        d = torch.sqrt(xx * xx + yy * yy)
    return torch.clamp(radius - d, min=0.0)


def density_filter(x: torch.Tensor, radius: float = 2.0) -> torch.Tensor:
    """Linear-cone density filter, normalised by the covered weight (so a
    constant field is unchanged up to the edges).  x has shape (nz, ny, nx)."""
    k = cone_kernel(radius, 3, x.dtype, x.device)[None, None]
    pad = k.shape[-1] // 2
    num = F.conv3d(x[None, None], k, padding=pad)
    den = F.conv3d(torch.ones_like(x)[None, None], k, padding=pad)
    return (num / den)[0, 0]


def heaviside_projection(x: torch.Tensor, beta: float = 8.0, eta: float = 0.5) -> torch.Tensor:
    """Smoothed Heaviside (tanh) projection onto [0, 1]."""
    a = math.tanh(beta * eta)
    return (a + torch.tanh(beta * (x - eta))) / (a + math.tanh(beta * (1.0 - eta)))


def design_to_gamma(rho: torch.Tensor, design_mask: torch.Tensor, fixed_gamma: torch.Tensor,
                    radius: float = 2.0, beta: float = 8.0, eta: float = 0.5) -> torch.Tensor:
    """gamma = projection(filter(rho)) on design nodes, fixed values elsewhere."""
    g = heaviside_projection(density_filter(rho, radius), beta, eta)
    return torch.where(design_mask, g, fixed_gamma)


def projected_gradient_loop(solver: Solver, lat, iters: int = 50, step: float = 0.05,
                            radius: float = 2.0, beta: float = 8.0, eta: float = 0.5,
                            volume: float | None = None, vol_weight: float = 10.0,
                            opts: SolveOpts | None = None, rho0: torch.Tensor | None = None):
    """Minimise J(gamma(rho)) (+ an optional volume-fraction penalty) over the
    design density rho in [0, 1] with projected gradient steps whose size is
    normalised by the largest gradient entry.  Returns (rho, history)."""
    opts = opts or SolveOpts(tol=1e-4, max_steps=100000, check_every=500, warm=True)
    dev = solver.device
    shape = (lat.nz, lat.ny, lat.nx)
    fixed = torch.as_tensor(lat.gamma, dtype=torch.float32, device=dev).reshape(shape)
    kind = torch.as_tensor(lat.flags & 7, device=dev).reshape(shape)
    mask = kind == 0  # fluid / design nodes; walls and openings keep their gamma
    rho = (rho0.clone() if rho0 is not None else fixed.clone()).clamp(0, 1)
    hist = []
    first = True
    for it in range(iters):
        x = rho.clone().requires_grad_(True)
        gam = design_to_gamma(x, mask, fixed, radius, beta, eta)
        o = SolveOpts(opts.tol, opts.max_steps, opts.check_every, warm=opts.warm and not first)
        J = lbm_objective(gam.reshape(-1), solver, o)
        loss = J
        if volume is not None:
            vf = gam[mask].mean()
            loss = loss + vol_weight * (vf - volume) ** 2
        loss.backward()
        g = x.grad
        gmax = g[mask].abs().max().clamp_min(1e-30)
        with torch.no_grad():
            rho = torch.where(mask, (rho - step * g / gmax).clamp(0.0, 1.0), rho)
        hist.append({"iter": it, "J": float(J.item()), "loss": float(loss.item())})
        first = False
    return rho, hist
