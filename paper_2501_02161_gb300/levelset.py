"""Level-set design update of the paper's optimiser (Sec. 2.2, Eq. 13-15;
Sec. 2.4, Eq. 66-67).

The design variable alpha (the solver's gamma) is the 0/1 image of a level-set
function phi in [-1, 1] (Eq. 13, 15).  Each optimisation iteration moves phi
along the reaction-diffusion equation dphi/dxi = -K (J' - sigma lap(phi))
(Eq. 14), with J' = J_W' + lambda (Eq. 66): J_W' is the sensitivity dJ/dgamma
the CUDA solver returns, lambda the volume multiplier of Eq. 67.

Readings where the paper is silent (they are the oracle's too):
- G in exp(G) is the volume-fraction excess mean(alpha) - V_max: Eq. 34 writes
  G as a node count, whose exponential overflows for any lattice of interest,
  and the fraction keeps its sign and zero;
- one explicit Euler step of unit fictitious time per iteration (K absorbs the
  step), then phi is clipped to [-1, 1] (the range Eq. 13 allows);
- lap(phi) is the 5-point (2D) / 7-point (3D) Laplacian with zero-gradient
  (mirror) values beyond the lattice edges; an anisotropic sigma =
  diag(s_x, s_y, s_z) (Sec. 3.3.4) weights each axis' second difference;
- nodes outside the design mask (walls, openings) keep phi and alpha.
All of this is plain tensor code on the design side; it runs on the device
the tensors live on.  Arrays are (nz, ny, nx) or (ny, nx).
"""
from __future__ import annotations

import math

import torch


def _second_difference(phi: torch.Tensor, dim: int) -> torch.Tensor:
    """phi(i+1) - 2 phi(i) + phi(i-1) along `dim`, mirrored at both ends."""
    n = phi.shape[dim]
    if n == 1:
        return torch.zeros_like(phi)
    up = torch.cat([phi.narrow(dim, 1, n - 1), phi.narrow(dim, n - 1, 1)], dim)
    down = torch.cat([phi.narrow(dim, 0, 1), phi.narrow(dim, 0, n - 1)], dim)
    return up - 2 * phi + down


def laplacian(phi: torch.Tensor, sigma=1.0) -> torch.Tensor:
    """sigma-weighted Laplacian: sum over axes of s_axis * second difference.
    sigma is a number (isotropic) or one weight per axis in x, y(, z) order."""
    nd = phi.dim()
    weights = [float(sigma)] * nd if isinstance(sigma, (int, float)) else [float(s) for s in sigma]
    if len(weights) != nd:
        raise ValueError("sigma needs one weight per lattice axis")
    out = torch.zeros_like(phi)
    for axis_xyz, w in enumerate(weights):
        if w != 0.0:
            out = out + w * _second_difference(phi, nd - 1 - axis_xyz)
    return out


def alpha_from_phi(phi: torch.Tensor) -> torch.Tensor:
    """Eq. 15: solid (0) where phi < 0, fluid (1) where phi >= 0."""
    return (phi >= 0).to(phi.dtype)


def volume_excess(alpha: torch.Tensor, vmax: float, mask: torch.Tensor | None = None) -> float:
    """G of Eq. 34 as a fraction: mean(alpha) - V_max over the design nodes."""
    a = alpha[mask] if mask is not None else alpha
    return float(a.mean()) - vmax


def lagrange_multiplier(jw: torch.Tensor, sig_lap: torch.Tensor, G: float,
                        mask: torch.Tensor | None = None) -> float:
    """Eq. 67: lambda = exp(G)/N sum_j |J_W'(x_j) - sigma lap(phi)(x_j)|,
    over the N design nodes."""
    r = (jw - sig_lap).abs()
    r = r[mask] if mask is not None else r
    return math.exp(G) * float(r.sum()) / r.numel()


def level_set_step(phi: torch.Tensor, jw: torch.Tensor, K: float, sigma, vmax: float,
                   mask: torch.Tensor | None = None):
    """One optimisation update.  phi: level set; jw: J_W' = dJ/dgamma from the
    solver (same shape); K: step size; sigma: regularisation (number or per
    axis); vmax: fluid volume fraction bound; mask: design nodes (None: all).
    Returns (phi, alpha, lambda, G) after the update."""
    alpha = alpha_from_phi(phi)
    G = volume_excess(alpha, vmax, mask)
    sl = laplacian(phi, sigma)
    lam = lagrange_multiplier(jw, sl, G, mask)
    rate = -K * ((jw + lam) - sl)          # Eq. 14 with J' = J_W' + lambda (Eq. 66)
    new = (phi + rate).clamp(-1.0, 1.0)
    if mask is not None:
        new = torch.where(mask, new, phi)
    return new, alpha_from_phi(new), lam, G


def level_set_loop(solver, lat, iters: int = 50, K: float = 0.1, sigma=5e-3, vmax: float = 0.5,
                   phi0: torch.Tensor | None = None, tol: float = 1e-4, max_steps: int = 100000,
                   check_every: int = 500, normalise: bool = True):
    """Drive the optimisation: gamma = alpha(phi), forward + adjoint solve and
    dJ/dgamma on the GPU solver (warm-started after the first iteration), then
    one level-set step.  normalise scales J_W' by its largest magnitude so that
    K is a fraction of the phi range per iteration.  Returns (phi, history)."""
    dev = solver.device
    shape = (lat.nz, lat.ny, lat.nx) if lat.nz > 1 else (lat.ny, lat.nx)
    kind = torch.as_tensor(lat.flags & 7, device=dev).reshape(shape)
    mask = kind == 0
    fixed = torch.as_tensor(lat.gamma, dtype=torch.float64, device=dev).reshape(shape)
    phi = (phi0.clone() if phi0 is not None else torch.ones(shape, dtype=torch.float64, device=dev))
    hist = []
    for it in range(iters):
        gamma = torch.where(mask, alpha_from_phi(phi), fixed)
        solver.set_gamma(gamma.reshape(-1).to(solver.rdtype))
        rf = solver.forward(tol=tol, max_steps=max_steps, check_every=check_every, reset=it == 0)
        solver.adjoint(tol=tol, max_steps=max_steps, check_every=check_every, reset=it == 0)
        jw = solver.sensitivity(dtype=torch.float64).reshape(shape)
        if normalise:
            jw = jw / jw[mask].abs().max().clamp_min(1e-300)
        phi, alpha, lam, G = level_set_step(phi, jw, K, sigma, vmax, mask)
        hist.append({"iter": it, "J": rf.J, "lambda": lam, "G": G,
                     "fluid_fraction": float(alpha[mask].mean())})
    return phi, hist
