"""FP64 reference of the level-set design update (Eq. 13-15, 66-67).

Test infrastructure only: the tests import it; the product path never does.
Plain Python loops over nodes, written from the equations, sharing no code
with the package.  Same readings as the package: G = mean(alpha) - V_max over
the design nodes, one explicit unit step of Eq. 14 then phi clipped to
[-1, 1], the Laplacian with mirrored values beyond the edges, sigma one
weight per axis, non-design nodes unchanged.  Arrays are nested (z, y, x)
(or (y, x) in 2D) numpy arrays; loops make it slow, so keep lattices small.
"""
import math

import numpy as np


def _at(phi, idx):
    """phi at an index tuple, mirrored (clamped) to the nearest edge node."""
    clamped = tuple(min(max(i, 0), n - 1) for i, n in zip(idx, phi.shape))
    return phi[clamped]


def sigma_laplacian(phi, sigma):
    """sum over axes a of sigma_a (phi(x+e_a) - 2 phi(x) + phi(x-e_a))."""
    phi = np.asarray(phi, dtype=np.float64)
    nd = phi.ndim
    w = [float(sigma)] * nd if np.isscalar(sigma) else [float(s) for s in sigma]
    out = np.zeros_like(phi)
    for idx in np.ndindex(*phi.shape):
        total = 0.0
        for axis_xyz in range(nd):
            d = nd - 1 - axis_xyz  # array dimension of lattice axis x, y, z
            if phi.shape[d] == 1:
                continue
            plus = list(idx)
            minus = list(idx)
            plus[d] += 1
            minus[d] -= 1
            total += w[axis_xyz] * (_at(phi, plus) - 2.0 * phi[idx] + _at(phi, minus))
        out[idx] = total
    return out


def alpha_of(phi):
    """Eq. 15."""
    phi = np.asarray(phi, dtype=np.float64)
    out = np.zeros_like(phi)
    for idx in np.ndindex(*phi.shape):
        out[idx] = 0.0 if phi[idx] < 0.0 else 1.0
    return out


def step(phi, jw, K, sigma, vmax, mask=None):
    """One update; returns (phi_new, alpha_new, lambda, G)."""
    phi = np.asarray(phi, dtype=np.float64)
    jw = np.asarray(jw, dtype=np.float64)
    mask = np.ones(phi.shape, bool) if mask is None else np.asarray(mask, bool)
    alpha = alpha_of(phi)
    n_design = 0
    fluid = 0.0
    for idx in np.ndindex(*phi.shape):
        if mask[idx]:
            n_design += 1
            fluid += alpha[idx]
    G = fluid / n_design - vmax
    lap = sigma_laplacian(phi, sigma)
    s = 0.0
    for idx in np.ndindex(*phi.shape):
        if mask[idx]:
            s += abs(jw[idx] - lap[idx])
    lam = math.exp(G) * s / n_design                      # Eq. 67
    new = phi.copy()
    for idx in np.ndindex(*phi.shape):
        if mask[idx]:
            jprime = jw[idx] + lam                         # Eq. 66
            v = phi[idx] - K * (jprime - lap[idx])         # Eq. 14, unit step
            new[idx] = min(1.0, max(-1.0, v))              # Eq. 13 range
    return new, alpha_of(new), lam, G
