"""Brute-force periodic Ewald sum of the force of one point mass, FP64.

Test infrastructure only (see the package docstring).

Used to pin the PM force (the paper's solver, §1/§2.3) against the exact
periodic Newtonian force.  A plain sum over periodic images converges only
conditionally, so the sum is split as in Hernquist, Bouchet & Suto (1991):
for a unit source with a uniform neutralising background,
psi(r) = sum_n erfc(alpha d_n)/d_n + (4 pi / L^3) sum_{k != 0} e^{-k^2 / 4 alpha^2} cos(k.r) / k^2,
with d_n = |r + n L|, and grad psi ~ -r_hat / r^2 at small r.

In the PM units (nabla^2 phi = 1.5 Omega_m0 delta with delta = rho / rho_bar - 1
and a particle of mass m in units of the mean mass per cell of side H),
the force on a test particle at separation vector r from the source is
F = 1.5 Omega_m0 m H^3 / (4 pi) grad psi(r).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def grad_psi(r, box, alpha=None, nreal=2, nk=8):
    """grad psi at separation vectors r, shape (n, 3) (Mpc/h), FP64."""
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    if alpha is None:
        alpha = 2.5 / box
    out = np.zeros_like(r)
    rng = range(-nreal, nreal + 1)
    for nx in rng:
        for ny in rng:
            for nz in rng:
                d = r + box * np.array([nx, ny, nz], dtype=np.float64)
                dn = np.sqrt((d ** 2).sum(axis=1))
                term = erfc(alpha * dn) / dn ** 2 + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * dn) ** 2) / dn
                out -= d / dn[:, None] * term[:, None]
    kf = 2.0 * math.pi / box
    m = np.arange(-nk, nk + 1)
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    kv = kf * np.stack([MX.ravel(), MY.ravel(), MZ.ravel()], axis=1).astype(np.float64)
    kv = kv[(kv ** 2).sum(axis=1) > 0]                       # k = 0 excluded
    k2 = (kv ** 2).sum(axis=1)
    coef = 4.0 * math.pi / box ** 3 * np.exp(-k2 / (4.0 * alpha ** 2)) / k2
    for lo in range(0, len(r), 2048):                         # chunked sum over k vectors
        s = np.sin(r[lo:lo + 2048] @ kv.T) * coef[None, :]
        out[lo:lo + 2048] -= s @ kv
    return out


def point_mass_force(r, box, mass, cell, omega_m0):
    """Force on test particles at separations r from a source of mass m (PM units)."""
    return 1.5 * omega_m0 * mass * cell ** 3 / (4.0 * math.pi) * grad_psi(r, box)
