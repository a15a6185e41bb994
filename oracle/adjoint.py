"""FP64 adjoint (vector-Jacobian products) of the particle-mesh evolution.

Test infrastructure only (see the package docstring).

The paper has no adjoint; the reconstruction workload needs gradients of a final-field
loss with respect to the initial linear modes.  This module writes the chain rule of
the forward oracle out step by step:

* CIC paint rho(c) = sum_i m_i W(x_i - c) with W = prod_d w(x_d - c_d), w the
  1D tent; readout R[M](x) = sum_c W(x - c) M(c).  Their position derivatives use
  dw/dx = -sign(x - c) / H inside the support (piecewise constant; at a cell face
  the one-sided value of the cell the particle is in).
* Force F_j(x_i) = R[G_j rho](x_i) with G_j the linear mesh operator of
  :func:`oracle.pm.force_mesh` o :func:`oracle.pm.potential_k`.  G_j is a real
  convolution with an odd kernel (-i D(k_j) times a real even Green's function,
  D the gradient kernel of :mod:`oracle.pm`), so
  G_j^T = -G_j.  Hence for a cotangent lambda_F:
  dL/dx_i = sum_j lambda_F,ij grad R[G_j rho](x_i)
            + m_i grad R[B](x_i),  B = -sum_j G_j(paint(lambda_F,j)).
* KDK step (p_h = p0 + K1 F(x0), x1 = x0 + Delta p_h, p1 = p_h + K2 F(x1)):
  lambda_x1' = lambda_x1 + F_vjp(x1; K2 lambda_p1), lambda_ph = lambda_p1 +
  Delta lambda_x1', lambda_x0 = lambda_x1' + F_vjp(x0; K1 lambda_ph),
  lambda_p0 = lambda_ph.  Positions are treated as continuous (the fixed-point
  rounding of the drift is a step of 2^-32 L, far below every finite difference).
* Zel'dovich ICs are linear in the white noise omega: s_j = T_j omega with
  T_j = IFFT diag(S_j) FFT, S_j = i k_j amp(k) / k^2 (Hermitian, odd), so
  T_j^T = IFFT diag(conj S_j) FFT = -T_j; neutrino sites add the filter and the
  phase e^{i k.d}, whose transpose is e^{-i k.d}.
"""
from __future__ import annotations

import numpy as np

from . import background as bgm
from . import ic as oic
from . import pm


def _corners(u, n):
    """Yield (flat index, weight, d weight / d x_d for d = 0, 1, 2 in units of 1/H)."""
    cells, fracs = zip(*[pm.cell_and_fraction(u[d], n) for d in range(3)])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                o = (dx, dy, dz)
                idx = [(cells[d] + o[d]) % n for d in range(3)]
                w1 = [fracs[d] if o[d] else 1.0 - fracs[d] for d in range(3)]
                dw1 = [1.0 if o[d] else -1.0 for d in range(3)]
                w = w1[0] * w1[1] * w1[2]
                g = (dw1[0] * w1[1] * w1[2], w1[0] * dw1[1] * w1[2], w1[0] * w1[1] * dw1[2])
                yield (idx[0] * n + idx[1]) * n + idx[2], w, g


def readout_grad(u, mesh, n, box):
    """Gradient with respect to the particle position of the CIC readout of a mesh, (3, np)."""
    h = box / n
    flat = mesh.reshape(-1)
    out = np.zeros((3, u.shape[1]))
    for idx, _, g in _corners(u, n):
        v = flat[idx]
        for d in range(3):
            out[d] += g[d] * v
    return out / h


def paint_vjp_positions(u, mass, lam_mesh, n, box):
    """d/dx_i of sum_c lam(c) paint(x)(c) = m_i grad R[lam](x_i)."""
    return np.asarray(mass)[None, :] * readout_grad(u, lam_mesh, n, box)


def force_vjp(u, mass, lam_f, n, box, omega_m0, kfactor=None):
    """d <lam_f, F(x)> / d x, shape (3, np).  kfactor: a real even multiplier of the
    Green's function (the learned correction); G_j stays odd, so G_j^T = -G_j still."""
    phi = pm.potential_k(pm.paint(u, mass, n), box, omega_m0, kfactor)
    out = np.zeros((3, u.shape[1]))
    for j in range(3):
        out += lam_f[j][None, :] * readout_grad(u, pm.force_mesh(phi, box, n, j), n, box)
    b = np.zeros((n, n, n))
    for j in range(3):
        a_j = pm.paint(u, lam_f[j], n)
        b -= pm.force_mesh(pm.potential_k(a_j, box, omega_m0, kfactor), box, n, j)
    return out + np.asarray(mass)[None, :] * readout_grad(u, b, n, box)


def kdk_step_vjp(u0, p0, f0, coeffs, lam_x1, lam_p1, mass, n, box, omega_m0):
    """VJP of one KDK step: cotangents of (x1, p1) -> cotangents of (x0, p0)."""
    K1, delta, K2 = coeffs
    ph = p0 + K1 * f0
    u1 = pm.drift(u0, ph, delta, box)
    lam_x1t = lam_x1 + force_vjp(u1, mass, K2 * lam_p1, n, box, omega_m0)
    lam_ph = lam_p1 + delta * lam_x1t
    lam_x0 = lam_x1t + force_vjp(u0, mass, K1 * lam_ph, n, box, omega_m0)
    return lam_x0, lam_ph


def ic_vjp(lam_s_cdm, lam_s_nu_sites, box, pk, n_sites=0, k_fs=0.0, nc=None):
    """d L / d omega from displacement cotangents.

    lam_s_cdm: (3, nc^3) cotangent of s at the CDM lattice nodes; lam_s_nu_sites:
    (3, n_sites^3) cotangent of s_nu at the sites (summed over each site's particles).
    """
    nc = nc or round(lam_s_cdm.shape[1] ** (1 / 3))
    KX, KY, KZ, nyq = oic._kgrid(nc, box)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k = np.sqrt(k2)
    amp = np.sqrt(pk(k) / box ** 3) * nc ** 1.5
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    mask = (~nyq) & (k2 > 0)
    grad_k = np.zeros((nc, nc, nc // 2 + 1), dtype=complex)
    for j, kj in enumerate((KX, KY, KZ)):
        S = 1j * kj * amp * inv * mask
        L = np.fft.rfftn(lam_s_cdm[j].reshape(nc, nc, nc))
        grad_k = grad_k + np.conj(S) * L
    if n_sites:
        r, j0, sh = oic.neutrino_site_offset(nc, n_sites)
        filt = 1.0 / (1.0 + k2 / k_fs ** 2) if k_fs > 0 else 1.0
        phase = np.exp(1j * (KX + KY + KZ) * sh * box / nc)
        idx = (j0 + r * np.arange(n_sites)) % nc
        for j, kj in enumerate((KX, KY, KZ)):
            S = 1j * kj * amp * inv * mask * filt * phase
            m = np.zeros((nc, nc, nc))
            m[np.ix_(idx, idx, idx)] = lam_s_nu_sites[j].reshape(n_sites, n_sites, n_sites)
            grad_k = grad_k + np.conj(S) * np.fft.rfftn(m)
    # T^T lam = IFFT(conj S FFT lam) with the normalised inverse of the forward map
    return np.fft.irfftn(grad_k, s=(nc, nc, nc), axes=(0, 1, 2))


class Reconstruction:
    """Forward model omega -> ICs -> KDK steps -> final CIC density, and its loss
    L = mean((rho - rho_target)^2), with the gradient dL/domega by the adjoint."""

    def __init__(self, cfg, steps, a0, k_fs=0.0):
        from . import neutrinos as onu
        self.cfg, self.steps, self.a0, self.k_fs = cfg, steps, a0, k_fs
        self.bg = bgm.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
        self.pk = oic.linear_power(cfg.omega_m, cfg.h, cfg.ns, cfg.sigma8)
        _, self.q, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
        mc, mn = onu.species_masses(cfg.nmesh, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib,
                                    self.bg.omega_c, self.bg.omega_nu_poisson, m_shell)
        self.n_cdm = cfg.nc ** 3
        self.n_nu = cfg.nsites ** 3 * cfg.nshell * (2 * cfg.nfib + 1) if cfg.nsites else 0
        self.mass = onu.particle_masses(self.n_cdm, self.n_nu, cfg.nshell, cfg.nfib, mc, mn)
        self.p_scale = onu.thermal_momentum_scale(self.bg.kT_nu0, max(cfg.m_nu))

    def ics(self, noise):
        bg, c = self.bg, self.cfg
        D0, gp0 = bg.D(self.a0), bg.gp(self.a0)
        uc, pc = oic.cdm_particles(noise, c.box, self.pk, D0, gp0)
        if not self.n_nu:
            return uc, pc
        un, pn = oic.neutrino_particles(noise, c.box, self.pk, D0, gp0, c.nsites, c.nshell, c.nfib, self.q,
                                        self.p_scale, k_fs=self.k_fs)
        return np.hstack([uc, un]), np.hstack([pc, pn])

    def forward(self, noise):
        c, bg = self.cfg, self.bg
        u, p = self.ics(noise)
        f = pm.force(u, self.mass, c.nmesh, c.box, bg.omega_m0)
        states = []
        for (a, ah, b) in self.steps:
            states.append((u, p, f, bgm.step_coefficients(bg, a, ah, b)))
            u, p, f = pm.kdk_step(u, p, f, states[-1][3], self.mass, c.nmesh, c.box, bg.omega_m0)
        return u, p, states

    def loss(self, noise, target):
        u, _, _ = self.forward(noise)
        rho = pm.paint(u, self.mass, self.cfg.nmesh)
        return float(np.mean((rho - target) ** 2))

    def grad(self, noise, target):
        c, bg = self.cfg, self.bg
        n = c.nmesh
        u, p, states = self.forward(noise)
        rho = pm.paint(u, self.mass, n)
        lam_rho = 2.0 * (rho - target) / n ** 3
        lam_x = paint_vjp_positions(u, self.mass, lam_rho, n, c.box)
        lam_p = np.zeros_like(lam_x)
        for (u0, p0, f0, coeffs) in reversed(states):
            lam_x, lam_p = kdk_step_vjp(u0, p0, f0, coeffs, lam_x, lam_p, self.mass, n, c.box, bg.omega_m0)
        D0, gp0 = bg.D(self.a0), bg.gp(self.a0)
        lam_s = D0 * lam_x + gp0 * lam_p
        lam_c = lam_s[:, : self.n_cdm]
        lam_nu = None
        if self.n_nu:
            per_site = c.nshell * (2 * c.nfib + 1)
            lam_nu = lam_s[:, self.n_cdm:].reshape(3, c.nsites ** 3, per_site).sum(axis=2)
        return ic_vjp(lam_c, lam_nu, c.box, self.pk, n_sites=c.nsites, k_fs=self.k_fs, nc=c.nc)
