"""FP64 learned correction of the particle-mesh Green's function, its gradients and
the training loss it is fitted to.

Test infrastructure only (see the package docstring).

The paper has no learned part; this is the production pattern layered on the
method: a small network m_theta(kappa, a) multiplies the Green's function of the
potential (the phi_k of :func:`oracle.pm.potential_k`), with kappa = |k| / k_Ny,
k_Ny = pi N / L and a the scale factor at which the force is evaluated.

Readings (none of them is in the paper):
* network: Linear(2, 64) -> SiLU -> Linear(64, 64) -> SiLU -> Linear(64, 1),
  m = 1 + out, SiLU(z) = z / (1 + e^-z); the last layer starts at zero so the
  untrained network is the plain kernel exactly;
* flat parameter vector theta (NPARAM = 4417 values): W1[64][2] (row j holds
  the weights of kappa and a into unit j), b1[64], W2[64][64] (row = output
  unit), b2[64], w3[64], b3;
* training loss: the mass-weighted mean of the periodic squared displacement
  between the corrected run and a target run from the same initial conditions,
  L = sum_i m_i |x_i - y_i|^2 / sum_i m_i, with x_i - y_i the wrapped difference
  (the int32 difference of the fixed-point positions times L / 2^32);
* gradient: the FastPM step adjoint of :mod:`oracle.adjoint` plus, at every
  force evaluation F(x; a), the derivative with respect to the factor.  With
  F_j = IFFT[h_j rho_k], h_j = -i D(k_j) c(k) m(k), c the plain Green's function
  and D the gradient kernel of :mod:`oracle.pm`,
  and A_j = FFT(paint(lambda_F,j)):
      <lambda_F, F> = sum_j sum_k h_j(k) rho_k conj(A_j,k)   (full k grid),
  so d<lambda_F, F>/dm(k) = Re sum_j (-i D(k_j)) c(k) rho_k conj(A_j,k), counted
  twice for r2c modes with 0 < n_z < N/2, and the theta gradient is the
  network's backward pass weighted by it.
"""
from __future__ import annotations

import numpy as np

from . import adjoint as oad
from . import background as bgm
from . import pm

HIDDEN = 64
NPARAM = 2 * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(theta):
    """Views (W1 (64, 2), b1, W2 (64, 64), b2, w3, b3) of the flat parameter vector."""
    t = np.asarray(theta, dtype=np.float64)
    assert t.shape == (NPARAM,)
    o = 0
    W1 = t[o:o + 2 * HIDDEN].reshape(HIDDEN, 2); o += 2 * HIDDEN
    b1 = t[o:o + HIDDEN]; o += HIDDEN
    W2 = t[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = t[o:o + HIDDEN]; o += HIDDEN
    w3 = t[o:o + HIDDEN]; o += HIDDEN
    b3 = t[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _layers(theta, kappa, a):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    x = np.stack([np.ravel(kappa), np.broadcast_to(a, np.shape(np.ravel(kappa)))], axis=1)  # (n, 2)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    return x, z1, h1, z2, h2, h2 @ w3 + b3


def forward(theta, kappa, a):
    """m(kappa, a) = 1 + MLP(kappa, a) at every kappa (same shape as kappa)."""
    out = _layers(theta, kappa, a)[-1]
    return (1.0 + out).reshape(np.shape(kappa))


def vjp(theta, kappa, a, gm):
    """sum_i gm_i dm(kappa_i, a) / dtheta, a flat vector of NPARAM values."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    x, z1, h1, z2, h2, _ = _layers(theta, kappa, a)
    g = np.ravel(gm).astype(np.float64)
    dw3 = h2.T @ g
    db3 = g.sum()
    dz2 = (g[:, None] * w3[None, :]) * dsilu(z2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    dW1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dw3, db3)


# ------------------------------------------------------------------ k-space grid
def kappa_half(n):
    """|k| / k_Ny on the r2c half grid (N, N, N/2 + 1): sqrt(n_x^2 + n_y^2 + n_z^2) / (N/2)."""
    _, _, nfull, nhalf = pm.wavenumbers(n, 1.0)
    n2 = nfull[:, None, None] ** 2 + nfull[None, :, None] ** 2 + nhalf[None, None, :] ** 2
    return np.sqrt(n2) / (n / 2)


def factor_mesh(theta, n, a):
    """m(|k| / k_Ny, a) on the r2c half grid."""
    return forward(theta, kappa_half(n), a)


def force(u, mass, n, box, omega_m0, theta, a):
    """Learned PM force: the plain force with phi_k multiplied by m(|k| / k_Ny, a)."""
    return pm.force(u, mass, n, box, omega_m0, factor_mesh(theta, n, a))


def dloss_dfactor(u, mass, lam_f, n, box, omega_m0, kernel="fd4"):
    """d <lam_f, F> / d m(k) per r2c mode (with its r2c multiplicity), shape (N, N, N/2+1)."""
    rho_k = np.fft.rfftn(pm.paint(u, mass, n))
    cg = pm.green_half(n, box, omega_m0, kernel)          # plain Green's function c(k)
    dfull, dhalf = pm.gradient_kernel(n, box, kernel)
    _, _, _, nhalf = pm.wavenumbers(n, box)
    q = np.zeros(rho_k.shape)
    for j, dj in enumerate((dfull[:, None, None], dfull[None, :, None], dhalf[None, None, :])):
        a_j = np.fft.rfftn(pm.paint(u, lam_f[j], n))
        q += np.real(-1j * dj * cg * rho_k * np.conj(a_j))
    mult = np.where((nhalf > 0) & (nhalf < n // 2), 2.0, 1.0)[None, None, :]
    return q * mult


def force_theta_vjp(u, mass, lam_f, n, box, omega_m0, theta, a):
    """d <lam_f, F(x; theta, a)> / d theta (flat, NPARAM)."""
    gm = dloss_dfactor(u, mass, lam_f, n, box, omega_m0)
    return vjp(theta, kappa_half(n), a, gm)


# ----------------------------------------------------------------- training loss
def wrapped_displacement(u, v, box):
    """x - y for fixed-point positions, wrapped to [-L/2, L/2): int32(u - v) L / 2^32."""
    d = (np.asarray(u, dtype=np.int64) - np.asarray(v, dtype=np.int64)) % (1 << 32)
    d = np.where(d >= (1 << 31), d - (1 << 32), d)
    return d.astype(np.float64) * (box / pm.TWO32)


def displacement_loss(u, v, mass, box):
    """L = sum_i m_i |x_i - y_i|^2 / sum_i m_i and dL/dx (3, n_particles)."""
    d = wrapped_displacement(u, v, box)
    m = np.asarray(mass, dtype=np.float64)
    w = m.sum()
    return float((m[None, :] * d * d).sum() / w), 2.0 * m[None, :] * d / w


class LearnedRun:
    """ICs from white noise -> KDK steps with the learned force -> final positions,
    and dL/dtheta of the displacement loss against target positions by the adjoint."""

    def __init__(self, cfg, steps, a0, k_fs=0.0):
        self.rec = oad.Reconstruction(cfg, steps, a0, k_fs)
        self.cfg, self.steps, self.a0 = cfg, steps, a0

    def _force(self, u, theta, a):
        c, bg = self.cfg, self.rec.bg
        return force(u, self.rec.mass, c.nmesh, c.box, bg.omega_m0, theta, a)

    def forward(self, noise, theta):
        c, bg = self.cfg, self.rec.bg
        u, p = self.rec.ics(noise)
        f = self._force(u, theta, self.a0)
        states = []
        for (a, ah, b) in self.steps:
            coeffs = bgm.step_coefficients(bg, a, ah, b)
            states.append((u, p, f, coeffs, a, b))
            K1, delta, K2 = coeffs
            ph = p + K1 * f
            u = pm.drift(u, ph, delta, c.box)
            f = self._force(u, theta, b)
            p = ph + K2 * f
        return u, p, states

    def loss(self, noise, theta, target_u):
        u, _, _ = self.forward(noise, theta)
        return displacement_loss(u, target_u, self.rec.mass, self.cfg.box)[0]

    def grad(self, noise, theta, target_u):
        """(L, dL/dtheta)."""
        c, bg = self.cfg, self.rec.bg
        n, box, om, mass = c.nmesh, c.box, bg.omega_m0, self.rec.mass
        u, _, states = self.forward(noise, theta)
        L, lam_x = displacement_loss(u, target_u, mass, box)
        lam_p = np.zeros_like(lam_x)
        g = np.zeros(NPARAM)
        for (u0, p0, f0, (K1, delta, K2), a, b) in reversed(states):
            m0, m1 = factor_mesh(theta, n, a), factor_mesh(theta, n, b)
            ph = p0 + K1 * f0
            u1 = pm.drift(u0, ph, delta, box)
            lf1 = K2 * lam_p
            g += force_theta_vjp(u1, mass, lf1, n, box, om, theta, b)
            lam_x = lam_x + oad.force_vjp(u1, mass, lf1, n, box, om, m1)
            lam_ph = lam_p + delta * lam_x
            lf0 = K1 * lam_ph
            g += force_theta_vjp(u0, mass, lf0, n, box, om, theta, a)
            lam_x = lam_x + oad.force_vjp(u0, mass, lf0, n, box, om, m0)
            lam_p = lam_ph
        return L, g


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2014, Algorithm 1): returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------------------- spectrum loss
def power_vjp(u, mass, n, box, nbins, dL_dP):
    """d L / d x (3, n_particles) for L depending on the binned auto-spectrum of the painted
    mass (:func:`oracle.pm.power_spectrum` of paint(u, mass)) through dL_dP[b].

    With F = FFT(rho), rho_bar its mean, P_b = (V / N^6) sum_{k in b} |F_k|^2 /
    (rho_bar^2 W_k^2) / N_b over the full grid (N_b its mode count) and rho_bar fixed by
    the total mass: dL/drho(x) = 2 sum_k c_k F_k e^{ikx}, c_k = dL/dP_b V / (N^6 rho_bar^2
    W_k^2 N_b) for k in bin b; then the paint's position VJP.
    """
    mass = np.broadcast_to(np.asarray(mass, dtype=np.float64), (u.shape[1],))
    rho = pm.paint(u, mass, n)
    F = np.fft.rfftn(rho)
    rho_bar = rho.mean()
    kfull, khalf, nfull, nhalf = pm.wavenumbers(n, box)
    kmag = np.sqrt(kfull[:, None, None] ** 2 + kfull[None, :, None] ** 2 + khalf[None, None, :] ** 2)
    kf = 2.0 * np.pi / box
    b = np.floor((kmag - 0.5 * kf) / kf).astype(np.int64)
    ok = (kmag >= 0.5 * kf) & (b < nbins)
    mult = np.where((nhalf > 0) & (nhalf < n // 2), 2.0, 1.0)[None, None, :] * np.ones_like(kmag)
    counts = np.bincount(b[ok], weights=mult[ok], minlength=nbins)
    wfull, whalf = pm.cic_window(n)
    w2 = (wfull[:, None, None] * wfull[None, :, None] * whalf[None, None, :]) ** 2
    g = np.asarray(dL_dP, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        per_bin = np.where(counts > 0, g / counts, 0.0)
    c = np.zeros(F.shape)
    c[ok] = per_bin[b[ok]]
    c = c * box ** 3 / (float(n) ** 6 * rho_bar ** 2 * w2)
    lam = 2.0 * n ** 3 * np.fft.irfftn(c * F, s=(n, n, n), axes=(0, 1, 2))
    return oad.paint_vjp_positions(u, mass, lam, n, box)


def power_loss(u, mass, n, box, nbins, p_ref, bins):
    """Spectrum-matching loss L = mean_{b in bins} (P_b / P_ref,b - 1)^2 of the total
    painted mass and dL/dP (length nbins, zero outside bins)."""
    _, P, _ = pm.power_spectrum(pm.paint(u, mass, n), None, box, nbins)
    sel = np.zeros(nbins, dtype=bool)
    sel[list(bins)] = True
    r = P[sel] / np.asarray(p_ref)[sel] - 1.0
    g = np.zeros(nbins)
    g[sel] = 2.0 * r / (sel.sum() * np.asarray(p_ref)[sel])
    return float(np.mean(r ** 2)), g
