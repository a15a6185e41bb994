"""FP64 particle-mesh force, kick-drift-kick step and power spectrum.

Test infrastructure only (see the package docstring).

The paper runs FastPM's particle-mesh solver (§1 "implements a particle-mesh
approach", §2.3 first paragraph, §3 mesh N_mesh^(1/3) = 2 N_c^(1/3)) but does
not spell the solver out.  This module writes out the plain definitions the
GPU path is held to:

* positions are 32-bit fixed point, x = u L / 2^32, periodic by integer
  wraparound; quantisation rounds half to even;
* cloud-in-cell (CIC) paint of rho / rho_bar: mass m at x gives
  m prod_d (1 - |x_d / H - i_d|) to the 8 nodes around it, periodic;
* delta_k = FFT(rho / rho_bar) (forward e^{-ikx}, unnormalised); k = 0 dropped;
* phi_k = -(3/2) Omega_m0 delta_k / N^3 / k^2, k_d = 2 pi n_d / L,
  n_d in [-N/2, N/2); Poisson source from §2.2 Eq. Om_pois (neutrinos count
  as matter);
* F_j(x) = IFFT[-i D(k_j) phi_k] (unnormalised inverse) with the 4-point
  finite-difference gradient D(k) = (8 sin(kH) - sin(2kH)) / (6H), which is
  real, odd and zero on the Nyquist index.  No CIC window deconvolution in the
  force (the paper inherits FastPM's solver and names no kernel; this one
  reproduces linear growth for a particle lattice coarser than the mesh, the
  paper's mesh twice the CDM grid, and the Ewald force of an isolated particle,
  where a spectral gradient with the W^-2 deconvolution does neither).  The
  alternative kernel="spectral" is that deconvolved form: phi_k / W(k)^2 with
  W(k) = prod_d sinc^2(k_d H / 2) and gradient k_j (0 at n_j = -N/2);
* CIC readout of F_j at each particle with the paint's weights;
* FastPM kick-drift-kick (§2.1 "Kick-Drift-Kick", §2.3) with the coefficients
  of :mod:`oracle.background`.
* P_ab(k) = (V / N^6) Re(delta_a delta_b^*) / W(k)^2 per mode, each delta_s the
  painted species over its own mean, no shot-noise
  subtraction, linear bins of width k_F = 2 pi / L starting at k_F / 2,
  mode-weighted mean |k| per bin, r2c modes with 0 < n_z < N/2 counted twice.

The sort contract (stable counting sort into tiles of mesh cells): tiles are
T^3 = 16^3 cells; tile id = (t_x * (N/T) + t_y) * (N/T) + t_z; the face class
of a cell is 4 [l_x = T-1] + 2 [l_y = T-1] + [l_z = T-1] for its in-tile
coordinates l; key = tile id * 8 + class; the order is the stable order of the
key with respect to the incoming particle index.
"""
from __future__ import annotations

import numpy as np

TWO32 = 2.0 ** 32
TILE = 16


# ----------------------------------------------------------------- fixed point
def quantise(x, box):
    """Position (any real, Mpc/h) -> uint32 fixed point, round half to even, mod 2^32."""
    v = np.rint(np.asarray(x, dtype=np.float64) * (TWO32 / box))
    return np.mod(v, TWO32).astype(np.uint64).astype(np.uint32)


def decode(u, box):
    """uint32 fixed point -> position in [0, L)."""
    return np.asarray(u, dtype=np.float64) * (box / TWO32)


def cell_and_fraction(u, n):
    """Cell index (u N) >> 32 and fractional offset ((u N) mod 2^32) / 2^32, exactly."""
    prod = np.asarray(u, dtype=np.uint64) * np.uint64(n)
    cell = (prod >> np.uint64(32)).astype(np.int64)
    frac = (prod & np.uint64(0xFFFFFFFF)).astype(np.float64) / TWO32
    return cell, frac


# ----------------------------------------------------------------------- sort
def sort_keys(u, n):
    """(tile, face class) key of every particle; u has shape (3, n_particles)."""
    nt = n // TILE
    c = [cell_and_fraction(u[d], n)[0] for d in range(3)]
    t = [ci // TILE for ci in c]
    l = [ci % TILE for ci in c]
    tile = (t[0] * nt + t[1]) * nt + t[2]
    cls = 4 * (l[0] == TILE - 1) + 2 * (l[1] == TILE - 1) + (l[2] == TILE - 1)
    return (tile * 8 + cls).astype(np.int64)


def sort_permutation(u, n):
    """Stable order of the keys: perm[i] = incoming index of the i-th sorted particle."""
    return np.argsort(sort_keys(u, n), kind="stable")


# ------------------------------------------------------------------------ CIC
def _corner_weights(u, n):
    cells, fracs = zip(*[cell_and_fraction(u[d], n) for d in range(3)])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                idx = []
                w = np.ones(u.shape[1])
                for d, o in enumerate((dx, dy, dz)):
                    idx.append((cells[d] + o) % n)
                    w = w * (fracs[d] if o else 1.0 - fracs[d])
                flat = (idx[0] * n + idx[1]) * n + idx[2]
                yield flat, w


def paint(u, mass, n):
    """CIC density rho / rho_bar on the N^3 mesh (mass in units of the mean mass per cell)."""
    mesh = np.zeros(n ** 3)
    mass = np.broadcast_to(np.asarray(mass, dtype=np.float64), (u.shape[1],))
    for flat, w in _corner_weights(u, n):
        mesh += np.bincount(flat, weights=mass * w, minlength=n ** 3)
    return mesh.reshape(n, n, n)


def readout(u, mesh, n):
    """CIC interpolation of a real N^3 mesh at the particles (the paint's transpose)."""
    flatmesh = mesh.reshape(-1)
    out = np.zeros(u.shape[1])
    for flat, w in _corner_weights(u, n):
        out += w * flatmesh[flat]
    return out


# ---------------------------------------------------------------- k-space ops
def wavenumbers(n, box):
    """k_d = 2 pi n_d / L for the full axis (n_d in [-N/2, N/2)) and the r2c half axis."""
    nfull = np.fft.fftfreq(n, d=1.0 / n)           # 0..N/2-1, -N/2..-1
    nhalf = np.arange(n // 2 + 1, dtype=np.float64)
    kf = 2.0 * np.pi / box
    return nfull * kf, nhalf * kf, nfull, nhalf


def cic_window(n):
    """Per-axis CIC window sinc^2(pi n_d / N) on the full and half axes."""
    _, _, nfull, nhalf = wavenumbers(n, 1.0)
    return np.sinc(nfull / n) ** 2, np.sinc(nhalf / n) ** 2      # np.sinc(x) = sin(pi x)/(pi x)


KERNELS = ("fd4", "spectral")


def gradient_kernel(n, box, kernel="fd4"):
    """Per-axis gradient multiplier D(k) on the full axis and on the r2c half axis."""
    kfull, khalf, nfull, nhalf = wavenumbers(n, box)
    if kernel == "fd4":
        H = box / n
        d = lambda k: (8.0 * np.sin(k * H) - np.sin(2.0 * k * H)) / (6.0 * H)  # noqa: E731
        dfull, dhalf = d(kfull), d(khalf)
    elif kernel == "spectral":
        dfull, dhalf = kfull.copy(), khalf.copy()
    else:
        raise ValueError(kernel)
    dfull[nfull == -n // 2] = 0.0      # Nyquist index: zero (exactly, for the odd kernel)
    dhalf[nhalf == n // 2] = 0.0
    return dfull, dhalf


def green_half(n, box, omega_m0, kernel="fd4"):
    """Real multiplier c(k) of FFT(rho / rho_bar) giving phi_k on the r2c half grid; c(0) = 0."""
    kfull, khalf, _, _ = wavenumbers(n, box)
    k2 = kfull[:, None, None] ** 2 + kfull[None, :, None] ** 2 + khalf[None, None, :] ** 2
    if kernel == "spectral":
        wfull, whalf = cic_window(n)
        k2 = k2 * (wfull[:, None, None] * wfull[None, :, None] * whalf[None, None, :]) ** 2
    elif kernel != "fd4":
        raise ValueError(kernel)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = -1.5 * omega_m0 / n ** 3 / k2
    g[0, 0, 0] = 0.0
    return g


def potential_k(mesh, box, omega_m0, kfactor=None, kernel="fd4"):
    """phi_k = c(k) FFT(rho/rho_bar), c = -(3/2) Omega_m0 / N^3 / k^2 (see green_half).

    kfactor: optional real multiplier of the Green's function on the r2c half grid
    (N, N, N/2 + 1), the learned correction m(|k|, a) of :mod:`oracle.mlp`.
    """
    n = mesh.shape[0]
    g = green_half(n, box, omega_m0, kernel)
    if kfactor is not None:
        g = g * kfactor
    return np.fft.rfftn(mesh) * g


def force_mesh(phi_k, box, n, component, kernel="fd4"):
    """F_j(x) = IFFT_unnormalised[-i D(k_j) phi_k]."""
    dfull, dhalf = gradient_kernel(n, box, kernel)
    if component == 0:
        kj = dfull[:, None, None]
    elif component == 1:
        kj = dfull[None, :, None]
    else:
        kj = dhalf[None, None, :]
    fk = -1j * kj * phi_k
    return np.fft.irfftn(fk, s=(n, n, n), axes=(0, 1, 2)) * n ** 3


def force(u, mass, n, box, omega_m0, kfactor=None, kernel="fd4"):
    """PM force (3, n_particles) at the particles (kfactor: see :func:`potential_k`)."""
    phi = potential_k(paint(u, mass, n), box, omega_m0, kfactor, kernel)
    return np.stack([readout(u, force_mesh(phi, box, n, j, kernel), n) for j in range(3)])


def force_at(u, mass, n, box, omega_m0, pick, kernel="fd4", workers=None):
    """The PM force of :func:`force` read out only at the particles ``pick`` (3, len(pick)).

    The mesh steps are the same definitions -- paint of every particle, phi_k, F_j =
    IFFT[-i D(k_j) phi_k] -- with the transforms on ``workers`` threads of scipy.fft (a
    library FFT like numpy's; the thread count changes only the speed).  For sampled
    checks on meshes where reading out every particle would be slow."""
    from scipy import fft as sfft
    phi = sfft.rfftn(paint(u, mass, n), workers=workers)
    phi *= green_half(n, box, omega_m0, kernel)
    dfull, dhalf = gradient_kernel(n, box, kernel)
    up = np.asarray(u)[:, pick]
    out = []
    for j, kj in enumerate((dfull[:, None, None], dfull[None, :, None], dhalf[None, None, :])):
        fj = sfft.irfftn(-1j * kj * phi, s=(n, n, n), axes=(0, 1, 2), workers=workers) * n ** 3
        out.append(readout(up, fj, n))
        del fj
    return np.stack(out)


# --------------------------------------------------------------- kick / drift
def drift(u, p, delta, box):
    """u_d <- (u_d + rne(Delta p_d 2^32 / L)) mod 2^32 (exact periodicity)."""
    step = np.rint(delta * np.asarray(p, dtype=np.float64) * (TWO32 / box))
    return np.mod(np.asarray(u, dtype=np.float64) + step, TWO32).astype(np.uint64).astype(np.uint32)


def kdk_step(u, p, f0, coeffs, mass, n, box, omega_m0, kernel="fd4"):
    """One FastPM KDK step with coefficients (K1, Delta, K2) and the force f0 at a0.

    Returns (u1, p1, f1) with f1 the force at a1 (the next step's first kick).
    """
    K1, delta, K2 = coeffs
    p = p + K1 * f0
    u = drift(u, p, delta, box)
    f1 = force(u, mass, n, box, omega_m0, kernel=kernel)
    p = p + K2 * f1
    return u, p, f1


# ------------------------------------------------------------ power spectrum
def power_spectrum(mesh_a, mesh_b, box, nbins):
    """Binned P_ab(k) of delta_s = rho_s / rho_bar_s - 1 (each mesh over its own mean).

    Returns (k_mean, P, n_modes) of length nbins.
    """
    n = mesh_a.shape[0]
    da = np.fft.rfftn(mesh_a / mesh_a.mean())
    db = da if mesh_b is None else np.fft.rfftn(mesh_b / mesh_b.mean())
    kfull, khalf, _, nhalf = wavenumbers(n, box)
    wfull, whalf = cic_window(n)
    kmag = np.sqrt(kfull[:, None, None] ** 2 + kfull[None, :, None] ** 2 + khalf[None, None, :] ** 2)
    w2 = (wfull[:, None, None] * wfull[None, :, None] * whalf[None, None, :]) ** 2
    vol = box ** 3
    pk = vol / float(n) ** 6 * np.real(da * np.conj(db)) / w2
    mult = np.where((nhalf > 0) & (nhalf < n // 2), 2.0, 1.0)[None, None, :] * np.ones_like(kmag)
    kf = 2.0 * np.pi / box
    b = np.floor((kmag - 0.5 * kf) / kf).astype(np.int64)
    ok = (kmag >= 0.5 * kf) & (b < nbins)
    b, mult, kmag, pk = b[ok], mult[ok], kmag[ok], pk[ok]
    cnt = np.bincount(b, weights=mult, minlength=nbins)
    ksum = np.bincount(b, weights=mult * kmag, minlength=nbins)
    psum = np.bincount(b, weights=mult * pk, minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt.astype(np.int64)
