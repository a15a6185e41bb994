"""Pins of the oracle's particle-mesh machinery: fixed point, sort, CIC, force, step, P(k).

Every test pins the oracle against brute force on tiny inputs, an exact
invariant, or a closed-form linear-response result; none re-types the
oracle's own formula.
"""
import math

import numpy as np
import pytest

from oracle import background as bgm
from oracle import ewald, pm

OM = 0.3


# ----------------------------------------------------------------- fixed point
def test_quantise_round_half_even_and_wrap():
    L = 2.0 ** 32          # one quantum per unit length
    u = pm.quantise(np.array([0.5, 1.5, 2.5, -0.5, -1.0, 2.0 ** 32 + 3.0, 2.0 ** 32 - 0.4]), L)
    assert u.tolist() == [0, 2, 2, 0, 2 ** 32 - 1, 3, 0]


def test_decode_quantise_roundtrip():
    rng = np.random.default_rng(0)
    u = rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(pm.quantise(pm.decode(u, 123.0), 123.0), u)


def test_cell_and_fraction_brute_force():
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2 ** 32, size=200, dtype=np.uint64).astype(np.uint32)
    for n in (32, 64, 2048):
        c, f = pm.cell_and_fraction(u, n)
        for ui, ci, fi in zip(u.tolist(), c.tolist(), f.tolist()):
            assert ci == (ui * n) // 2 ** 32
            assert fi == ((ui * n) % 2 ** 32) / 2 ** 32


# ----------------------------------------------------------------------- sort
def _key_brute(ux, uy, uz, n):
    T = 16
    cells = [(v * n) // 2 ** 32 for v in (ux, uy, uz)]
    t = [c // T for c in cells]
    l = [c % T for c in cells]
    nt = n // T
    cls = (4 if l[0] == T - 1 else 0) + (2 if l[1] == T - 1 else 0) + (1 if l[2] == T - 1 else 0)
    return ((t[0] * nt + t[1]) * nt + t[2]) * 8 + cls


def test_sort_keys_and_stable_permutation_brute_force():
    rng = np.random.default_rng(2)
    n = 64
    u = rng.integers(0, 2 ** 32, size=(3, 300), dtype=np.uint64).astype(np.uint32)
    u[:, 100:150] = u[:, 10:11]          # many equal keys to exercise stability
    keys = pm.sort_keys(u, n)
    brute = [_key_brute(*map(int, u[:, i]), n) for i in range(u.shape[1])]
    assert keys.tolist() == brute
    perm = pm.sort_permutation(u, n)
    expect = sorted(range(len(brute)), key=lambda i: (brute[i], i))
    assert perm.tolist() == expect


# ------------------------------------------------------------------------ CIC
def test_paint_brute_force_tiny():
    rng = np.random.default_rng(3)
    n, L = 8, 8.0
    x = rng.random((3, 5)) * L
    u = pm.quantise(x, L)
    m = rng.random(5) + 0.5
    mesh = pm.paint(u, m, n)
    ref = np.zeros((n, n, n))
    xs = pm.decode(u, L)
    for p in range(5):
        base = [math.floor(xs[d, p]) for d in range(3)]
        fr = [xs[d, p] - base[d] for d in range(3)]
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = 1.0
                    for d, o in enumerate((dx, dy, dz)):
                        w *= fr[d] if o else 1.0 - fr[d]
                    ref[(base[0] + dx) % n, (base[1] + dy) % n, (base[2] + dz) % n] += m[p] * w
    np.testing.assert_allclose(mesh, ref, rtol=1e-13, atol=1e-15)


def test_paint_conserves_mass_and_node_particle():
    rng = np.random.default_rng(4)
    u = rng.integers(0, 2 ** 32, size=(3, 1000), dtype=np.uint64).astype(np.uint32)
    m = rng.random(1000)
    assert pm.paint(u, m, 32).sum() == pytest.approx(m.sum(), rel=1e-13)
    node = pm.quantise(np.array([[3.0], [5.0], [7.0]]), 32.0)
    mesh = pm.paint(node, np.array([2.5]), 32)
    assert mesh[3, 5, 7] == 2.5 and mesh.sum() == 2.5


def test_readout_is_paint_transpose():
    rng = np.random.default_rng(5)
    n = 16
    u = rng.integers(0, 2 ** 32, size=(3, 50), dtype=np.uint64).astype(np.uint32)
    w = rng.normal(size=50)
    M = rng.normal(size=(n, n, n))
    assert (pm.paint(u, w, n) * M).sum() == pytest.approx((w * pm.readout(u, M, n)).sum(), rel=1e-12)


def test_window_definition():
    wf, wh = pm.cic_window(16)
    assert wf[0] == 1.0 and wh[0] == 1.0
    assert wh[8] == pytest.approx((2 / math.pi) ** 2, rel=1e-15)      # sinc^2 at Nyquist
    assert wf[8] == pytest.approx((2 / math.pi) ** 2, rel=1e-15)


# ---------------------------------------------------------------------- force
def _lattice(n, L):
    ax = (np.arange(n) + 0.5) * (L / n)
    return np.meshgrid(ax, ax, ax, indexing="ij")


def _fd4_ratio(k, H):
    """D(k) / k of the 4-point finite-difference gradient."""
    return (8 * math.sin(k * H) - math.sin(2 * k * H)) / (6 * H * k)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("mode", [1, 4, 8])
def test_plane_wave_linear_response_closed_form(axis, mode):
    """Displaced cell-centred lattice, s = A sin(k x_axis) e_axis.

    Linearising CIC paint and readout about cell centres gives, per mode, paint
    factor sinc(kH/2) and readout factor cos(kH/2); the potential is -1.5 Omega_m0
    delta / k^2 and the gradient D(k).  So F_PM / (1.5 Omega_m0 s) =
    cos(kH/2) sinc(kH/2) D(k)/k, exactly up to O(A^2).
    """
    n, L = 32, 32.0
    grid = _lattice(n, L)
    k = 2 * math.pi * mode / L
    A = 1e-4
    s = A * np.sin(k * grid[axis])
    pos = [g.ravel().copy() for g in grid]
    pos[axis] = pos[axis] + s.ravel()
    u = pm.quantise(np.stack(pos), L)
    F = pm.force(u, 1.0, n, L, OM)
    sq = (pm.decode(u[axis], L) - grid[axis].ravel() + L / 2) % L - L / 2
    x = k * L / n / 2
    pred = math.cos(x) * (math.sin(x) / x) * _fd4_ratio(k, L / n)
    ratio = (F[axis] * sq).sum() / (1.5 * OM * (sq * sq).sum())
    assert ratio == pytest.approx(pred, rel=1e-8)
    np.testing.assert_allclose(F[axis], pred * 1.5 * OM * sq, atol=3e-4 * 1.5 * OM * A)
    for other in range(3):
        if other != axis:
            assert np.abs(F[other]).max() < 1e-12 * 1.5 * OM * A


@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("mode", [1, 8])
def test_plane_wave_closed_form_spectral_kernel(axis, mode):
    """The deconvolved spectral kernel: cos(kH/2) / sinc^3(kH/2) (paint sinc, readout cos,
    Green's function / sinc^4, gradient k)."""
    n, L = 32, 32.0
    grid = _lattice(n, L)
    k = 2 * math.pi * mode / L
    A = 1e-4
    pos = [g.ravel().copy() for g in grid]
    pos[axis] = pos[axis] + (A * np.sin(k * grid[axis])).ravel()
    u = pm.quantise(np.stack(pos), L)
    F = pm.force(u, 1.0, n, L, OM, kernel="spectral")
    sq = (pm.decode(u[axis], L) - grid[axis].ravel() + L / 2) % L - L / 2
    x = k * L / n / 2
    pred = math.cos(x) / (math.sin(x) / x) ** 3
    assert (F[axis] * sq).sum() / (1.5 * OM * (sq * sq).sum()) == pytest.approx(pred, rel=1e-8)


def test_fd4_gradient_kernel_values():
    """D(k) = (8 sin kH - sin 2kH) / (6H): k (1 - (kH)^4 / 30 + ...) at small k, 4/(3H) at
    kH = pi/2, exactly zero on the Nyquist index, odd."""
    n, L = 32, 32.0
    dfull, dhalf = pm.gradient_kernel(n, L)
    kfull, khalf, nfull, _ = pm.wavenumbers(n, L)
    assert dfull[1] == pytest.approx(kfull[1] * (1 - (kfull[1]) ** 4 / 30), rel=1e-6)
    assert dhalf[8] == pytest.approx(4.0 / 3.0, rel=1e-14)
    assert dfull[n // 2] == 0.0 and dhalf[n // 2] == 0.0
    np.testing.assert_allclose(dfull[1:n // 2], -dfull[n - 1:n // 2:-1], rtol=1e-13)


@pytest.mark.parametrize("n", [16, 32])
def test_fd4_kernel_is_the_real_space_stencil(n):
    """IFFT(-i D(k_j) phi_k) = -[8 (phi(x + H) - phi(x - H)) - (phi(x + 2H) - phi(x - 2H))] / (12 H)
    along axis j, Nyquist planes included (the 4-point stencil's transfer function is
    i D(k), zero at k H = pi): the identity that lets the force be read out from the
    potential mesh with the stencil applied in real space."""
    L = 40.0
    H = L / n
    rng = np.random.default_rng(n)
    phi = rng.standard_normal((n, n, n))
    phik = np.fft.rfftn(phi) / n ** 3            # unnormalised inverse gives phi back
    for j in range(3):
        F = pm.force_mesh(phik, L, n, j, "fd4")
        r = lambda s: np.roll(phi, -s, axis=j)  # noqa: E731  phi(x + s H)
        ref = -(8.0 * (r(1) - r(-1)) - (r(2) - r(-2))) / (12.0 * H)
        np.testing.assert_allclose(F, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_momentum_conservation_and_self_force():
    rng = np.random.default_rng(6)
    n, L = 32, 50.0
    u = rng.integers(0, 2 ** 32, size=(3, 400), dtype=np.uint64).astype(np.uint32)
    m = rng.random(400) + 0.1
    F = pm.force(u, m, n, L, OM)
    assert np.abs((F * m).sum(axis=1)).max() < 1e-12 * np.abs(F * m).sum()
    lone = pm.force(u[:, :1], np.array([3.0]), n, L, OM)
    assert np.abs(lone).max() < 1e-13


def test_two_particle_action_reaction():
    rng = np.random.default_rng(7)
    n, L = 32, 32.0
    u = rng.integers(0, 2 ** 32, size=(3, 2), dtype=np.uint64).astype(np.uint32)
    F = pm.force(u, np.array([1.0, 1.0]), n, L, OM)
    np.testing.assert_allclose(F[:, 0], -F[:, 1], rtol=1e-11, atol=1e-15)


def test_ewald_reference_limits():
    L = 32.0
    r = np.array([[0.05, 0.0, 0.0], [0.02, 0.03, -0.01]])
    g = ewald.grad_psi(r, L)
    np.testing.assert_allclose(g, -r / np.linalg.norm(r, axis=1)[:, None] ** 3, rtol=1e-4, atol=1e-12)
    np.testing.assert_allclose(ewald.grad_psi(np.array([[L / 2, 0, 0]]), L), 0.0, atol=1e-14)
    r2 = np.array([[3.1, -2.2, 7.5]])
    np.testing.assert_allclose(ewald.grad_psi(r2 + L, L), ewald.grad_psi(r2, L), rtol=1e-8)
    np.testing.assert_allclose(ewald.grad_psi(-r2, L), -ewald.grad_psi(r2, L), rtol=1e-12)
    # converged in alpha and truncation
    np.testing.assert_allclose(ewald.grad_psi(r2, L, alpha=1.2 / L, nreal=4, nk=10),
                               ewald.grad_psi(r2, L), rtol=1e-10)


@pytest.mark.slow
def test_smooth_source_force_matches_ewald_sum():
    """PM force of a Gaussian blob (sigma = 1.5 H) vs the periodic Ewald sum over its particles.

    Tolerance 1% rms, 3% max at separations >= 4 sigma.
    """
    n, L, H = 32, 32.0, 1.0
    rng = np.random.default_rng(5)
    sig = 1.5
    c0 = np.array([10.37, 12.81, 15.29])
    g = (np.arange(-10, 10) + 0.5) * 0.5
    GX, GY, GZ = np.meshgrid(g, g, g, indexing="ij")
    r2 = GX ** 2 + GY ** 2 + GZ ** 2
    keep = r2 < (3.2 * sig) ** 2
    w = np.exp(-r2[keep] / (2 * sig ** 2))
    w /= w.sum()
    blob = np.stack([GX[keep], GY[keep], GZ[keep]], 1) + c0
    nprobe = 60
    dirs = rng.normal(size=(nprobe, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    rr = rng.uniform(4 * sig, L / 4, nprobe)
    probes = (c0 + dirs * rr[:, None]) % L
    u = pm.quantise(np.vstack([blob % L, probes]).T, L)
    mass = np.concatenate([w, np.zeros(nprobe)])
    x = pm.decode(u, L).T
    F = pm.force(u, mass, n, L, OM)[:, len(w):].T
    Fe = np.zeros((nprobe, 3))
    for i in range(nprobe):
        sep = (x[len(w) + i] - x[:len(w)] + L / 2) % L - L / 2
        Fe[i] = (ewald.point_mass_force(sep, L, 1.0, H, OM) * w[:, None]).sum(0)
    err = np.linalg.norm(F - Fe, axis=1) / np.linalg.norm(Fe, axis=1)
    assert np.sqrt(np.mean(err ** 2)) < 0.01
    assert err.max() < 0.03


@pytest.mark.slow
def test_single_particle_force_matches_ewald_sum():
    """One massive particle at random sub-cell offsets, probes at 3-8 cells in random
    directions, against the brute-force periodic Ewald sum: the radial force per
    one-cell shell within 0.5 % on average, the rms relative error of the force vector
    below 2.5 % at 4-5 cells and 1.2 % beyond, the largest below 6 % beyond 4 cells,
    and the tangential part averaging out below 1 %."""
    n, L = 32, 32.0
    rng = np.random.default_rng(3)
    nprobe = 1500
    ratios = {lo: [] for lo in range(3, 8)}
    errs = {lo: [] for lo in range(3, 8)}
    tang_mean = []
    for trial in range(3):
        src = rng.random(3) * L
        dirs = rng.normal(size=(nprobe, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        rr = rng.uniform(3, L / 4, nprobe)
        u = pm.quantise(np.vstack([src[None, :], (src + dirs * rr[:, None]) % L]).T, L)
        mass = np.zeros(nprobe + 1)
        mass[0] = 1.0
        x = pm.decode(u, L).T
        sep = (x[1:] - x[0] + L / 2) % L - L / 2
        Fe = ewald.point_mass_force(sep, L, 1.0, 1.0, OM, )
        F = pm.force(u, mass, n, L, OM)[:, 1:].T
        rhat = sep / np.linalg.norm(sep, axis=1)[:, None]
        Fr, Fer = (F * rhat).sum(1), (Fe * rhat).sum(1)
        err = np.linalg.norm(F - Fe, axis=1) / np.linalg.norm(Fe, axis=1)
        for lo in ratios:
            m = (rr >= lo) & (rr < lo + 1)
            ratios[lo].append(Fr[m].sum() / Fer[m].sum())
            errs[lo].append(err[m])
        tang = F - Fr[:, None] * rhat
        tang_mean.append(np.linalg.norm(tang.mean(0)) / np.abs(Fer).mean())
    for lo, v in ratios.items():
        assert abs(np.mean(v) - 1.0) < 0.005, (lo, v)
    rms = {lo: float(np.sqrt(np.mean(np.concatenate(e) ** 2))) for lo, e in errs.items()}
    assert rms[4] < 0.025, rms
    assert max(rms[lo] for lo in (5, 6, 7)) < 0.012, rms
    assert max(np.concatenate(errs[lo]).max() for lo in (4, 5, 6, 7)) < 0.06
    assert max(tang_mean) < 0.01


def test_boosted_lattice_linear_response():
    """A CDM lattice two and four times coarser than the mesh (the paper runs the mesh at
    twice the CDM grid) displaced by a fundamental-mode plane wave: the force follows
    1.5 Omega_m0 s within 3 %.  The deconvolved spectral kernel is several times off
    here, from the lattice's alias modes inside the mesh's Brillouin zone."""
    nc, L = 16, 32.0
    ax = np.arange(nc) * (L / nc)
    grid = np.meshgrid(ax, ax, ax, indexing="ij")
    k = 2 * math.pi / L
    A = 1e-3
    s = A * np.sin(k * grid[0]).ravel()
    pos = np.stack([g.ravel() for g in grid])
    pos[0] += s
    u = pm.quantise(pos, L)
    sel = np.abs(s) > 0.5 * A
    for boost in (2, 4):
        n = nc * boost
        F = pm.force(u, float(boost ** 3), n, L, OM)
        assert np.median(F[0][sel] / (1.5 * OM * s[sel])) == pytest.approx(1.0, abs=0.03), boost
        Fs = pm.force(u, float(boost ** 3), n, L, OM, kernel="spectral")
        assert np.median(Fs[0][sel] / (1.5 * OM * s[sel])) > 3.0


def test_linear_step_reproduces_zeldovich_growth():
    """One full PM KDK step on a fundamental-mode plane wave (cell-centred lattice, N = N_c).

    The PM force of this lattice is T 1.5 Omega_m0 (x - q) with the closed-form response
    T = cos(kH/2) sinc(kH/2) D(k)/k (previous test), so the step must equal the linear KDK
    recursion with that force exactly, and the Zel'dovich solution x = q + D(a) s,
    p = g_p(a) s up to |1 - T| = O((k_F H)^2)."""
    n, L = 32, 32.0
    bg = bgm.Background.physical(0.68, 0.31, nu_masses_ev=(0.1 / 3,) * 3)
    om = bg.omega_m0
    grid = _lattice(n, L)
    k = 2 * math.pi / L
    A = 1e-3
    s = A * np.sin(k * grid[0]).ravel()
    q = np.stack([g.ravel() for g in grid])
    a0, a1 = 0.1, 0.2
    ah = 0.5 * (a0 + a1)
    x0 = q.copy()
    x0[0] += bg.D(a0) * s
    u = pm.quantise(x0, L)
    p = np.zeros_like(q)
    p[0] = bg.gp(a0) * s
    f0 = pm.force(u, 1.0, n, L, om)
    K1, delta, K2 = bgm.step_coefficients(bg, a0, ah, a1)
    u1, p1, _ = pm.kdk_step(u, p, f0, (K1, delta, K2), 1.0, n, L, om)
    d1 = (pm.decode(u1[0], L) - q[0] + L / 2) % L - L / 2
    x = k * L / n / 2
    T = math.cos(x) * (math.sin(x) / x) * _fd4_ratio(k, L / n)
    d0 = (pm.decode(u[0], L) - q[0] + L / 2) % L - L / 2
    ph = p[0] + K1 * T * 1.5 * om * d0
    d_lin = d0 + delta * ph
    p_lin = ph + K2 * T * 1.5 * om * d1                # the force at the rounded positions
    np.testing.assert_allclose(d1, d_lin, atol=2 * L / 2 ** 32)        # two fixed-point quanta
    np.testing.assert_allclose(p1[0], p_lin, atol=1e-4 * bg.gp(a1) * A)   # O(k s) nonlinearity
    np.testing.assert_allclose(d1, bg.D(a1) * s, atol=(abs(1 - T) + 1e-3) * bg.D(a1) * A)
    np.testing.assert_allclose(p1[0], bg.gp(a1) * s, atol=(abs(1 - T) + 1e-3) * bg.gp(a1) * A)


# ------------------------------------------------------------- power spectrum
def test_power_of_a_single_mode_closed_form():
    n, L = 32, 100.0
    ax = np.arange(n) * (L / n)
    X = ax[:, None, None] * np.ones((1, n, n))
    m, A = 3, 0.2
    mesh = 1.0 + A * np.cos(2 * math.pi * m * X / L)
    nb = 10
    k, P, cnt = pm.power_spectrum(mesh, None, L, nb)
    # modes (+-m, 0, 0) each carry |delta_k|^2 = (A N^3 / 2)^2; P = V/N^6 |delta_k|^2 / W^2
    W = math.sin(math.pi * m / n) / (math.pi * m / n)
    W = W ** 2
    b = m - 1
    expect = 2 * (L ** 3 / n ** 6) * (A * n ** 3 / 2) ** 2 / W ** 2 / cnt[b]
    assert P[b] == pytest.approx(expect, rel=1e-10)
    others = np.delete(np.arange(nb), b)
    assert np.abs(P[others]).max() < 1e-20 * expect
    # bin 0 holds |n| in [0.5, 1.5): 6 modes with |n| = 1 and 12 with |n| = sqrt(2)
    assert cnt[0] == 18
    assert k[0] == pytest.approx((6 + 12 * math.sqrt(2)) / 18 * 2 * math.pi / L, rel=1e-14)


def test_power_mode_counts_match_full_grid():
    n, L = 16, 1.0
    nb = 8
    _, _, cnt = pm.power_spectrum(np.ones((n, n, n)), None, L, nb)
    f = np.fft.fftfreq(n, 1.0 / n)
    KX, KY, KZ = np.meshgrid(f, f, f, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    b = np.floor(kk - 0.5).astype(int)
    ok = (kk >= 0.5) & (b < nb)
    brute = np.bincount(b[ok], minlength=nb)
    # every full-grid mode counted once, except the n_z = -N/2 plane the r2c half stores as +N/2
    np.testing.assert_array_equal(cnt, brute)


def test_cross_power_linearity_identity():
    rng = np.random.default_rng(8)
    n, L = 32, 64.0
    uc = rng.integers(0, 2 ** 32, size=(3, 3000), dtype=np.uint64).astype(np.uint32)
    un = rng.integers(0, 2 ** 32, size=(3, 800), dtype=np.uint64).astype(np.uint32)
    mc, mn = 1.7, 0.4
    dc = pm.paint(uc, mc, n)
    dn = pm.paint(un, mn, n)
    dm = pm.paint(np.hstack([uc, un]), np.concatenate([np.full(3000, mc), np.full(800, mn)]), n)
    fnu = 800 * mn / (3000 * mc + 800 * mn)
    rc, rn, rm = dc / dc.mean(), dn / dn.mean(), dm / dm.mean()
    _, Pcc, _ = pm.power_spectrum(rc, None, L, 12)
    _, Pnn, _ = pm.power_spectrum(rn, None, L, 12)
    _, Pcn, _ = pm.power_spectrum(rc, rn, L, 12)
    _, Pmm, _ = pm.power_spectrum(rm, None, L, 12)
    np.testing.assert_allclose(Pmm, (1 - fnu) ** 2 * Pcc + 2 * fnu * (1 - fnu) * Pcn + fnu ** 2 * Pnn,
                               rtol=1e-11)


def test_force_at_equals_the_full_force_at_the_picked_particles():
    """The sampled oracle force (scipy transforms, readout at a subset) is the full force
    restricted to that subset."""
    rng = np.random.default_rng(11)
    n, box = 32, 100.0
    u = rng.integers(0, 2 ** 32, size=(3, 500), dtype=np.uint64).astype(np.uint32)
    mass = rng.uniform(0.5, 2.0, 500)
    pick = rng.choice(500, 37, replace=False)
    full = pm.force(u, mass, n, box, 0.31)
    for kernel in pm.KERNELS:
        full = pm.force(u, mass, n, box, 0.31, kernel=kernel)
        got = pm.force_at(u, mass, n, box, 0.31, pick, kernel=kernel, workers=2)
        np.testing.assert_allclose(got, full[:, pick], rtol=1e-12, atol=1e-14 * np.abs(full).max())
