"""Pins of the oracle's synthetic Zel'dovich initial conditions (stand-in for the paper's §2.2)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import ic, neutrinos, pm
from paper_2007_13394_gb300 import inputs


def test_bbks_and_tophat_limits():
    assert ic.bbks_transfer(np.array([1e-8]), 0.31, 0.68)[0] == pytest.approx(1.0, rel=1e-6)
    assert float(ic.tophat_window(np.array([1e-4]))[0]) == pytest.approx(1.0, rel=1e-7)
    # large-q BBKS tail: T ~ ln(2.34 q) / (2.34 q) / (6.71 q)
    q = 1e4
    t = ic.bbks_transfer(np.array([q * 0.31 * 0.68]), 0.31, 0.68)[0]
    assert t == pytest.approx(math.log(2.34 * q) / (2.34 * q) / (6.71 * q), rel=1e-3)


def test_sigma8_normalisation_by_independent_quadrature():
    pk = ic.linear_power(0.31, 0.68, 0.965, 0.81)
    lnk = np.linspace(math.log(1e-5), math.log(1e2), 200001)
    k = np.exp(lnk)
    x = 8.0 * k
    w = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    s2 = np.trapezoid(k ** 3 * pk(k) * w ** 2 / (2 * math.pi ** 2), lnk)
    assert math.sqrt(s2) == pytest.approx(0.81, rel=1e-6)


def test_delta_k_spectrum_matches_input_within_cosmic_variance():
    nc, L = 32, 256.0
    noise = inputs.white_noise(nc, seed=11).astype(np.float64)
    pk = ic.linear_power(0.31, 0.68, 0.965, 0.81)
    dk = ic.delta_k(noise, L, pk)
    mesh = np.fft.irfftn(dk, s=(nc,) * 3)
    # raw estimator without the CIC window: divide P_est by W^2 back out
    k, P, cnt = pm.power_spectrum(mesh + 1.0, None, L, 8)
    wf, wh = pm.cic_window(nc)
    # compare on bins whose modes have W close to 1 and enough modes
    for b in range(1, 6):
        expect = float(pk(k[b]))
        sigma = expect * math.sqrt(2.0 / cnt[b])
        kb = k[b]
        wcorr = (math.sin(kb * L / nc / 2) / (kb * L / nc / 2)) ** 4   # approximate window on the bin centre
        assert abs(P[b] * wcorr - expect) < 4 * sigma + 0.05 * expect, (b, P[b], expect)


def test_displacement_divergence_is_minus_delta():
    nc, L = 16, 64.0
    noise = inputs.white_noise(nc, seed=3).astype(np.float64)
    pk = ic.linear_power(0.31, 0.68, 0.965, 0.81)
    dk = ic.delta_k(noise, L, pk)
    s = ic.displacement(dk, L)
    kfull, khalf, _, _ = pm.wavenumbers(nc, L)
    div_k = (1j * kfull[:, None, None] * np.fft.rfftn(s[0]) + 1j * kfull[None, :, None] * np.fft.rfftn(s[1])
             + 1j * khalf[None, None, :] * np.fft.rfftn(s[2]))
    np.testing.assert_allclose(div_k, -dk, atol=1e-10 * np.abs(dk).max())


def test_neutrino_site_displacement_equals_fourier_series_at_site():
    nc, L, ns = 16, 64.0, 4
    noise = inputs.white_noise(nc, seed=5).astype(np.float64)
    pk = ic.linear_power(0.31, 0.68, 0.965, 0.81)
    dk = ic.delta_k(noise, L, pk)
    full = np.zeros((nc, nc, nc), dtype=complex)
    full[:, :, : nc // 2 + 1] = dk
    for kz in range(1, nc // 2):                       # Hermitian completion
        full[:, :, nc - kz] = np.conj(dk[(-np.arange(nc)) % nc][:, (-np.arange(nc)) % nc][:, :, kz])
    f = np.fft.fftfreq(nc, 1.0 / nc) * (2 * math.pi / L)
    KX, KY, KZ = np.meshgrid(f, f, f, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    sites = neutrinos.site_positions(ns, nc, L)
    r, j0, sh = ic.neutrino_site_offset(nc, ns)
    s_sites = ic.displacement(dk, L, shift=sh * L / nc)
    idx = j0 + r * np.arange(ns)
    got = s_sites[:, idx][:, :, idx][:, :, :, idx].reshape(3, -1)
    for si in (0, 7, 33, 63):
        q = sites[si]
        ph = np.exp(1j * (KX * q[0] + KY * q[1] + KZ * q[2]))
        for d, K in enumerate((KX, KY, KZ)):
            val = (1j * K * full / k2 * ph).sum().real / nc ** 3
            assert got[d, si] == pytest.approx(val, rel=1e-9, abs=1e-12)


def test_particle_layout_and_thermal_terms():
    nc, L, ns, nshell, nfib = 16, 64.0, 4, 3, 1
    noise = inputs.white_noise(nc, seed=9).astype(np.float64)
    pk = ic.linear_power(0.31, 0.68, 0.965, 0.81)
    _, q, _ = neutrinos.shell_table(nshell, [0.1])
    uc, pc = ic.cdm_particles(noise, L, pk, 0.0, 0.0)
    # zero growth: CDM exactly on lattice nodes with zero momentum
    ax = np.arange(nc) * (L / nc)
    assert pm.decode(uc[0], L).reshape(nc, nc, nc)[:, 0, 0] == pytest.approx(ax)
    assert np.all(pc == 0)
    un, pn = ic.neutrino_particles(noise, L, pk, 0.0, 0.0, ns, nshell, nfib, q, p_scale=2.0)
    assert un.shape == (3, ns ** 3 * nshell * (2 * nfib + 1))
    # momentum of particle (site 0, shell i, dir j) = 2 q_i n_j; positions = site + radius n_j
    dirs = neutrinos.fibonacci_directions(nfib)
    site0 = neutrinos.site_positions(ns, nc, L)[0]
    for shell in range(nshell):
        for d in range(3):
            i = shell * 3 + d
            np.testing.assert_allclose(pn[:, i], 2.0 * q[shell] * dirs[d], rtol=1e-14)
            rad = 0.45 * (L / ns) * q[shell] / q.max()
            np.testing.assert_allclose(pm.decode(un[:, i], L), (site0 + rad * dirs[d]) % L, atol=1e-7)


def test_free_streaming_k_limits():
    # today (a = 1, flat) k_fs = 0.82 (m / 1 eV) h/Mpc; deep in matter domination it grows as
    # sqrt(Omega_m a): k_fs(a) / k_fs(a / 4) -> 2
    assert ic.free_streaming_k([0.1, 0.1, 0.1], 1.0, 0.31) == pytest.approx(0.082, rel=1e-14)
    assert ic.free_streaming_k([0.3], 1.0, 0.5) == pytest.approx(0.82 * 0.3, rel=1e-14)
    r = ic.free_streaming_k([0.2], 4e-4, 0.31) / ic.free_streaming_k([0.2], 1e-4, 0.31)
    assert r == pytest.approx(2.0, rel=1e-6)
