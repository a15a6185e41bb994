"""Pins of the FP64 oracle's background, growth ODE and KDK coefficients.

Each test checks the oracle against something other than itself: a closed
form, a limit, an identity between independently computed quantities, or a
textbook value.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import background as bgm

ZETA3 = 1.2020569031595942
ZETA5 = 1.0369277551433699


def test_F_massless_limit_closed_form():
    # F(0) = int x^3 / (1 + e^x) = (7/8) 3! zeta(4) = 7 pi^4 / 120
    assert bgm.fd_F(0.0) == pytest.approx(7.0 * math.pi ** 4 / 120.0, rel=1e-12)


def test_F_nonrelativistic_limit():
    # sqrt(x^2 + y^2) ~ y + x^2/(2y): F(y) ~ 1.5 zeta(3) y + 22.5 zeta(5) / (2 y)
    for y in (1e3, 1e4):
        expect = 1.5 * ZETA3 * y + 22.5 * ZETA5 / (2.0 * y)
        assert bgm.fd_F(y) == pytest.approx(expect, rel=1e-9)


def test_dF_matches_finite_difference():
    for y in (0.3, 3.0, 30.0):
        h = 1e-4 * y
        fd = (bgm.fd_F(y + h) - bgm.fd_F(y - h)) / (2 * h)
        assert bgm.fd_dF(y) == pytest.approx(fd, rel=1e-7)


def test_massless_neutrinos_are_seven_eighths_photons():
    # textbook: rho_nu / rho_gamma = 3 (7/8) Gamma^4 for three massless species
    bg = bgm.Background(omega_gamma=5e-5, omega_c=0.3, omega_lambda=0.7,
                        nu_masses_ev=(0.0, 0.0, 0.0), gamma_nu=(4 / 11) ** (1 / 3), kT_nu0_ev=1.7e-4)
    a = 0.37
    assert bg.omega_nu_E2(a) == pytest.approx(3 * 7 / 8 * bg.gamma_nu ** 4 * 5e-5 / a ** 4, rel=1e-12)


def test_omega_gamma_textbook_value():
    # Omega_gamma h^2 = 2.47e-5 for T_cmb = 2.7255 K (Fixsen 2009 temperature)
    assert bgm.omega_gamma_h2(2.7255) == pytest.approx(2.4728e-5, rel=2e-4)


def test_physical_background_is_flat_and_splits_omega_m():
    bg = bgm.Background.physical(0.68, 0.31, nu_masses_ev=(0.2 / 3,) * 3)
    assert bg.E(1.0) == pytest.approx(1.0, abs=1e-14)
    assert bg.omega_m0 == pytest.approx(0.31, abs=1e-15)
    assert bg.omega_nu_poisson == pytest.approx(0.2 / (93.14 * 0.68 ** 2), rel=1e-14)
    # F-based neutrino density today agrees with 93.14 eV to ~1e-3 (they are different conventions)
    assert bg.omega_nu_E2(1.0) == pytest.approx(bg.omega_nu_poisson, rel=5e-3)


def test_growth_einstein_de_sitter_is_exactly_a():
    bg = bgm.Background(omega_gamma=0.0, omega_c=1.0, omega_lambda=0.0)
    for a in (0.01, 0.05, 0.3, 0.77, 1.0):
        assert bg.D(a) == pytest.approx(a, rel=1e-10)
        assert bg.gp(a) == pytest.approx(a ** 1.5, rel=1e-10)      # a^2 E D' with E = a^-1.5
        assert bg.gf(a) == pytest.approx(1.5 * a, rel=1e-10)


def test_growth_lcdm_matches_heath_integral():
    om, ol = 0.31, 0.69
    bg = bgm.Background(omega_gamma=0.0, omega_c=om, omega_lambda=ol)
    E = lambda a: math.sqrt(om / a ** 3 + ol)

    def heath(a):
        v, _ = integrate.quad(lambda x: 1.0 / (x * E(x)) ** 3, 0.0, a, epsabs=0, epsrel=1e-13)
        return E(a) * v
    h1 = heath(1.0)
    for a in (0.05, 0.2, 0.5, 0.8, 1.0):
        assert bg.D(a) == pytest.approx(heath(a) / h1, rel=1e-9)


def test_gf_identity_by_differencing_gp():
    # g_f = a^2 E dg_p/da must equal 1.5 Omega_m0 D when the ODE is solved right
    bg = bgm.Background.physical(0.68, 0.31, nu_masses_ev=(0.2 / 3,) * 3)
    for a in (0.02, 0.1, 0.4, 0.9):
        h = 1e-4 * a
        dgp = (bg.gp(a + h) - bg.gp(a - h)) / (2 * h)
        assert a * a * bg.E(a) * dgp == pytest.approx(1.5 * bg.omega_m0 * bg.D(a), rel=1e-7)


def test_radiation_lowers_growth_rate_at_z99():
    # growth rate f = dln D / dln a is 1 in matter domination; radiation (photons plus
    # relativistic neutrinos) holds it below 1 at z = 99, Lambda alone does not
    bg_r = bgm.Background.physical(0.68, 0.31, nu_masses_ev=(0.0, 0.0, 0.0))
    bg_l = bgm.Background(omega_gamma=0.0, omega_c=0.31, omega_lambda=0.69)
    f = lambda bg: bg.dD_dlna(0.01) / bg.D(0.01)
    assert f(bg_l) == pytest.approx(1.0, abs=1e-5)
    assert 0.98 < f(bg_r) < 0.995


@pytest.mark.parametrize("sched", ["linear", "paper"])
def test_kdk_coefficients_reproduce_zeldovich_exactly(sched):
    # c.f. §2.3: FastPM factors make x = q + D(a) s exact for F = g_f(a) s
    bg = bgm.Background.physical(0.68, 0.31, nu_masses_ev=(0.1 / 3,) * 3)
    steps = bgm.schedule_linear(0.01, 1.0, 10) if sched == "linear" else bgm.schedule_paper(25)
    s = np.array([0.3, -1.2, 2.5])
    a0 = steps[0][0]
    x = bg.D(a0) * s
    p = bg.gp(a0) * s
    for (ai, ah, a1) in steps:
        K1, Dl, K2 = bgm.step_coefficients(bg, ai, ah, a1)
        p = p + K1 * bg.gf(ai) * s
        x = x + Dl * p
        p = p + K2 * bg.gf(a1) * s
        np.testing.assert_allclose(x, bg.D(a1) * s, rtol=1e-12)
        np.testing.assert_allclose(p, bg.gp(a1) * s, rtol=1e-12)


def test_paper_schedule_shape():
    st = bgm.schedule_paper(25)
    assert len(st) == 25
    assert st[0][0] == 0.01 and st[4][2] == 0.05 and st[-1][2] == pytest.approx(1.0)
    for a, h, b in st[:5]:
        assert h == pytest.approx(math.sqrt(a * b), rel=1e-14)
    for a, h, b in st[5:]:
        assert h == pytest.approx(0.5 * (a + b), rel=1e-14)
