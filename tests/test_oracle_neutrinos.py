"""Pins of the oracle's quasi-random Fermi-Dirac sampling (paper §2.1, Appendix A)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import neutrinos as nu

ZETA3 = 1.2020569031595942
ZETA5 = 1.0369277551433699
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


@pytest.fixture(scope="module")
def table10():
    return nu.shell_table(10, [0.2 / 3] * 3)


def test_shell_mass_fractions_sum_to_one(table10):
    _, _, m = table10
    assert m.sum() == pytest.approx(1.0, abs=1e-13)


def test_second_moment_is_exact(table10):
    # sum_i m_i q_i^2 = int q^4 f / int q^2 f, untruncated 15 zeta(5) / zeta(3)
    _, q, m = table10
    assert (m * q ** 2).sum() == pytest.approx(15.0 * ZETA5 / ZETA3, rel=1e-10)


def test_first_moment_bounded_and_converging():
    # Jensen: sum m_i q_i >= <q> = 7 pi^4 / (180 zeta(3)); approaches it as N_shell grows
    mean_q = 7.0 * math.pi ** 4 / (180.0 * ZETA3)
    errs = []
    for ns in (5, 10, 40):
        _, q, m = nu.shell_table(ns, [0.05] * 3)
        first = (m * q).sum()
        assert first >= mean_q
        errs.append(first - mean_q)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1.5e-2


def test_equal_area_under_g_closed_form(table10):
    # int_0^Q x/(e^x + 1) dx = Q^2/2 - Q ln(1 + e^Q) - Li2(-e^Q) + Li2(-1)  (independent of scipy)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    edges, _, _ = table10

    def G(Q):
        Q = mp.mpf(Q)
        return Q ** 2 / 2 - Q * mp.log(1 + mp.e ** Q) - mp.polylog(2, -mp.e ** Q) + mp.polylog(2, -1)
    areas = [float(G(edges[i + 1]) - G(edges[i])) for i in range(10)]
    total = float(G(edges[-1]))
    for a in areas:
        assert a == pytest.approx(total / 10.0, rel=1e-11)


def test_shell_speed_and_mass_by_independent_quadrature(table10):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    edges, q, m = table10
    f = lambda x: 1 / (mp.e ** x + 1)
    z2 = mp.quad(lambda x: x ** 2 * f(x), [0, 5, 10, 40])
    for i in (0, 4, 9):
        lo, hi = edges[i], edges[i + 1]
        pts = [lo, hi] if hi < 10 else [lo, 10, 20, hi]
        m2 = mp.quad(lambda x: x ** 2 * f(x), pts)
        m4 = mp.quad(lambda x: x ** 4 * f(x), pts)
        assert q[i] == pytest.approx(float(mp.sqrt(m4 / m2)), rel=1e-11)
        assert m[i] == pytest.approx(float(m2 / z2), rel=1e-11)


def test_degenerate_limit_reduces_to_fermi_dirac():
    # Eq. FD_deg: alpha_j -> 1 gives f~ = N_nu f, and the table does not depend on N_nu
    a = nu.shell_table(6, [0.1])
    b = nu.shell_table(6, [0.1, 0.1, 0.1])
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-12)


def test_effective_distribution_conserves_mass_and_second_moment():
    # Appendix A: int q^2 f~ = 1.5 zeta(3) sum_j alpha_j, int q^4 f~ = 22.5 zeta(5) sum_j 1/alpha_j
    masses = [0.12, 0.06, 0.02]
    alphas = nu.mass_ratios(masses)
    from scipy import integrate
    ft = lambda q: nu.effective_fd(q, alphas)
    z2, _ = integrate.quad(lambda q: q * q * ft(q), 0, 600, limit=800, epsrel=1e-13)
    z4, _ = integrate.quad(lambda q: q ** 4 * ft(q), 0, 600, limit=800, epsrel=1e-13)
    assert z2 == pytest.approx(1.5 * ZETA3 * sum(alphas), rel=1e-11)
    assert z4 == pytest.approx(22.5 * ZETA5 * sum(1 / a for a in alphas), rel=1e-11)
    # with q_max = 40 / alpha_min the table's second moment reproduces the ratio
    _, q, m = nu.shell_table(10, masses, q_max=40.0 / min(alphas))
    assert (m * q ** 2).sum() == pytest.approx(z4 / z2, rel=1e-9)


def test_fibonacci_directions_symmetric_sums():
    for nfib in (1, 3, 20):
        d = nu.fibonacci_directions(nfib)
        assert d.shape == (2 * nfib + 1, 3)
        np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=1e-15)
        assert abs(d[:, 2].sum()) < 1e-14          # sin(lat) antisymmetric in i
        assert abs(d[:, 1].sum()) < 1e-14          # sin(lon) antisymmetric in i


FIBONACCI_NUMBERS = {1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377, 610, 987, 1597}


def golden_lattice_defects(d):
    """Properties that the Fibonacci (golden-angle) sphere lattice of 2 N_fib + 1 points
    fixes (González 2010, the lattice cited for the directions of §2.1, Eq. N_n), each
    checked without the lattice's own formula.  Returns the list of violated properties.

    1. Equal-area zones: by Archimedes' hat-box theorem a zone of the unit sphere between
       heights z_a < z_b has area 2 pi (z_b - z_a), so n points that each own an equal
       share of the area sit one per zone of height 2 / n, at its centre: sorted heights
       -1 + (2k + 1) / n.
    2. Packing: the smallest distance between two points is ~3.09 / sqrt(n), i.e. 0.87 of
       sqrt(4 pi / n), the side of a square of the mean area per point (González's
       figure), for every n; a spiral with another turning angle packs worse.
    3. Parastichies: in index order the longitude advances by the golden angle, whose
       continued fraction [1; 1, 1, ...] makes the nearest neighbours of every point
       away from the poles lie at Fibonacci-number index offsets.
    """
    n = len(d)
    bad = []
    z = np.sort(d[:, 2])
    if np.abs(z - (-1.0 + (2.0 * np.arange(n) + 1.0) / n)).max() > 1e-14:
        bad.append("equal-area zones")
    dist = np.linalg.norm(d[:, None, :] - d[None, :, :], axis=2)
    np.fill_diagonal(dist, np.inf)
    if dist.min() < 0.86 * math.sqrt(4.0 * math.pi / n):
        bad.append("packing")
    if n >= 41:
        away = np.abs(d[:, 2]) < 0.8
        nearest = np.argsort(dist, axis=1)[:, :2]
        offsets = np.abs(nearest - np.arange(n)[:, None])[away]
        if not all(int(o) in FIBONACCI_NUMBERS for o in offsets.ravel()):
            bad.append("parastichies")
    return bad


def test_fibonacci_directions_are_the_golden_angle_lattice():
    for nfib in (3, 20, 100, 500):
        assert golden_lattice_defects(nu.fibonacci_directions(nfib)) == [], nfib
    # the second moments approach isotropy (sum v v^T / n -> I / 3) as the lattice grows
    aniso = [np.abs(d.T @ d / len(d) - np.eye(3) / 3).max()
             for d in (nu.fibonacci_directions(k) for k in (20, 100, 500))]
    assert aniso[0] < 1e-3 and aniso[2] < 1e-4 and aniso[2] < aniso[0]


def _spiral(nfib, turn):
    """Planted mistakes: the lattice with the longitude of point i replaced by turn(i, n)."""
    n = 2 * nfib + 1
    i = np.arange(-nfib, nfib + 1)
    lat = np.arcsin(2.0 * i / n)
    lon = turn(i, n)
    return np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], axis=1)


@pytest.mark.parametrize("name,turn", [
    ("single turn", lambda i, n: 2.0 * math.pi * i / n),
    ("half the golden turn", lambda i, n: math.pi * i / ((1.0 + math.sqrt(5.0)) / 2.0)),
    ("sqrt(2) turn", lambda i, n: 2.0 * math.pi * i / math.sqrt(2.0)),
])
def test_fibonacci_pins_reject_other_spirals(name, turn):
    for nfib in (20, 100):
        assert golden_lattice_defects(_spiral(nfib, turn)), (name, nfib)
    # a shifted height rule breaks the equal-area zones
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    d = _spiral(20, lambda i, n: 2.0 * math.pi * i / golden)
    assert golden_lattice_defects(d) == []
    d[:, 2] *= 1.0 - 1e-3
    assert "equal-area zones" in golden_lattice_defects(d)


def test_particle_counts_match_paper():
    g = json.load(open(GOLDEN))
    for row in g["table1"]["rows"]:
        n_n = nu.neutrino_count(row["nsites"], row["nshell"], row["nfib"])
        assert n_n == row["nsites"] ** 3 * row["nshell"] * (2 * row["nfib"] + 1)
        assert row["nmesh"] == 2 * row["nc"]                      # Table 1: mesh twice the CDM grid
    r = nu.neutrino_count(128, 10, 3) / 512 ** 3
    assert round(r, g["nn_over_nc_nc512_nf3"]["printed_digits"] - 1) == g["nn_over_nc_nc512_nf3"]["value"]
    r2 = nu.neutrino_count(128, 10, 25) / 1024 ** 3
    assert round(r2, g["nn_over_nn_pseudo"]["printed_digits"]) == g["nn_over_nn_pseudo"]["value"]
    kn = 2 * math.pi * g["k_n_hmpc"]["nsites"] / g["k_n_hmpc"]["box_mpc_h"]
    assert round(kn, g["k_n_hmpc"]["printed_digits"]) == g["k_n_hmpc"]["value"]


def test_species_masses_give_unit_mean_density():
    _, _, m_shell = nu.shell_table(10, [0.2 / 3] * 3)
    mc, mn = nu.species_masses(64, 32, 8, 10, 3, 0.3, 0.01, m_shell)
    total = mc * 32 ** 3 + (mn * 7).sum() * 8 ** 3
    assert total == pytest.approx(64.0 ** 3, rel=1e-14)
    masses = nu.particle_masses(32 ** 3, 8 ** 3 * 70, 10, 3, mc, mn)
    assert masses.sum() == pytest.approx(64.0 ** 3, rel=1e-13)


def test_thermal_momentum_scale():
    # q kT/(m c^2) c/H0 in Mpc/h; kT_nu0 = 1.6764e-4 eV for N_eff = 3 gives 7.54 per unit q at m = 0.2/3 eV
    assert nu.thermal_momentum_scale(1.6764e-4, 0.2 / 3) == pytest.approx(7.54, rel=1e-3)


def test_sites_are_staggered_from_cdm_lattice():
    box, nc, ns = 64.0, 32, 8
    s = nu.site_positions(ns, nc, box)
    dc = box / nc
    frac = (s / dc) % 1.0
    assert np.all(np.abs(frac - 0.5) < 1e-12)        # half a CDM spacing off every lattice plane


def _fd2_integral(q):
    """int_0^q x^2 / (e^x + 1) dx in closed form: -q^2 ln(1 + e^-q) + 2 q Li2(-e^-q)
    + 2 Li3(-e^-q) + 3 zeta(3) / 2 (differentiate to check; zero at q = 0)."""
    mpmath = pytest.importorskip("mpmath")
    z = -mpmath.e ** (-q)
    return float(-q * q * mpmath.log(1 + mpmath.e ** (-q)) + 2 * q * mpmath.polylog(2, z)
                 + 2 * mpmath.polylog(3, z) + 1.5 * mpmath.zeta(3))


@pytest.mark.parametrize("masses", [(0.1, 0.1, 0.1), (0.12, 0.06, 0.02)])
def test_speed_cdf_matches_polylog_closed_form(masses):
    """F(q) = sum_j alpha_j^4 int_0^q x^2 f(alpha_j x) dx / total; each term is
    alpha_j^-3 times the closed form at alpha_j q."""
    al = nu.mass_ratios(list(masses))
    tot = sum(a ** 4 / a ** 3 * _fd2_integral(a * nu.Q_MAX) for a in al)
    for q in (0.3, 1.0, 3.15, 7.0, 15.0):
        ref = sum(a * _fd2_integral(a * q) for a in al) / tot
        assert nu.speed_cdf(q, list(masses)) == pytest.approx(ref, rel=1e-10)


def test_speed_quantile_inverts_cdf_and_reproduces_moments():
    """q(F(q)) = q; the mean and mean square of q(u) over u in (0, 1) are the first two
    moments of the speed density q^2 f(q): 7 pi^4 / (180 zeta(3)) and 15 zeta(5) / zeta(3)."""
    import math
    from scipy.special import zeta
    m = [0.1, 0.1, 0.1]
    for q in (0.5, 2.0, 6.0, 12.0):
        assert nu.speed_quantile(nu.speed_cdf(q, m), m) == pytest.approx(q, rel=1e-10)
    # Gauss-Legendre in t with u = 1 - (1 - t^3)^4: q ~ u^(1/3) ~ t near t = 0 and the
    # q ~ -ln(1 - u) tail damped by (1 - t^3)^3 near t = 1
    t, w = np.polynomial.legendre.leggauss(80)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    u = 1.0 - (1.0 - t ** 3) ** 4
    du = 12.0 * t ** 2 * (1.0 - t ** 3) ** 3
    q = np.array([nu.speed_quantile(v, m) for v in u])
    assert float((w * du * q).sum()) == pytest.approx(7 * math.pi ** 4 / (180 * zeta(3)), rel=1e-6)
    assert float((w * du * q * q).sum()) == pytest.approx(15 * zeta(5) / zeta(3), rel=1e-5)
