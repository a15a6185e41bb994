"""Pins of the oracle's adjoint: finite differences (exact for the piecewise-polynomial
CIC maps when the perturbation stays inside a cell), dot-product tests, and a
finite-difference check of the full reconstruction gradient."""
import numpy as np
import pytest

from oracle import adjoint as oad
from oracle import background as obg
from oracle import ic as oic
from oracle import pm as opm
from paper_2007_13394_gb300 import inputs

OM = 0.3


def _safe_particles(n, npart, seed):
    """Positions at least 1e-3 of a cell away from every face (safe for +-eps moves)."""
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, n, size=(3, npart))
    frac = rng.uniform(0.01, 0.99, size=(3, npart))
    return ((cell + frac) * (2.0 ** 32 / n)).astype(np.uint64).astype(np.uint32)


def _shift(u, i, d, k):
    v = u.copy()
    v[d, i] = np.uint32((int(v[d, i]) + k) % 2 ** 32)
    return v


def test_readout_grad_is_exact_derivative():
    n, L = 8, 8.0
    u = _safe_particles(n, 40, 1)
    M = inputs.normal_values((n, n, n), seed=2)
    g = oad.readout_grad(u, M, n, L)
    k = 4096
    dx = k * L / 2 ** 32
    for i in (0, 7, 33):
        for d in range(3):
            fp = opm.readout(_shift(u, i, d, k), M, n)[i]
            fm = opm.readout(_shift(u, i, d, -k), M, n)[i]
            assert (fp - fm) / (2 * dx) == pytest.approx(g[d, i], rel=1e-7, abs=1e-9)


def test_force_vjp_matches_finite_differences():
    n, L = 16, 16.0
    u = _safe_particles(n, 120, 3)
    mass = inputs.uniform_masses(120, seed=4)
    lam = inputs.normal_values((3, 120), seed=5)
    g = oad.force_vjp(u, mass, lam, n, L, OM)
    k = 2048
    dx = k * L / 2 ** 32
    obj = lambda v: float((lam * opm.force(v, mass, n, L, OM)).sum())
    for i in (0, 50, 119):
        for d in range(3):
            fd = (obj(_shift(u, i, d, k)) - obj(_shift(u, i, d, -k))) / (2 * dx)
            assert fd == pytest.approx(g[d, i], rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_kdk_step_vjp_matches_finite_differences():
    n, L = 16, 16.0
    bg = obg.Background(omega_gamma=0.0, omega_c=OM, omega_lambda=1 - OM)
    coeffs = obg.step_coefficients(bg, 0.3, 0.35, 0.4)
    u0 = _safe_particles(n, 60, 6)
    mass = inputs.uniform_masses(60, seed=7)
    p0 = 0.01 * inputs.normal_values((3, 60), seed=8)
    f0 = opm.force(u0, mass, n, L, OM)
    lx, lp = inputs.normal_values((3, 60), seed=9), inputs.normal_values((3, 60), seed=10)

    def obj(u, p):
        f = opm.force(u, mass, n, L, OM)
        u1, p1, _ = opm.kdk_step(u, p, f, coeffs, mass, n, L, OM)
        x1 = opm.decode(u1, L)
        return float((lx * x1).sum() + (lp * p1).sum())
    gx, gp = oad.kdk_step_vjp(u0, p0, f0, coeffs, lx, lp, mass, n, L, OM)
    eps = 1e-3   # moves x1 by ~3e4 fixed-point quanta: the drift's rounding stays negligible
    for i in (0, 31):
        for d in range(3):
            pp, pm_ = p0.copy(), p0.copy()
            pp[d, i] += eps
            pm_[d, i] -= eps
            fd = (obj(u0, pp) - obj(u0, pm_)) / (2 * eps)
            assert fd == pytest.approx(gp[d, i], rel=1e-4)
            k = 1 << 20   # 4e-3 cells: the drift's rounding of the force change stays negligible
            dx = k * L / 2 ** 32
            fdx = (obj(_shift(u0, i, d, k), p0) - obj(_shift(u0, i, d, -k), p0)) / (2 * dx)
            assert fdx == pytest.approx(gx[d, i], rel=1e-4, abs=1e-5 * np.abs(gx).max())


def test_ic_transpose_dot_product():
    nc, L = 16, 64.0
    pk = oic.linear_power(0.31, 0.68, 0.965, 0.81)
    om = inputs.normal_values((nc, nc, nc), seed=11)
    lam_c = inputs.normal_values((3, nc ** 3), seed=12)
    ns = 4
    lam_n = inputs.normal_values((3, ns ** 3), seed=13)
    kfs = 0.2
    grad = oad.ic_vjp(lam_c, lam_n, L, pk, n_sites=ns, k_fs=kfs, nc=nc)
    s = oic.displacement(oic.delta_k(om, L, pk), L).reshape(3, -1)
    r, j0, sh = oic.neutrino_site_offset(nc, ns)
    sn = oic.displacement(oic.delta_k(om, L, pk), L, shift=sh * L / nc, k_fs=kfs)
    idx = (j0 + r * np.arange(ns)) % nc
    sn = sn[:, idx][:, :, idx][:, :, :, idx].reshape(3, -1)
    lhs = (lam_c * s).sum() + (lam_n * sn).sum()
    assert (grad * om).sum() == pytest.approx(lhs, rel=1e-11)


def test_reconstruction_gradient_finite_differences():
    from paper_2007_13394_gb300.pm import RunConfig
    cfg = RunConfig(box=64.0, nmesh=16, nc=8, nsites=2, nshell=2, nfib=1, m_nu=(0.2 / 3,) * 3)
    steps = obg.schedule_linear(0.05, 0.3, 2)
    rec = oad.Reconstruction(cfg, steps, a0=0.05)
    om = inputs.white_noise(8, seed=1).astype(np.float64)
    target = opm.paint(rec.forward(inputs.white_noise(8, seed=2).astype(np.float64))[0], rec.mass, 16)
    g = rec.grad(om, target)
    rng = np.random.default_rng(0)
    eps = 1e-4
    for _ in range(6):
        idx = tuple(rng.integers(0, 8, size=3))
        op, omn = om.copy(), om.copy()
        op[idx] += eps
        omn[idx] -= eps
        fd = (rec.loss(op, target) - rec.loss(omn, target)) / (2 * eps)
        assert fd == pytest.approx(g[idx], rel=2e-3, abs=1e-3 * np.abs(g).max())
