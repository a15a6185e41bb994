"""Pins of the FP64 learned-factor oracle (oracle/mlp.py): the network against torch's
own layers and autograd, central differences, closed forms of the factor's gradient,
the antisymmetry of the corrected gradient operator, and end-to-end differences of
the training loss through a short run."""
import numpy as np
import pytest

from oracle import adjoint as oad
from oracle import background as obg
from oracle import mlp as om
from oracle import pm as opm
from paper_2007_13394_gb300 import inputs
from paper_2007_13394_gb300.pm import RunConfig

torch = pytest.importorskip("torch")

OM0 = 0.31


def _theta(seed, last=1.0):
    return inputs.mlp_parameters(seed, last_scale=last).astype(np.float64)


def _torch_net(theta):
    W1, b1, W2, b2, w3, b3 = (torch.tensor(np.array(x), dtype=torch.float64, requires_grad=True)
                              for x in om.unpack(theta))
    return [W1, b1, W2, b2, w3, b3]


def test_layout_and_count():
    assert om.NPARAM == 4417
    th = _theta(0)
    back = om.pack(*om.unpack(th))
    assert np.array_equal(back, th)


def test_forward_and_vjp_match_torch_autograd():
    """Independent restatement with torch.nn.functional (linear, silu) and autograd."""
    th = _theta(1)
    rng = np.random.default_rng(2)
    kappa = rng.uniform(0, np.sqrt(3), size=257)
    a = 0.37
    gm = rng.standard_normal(kappa.size)
    P = _torch_net(th)
    x = torch.stack([torch.tensor(kappa), torch.full((kappa.size,), a, dtype=torch.float64)], dim=1)
    h = torch.nn.functional.silu(torch.nn.functional.linear(x, P[0], P[1]))
    h = torch.nn.functional.silu(torch.nn.functional.linear(h, P[2], P[3]))
    m = 1.0 + h @ P[4] + P[5]
    np.testing.assert_allclose(om.forward(th, kappa, a), m.detach().numpy(), rtol=1e-13, atol=1e-13)
    (m * torch.tensor(gm)).sum().backward()
    ref = om.pack(*[p.grad.numpy() for p in P])
    np.testing.assert_allclose(om.vjp(th, kappa, a, gm), ref, rtol=1e-11, atol=1e-12)


def test_silu_derivative_and_vjp_central_differences():
    z = np.linspace(-6, 6, 101)
    eps = 1e-6
    np.testing.assert_allclose(om.dsilu(z), (om.silu(z + eps) - om.silu(z - eps)) / (2 * eps), rtol=1e-8,
                               atol=1e-10)
    th = _theta(3)
    rng = np.random.default_rng(4)
    kappa = rng.uniform(0, 1.7, size=50)
    gm = rng.standard_normal(50)
    g = om.vjp(th, kappa, 0.8, gm)
    for _ in range(4):
        v = rng.standard_normal(th.size)
        fd = ((om.forward(th + eps * v, kappa, 0.8) - om.forward(th - eps * v, kappa, 0.8)) @ gm) / (2 * eps)
        assert fd == pytest.approx(g @ v, rel=1e-7)


def test_zero_last_layer_is_the_plain_kernel_exactly():
    th = _theta(5, last=0.0)
    assert np.all(om.factor_mesh(th, 16, 0.5) == 1.0)
    u = inputs.uniform_positions(300, seed=6)
    m = inputs.uniform_masses(300, seed=7)
    assert np.array_equal(om.force(u, m, 16, 50.0, OM0, th, 0.5), opm.force(u, m, 16, 50.0, OM0))


def test_constant_factor_scales_the_force():
    """w3 = 0, b3 = c - 1 gives m = c everywhere, so F = c F_plain (linearity in phi)."""
    th = _theta(8, last=0.0)
    th[-1] = 0.75 - 1.0
    u = inputs.uniform_positions(200, seed=9)
    m = inputs.uniform_masses(200, seed=10)
    np.testing.assert_allclose(om.force(u, m, 16, 40.0, OM0, th, 0.3), 0.75 * opm.force(u, m, 16, 40.0, OM0),
                               rtol=1e-12, atol=1e-14)


def test_bias_gradient_is_the_plain_force_projection():
    """dm/db3 = 1, so d<lam, F>/db3 = <lam, F_plain> whatever theta is: pins the mode sum,
    its r2c multiplicities and the sign of d<lam, F>/dm."""
    th = _theta(11)
    u = inputs.uniform_positions(400, seed=12)
    m = inputs.uniform_masses(400, seed=13)
    lam = inputs.normal_values((3, 400), seed=14)
    g = om.force_theta_vjp(u, m, lam, 16, 30.0, OM0, th, 0.6)
    ref = float((lam * opm.force(u, m, 16, 30.0, OM0)).sum())
    assert g[-1] == pytest.approx(ref, rel=1e-11)


def test_force_theta_vjp_central_differences():
    th = _theta(15)
    u = inputs.uniform_positions(300, seed=16)
    m = inputs.uniform_masses(300, seed=17)
    lam = inputs.normal_values((3, 300), seed=18)
    g = om.force_theta_vjp(u, m, lam, 16, 30.0, OM0, th, 0.45)
    rng = np.random.default_rng(19)
    eps = 1e-5
    for _ in range(3):
        v = rng.standard_normal(th.size)
        fp = (lam * om.force(u, m, 16, 30.0, OM0, th + eps * v, 0.45)).sum()
        fm = (lam * om.force(u, m, 16, 30.0, OM0, th - eps * v, 0.45)).sum()
        assert (fp - fm) / (2 * eps) == pytest.approx(g @ v, rel=1e-7)


def test_corrected_gradient_operator_stays_antisymmetric():
    """m is real and even in k, so G_j with the factor is still odd: <X, G_j Y> = -<G_j X, Y>."""
    th = _theta(20)
    n, box = 16, 25.0
    kf = om.factor_mesh(th, n, 0.7)
    X = inputs.normal_values((n, n, n), seed=21)
    Y = inputs.normal_values((n, n, n), seed=22)
    for j in range(3):
        gy = opm.force_mesh(opm.potential_k(Y, box, OM0, kf), box, n, j)
        gx = opm.force_mesh(opm.potential_k(X, box, OM0, kf), box, n, j)
        a, b = (X * gy).sum(), (gx * Y).sum()
        assert a == pytest.approx(-b, rel=1e-10, abs=1e-12 * np.abs(X * gy).sum())


def test_wrapped_displacement_and_loss_cotangent():
    box = 10.0
    u = np.array([[2 ** 32 - 10, 5, 2 ** 31], [0, 0, 0], [7, 7, 7]], dtype=np.uint32)
    v = np.array([[5, 2 ** 32 - 10, 0], [0, 0, 0], [7, 7, 7]], dtype=np.uint32)
    d = om.wrapped_displacement(u, v, box)
    q = box / 2 ** 32
    assert d[0, 0] == pytest.approx(-15 * q) and d[0, 1] == pytest.approx(15 * q)
    assert d[0, 2] == pytest.approx(-box / 2)     # 2^31 apart wraps to -L/2
    m = np.array([1.0, 2.0, 3.0])
    L, lam = om.displacement_loss(u, v, m, box)
    assert L == pytest.approx(((d ** 2).sum(0) * m).sum() / 6.0)
    np.testing.assert_allclose(lam, 2 * m * d / 6.0)


def test_training_gradient_central_differences_through_a_run():
    """dL/dtheta of the displacement loss through three learned KDK steps (ICs, forces,
    drifts, the factor at each force's scale factor) against central differences."""
    cfg = RunConfig(box=32.0, nmesh=16, nc=8, nsites=2, nshell=2, nfib=1, m_nu=(0.1, 0.1, 0.1))
    steps = obg.schedule_linear(0.1, 0.4, 3)
    a0 = steps[0][0]
    run = om.LearnedRun(cfg, steps, a0)
    noise = 3.0 * inputs.white_noise(8, seed=1).astype(np.float64)
    target = oad.Reconstruction(cfg, obg.schedule_linear(0.1, 0.4, 8), a0).forward(noise)[0]
    th = _theta(3)
    L, g = run.grad(noise, th, target)
    assert L == pytest.approx(run.loss(noise, th, target), rel=1e-14)
    rng = np.random.default_rng(0)
    eps = 3e-5
    for _ in range(3):
        v = rng.standard_normal(th.size)
        fd = (run.loss(noise, th + eps * v, target) - run.loss(noise, th - eps * v, target)) / (2 * eps)
        assert fd == pytest.approx(g @ v, rel=5e-4)


def test_adam_matches_torch_optimizer():
    th = _theta(30)
    rng = np.random.default_rng(31)
    p = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.8, 0.99), eps=1e-7)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    x = th.copy()
    for t in range(1, 6):
        g = rng.standard_normal(th.size)
        opt.zero_grad()
        p.grad = torch.tensor(g)
        opt.step()
        x, m, v = om.adam_step(x, g, m, v, t, lr=3e-3, beta1=0.8, beta2=0.99, eps=1e-7)
    np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_power_vjp_central_differences():
    """Gradient of a spectrum-matching loss with respect to particle positions against
    central differences of the estimator itself (positions moved far less than a cell,
    so no particle crosses a cell face)."""
    n, L = 16, 40.0
    rng = np.random.default_rng(40)
    x = rng.uniform(0, L, size=(3, 600))
    m = inputs.uniform_masses(600, seed=41)
    nb = 10
    p_ref = np.linspace(5.0, 1.0, nb) * 1e3
    bins = range(1, 8)
    u = opm.quantise(x, L)
    xq = opm.decode(u, L)
    L0, g_P = om.power_loss(u, m, n, L, nb, p_ref, bins)
    g = om.power_vjp(u, m, n, L, nb, g_P)
    eps = 1e-4
    frac = np.stack([opm.cell_and_fraction(u[d], n)[1] for d in range(3)])
    near_node = np.minimum(frac, 1 - frac) < 1e-3    # a step of eps would cross the CIC kink
    for _ in range(3):
        v = np.where(near_node, 0.0, rng.standard_normal(x.shape))
        lp = om.power_loss(opm.quantise(xq + eps * v, L), m, n, L, nb, p_ref, bins)[0]
        lm = om.power_loss(opm.quantise(xq - eps * v, L), m, n, L, nb, p_ref, bins)[0]
        assert (lp - lm) / (2 * eps) == pytest.approx((g * v).sum(), rel=2e-4)
    assert L0 > 0


def test_power_vjp_single_mode_closed_form():
    """Weight dL/dP only on the bin of one plane-wave density mode: the cotangent mesh is
    2 c F_k e^{ikx} + c.c., so the position gradient of sum_b w_b P_b equals the direct
    derivative of the closed-form P of the displaced lattice's mode (cross-checked by the
    power spectrum's own value change)."""
    n, L = 16, 16.0
    ax = (np.arange(n) + 0.5) * (L / n)
    grid = np.meshgrid(ax, ax, ax, indexing="ij")
    q = np.stack([gg.ravel() for gg in grid])
    k = 2 * np.pi * 2 / L
    A = 1e-3
    x = q.copy()
    x[0] += A * np.sin(k * q[0])
    u = opm.quantise(x, L)
    nb = 4
    g_P = np.zeros(nb)
    g_P[1] = 1.0                           # bin of |n| = 2
    g = om.power_vjp(u, 1.0, n, L, nb, g_P)
    # moving every particle along the mode's own displacement changes A -> A (1 + t):
    # P ~ A^2 near A = 0, so dP/dt = 2 P
    _, P, _ = opm.power_spectrum(opm.paint(u, 1.0, n), None, L, nb)
    d = (opm.decode(u[0], L) - q[0] + L / 2) % L - L / 2
    v = np.zeros_like(x)
    v[0] = d
    assert (g * v).sum() == pytest.approx(2 * P[1], rel=1e-4)
