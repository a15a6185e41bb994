"""Learned Green's-function factor on the GPU against the FP64 oracle (oracle/mlp.py):
the network table, the corrected force on both force paths, the plain kernel at zero
last layer, the adjoint with the parameter gradient, the displacement loss, Adam, and
the training gradient through a short run."""
import numpy as np
import pytest

from oracle import adjoint as oad
from oracle import background as obg
from oracle import mlp as om
from oracle import pm as opm
from paper_2007_13394_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__ as g
    g.build()
    from paper_2007_13394_gb300 import pm as _pm
    return _pm


def _cfg(pm, **kw):
    base = dict(box=64.0, nmesh=64, nc=32, nsites=4, nshell=4, nfib=1, m_nu=(0.2 / 3,) * 3)
    base.update(kw)
    return pm.RunConfig(**base)


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def _theta(seed, last=0.5):
    return inputs.mlp_parameters(seed, last_scale=last)


def test_mlp_eval_and_table_match_oracle(pm):
    ctx = pm.ParticleMesh(_cfg(pm))
    th = _theta(1, last=1.0)
    ctx.set_mlp(th)
    assert np.array_equal(ctx.get_mlp(), th)
    rng = np.random.default_rng(2)
    kap = rng.uniform(0, np.sqrt(3), 4096).astype(np.float32)
    av = rng.uniform(0.01, 1.0, 4096).astype(np.float32)
    m = ctx.mlp_eval(torch.from_numpy(kap).cuda(), torch.from_numpy(av).cuda()).double().cpu().numpy()
    ctx.sync()
    ref = np.array([om.forward(th.astype(np.float64), kap[i:i + 1].astype(np.float64), float(av[i]))[0]
                    for i in range(kap.size)])
    np.testing.assert_allclose(m, ref, rtol=0, atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("flags", [0, 8, 9], ids=["stencil", "kspace_fused_x", "kspace_per_component"])
def test_learned_force_matches_oracle(pm, flags):
    cfg = _cfg(pm, flags=flags)
    ctx = pm.ParticleMesh(cfg)
    rec = oad.Reconstruction(cfg, [], 0.1)
    u, _ = rec.ics(inputs.white_noise(cfg.nc, seed=3).astype(np.float64))
    th = _theta(4)
    ctx.set_mlp(th)
    ctx.set_force_time(0.37)
    F = ctx.force(pm.as_u32_tensor(u), None).double().cpu().numpy()
    ctx.sync()
    ref = om.force(u, rec.mass, cfg.nmesh, cfg.box, rec.bg.omega_m0, th.astype(np.float64), 0.37)
    plain = opm.force(u, rec.mass, cfg.nmesh, cfg.box, rec.bg.omega_m0)
    assert _rel(ref, plain) > 3e-3          # the factor does something
    assert _rel(F, ref) < 1e-5


def test_zero_last_layer_is_bitwise_plain(pm):
    cfg = _cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    n = cfg.n_particles()
    u = pm.as_u32_tensor(inputs.uniform_positions(n, seed=5))
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    plain = ctx.force(u, ids).cpu().numpy()
    ctx.set_mlp(_theta(6, last=0.0))
    ctx.set_force_time(0.5)
    learned = ctx.force(u, ids).cpu().numpy()
    ctx.set_mlp(None)
    again = ctx.force(u, ids).cpu().numpy()
    ctx.sync()
    assert np.array_equal(plain, learned) and np.array_equal(plain, again)


def test_learned_force_vjp_and_parameter_gradient_match_oracle(pm):
    cfg = _cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    rec = oad.Reconstruction(cfg, [], 0.1)
    u, _ = rec.ics(inputs.white_noise(cfg.nc, seed=7).astype(np.float64))
    th = _theta(8).astype(np.float64)
    lam = inputs.normal_values((3, u.shape[1]), seed=9)
    ctx.set_mlp(th.astype(np.float32))
    ctx.set_force_time(0.6)
    ctx.mlp_grad(reset=True)
    g = ctx.force_vjp(pm.as_u32_tensor(u), None, torch.from_numpy(lam.astype(np.float32)).cuda())
    gt = ctx.mlp_grad(reset=True).double().cpu().numpy()
    ctx.sync()
    kf = om.factor_mesh(th, cfg.nmesh, 0.6)
    ref = oad.force_vjp(u, rec.mass, lam, cfg.nmesh, cfg.box, rec.bg.omega_m0, kf)
    assert _rel(g.double().cpu().numpy(), ref) < 1e-4
    ref_t = om.force_theta_vjp(u, rec.mass, lam, cfg.nmesh, cfg.box, rec.bg.omega_m0, th, 0.6)
    assert _rel(gt, ref_t) < 1e-4
    # b3 entry: <lam, F_plain> exactly in exact arithmetic
    assert gt[-1] == pytest.approx(ref_t[-1], rel=1e-4)


def test_displacement_loss_matches_oracle(pm):
    cfg = _cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    n = cfg.n_particles()
    rng = np.random.default_rng(10)
    ref_u = inputs.uniform_positions(n, seed=11)
    u = (ref_u.astype(np.int64) + rng.integers(-2 ** 28, 2 ** 28, size=ref_u.shape)).astype(np.uint32)
    # state in a shuffled order, reference in another
    o1, o2 = rng.permutation(n).astype(np.uint32), rng.permutation(n).astype(np.uint32)
    st = {"u": pm.as_u32_tensor(np.ascontiguousarray(u[:, o1])), "id": pm.as_u32_tensor(o1)}
    ref = {"u": pm.as_u32_tensor(np.ascontiguousarray(ref_u[:, o2])), "id": pm.as_u32_tensor(o2)}
    rec = oad.Reconstruction(cfg, [], 0.1)
    cdm_only = np.where(np.arange(n) < rec.n_cdm, rec.mass, 0.0)
    for species, mass in ((pm.SPECIES_ALL, rec.mass), (pm.SPECIES_CDM, cdm_only)):
        L, lam = ctx.displacement_loss(st, ref, species)
        L_ref, lam_ref = om.displacement_loss(u, ref_u, mass, cfg.box)
        assert L == pytest.approx(L_ref, rel=1e-6)
        assert _rel(lam.double().cpu().numpy(), lam_ref) < 1e-6


def test_adam_matches_oracle(pm):
    ctx = pm.ParticleMesh(_cfg(pm))
    th = _theta(12, last=1.0)
    ctx.set_mlp(th)
    x = th.astype(np.float64)
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    rng = np.random.default_rng(13)
    for t in range(1, 4):
        g = rng.standard_normal(x.size).astype(np.float32)
        ctx.mlp_adam(torch.from_numpy(g).cuda(), t, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-6)
        x, m, v = om.adam_step(x, g.astype(np.float64), m, v, t, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-6)
    np.testing.assert_allclose(ctx.get_mlp(), x, rtol=0, atol=1e-6)


def test_training_gradient_matches_oracle(pm):
    """dL/dtheta of the displacement loss through 3 learned KDK steps (GPU adjoint with
    the parameter gradient at every force) against the FP64 oracle; the target run (8
    plain steps) is the oracle's and is handed to both sides."""
    from paper_2007_13394_gb300 import learned
    cfg = _cfg(pm, box=64.0, nmesh=64, nc=32, nsites=4, nshell=4, nfib=1)
    steps = obg.schedule_linear(0.1, 0.4, 3)
    a0 = steps[0][0]
    noise = inputs.white_noise(cfg.nc, seed=14)
    target = oad.Reconstruction(cfg, obg.schedule_linear(0.1, 0.4, 8), a0).forward(noise.astype(np.float64))[0]
    th = _theta(15, last=0.3)
    ctx = pm.ParticleMesh(cfg)
    ctx.set_mlp(th)
    ctx.mlp_grad(reset=True)
    ref = {"u": pm.as_u32_tensor(target), "id": None}
    L = learned.loss_and_grad(ctx, torch.from_numpy(noise).cuda(), ref, steps, a0, species=pm.SPECIES_ALL)
    g = ctx.mlp_grad(reset=True).double().cpu().numpy()
    ctx.sync()
    run = om.LearnedRun(cfg, steps, a0)
    L_ref, g_ref = run.grad(noise.astype(np.float64), th.astype(np.float64), target)
    assert L == pytest.approx(L_ref, rel=1e-3)
    assert _rel(g, g_ref) < 2e-3


def test_power_vjp_matches_oracle(pm):
    cfg = _cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    rec = oad.Reconstruction(cfg, [], 0.1)
    u, _ = rec.ics(inputs.white_noise(cfg.nc, seed=20).astype(np.float64) * 30.0)
    nb = 20
    dL_dP = inputs.normal_values(nb, seed=21)
    rng = np.random.default_rng(22)
    order = rng.permutation(u.shape[1]).astype(np.uint32)         # input order != canonical
    g = ctx.power_vjp(pm.as_u32_tensor(np.ascontiguousarray(u[:, order])), pm.as_u32_tensor(order), dL_dP)
    ctx.sync()
    ref = om.power_vjp(u, rec.mass, cfg.nmesh, cfg.box, nb, dL_dP)[:, order]
    assert _rel(g.double().cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("nmesh", [64, 256])
def test_mlp_tables_fp32_and_tensor_core_match_oracle(pm, nmesh):
    """The |n|^2 table of the factor: FP32 (default) within 2e-6 of the FP64 network, the
    tensor-core form (tcgen05, BF16 operands, FP32 accumulation) within the BF16 bound,
    max error < 1 % of max |m - 1|."""
    th = _theta(21, last=1.0)
    th64 = th.astype(np.float64)
    ctx32 = pm.ParticleMesh(_cfg(pm, nmesh=nmesh))
    ctxtc = pm.ParticleMesh(_cfg(pm, nmesh=nmesh, flags=pm.FLAG_MLP_TENSOR))
    ctx32.set_mlp(th)
    ctxtc.set_mlp(th)
    for a in (0.05, 0.5, 1.0):
        t32 = ctx32.mlp_table(a).double().cpu().numpy()
        ttc = ctxtc.mlp_table(a).double().cpu().numpy()
        ctxtc.sync()
        s = np.arange(t32.size)
        ref = om.forward(th64, np.sqrt(s) / (nmesh / 2), a)
        scale = np.abs(ref - 1.0).max()
        assert np.abs(t32 - ref).max() < 2e-6 * max(1.0, np.abs(ref).max())
        err = np.abs(ttc - ref).max() / scale
        print(f"\nnmesh {nmesh} a {a}: tensor-core table max error / max|m-1| = {err:.2e}")
        assert err < 1e-2


def test_learned_force_with_tensor_core_table(pm):
    cfg = _cfg(pm, flags=pm.FLAG_MLP_TENSOR)
    ctx = pm.ParticleMesh(cfg)
    rec = oad.Reconstruction(cfg, [], 0.1)
    u, _ = rec.ics(inputs.white_noise(cfg.nc, seed=3).astype(np.float64))
    th = _theta(4)
    ctx.set_mlp(th)
    ctx.set_force_time(0.37)
    F = ctx.force(pm.as_u32_tensor(u), None).double().cpu().numpy()
    ctx.sync()
    ref = om.force(u, rec.mass, cfg.nmesh, cfg.box, rec.bg.omega_m0, th.astype(np.float64), 0.37)
    assert _rel(F, ref) < 3e-3
