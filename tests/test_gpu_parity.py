"""GPU parity: each stage of the CUDA path through the C-ABI against the FP64 oracle.

Tolerances: integer work (sort keys, permutation) bit-exact; FP32 mesh and FFT
work relative to the field's scale at the FP32 level (1e-6 .. 1e-5); the force
relative RMS < 1e-5; P(k) per bin < 1e-3 for k < k_Ny / 2.
"""
import numpy as np
import pytest

from oracle import background as obg
from oracle import ic as oic
from oracle import neutrinos as onu
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


def make_cfg(pm, nmesh=64, nc=32, nsites=8, box=128.0, nshell=4, nfib=1, m_nu=(0.2 / 3,) * 3, n_max=0,
             flags=0):
    return pm.RunConfig(box=box, nmesh=nmesh, nc=nc, nsites=nsites, nshell=nshell, nfib=nfib,
                        m_nu=m_nu, n_max=n_max, flags=flags)


def oracle_setup(cfg, a0=0.05, seed=1, kfs=0.0):
    """Oracle ICs (positions, momenta, masses) and background for a config."""
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    noise = inputs.white_noise(cfg.nc, seed=seed).astype(np.float64)
    plin = oic.linear_power(cfg.omega_m, cfg.h, cfg.ns, cfg.sigma8)
    uc, pc = oic.cdm_particles(noise, cfg.box, plin, bg.D(a0), bg.gp(a0))
    mm = max(cfg.m_nu)
    if cfg.nsites:
        _, q, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
        pscale = onu.thermal_momentum_scale(bg.kT_nu0, mm) if mm > 0 else 0.0
        un, pn = oic.neutrino_particles(noise, cfg.box, plin, bg.D(a0), bg.gp(a0), cfg.nsites, cfg.nshell,
                                        cfg.nfib, q, p_scale=pscale, k_fs=kfs)
    else:
        m_shell = np.zeros(0)
        un, pn = np.zeros((3, 0), np.uint32), np.zeros((3, 0))
    mc, mn = onu.species_masses(cfg.nmesh, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                                bg.omega_nu_poisson, m_shell)
    mass = onu.particle_masses(uc.shape[1], un.shape[1], cfg.nshell, cfg.nfib, mc, mn)
    return dict(bg=bg, u=np.hstack([uc, un]), p=np.hstack([pc, pn]), mass=mass, noise=noise,
                n_cdm=uc.shape[1])


# ------------------------------------------------------------------- sort
@pytest.mark.parametrize("n", [1, 4095, 4096, 70001])
def test_sort_bit_exact_uniform(pm, n):
    cfg = make_cfg(pm, nmesh=64, n_max=70001)
    ctx = pm.ParticleMesh(cfg)
    u = inputs.uniform_positions(n, seed=n)
    perm, keys = ctx.sort(pm.as_u32_tensor(u))
    ctx.sync()
    np.testing.assert_array_equal(pm.to_u32(keys), np.sort(opm.sort_keys(u, 64)).astype(np.uint32))
    np.testing.assert_array_equal(pm.to_u32(perm), opm.sort_permutation(u, 64).astype(np.uint32))


def test_sort_bit_exact_clustered_and_face_classes(pm):
    cfg = make_cfg(pm, nmesh=128, n_max=200000)
    ctx = pm.ParticleMesh(cfg)
    rng = np.random.default_rng(7)
    n = 200000
    # half the particles in a few cells (many equal keys), many on tile faces
    u = inputs.uniform_positions(n, seed=3)
    cells = rng.integers(0, 128, size=(3, n // 2))
    cells[:, : n // 4] = (cells[:, : n // 4] // 16) * 16 + 15          # on the high face layer
    u[:, : n // 2] = (cells.astype(np.uint64) * (2 ** 32 // 128) + rng.integers(0, 2 ** 25, size=(3, n // 2))
                      ).astype(np.uint32)
    perm, keys = ctx.sort(pm.as_u32_tensor(u))
    ctx.sync()
    np.testing.assert_array_equal(pm.to_u32(perm), opm.sort_permutation(u, 128).astype(np.uint32))


def test_sort_2048_mesh_keys(pm):
    # keys at the largest mesh use 24 bits (three radix passes); small n
    cfg = make_cfg(pm, nmesh=2048, nc=0, nsites=0, n_max=50000)
    ctx = pm.ParticleMesh(cfg)
    u = inputs.uniform_positions(50000, seed=11)
    perm, keys = ctx.sort(pm.as_u32_tensor(u))
    ctx.sync()
    np.testing.assert_array_equal(pm.to_u32(perm), opm.sort_permutation(u, 2048).astype(np.uint32))


# ------------------------------------------------------------------ paint
def test_paint_matches_oracle_and_is_deterministic(pm):
    cfg = make_cfg(pm)
    o = oracle_setup(cfg)
    ctx = pm.ParticleMesh(cfg)
    ud = pm.as_u32_tensor(o["u"])
    m1 = ctx.paint(ud).cpu().numpy()
    m2 = ctx.paint(ud).cpu().numpy()
    ctx.sync()
    ref = opm.paint(o["u"], o["mass"], cfg.nmesh)
    assert np.array_equal(m1, m2)                          # bitwise reproducible
    np.testing.assert_allclose(m1, ref, rtol=2e-6, atol=2e-6 * ref.max())
    assert m1.astype(np.float64).sum() == pytest.approx(cfg.nmesh ** 3, rel=1e-6)   # mean 1


@pytest.mark.parametrize("species", [1, 2])
def test_paint_species_selection(pm, species):
    cfg = make_cfg(pm)
    o = oracle_setup(cfg)
    ctx = pm.ParticleMesh(cfg)
    m = ctx.paint(pm.as_u32_tensor(o["u"]), species=species).cpu().numpy()
    ctx.sync()
    sel = np.arange(o["u"].shape[1]) < o["n_cdm"]
    if species == 2:
        sel = ~sel
    ref = opm.paint(o["u"][:, sel], o["mass"][sel], cfg.nmesh)
    np.testing.assert_allclose(m, ref, rtol=2e-6, atol=2e-6 * ref.max())


def test_paint_uniform_random_and_empty(pm):
    cfg = make_cfg(pm, nmesh=128, n_max=300000)
    ctx = pm.ParticleMesh(cfg)
    n = 300000
    u = inputs.uniform_positions(n, seed=5)
    ids = np.arange(n, dtype=np.uint32) % (cfg.n_particles())
    m = ctx.paint(pm.as_u32_tensor(u), pm.as_u32_tensor(ids)).cpu().numpy()
    mass = np.where(ids < cfg.n_cdm(), 0, 0)  # placeholder replaced below
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    _, _, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
    mc, mn = onu.species_masses(128, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                                bg.omega_nu_poisson, m_shell)
    table = onu.particle_masses(cfg.n_cdm(), cfg.n_nu(), cfg.nshell, cfg.nfib, mc, mn)
    mass = table[ids]
    ref = opm.paint(u, mass, 128)
    np.testing.assert_allclose(m, ref, rtol=2e-6, atol=2e-6 * ref.max())
    empty = ctx.paint(pm.as_u32_tensor(np.zeros((3, 0), np.uint32))).cpu().numpy()
    ctx.sync()
    assert not empty.any()


def test_paint_clustered_tiles(pm):
    """Most particles in a few cells and on tile faces: tiles far above one chunk of the
    paint's per-tile staging, columns with thousands of particles, halo classes."""
    cfg = make_cfg(pm, nmesh=128, n_max=300000)
    ctx = pm.ParticleMesh(cfg)
    rng = np.random.default_rng(12)
    n = 300000
    u = inputs.uniform_positions(n, seed=13)
    cells = rng.integers(0, 8, size=(3, 2 * n // 3)) * 16 + rng.integers(14, 16, size=(3, 2 * n // 3))
    u[:, : 2 * n // 3] = (cells.astype(np.uint64) * (2 ** 32 // 128)
                          + rng.integers(0, 2 ** 25, size=(3, 2 * n // 3))).astype(np.uint32)
    ids = np.arange(n, dtype=np.uint32) % cfg.n_cdm()
    m = ctx.paint(pm.as_u32_tensor(u), pm.as_u32_tensor(ids)).cpu().numpy()
    m2 = ctx.paint(pm.as_u32_tensor(u), pm.as_u32_tensor(ids)).cpu().numpy()
    ctx.sync()
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    _, _, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
    mc, _ = onu.species_masses(128, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                               bg.omega_nu_poisson, m_shell)
    ref = opm.paint(u, np.full(n, mc), 128)
    assert np.array_equal(m, m2)
    np.testing.assert_allclose(m, ref, rtol=2e-6, atol=2e-6 * ref.max())


@pytest.mark.parametrize("cell", [(80, 48, 48), (79, 47, 47), (5, 6, 7)], ids=["tile_origin", "tile_corner", "interior"])
def test_paint_dense_cells_that_wrap_32_bit_words(pm, cell):
    """Cells above 256 mean cell masses wrap the paint's 32-bit fixed-point words: such tiles
    are repainted whole in the carry form.  A cell with 100 (no wrap), 300 and 1000 particles
    (one to four wraps in each of the 8 cells around it), at a tile's origin, at a tile's far
    corner (its 8 CIC cells in 8 tiles) and inside a tile: the whole mesh against the
    oracle, on meshes reused between calls (a tile left unwritten would show stale values)."""
    cfg = make_cfg(pm, nmesh=256, nc=128, nsites=0, box=256.0, m_nu=(0.0, 0.0, 0.0), n_max=4000)
    ctx = pm.ParticleMesh(cfg)
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    mc, _ = onu.species_masses(256, 128, 0, cfg.nshell, cfg.nfib, bg.omega_c, bg.omega_nu_poisson, np.zeros(0))
    rng = np.random.default_rng(sum(cell))
    for count in (100, 300, 1000, 300):
        u = np.empty((3, count), np.uint32)
        for d in range(3):
            u[d] = (cell[d] * (2 ** 32 // 256) + rng.integers(0, 2 ** 32 // 256, count)).astype(np.uint32)
        m = ctx.paint(pm.as_u32_tensor(u)).cpu().numpy()
        ctx.sync()
        ref = opm.paint(u, np.full(count, mc), 256)
        assert ref.max() > 256 or count == 100
        np.testing.assert_allclose(m, ref, rtol=2e-6, atol=2e-6 * ref.max())


def test_paint_rejects_unknown_ids(pm):
    cfg = make_cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    u = inputs.uniform_positions(10, seed=1)
    ids = np.full(10, 10 ** 9, dtype=np.uint32)
    ctx.paint(pm.as_u32_tensor(u), pm.as_u32_tensor(ids))
    with pytest.raises(pm.PMError) as ei:
        ctx.sync()
    assert ei.value.status == pm.PM_EKERNEL
    ctx.sync()                         # the error word is cleared once reported


# -------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_fft_r2c_c2r_match_numpy(pm, n):
    cfg = make_cfg(pm, nmesh=n, nc=0, nsites=0)
    ctx = pm.ParticleMesh(cfg)
    x = inputs.normal_values((n, n, n), seed=n).astype(np.float32)
    X = ctx.fft_r2c(torch.from_numpy(x).cuda()).cpu().numpy()
    Xc = X[..., 0] + 1j * X[..., 1]
    ref = np.fft.rfftn(x.astype(np.float64))
    err = np.abs(Xc - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
    y = ctx.fft_c2r(torch.from_numpy(X).cuda()).cpu().numpy()
    ctx.sync()
    yref = np.fft.irfftn(Xc, s=(n, n, n), axes=(0, 1, 2)) * n ** 3
    err2 = np.abs(y - yref).max() / np.abs(yref).max()
    assert err2 < 2e-6, err2


def test_potential_and_force_mesh_match_oracle(pm):
    cfg = make_cfg(pm)
    o = oracle_setup(cfg)
    ctx = pm.ParticleMesh(cfg)
    rho = opm.paint(o["u"], o["mass"], cfg.nmesh)
    phi = ctx.potential(torch.from_numpy(rho.astype(np.float32)).cuda())
    pc = phi.cpu().numpy()
    phic = pc[..., 0] + 1j * pc[..., 1]
    ref = opm.potential_k(rho, cfg.box, o["bg"].omega_m0)
    assert np.abs(phic - ref).max() / np.abs(ref).max() < 5e-6
    for j in range(3):
        Fm = ctx.force_mesh(phi, j).cpu().numpy()
        Fr = opm.force_mesh(ref, cfg.box, cfg.nmesh, j)
        assert np.abs(Fm - Fr).max() / np.abs(Fr).max() < 5e-6
    ctx.sync()


def test_readout_matches_oracle(pm):
    cfg = make_cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    u = inputs.uniform_positions(50000, seed=9)
    M = inputs.normal_values((64, 64, 64), seed=2).astype(np.float32)
    r = ctx.readout(pm.as_u32_tensor(u), torch.from_numpy(M).cuda()).cpu().numpy()
    ctx.sync()
    ref = opm.readout(u, M.astype(np.float64), 64)
    np.testing.assert_allclose(r, ref, rtol=1e-5, atol=1e-6)


# ------------------------------------------------------------------ force
@pytest.mark.parametrize("flags", [0, 8, 9, 2, 3], ids=["stencil", "kspace_fused_x", "kspace_per_component",
                                                        "spectral_fused_x", "spectral_per_component"])
@pytest.mark.parametrize("size", ["mesh32", "cfg1", "cfg2_parity"])
def test_force_relative_rms_below_1e5(pm, size, flags):
    if size == "mesh32":  # two tiles per side: the stencil halo wraps across the whole mesh
        cfg = make_cfg(pm, nmesh=32, nc=16, nsites=4, box=128.0, nshell=4, nfib=1, flags=flags)
    elif size == "cfg1":
        cfg = make_cfg(pm, nmesh=64, nc=32, nsites=8, box=256.0, nshell=10, nfib=3, flags=flags)
    else:
        cfg = make_cfg(pm, nmesh=256, nc=128, nsites=16, box=256.0, nshell=10, nfib=3, m_nu=(0.1 / 3,) * 3,
                       flags=flags)
    o = oracle_setup(cfg)
    ctx = pm.ParticleMesh(cfg)
    F = ctx.force(pm.as_u32_tensor(o["u"])).cpu().numpy().astype(np.float64)
    ctx.sync()
    ref = opm.force(o["u"], o["mass"], cfg.nmesh, cfg.box, o["bg"].omega_m0,
                    kernel="spectral" if flags & 2 else "fd4")
    rel = np.sqrt(((F - ref) ** 2).sum() / (ref ** 2).sum())
    assert rel < 1e-5, rel


@pytest.mark.parametrize("flags", [0, 8], ids=["stencil", "kspace_fused_x"])
def test_force_clustered_tiles(pm, flags):
    """Force on particles packed into a few cells on tile faces (tiles holding tens of
    thousands of particles, runs of many CTA-strides in the stencil readout) against the
    oracle."""
    cfg = make_cfg(pm, nmesh=128, n_max=300000, flags=flags)
    ctx = pm.ParticleMesh(cfg)
    rng = np.random.default_rng(14)
    n = 300000
    u = inputs.uniform_positions(n, seed=15)
    k = 2 * n // 3
    cells = rng.integers(0, 8, size=(3, k)) * 16 + rng.integers(14, 16, size=(3, k))
    u[:, :k] = (cells.astype(np.uint64) * (2 ** 32 // 128) + rng.integers(0, 2 ** 25, size=(3, k))).astype(np.uint32)
    ids = np.arange(n, dtype=np.uint32) % cfg.n_cdm()
    F = ctx.force(pm.as_u32_tensor(u), pm.as_u32_tensor(ids)).cpu().numpy().astype(np.float64)
    ctx.sync()
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    _, _, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
    mc, _ = onu.species_masses(128, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                               bg.omega_nu_poisson, m_shell)
    ref = opm.force(u, np.full(n, mc), 128, cfg.box, bg.omega_m0)
    rel = np.sqrt(((F - ref) ** 2).sum() / (ref ** 2).sum())
    assert rel < 1e-5, rel


def test_force_conserves_momentum(pm):
    cfg = make_cfg(pm, nmesh=128, n_max=100000)
    ctx = pm.ParticleMesh(cfg)
    n = 100000
    u = inputs.uniform_positions(n, seed=4)
    ids = (np.arange(n) % cfg.n_cdm()).astype(np.uint32)     # all CDM: equal masses
    F = ctx.force(pm.as_u32_tensor(u), pm.as_u32_tensor(ids)).cpu().numpy().astype(np.float64)
    ctx.sync()
    assert np.abs(F.sum(axis=1)).max() < 1e-5 * np.abs(F).sum(axis=1).max()


# -------------------------------------------------------------------- step
@pytest.mark.parametrize("flags", [0, 8, 9], ids=["stencil", "kspace_fused_x", "kspace_per_component"])
def test_step_matches_oracle(pm, flags):
    cfg = make_cfg(pm, nmesh=64, nc=32, nsites=8, box=256.0, nshell=10, nfib=3, flags=flags)
    a0, a1 = 0.05, 0.07
    o = oracle_setup(cfg, a0=a0)
    ctx = pm.ParticleMesh(cfg)
    st = ctx.new_state(o["u"].shape[1])
    st["u"].copy_(pm.as_u32_tensor(o["u"]))
    st["p"].copy_(torch.from_numpy(o["p"].astype(np.float32)))
    st["id"].copy_(torch.arange(o["u"].shape[1], dtype=torch.int32))
    ah = 0.5 * (a0 + a1)
    ctx.step(st, a0, ah, a1)
    ctx.sync()
    ids = pm.to_u32(st["id"])
    assert np.array_equal(np.sort(ids), np.arange(len(ids)))
    u_gpu = np.empty_like(o["u"])
    u_gpu[:, ids] = pm.to_u32(st["u"])
    p_gpu = np.empty_like(o["p"])
    p_gpu[:, ids] = st["p"].cpu().numpy()
    f_gpu = np.empty_like(o["p"])
    f_gpu[:, ids] = st["f"].cpu().numpy()
    bg = o["bg"]
    f0 = opm.force(o["u"], o["mass"], cfg.nmesh, cfg.box, bg.omega_m0)
    u1, p1, f1 = opm.kdk_step(o["u"], o["p"], f0, obg.step_coefficients(bg, a0, ah, a1), o["mass"],
                              cfg.nmesh, cfg.box, bg.omega_m0)
    wrap = lambda d: ((d + 2 ** 31) % 2 ** 32) - 2 ** 31
    du = wrap(u_gpu.astype(np.int64) - u1.astype(np.int64))
    moved = wrap(u1.astype(np.int64) - o["u"].astype(np.int64))
    # FP32 momenta and drift product: error relative to this step's displacement, in quanta
    assert np.all(np.abs(du) <= 64 + 4e-6 * np.abs(moved)), np.abs(du).max()
    assert np.sqrt(((p_gpu - p1) ** 2).sum() / (p1 ** 2).sum()) < 1e-5
    assert np.sqrt(((f_gpu - f1) ** 2).sum() / (f1 ** 2).sum()) < 1e-5
    # the state is now in tile order: the sort of the stored positions is the identity
    perm, _ = ctx.sort(st["u"])
    ctx.sync()
    assert np.array_equal(pm.to_u32(perm), np.arange(len(ids), dtype=np.uint32))


# ------------------------------------------------------------------- power
@pytest.mark.parametrize("pair", [(3, 3), (1, 1), (1, 2), (2, 2)])
def test_power_matches_oracle(pm, pair):
    cfg = make_cfg(pm, nmesh=64, nc=32, nsites=8, box=256.0, nshell=10, nfib=3)
    o = oracle_setup(cfg, a0=0.5)
    ctx = pm.ParticleMesh(cfg)
    nb = 20
    k, P, nm = ctx.power(pm.as_u32_tensor(o["u"]), species_a=pair[0], species_b=pair[1], nbins=nb)
    ctx.sync()
    sel = {1: np.arange(o["u"].shape[1]) < o["n_cdm"], 2: np.arange(o["u"].shape[1]) >= o["n_cdm"],
           3: np.ones(o["u"].shape[1], bool)}
    meshes = {s: opm.paint(o["u"], np.where(sel[s], o["mass"], 0.0), 64) for s in set(pair)}
    ka, Pa, na = opm.power_spectrum(meshes[pair[0]], meshes[pair[1]], cfg.box, nb)
    np.testing.assert_array_equal(nm, na)
    ok = na > 0
    np.testing.assert_allclose(k[ok], ka[ok], rtol=1e-12)
    kny = np.pi * 64 / cfg.box
    sel_k = ok & (ka < kny / 2)
    np.testing.assert_allclose(P[sel_k], Pa[sel_k], rtol=1e-3)


# --------------------------------------------------------------- edge cases
def test_invalid_arguments_fail_loudly(pm):
    cfg = make_cfg(pm)
    ctx = pm.ParticleMesh(cfg)
    u = inputs.uniform_positions(10, seed=1)
    with pytest.raises(pm.PMError):
        ctx.power(pm.as_u32_tensor(u), nbins=0)
    st = ctx.new_state(10)
    with pytest.raises(pm.PMError):
        ctx.step(st, 0.5, 0.4, 0.3)
    with pytest.raises(pm.PMError):
        pm.ParticleMesh(make_cfg(pm, nmesh=96))


def test_fft_2048_plane_wave_closed_form(pm):
    """The 2048^3 transforms (per-component force path, 16.8 MB-strided x lines) on one plane
    wave cos(2 pi n.x / N + phi) with all three n_d nonzero: r2c is N^3/2 e^{i phi} at n and
    zero elsewhere (sampled), c2r of it is N^3 times the wave (sampled planes)."""
    import math
    N = 2048
    cfg = make_cfg(pm, nmesh=N, nc=0, nsites=0, n_max=16)
    ctx = pm.ParticleMesh(cfg)
    nv, phi = (3, 5, 7), 0.3
    ax = torch.arange(N, device="cuda", dtype=torch.float64)
    px, py, pz = (2 * math.pi * nv[d] * ax / N for d in range(3))
    mesh = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    for x in range(N):
        mesh[x] = torch.cos(px[x] + py[:, None] + pz[None, :] + phi).float()
    out = ctx.fft_r2c(mesh)
    ctx.sync()
    half = N ** 3 / 2
    v = out[nv[0], nv[1], nv[2]].double().cpu().numpy()
    assert v[0] == pytest.approx(half * math.cos(phi), rel=1e-5)
    assert v[1] == pytest.approx(half * math.sin(phi), rel=1e-5)
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j, k = int(rng.integers(0, N)), int(rng.integers(0, N)), int(rng.integers(0, N // 2 + 1))
        if (i, j, k) == nv:
            continue
        w = out[i, j, k].double().cpu().numpy()
        assert np.abs(w).max() < 1e-5 * half
    back = ctx.fft_c2r(out)
    ctx.sync()
    for x in (0, 1, 777, N - 1):
        ref = (N ** 3) * torch.cos(px[x] + py[:, None] + pz[None, :] + phi)
        err = (back[x].double() - ref).abs().max().item()
        assert err < 1e-5 * N ** 3, (x, err)


@pytest.mark.parametrize("N", [512, 1024, 2048])
def test_fft_random_rows_match_numpy(pm, N):
    """Random data on three z rows (i_r, j_r) of an otherwise empty N^3 mesh, N up to the
    2048-point rows of the scale run: the r2c transform is, by linearity and the shift
    theorem, sum_r e^{-2 pi i (k_x i_r + k_y j_r) / N} rfft(row_r)(k_z) -- every k_z mode of
    each row's real transform, checked on whole (k_x, k_y) lines and sampled modes -- and
    c2r of it is N^3 times the input (the rows, and zero elsewhere on sampled planes)."""
    cfg = make_cfg(pm, nmesh=N, nc=0, nsites=0, n_max=16)
    ctx = pm.ParticleMesh(cfg)
    rows = ((0, 0), (5, N - 3), (N // 2 + 1, 17))
    data = inputs.normal_values((len(rows), N), seed=N + 7).astype(np.float32)
    mesh = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    for (i, j), r in zip(rows, data):
        mesh[i, j] = torch.from_numpy(r).cuda()
    out = ctx.fft_r2c(mesh)
    ctx.sync()
    R = np.fft.rfft(data.astype(np.float64), axis=1)          # (rows, N/2 + 1)
    scale = np.abs(R).max() * len(rows)

    def expected(kx, ky):
        ph = np.array([np.exp(-2j * np.pi * (kx * i + ky * j) / N) for i, j in rows])
        return (ph[:, None] * R).sum(axis=0)

    rng = np.random.default_rng(N)
    lines = [(0, 0), (1, 0), (0, N - 1), (N // 2, N // 2), (N - 1, 3)]
    lines += [(int(rng.integers(0, N)), int(rng.integers(0, N))) for _ in range(20)]
    for kx, ky in lines:
        got = out[kx, ky].double().cpu().numpy()
        err = np.abs(got[:, 0] + 1j * got[:, 1] - expected(kx, ky)).max() / scale
        assert err < 3e-6, (kx, ky, err)
    back = ctx.fft_c2r(out)
    ctx.sync()
    for (i, j), r in zip(rows, data):
        err = np.abs(back[i, j].double().cpu().numpy() / N ** 3 - r).max() / np.abs(data).max()
        assert err < 5e-6, (i, j, err)
    for x in (1, N // 3, N - 1):
        assert back[x].abs().max().item() < 5e-6 * N ** 3 * np.abs(data).max()


def test_force_2048_stencil_matches_kspace_path(pm):
    """At 2048^3 there is no oracle: the default force (potential x pass on the TMA kernel,
    stencil readout) against the k-space per-component path (classic kernels, three
    inverse transforms) on the same 2^21 particles; both are checked against the oracle
    at the smaller meshes above."""
    n = 1 << 21
    u = pm.as_u32_tensor(inputs.uniform_positions(n, seed=21))
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    F = {}
    for flags in (0, 9):
        cfg = make_cfg(pm, nmesh=2048, nc=128, nsites=0, box=1024.0, m_nu=(0.0, 0.0, 0.0), n_max=n,
                       flags=flags)
        ctx = pm.ParticleMesh(cfg)
        F[flags] = ctx.force(u, ids).double().cpu().numpy()
        ctx.sync()
        ctx.close()
    rel = np.sqrt(((F[0] - F[9]) ** 2).sum() / (F[9] ** 2).sum())
    assert rel < 1e-5, rel
