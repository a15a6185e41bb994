"""The allocation-free spectrum entry point against the regular one.

pm_power_bin_noalloc serves callers that cannot allocate device memory (memory
pools or arenas that own the device, allocation-free graph replays): it keeps
its partial sums in a fixed file-scope device array instead of context
scratch.  Here it bins the half spectra of painted species meshes and must
reproduce pm_power on the same particles, on two calls in a row (the second
call reuses the array the first one left behind).  This file sorts last so a
run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

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


def test_noalloc_binning_matches_pm_power_twice(pm):
    from paper_2007_13394_gb300 import workloads
    cfg = workloads.cfg1()
    ctx = pm.ParticleMesh(cfg)
    noise = torch.from_numpy(inputs.white_noise(cfg.nc, seed=4)).cuda()
    st = ctx.ic(noise, 0.5, k_fs=0.0)
    u, ids = st["u"], st["id"]
    nb = 24
    spectra = {}
    for s in (pm.SPECIES_CDM, pm.SPECIES_ALL):
        spectra[s] = ctx.fft_r2c(ctx.paint(u, ids, species=s))
    for call in range(2):
        for (sa, sb) in ((pm.SPECIES_ALL, pm.SPECIES_ALL), (pm.SPECIES_CDM, pm.SPECIES_ALL)):
            k0, P0, n0 = ctx.power(u, ids, species_a=sa, species_b=sb, nbins=nb)
            k1, P1, n1 = pm.power_bin_noalloc(spectra[sa], spectra[sb], cfg.nmesh, cfg.box, nb)
            torch.cuda.synchronize()
            k1, P1, n1 = k1.cpu().numpy(), P1.cpu().numpy(), n1.cpu().numpy()
            np.testing.assert_array_equal(n1.astype(np.int64), n0)
            ok = n0 > 0
            np.testing.assert_allclose(k1[ok], k0[ok], rtol=1e-12)
            np.testing.assert_allclose(P1[ok], P0[ok], rtol=1e-5)
    ctx.sync()


def test_noalloc_binning_at_512_with_the_most_bins(pm):
    """A 512^3 mesh (more x planes than the 256 CTAs of the binning kernel, so each CTA
    loops over two planes) with nbins = 512, the array's limit: equal to pm_power on the
    same particles, on two calls in a row."""
    cfg = pm.RunConfig(box=512.0, nmesh=512, nc=128)
    ctx = pm.ParticleMesh(cfg)
    noise = torch.from_numpy(inputs.white_noise(cfg.nc, seed=5)).cuda()
    st = ctx.ic(noise, 0.2, k_fs=0.0)
    u, ids = st["u"], st["id"]
    nb = 512
    spec = ctx.fft_r2c(ctx.paint(u, ids, species=pm.SPECIES_ALL))
    k0, P0, n0 = ctx.power(u, ids, species_a=pm.SPECIES_ALL, species_b=pm.SPECIES_ALL, nbins=nb)
    for call in range(2):
        k1, P1, n1 = pm.power_bin_noalloc(spec, spec, cfg.nmesh, cfg.box, nb)
        torch.cuda.synchronize()
        k1, P1, n1 = k1.cpu().numpy(), P1.cpu().numpy(), n1.cpu().numpy()
        np.testing.assert_array_equal(n1.astype(np.int64), n0)
        assert (n0 > 0).sum() > 400          # every |n| up to sqrt(3) 256 has modes
        ok = n0 > 0
        np.testing.assert_allclose(k1[ok], k0[ok], rtol=1e-12)
        np.testing.assert_allclose(P1[ok], P0[ok], rtol=1e-5)
    ctx.sync()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(pm):
    x = torch.zeros((64, 64, 33, 2), dtype=torch.float32, device="cuda")
    for bad in (dict(nbins=513), dict(nbins=0), dict(nmesh=48), dict(box=0.0)):
        args = dict(nmesh=64, box=100.0, nbins=16)
        args.update(bad)
        with pytest.raises(pm.PMError) as ei:
            pm.power_bin_noalloc(x, x, args["nmesh"], args["box"], args["nbins"])
        assert ei.value.status == pm.PM_EINVAL
