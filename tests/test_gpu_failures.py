"""Failure paths of the library, made on the host or by a copy that is never issued --
nothing here faults, traps or hangs the GPU.

* A bounded wait that runs out: pm_test_inject makes the first CTA of the next
  TMA-pipelined FFT pass skip its first tile copy; its wait on that copy gives up after a
  short limit, the CTA waits for its other copies in flight and returns, pm_sync reports
  PM_ETIMEOUT, and the same context then computes the force again bit for bit.
* A NaN or infinite momentum reaches the kick kernels: pm_sync reports PM_ENONFINITE.
* An allocation that would pass the context's memory limit: PM_ENOMEM, from pm_init (which
  then holds nothing) and from a call that allocates on first use (the context stays usable).
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


def _cfg1_state(pm, ctx, cfg, seed=1, a0=0.05):
    noise = torch.from_numpy(inputs.white_noise(cfg.nc, seed=seed)).cuda()
    return ctx.ic(noise, a0, k_fs=0.0)


def test_dropped_tma_copy_times_out_and_the_context_recovers(pm):
    from paper_2007_13394_gb300 import workloads
    cfg = workloads.cfg1()                       # 64^3 mesh: the y and x passes run on TMA tiles
    ctx = pm.ParticleMesh(cfg)
    st = _cfg1_state(pm, ctx, cfg)
    F0 = ctx.force(st["u"], st["id"]).clone()
    ctx.sync()
    ctx.test_inject(pm.PM_INJECT_DROP_COPY)
    ctx.force(st["u"], st["id"])
    with pytest.raises(pm.PMError) as ei:
        ctx.sync()
    assert ei.value.status == pm.PM_ETIMEOUT
    ctx.sync()                                   # the error word was read and cleared
    F1 = ctx.force(st["u"], st["id"])
    ctx.sync()
    assert torch.equal(F0, F1)                   # deterministic force, same bits as before
    with pytest.raises(pm.PMError) as ei:
        ctx.test_inject(7)
    assert ei.value.status == pm.PM_EINVAL
    ctx.close()


def test_nonfinite_momentum_is_reported(pm):
    from paper_2007_13394_gb300 import workloads
    cfg = workloads.cfg1()
    ctx = pm.ParticleMesh(cfg)
    for bad in (float("nan"), float("inf")):
        st = _cfg1_state(pm, ctx, cfg)
        ctx.step(st, 0.05, 0.055, 0.06)
        ctx.sync()
        st["p"][1, 123] = bad                    # one particle's momentum
        ctx.step(st, 0.06, 0.065, 0.07)
        with pytest.raises(pm.PMError) as ei:
            ctx.sync()
        assert ei.value.status == pm.PM_ENONFINITE
    # a clean state steps without error on the same context
    st = _cfg1_state(pm, ctx, cfg)
    ctx.step(st, 0.05, 0.055, 0.06)
    ctx.sync()
    assert torch.isfinite(st["p"]).all()
    ctx.close()


def test_memory_limit_returns_enomem(pm):
    from paper_2007_13394_gb300 import workloads
    base = workloads.cfg1()
    ctx = pm.ParticleMesh(base)
    need = ctx.memory_used()
    assert need > 3 * 64 * 64 * 34 * 8       # at least the padded meshes
    st = _cfg1_state(pm, ctx, base)          # initial conditions from an unlimited context
    ctx.sync()
    ctx.close()
    free0 = torch.cuda.mem_get_info()[0]
    import dataclasses
    for limit in (1 << 20, need // 2, need - 1):
        with pytest.raises(pm.PMError) as ei:
            pm.ParticleMesh(dataclasses.replace(base, mem_limit=limit))
        assert ei.value.status == pm.PM_ENOMEM
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)   # nothing left allocated
    # exactly enough for pm_init: the host-buffer step, which allocates its device copy of the
    # state on first use, is refused; the device path still works
    ctx = pm.ParticleMesh(dataclasses.replace(base, mem_limit=need))
    assert ctx.memory_used() == need
    n = st["u"].shape[1]
    hu = pm.to_u32(st["u"]).copy()
    hp = st["p"].cpu().numpy().copy()
    hid = pm.to_u32(st["id"]).copy()
    hf = np.zeros_like(hp)
    with pytest.raises(pm.PMError) as ei:
        ctx.step_host(hu, hp, hid, hf, 0, 0.05, 0.055, 0.06)
    assert ei.value.status == pm.PM_ENOMEM
    assert ctx.memory_used() == need
    ctx.step(st, 0.05, 0.055, 0.06)
    ctx.sync()
    assert torch.isfinite(st["p"]).all() and n == st["p"].shape[1]
    ctx.close()
