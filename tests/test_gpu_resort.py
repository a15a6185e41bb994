"""The order pm_step leaves the state in, through the near-sorted re-sort, on the GPU.

After every step the state must be the stable sort, by the oracle's tile key of the
drifted positions, of the order the step started from (bit-exact); the context reports
which way it sorted (pm_sort_stats).  A state shuffled between steps is not in the
order of the last sort: the step must notice, sort from scratch and give the same
stable order.
"""
import numpy as np
import pytest

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


def _state(pm, ctx, cfg, seed=1, a0=0.05):
    noise = torch.from_numpy(inputs.white_noise(cfg.nc, seed=seed)).cuda()
    return ctx.ic(noise, a0)


def _host(pm, st):
    return pm.to_u32(st["u"]), pm.to_u32(st["id"])


def _expected_order(pm, ids_before, u_after, ids_after, nmesh):
    """ids in the stable order of the drifted keys, taken in the pre-step order."""
    where = np.empty(len(ids_after), np.int64)
    where[ids_after] = np.arange(len(ids_after))
    u_prev_order = u_after[:, where[ids_before]]
    keys = opm.sort_keys(u_prev_order, nmesh)
    return ids_before[np.argsort(keys, kind="stable")]


@pytest.mark.parametrize("nmesh,nc,nsites", [(64, 32, 8), (128, 64, 8)])
def test_step_order_is_the_stable_sort_of_the_drifted_keys(pm, nmesh, nc, nsites):
    cfg = pm.RunConfig(box=256.0, nmesh=nmesh, nc=nc, nsites=nsites, nshell=10, nfib=3, m_nu=(0.1,) * 3)
    ctx = pm.ParticleMesh(cfg)
    st = _state(pm, ctx, cfg)
    # steps long enough that particles cross face layers and tiles (neutrinos several cells)
    sched = [(0.05, 0.1), (0.1, 0.2), (0.2, 0.4), (0.4, 0.7), (0.7, 1.0)]
    for a0, a1 in sched:
        u0, ids0 = _host(pm, st)
        if a0 == sched[0][0]:  # the first step's force sorts the caller's order from scratch
            perm0 = np.argsort(opm.sort_keys(u0, nmesh), kind="stable")
            ids0 = ids0[perm0]
        ctx.step(st, a0, 0.5 * (a0 + a1), a1)
        ctx.sync()
        u1, ids1 = _host(pm, st)
        assert np.array_equal(np.sort(ids1), np.arange(len(ids1)))
        assert np.array_equal(ids1, _expected_order(pm, ids0, u1, ids1, nmesh)), (a0, a1)
    fast, full, movers = ctx.sort_stats()
    assert (fast, full) == (len(sched), 0)
    assert 0 < movers < cfg.n_particles()


def test_shuffled_state_sorts_from_scratch(pm):
    cfg = pm.RunConfig(box=256.0, nmesh=64, nc=32, nsites=8, nshell=10, nfib=3, m_nu=(0.1,) * 3)
    ctx = pm.ParticleMesh(cfg)
    st = _state(pm, ctx, cfg, seed=2)
    ctx.step(st, 0.05, 0.075, 0.1)
    rng = np.random.default_rng(3)
    perm = torch.from_numpy(rng.permutation(cfg.n_particles())).cuda()
    for k in ("u", "p", "f"):
        st[k].copy_(st[k][:, perm].contiguous())
    st["id"].copy_(st["id"][perm].contiguous())
    u0, ids0 = _host(pm, st)
    ctx.step(st, 0.1, 0.15, 0.2)
    ctx.sync()
    u1, ids1 = _host(pm, st)
    assert np.array_equal(ids1, _expected_order(pm, ids0, u1, ids1, 64))
    fast, full, _ = ctx.sort_stats()
    assert (fast, full) == (1, 1)
    # the next step is in order again
    ctx.step(st, 0.2, 0.3, 0.4)
    ctx.sync()
    u2, ids2 = _host(pm, st)
    assert np.array_equal(ids2, _expected_order(pm, ids1, u2, ids2, 64))
    assert ctx.sort_stats()[:2] == (2, 1)


@pytest.mark.parametrize("warm,learned", [(False, False), (True, False), (False, True)],
                         ids=["from_ics", "after_a_step", "learned_factor"])
def test_run_equals_repeated_steps_bitwise(pm, warm, learned):
    """pm_run fuses each step's last readout with the next step's first half kick and
    drift; the state after it must be that of pm_step called once per step, bit for bit."""
    cfg = pm.RunConfig(box=256.0, nmesh=64, nc=32, nsites=8, nshell=10, nfib=3, m_nu=(0.1,) * 3)
    ca, cb = pm.ParticleMesh(cfg), pm.ParticleMesh(cfg)
    if learned:  # the factor's table is refreshed at every force evaluation in both forms
        th = inputs.mlp_parameters(6, last_scale=0.5)
        ca.set_mlp(th)
        cb.set_mlp(th)
    sa, sb = _state(pm, ca, cfg, seed=4), _state(pm, cb, cfg, seed=4)
    if warm:
        ca.step(sa, 0.05, 0.075, 0.1)
        cb.step(sb, 0.05, 0.075, 0.1)
        sched = [(0.1, 0.15, 0.2), (0.2, 0.3, 0.4), (0.4, 0.55, 0.7), (0.7, 0.85, 1.0)]
    else:
        sched = [(0.05, 0.1, 0.15), (0.15, 0.3, 0.45), (0.45, 0.7, 1.0)]
    for t in sched:
        ca.step(sa, *t)
    cb.run(sb, sched)
    ca.sync()
    cb.sync()
    for k in ("u", "p", "f", "id"):
        assert torch.equal(sa[k], sb[k]), k
    assert sb["a"] == sched[-1][2] and sb["f_valid"] == 1
    assert cb.sort_stats()[:2] == ca.sort_stats()[:2]


def test_run_rejects_a_broken_schedule(pm):
    cfg = pm.RunConfig(box=256.0, nmesh=64, nc=32, nsites=8, nshell=10, nfib=3, m_nu=(0.1,) * 3)
    ctx = pm.ParticleMesh(cfg)
    st = _state(pm, ctx, cfg, seed=5)
    with pytest.raises(pm.PMError):
        ctx.run(st, [(0.05, 0.06, 0.07), (0.08, 0.09, 0.1)])  # a0 of the second != a1 of the first
    ctx.run(st, [])
    assert st["f_valid"] == 0
