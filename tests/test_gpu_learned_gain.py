"""What the trained factor gains over the plain kernel, on the GPU.

Reduced version of the learned-correction workload: 128 Mpc/h, 64^3 CDM + 4^3 x 70
neutrinos (M_nu = 0.3 eV), force mesh 64^3 (boost 1, 2 Mpc/h spacing, k_Ny = 1.57
h/Mpc).  Targets are 40-step runs on a 256^3 mesh (boost 4: the mesh sizes are powers of
two) from the same initial conditions.  The factor is trained (spectrum-matching loss up to
k = 1 h/Mpc, Adam, 120 passes) on four seeds with 10-step runs, then judged on an unseen
seed by max_{k <= 1 h/Mpc} |P_m / P_m,target - 1| against plain 10-step and plain 25-step
runs (P_m on one 128^3 measuring mesh): it must beat plain 25 steps and halve the plain
10-step error.  (At boost 1 against boost-4 targets even plain 40 steps stay ~30 % off
at k = 1 h/Mpc: the mesh resolution, not the step count, sets the error there.)"""
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


def test_trained_factor_beats_plain_ten_steps(pm):
    from paper_2007_13394_gb300 import learned, workloads
    cfg = pm.RunConfig(box=128.0, nmesh=64, nc=64, nsites=4, nshell=10, nfib=3, m_nu=(0.1,) * 3)
    s10, s25, s40 = (workloads.schedule_paper(n) for n in (10, 25, 40))
    a0 = s10[0][0]
    coarse = pm.ParticleMesh(cfg)
    fine = pm.ParticleMesh(learned.boosted(cfg, 4))
    meas = pm.ParticleMesh(learned.boosted(cfg, 2))

    def noise(seed):
        return torch.from_numpy(inputs.white_noise(cfg.nc, seed=seed)).cuda()

    examples = [(noise(s), learned.final_positions(fine, noise(s), s40, a0)) for s in range(1000, 1004)]
    coarse.set_mlp(learned.zero_factor(0))
    log = learned.train(coarse, examples, s10, a0, iters=120, lr=1e-2, loss="spectrum", k_max=1.0)
    print("\nloss every 10 passes:", " ".join(f"{x:.3e}" for x in log.losses[::10]))
    assert log.losses[-1] < 0.2 * log.losses[0]

    ev = noise(9001)
    nb = 40
    k, P_ref = learned.matter_power(meas, learned.final_positions(fine, ev, s40, a0), nb)
    _, P_corr = learned.matter_power(meas, learned.final_positions(coarse, ev, s10, a0), nb)
    coarse.set_mlp(None)
    _, P10 = learned.matter_power(meas, learned.final_positions(coarse, ev, s10, a0), nb)
    _, P25 = learned.matter_power(meas, learned.final_positions(coarse, ev, s25, a0), nb)
    e_corr, e10, e25 = (learned.max_power_error(k, P, P_ref, 1.0) for P in (P_corr, P10, P25))
    print(f"\nmax |P/P_ref - 1| for k <= 1 h/Mpc: corrected-10 {e_corr:.4f}  plain-10 {e10:.4f}  "
          f"plain-25 {e25:.4f}; loss {log.losses[0]:.4e} -> {log.losses[-1]:.4e} in {log.seconds:.1f} s")
    assert e_corr < 0.5 * e10
    assert e_corr < e25
