"""Host-side schedule and bench bookkeeping (no GPU)."""
import importlib.util
import math
import os

import pytest

from paper_2007_13394_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n", [6, 10, 25, 40, 66])
def test_paper_schedule_chains_exactly(n):
    """pm_run takes chained steps only (each a0 equal to the previous a1, bit for bit):
    the schedule must produce them, with log-a steps to a = 0.05 (geometric half points)
    and linear-a steps to a = 1 (arithmetic half points)."""
    s = workloads.schedule_paper(n)
    assert len(s) == n
    assert s[0][0] == 0.01 and s[-1][2] == 1.0
    for (a0, ah, a1), nxt in zip(s, s[1:] + [None]):
        assert a0 < ah < a1
        if nxt is not None:
            assert nxt[0] == a1
    for a0, ah, a1 in s[:5]:
        assert ah == pytest.approx(math.sqrt(a0 * a1), rel=1e-12)
    assert s[4][2] == 0.05
    for a0, ah, a1 in s[5:]:
        assert ah == pytest.approx(0.5 * (a0 + a1), rel=1e-12)


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_run_readout_bytes_average():
    """The readout of a pm_run of K steps: K - 1 launches carry the next kick and drift
    (60 B a particle: u, p, id read; p, u, id, key written), the last is the plain readout
    (68 B: also the force cache); 4 B a cell for the potential either way."""
    b = _bench()
    n, nm = 1000, 32
    plain = b.algorithmic_bytes("readout_fd4_kick", nm, n)
    assert plain == 68 * n + 4 * nm ** 3
    assert b.run_readout_bytes(nm, n, 1) == plain
    assert b.run_readout_bytes(nm, n, 4) == pytest.approx((3 * (60 * n + 4 * nm ** 3) + plain) / 4)


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3"])
def test_free_streaming_k_equals_oracle(name):
    """The product's k_fs (the initial-condition suppression scale it hands to pm_ic) equals
    the oracle's own restatement."""
    from oracle import ic as oic
    cfg = workloads.PRESETS[name]()
    for a in (0.01, 0.1, 1.0):
        assert workloads.free_streaming_k(cfg, a) == pytest.approx(
            oic.free_streaming_k(list(cfg.m_nu), a, cfg.omega_m), rel=1e-14)
