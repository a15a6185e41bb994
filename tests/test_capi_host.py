"""CPU checks of the C-ABI library: it loads, exports every symbol include/pm.h
declares, and its host FP64 code (growth ODE, KDK factors, shell tables) agrees
with the oracle.  No GPU call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import background as obg
from oracle import neutrinos as onu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2007_13394_gb300 import pm
    return pm.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_five_required_calls():
    names = declared_functions()
    for req in ("pm_init", "pm_paint", "pm_force", "pm_step", "pm_power"):
        assert req in names


def test_required_calls_cite_the_passage_that_defines_them():
    """Each of the five calls of the boundary carries, in the comment right above its
    declaration, a citation (§ section, equation, table) of the passage it implements."""
    text = open(os.path.join(ROOT, "include", "pm.h")).read()
    want = {"pm_init": ["Eq. growthDE", "Eq. Hubble", "m_shell"],
            "pm_paint": ["Eq. Om_pois"],
            "pm_force": ["Eq. Om_pois", "Table 1"],
            "pm_step": ["Kick-Drift-Kick", "§2.3"],
            "pm_power": ["§3"]}
    for name, cites in want.items():
        m = re.search(r"/\*((?:(?!\*/).)*)\*/\s*int " + name + r"\(", text, flags=re.S)
        assert m, name
        comment = m.group(1)
        assert "§" in comment, name
        for c in cites:
            assert c in comment, (name, c)


def test_library_exports_every_declared_symbol(lib):
    so = os.path.join(ROOT, "paper_2007_13394_gb300", "libpmnu.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(pm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_strerror(lib):
    from paper_2007_13394_gb300 import pm
    assert pm.strerror(0) == "ok"
    assert "invalid" in pm.strerror(-1)


def _cfg(**kw):
    from paper_2007_13394_gb300 import pm
    base = dict(box=256.0, nmesh=64, nc=32, nsites=8, nshell=10, nfib=3, m_nu=(0.2 / 3,) * 3)
    base.update(kw)
    return pm.RunConfig(**base)


@pytest.mark.parametrize("masses", [(0.2 / 3,) * 3, (0.19786, 0.19805, 0.20408), (0.0, 0.0, 0.0)])
def test_host_growth_and_coefficients_match_oracle(lib, masses):
    from paper_2007_13394_gb300 import pm
    cfg = _cfg(m_nu=masses, nsites=0)
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=masses)
    for a in (0.01, 0.05, 0.3, 1.0):
        D, gp, gf, E = pm.cosmo_growth(cfg, a)
        assert D == pytest.approx(bg.D(a), rel=1e-9)
        assert gp == pytest.approx(bg.gp(a), rel=1e-9)
        assert gf == pytest.approx(bg.gf(a), rel=1e-9)
        assert E == pytest.approx(bg.E(a), rel=1e-12)
    for (a0, ah, a1) in obg.schedule_paper(25)[::6]:
        got = pm.cosmo_coeffs(cfg, a0, ah, a1)
        np.testing.assert_allclose(got, obg.step_coefficients(bg, a0, ah, a1), rtol=1e-9)
    prm = pm.cosmo_params(cfg)
    assert prm["omega_lambda"] == pytest.approx(bg.omega_lambda, rel=1e-12)
    assert prm["omega_gamma"] == pytest.approx(bg.omega_gamma, rel=1e-12)
    assert prm["kT_nu0"] == pytest.approx(bg.kT_nu0, rel=1e-12)


@pytest.mark.parametrize("masses", [(0.2 / 3,) * 3, (0.12, 0.06, 0.02)])
def test_host_shell_table_matches_oracle(lib, masses):
    from paper_2007_13394_gb300 import pm
    cfg = _cfg(m_nu=masses)
    e, q, m = pm.nu_shells(cfg)
    e0, q0, m0 = onu.shell_table(10, list(masses))
    np.testing.assert_allclose(e, e0, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(q, q0, rtol=1e-11)
    np.testing.assert_allclose(m, m0, rtol=1e-11)


def test_host_rejects_bad_configs(lib):
    from paper_2007_13394_gb300 import pm
    for bad in (dict(nmesh=48), dict(nmesh=16), dict(box=-1.0), dict(nmesh=4096), dict(m_nu=(0.0, 0.0, 0.0))):
        with pytest.raises(pm.PMError) as ei:
            pm.cosmo_growth(_cfg(**bad), 0.5) if "m_nu" not in bad else pm.nu_shells(_cfg(**bad))
        assert ei.value.status == pm.PM_EINVAL
    with pytest.raises(pm.PMError):
        pm.cosmo_coeffs(_cfg(), 0.5, 0.4, 0.6)     # half point outside the step


def test_noalloc_wrapper_rejects_short_or_foreign_spectra():
    """pm_power_bin_noalloc receives raw pointers, so its binding checks the spectra before
    any device work: a 64^3 half spectrum passed with nmesh = 128 would be read past its end."""
    torch = pytest.importorskip("torch")
    from paper_2007_13394_gb300 import pm
    ok64 = torch.zeros((64, 64, 33, 2), dtype=torch.float32)
    with pytest.raises(ValueError, match="half spectrum needs"):
        pm.check_half_spectrum(ok64, 128)
    with pytest.raises(ValueError, match="half spectrum needs"):
        pm.power_bin_noalloc(ok64, ok64, 128, 100.0, 16)       # rejected before any GPU call
    with pytest.raises(ValueError, match="float32"):
        pm.check_half_spectrum(ok64.double(), 64)
    with pytest.raises(ValueError, match="contiguous"):
        pm.check_half_spectrum(torch.zeros((64, 64, 66, 2), dtype=torch.float32)[:, :, ::2], 64)
    with pytest.raises(ValueError, match="CUDA"):
        pm.check_half_spectrum(ok64, 64)
    with pytest.raises(ValueError, match="torch tensor"):
        pm.check_half_spectrum(np.zeros(64 * 64 * 33 * 2, dtype=np.float32), 64)
