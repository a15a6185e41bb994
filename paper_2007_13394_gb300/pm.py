"""Thin ctypes binding over libpmnu (include/pm.h).

Argument marshalling only: every step of the particle-mesh path runs in the
library's CUDA kernels.  Torch tensors supply device memory and the current
stream; uint32 arrays (positions, ids, permutations) travel as int32 tensors
with the same bits.  A missing or unloadable library raises ``RuntimeError``:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmnu.so")

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_EKERNEL, PM_ETIMEOUT, PM_ENOTINIT = 0, -1, -2, -3, -4, -5, -6
PM_ENONFINITE = -7
PM_FLAG_TWO_MESH, PM_FLAG_SPECTRAL_KERNEL, PM_FLAG_MLP_TENSOR, PM_FLAG_KSPACE_GRADIENT = 1, 2, 4, 8
PM_INJECT_DROP_COPY = 1
SPECIES_CDM, SPECIES_NU, SPECIES_ALL = 1, 2, 3
MLP_HIDDEN, MLP_NPARAM = 64, 4417
FLAG_TWO_MESH, FLAG_SPECTRAL_KERNEL, FLAG_MLP_TENSOR, FLAG_KSPACE_GRADIENT = 1, 2, 4, 8


class PMError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {status} ({strerror(status)})")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double), ("nmesh", ctypes.c_int32), ("nc", ctypes.c_int32),
        ("nsites", ctypes.c_int32), ("nshell", ctypes.c_int32), ("nfib", ctypes.c_int32),
        ("h", ctypes.c_double), ("omega_m", ctypes.c_double), ("t_cmb", ctypes.c_double),
        ("n_eff", ctypes.c_double), ("n_nu", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("m_nu", ctypes.c_double * 3), ("a_ini_ode", ctypes.c_double), ("n_max", ctypes.c_int64),
        ("ns", ctypes.c_double), ("sigma8", ctypes.c_double), ("flags", ctypes.c_uint32),
        ("pad1", ctypes.c_int32), ("mem_limit", ctypes.c_int64),
    ]


class State(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_void_p), ("p", ctypes.c_void_p), ("id", ctypes.c_void_p), ("f", ctypes.c_void_p),
        ("n", ctypes.c_int64), ("a", ctypes.c_double), ("f_valid", ctypes.c_int32), ("pad0", ctypes.c_int32),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpmnu.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpmnu.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "pm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "pm_cosmo_growth": (ctypes.c_int, [ctypes.POINTER(Config), d, dp]),
        "pm_cosmo_coeffs": (ctypes.c_int, [ctypes.POINTER(Config), d, d, d, dp]),
        "pm_cosmo_params": (ctypes.c_int, [ctypes.POINTER(Config), dp]),
        "pm_nu_shells": (ctypes.c_int, [ctypes.POINTER(Config), dp, dp, dp]),
        "pm_init": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
        "pm_destroy": (ctypes.c_int, [vp]),
        "pm_sync": (ctypes.c_int, [vp, vp]),
        "pm_coeffs": (ctypes.c_int, [vp, d, d, d, dp]),
        "pm_sort": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "pm_paint": (ctypes.c_int, [vp, vp, vp, i64, i32, vp, vp]),
        "pm_force": (ctypes.c_int, [vp, vp, vp, i64, vp, vp]),
        "pm_step": (ctypes.c_int, [vp, ctypes.POINTER(State), d, d, d, vp]),
        "pm_run": (ctypes.c_int, [vp, ctypes.POINTER(State), dp, i64, vp]),
        "pm_step_host": (ctypes.c_int, [vp, vp, vp, vp, vp, i64, ctypes.POINTER(i32), d, d, d, vp]),
        "pm_power": (ctypes.c_int, [vp, vp, vp, i64, i32, i32, i32, vp, vp, vp, vp]),
        "pm_ic": (ctypes.c_int, [vp, vp, d, d, ctypes.POINTER(State), vp]),
        "pm_ic_pseudo": (ctypes.c_int, [vp, vp, vp, d, d, ctypes.POINTER(State), vp]),
        "pm_state_save": (ctypes.c_int, [vp, ctypes.POINTER(State), ctypes.c_char_p]),
        "pm_state_load": (ctypes.c_int, [vp, ctypes.POINTER(State), ctypes.c_char_p]),
        "pm_fft_r2c": (ctypes.c_int, [vp, vp, vp, vp]),
        "pm_fft_c2r": (ctypes.c_int, [vp, vp, vp, vp]),
        "pm_potential": (ctypes.c_int, [vp, vp, vp, vp]),
        "pm_force_mesh": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "pm_readout": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "pm_power_bin_noalloc": (ctypes.c_int, [vp, vp, i32, d, i32, vp, vp, vp, vp]),
        "pm_paint_T": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "pm_readout_T": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
        "pm_paint_vjp": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "pm_force_vjp": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "pm_power_vjp": (ctypes.c_int, [vp, vp, vp, i64, i32, i32, vp, vp, vp]),
        "pm_step_vjp": (ctypes.c_int, [vp, ctypes.POINTER(State), d, d, d, vp, vp, vp, vp, vp]),
        "pm_ic_vjp": (ctypes.c_int, [vp, vp, vp, d, d, vp, vp]),
        "pm_set_mlp": (ctypes.c_int, [vp, vp, i64]),
        "pm_get_mlp": (ctypes.c_int, [vp, vp, i64]),
        "pm_set_force_time": (ctypes.c_int, [vp, d]),
        "pm_mlp_eval": (ctypes.c_int, [vp, vp, vp, i64, vp, vp]),
        "pm_mlp_table": (ctypes.c_int, [vp, d, vp, vp]),
        "pm_mlp_grad": (ctypes.c_int, [vp, vp, i64, i32, vp]),
        "pm_mlp_adam": (ctypes.c_int, [vp, vp, i64, d, d, d, d, i64, vp]),
        "pm_displacement_loss": (ctypes.c_int, [vp, vp, vp, vp, vp, i64, i32, vp, dp, vp]),
        "pm_launch_count": (i64, [vp]),
        "pm_memory_used": (i64, [vp]),
        "pm_test_inject": (ctypes.c_int, [vp, i32]),
        "pm_profile_enable": (ctypes.c_int, [vp, i32]),
        "pm_profile_read": (ctypes.c_int, [vp, i32, dp, ctypes.POINTER(i64), i32]),
        "pm_kernel_kinds": (i32, []),
        "pm_kernel_name": (ctypes.c_char_p, [i32]),
        "pm_sort_stats": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load_library().pm_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return "?"


def _check(status, what):
    if status != PM_OK:
        raise PMError(status, what)


@dataclass
class RunConfig:
    """Python mirror of pm_config with the defaults of the synthetic workloads."""
    box: float
    nmesh: int
    nc: int
    nsites: int = 0
    nshell: int = 10
    nfib: int = 3
    h: float = 0.68
    omega_m: float = 0.31
    t_cmb: float = 2.7255
    n_eff: float = 3.046
    m_nu: tuple = (0.0, 0.0, 0.0)
    a_ini_ode: float = 1.0 / 160.0
    n_max: int = 0
    ns: float = 0.965
    sigma8: float = 0.81
    flags: int = 0
    mem_limit: int = 0
    extra: dict = field(default_factory=dict)

    def n_cdm(self) -> int:
        return self.nc ** 3

    def n_nu(self) -> int:
        return self.nsites ** 3 * self.nshell * (2 * self.nfib + 1) if self.nsites else 0

    def n_particles(self) -> int:
        return self.n_cdm() + self.n_nu()

    def to_c(self) -> Config:
        c = Config()
        c.box, c.nmesh, c.nc, c.nsites = self.box, self.nmesh, self.nc, self.nsites
        c.nshell, c.nfib, c.h, c.omega_m = self.nshell, self.nfib, self.h, self.omega_m
        c.t_cmb, c.n_eff = self.t_cmb, self.n_eff
        m = [float(x) for x in self.m_nu]
        c.n_nu = len(m)
        for i, x in enumerate(m[:3]):
            c.m_nu[i] = x
        c.a_ini_ode = self.a_ini_ode
        c.n_max = self.n_max or self.n_particles()
        c.ns, c.sigma8 = self.ns, self.sigma8
        c.flags = self.flags
        c.mem_limit = self.mem_limit
        return c


# ----------------------------------------------------------------- host-only
def cosmo_growth(cfg: RunConfig, a: float):
    out = (ctypes.c_double * 4)()
    _check(load_library().pm_cosmo_growth(ctypes.byref(cfg.to_c()), a, out), "pm_cosmo_growth")
    return tuple(out)


def cosmo_coeffs(cfg: RunConfig, a0: float, ah: float, a1: float):
    out = (ctypes.c_double * 3)()
    _check(load_library().pm_cosmo_coeffs(ctypes.byref(cfg.to_c()), a0, ah, a1, out), "pm_cosmo_coeffs")
    return tuple(out)


def cosmo_params(cfg: RunConfig):
    out = (ctypes.c_double * 5)()
    _check(load_library().pm_cosmo_params(ctypes.byref(cfg.to_c()), out), "pm_cosmo_params")
    return dict(zip(["omega_gamma", "omega_c", "omega_nu", "omega_lambda", "kT_nu0"], out))


def nu_shells(cfg: RunConfig):
    e = (ctypes.c_double * (cfg.nshell + 1))()
    q = (ctypes.c_double * cfg.nshell)()
    m = (ctypes.c_double * cfg.nshell)()
    _check(load_library().pm_nu_shells(ctypes.byref(cfg.to_c()), e, q, m), "pm_nu_shells")
    return np.array(e), np.array(q), np.array(m)


# ----------------------------------------------------------------- device
def power_bin_noalloc(delta_a, delta_b, nmesh: int, box: float, nbins: int):
    """Allocation-free binning of two half spectra (device tensors as pm_fft_r2c writes them).

    Returns device tensors (k, P, n_modes) of float64; the library itself allocates
    nothing (the output tensors are the caller's).
    """
    # the library sees raw pointers only: a spectrum shorter than the mesh's half spectrum
    # would be read past its end on the device, so the shapes are checked here
    for name, t in (("delta_a", delta_a), ("delta_b", delta_b)):
        check_half_spectrum(t, nmesh, name)
    torch = _torch()
    k = torch.empty(nbins, dtype=torch.float64, device="cuda")
    P = torch.empty(nbins, dtype=torch.float64, device="cuda")
    nm = torch.empty(nbins, dtype=torch.float64, device="cuda")
    _check(load_library().pm_power_bin_noalloc(_ptr(delta_a), _ptr(delta_b), nmesh, box, nbins, _ptr(k), _ptr(P),
                                               _ptr(nm), _stream()), "pm_power_bin_noalloc")
    return k, P, nm


def check_half_spectrum(t, nmesh: int, name: str = "spectrum") -> None:
    """Raise ValueError unless t is a contiguous float32 CUDA tensor on the current device
    holding at least the nmesh * nmesh * (nmesh // 2 + 1) complex values (interleaved
    floats) of an r2c half spectrum.  Sizes are checked before the device, so the rule
    can be exercised on CPU tensors."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if t.dtype != torch.float32:
        raise ValueError(f"{name}: float32 required (interleaved complex), got {t.dtype}")
    need = int(nmesh) * int(nmesh) * (int(nmesh) // 2 + 1) * 2
    if t.numel() < need:
        raise ValueError(f"{name}: {t.numel()} floats, the {nmesh}^3 half spectrum needs {need}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if not t.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required for the particle-mesh path")
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def as_u32_tensor(a: np.ndarray):
    """Host uint32 array -> CUDA int32 tensor with the same bits."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def to_u32(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


class ParticleMesh:
    """One library context (scratch meshes, sort buffers, FP64 growth tables)."""

    def __init__(self, cfg: RunConfig):
        self.cfg = cfg
        self.lib = load_library()
        _torch()
        h = ctypes.c_void_p()
        self._c = cfg.to_c()
        _check(self.lib.pm_init(ctypes.byref(self._c), ctypes.byref(h)), "pm_init")
        self.h = h
        self.n = cfg.nmesh

    def close(self):
        if self.h:
            self.lib.pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def sync(self):
        _check(self.lib.pm_sync(self.h, _stream()), "pm_sync")

    def coeffs(self, a0, ah, a1):
        out = (ctypes.c_double * 5)()
        _check(self.lib.pm_coeffs(self.h, a0, ah, a1, out), "pm_coeffs")
        return tuple(out)

    def sort(self, u):
        torch = _torch()
        n = u.shape[1]
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(self.lib.pm_sort(self.h, _ptr(u), n, _ptr(perm), _ptr(keys), _stream()), "pm_sort")
        return perm, keys

    def paint(self, u, ids=None, species=SPECIES_ALL):
        torch = _torch()
        mesh = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_paint(self.h, _ptr(u), _ptr(ids), u.shape[1], species, _ptr(mesh), _stream()),
               "pm_paint")
        return mesh

    def force(self, u, ids=None):
        torch = _torch()
        n = u.shape[1]
        F = torch.empty((3, n), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_force(self.h, _ptr(u), _ptr(ids), n, _ptr(F), _stream()), "pm_force")
        return F

    def step(self, st: dict, a0, ah, a1):
        s = State(_ptr(st["u"]).value, _ptr(st["p"]).value, _ptr(st["id"]).value, _ptr(st["f"]).value,
                  st["u"].shape[1], st.get("a", a0), int(st.get("f_valid", 0)), 0)
        _check(self.lib.pm_step(self.h, ctypes.byref(s), a0, ah, a1, _stream()), "pm_step")
        st["a"], st["f_valid"] = s.a, s.f_valid
        return st

    def run(self, st: dict, steps):
        """Chained KDK steps [(a0, ah, a1), ...] through pm_run (same result as step() per step)."""
        steps = [tuple(float(x) for x in t) for t in steps]
        if not steps:
            return st
        sched = (ctypes.c_double * (3 * len(steps)))(*[x for t in steps for x in t])
        s = State(_ptr(st["u"]).value, _ptr(st["p"]).value, _ptr(st["id"]).value, _ptr(st["f"]).value,
                  st["u"].shape[1], st.get("a", steps[0][0]), int(st.get("f_valid", 0)), 0)
        _check(self.lib.pm_run(self.h, ctypes.byref(s), sched, len(steps), _stream()), "pm_run")
        st["a"], st["f_valid"] = s.a, s.f_valid
        return st

    def step_host(self, u, p, ids, f, f_valid, a0, ah, a1, stream=None):
        fv = ctypes.c_int32(int(f_valid))
        rc = self.lib.pm_step_host(self.h, u.ctypes.data_as(ctypes.c_void_p), p.ctypes.data_as(ctypes.c_void_p),
                                   ids.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p),
                                   u.shape[1], ctypes.byref(fv), a0, ah, a1,
                                   stream if stream is not None else _stream())
        _check(rc, "pm_step_host")
        return fv.value

    def _state_struct(self, st):
        return State(_ptr(st["u"]).value, _ptr(st["p"]).value, _ptr(st["id"]).value, _ptr(st["f"]).value,
                     st["u"].shape[1], st.get("a", 0.0), int(st.get("f_valid", 0)), 0)

    def save_state(self, st: dict, path: str):
        s = self._state_struct(st)
        _check(self.lib.pm_state_save(self.h, ctypes.byref(s), path.encode()), "pm_state_save")

    def load_state(self, st: dict, path: str):
        s = self._state_struct(st)
        _check(self.lib.pm_state_load(self.h, ctypes.byref(s), path.encode()), "pm_state_load")
        st["a"], st["f_valid"] = s.a, s.f_valid
        return st

    def new_state(self, n):
        torch = _torch()
        return {"u": torch.empty((3, n), dtype=torch.int32, device="cuda"),
                "p": torch.empty((3, n), dtype=torch.float32, device="cuda"),
                "id": torch.empty(n, dtype=torch.int32, device="cuda"),
                "f": torch.zeros((3, n), dtype=torch.float32, device="cuda"),
                "a": 0.0, "f_valid": 0}

    def ic(self, noise, a0, k_fs=0.0):
        """Zel'dovich ICs from device white noise (float32, nc^3)."""
        st = self.new_state(self.cfg.n_particles())
        s = State(_ptr(st["u"]).value, _ptr(st["p"]).value, _ptr(st["id"]).value, _ptr(st["f"]).value,
                  st["u"].shape[1], a0, 0, 0)
        _check(self.lib.pm_ic(self.h, _ptr(noise), a0, k_fs, ctypes.byref(s), _stream()), "pm_ic")
        st["a"], st["f_valid"] = s.a, s.f_valid
        return st

    def ic_pseudo(self, noise, uniforms, a0, k_fs=0.0):
        """Zel'dovich ICs with pseudo-random neutrino speeds and directions (one particle per
        site; the configuration must have nshell = 1, nfib = 0).  uniforms: device float32
        (3, nsites^3) in [0, 1)."""
        st = self.new_state(self.cfg.n_particles())
        s = State(_ptr(st["u"]).value, _ptr(st["p"]).value, _ptr(st["id"]).value, _ptr(st["f"]).value,
                  st["u"].shape[1], a0, 0, 0)
        _check(self.lib.pm_ic_pseudo(self.h, _ptr(noise), _ptr(uniforms), a0, k_fs, ctypes.byref(s), _stream()),
               "pm_ic_pseudo")
        st["a"], st["f_valid"] = s.a, s.f_valid
        return st

    def power(self, u, ids=None, species_a=SPECIES_ALL, species_b=SPECIES_ALL, nbins=32):
        k = np.zeros(nbins)
        P = np.zeros(nbins)
        nm = np.zeros(nbins, dtype=np.int64)
        _check(self.lib.pm_power(self.h, _ptr(u), _ptr(ids), u.shape[1], species_a, species_b, nbins,
                                 k.ctypes.data_as(ctypes.c_void_p), P.ctypes.data_as(ctypes.c_void_p),
                                 nm.ctypes.data_as(ctypes.c_void_p), _stream()), "pm_power")
        return k, P, nm

    def fft_r2c(self, mesh):
        torch = _torch()
        out = torch.empty((self.n, self.n, self.n // 2 + 1, 2), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_fft_r2c(self.h, _ptr(mesh), _ptr(out), _stream()), "pm_fft_r2c")
        return out

    def fft_c2r(self, cplx):
        torch = _torch()
        out = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_fft_c2r(self.h, _ptr(cplx), _ptr(out), _stream()), "pm_fft_c2r")
        return out

    def potential(self, mesh):
        torch = _torch()
        out = torch.empty((self.n, self.n, self.n // 2 + 1, 2), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_potential(self.h, _ptr(mesh), _ptr(out), _stream()), "pm_potential")
        return out

    def force_mesh(self, phi, comp):
        torch = _torch()
        out = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_force_mesh(self.h, _ptr(phi), comp, _ptr(out), _stream()), "pm_force_mesh")
        return out

    def readout(self, u, mesh):
        torch = _torch()
        out = torch.empty(u.shape[1], dtype=torch.float32, device="cuda")
        _check(self.lib.pm_readout(self.h, _ptr(u), u.shape[1], _ptr(mesh), _ptr(out), _stream()), "pm_readout")
        return out

    # ---- adjoint ----------------------------------------------------------------
    def readout_T(self, u, w):
        """Paint of signed per-particle weights (the readout's transpose)."""
        torch = _torch()
        mesh = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_readout_T(self.h, _ptr(u), u.shape[1], _ptr(w), _ptr(mesh), _stream()), "pm_readout_T")
        return mesh

    def paint_T(self, u, mesh):
        torch = _torch()
        out = torch.empty(u.shape[1], dtype=torch.float32, device="cuda")
        _check(self.lib.pm_paint_T(self.h, _ptr(u), u.shape[1], _ptr(mesh), _ptr(out), _stream()), "pm_paint_T")
        return out

    def paint_vjp(self, u, ids, lam_mesh):
        torch = _torch()
        g = torch.empty((3, u.shape[1]), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_paint_vjp(self.h, _ptr(u), _ptr(ids), u.shape[1], _ptr(lam_mesh), _ptr(g), _stream()),
               "pm_paint_vjp")
        return g

    def power_vjp(self, u, ids, dL_dP, species=SPECIES_ALL):
        """d L / d x (input order) for L depending on the binned auto-spectrum through dL_dP."""
        torch = _torch()
        w = np.ascontiguousarray(np.asarray(dL_dP, dtype=np.float64))
        g = torch.empty((3, u.shape[1]), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_power_vjp(self.h, _ptr(u), _ptr(ids), u.shape[1], species, w.size,
                                     w.ctypes.data_as(ctypes.c_void_p), _ptr(g), _stream()), "pm_power_vjp")
        return g

    def force_vjp(self, u, ids, lam_f):
        torch = _torch()
        g = torch.empty((3, u.shape[1]), dtype=torch.float32, device="cuda")
        _check(self.lib.pm_force_vjp(self.h, _ptr(u), _ptr(ids), u.shape[1], _ptr(lam_f), _ptr(g), _stream()),
               "pm_force_vjp")
        return g

    def step_vjp(self, st, a0, ah, a1, lam_x1, lam_p1):
        """Cotangents (canonical id order) of the state after a step -> before it; st is the
        checkpoint at a0 (u, p, id, f)."""
        torch = _torch()
        lx0 = torch.empty_like(lam_x1)
        lp0 = torch.empty_like(lam_p1)
        s = self._state_struct(st)
        _check(self.lib.pm_step_vjp(self.h, ctypes.byref(s), a0, ah, a1, _ptr(lam_x1), _ptr(lam_p1), _ptr(lx0),
                                    _ptr(lp0), _stream()), "pm_step_vjp")
        return lx0, lp0

    def ic_vjp(self, lam_x0, lam_p0, a0, k_fs=0.0):
        torch = _torch()
        g = torch.empty((self.cfg.nc,) * 3, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_ic_vjp(self.h, _ptr(lam_x0), _ptr(lam_p0), a0, k_fs, _ptr(g), _stream()), "pm_ic_vjp")
        return g

    # ---- learned Green's-function factor ---------------------------------------
    def set_mlp(self, theta):
        """Switch the learned factor on with host parameters (MLP_NPARAM floats); None: off."""
        if theta is None:
            _check(self.lib.pm_set_mlp(self.h, None, 0), "pm_set_mlp")
            return
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        _check(self.lib.pm_set_mlp(self.h, t.ctypes.data_as(ctypes.c_void_p), t.size), "pm_set_mlp")

    def get_mlp(self):
        t = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(self.lib.pm_get_mlp(self.h, t.ctypes.data_as(ctypes.c_void_p), t.size), "pm_get_mlp")
        return t

    def set_force_time(self, a):
        _check(self.lib.pm_set_force_time(self.h, a), "pm_set_force_time")

    def mlp_eval(self, kappa, a):
        torch = _torch()
        out = torch.empty_like(kappa)
        _check(self.lib.pm_mlp_eval(self.h, _ptr(kappa), _ptr(a), kappa.numel(), _ptr(out), _stream()),
               "pm_mlp_eval")
        return out

    def mlp_table(self, a):
        """The factor's table m(sqrt(s) / (N/2), a), s = 0 .. 3 (N/2)^2, as the context computes it."""
        torch = _torch()
        out = torch.empty(3 * (self.n // 2) ** 2 + 1, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_mlp_table(self.h, a, _ptr(out), _stream()), "pm_mlp_table")
        return out

    def mlp_grad(self, reset=True):
        torch = _torch()
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        _check(self.lib.pm_mlp_grad(self.h, _ptr(g), MLP_NPARAM, 1 if reset else 0, _stream()), "pm_mlp_grad")
        return g

    def mlp_adam(self, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self.lib.pm_mlp_adam(self.h, _ptr(grad), MLP_NPARAM, lr, beta1, beta2, eps, int(t), _stream()),
               "pm_mlp_adam")

    def displacement_loss(self, st, ref, species=SPECIES_ALL):
        """(L, dL/dx in canonical order) of a state against a reference state (same ICs),
        over the particles of the selected species."""
        torch = _torch()
        n = st["u"].shape[1]
        lam = torch.empty((3, n), dtype=torch.float32, device="cuda")
        out = ctypes.c_double()
        _check(self.lib.pm_displacement_loss(self.h, _ptr(st["u"]), _ptr(st["id"]), _ptr(ref["u"]),
                                             _ptr(ref.get("id")), n, species, _ptr(lam), ctypes.byref(out),
                                             _stream()),
               "pm_displacement_loss")
        return out.value, lam

    def memory_used(self):
        """Bytes of device memory the context holds (checked against RunConfig.mem_limit)."""
        return int(self.lib.pm_memory_used(self.h))

    def test_inject(self, what):
        """Arm a one-shot failure of the next launch of the selected kind (PM_INJECT_*)."""
        _check(self.lib.pm_test_inject(self.h, what), "pm_test_inject")

    def launch_count(self):
        return int(self.lib.pm_launch_count(self.h))

    def sort_stats(self):
        """(steps re-sorted the near-sorted way, steps sorted from scratch, movers of the last
        near-sorted re-sort)."""
        out = (ctypes.c_int64 * 3)()
        _check(self.lib.pm_sort_stats(self.h, out), "pm_sort_stats")
        return int(out[0]), int(out[1]), int(out[2])

    def kernel_kinds(self):
        return [self.lib.pm_kernel_name(k).decode() for k in range(self.lib.pm_kernel_kinds())]

    def profile(self, kinds=None):
        """Time the named kernel kinds with CUDA events (None: all, []: off)."""
        if kinds is None:
            mask = -1
        else:
            names = self.kernel_kinds()
            mask = 0
            for k in kinds:
                mask |= 1 << names.index(k)
        _check(self.lib.pm_profile_enable(self.h, mask), "pm_profile_enable")

    def profile_read(self, reset=True):
        out = {}
        for k in range(self.lib.pm_kernel_kinds()):
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            _check(self.lib.pm_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0),
                   "pm_profile_read")
            if n.value:
                out[self.lib.pm_kernel_name(k).decode()] = (ms.value, n.value)
        return out
