"""Throughput of the particle-mesh kick-drift-kick step on GB300.

A "step" is one full KDK step (first half kick + drift + sort + paint + r2c FFT
with the Green's function + 3 x (inverse FFT + readout + second half kick)) over
every particle of the workload, inputs resident in HBM.  Default workload: 512
Mpc/h, 256^3 CDM + 32^3 x 70 neutrinos (M_nu = 0.1 eV), mesh 512^3, started
from Zel'dovich initial conditions at z = 99 and advanced along the paper's
schedule (5 log-a steps, then linear a).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s per PM step"
UNIT = "particle-updates/s"


# ------------------------------------------------------------------ helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(kind, n_mesh, n_particles):
    """Compulsory DRAM bytes of one launch of a kernel kind."""
    cells = n_mesh ** 3
    half = n_mesh * n_mesh * (n_mesh // 2 + 1) * 8      # complex half spectrum
    table = {
        "fft_y": 2 * half,
        "fft_x_green": 2 * half,
        "fft_x_grad": 2 * half,
        "fft_z_r2c": 4 * cells + half,
        "fft_z_c2r": half + 4 * cells,
        "paint_tiles": 16 * n_particles + 4 * cells,           # u + id read, mesh written once
        # u 12 + p_j 4 read, p_j 4 + f_j 4 written, mesh read once; u, id copy-back on 1 of 3
        "readout_kick": 24 * n_particles + 4 * cells + (12 + 4 + 4 + 8) * n_particles // 3,
        "fft_x_fused": 4 * half,                                # read once, three components written
        # u, p, id read; p, f, u, id written (tile order); three meshes read once
        "readout3_kick": 68 * n_particles + 12 * cells,
        "fft_x_plain": 2 * half,
        "fft_x_potential": 2 * half,                            # forward, Green's function, inverse
        # u, p, id read; p, f, u, id written (tile order); the potential read once
        "readout_fd4_kick": 68 * n_particles + 4 * cells,
        # stayers copied into tile order (u, p, id read and written) + key, flag, scan read
        "resort_place": 68 * n_particles,
        "kick_drift_keys": 64 * n_particles,
        "gather": 64 * n_particles,
        "radix_scatter": 16 * n_particles,
        "radix_hist": 4 * n_particles,
        "keys": 16 * n_particles,
    }
    return table.get(kind)


def run_readout_bytes(n_mesh, n_particles, k_steps):
    """Average algorithmic bytes of one k_readout_fd4_kick launch over a pm_run of k_steps:
    k - 1 launches carry the next step's kick and drift (u, p, id read 28 B; p, u, id, key
    written 32 B; no force cache), the last one is the plain readout (68 B)."""
    fused = 60 * n_particles + 4 * n_mesh ** 3
    plain = algorithmic_bytes("readout_fd4_kick", n_mesh, n_particles)
    return (fused * (k_steps - 1) + plain) / k_steps


def source_digest(files=None):
    """sha256 prefix of the given CUDA source files (default: all of them)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2007_13394_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# (profiles/ncu_readout_fd4_kick_cfg2.md), keyed by (kernel kind, workload): ((bytes of the
# launch that carries the next step's kick and drift, bytes of the plain launch), digest,
# the source files that define the kernel).  Reported only while those files hash to the
# digest.
NCU_TRAFFIC = {
    ("readout_fd4_kick", "cfg2"): ((1685900800.0, 1807801088.0), "01e217c7dd44", ("k_particles.cu", "pm_internal.cuh")),
}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_replicas(ms_local, n_local, world, device="cpu"):
    """Replicas only: every rank ran its own problem.  Returns (ms_max, total particles,
    updates per second) -- the slowest rank's step time over all ranks' particles."""
    import torch
    t = torch.tensor([ms_local, float(n_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms_max, n_tot = float(mx.item()), float(tot.item())
    else:
        ms_max, n_tot = ms_local, float(n_local)
    return ms_max, int(n_tot), n_tot / (ms_max / 1e3)


# --------------------------------------------------------------- oracle arm
def oracle_sample_cfg(steps_total, budget_s=120.0):
    """A bounded sample of the cfg2 workload: same 2 Mpc/h spacing, boost-2 mesh and
    neutrino-to-CDM ratio in a smaller box, the largest whose steps fit the budget
    (about 10 s, 0.8 s and 0.08 s per FP64 step on one core)."""
    from paper_2007_13394_gb300.pm import RunConfig
    for box, nc, ns, t_est in ((256.0, 128, 16, 10.0), (128.0, 64, 8, 0.8), (64.0, 32, 4, 0.08)):
        if steps_total * t_est <= budget_s or nc == 32:
            return (RunConfig(box=box, nmesh=2 * nc, nc=nc, nsites=ns, nshell=10, nfib=3, m_nu=(0.1 / 3,) * 3),
                    f"{box:g} Mpc/h box, {nc}^3 CDM + {ns}^3 x 70 nu, mesh {2 * nc}^3 (cfg2 density and boost)")


def oracle_run(cfg, n_warm, n_timed):
    """Time the oracle's KDK step (force, kicks, drift) on cfg; returns (s/step, n, cores)."""
    from oracle import background as obg
    from oracle import ic as oic
    from oracle import neutrinos as onu
    from oracle import pm as opm
    from paper_2007_13394_gb300 import inputs
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    plin = oic.linear_power(cfg.omega_m, cfg.h, cfg.ns, cfg.sigma8)
    a0 = 0.01
    noise = inputs.white_noise(cfg.nc, seed=1).astype(np.float64)
    uc, pc = oic.cdm_particles(noise, cfg.box, plin, bg.D(a0), bg.gp(a0))
    _, q, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
    un, pn = oic.neutrino_particles(noise, cfg.box, plin, bg.D(a0), bg.gp(a0), cfg.nsites, cfg.nshell,
                                    cfg.nfib, q, onu.thermal_momentum_scale(bg.kT_nu0, max(cfg.m_nu)),
                                    k_fs=oic.free_streaming_k(list(cfg.m_nu), a0, cfg.omega_m))
    u, p = np.hstack([uc, un]), np.hstack([pc, pn])
    mc, mn = onu.species_masses(cfg.nmesh, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                                bg.omega_nu_poisson, m_shell)
    mass = onu.particle_masses(uc.shape[1], un.shape[1], cfg.nshell, cfg.nfib, mc, mn)
    sched = obg.schedule_paper(max(25, n_warm + n_timed))
    f = opm.force(u, mass, cfg.nmesh, cfg.box, bg.omega_m0)
    t = 0.0
    for i, (a, ah, b) in enumerate(sched[: n_warm + n_timed]):
        t0 = time.perf_counter()
        u, p, f = opm.kdk_step(u, p, f, obg.step_coefficients(bg, a, ah, b), mass, cfg.nmesh, cfg.box,
                               bg.omega_m0)
        if i >= n_warm:
            t += time.perf_counter() - t0
    return t / max(1, n_timed), u.shape[1], 1


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    cfg, desc = oracle_sample_cfg(args.steps + args.warmup)
    sec, n, cores = oracle_run(cfg, args.warmup, args.steps)
    value = n / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cfg2 sample: " + desc, "n_particles": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc + f"; {args.steps} timed KDK steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def fft_reference(ctx, n, reps=10):
    """Our 3D r2c / c2r (the z, y, x passes of pm_fft_r2c / pm_fft_c2r, timed per kernel
    with CUDA events, without the stage calls' layout repacks) beside cuFFT (through
    torch.fft.rfftn / irfftn, out of place) on the same N^3 mesh, ms per transform."""
    import torch
    mesh = torch.randn((n, n, n), dtype=torch.float32, device="cuda")
    out = {"mesh": n}
    c = ctx.fft_r2c(mesh)
    ctx.fft_c2r(c)
    ctx.profile(None)
    for name, fn in (("ours_r2c_ms", lambda: ctx.fft_r2c(mesh)), ("ours_c2r_ms", lambda: ctx.fft_c2r(c))):
        ctx.profile_read(reset=True)
        for _ in range(reps):
            fn()
        prof = ctx.profile_read(reset=True)
        out[name] = round(sum(ms for kind, (ms, _) in prof.items() if kind != "repack") / reps, 4)
    ctx.profile([])
    y = torch.fft.rfftn(mesh)
    torch.fft.irfftn(y, s=mesh.shape)
    for name, fn in (("cufft_r2c_ms", lambda: torch.fft.rfftn(mesh)),
                     ("cufft_c2r_ms", lambda: torch.fft.irfftn(y, s=mesh.shape))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / reps, 4)
    out["note"] = ("ours: z, y, x passes of pm_fft_r2c / pm_fft_c2r (CUDA events per kernel, repacks "
                   "excluded); cuFFT: torch.fft.rfftn / irfftn out of place; reference point only")
    del mesh, c, y
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    from paper_2007_13394_gb300 import build as _build
    from paper_2007_13394_gb300 import inputs, pm, workloads

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    cfg = workloads.PRESETS[args.config]()
    if args.kspace_gradient:
        cfg.flags |= 8
    if args.two_mesh:
        cfg.flags |= 1 | 8
    if args.no_nu:  # the same run without neutrino particles (massless neutrinos)
        cfg = dataclasses.replace(cfg, nsites=0, m_nu=(0.0, 0.0, 0.0))
    ctx = pm.ParticleMesh(cfg)
    n = cfg.n_particles()
    # initial conditions on the GPU from seeded white noise (one independent replica per rank)
    noise = torch.from_numpy(inputs.white_noise(cfg.nc, seed=1 + rank)).cuda()
    a_start = 0.01
    st = ctx.ic(noise, a_start, k_fs=workloads.free_streaming_k(cfg, a_start))
    del noise
    sched = workloads.schedule_paper(max(25, args.warmup + args.steps + 16))
    stream = torch.cuda.current_stream()

    def step(i):
        a0, ah, a1 = sched[i]
        ctx.step(st, a0, ah, a1)

    # warm-up, the first one also profiles every kernel kind to find the dominant one
    ctx.profile(None)
    step(0)
    prof_all = ctx.profile_read()
    ctx.profile([])
    for i in range(1, args.warmup):
        step(i)
    ctx.sync()
    shares = {k: v[0] for k, v in prof_all.items()}
    dominant = max(shares, key=shares.get)
    # timed region: only the dominant kind is bracketed with events (on its launch stream)
    ctx.profile([dominant])
    ctx.profile_read(reset=True)
    launches0 = ctx.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        # the K steps through pm_run: each step's last readout carries the next step's
        # first half kick and drift (same state as K pm_step calls, bit for bit)
        ctx.run(st, sched[args.warmup:args.warmup + args.steps])
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctx.sync()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - launches0
    dom = ctx.profile_read(reset=True).get(dominant, (0.0, 0))
    ctx.profile([])
    # one more steady step with every kernel kind timed: per-kernel algorithmic bandwidth
    peak_bw, _ = peaks()
    ctx.profile(None)
    ctx.profile_read(reset=True)
    base = args.warmup + args.steps
    ctx.run(st, sched[base:base + 3])  # steady steps of the pm_run path, per launch below
    per_kind = {}
    sort_fast, sort_full, movers = ctx.sort_stats()
    for kind, (kms, kn) in ctx.profile_read(reset=True).items():
        # the near-sorted re-sort radix-sorts only the movers
        n_kind = movers if kind.startswith("radix") and sort_fast > 0 and sort_full == 0 else n
        alg_b = algorithmic_bytes(kind, cfg.nmesh, n_kind)
        if kind == "readout_fd4_kick":
            alg_b = run_readout_bytes(cfg.nmesh, n, 3)
        per = kms / kn
        per_kind[kind] = {"launches": kn, "ms_per_launch": round(per, 4),
                          "gbs": round(alg_b / (per / 1e3) / 1e9, 1) if alg_b else None,
                          "frac": round(alg_b / (per / 1e3) / 1e9 / peak_bw, 3) if alg_b else None}
    ctx.profile([])
    ms_max, n_total, value = aggregate_replicas(ms, n, world, device="cuda")

    out = None
    if rank == 0:
        peak, peak_kind = peaks()
        dom_ms = dom[0] / max(1, dom[1])
        alg = algorithmic_bytes(dominant, cfg.nmesh, n)
        if dominant == "readout_fd4_kick":
            alg = run_readout_bytes(cfg.nmesh, n, args.steps)
        achieved = alg / (dom_ms / 1e3) / 1e9 if alg and dom_ms > 0 else None
        key = (dominant, args.config)
        traffic = None
        if key in NCU_TRAFFIC and NCU_TRAFFIC[key][1] == source_digest(NCU_TRAFFIC[key][2]):
            fused, plain = NCU_TRAFFIC[key][0]
            traffic = (fused * (args.steps - 1) + plain) / args.steps  # per launch, like achieved
        roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_source": f"hbm_gbs of {peak_kind}", "algorithmic_bytes_per_launch": alg,
                "ms_per_launch": dom_ms, "launches_timed": dom[1],
                "step_share": shares[dominant] / sum(shares.values())}
        # end to end through the C-ABI with host buffers: copies in, step, copies out, every step
        e2e = None
        if not args.no_e2e and args.config not in ("cfg3", "cfg_mid"):
            # pinned (page-locked) host buffers, viewed as numpy arrays for the C-ABI call
            pinned = {k: torch.empty(st[k].shape, dtype=st[k].dtype, pin_memory=True) for k in ("u", "p", "id", "f")}
            for k, v in pinned.items():
                v.copy_(st[k])
            hu, hp, hid, hf = (pinned[k].numpy() for k in ("u", "p", "id", "f"))
            fv = st["f_valid"]
            k_e2e = max(3, min(args.steps, 10))
            base = args.warmup + args.steps + 3  # after the profiled steady steps
            fv = ctx.step_host(hu, hp, hid, hf, fv, *sched[base % len(sched)])  # warm the host path
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for j in range(k_e2e):
                fv = ctx.step_host(hu, hp, hid, hf, fv, *sched[(base + 1 + j) % len(sched)])
            t_e2e = (time.perf_counter() - t0) / k_e2e
            e2e = {"value": n / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 40 * n,
                   "d2h_bytes_per_step": 40 * n, "steps": k_e2e,
                   "note": "pm_step_host: u, p, id, f copied from pinned host memory to the device, "
                           "one KDK step, copied back"}
        fft_ref = None
        if not args.no_fft_reference and args.config not in ("cfg3", "cfg_mid"):  # 2048^3 / 1024^3: skipped
            fft_ref = fft_reference(ctx, cfg.nmesh)
        cpu = None
        if not args.no_cpu_baseline and world == 1 and args.config not in ("cfg3", "cfg_mid"):
            ocfg, desc = oracle_sample_cfg(1)
            sec, n_o, cores = oracle_run(ocfg, 0, 1)
            cpu = {"value": n_o / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": desc + "; one FP64 KDK step (force, kicks, drift)",
                   "host_cores_available": os.cpu_count()}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.config}: {cfg.box:g} Mpc/h, {cfg.nc}^3 CDM + {cfg.nsites}^3 x "
                                   f"{cfg.nshell * (2 * cfg.nfib + 1)} nu (M_nu = {sum(cfg.m_nu):g} eV), "
                                   f"mesh {cfg.nmesh}^3, one KDK PM step",
                       "n_particles": n, "nmesh": cfg.nmesh, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (padded force mesh of "
                             f"{cfg.nmesh ** 2 * (cfg.nmesh // 2 + 2) * 8 / 1e6:.0f} MB, particles "
                             f"{40 * n / 1e6:.0f} MB)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "sort": {"near_sorted_steps": sort_fast, "from_scratch_steps": sort_full,
                     "movers_last_step": movers},
            "fft_reference": fft_ref,
            "clocks": clk.summary(), "kernels_steady_step": per_kind,
        }
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["cfg1", "cfg2", "cfg2_parity", "cfg_mid", "cfg3"], default="cfg2")
    ap.add_argument("--kspace-gradient", action="store_true",
                    help="gradient in k-space with three inverse transforms (flags bit 3)")
    ap.add_argument("--two-mesh", action="store_true",
                    help="k-space gradient one component at a time (flags bits 0 and 3)")
    ap.add_argument("--no-nu", action="store_true",
                    help="the same workload without neutrino particles (massless neutrinos)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fft-reference", action="store_true", help="skip the FFT beside cuFFT")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
