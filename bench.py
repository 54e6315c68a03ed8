"""Benchmark of the MPS lattice Boltzmann step on GB300.

Default workload (the configuration the metric is quoted on): porous medium,
128^3 D3Q19 BGK, tau = 0.7, seeded sphere pack (radius 10 cells, 35 % solid,
periodic), mask compressed as an MPS (chi_mask = 64), body force 1e-5 along x
standing in for the pressure drive, chi_max = 64, FP32 storage and contractions
with FP64 singular-value tails, variational products (2 sweeps), and a smooth
rank-saturating start (31 seeded Fourier modes of density and velocity, so
bonds sit at chi from the first step).

Prints one JSON line (rank 0):
  value      represented MLUPS = N^3 * steps / device seconds, all ranks
  e2e        the same through the C ABI with the populations copied host ->
             device before and device -> host after every step
  roofline   dominant kernel class of one profiled step against its peak
  cpu_baseline  the CPU oracle on a bounded sample of the same step
  clocks     nvidia-smi samples taken during the timed region
  batched    eight 64^3 simulations stepped in one graph, against the same
             eight one after another and one plain FP64 full-SVD simulation

--impl reference times the CPU oracle instead (the reference arm).
Multi-GPU: independent replicas, one per rank (nothing is exchanged).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "porous128": dict(n=7, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                      chi=64, eps=1e-7, chi_mask=64, eps_mask=1e-8, precision=1, geometry="spheres",
                      radius=10.0, solid_fraction=0.35, geo_seed=0, n_modes=31, mode_seed=0),
    # same chi and per-job matrix shapes as porous128 on 64^3 (for kernel captures)
    "porous64": dict(n=6, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                     chi=64, eps=1e-7, chi_mask=64, eps_mask=1e-8, precision=1, geometry="spheres",
                     radius=5.0, solid_fraction=0.35, geo_seed=0, n_modes=31, mode_seed=0),
    # Taylor-Green vortex, 256^3, Re = 800 at u0 = 0.05 (nu = u0 (N / 2 pi) / Re)
    "tgv256": dict(n=8, lattice=19, tau=0.5 + 3.0 * 0.05 * (256 / (2 * 3.141592653589793)) / 800.0,
                   periodic=(1, 1, 1), force=(0.0, 0.0, 0.0), chi=64, eps=1e-7, chi_mask=1, eps_mask=1e-12,
                   precision=1, geometry=None, n_modes=0, mode_seed=0, tgv_u0=0.05),
    # branching vessel, 256^3: binary tree of cylinders (depth 4, Murray radii
    # from 24 cells, bifurcation half-angles 25-45 deg), body force along the
    # root axis in the fluid; FP32 storage and contractions (no BF16 path)
    "vessel256": dict(n=8, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                      chi=128, eps=1e-7, chi_mask=128, eps_mask=1e-8, precision=1, geometry="vessel",
                      radius=24.0, depth=4, geo_seed=0, n_modes=31, mode_seed=0),
    # the vessel's per-job shapes (chi 128: 256-wide centre matrices, Jacobi in
    # global memory) on 64^3, for kernel captures
    "vessel64": dict(n=6, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                     chi=128, eps=1e-7, chi_mask=128, eps_mask=1e-8, precision=1, geometry="vessel",
                     radius=6.0, depth=4, geo_seed=0, n_modes=31, mode_seed=0),
    "channel32": dict(n=5, lattice=19, tau=0.8, periodic=(1, 1, 0), force=(1e-6, 0.0, 0.0),
                      chi=16, eps=1e-10, chi_mask=1, eps_mask=1e-12, precision=0, geometry=None,
                      n_modes=0, mode_seed=0),
}

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 SIMT throughput of cuBLAS SGEMM (no TF32) measured on this machine's GB300
# (8192^3, CUDA events): the peak used for the FP32 SIMT contraction kernels.
FP32_SIMT_MEASURED_TFLOPS = 69.8


def geometry(w):
    import synth
    if w["geometry"] == "spheres":
        return synth.sphere_pack(w["n"], w["radius"], w["solid_fraction"], w["geo_seed"])
    if w["geometry"] == "vessel":
        return synth.vessel_tree(w["n"], w["radius"], w["depth"], w["geo_seed"])
    return None


def make_sim(w, solid, modes):
    import paper_2512_07615_gb300 as tl
    return tl.Sim(w["n"], lattice=w["lattice"], tau=w["tau"], periodic=w["periodic"], solid=solid,
                  chi_mask=w["chi_mask"], eps_mask=w["eps_mask"], force=w["force"], chi_max=w["chi"],
                  eps=w["eps"], precision=w["precision"], hadamard=0, sweeps=2, modes=modes,
                  conserve_mass=w["precision"] != 0)


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.f.read().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(w, solid, modes, budget_s=25.0, pops=None):
    """Time the oracle on the first phases of the same step (moments, rho_0,
    Taylor 1/rho, velocity and second-order products: roundings and fits of
    the real populations) and extrapolate to one whole step by the step's
    counts of roundings and fits.  pops: the populations (lists of cores) of
    the state the GPU timed, else the workload's initial state.  Returns
    (seconds per step, description, seconds spent)."""
    import oracle.mps as M
    import oracle.mps_lbm as ml
    from oracle import lattice as olat
    lat = olat.get("D3Q19" if w["lattice"] == 19 else "D3Q15")
    # job counts of one step, from a dry run of the step's structure on 2^3 cells
    cnt = {"round": 0, "fit": 0}
    r0, f0 = M.lincomb_round, M.hadamard_fit

    def c_round(*a, **k):
        cnt["round"] += 1
        return r0(*a, **k)

    def c_fit(*a, **k):
        cnt["fit"] += 1
        return f0(*a, **k)

    M.lincomb_round, M.hadamard_fit = c_round, c_fit
    try:
        tiny_mask = M.scale(M.ones(3), 0.1) if solid is not None else None
        tcfg = ml.Config(1, lat, w["tau"], force=w["force"], periodic=w["periodic"], chi_max=4,
                         eps=w["eps"], hadamard="fit", mask=tiny_mask)
        ml.step(tcfg, ml.initial_rest(tcfg))
    finally:
        M.lincomb_round, M.hadamard_fit = r0, f0
    n_round, n_fit = cnt["round"], cnt["fit"]
    # the real populations of the workload (setup, not timed)
    cfg = ml.Config(w["n"], lat, w["tau"], force=w["force"], periodic=w["periodic"], chi_max=w["chi"],
                    eps=w["eps"], hadamard="fit", mask=None)
    if pops is not None:
        f = [[np.asarray(c, dtype=np.float64) for c in x] for x in pops]
    else:
        f = ml.initial_perturbed(cfg, modes) if modes is not None else ml.initial_rest(cfg)
    t_round, t_fit = [], []
    t_start = time.perf_counter()
    # a1: moments
    items = [(1.0, f[i]) for i in range(lat.Q)]
    rho = None
    while len(items) > 1 and time.perf_counter() - t_start < budget_s:
        nxt = []
        for p in range(0, len(items) - 1, 2):
            t = time.perf_counter()
            nxt.append((1.0, M.lincomb_round([items[p], items[p + 1]], cfg.chi, cfg.eps)))
            t_round.append(time.perf_counter() - t)
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
    rho = items[0][1]
    # a3-a5 style products on the same fields
    one = M.ones(cfg.L)
    rho0 = M.inner_ones(rho) / float(cfg.N ** 3)
    t = time.perf_counter()
    drho = M.lincomb_round([(1.0, rho), (-rho0, one)], cfg.chi, cfg.eps)
    t_round.append(time.perf_counter() - t)
    fac = [drho] + [f[i] for i in range(1, 4)]
    for k in range(len(fac)):
        if time.perf_counter() - t_start > budget_s and t_fit:
            break
        t = time.perf_counter()
        M.hadamard_fit(fac[k], drho, 2)
        t_fit.append(time.perf_counter() - t)
    per_step = n_round * float(np.mean(t_round)) + n_fit * float(np.mean(t_fit))
    desc = ("oracle (numpy FP64) on %d roundings and %d fits of the same step (moments tree and "
            "products of the %s populations), extrapolated to the step's %d roundings and %d fits"
            % (len(t_round), len(t_fit), "timed" if pops is not None else "initial", n_round, n_fit))
    return per_step, desc, time.perf_counter() - t_start


BATCH_CHIS = (32, 48, 64, 40, 56, 32, 64, 48)


def batch_configs(precision=1, chis=BATCH_CHIS):
    """Eight independent 64^3 porous media (sphere packs of radius 5 at 30 %
    solid, seeds 0-7), chi 32-64, eps 1e-7, smooth seeded starts."""
    import synth
    out = []
    for i, chi in enumerate(chis):
        out.append(dict(n_per_axis=6, tau=0.7, periodic=(1, 1, 1), solid=synth.sphere_pack(6, 5.0, 0.3, i),
                        chi_mask=chi, eps_mask=1e-8, force=(1e-5, 0, 0), chi_max=chi, eps=1e-7,
                        precision=precision, hadamard=0, sweeps=2,
                        modes=synth.fourier_modes(15, 10 + i, kmax=3, amp_rho=1e-3, amp_u=1e-3),
                        conserve_mass=precision == 1))
    return out


def batched_measurement(warmup=2, steps=2):
    """The batched workload: eight simulations stepped in one graph against the
    same eight stepped one after another, and against one plain FP64
    full-SVD simulation of the largest chi."""
    import paper_2512_07615_gb300 as tl
    N3 = 64 ** 3
    cfgs = batch_configs()
    b = tl.Batch(cfgs)
    info = b.info()
    b.step(warmup)
    ms = b.step_timed(steps) / steps
    b.close()
    seq = 0.0
    for c in cfgs:
        c = dict(c)
        n = c.pop("n_per_axis")
        s = tl.Sim(n, **c)
        s.step(1)
        seq += s.step_timed(1)
        s.close()
    c = dict(batch_configs(precision=0)[2])
    n = c.pop("n_per_axis")
    s = tl.Sim(n, **c)
    s.step(1)
    ms64 = s.step_timed(1)
    s.close()
    return {"workload": "batched8_porous64: eight 64^3 sphere packs (seeds 0-7), chi %s, eps 1e-7, FP32"
                        % "/".join(map(str, BATCH_CHIS)),
            "value": len(cfgs) * N3 / (ms * 1e3), "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "launches_per_step": info["launches_per_step"],
            "jobs_per_step": info["jobs_per_step"],
            "unbatched_value": len(cfgs) * N3 / (seq * 1e3), "unbatched_ms_per_round": seq,
            "fp64_unbatched_full_svd_value": N3 / (ms64 * 1e3), "fp64_chi": cfgs[2]["chi_max"]}


MIXED_SIZES = (6, 7, 8, 6, 7, 6, 8, 7)
MIXED_CHIS = (32, 64, 128)


def mixed_batch_configs():
    """Eight simulations of uneven size: 64^3 / 128^3 / 256^3 in the order of
    MIXED_SIZES, chi cycling 32 / 64 / 128; even seeds are sphere packs (radius
    10 cells per 128, 35 % solid), odd seeds branching vessels (root radius 24
    cells per 256, depth 4); FP32, eps 1e-7, seeded smooth starts."""
    import synth
    out = []
    for i, n in enumerate(MIXED_SIZES):
        N = 1 << n
        chi = MIXED_CHIS[i % 3]
        solid = synth.sphere_pack(n, 10.0 * N / 128, 0.35, i) if i % 2 == 0 else \
            synth.vessel_tree(n, 24.0 * N / 256, 4, i)
        out.append(dict(n_per_axis=n, tau=0.7, periodic=(1, 1, 1), solid=solid, chi_mask=chi, eps_mask=1e-8,
                        force=(1e-5, 0, 0), chi_max=chi, eps=1e-7, precision=1, hadamard=0, sweeps=2,
                        modes=synth.fourier_modes(31, i, kmax=4, amp_rho=1e-3, amp_u=1e-3), conserve_mass=True))
    return out


def mixed_batch_measurement(warmup=1, steps=2):
    """The uneven batch stepped in one graph against the same simulations
    stepped one after another (one step each, after one untimed step)."""
    import paper_2512_07615_gb300 as tl
    cfgs = mixed_batch_configs()
    cells = sum((1 << c["n_per_axis"]) ** 3 for c in cfgs)
    b = tl.Batch(cfgs)
    info = b.info()
    b.step(warmup)
    ms = b.step_timed(steps) / steps
    bonds = [s.stats()["max_bond"] for s in b.sims]
    b.close()
    alone = []
    for c in cfgs:
        c = dict(c)
        n = c.pop("n_per_axis")
        s = tl.Sim(n, **c)
        s.step(1)
        alone.append(s.step_timed(1))
        s.close()
    return {"workload": "mixed8: sizes %s^3, chi %s cycling, sphere packs (even seeds) and vessels (odd seeds), "
                        "FP32" % ("/".join(str(1 << n) for n in MIXED_SIZES), "/".join(map(str, MIXED_CHIS))),
            "value": cells / (ms * 1e3), "unit": "MLUPS", "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "launches_per_step": info["launches_per_step"], "jobs_per_step": info["jobs_per_step"],
            "max_bonds": bonds, "unbatched_ms_per_round": sum(alone), "unbatched_ms_each": alone,
            "unbatched_value": cells / (sum(alone) * 1e3)}


def max_over_ranks(x, world, device):
    """Max of a per-rank float over all ranks (replicas are timed by the
    slowest one); identity for one process."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms, world, cells, steps):
    """Whole-job represented MLUPS: every rank steps its own replica of
    `cells` cells `steps` times; ms is the max over ranks of the timed region."""
    return world * cells * steps / (ms / 1e3) / 1e6


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="porous128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "fp32", "tf32"], default=None,
                    help="override the workload's precision (tf32: FP32 storage, fit contractions on the "
                         "tensor cores with TF32 operands)")
    ap.add_argument("--batched-mixed", action="store_true",
                    help="also time the eight uneven simulations (64^3-256^3, chi 32-128) in one graph")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["precision"] = {"fp64": 0, "fp32": 1, "tf32": 2}[args.precision]
    N3 = float((1 << w["n"]) ** 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import synth
    if w.get("tgv_u0"):
        modes = synth.taylor_green_modes(w["tgv_u0"])
    else:
        modes = synth.fourier_modes(w["n_modes"], w["mode_seed"], kmax=4, amp_rho=1e-3, amp_u=1e-3) \
            if w["n_modes"] > 0 else None
    solid = geometry(w)
    config = {"workload": args.workload, "lattice": "D3Q%d" % w["lattice"], "cells": "%d^3" % (1 << w["n"]),
              "chi_max": w["chi"], "chi_mask": w["chi_mask"] if solid is not None else None,
              "eps": w["eps"], "tau": w["tau"], "products": "variational fit, 2 sweeps",
              "storage": "fp64" if w["precision"] == 0 else "fp32",
              "contractions": {0: "fp64 SIMT", 1: "fp32 SIMT", 2: "tf32 tensor cores (fit), fp32 SIMT (rounding)"}[
                  w["precision"]],
              "mass_correction": w["precision"] != 0,
              "start": ("Taylor-Green vortex u0 = %g" % w["tgv_u0"]) if w.get("tgv_u0") else
                       ("%d seeded Fourier modes" % w["n_modes"] if w["n_modes"] else "rest"),
              "l2_flush": "working set > L2 (129 MB) is not claimed; each step touches ~GBs of environments"}

    if args.impl == "reference":
        if rank != 0:
            return
        per = []
        desc = ""
        for i in range(args.warmup + args.steps):
            sec, desc, _ = oracle_sample(w, solid, modes, budget_s=8.0)
            if i >= args.warmup:
                per.append(sec)
        T = float(np.sum(per))
        val = N3 * args.steps / T / 1e6
        out = {"impl": "reference", "metric": "represented MLUPS at fixed chi", "value": val, "unit": "MLUPS",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
               "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
                                "sample": desc},
               "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_07615_gb300 as tl
    from paper_2512_07615_gb300 import native as nat

    t0 = time.time()
    sim = make_sim(w, solid, modes)
    setup_s = time.time() - t0
    rho_start, _ = sim.macroscopic()
    mass_start = float(rho_start.sum())
    sim.step(args.warmup)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as clk:
        ms = sim.step_timed(args.steps)
    barrier()
    clocks = clk.summary()
    ms = max_over_ranks(ms, world, "cuda")
    st = sim.stats()
    value = replica_value(ms, world, N3, args.steps)
    rho_end, _ = sim.macroscopic()
    mass_drift = abs(float(rho_end.sum()) - mass_start) / mass_start

    # one profiled (eager, serialised) step: per kernel class time and FLOPs
    prof = sim.profile_step()
    round_phases = prof["round"].pop("phase_cycles")
    total_prof_ms = sum(v["ms"] for v in prof.values())
    dom = max(prof, key=lambda c: prof[c]["ms"])
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    fp32 = w["precision"] != 0
    if fp32:
        peak_tf, peak_src = FP32_SIMT_MEASURED_TFLOPS, "measured FP32 SIMT SGEMM on this pool (no TF32)"
    else:
        peak_tf, peak_src = 1.06, "measured FP64 DGEMM on this pool"
    launches = max(prof[dom]["launches"], 1)
    # DRAM bytes of the rounding kernel: ncu (dram__bytes_read.sum +
    # dram__bytes_write.sum) on the porous 64^3 workload at chi 64 measured
    # 1.156 MB for a launch of 4 jobs; scaled by the jobs of an average
    # launch here (each job reads its terms and writes its result).  Only for
    # the FP32 chi-64 sphere packs it was measured on.
    traffic = None
    if dom == "round" and fp32 and w["chi"] == 64 and w["geometry"] == "spheres":
        traffic = 1.156e6 / 4 * st["round_jobs_per_step"] / launches
    ach = prof[dom]["flops"] / (prof[dom]["ms"] / 1e3) / 1e12 if prof[dom]["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": traffic,
                "traffic_source": ("ncu DRAM bytes per rounding job (porous 64^3, chi 64) x jobs per launch"
                                   if traffic is not None else None),
                "peak_source": peak_src,
                "flops_per_launch": prof[dom]["flops"] / launches, "launches_per_step": prof[dom]["launches"],
                "share_of_profiled_step": prof[dom]["ms"] / total_prof_ms if total_prof_ms else None,
                "classes": {c: {"ms": round(v["ms"], 3), "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12
                                                                    if v["ms"] > 0 else 0.0),
                                "launches": v["launches"]} for c, v in prof.items()},
                "round_phase_share": {p: round(round_phases[p] / max(sum(round_phases[q] for q in
                                      ("terms", "gemm_rw", "qr", "jacobi", "svd_out", "gemm_qus")), 1.0), 4)
                                      for p in ("terms", "gemm_rw", "qr", "jacobi", "svd_out", "gemm_qus")},
                "jacobi_sweeps_per_svd": round_phases["jacobi_sweeps"] / max(round_phases["svd_count"], 1.0)}
    if w["precision"] == 2 and prof["fit_gemm"]["ms"] > 0:
        # the fit's GEMM stages on the tensor cores: against the TF32 peak, taken
        # as the measured BF16 burst peak times the nominal TF32 / BF16 ratio
        tf32_peak = peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25
        ach_tc = prof["fit_gemm"]["flops"] / (prof["fit_gemm"]["ms"] / 1e3) / 1e12
        roofline["tensor"] = {"kernel": "fit_gemm_tc", "bound": "tensor", "achieved": ach_tc, "peak": tf32_peak,
                              "unit": "TFLOP/s", "frac": ach_tc / tf32_peak,
                              "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}

    # end to end through the C ABI: populations host -> device, step, device -> host
    e2e = None
    if not args.no_e2e:
        pops = sim.get_populations()
        L = 3 * w["n"]
        ms_size = tl.tnlbm.mps_size(L, w["chi"])
        bytes_io = w["lattice"] * (ms_size * 8 + (L + 1) * 4)
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            sim.set_populations(pops)
            sim.step(1)
            pops = sim.get_populations()
        barrier()
        el_ms = max_over_ranks((time.perf_counter() - t) * 1e3, world, "cuda")
        e2e = {"value": replica_value(el_ms, world, N3, args.steps), "unit": "MLUPS",
               "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sec, desc, spent = oracle_sample(w, solid, modes, pops=sim.get_populations())
        cpu = {"value": N3 / sec / 1e6, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
               "sample": desc, "sample_seconds": round(spent, 1)}

    batched = None
    if rank == 0 and not args.no_batched and args.workload == "porous128":
        batched = batched_measurement()
    batched_mixed = None
    if rank == 0 and args.batched_mixed:
        batched_mixed = mixed_batch_measurement()

    if rank == 0:
        out = {"metric": "represented MLUPS at fixed chi", "value": value, "unit": "MLUPS",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": ("tf32" if w["precision"] == 2 else "f32") if fp32 else "f64", "data": "synthetic", "config": config,
               "gpu_launches": st["gpu_launches_per_step"] * args.steps,
               "bonds": {"max": st["max_bond"], "mean": round(st["mean_bond"], 2)},
               "compression_ratio": st["compression_ratio"], "setup_s": round(setup_s, 2),
               "mass_drift": mass_drift, "mass_drift_steps": args.warmup + args.steps,
               "clocks": clocks, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
               "batched": batched, "batched_mixed": batched_mixed}
        print(json.dumps(out))
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
