"""Benchmark of the MPS lattice Boltzmann step on GB300.

Default workload (the configuration the metric is quoted on): porous medium,
128^3 D3Q19 BGK, tau = 0.7, seeded sphere pack (radius 10 cells, 35 % solid,
periodic), mask compressed as an MPS (chi_mask = 64), body force 1e-5 along x
standing in for the pressure drive, chi_max = 64, precision TNLBM_MIXED (FP32
cores, contractions and QR sweeps; every centre SVD an FP64 one-sided Jacobi
shared by a thread-block cluster), variational products (2 sweeps), and a
smooth rank-saturating start (31 seeded Fourier modes of density and
velocity, so bonds sit at chi from the first step).

Prints one JSON line (rank 0):
  value        represented MLUPS = N^3 * steps / device seconds, all ranks
  vs_baseline  value / that of the plain FP64 unbatched full-SVD GPU path on the
               same workload (the baseline the metric names)
  rel_l2_u     ||u - u_64|| / ||u_64|| against that FP64 path after the same
               steps from the same start
  e2e          the same metric through the C ABI with the populations copied
               host -> device before and device -> host after every step
  roofline     the rounding kernel (the dominant one) against its peak
  cpu_baseline the CPU oracle timed on one whole step of the timed state
  clocks       nvidia-smi samples taken during the timed region
  batched      eight 64^3 simulations stepped in one graph (mixed precision,
               cluster sizes tuned per level) against the same eight stepped
               one after another, in mixed precision and in plain FP64

--impl reference times the CPU oracle instead (the reference arm): one oracle
step of the workload's start is recorded call by call (roundings and products
with their inputs), and every bench step replays a fifth of those calls, so
that 5 bench steps re-run one whole oracle step.
--probe-peaks measures the FP32 (no TF32), TF32 and FP64 GEMM peaks with
torch.matmul (the record the roofline reads is profiles/peaks_gb300.md).
Multi-GPU: independent replicas, one per rank (nothing is exchanged).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "mixed": 3, "bf16": 4}
PREC_NAME = {v: k for k, v in PREC.items()}

WORKLOADS = {
    "porous128": dict(n=7, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                      chi=64, eps=1e-7, chi_mask=64, eps_mask=1e-8, precision=3, geometry="spheres",
                      radius=10.0, solid_fraction=0.35, geo_seed=0, n_modes=31, mode_seed=0),
    # same chi and per-job matrix shapes as porous128 on 64^3 (for kernel captures)
    "porous64": dict(n=6, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                     chi=64, eps=1e-7, chi_mask=64, eps_mask=1e-8, precision=3, geometry="spheres",
                     radius=5.0, solid_fraction=0.35, geo_seed=0, n_modes=31, mode_seed=0),
    # Taylor-Green vortex, 256^3, Re = 800 at u0 = 0.05 (nu = u0 (N / 2 pi) / Re)
    "tgv256": dict(n=8, lattice=19, tau=0.5 + 3.0 * 0.05 * (256 / (2 * 3.141592653589793)) / 800.0,
                   periodic=(1, 1, 1), force=(0.0, 0.0, 0.0), chi=64, eps=1e-7, chi_mask=1, eps_mask=1e-12,
                   precision=3, geometry=None, n_modes=0, mode_seed=0, tgv_u0=0.05),
    # branching vessel, 256^3: binary tree of cylinders (depth 4, Murray radii
    # from 24 cells, bifurcation half-angles 25-45 deg), body force along the
    # root axis in the fluid
    "vessel256": dict(n=8, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                      chi=128, eps=1e-7, chi_mask=128, eps_mask=1e-8, precision=3, geometry="vessel",
                      radius=24.0, depth=4, geo_seed=0, n_modes=31, mode_seed=0),
    # the vessel's per-job shapes (chi 128: 256-wide centre matrices) on 64^3, for kernel captures
    "vessel64": dict(n=6, lattice=19, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0),
                     chi=128, eps=1e-7, chi_mask=128, eps_mask=1e-8, precision=3, geometry="vessel",
                     radius=6.0, depth=4, geo_seed=0, n_modes=31, mode_seed=0),
    "channel32": dict(n=5, lattice=19, tau=0.8, periodic=(1, 1, 0), force=(1e-6, 0.0, 0.0),
                      chi=16, eps=1e-10, chi_mask=1, eps_mask=1e-12, precision=0, geometry=None,
                      n_modes=0, mode_seed=0),
}

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
PEAKS_RECORD = os.path.join(ROOT, "profiles", "peaks_gb300.md")


def load_peaks():
    """HBM and BF16 peaks from the driver's record; FP32 (no TF32), TF32 and
    FP64 GEMM peaks from the committed probe record (key = value lines)."""
    peaks = {}
    if os.path.exists(MEASURED_PEAKS):
        peaks.update(json.load(open(MEASURED_PEAKS)))
    if os.path.exists(PEAKS_RECORD):
        for line in open(PEAKS_RECORD):
            line = line.strip().strip("`")
            if "=" in line and not line.startswith("#"):
                k, v = [t.strip() for t in line.split("=", 1)]
                try:
                    peaks[k] = float(v.split()[0])
                except ValueError:
                    pass
    return peaks


def probe_peaks():
    """FP32 (TF32 off), TF32 and FP64 dense GEMM throughput with torch.matmul,
    CUDA events, best of 5 after 2 warm-up products."""
    import torch
    torch.cuda.set_device(0)
    out = {}
    for name, dt, n, tf32 in (("fp32_simt_tflops", torch.float32, 8192, False),
                              ("tf32_tflops", torch.float32, 8192, True),
                              ("fp64_tflops", torch.float64, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(2):
            torch.matmul(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        print("%s = %.1f   (torch.matmul %s %d^3, TF32 %s, best of 5: %.3f ms)"
              % (name, out[name], str(dt).replace("torch.", ""), n, "on" if tf32 else "off", best))
    torch.backends.cuda.matmul.allow_tf32 = False
    return out


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
                  conserve_mass=w["precision"] != 0, max_cluster=w.get("max_cluster", 0))


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


# ------------------------------------------------------------------ CPU oracle
def oracle_config(w, solid):
    """The oracle's configuration of the workload (products by the fit; the
    mask MPS by the oracle's own TT-SVD of the voxels at chi_mask / eps_mask)."""
    import oracle.mps as M
    import oracle.mps_lbm as ml
    from oracle import lattice as olat, quantics as q
    lat = olat.get("D3Q19" if w["lattice"] == 19 else "D3Q15")
    mask = M.tt_svd(q.encode(solid.astype(np.float64)), w["chi_mask"], w["eps_mask"]) if solid is not None else None
    return ml.Config(w["n"], lat, w["tau"], force=w["force"], periodic=w["periodic"], chi_max=w["chi"],
                     eps=w["eps"], hadamard="fit", mask=mask)


def oracle_start(cfg, modes):
    import oracle.mps_lbm as ml
    return ml.initial_perturbed(cfg, modes) if modes is not None else ml.initial_rest(cfg)


def oracle_whole_step(w, solid, pops):
    """Seconds of one whole oracle step (oracle.mps_lbm.step: moments, Taylor
    1/rho, products, collision, streaming, walls and object bounce-back with
    the mask products) on the given populations (lists of cores)."""
    import oracle.mps_lbm as ml
    cfg = oracle_config(w, solid)
    f = [[np.asarray(c, dtype=np.float64) for c in x] for x in pops]
    t = time.perf_counter()
    ml.step(cfg, f)
    return time.perf_counter() - t


class OracleReplay:
    """One oracle step recorded call by call: every rounding (lincomb_round)
    and product (hadamard_fit) with its inputs and its duration; replay(c)
    re-runs the calls of chunk c of `parts` contiguous chunks of about equal
    recorded time and returns (seconds, fraction of the step's recorded time)."""

    def __init__(self, w, solid, modes, parts=5):
        import oracle.mps as M
        import oracle.mps_lbm as ml
        cfg = oracle_config(w, solid)
        f = oracle_start(cfg, modes)
        calls = []
        r0, f0 = M.lincomb_round, M.hadamard_fit

        def rec(fn):
            def wrapped(*a, **k):
                t = time.perf_counter()
                out = fn(*a, **k)
                calls.append((fn, a, k, time.perf_counter() - t))
                return out
            return wrapped

        M.lincomb_round, M.hadamard_fit = rec(r0), rec(f0)
        try:
            t = time.perf_counter()
            ml.step(cfg, f)
            self.record_s = time.perf_counter() - t
        finally:
            M.lincomb_round, M.hadamard_fit = r0, f0
        total = sum(c[3] for c in calls)
        self.chunks, self.frac = [], []
        acc, cur, cur_t = 0.0, [], 0.0
        for c in calls:
            cur.append(c)
            cur_t += c[3]
            acc += c[3]
            if acc >= total * (len(self.chunks) + 1) / parts and len(self.chunks) < parts - 1:
                self.chunks.append(cur)
                self.frac.append(cur_t / total)
                cur, cur_t = [], 0.0
        self.chunks.append(cur)
        self.frac.append(cur_t / total)
        self.ncalls = len(calls)

    def replay(self, c):
        c %= len(self.chunks)
        t = time.perf_counter()
        for fn, a, k, _ in self.chunks[c]:
            fn(*a, **k)
        return time.perf_counter() - t, self.frac[c]


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
                        conserve_mass=precision != 0))
    return out


def batched_measurement(precision=3, warmup=1, steps=2, tune=True):
    """The batched workload: eight 64^3 simulations stepped in one graph, with
    the cluster sizes of the occupancy rule and after the per-level tuner,
    against the same eight stepped one after another in this precision and in
    the plain FP64 full-SVD path (one untimed step each, then one timed)."""
    import paper_2512_07615_gb300 as tl
    N3 = 64 ** 3
    cfgs = batch_configs(precision)
    b = tl.Batch(cfgs)
    info = b.info()
    sizes0, jobs = b.clusters()
    b.step(1)
    ms0 = b.step_timed(1)
    tuned = None
    if tune and precision in (0, 3, 4):
        t = time.perf_counter()
        r = b.tune_clusters(reps=1)
        tuned = {"tune_s": round(time.perf_counter() - t, 2), "sizes": r["sizes"], "occupancy_sizes": sizes0,
                 "jobs_per_level": jobs}
    b.step(warmup)
    ms = b.step_timed(steps) / steps
    b.close()

    def alone(prec):
        tot = 0.0
        for c in batch_configs(prec):
            c = dict(c)
            n = c.pop("n_per_axis")
            s = tl.Sim(n, **c)
            s.step(1)
            tot += s.step_timed(1)
            s.close()
        return tot

    seq = alone(precision)
    seq64 = alone(0) if precision != 0 else seq
    cells = len(cfgs) * N3
    return {"workload": "batched8_porous64: eight 64^3 sphere packs (seeds 0-7), chi %s, eps 1e-7, %s"
                        % ("/".join(map(str, BATCH_CHIS)), PREC_NAME[precision]),
            "value": cells / (ms * 1e3), "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "launches_per_step": info["launches_per_step"],
            "jobs_per_step": info["jobs_per_step"],
            "occupancy_rule_value": cells / (ms0 * 1e3), "occupancy_rule_ms_per_step": ms0,
            "cluster_tuning": tuned,
            "unbatched_value": cells / (seq * 1e3), "unbatched_ms_per_round": seq,
            "fp64_unbatched_full_svd_value": cells / (seq64 * 1e3), "fp64_unbatched_ms_per_round": seq64,
            "vs_fp64_unbatched": seq64 / ms}


MIXED_SIZES = (6, 7, 8, 6, 7, 6, 8, 7)
MIXED_CHIS = (32, 64, 128)


def mixed_batch_configs(precision=1):
    """Eight simulations of uneven size: 64^3 / 128^3 / 256^3 in the order of
    MIXED_SIZES, chi cycling 32 / 64 / 128; even seeds are sphere packs (radius
    10 cells per 128, 35 % solid), odd seeds branching vessels (root radius 24
    cells per 256, depth 4); eps 1e-7, seeded smooth starts; FP32 unless
    another precision is given."""
    import synth
    out = []
    for i, n in enumerate(MIXED_SIZES):
        N = 1 << n
        chi = MIXED_CHIS[i % 3]
        solid = synth.sphere_pack(n, 10.0 * N / 128, 0.35, i) if i % 2 == 0 else \
            synth.vessel_tree(n, 24.0 * N / 256, 4, i)
        out.append(dict(n_per_axis=n, tau=0.7, periodic=(1, 1, 1), solid=solid, chi_mask=chi, eps_mask=1e-8,
                        force=(1e-5, 0, 0), chi_max=chi, eps=1e-7, precision=precision, hadamard=0, sweeps=2,
                        modes=synth.fourier_modes(31, i, kmax=4, amp_rho=1e-3, amp_u=1e-3), conserve_mass=True))
    return out


def mixed_batch_measurement(precision=1, warmup=1, steps=2, tune=True):
    """The uneven batch stepped in one graph (cluster sizes tuned per level
    first where the precision runs clusters) against the same simulations
    stepped one after another (one step each, after one untimed step)."""
    import paper_2512_07615_gb300 as tl
    cfgs = mixed_batch_configs(precision)
    cells = sum((1 << c["n_per_axis"]) ** 3 for c in cfgs)
    b = tl.Batch(cfgs)
    info = b.info()
    tuned = None
    if tune and precision in (0, 3, 4):
        b.step(1)                       # bonds at their working size before the sizes are measured
        t = time.perf_counter()
        r = b.tune_clusters(reps=1)
        tuned = {"tune_s": round(time.perf_counter() - t, 2), "sizes": r["sizes"], "jobs_per_level": r["jobs"]}
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
                        "%s" % ("/".join(str(1 << n) for n in MIXED_SIZES), "/".join(map(str, MIXED_CHIS)),
                                PREC_NAME[precision]),
            "cluster_tuning": tuned,
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
def precision_desc(p):
    svd64 = ("fp64 one-sided Jacobi (cluster of CTAs, started from fp32 sweeps made orthogonal by an fp64 "
             "Newton-Schulz step), fp64 norms and tails")
    return {0: dict(storage="fp64", contractions="fp64 SIMT", qr="fp64", svd="fp64 one-sided Jacobi"),
            1: dict(storage="fp32", contractions="fp32 SIMT", qr="fp32 (scaled fp32 column norms)",
                    svd="fp32 one-sided Jacobi, fp64 tails"),
            2: dict(storage="fp32", contractions="tf32 tensor cores (fit), fp32 SIMT (rounding)",
                    qr="fp32 (scaled fp32 column norms)", svd="fp32 one-sided Jacobi, fp64 tails"),
            3: dict(storage="fp32", contractions="fp32 SIMT", qr="fp32 (scaled fp32 column norms)", svd=svd64),
            4: dict(storage="fp32", contractions="bf16 x bf16 -> fp32 tensor cores (fit), fp32 SIMT (rounding)",
                    qr="fp32 (scaled fp32 column norms)", svd=svd64)}[p]


def reference_arm(args, w, solid, modes, config, N3, rank):
    """The CPU oracle as the reference arm: W + K bench steps, each replaying a
    fifth of one recorded oracle step (see OracleReplay)."""
    if rank != 0:
        return
    rep = OracleReplay(w, solid, modes)
    t_tot, cells = 0.0, 0.0
    for i in range(args.warmup + args.steps):
        sec, frac = rep.replay(i)
        if i >= args.warmup:
            t_tot += sec
            cells += frac * N3
    val = cells / t_tot / 1e6
    desc = ("oracle (numpy FP64) step of the workload's start recorded call by call (%d roundings and fits, "
            "%.1f s including its unrecorded glue); each bench step replays one fifth of those calls by "
            "recorded time, so %d bench steps re-ran %.2f whole oracle steps"
            % (rep.ncalls, rep.record_s, args.steps, cells / N3))
    out = {"impl": "reference", "metric": "represented MLUPS at fixed chi", "value": val, "unit": "MLUPS",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
           "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


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
    ap.add_argument("--batched-precision", choices=sorted(PREC), default="mixed",
                    help="precision of the batched eight-simulation leg")
    ap.add_argument("--uneven-precision", choices=sorted(PREC), default="fp32",
                    help="precision of the uneven batch (--batched-mixed)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the occupancy rule's cluster sizes (no per-level tuning)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison (vs_baseline, rel_l2_u)")
    ap.add_argument("--precision", choices=sorted(PREC), default=None,
                    help="override the workload's precision (mixed: FP32 storage and contractions, FP64 SVD)")
    ap.add_argument("--max-cluster", type=int, default=0, help="CTAs per rounding job cap (0 = automatic)")
    ap.add_argument("--batched-mixed", action="store_true",
                    help="also time the eight uneven simulations (64^3-256^3, chi 32-128) in one graph")
    ap.add_argument("--probe-peaks", action="store_true", help="measure the FP32 / TF32 / FP64 GEMM peaks")
    args = ap.parse_args()
    if args.probe_peaks:
        probe_peaks()
        return
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["precision"] = PREC[args.precision]
    w["max_cluster"] = args.max_cluster
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
    pd = precision_desc(w["precision"])
    config = {"workload": args.workload, "lattice": "D3Q19" if w["lattice"] == 19 else "D3Q15",
              "cells": "%d^3" % (1 << w["n"]), "chi_max": w["chi"],
              "chi_mask": w["chi_mask"] if solid is not None else None, "eps": w["eps"], "tau": w["tau"],
              "products": "variational fit, 2 sweeps", "precision": PREC_NAME[w["precision"]], **pd,
              "mass_correction": w["precision"] != 0,
              "start": ("Taylor-Green vortex u0 = %g" % w["tgv_u0"]) if w.get("tgv_u0") else
                       ("%d seeded Fourier modes" % w["n_modes"] if w["n_modes"] else "rest"),
              "l2_flush": "none: each step streams GBs of environments and rounding scratch through HBM"}

    if args.impl == "reference":
        reference_arm(args, w, solid, modes, config, N3, rank)
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

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # plain FP64 unbatched full-SVD path on the same workload: its MLUPS (the
    # baseline the metric names) and the velocity field after n_cmp steps from
    # the same start, against which the timed precision's field is compared
    cmp = None
    n_cmp = 3
    if rank == 0 and not args.no_fp64:
        w64 = dict(w, precision=0)
        s64 = make_sim(w64, solid, modes)
        s64.step(1)
        ms64 = s64.step_timed(1)
        s64.step(n_cmp - 2)
        _, u64 = s64.macroscopic()
        s64.close()
        sx = make_sim(w, solid, modes)
        sx.step(n_cmp)
        _, ux = sx.macroscopic()
        sx.close()
        cmp = {"fp64_ms_per_step": ms64, "fp64_value": N3 / (ms64 * 1e3),
               "rel_l2_u": float(np.linalg.norm(ux - u64) / np.linalg.norm(u64)), "steps": n_cmp}
        # conditioning of the workload: the FP64 path from a start whose mode
        # amplitudes are scaled by 1 + 1e-12
        if modes is not None:
            mp = np.array(modes, dtype=np.float64)
            mp[:, 4:] *= 1.0 + 1e-12
            sp = make_sim(w64, solid, mp)
            sp.step(n_cmp)
            _, up = sp.macroscopic()
            sp.close()
            cmp["rel_l2_u_fp64_perturbed"] = float(np.linalg.norm(up - u64) / np.linalg.norm(u64))
            del up
        del u64, ux

    t0 = time.time()
    sim = make_sim(w, solid, modes)
    setup_s = time.time() - t0
    rho_start, _ = sim.macroscopic()
    mass_start = float(rho_start.sum())
    sim.step(args.warmup)
    tuning = None
    if not args.no_tune and w["precision"] in (0, 3, 4):
        # per-level cluster sizes measured once, after the warm-up steps and
        # before the timed ones (one eager step without its final copy: the
        # state is unchanged), then one more untimed step of the new graph
        sizes0, _ = sim.clusters()
        t0 = time.time()
        r = sim.tune_clusters(reps=1)
        tuning = {"tune_s": round(time.time() - t0, 2), "sizes": r["sizes"], "occupancy_sizes": sizes0}
        sim.step(1)
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
    ph = prof["round"].pop("phase_cycles")
    total_prof_ms = sum(v["ms"] for v in prof.values())
    peaks = load_peaks()
    rd = prof["round"]
    per_launch_ms = rd["ms"] / max(rd["launches"], 1)
    phase_keys = ("terms", "gemm_rw", "qr", "jacobi32", "jacobi", "svd_out", "gemm_qus")
    phase_tot = max(sum(ph[q] for q in phase_keys), 1.0)
    roofline = {"kernel": "round_kernel", "launches_per_step": rd["launches"],
                "ms_per_launch": per_launch_ms,
                "share_of_profiled_step": rd["ms"] / total_prof_ms if total_prof_ms else None,
                "flops_per_launch": rd["flops"] / max(rd["launches"], 1),
                "classes": {c: {"ms": round(v["ms"], 3),
                                "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0),
                                "launches": v["launches"]} for c, v in prof.items()},
                "round_phase_share": {q: round(ph[q] / phase_tot, 4) for q in phase_keys},
                "jacobi_sweeps_per_svd": ph["jacobi_sweeps"] / max(ph["svd_count"], 1.0),
                "traffic": None,
                "traffic_note": "the rounding kernel reads its terms and writes its result once per job; "
                                "DRAM bytes per launch are in profiles/ (ncu), not re-measured per run"}
    if w["precision"] in (0, 3, 4):
        # the centre SVDs are FP64 one-sided Jacobis bound by the FP64 pipes:
        # achieved = the kernel's algorithmic FLOPs (QR, SVD by the Golub-Kahan
        # count, GEMMs) per launch / launch time, against the FP64 GEMM peak
        peak = peaks.get("fp64_tflops")
        ach = rd["flops"] / (rd["ms"] / 1e3) / 1e12 if rd["ms"] > 0 else 0.0
        jac_ms = rd["ms"] * ph["jacobi"] / phase_tot
        roofline.update({"bound": "fp64", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if peak else None,
                         "peak_source": "FP64 torch.matmul on this pool (profiles/peaks_gb300.md)",
                         "svd64_algorithmic_tflops": ph["svd64_flops"] / (jac_ms / 1e3) / 1e12 if jac_ms else None,
                         "svd64_executed_tflops": ph["svd64_exec_flops"] / (jac_ms / 1e3) / 1e12 if jac_ms else None})
        if peak and jac_ms:
            roofline["svd64_executed_frac"] = roofline["svd64_executed_tflops"] / peak
        if w["precision"] == 3 and w.get("geometry") == "spheres":
            # DRAM bytes of one rounding launch: the ncu capture of this kernel
            # on the porous 64^3 workload (1.698 MB for a launch of 4 jobs,
            # profiles/round_kernel_porous64_mixed.md) scaled by the jobs of
            # an average launch of this run
            per_job = 1.698e6 / 4.0
            roofline["traffic"] = per_job * st["round_jobs_per_step"] / max(rd["launches"], 1)
            roofline["traffic_note"] = ("bytes per launch: dram__bytes_read + write of the porous 64^3 capture "
                                        "(0.42 MB per job) x jobs per launch; the kernel is FP64-latency bound, "
                                        "not DRAM bound")
    else:
        peak = peaks.get("fp32_simt_tflops")
        ach = rd["flops"] / (rd["ms"] / 1e3) / 1e12 if rd["ms"] > 0 else 0.0
        roofline.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if peak else None,
                         "peak_source": "FP32 (no TF32) torch.matmul on this pool (profiles/peaks_gb300.md)"})
    if w["precision"] in (2, 4) and prof["fit_gemm"]["ms"] > 0:
        # the fit's contractions on the tensor cores: TF32 against the measured
        # TF32 GEMM peak, BF16 against the driver's measured BF16 burst peak
        if w["precision"] == 2:
            tc_peak, src = peaks.get("tf32_tflops"), "TF32 torch.matmul on this pool (profiles/peaks_gb300.md)"
        else:
            tc_peak, src = peaks.get("bf16_tflops"), "BF16 torch.matmul burst on this pool (MEASURED_PEAKS.json)"
        ach_tc = prof["fit_gemm"]["flops"] / (prof["fit_gemm"]["ms"] / 1e3) / 1e12
        roofline["tensor"] = {"kernel": "fit_gemm_tc", "bound": "tensor", "achieved": ach_tc, "peak": tc_peak,
                              "unit": "TFLOP/s", "frac": ach_tc / tc_peak if tc_peak else None,
                              "peak_source": src}

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
        sec = oracle_whole_step(w, solid, sim.get_populations())
        cpu = {"value": N3 / sec / 1e6, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
               "sample": "one whole oracle step (numpy FP64, mask products included) on the populations the "
                         "GPU reached after its timed steps (%.1f s)" % sec}

    batched = None
    if rank == 0 and not args.no_batched and args.workload == "porous128":
        batched = batched_measurement(PREC[args.batched_precision], tune=not args.no_tune)
    batched_mixed = None
    if rank == 0 and args.batched_mixed:
        batched_mixed = mixed_batch_measurement(PREC[args.uneven_precision], tune=not args.no_tune)

    if rank == 0:
        out = {"metric": "represented MLUPS at fixed chi", "value": value, "unit": "MLUPS",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
               "higher_is_better": True, "scaling": "weak",
               "vs_baseline": (value / world) / cmp["fp64_value"] if cmp else None,
               "vs_baseline_def": "per-GPU value / MLUPS of the plain FP64 unbatched full-SVD GPU path on the "
                                  "same workload (fp64_baseline)",
               "rel_l2_u": cmp["rel_l2_u"] if cmp else None,
               "rel_l2_u_def": ("||u - u_fp64|| / ||u_fp64|| after %d steps from the same start, u_fp64 from the "
                                "plain FP64 GPU path" % n_cmp) if cmp else None,
               "rel_l2_u_fp64_perturbed": cmp.get("rel_l2_u_fp64_perturbed") if cmp else None,
               "rel_l2_u_fp64_perturbed_def": "the same distance between the FP64 path and the FP64 path started "
                                              "from mode amplitudes scaled by 1 + 1e-12 (the workload's own "
                                              "sensitivity: chi-capped bonds and variational products)",
               "fp64_baseline": ({"value": cmp["fp64_value"], "unit": "MLUPS", "ms_per_step": cmp["fp64_ms_per_step"]}
                                 if cmp else None),
               "dtype": {0: "f64", 1: "f32", 2: "tf32", 3: "f32+f64svd", 4: "bf16+f32+f64svd"}[w["precision"]],
               "data": "synthetic", "config": config,
               "gpu_launches": st["gpu_launches_per_step"] * args.steps,
               "bonds": {"max": st["max_bond"], "mean": round(st["mean_bond"], 2)},
               "rounding_launch": {"jobs_per_step": st["round_jobs_per_step"], "ctas_per_step": st["round_ctas_per_step"],
                                   "max_cluster": st["max_cluster"], "cluster_tuning": tuning},
               "compression_ratio": st["compression_ratio"], "setup_s": round(setup_s, 2),
               "mass_drift": mass_drift, "mass_drift_steps": args.warmup + args.steps + (1 if tuning else 0),
               "clocks": clocks, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
               "batched": batched, "batched_mixed": batched_mixed}
        print(json.dumps(out))
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
