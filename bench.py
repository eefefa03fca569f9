#!/usr/bin/env python
"""Throughput of the coupled electrohydrodynamic lattice step on GB300.

Workload: the dielectric droplet of the model (arXiv:1712.08494 Sec. III.B
geometry, 3D): 128^3 periodic box, two Shan-Chen components (G = 4, tau = 1),
blue drop of radius 24 at the centre, +-1% seeded density noise, two
monovalent ion species at 1e-3, D = 0.05, Bjerrum length 0.4, permittivity
ratio 2, applied field 1e-3 along z, Poisson relative residual 1e-6.  A step
is one full coupled timestep (macro fields, Poisson solve, forces and ion
fluxes, Nernst-Planck update, collision, streaming).

Prints one JSON line: FP32 MLUPS (value), BF16-storage MLUPS and its speedup
and deviation from the FP32 run, the roofline of the dominant kernel
(k_collide) against the measured HBM bandwidth, the end-to-end rate through
the C-ABI with host buffers, the CPU oracle baseline, clocks and launch count.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS & % HBM roofline; BF16 vs FP32 speedup at stated error"
SIZE = 128
# algorithmic bytes per site of one k_collide launch (two components, two ion
# species, no colloids): populations read + written, then rho_a rho_b, J (3),
# psi_a psi_b, eps, phi (compute-type copy) and n+ n- read once, u (3) and
# the three owned face fluxes per species written
_FIELDS = (2 + 3 + 2 + 1 + 1 + 2) * 4 + (3 + 6) * 4
COLLIDE_BYTES = {"fp32": 2 * 19 * 4 * 2 + _FIELDS, "bf16": 2 * 19 * 2 * 2 + _FIELDS}


# Poisson solve, multigrid: 16 B/site per fine-level sweep (potential read
# and written, eps and q read), V(NU_SMOOTH, NU_SMOOTH) cycles
POISSON_BYTES_PER_SWEEP = 16
NU_SMOOTH = 2
# Poisson solve, spectral conjugate gradients (FP32 words, bytes per site):
# initial guess and sum of q 36, exact residual 20, final update 20; per
# iteration 88 = update + x pass 28, y, z, y passes 8 each, x pass with r.z 12,
# matvec and search direction 24
SPECTRAL_FIXED_BYTES = 76
SPECTRAL_ITER_BYTES = 88


def collide_bytes(ncomp, pop_bytes, solids):
    """Algorithmic bytes per site of k_collide with ions and a field: populations
    read + written, rho (ncomp), J (3), psi (two components only), eps, phi,
    n+ n- read once, psi_f and the solid mask with colloids; u (3) and the three
    owned face fluxes per species written."""
    reads = ncomp + 3 + (2 if ncomp == 2 else 0) + 1 + 1 + 2 + (1 if solids else 0)
    return ncomp * 19 * pop_bytes * 2 + reads * 4 + (1 if solids else 0) + (3 + 6) * 4


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class Ranks:
    """Replica bookkeeping of a torchrun launch: one independent box per rank,
    no collective on the data path; a barrier around the timed region and the
    max of the per-rank times (nccl on GPUs, gloo on CPU)."""

    def __init__(self, backend=None):
        self.rank, self.world, self.local = env_rank()
        self.dist = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.dist = dist
            self.device = "cuda" if backend == "nccl" else "cpu"

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v):
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("step_kernels.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1712_08494_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(prec):
    """DRAM bytes per k_collide launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "k_collide_droplet128.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(r"traffic_%s_bytes_per_launch:\s*([0-9.eE+]+)" % prec, txt)
    return float(m.group(1)) if m else None


def poisson_source_hash():
    h = hashlib.sha256()
    for f in ("poisson_dev.cuh", "poisson.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1712_08494_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_spectral_traffic(iters_per_solve):
    """DRAM bytes per k_spectral launch from the committed ncu summary when it
    was taken on the current solver source, scaled from the captured launch's
    iterations to an average solve's by the algorithmic byte rule (else None)."""
    p = os.path.join(ROOT, "profiles", "k_spectral_droplet128.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != spectral_source_hash():
        return None
    b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    c = re.search(r"iterations_of_captured_launch:\s*([0-9.eE+]+)", txt)
    if not b or not c:
        return None
    k = float(c.group(1))
    scale = (SPECTRAL_FIXED_BYTES + SPECTRAL_ITER_BYTES * iters_per_solve) / (SPECTRAL_FIXED_BYTES + SPECTRAL_ITER_BYTES * k)
    return float(b.group(1)) * scale


def spectral_source_hash():
    h = hashlib.sha256()
    for f in ("spectral.cu", "spectral.cuh", "poisson_dev.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1712_08494_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_poisson_traffic(cycles_per_solve):
    """DRAM bytes per k_poisson launch from the committed ncu summary when it
    was taken on the current solver source: the captured launch's bytes per
    multigrid cycle times the cycles of an average solve (else None)."""
    p = os.path.join(ROOT, "profiles", "k_poisson_droplet128.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != poisson_source_hash():
        return None
    b = re.search(r"traffic_fp32_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    c = re.search(r"cycles_of_captured_launch:\s*([0-9.eE+]+)", txt)
    if not b or not c:
        return None
    return float(b.group(1)) / float(c.group(1)) * cycles_per_solve


def _oracle_worker(args):
    """One host process: the oracle stepping its own seeded copy of the droplet
    workload; returns the wall-clock interval of the timed steps."""
    n, seed, untimed, timed = args
    sys.path.insert(0, ROOT)
    import synth
    from oracle import OracleSystem
    w = synth.droplet(n=n, r=24.0 * n / 128.0, prec="fp32", seed=seed)
    s = OracleSystem(w.params, w.rho, w.n)
    for _ in range(untimed):
        s.step()
    t0 = time.time()
    for _ in range(timed):
        s.step()
    return t0, time.time()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_throughput(n, untimed, timed, procs=None):
    """The FP64 oracle, as it stands (numpy, one thread per process), on every
    host core: one process per core, each stepping its own copy of the n^3
    droplet.  Processes are spawned (never forked from a process that has used
    the GPU).  Aggregate MLUPS = all sites stepped / the wall-clock span of the
    timed steps."""
    import multiprocessing as mp
    procs = procs or host_cores()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        spans = pool.map(_oracle_worker, [(n, 1 + k, untimed, timed) for k in range(procs)])
    t0 = min(a for a, _ in spans)
    t1 = max(b for _, b in spans)
    return procs * n ** 3 * timed / (t1 - t0) / 1e6, procs, t1 - t0


def cpu_baseline(n):
    """Time the FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload: on every host core, one copy of the n^3 droplet per core, one
    untimed step then one timed step."""
    val, procs, span = oracle_throughput(n, 1, 1)
    return {"value": val, "unit": "MLUPS", "cores": procs, "kind": "oracle",
            "sample": "%d processes (one per host core), each one timed step (after one untimed) of its own %d^3 "
                      "droplet, numpy FP64; %.1f s wall" % (procs, n, span)}


def run_reference(args):
    """CPU oracle timed on all host cores, each step a bounded sample: every
    core steps its own copy of a reduced droplet box."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    procs = host_cores()
    n = 64
    # size the box so that warm-up + timed steps end within a few minutes
    while n > 16:
        val, _, span = oracle_throughput(n, 0, 1, procs)
        if span * (args.steps + args.warmup) < 150.0:
            break
        n //= 2
    val, _, span = oracle_throughput(n, args.warmup, args.steps, procs)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * span / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "dielectric droplet, sampled at %d^3 per core per step (oracle)" % n},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                             "sample": "each step: one oracle step of a %d^3 droplet on each of %d cores" % (n, procs)},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import paper_1712_08494_gb300 as pkg
    import synth

    rank, world, local = env_rank()
    pkg.build()
    lbeh = pkg.load()
    torch.cuda.set_device(local)
    ranks = Ranks()
    stream = torch.cuda.current_stream()
    n = args.size
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    results = {}
    fields = {}
    sampler = None
    for prec in ("fp32", "bf16", "fp16"):
        w = synth.droplet(n=n, r=24.0 * n / 128.0, prec=prec, seed=1 + rank)
        w.params.poisson_solver = args.solver
        sysg = lbeh.System(w.params, stream.cuda_stream)
        sysg.set_fields(rho=list(w.rho), n=list(w.n))
        if args.relax:
            sysg.step(args.relax)  # state preparation: past the start-up transient
        if prec == "fp32":
            # the restart checkpoint the end-to-end leg loads every step
            checkpoint = sysg.get(("rho", "n", "phi"))
        sysg.step(args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sysg.profile_enable(False)  # reset the launch counter; whole-step graphs stay on
        smp = ClockSampler(local) if prec == "fp32" else None
        if smp:
            smp.__enter__()
        e0.record(stream)
        rc = sysg.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if smp:
            smp.__exit__()
            sampler = smp
        barrier()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        pr0 = sysg.profile_read()
        launches, cycles = pr0["launches"], pr0["poisson_cycles"]
        obs = sysg.observables()
        # per-kernel device times: CUDA events recorded by the library around
        # each stage on the stream it launches on (eager launches, same kernels)
        sysg.profile_enable(True)
        sysg.step(min(args.steps, 100))
        prof = sysg.profile_read()
        sysg.profile_enable(False)
        prof["launches"] = launches
        results[prec] = {"ms": ms, "prof": prof, "rc": rc, "obs": obs, "cycles": cycles}
        fields[prec] = sysg.get(("rho",))["rho"]
        sysg.close()
        del sysg

    N = n ** 3
    ms32 = results["fp32"]["ms"]
    mlups32 = world * N * args.steps / (ms32 * 1e3)
    msbf = results["bf16"]["ms"]
    mlupsbf = world * N * args.steps / (msbf * 1e3)
    err_bf = max(float(np.abs(fields["bf16"][s] - fields["fp32"][s]).max() / np.abs(fields["fp32"][s]).max())
                 for s in range(2))
    rms_bf = max(float(np.sqrt(((fields["bf16"][s] - fields["fp32"][s]) ** 2).mean() / (fields["fp32"][s] ** 2).mean()))
                 for s in range(2))

    # end-to-end through the C-ABI with pinned host buffers: every step
    # restarts from a checkpoint in host memory (densities, ion concentrations
    # and the potential, the solve's starting guess, of the relaxed state),
    # advances one step and reads the observables back
    w = synth.droplet(n=n, r=24.0 * n / 128.0, prec="fp32", seed=1 + rank)
    w.params.poisson_solver = args.solver
    host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
            for a in (checkpoint["rho"][0], checkpoint["rho"][1], checkpoint["n"][0], checkpoint["n"][1],
                      checkpoint["phi"])]
    sysg = lbeh.System(w.params, stream.cuda_stream)
    ke = max(3, min(10, args.steps))
    for it in range(2 + ke):
        if it == 2:
            torch.cuda.synchronize()
            barrier()
            sysg.profile_enable(False)  # reset the counters; graphs stay on
            t0 = time.perf_counter()
        sysg.set_fields(rho=host[:2], n=host[2:4], phi=host[4])
        sysg.step(1)
        sysg.observables()
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - t0)
    pre = sysg.profile_read()
    sysg.close()
    e2e = {"value": world * N * ke / te / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in host)),
           "d2h_bytes_per_step": 16 * 8, "poisson_iterations_per_step": pre["poisson_cycles"] / ke,
           "input": "checkpoint of the state relaxed for %d steps: rho, n and phi in FP32, populations "
                    "rebuilt at equilibrium" % args.relax}

    peak, peak_kind = measured_peaks()
    prof = results["fp32"]["prof"]
    calls = max(1, prof["calls"]["collide"])
    t_coll = prof["ms"]["collide"] / calls * 1e-3
    achieved = COLLIDE_BYTES["fp32"] * N / t_coll / 1e9
    profb = results["bf16"]["prof"]
    t_collb = profb["ms"]["collide"] / max(1, profb["calls"]["collide"]) * 1e-3
    achievedb = COLLIDE_BYTES["bf16"] * N / t_collb / 1e9
    tr = ncu_traffic("fp32")
    # the Poisson kernel: one launch is one solve
    calls_p = max(1, prof["calls"]["poisson"])
    t_pois = prof["ms"]["poisson"] / calls_p * 1e-3
    cyc_solve = prof["poisson_cycles"] / calls_p
    spectral = results["fp32"]["obs"].poisson_solver == lbeh.LBEH_POISSON_SPECTRAL
    if spectral:
        pois_kernel = "k_spectral"
        pois_bytes = (SPECTRAL_FIXED_BYTES + SPECTRAL_ITER_BYTES * cyc_solve) * N
        pois_rule = "%d + %d k B/site, k = conjugate-gradient iterations of the solve" % (
            SPECTRAL_FIXED_BYTES, SPECTRAL_ITER_BYTES)
        tr_p = ncu_spectral_traffic(cyc_solve)
    else:
        pois_kernel = "k_poisson"
        pois_bytes = POISSON_BYTES_PER_SWEEP * 2 * NU_SMOOTH * cyc_solve * N
        pois_rule = "16 B/site x 2*%d fine sweeps per V(%d,%d) cycle" % (NU_SMOOTH, NU_SMOOTH, NU_SMOOTH)
        tr_p = ncu_poisson_traffic(cyc_solve)
    achieved_p = pois_bytes / t_pois / 1e9 if t_pois > 0 else 0.0

    # whole-step roofline: 340 B/site for the lattice passes (FP32, two
    # components: macro, collide, Nernst-Planck) + 16 s B/site for the
    # Poisson solve, s = its bytes expressed as 16-B/site sweep equivalents
    s_eq = pois_bytes / N / POISSON_BYTES_PER_SWEEP * (prof["calls"]["poisson"] / max(1, prof["calls"]["collide"]))
    step_bytes = 340 + POISSON_BYTES_PER_SWEEP * s_eq
    step_gbs = step_bytes * N * args.steps / (ms32 * 1e-3) / 1e9
    step_roof = {"bytes_per_site": step_bytes, "achieved_gbs": step_gbs, "peak": peak, "frac": step_gbs / peak,
                 "rule": "340 + 16 s B/site, s = Poisson bytes per site / 16"}
    roof_p = {"bound": "hbm", "kernel": pois_kernel, "achieved": achieved_p, "peak": peak, "peak_kind": peak_kind,
              "unit": "GB/s", "frac": achieved_p / peak, "traffic": tr_p, "algorithmic_bytes_per_launch": pois_bytes,
              "avg_launch_ms": t_pois * 1e3, "iterations_per_launch": cyc_solve, "bytes_rule": pois_rule}
    roof_c = {"bound": "hbm", "kernel": "k_collide", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
              "unit": "GB/s", "frac": achieved / peak, "traffic": tr,
              "algorithmic_bytes_per_launch": COLLIDE_BYTES["fp32"] * N, "avg_launch_ms": t_coll * 1e3,
              "bytes_rule": "%d B/site: populations read and written, fields read once, u and face fluxes written"
                            % COLLIDE_BYTES["fp32"]}
    # `roofline` is the kernel with the larger share of the step
    if prof["ms"]["poisson"] >= prof["ms"]["collide"]:
        roof_main, roof_other_key, roof_other = roof_p, "roofline_collide", roof_c
    else:
        roof_main, roof_other_key, roof_other = roof_c, "roofline_poisson", roof_p
    if rank != 0:
        return
    extra = {}
    if not args.no_extra:
        runs = {"suspension": lambda: suspension_run(lbeh, stream, peak, peak_kind, args, n=args.suspension_size),
                "showcase": lambda: showcase_run(lbeh, stream, args),
                "coated_droplet": lambda: coated_run(lbeh, stream, args),
                "batch": lambda: batch_run(lbeh, stream, args),
                "adjoint": lambda: adjoint_run(lbeh, stream, args)}
        want = set(args.extras.split(","))
        for name in EXTRAS:
            if name in want:
                extra[name] = runs[name]()
    cpu = None if args.no_cpu_baseline else cpu_baseline(n)
    clocks = sampler.summary() if sampler else {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
    total_ms = sum(prof["ms"].values())

    def half_storage(prec):
        """Rate and deviation from the FP32 run of a reduced-precision storage mode."""
        r = results[prec]
        mlups = world * N * args.steps / (r["ms"] * 1e3)
        dev = max(float(np.abs(fields[prec][s] - fields["fp32"][s]).max() / np.abs(fields["fp32"][s]).max())
                  for s in range(2))
        rms = max(float(np.sqrt(((fields[prec][s] - fields["fp32"][s]) ** 2).mean() / (fields["fp32"][s] ** 2).mean()))
                  for s in range(2))
        pr = r["prof"]
        return {"value": mlups, "unit": "MLUPS", "speedup_vs_fp32": mlups / mlups32, "max_rel_dev_rho_vs_fp32": dev,
                "rms_rel_dev_rho_vs_fp32": rms, "deformation": r["obs"].deformation,
                "ms_per_step": r["ms"] / args.steps, "poisson_iterations_per_step": r["cycles"] / args.steps,
                "stage_ms_per_step": {k: v / max(1, pr["calls"]["collide"]) for k, v in pr["ms"].items()}}

    line = {
        "metric": METRIC, "value": mlups32, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "dielectric droplet %d^3, 2 components + 2 ion species, E_z=1e-3" % n,
                   "sites": N, "populations": "fp32", "poisson_tol": 1e-6,
                   "poisson_solver": "spectral" if spectral else "multigrid",
                   "state": ("relaxed for %d steps before the warm-up (the workload runs 5000 steps; the first "
                             "steps are its start-up transient)" % args.relax) if args.relax else "initial",
                   "l2": "inputs larger than L2 (populations %.0f MB)" % (2 * 19 * 4 * N / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "fp16_storage": half_storage("fp16"),
        "bf16_storage": {"value": mlupsbf, "unit": "MLUPS", "speedup_vs_fp32": mlupsbf / mlups32,
                         "max_rel_dev_rho_vs_fp32": err_bf, "rms_rel_dev_rho_vs_fp32": rms_bf,
                         "deformation_fp32": results["fp32"]["obs"].deformation,
                         "deformation_bf16": results["bf16"]["obs"].deformation,
                         "ms_per_step": msbf / args.steps,
                         "collide_gbs": achievedb,
                         "poisson_iterations_per_step": results["bf16"]["cycles"] / args.steps,
                         "stage_ms_per_step": {k: v / max(1, profb["calls"]["collide"]) for k, v in profb["ms"].items()}},
        "roofline": roof_main,
        roof_other_key: roof_other,
        "stage_share": {k: (v / total_ms if total_ms else None) for k, v in prof["ms"].items()},
        "stage_ms_per_step": {k: v / max(1, prof["calls"]["collide"]) for k, v in prof["ms"].items()},
        "step_roofline": step_roof,
        "poisson_iterations_per_step": results["fp32"]["cycles"] / args.steps,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": prof["launches"],
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def _timed(step, stream, steps):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), rc


EXTRAS = ("suspension", "showcase", "coated_droplet", "batch", "adjoint")


def suspension_run(lbeh, stream, peak, peak_kind, args, n=256, steps=100):
    """256^3 electrophoresis suspension: one fluid, 1e-3 salt, 200 moving
    charged spheres of radius 6, E_x = 1e-3; FP32 and BF16 storage.  Other
    box edges keep the number density of the spheres."""
    import numpy as np
    import synth
    ncoll = max(1, int(round(200 * (n / 256.0) ** 3)))
    out = {"workload": "suspension %d^3, %d moving colloids r=6, salt 1e-3, E_x=1e-3" % (n, ncoll), "steps": steps}
    vx = {}
    for prec in ("fp32", "bf16"):
        w = synth.suspension(n=n, ncoll=ncoll, r=6.0, prec=prec)
        s = lbeh.System(w.params, stream.cuda_stream)
        s.set_fields(rho=list(w.rho), n=list(w.n), colloid_x=w.colloid_x, colloid_v=w.colloid_v,
                     colloid_q=w.colloid_q, colloid_r=w.colloid_r)
        s.step(5)
        s.profile_enable(False)  # resets the launch and cycle counters
        ms, rc = _timed(s.step, stream, steps)
        cycles = s.profile_read()["poisson_cycles"]
        s.profile_enable(True)
        s.step(min(steps, 50))
        prof = s.profile_read()
        s.profile_enable(False)
        vx[prec] = np.array(s.get(("rho",))["cv"])[:, 0]
        s.close()
        t_coll = prof["ms"]["collide"] / max(1, prof["calls"]["collide"]) * 1e-3
        gbs = collide_bytes(1, 4 if prec == "fp32" else 2, True) * n ** 3 / t_coll / 1e9
        total = sum(prof["ms"].values())
        # whole-step roofline: 172 B/site (FP32) or 96 (BF16) for the lattice
        # passes of one component + 16 s B/site for the multigrid, s = fine
        # sweeps per step
        sweeps = 2 * NU_SMOOTH * cycles / steps
        step_bytes = (172 if prec == "fp32" else 96) + POISSON_BYTES_PER_SWEEP * sweeps
        step_gbs = step_bytes * n ** 3 * steps / (ms * 1e-3) / 1e9
        out[prec] = {"mlups": n ** 3 * steps / (ms * 1e3), "ms_per_step": ms / steps, "status": rc,
                     "poisson_cycles_per_step": cycles / steps,
                     "step_roofline": {"bytes_per_site": step_bytes, "achieved_gbs": step_gbs, "peak": peak,
                                       "frac": step_gbs / peak,
                                       "rule": "%d + 16 s B/site, s = 4 fine sweeps x multigrid cycles per step"
                                               % (172 if prec == "fp32" else 96)},
                     "collide_gbs": gbs, "collide_frac": gbs / peak, "peak_kind": peak_kind,
                     "stage_share": {k: (v / total if total else None) for k, v in prof["ms"].items()}}
    out["bf16_speedup"] = out["bf16"]["mlups"] / out["fp32"]["mlups"]
    out["bf16_colloid_vx_rel_dev"] = float(np.abs(vx["bf16"] - vx["fp32"]).max() / max(np.abs(vx["fp32"]).max(), 1e-30))
    return out


def showcase_run(lbeh, stream, args, n=384, r=64.0, steps=20):
    """The paper's largest run (Sec. III.D, 3D charged droplet): a drop of
    radius 64 in a 384^3 periodic box, two components (G = 4), salt 1e-3,
    Gibbs transfer energies +-4 kT (the drop takes a negative net charge),
    equal permittivities, applied field 1e-3 along z; FP32.  Device memory of
    the system and MLUPS over `steps` steps after 5 warm-up steps."""
    import torch
    import synth
    free0, total = torch.cuda.mem_get_info()
    w = synth.droplet(n=n, r=r, prec="fp32", salt=1e-3, Ez=1e-3, eps_r=(1.0, 1.0), noise=0.01)
    w.params.dmu = (4.0, -4.0)
    s = lbeh.System(w.params, stream.cuda_stream)
    s.set_fields(rho=list(w.rho), n=list(w.n))
    del w
    free1, _ = torch.cuda.mem_get_info()
    s.step(5)
    ms, rc = _timed(s.step, stream, steps)
    o = s.observables()
    s.close()
    return {"workload": "charged droplet %d^3, r=%g, salt 1e-3, dmu +-4, E_z=1e-3, FP32" % (n, r), "sites": n ** 3,
            "steps": steps, "mlups": n ** 3 * steps / (ms * 1e3), "ms_per_step": ms / steps, "status": rc,
            "device_gb": (free0 - free1) / 1e9, "poisson_solver": "spectral" if o.poisson_solver == 2 else "multigrid",
            "poisson_iterations_last_step": o.poisson_iters}


def coated_run(lbeh, stream, args, n=128, steps=50):
    """Sec. III.G: a drop of radius 32 coated by 80 uncharged moving spheres of
    radius 5 (covering fraction 0.49) in the charged-drop setting of
    Sec. III.D, 128^3, FP32: MLUPS over `steps` steps after 5 warm-up steps,
    with the multigrid cycles per step (colloids bring the permittivity
    contrast 8)."""
    import synth
    w = synth.coated_droplet(n=n)
    s = lbeh.System(w.params, stream.cuda_stream)
    s.set_fields(rho=list(w.rho), n=list(w.n), colloid_x=w.colloid_x, colloid_v=w.colloid_v,
                 colloid_q=w.colloid_q, colloid_r=w.colloid_r)
    s.step(5)
    s.profile_enable(False)  # resets the cycle counter
    ms, rc = _timed(s.step, stream, steps)
    cycles = s.profile_read()["poisson_cycles"]
    o = s.observables()
    s.close()
    return {"workload": "colloid-coated drop %d^3, r_d=32, 80 spheres r_p=5, salt 1e-3, dmu +-4, E_z=1e-3, FP32" % n,
            "sites": n ** 3, "steps": steps, "mlups": n ** 3 * steps / (ms * 1e3), "ms_per_step": ms / steps,
            "status": rc, "poisson_solver": "spectral" if o.poisson_solver == 2 else "multigrid",
            "poisson_cycles_per_step": cycles / steps}


def batch_run(lbeh, stream, args, steps=50):
    """96 independent charged droplets (edges 32..64) in one cluster launch per
    step call, against the single-system kernels stepping the boxes in turn."""
    import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    ws = synth.batch_boxes(nbox=96, steps=steps)
    sites = sum(w.params.nx * w.params.ny * w.params.nz for w in ws)
    bt = lbeh.Batch([w.params for w in ws], stream.cuda_stream)
    for box, w in zip(bt.boxes, ws):
        box.set_fields(rho=list(w.rho), n=list(w.n))
    shape, _ = bt.tune(4)
    bt.step(3)
    ms, rc = _timed(bt.step, stream, steps)
    bt.close()
    singles = []
    for w in ws:
        s = lbeh.System(w.params, stream.cuda_stream)
        s.set_fields(rho=list(w.rho), n=list(w.n))
        s.step(2)
        singles.append(s)
    k = 5
    ms_seq, _ = _timed(lambda m: [s.step(m) for s in singles], stream, k)
    for s in singles:
        s.close()
    return {"workload": "96 charged droplets, edges {32..64}, FP32", "sites": sites, "steps": steps,
            "cluster_blocks": shape, "mlups": sites * steps / (ms * 1e3), "ms_per_step": ms / steps,
            "status": rc, "single_system_in_turn_mlups": sites * k / (ms_seq * 1e3),
            "speedup_vs_single_system_in_turn": (sites * steps / ms) / (sites * k / ms_seq)}


def adjoint_run(lbeh, stream, args, n=96, steps=800, ckpt=50):
    """Gradient of the drop deformation after 800 steps (96^3, r=18, Q=50,
    E_z=1.5e-3, FP32, checkpoints every 50) by the discrete adjoint."""
    import synth
    w = synth.droplet(n=n, r=18.0, seed=4, prec="fp32", salt=1e-3, Ez=1.5e-3, charge=50.0, steps=steps)
    one = synth.droplet(n=n, r=18.0, seed=4, prec="fp32", salt=1e-3, Ez=1.5e-3, charge=1.0)
    zero = synth.droplet(n=n, r=18.0, seed=4, prec="fp32", salt=1e-3, Ez=1.5e-3, charge=0.0)
    s = lbeh.System(w.params, stream.cuda_stream)
    s.set_fields(rho=list(w.rho), n=list(w.n))
    g = s.step_adjoint(steps, ckpt, d_deformation=1.0, dn0_dQ=one.n - zero.n)
    s.close()
    return {"workload": "adjoint drop %d^3 r=18 Q=50 E_z=1.5e-3, %d steps, checkpoints every %d, FP32" % (n, steps, ckpt),
            "forward_ms": g["forward_ms"], "reverse_ms": g["adjoint_ms"],
            "reverse_over_forward": g["adjoint_ms"] / g["forward_ms"], "deformation": g["deformation"],
            "dD_dEz": float(g["dE_ext"][2]), "dD_dG": g["dG"], "dD_dQ": g["dQ"], "status": g["status"],
            "adjoint_poisson_cycles": g["adjoint_poisson_cycles"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=SIZE)
    ap.add_argument("--relax", type=int, default=200,
                    help="untimed steps before the warm-up that take the droplet past its start-up transient")
    ap.add_argument("--solver", default="auto", choices=["auto", "spectral", "multigrid"],
                    help="Poisson solver of the droplet runs (auto: spectral for the droplet)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the suspension, showcase, coated-droplet, batch and adjoint measurements")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma-separated extra measurements to run (default: all of %s)" % ", ".join(EXTRAS))
    ap.add_argument("--suspension-size", type=int, default=256,
                    help="edge of the suspension box (the sphere count keeps the density of 200 in 256^3)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
