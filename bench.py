#!/usr/bin/env python3
"""Benchmark: short-range tree-gravity forces/s at N = 256^3 on one GB300.

Workload (the headline configuration): periodic box L = 500 with 256^3 equal-mass particles,
lattice plus Zel'dovich displacements from a seeded Gaussian field with P(k) ~ k^-2 and rms
displacement 2 grid spacings (strongly clustered), 32-bit integer coordinates, TreePM split
r_s = 1.25 L / 512, cutoff 4.5 r_s, softening eps = L / 256 / 30, one-sided tree of order
p = 3 with the relative opening criterion alpha = 0.0025, leaf threshold 32.

One step = one complete force computation through the C ABI: Peano-Hilbert keys + radix sort,
PH-order gather, oct-tree build, upward moments, tree walk (with |a_old| of the previous step)
writing its results in input order (the scatter fused into the walk's epilogue).  |a_old| comes from one geometric-criterion walk before timing
(the paper's first-step bootstrap).  Inputs (about 335 MB) are larger than the 129 MB L2.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tree-gravity forces/sec at N=256^3 (FP32 vs FP64-judged, 99% err<=1e-3)"
UNIT = "forces/s"
N_SIDE = 256
L_BOX = 500.0
RMS = 2.0
SEED = 1003
# algorithmic work per interaction (operations of the kernel formulas; erfc, exp and rsqrt
# count as one operation each)
FLOPS_PP = 35
FLOPS_PN = {1: 40, 2: 110, 3: 170, 4: 300, 5: 480}
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per SM (Blackwell)
SM_CLOCK_MAX_GHZ = 2.070    # maximum SM clock of a GB300


def fp32_peak_tflops():
    """FP32 FMA peak of the current GPU: its SM count x 128 lanes x 2 flops x maximum clock
    (no FP32 figure is measured for this GPU type, so the unit counts and clock are used)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * SM_CLOCK_MAX_GHZ * 1e9 / 1e12, \
        f"{sms} SMs (device property) x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {SM_CLOCK_MAX_GHZ} GHz"


# DRAM bytes (read + write) of one k_walk launch of the headline workload: the single-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the timed walk, 762,177,280 +
# 763,437,056 bytes.  Reported as roofline.traffic for the default workload only; set to
# None whenever the walk kernel changes until it is captured again.
WALK_DRAM_BYTES_256 = 1525614336


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU type (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# algorithmic bytes per particle / per node of the HBM-bound stages (keys: 12 B read + 8 B
# written; sort: 8 passes of (8 + 4) B read and written; gather: perm + 20 B in, 20 B out;
# build: keys and positions read plus ~64 B per node; multipoles: particles read once, node
# records and p = 3 moments (64 + 64 B) written; the walk writes its results in input order)
STAGE_BYTES = {"keys_sort": (20 + 8 * 2 * 12, 0), "gather": (44, 0), "build": (24, 64),
               "multipoles": (16, 128)}


LEAF_MAX = 32          # tuned on GB300 with autotune.tune_leaf on the 256^3 box


def workload_params(n_side=N_SIDE, L=L_BOX, leaf_max=None):
    d = L / n_side
    return dict(box_size=L, periodic=1, r_s=1.25 * L / (2 * n_side), r_cut_factor=4.5,
                eps=[d / 30.0], alpha=0.0025, order_p=3, leaf_max=leaf_max or LEAF_MAX)


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ---------------------------------------------------------------------------------------------
def oracle_workload_sample(n_side=N_SIDE, k_sinks=262144):
    """The FP64 oracle on the headline box itself: keys, sort, build and multipoles over all
    N particles, then the relative-criterion walk for a seeded subset of k_sinks sinks.  The
    step time is extrapolated to all N sinks: t_prepare + t_walk * N / k_sinks."""
    import oracle
    from paper_2010_03567_gb300 import synth
    L = L_BOX * n_side / N_SIDE
    ps = synth.zeldovich(n_side, L, RMS, SEED)
    wp = workload_params(n_side, L)
    kw = dict(box=L, periodic=True, eps=np.array(wp["eps"]), r_s=wp["r_s"], r_cut_factor=4.5, order=3)
    OP = oracle.OracleParams(**kw, alpha=wp["alpha"])
    OB = oracle.OracleParams(**kw, criterion=1, theta=0.5)
    q = oracle.int_coords_periodic(ps.pos, L)
    sinks = synth.subset(ps.n, k_sinks, 2002)
    run = oracle.prepare(q, ps.mass, None, None, OB, LEAF_MAX)
    ab, _, _ = oracle.tree_forces(run, sinks)
    aold = np.zeros(ps.n)
    aold[sinks] = np.linalg.norm(ab, axis=1)

    def step():
        t0 = time.perf_counter()
        r = oracle.prepare(q, ps.mass, None, aold, OP, LEAF_MAX)
        t1 = time.perf_counter()
        oracle.tree_forces(r, sinks)
        t2 = time.perf_counter()
        return (t1 - t0) + (t2 - t1) * ps.n / len(sinks), t2 - t0

    sample = (f"FP64 oracle on the {n_side}^3 headline box: keys, sort, build and multipoles of all "
              f"{ps.n} particles plus the relative-criterion walk of a {len(sinks)}-sink subset; "
              f"step time extrapolated as t_prepare + t_walk * N / {len(sinks)}")
    return ps.n, step, sample


def stage_breakdown(tg, pos_int, mass, aold, P, n, n_nodes, reps=3):
    """CUDA-event time of each pipeline stage (same calls as a timed step) and the achieved
    algorithmic HBM bandwidth of the memory-bound ones."""
    import torch
    from paper_2010_03567_gb300 import g4
    stages = [
        ("keys_sort", lambda: g4.g4_keys_sort(pos_int, tg.keys, tg.perm, tg.ws)),
        ("gather", lambda: g4.g4_gather(tg.perm, pos_int, mass, None, aold,
                                        out=(tg.pos_s, tg.mass_s, None, tg.aold_s))),
        ("build", lambda: tg.tree.build(tg.keys, tg.pos_s, P)),
        ("multipoles", lambda: tg.tree.multipoles(tg.pos_s, tg.mass_s, None, tg.aold_s, P)),
        ("walk", lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, acc=tg.acc,
                                              pot=tg.pot, counts=tg.counts, perm=tg.perm)),
    ]
    s = torch.cuda.current_stream()
    tot = {k: 0.0 for k, _ in stages}
    for r in range(reps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
        ev[0].record(s)
        for i, (_, fn) in enumerate(stages):
            fn()
            ev[i + 1].record(s)
        torch.cuda.synchronize()
        if r > 0:
            for i, (k, _) in enumerate(stages):
                tot[k] += ev[i].elapsed_time(ev[i + 1]) / reps
    peak, src = hbm_peak_gbs()
    out = {}
    for k, _ in stages:
        d = {"ms": tot[k]}
        if k in STAGE_BYTES:
            bpp, bpn = STAGE_BYTES[k]
            b = bpp * n + bpn * n_nodes
            d.update({"bytes": int(b), "GB/s": b / (tot[k] * 1e-3) / 1e9,
                      "frac_hbm": b / (tot[k] * 1e-3) / 1e9 / peak})
        out[k] = d
    out["hbm_peak_GB/s"] = peak
    out["hbm_peak_source"] = src
    return out


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n, step, sample = oracle_workload_sample()
    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    t = sum(x[0] for x in ts)
    val = n * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(x, device, dist):
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if not dist:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_per_rank, ms):
    """Whole-job forces per second: every rank solves its own n_per_rank-particle box."""
    return world * n_per_rank / (ms * 1e-3)


def config_block(world, n_side=N_SIDE, leaf_max=None):
    L = L_BOX * n_side / N_SIDE
    return {"workload": f"periodic Zel'dovich box, {n_side}^3 particles, L={L:g}, rms displacement 2 "
                        f"spacings, TreePM short range r_s=1.25L/{2 * n_side}, R_cut=4.5, eps=L/{30 * n_side}, "
                        f"tree p=3, alpha=0.0025, leaf {leaf_max or LEAF_MAX}",
            "n_particles": n_side ** 3, "order_p": 3, "alpha": 0.0025, "leaf_max": leaf_max or LEAF_MAX,
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": (f"inputs ({n_side ** 3 * 20 / 1e6:.0f} MB: positions, masses, |a_old|) larger than "
                   f"L2 (129 MB); no flush") if n_side ** 3 * 20 > 129e6 else
                  (f"inputs ({n_side ** 3 * 20 / 1e6:.0f} MB) fit in L2 (129 MB): small profiling case, "
                   f"not a bench configuration")}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    from paper_2010_03567_gb300 import g4, synth

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    n_side = args.n_side
    L = L_BOX * n_side / N_SIDE          # same spacing, split and softening at any size
    ps = synth.zeldovich(n_side, L, RMS, SEED + rank)
    n = ps.n
    wp = workload_params(n_side, L, args.leaf_max)
    P = g4.params(**wp)
    PB = g4.params(**{**wp, "criterion": 1, "theta": 0.5})
    pos = torch.from_numpy(ps.pos).cuda()
    pos_int, _ = g4.g4_int_coords(pos, True, L)
    del pos
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    tg = g4.TreeGravity(n, P)
    # bootstrap |a_old| (geometric criterion), then the relative-criterion steps
    acc0, _ = tg.forces(pos_int, mass, None, None, PB)
    aold = torch.linalg.vector_norm(acc0, dim=0).contiguous()
    torch.cuda.synchronize()
    nn, ml = tg.tree.status()

    stream = torch.cuda.current_stream()
    ev_walk = []

    def step(record=False):
        tg.prepare(pos_int, mass, None, aold, P)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        tg.walk(P)
        if record:
            e1.record(stream)
            ev_walk.append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tg.tree.status()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    l0 = g4.launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = g4.launch_count() - l0
    ms = t0.elapsed_time(t1) / args.steps
    walk_ms = sum(a.elapsed_time(b) for a, b in ev_walk) / len(ev_walk)
    ms = max_over_ranks(ms, "cuda", dist)
    clk = clocks.stop()
    counts = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    flops = counts[0] * FLOPS_PP + counts[1] * FLOPS_PN[3]
    achieved = flops / (walk_ms * 1e-3) / 1e12

    # ---- end to end through the public API with host buffers (pinned), copies inside the
    # region: g4.HostPipeline overlaps the next step's input copy and the previous step's
    # result copy with the current step's computation (every step moves all its bytes)
    h_pos = pos_int.cpu().pin_memory()
    h_mass = mass.cpu().pin_memory()
    h_aold = aold.cpu().pin_memory()
    h_acc = [torch.empty((3, n), dtype=torch.float32).pin_memory() for _ in range(2)]
    h_pot = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    pipe = g4.HostPipeline(n, P)
    for k in range(2):
        pipe.submit(h_pos, h_mass, h_aold, h_acc[k & 1], h_pot[k & 1])
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e0.record(pipe.h2d)
    done = None
    for k in range(args.steps):
        done = pipe.submit(h_pos, h_mass, h_aold, h_acc[k & 1], h_pot[k & 1])
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(done) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, "cuda", dist)
    e2e_same = bool(torch.equal(h_acc[(args.steps - 1) & 1], tg.acc.cpu()))
    del pipe

    # ---- accuracy on a sample against the FP64 direct sum (pairs with r < r_cut)
    accuracy = None
    if rank == 0 and not args.no_check:
        import oracle
        sinks = synth.subset(n, 4096, 2002)
        q = pos_int.cpu().numpy().view(np.uint32)
        OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(wp["eps"]), r_s=wp["r_s"],
                                 r_cut_factor=4.5)
        ad, _ = oracle.direct(q, ps.mass, None, sinks, OP, r_max=OP.r_cut)
        ag = tg.acc.cpu().numpy().T[sinks].astype(np.float64)
        e = np.linalg.norm(ag - ad, axis=1) / np.linalg.norm(ad, axis=1)
        accuracy = {"reference": "FP64 direct sum over pairs with r < r_cut (oracle)",
                    "sample": int(len(sinks)), "p50": float(np.percentile(e, 50)),
                    "p99": float(np.percentile(e, 99)), "max": float(np.max(e))}

    stages = stage_breakdown(tg, pos_int, mass, aold, P, n, nn) if rank == 0 else None

    extras = {}
    if rank == 0 and not args.no_extras:
        sample_ref = None
        if accuracy is not None:
            sample_ref = (sinks, ad)
        collect_cost_samples("C3_256cubed", tg.tree, P, n, tg.aold_s, tg.counts)
        for name, fn in (("cost_model", lambda: extra_cost_model(tg, P, n)),
                         ("fmm", lambda: extra_fmm(pos_int, mass, aold, wp, n, sample_ref,
                                                   cpu=not args.no_cpu)),
                         ("treepm", lambda: extra_treepm(pos_int, mass, aold, wp, n)),
                         ("fp64_walk", lambda: extra_fp64(tg, P, n, sample_ref)),
                         ("batched_systems", lambda: extra_forest(wp["leaf_max"])),
                         ("plummer_16k", lambda: extra_plummer(wp["leaf_max"])),
                         ("box_128cubed", lambda: extra_box128(wp["leaf_max"])),
                         ("cost_model_frozen", extra_frozen_model),
                         ("hierarchical_bins", lambda: extra_bins(wp["leaf_max"])),
                         ("softened_nodes", lambda: extra_softened(wp["leaf_max"])),
                         ("ewald_periodic_tree", lambda: extra_ewald(wp["leaf_max"])),
                         ("cost_model_512cubed", lambda: extra_c5(wp["leaf_max"]))):
            if args.extras and name not in args.extras.split(","):
                continue
            try:
                extras[name] = fn()
            except Exception as ex:           # report, keep the headline line
                extras[name] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu:
        nb, cstep, csample = oracle_workload_sample(n_side)
        text, treal = cstep()
        cpu = {"value": nb / text, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": csample + f" ({treal:.1f} s of CPU time measured)"}

    if rank == 0:
        peak, peak_src = fp32_peak_tflops()
        value = job_throughput(world, n, ms)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_block(world, n_side, args.leaf_max), "clocks": clk,
                "e2e": {"value": job_throughput(world, n, e2e_ms), "unit": UNIT,
                        "h2d_bytes_per_step": int(n * (12 + 4 + 4)),
                        "d2h_bytes_per_step": int(n * (12 + 4)),
                        "api": "g4.HostPipeline (double-buffered copies on two copy streams)",
                        "results_equal_device_run": e2e_same},
                "gpu_launches": int(launches),
                "roofline": {"bound": "alu", "kernel": "k_walk (tree walk, p=3, TreePM)",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "peak_source": peak_src, "frac": achieved / peak,
                             "traffic": WALK_DRAM_BYTES_256 if (n_side == N_SIDE and WALK_DRAM_BYTES_256) else None,
                             "traffic_per_sink_bytes": (WALK_DRAM_BYTES_256 / n) if (n_side == N_SIDE and WALK_DRAM_BYTES_256) else None,
                             "walk_ms": walk_ms,
                             "interactions_per_step": {"pp": int(counts[0]), "pn": int(counts[1])}},
                "tree": {"nodes": nn, "max_level": ml},
                "interactions_per_s": {"pp": float(counts[0] / (walk_ms * 1e-3)),
                                       "pn": float(counts[1] / (walk_ms * 1e-3)),
                                       "nn": None},
                "accuracy": accuracy, "stages": stages, "cpu_baseline": cpu, **extras}
        print(json.dumps(line), flush=True)
    if dist:
        tdist.barrier()
    return 0


# ---------------------------------------------------------------------------------------------
# further rows of the path, measured after the headline (each guarded: a failure is reported,
# never fatal to the headline line)
# ---------------------------------------------------------------------------------------------
def _time(fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def oracle_fmm_throughput(n_side_cpu=40):
    """The FP64 oracle's FMM (p = 4, relative criterion, leaf 32) on a box of the headline's
    spacing, split and cutoff with n_side_cpu^3 particles (the FMM's work per particle does not
    grow with N), on the host: forces/s."""
    import oracle
    from paper_2010_03567_gb300 import synth
    L = 500.0 * n_side_cpu / N_SIDE
    ps = synth.zeldovich(n_side_cpu, L, 2.0, 1003)
    q = oracle.int_coords_periodic(ps.pos, L)
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array([L / n_side_cpu / 30.0]),
                             r_s=1.25 * L / (2 * n_side_cpu), r_cut_factor=4.5, alpha=0.0025, order=4)
    t0 = time.perf_counter()
    run = oracle.prepare(q, ps.mass, None, np.full(ps.n, 20.0), OP, LEAF_MAX)
    run.tree.fmm(OP)
    t = time.perf_counter() - t0
    return {"value": ps.n / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle FMM (keys, sort, tree, multipoles, dual walk; p = 4, alpha = 0.0025, "
                      f"|a_old| = 20, leaf {LEAF_MAX}) on a {n_side_cpu}^3 box with the headline's spacing, "
                      f"r_s / spacing and R_cut, one thread; {t:.1f} s"}


def extra_fmm(pos_int, mass, aold, wp, n, sample_ref, cpu=True):
    """Symmetric FMM (p = 4, relative criterion) on the headline box; the same FMM run all in
    FP64 on the GPU, and the FP32 run's error against it; the oracle's FMM on a bounded sample
    of the same workload on the host."""
    import torch
    from paper_2010_03567_gb300 import g4
    P4 = g4.params(**{**wp, "order_p": 4})
    tg = g4.TreeGravity(n, P4)
    tg.prepare(pos_int, mass, None, aold, P4)
    ws = torch.empty(tg.tree.fmm_workspace(P4) + 256, dtype=torch.uint8, device="cuda")
    out = {}

    def step():
        tg.prepare(pos_int, mass, None, aold, P4)
        out["r"] = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P4, workspace=ws)
        g4.g4_scatter(tg.perm, out["r"][0], out["r"][1], out=(tg.acc, tg.pot))

    ms = _time(step, 3)
    tg.tree.status()
    acc_s, _, cnt, mom = out["r"]
    m = mass.double()
    amag = torch.linalg.vector_norm(acc_s.double(), dim=0)
    ms_s = tg.mass_s.double()
    res = {"ms_per_step": ms, "forces_per_s": n / (ms * 1e-3), "order_p": 4,
           "momentum_rel": float(torch.linalg.vector_norm(mom).item() / (ms_s * amag).sum().item()),
           # ordered particle pairs (each pair counted at both particles), particle-node terms
           "pp_per_step": int(cnt[0].to(torch.int64).sum().item()),
           "pn_per_step": int(cnt[1].to(torch.int64).sum().item()),
           # node-node (M2L) fields acting on each particle through its ancestors, summed
           "nn_per_particle_sum": int(cnt[2].to(torch.int64).sum().item())}
    # interactions per second by kind (ordered particle pairs, particle-node terms, node-node
    # fields counted at the particles they reach)
    res["interactions_per_s"] = {k: res[f"{k}_per_step"] / (ms * 1e-3) for k in ("pp", "pn")}
    res["interactions_per_s"]["nn_per_particle"] = res["nn_per_particle_sum"] / (ms * 1e-3)
    if sample_ref is not None:
        sinks, ad = sample_ref
        ag = tg.acc.cpu().numpy().T[sinks].astype(np.float64)
        e = np.linalg.norm(ag - ad, axis=1) / np.linalg.norm(ad, axis=1)
        res["accuracy_vs_direct"] = {"p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99))}
    del ws
    # the all-FP64 GPU run of the same FMM (precision 1: FP64 node data, expansions, fields and
    # pairs; the decisions as in FP32): the FP32 run's error against it
    a32 = acc_s.clone()
    P4d = g4.G4Params.from_buffer_copy(P4)
    P4d.precision = 1
    tg.tree.multipoles(tg.pos_s, tg.mass_s, None, tg.aold_s, P4d)
    ws64 = torch.empty(tg.tree.fmm_workspace(P4d) + 256, dtype=torch.uint8, device="cuda")
    r64 = {}
    ms64 = _time(lambda: r64.__setitem__("r", tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s,
                                                                   P4d, workspace=ws64)), 1)
    tg.tree.status()
    a64, _, c64, mom64 = r64["r"]
    amag64 = torch.linalg.vector_norm(a64.double(), dim=0)
    fp64 = {"ms_per_step": ms64,
            "momentum_rel": float(torch.linalg.vector_norm(mom64).item() / (ms_s * amag64).sum().item()),
            "counts_identical_frac": float((c64 == cnt).all(dim=0).double().mean().item()),
            "fp32_vs_fp64_gpu": _errors(a32.double().cpu().numpy().T, a64.double().cpu().numpy().T)}
    if sample_ref is not None:
        sinks, ad = sample_ref
        inv = torch.empty_like(tg.perm)
        inv[tg.perm.long()] = torch.arange(n, dtype=torch.int32, device="cuda")
        rows = inv[torch.from_numpy(sinks).cuda().long()].long()
        fp64["fp64_gpu_vs_direct"] = _errors(a64[:, rows].double().cpu().numpy().T, ad)
    res["fp64_gpu"] = fp64
    del ws64
    if cpu:
        res["cpu_oracle"] = oracle_fmm_throughput()
    return res


def extra_treepm(pos_int, mass, aold, wp, n):
    """Total TreePM forces on the headline box (Sec. 2.3): the tree's short-range walk plus
    the PM long-range force on a 512^3 mesh (A_smth = r_s / (L / N_grid) = 1.25), with the
    relative criterion fed the total |a| of the previous step; the PM call alone, and its
    mesh traffic against the measured HBM bandwidth."""
    import torch
    from paper_2010_03567_gb300 import g4
    ng = 2 * N_SIDE if n == N_SIDE ** 3 else 2 * round(n ** (1 / 3))
    P = g4.params(**wp)
    tp = g4.TreePMGravity(n, P, ng)
    tp.forces(pos_int, mass, None, aold, P)
    aold_tot = torch.linalg.vector_norm(tp.tg.acc, dim=0).contiguous()   # total |a|
    ms_step = _time(lambda: tp.forces(pos_int, mass, None, aold_tot, P), 3)
    tg = tp.tg
    acc = torch.zeros_like(tg.acc_s)
    pm = lambda: g4.g4_pm_long_range(tg.pos_s, tg.mass_s, P, ng, acc=acc, pot=None, workspace=tp.ws)
    ms_pm = _time(pm, 5)
    # mesh bytes per call: clear (8 N^3), 6 FFT passes and the Green's function (2 x 8 N^3 each),
    # the CIC sums (8 atomics of 4 B per particle) and the interpolation reads (8 x 13 values
    # of 8 B per sink, mostly from cache)
    mesh = 8.0 * ng ** 3
    bytes_alg = mesh + 7 * 2 * mesh + n * 8 * 4 + n * (12 + 4) + n * 16
    peak, src = hbm_peak_gbs()
    cnt = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    return {"n_grid": ng, "A_smth": wp["r_s"] / (wp["box_size"] / ng), "ms_per_step": ms_step,
            "forces_per_s": n / (ms_step * 1e-3), "pm_ms": ms_pm,
            "pm_algorithmic_bytes": bytes_alg, "pm_GB/s": bytes_alg / (ms_pm * 1e-3) / 1e9,
            "pm_frac_hbm": bytes_alg / (ms_pm * 1e-3) / 1e9 / peak, "hbm_peak_source": src,
            "pp_per_step": int(cnt[0]), "pn_per_step": int(cnt[1]),
            "aold": "total |a| (tree + PM) of the previous step"}


def extra_forest(leaf_max):
    """256 independent Plummer spheres (N log-uniform in [1024, 65536]) in one call sequence."""
    import torch
    from paper_2010_03567_gb300 import g4, synth
    systems = synth.multi_plummer(256, 1005)
    sizes = [ps.n for ps in systems]
    n = sum(sizes)
    qs, boxes = [], []
    for ps in systems:
        q, fr = g4.g4_int_coords(torch.from_numpy(ps.pos).cuda(), False)
        qs.append(q)
        boxes.append(fr[3:4])
    pos = torch.cat(qs, dim=1).contiguous()
    box = torch.cat(boxes).contiguous()
    mass = torch.from_numpy(np.concatenate([ps.mass for ps in systems]).astype(np.float32)).cuda()
    PB = g4.params(periodic=0, eps=[0.01], criterion=1, theta=0.5, leaf_max=leaf_max)
    P = g4.params(periodic=0, eps=[0.01], alpha=0.0025, leaf_max=leaf_max)
    fg = g4.ForestGravity(sizes, P)
    acc0, _ = fg.forces(pos, mass, box, None, PB)
    aold = torch.linalg.vector_norm(acc0, dim=0).contiguous()
    l0 = g4.launch_count()
    ms = _time(lambda: fg.forces(pos, mass, box, aold, P), 3)
    launches = (g4.launch_count() - l0) / 4
    fg.tree.status()
    cnt = fg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    res = {"systems": len(sizes), "particles": n, "ms_per_step": ms, "forces_per_s": n / (ms * 1e-3),
           "launches_per_step": launches, "pp_per_step": int(cnt[0]), "pn_per_step": int(cnt[1])}
    # the same systems one at a time: every system its own sort, gather, tree build, moments,
    # walk and scatter launches (one handle and one set of buffers sized for the largest
    # system, reused in turn), eager and as one CUDA graph of all those launches
    first = np.concatenate([[0], np.cumsum(sizes)])
    nmax = max(sizes)
    tree1 = g4.Tree(nmax, 4096 + int(nmax * max(1.5, 3.5 / leaf_max)))
    keys1 = torch.empty(nmax, dtype=torch.int64, device="cuda")
    perm1 = torch.empty(nmax, dtype=torch.int32, device="cuda")
    ws1 = torch.empty(g4.g4_keys_sort_workspace(nmax) + 256, dtype=torch.uint8, device="cuda")
    flat = {k: torch.empty(3 * nmax, dtype=dt, device="cuda")
            for k, dt in (("pos", torch.int32), ("acc_s", torch.float32), ("acc", torch.float32))}
    one = {k: torch.empty(nmax, dtype=torch.float32, device="cuda")
           for k in ("mass", "aold", "pot_s", "pot")}
    cnt1 = torch.empty(2 * nmax, dtype=torch.int32, device="cuda")
    Ps = [g4.params(periodic=0, eps=[0.01], alpha=0.0025, leaf_max=leaf_max,
                    box_size=float(box[k].item())) for k in range(len(sizes))]

    def one_system(k):
        a, b = int(first[k]), int(first[k + 1])
        m = b - a
        q_, P_ = pos[:, a:b].contiguous(), Ps[k]
        ps_ = flat["pos"][:3 * m].view(3, m)
        g4.g4_keys_sort(q_, keys1[:m], perm1[:m], ws1)
        g4.g4_gather(perm1[:m], q_, mass[a:b], None, aold[a:b],
                     out=(ps_, one["mass"][:m], None, one["aold"][:m]))
        tree1.build(keys1[:m], ps_, P_)
        tree1.multipoles(ps_, one["mass"][:m], None, one["aold"][:m], P_)
        tree1.gravity_tree(ps_, one["mass"][:m], None, one["aold"][:m], P_,
                           acc=flat["acc_s"][:3 * m].view(3, m), pot=one["pot_s"][:m],
                           counts=cnt1[:2 * m].view(2, m))
        g4.g4_scatter(perm1[:m], flat["acc_s"][:3 * m].view(3, m), one["pot_s"][:m],
                      out=(flat["acc"][:3 * m].view(3, m), one["pot"][:m]))

    for k in range(len(sizes)):   # first calls outside any capture (walk buffers)
        one_system(k)
    ms_sys = _time(lambda: [one_system(k) for k in range(len(sizes))], 3)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        for k in range(len(sizes)):
            one_system(k)
    ms_sys_graph = _time(g.replay, 3)
    # the leaf threshold tuned for the forest (one complete forest step per candidate)
    leaf_ms = {}
    for lm in (8, 16, 32, 64):
        Pl = g4.params(periodic=0, eps=[0.01], alpha=0.0025, leaf_max=lm)
        fl = g4.ForestGravity(sizes, Pl)
        fl.forces(pos, mass, box, aold, Pl)
        leaf_ms[lm] = _time(lambda: fl.forces(pos, mass, box, aold, Pl), 2)
        del fl
    res["leaf_autotune"] = {"best": min(leaf_ms, key=leaf_ms.get), "step_ms": leaf_ms,
                            "forces_per_s_best": n / (min(leaf_ms.values()) * 1e-3)}
    res["per_system_launches"] = {"ms_per_step": ms_sys, "ms_per_step_graphs": ms_sys_graph,
                                  "forest_speedup": ms_sys / ms,
                                  "forest_speedup_vs_graphs": ms_sys_graph / ms}
    # accuracy: 512 sampled sinks of 16 systems against the oracle's FP64 direct sum over each
    # whole system
    import oracle
    acc = fg.acc.double().cpu().numpy().T
    pick = np.random.default_rng(3005).choice(len(sizes), 16, replace=False)
    errs = []
    for k in pick:
        ps = systems[k]
        qk = pos[:, int(first[k]):int(first[k + 1])].cpu().numpy().view(np.uint32)
        sinks = np.sort(np.random.default_rng(int(k)).choice(ps.n, min(512, ps.n), replace=False))
        OP = oracle.OracleParams(box=float(box[k].item()), periodic=False, eps=np.array([0.01]))
        ad, _ = oracle.direct(qk, ps.mass, None, sinks, OP)
        ak = acc[int(first[k]):int(first[k + 1])][sinks]
        errs.append(np.linalg.norm(ak - ad, axis=1) / np.linalg.norm(ad, axis=1))
    e = np.concatenate(errs)
    res["accuracy_vs_direct"] = {"p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99)),
                                 "max": float(e.max()), "sample": f"512 sinks of each of 16 systems"}
    del g, tree1
    return res


def extra_bins(leaf_max):
    """Zoom box with two softening classes and six nested active subsets (1..100%), one force
    call per subset with its own tree, eager and replayed as one CUDA graph."""
    import torch
    from paper_2010_03567_gb300 import g4, synth
    ps = synth.zoom(176, 100.0, 1004)
    n = ps.n
    rs = 1.25 * 100.0 / (2 * 176)
    pos = torch.from_numpy(ps.pos).cuda()
    q, _ = g4.g4_int_coords(pos, True, 100.0)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    cls = torch.from_numpy(ps.eps_class).cuda()
    base = dict(box_size=100.0, periodic=1, r_s=rs, r_cut_factor=4.5, eps=list(ps.eps_table),
                leaf_max=leaf_max)
    tg = g4.TreeGravity(n, g4.params(**base, criterion=1, theta=0.5), with_cls=True)
    acc0, _ = tg.forces(q, mass, cls, None)
    aold = torch.linalg.vector_norm(acc0, dim=0).contiguous()
    order = torch.argsort(aold, descending=True).cpu().numpy()
    fracs = [0.01, 0.03, 0.10, 0.30, 0.60, 1.00]
    lists = [np.sort(order[:max(32, int(round(f * n)))]) for f in fracs]
    del tg
    P = g4.params(**base, alpha=0.0025)
    bf = g4.BinnedForces(n, lists, P, with_cls=True)
    forces = sum(len(a) for a in lists)
    eager = _time(lambda: bf.run(q, mass, cls, aold), 3)
    ref = [a.clone() for a in bf.acc]
    # accuracy of every bin's forces: 2048 sampled sinks per bin against the oracle's FP64
    # direct sum over that bin's active set (r < r_cut, both softening classes)
    import oracle
    q_np = q.cpu().numpy().view(np.uint32)
    OPb = oracle.OracleParams(box=100.0, periodic=True, eps=np.array(ps.eps_table), r_s=rs,
                              r_cut_factor=4.5)
    acc_bins = []
    for b, ix in enumerate(lists):
        sel = np.sort(np.random.default_rng(4004 + b).choice(len(ix), min(2048, len(ix)), replace=False))
        ad, _ = oracle.direct(np.ascontiguousarray(q_np[:, ix]), ps.mass[ix], ps.eps_class[ix], sel,
                              OPb, r_max=OPb.r_cut)
        ag = ref[b].double().cpu().numpy().T[ix[sel]]
        # the relative criterion bounds each node's error by alpha |a_old| with |a_old| the
        # total acceleration, while a bin's force (from the bin's own particles) can be far
        # smaller: the error in units of |a_old| is the quantity the criterion controls
        a_o = aold.double().cpu().numpy()[ix[sel]]
        e_o = np.linalg.norm(ag - ad, axis=1) / a_o
        acc_bins.append({"fraction": fracs[b], **_errors(ag, ad), "sample": int(len(sel)),
                         "err_over_aold_p99": float(np.percentile(e_o, 99)),
                         "err_over_aold_max": float(e_o.max())})
    bf.capture(q, mass, cls, aold)
    graph = _time(bf.replay, 3)
    same = all(torch.equal(a, b) for a, b in zip(ref, bf.acc))
    per_bin = [_time(lambda b=b: bf.run_bin(b, q, mass, cls, aold), 3) for b in range(len(lists))]
    ref_counts = [tgb.counts.clone() for tgb, _ in bf.bins]
    # partition of every bin's walk (g4_schedule_items) by (a) the cost model trained on C1-C3
    # and frozen (it has never seen this box), (b) the paper's q_i: the measured interactions
    # of the bin's previous force computation; against the plain 32-sink groups
    part = {}
    qi = [c.clone() for c in bf.measured_costs()]
    schemes = [("q_i_measured", qi)]
    cm = FROZEN.get("model")
    if cm is not None:
        preds = [cm.predict(g4.cost_features(tgb.tree, P, int(ix.shape[0]), tgb.aold_s))
                 for ix, (tgb, _) in zip(bf.idx, bf.bins)]
        schemes.insert(0, ("mlp_frozen", preds))
        part["mlp_frozen_vs_measured"] = [_rank_and_err(pr, lb) for pr, lb in zip(preds, qi)]
    counts_same = True
    for name, pr in schemes:
        bf.set_partition(pr)
        e_ms = _time(lambda: bf.run(q, mass, cls, aold), 3)
        pb = [_time(lambda b=b: bf.run_bin(b, q, mass, cls, aold), 3) for b in range(len(lists))]
        counts_same = counts_same and all(torch.equal(tgb.counts, c) for (tgb, _), c in zip(bf.bins, ref_counts))
        bf.capture(q, mass, cls, aold)
        g_ms = _time(bf.replay, 3)
        part[name] = {"eager_ms": e_ms, "graph_ms": g_ms, "per_bin_ms": pb,
                      "forces_per_s_graph": forces / (g_ms * 1e-3), "speedup_graph": graph / g_ms}
    part["interaction_counts_identical"] = bool(counts_same)
    bf.set_cost_model(None)
    return {"particles": n, "active_fractions": fracs, "forces_per_step": forces,
            "accuracy_vs_direct": acc_bins,
            "eager_ms": eager, "graph_ms": graph, "forces_per_s_eager": forces / (eager * 1e-3),
            "forces_per_s_graph": forces / (graph * 1e-3), "graph_equals_eager": bool(same),
            "per_bin_ms": per_bin,
            "cost_partition": part}


def extra_cost_model(tg, P, n):
    """Train the cost model on the counts of the last walk, schedule the walk's groups
    heaviest first, and time the walk against the plain PH order."""
    import torch
    from paper_2010_03567_gb300 import g4
    feats = g4.cost_features(tg.tree, P, n, tg.aold_s)
    labels = g4.cost_labels(tg.counts)
    g = torch.Generator(device="cuda").manual_seed(7)
    sub = torch.randperm(n, device="cuda", generator=g)[: min(n, 1 << 18)]
    cm = g4.CostModel(seed=1)
    t_train = _time(lambda: None, 1, warm=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = cm.train(feats[sub].contiguous(), labels[sub].contiguous(), steps=400, lr=3e-3)
    e1.record()
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1)
    pred = cm.predict(feats)
    walk = lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, acc=tg.acc_s,
                                        pot=tg.pot_s, counts=tg.counts)
    g4.set_group_order(tg.tree, None)
    ph_ms = _time(walk, 5)
    ref, ref_cnt = tg.acc_s.clone(), tg.counts.clone()
    lpt = {}
    same, dmax = True, 0.0
    for chunk in (1, 64, 512):
        order = g4.schedule_lpt(pred, chunk)
        g4.set_group_order(tg.tree, order)
        lpt[chunk] = _time(walk, 5)
        same = same and bool(torch.equal(ref_cnt, tg.counts))
        dmax = max(dmax, _max_rel_diff(tg.acc_s, ref))
    g4.set_group_order(tg.tree, None)
    p_np, l_np = pred.cpu().numpy(), labels.cpu().numpy()
    rk = lambda a: np.argsort(np.argsort(a))
    return {"train_ms": t_train, "train_samples": int(sub.shape[0]), "steps": 400,
            "loss_first_last": [float(losses[0]), float(losses[-1])],
            "rank_corr": float(np.corrcoef(rk(p_np), rk(l_np))[0, 1]),
            "mean_abs_err_log_cost": float(np.mean(np.abs(p_np - l_np))),
            "walk_ms_ph_order": ph_ms,
            "walk_ms_lpt_order": {f"chunk{c}": v for c, v in lpt.items()},
            "interaction_counts_identical": same, "forces_max_rel_diff": dmax}


def _max_rel_diff(a, b):
    """Largest |a - b| / |b| over the particles (forces as (3, n) tensors): the PH-order walk
    shares one walk among runs of groups, the scheduled orders walk every group on its own, so
    the same interactions are summed in another order."""
    import torch
    d = torch.linalg.vector_norm((a - b).double(), dim=0) / torch.linalg.vector_norm(b.double(), dim=0).clamp_min(1e-30)
    return float(d.max().item())


def _graph_time(fn, reps):
    """Capture one call of fn (a whole allocation-free pipeline step) in a CUDA graph and time
    its replays: what the step costs without host launch overhead."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                                   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return _time(g.replay, reps, warm=2)


def partition_gain(tg, P, n, step, reps=10, train_steps=400):
    """The cost model trained on the counts of the last walk partitions the walk into work items
    (g4_schedule_items); the same step is timed with plain 32-sink groups, with items from the
    model's predictions, and with items from the measured counts (the paper's q_i of the last
    step).  Every sink's interaction counts must be unchanged."""
    import torch
    from paper_2010_03567_gb300 import g4
    ref_counts = tg.counts.clone()
    labels = g4.cost_labels(tg.counts)
    feats = g4.cost_features(tg.tree, P, n, tg.aold_s)
    cm = g4.CostModel(seed=1)
    cm.train(feats, labels, steps=train_steps, lr=3e-3)
    pred = cm.predict(feats)
    walk = lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, acc=tg.acc_s,
                                        pot=tg.pot_s, counts=tg.counts)
    out = {"plain": {"walk_ms": _time(walk, reps), "step_ms_graph": _graph_time(step, reps)}}
    same = True
    for name, src in (("model", pred), ("measured_counts", labels)):
        items, ni = g4.schedule_items(src)
        g4.set_work_items(tg.tree, items, ni, n)
        out[name] = {"walk_ms": _time(walk, reps), "step_ms_graph": _graph_time(step, reps),
                     "items": int(ni.item())}
        same = same and bool(torch.equal(tg.counts, ref_counts))
        g4.set_work_items(tg.tree, None)
    out["groups"] = (n + 31) // 32
    out["interaction_counts_identical"] = same
    out["speedup_step_model"] = out["plain"]["step_ms_graph"] / out["model"]["step_ms_graph"]
    # the partition granularity picked by the autotuner (items per resident warp; 0 = none)
    from paper_2010_03567_gb300 import autotune
    best, times = autotune.tune_partition(autotune.gpu_partition_timer(tg, P, pred),
                                          torch.cuda.get_device_name(), n, P, use_cache=False)
    out["autotuned_partition"] = {"items_per_warp": best, "walk_ms": times}
    return out


def _errors(a, ref):
    """Relative error percentiles |a - ref| / |ref|; sinks whose reference force is exactly zero
    (no source inside r_cut, e.g. in sparse active subsets) are counted apart, with the number
    of them where a is not zero as well."""
    rn = np.linalg.norm(ref, axis=1)
    z = rn == 0
    e = np.linalg.norm(a[~z] - ref[~z], axis=1) / rn[~z]
    out = {"p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99)), "max": float(e.max())}
    if z.any():
        out["zero_reference"] = int(z.sum())
        out["zero_reference_nonzero_result"] = int(np.count_nonzero(np.linalg.norm(a[z], axis=1)))
    return out


# Cost-model training samples logged from the walks of C1 (Plummer sphere), C2 (128^3 box) and
# C3 (the headline 256^3 box); the network trained once on them is frozen and applied to the
# time bins of the zoom box and to the 512^3 box, which it has never seen.
TRAIN_SAMPLES = {}
FROZEN = {}


def collect_cost_samples(name, tree, P, n, aold_s, counts, k=1 << 16):
    """Tree features and measured-cost labels (log(1 + PP + 5 PN)) of k sampled sinks."""
    import torch
    from paper_2010_03567_gb300 import g4
    feats = g4.cost_features(tree, P, n, aold_s)
    labels = g4.cost_labels(counts)
    gen = torch.Generator(device="cuda").manual_seed(11)
    sub = torch.randperm(n, device="cuda", generator=gen)[: min(n, k)]
    TRAIN_SAMPLES[name] = (feats[sub].contiguous().clone(), labels[sub].contiguous().clone())


def extra_frozen_model():
    """Train the cost model once on the samples of C1-C3 and freeze it."""
    import torch
    from paper_2010_03567_gb300 import g4
    if not TRAIN_SAMPLES:
        return {"error": "no training samples"}
    f = torch.cat([v[0] for v in TRAIN_SAMPLES.values()]).contiguous()
    lab = torch.cat([v[1] for v in TRAIN_SAMPLES.values()]).contiguous()
    cm = g4.CostModel(seed=1)
    losses = cm.train(f, lab, steps=600, lr=3e-3)
    FROZEN["model"] = cm
    return {"trained_on": {k: int(v[1].shape[0]) for k, v in TRAIN_SAMPLES.items()},
            "steps": 600, "loss_first_last": [float(losses[0]), float(losses[-1])]}


def _rank_and_err(pred, labels):
    p_np, l_np = pred.cpu().numpy(), labels.cpu().numpy()
    rk = lambda a: np.argsort(np.argsort(a))
    return {"rank_corr": float(np.corrcoef(rk(p_np), rk(l_np))[0, 1]),
            "mean_abs_err_log_cost": float(np.mean(np.abs(p_np - l_np))),
            "mean_rel_err_cost": float(np.mean(np.abs(np.expm1(p_np) - np.expm1(l_np)) /
                                               np.maximum(np.expm1(l_np), 1.0)))}


def extra_fp64(tg, P, n, sample_ref):
    """The same walk in FP64 (FP64 multipoles and interactions) on the headline box: the FP32
    walk's error against it, and both against the FP64 direct sum on the sample."""
    import torch
    from paper_2010_03567_gb300 import g4
    P64 = g4.G4Params.from_buffer_copy(P)
    P64.precision = 1
    a32, _, _ = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)   # FP32, sorted order
    tg.tree.multipoles(tg.pos_s, tg.mass_s, None, tg.aold_s, P64)
    acc64 = torch.zeros_like(tg.acc_s)
    ms = _time(lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P64, acc=acc64,
                                            pot=None, counts=None), 1)
    tg.tree.multipoles(tg.pos_s, tg.mass_s, None, tg.aold_s, P)    # restore the FP32 state
    res = {"walk_ms_fp64": ms, "fp32_vs_fp64_gpu": _errors(a32.double().cpu().numpy().T,
                                                           acc64.double().cpu().numpy().T)}
    if sample_ref is not None:
        sinks, ad = sample_ref
        inv = torch.empty_like(tg.perm)
        inv[tg.perm.long()] = torch.arange(n, dtype=torch.int32, device="cuda")
        rows = inv[torch.from_numpy(sinks).cuda().long()].long()
        res["fp64_gpu_vs_direct"] = _errors(acc64[:, rows].double().cpu().numpy().T, ad)
    return res


def extra_plummer(leaf_max):
    """Isolated Plummer sphere, N = 16384, p = 3, alpha = 0.0025 with |a_old| from the GPU
    direct sum; accuracy against the oracle's FP64 direct sum."""
    import torch
    import oracle
    from paper_2010_03567_gb300 import g4, synth
    ps = synth.plummer_16k()
    q, fr = g4.g4_int_coords(torch.from_numpy(ps.pos).cuda(), False)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    box = float(fr[3].item())
    PD = g4.params(box_size=box, periodic=0, eps=[0.01], leaf_max=leaf_max)
    ad_gpu, _ = g4.g4_direct(q, mass, None, PD)
    aold = torch.linalg.vector_norm(ad_gpu, dim=0).contiguous()
    P = g4.params(box_size=box, periodic=0, eps=[0.01], alpha=0.0025, leaf_max=leaf_max)
    tg = g4.TreeGravity(ps.n, P)
    ms = _time(lambda: tg.forces(q, mass, None, aold, P), 10)
    ms_graph = _graph_time(lambda: tg.forces(q, mass, None, aold, P), 10)
    acc = tg.acc.double().cpu().numpy().T
    OP = oracle.OracleParams(box=box, periodic=False, eps=np.array([0.01]))
    ad, _ = oracle.direct(q.cpu().numpy().view(np.uint32), ps.mass, None, np.arange(ps.n), OP)
    cnt = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    collect_cost_samples("C1_plummer16k", tg.tree, P, ps.n, tg.aold_s, tg.counts)
    part = partition_gain(tg, P, ps.n, lambda: tg.forces(q, mass, None, aold, P))
    # expansion orders p = 1..5 at the same alpha: time of a step and accuracy (Sec. 2.2.2)
    orders = {}
    for po in (1, 2, 3, 4, 5):
        Po = g4.params(box_size=box, periodic=0, eps=[0.01], alpha=0.0025, leaf_max=leaf_max, order_p=po)
        tgo = g4.TreeGravity(ps.n, Po)
        mso = _time(lambda: tgo.forces(q, mass, None, aold, Po), 5)
        co = tgo.counts.to(torch.int64).sum(dim=1).cpu().numpy()
        orders[po] = {"ms_per_step": mso, "pn_per_step": int(co[1]),
                      "accuracy_vs_direct": _errors(tgo.acc.double().cpu().numpy().T, ad)}
        del tgo
    # the leaf threshold tuned for this workload (one complete force computation per candidate)
    from paper_2010_03567_gb300 import autotune
    best_leaf, leaf_ms = autotune.tune(autotune.gpu_step_timer(q, mass, aold, P),
                                       torch.cuda.get_device_name(), ps.n, P, use_cache=False)
    return {"particles": ps.n, "ms_per_step": ms, "forces_per_s": ps.n / (ms * 1e-3),
            "ms_per_step_graph": ms_graph, "forces_per_s_graph": ps.n / (ms_graph * 1e-3),
            "pp_per_step": int(cnt[0]), "pn_per_step": int(cnt[1]),
            "accuracy_vs_direct": _errors(acc, ad), "cost_partition": part,
            "leaf_autotune": {"best": best_leaf, "step_ms": leaf_ms}, "orders": orders,
            "forces_per_s_graph_model_items": ps.n / (part["model"]["step_ms_graph"] * 1e-3)}


def extra_softened(leaf_max):
    """Softened node interactions (Sec. 2.7) on a set where softenings are comparable to the
    node sizes: the 16k Plummer sphere with two softening classes (eps = 0.3 and 0.08, every
    fourth particle in the second), tree walk (p = 3, alpha = 0.005, leaf 4) and FMM (p = 4)
    under the GADGET-3 rule (every pair closer than 2.8 eps_ij opened) and the GADGET-4 rule
    (the softened kernel's expansion unless both sides are mixed): time, interactions and
    accuracy against the oracle's FP64 direct sum with pair softening max(eps_i, eps_j)."""
    import torch
    import oracle
    from paper_2010_03567_gb300 import g4, synth
    ps = synth.plummer_16k()
    ps.eps_table = np.array([0.3, 0.08])
    ps.eps_class = np.zeros(ps.n, np.uint8)
    ps.eps_class[::4] = 1
    q, fr = g4.g4_int_coords(torch.from_numpy(ps.pos).cuda(), False)
    box = float(fr[3].item())
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    cls = torch.from_numpy(ps.eps_class).cuda()
    q_np = q.cpu().numpy().view(np.uint32)
    OP = oracle.OracleParams(box=box, periodic=False, eps=ps.eps_table)
    ad, _ = oracle.direct(q_np, ps.mass, ps.eps_class, np.arange(ps.n), OP)
    aold = torch.from_numpy(np.linalg.norm(ad, axis=1).astype(np.float32)).cuda()
    base = dict(box_size=box, periodic=0, eps=list(ps.eps_table), leaf_max=4, alpha=0.005)
    tg = g4.TreeGravity(ps.n, g4.params(**base), with_cls=True)
    ws = None
    out = {"particles": ps.n, "eps": [0.3, 0.08]}
    for soft in (0, 1):
        P = g4.params(**base, soft_nodes=soft)
        ms = _time(lambda: tg.forces(q, mass, cls, aold, P), 5)
        tg.tree.status()
        c = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
        ag = tg.acc.cpu().numpy().T.astype(np.float64)
        tree = {"ms_per_step": ms, "pp_per_step": int(c[0]), "pn_per_step": int(c[1]),
                "accuracy_vs_direct": _errors(ag, ad)}
        P4 = g4.params(**base, order_p=4, soft_nodes=soft)
        tg.prepare(q, mass, cls, aold, P4)
        if ws is None:
            ws = torch.empty(tg.tree.fmm_workspace(P4) + 256, dtype=torch.uint8, device="cuda")
        res = {}

        def step():
            tg.prepare(q, mass, cls, aold, P4)
            res["r"] = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, tg.cls_s, tg.aold_s, P4, workspace=ws)
            g4.g4_scatter(tg.perm, res["r"][0], res["r"][1], out=(tg.acc, tg.pot))

        fms = _time(step, 5)
        tg.tree.status()
        cnt = res["r"][2].to(torch.int64).sum(dim=1).cpu().numpy()
        af = tg.acc.cpu().numpy().T.astype(np.float64)
        fmm = {"ms_per_step": fms, "pp_per_step": int(cnt[0]), "pn_per_step": int(cnt[1]),
               "accuracy_vs_direct": _errors(af, ad)}
        out["gadget4_rule" if soft else "gadget3_rule"] = {"tree": tree, "fmm": fmm}
    g3, g4r = out["gadget3_rule"], out["gadget4_rule"]
    out["speedup_tree"] = g3["tree"]["ms_per_step"] / g4r["tree"]["ms_per_step"]
    out["speedup_fmm"] = g3["fmm"]["ms_per_step"] / g4r["fmm"]["ms_per_step"]
    del ws
    return out


def extra_ewald(leaf_max):
    """The pure periodic tree with the Ewald correction (Sec. 2.2.4, no PM): a 64^3 periodic
    box (L = 100, rms displacement 0.5 spacings), p = 3, relative criterion alpha = 0.0025 with
    |a_old| from a geometric bootstrap walk; forces/s (keys to scatter), parity on sampled sinks
    against the oracle's walk with exact Ewald tensors, the pure periodic FMM (p = 4) on the
    same box, and the tree's accuracy on a 16^3 box against the exact periodic direct sum (with
    the nearest images alone for contrast)."""
    import torch
    import oracle
    from paper_2010_03567_gb300 import g4, synth
    L, ns = 100.0, 64
    ps = synth.zeldovich(ns, L, 0.5, 1011)
    base = dict(box_size=L, periodic=1, eps=list(ps.eps_table), order_p=3, leaf_max=leaf_max,
                ewald=1)
    q, _ = g4.g4_int_coords(torch.from_numpy(ps.pos).cuda(), True, L)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    tg = g4.TreeGravity(ps.n, g4.params(**base, criterion=1, theta=0.5))
    a0, _ = tg.forces(q, mass, None, None)
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    P = g4.params(**base, alpha=0.0025)
    ms = _time(lambda: tg.forces(q, mass, None, aold, P), 3)
    tg.tree.status()
    c = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    sinks = np.sort(np.random.default_rng(4111).choice(ps.n, 64, replace=False))
    q_np = q.cpu().numpy().view(np.uint32)
    OP = oracle.OracleParams(box=L, periodic=True, eps=ps.eps_table, alpha=0.0025, order=3,
                             ewald=True)
    run = oracle.prepare(q_np, ps.mass, None, aold.double().cpu().numpy(), OP, leaf_max)
    ao, _, _ = oracle.tree_forces(run, sinks)
    ag = tg.acc.cpu().numpy().T[sinks].astype(np.float64)
    out = {"particles": ps.n, "ms_per_step": ms, "forces_per_s": ps.n / (ms * 1e-3),
           "pp_per_step": int(c[0]), "pn_per_step": int(c[1]),
           "parity_vs_oracle_walk": {**_errors(ag, ao), "sample": int(len(sinks))}}
    # the pure periodic FMM (p = 4) on the same box and |a_old|
    P4 = g4.params(**dict(base, order_p=4), alpha=0.0025)
    tg.prepare(q, mass, None, aold, P4)
    ws = torch.empty(tg.tree.fmm_workspace(P4) + 256, dtype=torch.uint8, device="cuda")
    res = {}

    def fstep():
        tg.prepare(q, mass, None, aold, P4)
        res["r"] = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P4, workspace=ws)

    fms = _time(fstep, 3)
    tg.tree.status()
    acc_s, _, cnt, mom = res["r"]
    amag = torch.linalg.vector_norm(acc_s.double(), dim=0)
    out["fmm"] = {"ms_per_step": fms, "forces_per_s": ps.n / (fms * 1e-3), "order_p": 4,
                  "momentum_rel": float(torch.linalg.vector_norm(mom).item()
                                        / (tg.mass_s.double() * amag).sum().item()),
                  "pp_per_step": int(cnt[0].to(torch.int64).sum().item()),
                  "pn_per_step": int(cnt[1].to(torch.int64).sum().item())}
    del ws
    # the method's accuracy against the exact periodic sum, 16^3 box
    ps2 = synth.zeldovich(16, L, 0.5, 1012)
    q2, _ = g4.g4_int_coords(torch.from_numpy(ps2.pos).cuda(), True, L)
    m2 = torch.from_numpy(ps2.mass.astype(np.float32)).cuda()
    s2 = np.sort(np.random.default_rng(4112).choice(ps2.n, 128, replace=False))
    q2_np = q2.cpu().numpy().view(np.uint32)
    ad, _ = oracle.ewald_direct(q2_np, ps2.mass, None, s2,
                                oracle.OracleParams(box=L, periodic=True, eps=ps2.eps_table))
    acc_small = {}
    for ew in (1, 0):
        b2 = dict(base, ewald=ew)
        t2 = g4.TreeGravity(ps2.n, g4.params(**b2, criterion=1, theta=0.5))
        x0, _ = t2.forces(q2, m2, None, None)
        ao2 = torch.linalg.vector_norm(x0, dim=0).contiguous()
        a2, _ = t2.forces(q2, m2, None, ao2, g4.params(**b2, alpha=0.0025))
        acc_small["ewald" if ew else "nearest_images_only"] = _errors(
            a2.cpu().numpy().T[s2].astype(np.float64), ad)
    out["accuracy_vs_exact_periodic_sum_16cubed"] = {**acc_small, "sample": int(len(s2))}
    return out


def extra_box128(leaf_max):
    """The 128^3 periodic box (L = 100, rms displacement 0.5 spacings), p = 3, alpha = 0.0025;
    accuracy on a 65536-particle subset against the oracle's FP64 direct sum (r < r_cut)."""
    import torch
    import oracle
    from paper_2010_03567_gb300 import g4, synth
    L, ns = 100.0, 128
    ps = synth.zeldovich(ns, L, 0.5, 1002)
    wp = dict(box_size=L, periodic=1, r_s=1.25 * L / 256, r_cut_factor=4.5, eps=[L / ns / 30],
              leaf_max=leaf_max)
    q, _ = g4.g4_int_coords(torch.from_numpy(ps.pos).cuda(), True, L)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    tg = g4.TreeGravity(ps.n, g4.params(**wp, criterion=1, theta=0.5))
    a0, _ = tg.forces(q, mass)
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    P = g4.params(**wp, alpha=0.0025)
    ms = _time(lambda: tg.forces(q, mass, None, aold, P), 10)
    ms_graph = _graph_time(lambda: tg.forces(q, mass, None, aold, P), 10)
    sinks = synth.subset(ps.n, 65536, 2002)
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(wp["eps"]), r_s=wp["r_s"],
                             r_cut_factor=4.5)
    ad, _ = oracle.direct(q.cpu().numpy().view(np.uint32), ps.mass, None, sinks, OP, r_max=OP.r_cut)
    acc = tg.acc.double().cpu().numpy().T[sinks]
    cnt = tg.counts.to(torch.int64).sum(dim=1).cpu().numpy()
    collect_cost_samples("C2_128cubed", tg.tree, P, ps.n, tg.aold_s, tg.counts)
    return {"particles": ps.n, "ms_per_step": ms, "forces_per_s": ps.n / (ms * 1e-3),
            "ms_per_step_graph": ms_graph, "forces_per_s_graph": ps.n / (ms_graph * 1e-3),
            "pp_per_step": int(cnt[0]), "pn_per_step": int(cnt[1]),
            "accuracy_vs_direct": {**_errors(acc, ad), "sample": len(sinks)}}


def extra_c5(leaf_max):
    """512^3 box (L = 1000, rms 0.5 spacings, r_s = 1.25 L/1024): the cost model trained on the
    counts logged by the first walk orders the groups of the next walks (heaviest first);
    forces/s against the plain PH order, prediction error against the measured counts."""
    import torch
    from paper_2010_03567_gb300 import g4, synth
    ns, L = 512, 1000.0
    pos = synth.zeldovich_gpu(ns, L, 0.5, 1006)
    q, _ = g4.g4_int_coords(pos, True, L)
    del pos
    torch.cuda.empty_cache()
    n = ns ** 3
    mass = torch.ones(n, dtype=torch.float32, device="cuda")
    wp = dict(box_size=L, periodic=1, r_s=1.25 * L / 1024, r_cut_factor=4.5, eps=[L / ns / 30],
              leaf_max=leaf_max)
    tg = g4.TreeGravity(n, g4.params(**wp, criterion=1, theta=0.5))
    a0, _ = tg.forces(q, mass)
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    del a0
    P = g4.params(**wp, alpha=0.0025)
    plain = _time(lambda: tg.forces(q, mass, None, aold, P), 2)
    # accuracy: 512 sampled sinks against the oracle's FP64 direct sum (r < r_cut) over all
    # 134M particles
    import oracle
    sinks = synth.subset(n, 512, 2006)
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(wp["eps"]), r_s=wp["r_s"],
                             r_cut_factor=4.5)
    q_np = q.cpu().numpy().view(np.uint32)
    ad, _ = oracle.direct(q_np, np.ones(n), None, sinks, OP, r_max=OP.r_cut)
    del q_np
    accuracy = {**_errors(tg.acc[:, torch.from_numpy(sinks).cuda().long()].double().cpu().numpy().T, ad),
                "sample": len(sinks)}
    # the cost model frozen after training on C1-C3 (it has never seen this box) against the
    # paper's q_i (the measured interactions of the previous walk): prediction quality and the
    # walk with groups ordered heaviest first (chunks of 64 groups) by either, against PH order
    walk = lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, acc=tg.acc_s,
                                        pot=tg.pot_s, counts=tg.counts)
    labels = g4.cost_labels(tg.counts).clone()
    frozen = {}
    cm = FROZEN.get("model")
    ph_ms = _time(walk, 3)
    ref, ref_cnt = tg.acc_s.clone(), tg.counts.clone()
    sources = [("q_i_measured", labels)]
    if cm is not None:
        pred = cm.predict(g4.cost_features(tg.tree, P, n, tg.aold_s))
        frozen["mlp_frozen_vs_measured"] = _rank_and_err(pred, labels)
        sources.insert(0, ("mlp_frozen", pred))
    for name, src in sources:
        g4.set_group_order(tg.tree, g4.schedule_lpt(src, 64))
        frozen[name] = {"walk_ms_lpt_chunk64": _time(walk, 3),
                        "interaction_counts_identical": bool(torch.equal(ref_cnt, tg.counts)),
                        "forces_max_rel_diff": _max_rel_diff(tg.acc_s, ref)}
    g4.set_group_order(tg.tree, None)
    frozen["walk_ms_ph_order"] = ph_ms
    res = {"out_of_sample": frozen, "in_sample": extra_cost_model(tg, P, n)}
    res.update({"particles": n, "ms_per_step_ph_order": plain,
                "forces_per_s_ph_order": n / (plain * 1e-3), "accuracy_vs_direct": accuracy})
    del tg
    return res


def run_pm_only(args):
    """PM long-range calls on the bench workload (for launch lists and captures of the PM
    kernels): mesh 2 N_side per axis."""
    import torch
    from paper_2010_03567_gb300 import g4, synth
    n_side = args.n_side
    L = L_BOX * n_side / N_SIDE
    ps = synth.zeldovich(n_side, L, RMS, SEED)
    wp = workload_params(n_side, L, args.leaf_max)
    pos = torch.from_numpy(ps.pos).cuda()
    q, _ = g4.g4_int_coords(pos, True, L)
    del pos
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    P = g4.params(**wp)
    tg = g4.TreeGravity(ps.n, P)
    tg.prepare(q, mass, None, None, P)          # PH order, as TreePMGravity calls it
    ng = 2 * n_side
    ws = torch.empty(g4.g4_pm_workspace(ng) + 256, dtype=torch.uint8, device="cuda")
    acc = torch.zeros((3, ps.n), dtype=torch.float32, device="cuda")
    call = lambda: g4.g4_pm_long_range(tg.pos_s, tg.mass_s, P, ng, acc=acc, workspace=ws)
    ms = _time(call, max(1, args.steps), warm=1)
    print(json.dumps({"pm_only": True, "n_particles": ps.n, "n_grid": ng, "calls": args.steps,
                      "ms_per_call": ms}), flush=True)
    return 0


def run_fmm_only(args):
    """FMM calls on the bench workload (for launch lists and captures of the FMM kernels)."""
    import torch
    from paper_2010_03567_gb300 import g4, synth
    n_side = args.n_side
    L = L_BOX * n_side / N_SIDE
    ps = synth.zeldovich(n_side, L, RMS, SEED)
    wp = workload_params(n_side, L, args.leaf_max)
    pos = torch.from_numpy(ps.pos).cuda()
    q, _ = g4.g4_int_coords(pos, True, L)
    del pos
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    tg = g4.TreeGravity(ps.n, g4.params(**{**wp, "criterion": 1, "theta": 0.5}))
    a0, _ = tg.forces(q, mass)
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    del tg, a0
    P4 = g4.params(**{**wp, "order_p": 4})
    tg = g4.TreeGravity(ps.n, P4)
    tg.prepare(q, mass, None, aold, P4)
    ws = torch.empty(tg.tree.fmm_workspace(P4) + 256, dtype=torch.uint8, device="cuda")
    call = lambda: tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P4, workspace=ws)
    ms = _time(call, max(1, args.steps), warm=1)
    tg.tree.status()
    print(json.dumps({"fmm_only": True, "n_particles": ps.n, "order_p": 4, "calls": args.steps,
                      "ms_per_call": ms}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FMM, batched-systems, time-bin and cost-model measurements")
    ap.add_argument("--extras", default=None,
                    help="comma-separated names of the extra entries to run (default: all)")
    ap.add_argument("--leaf-max", type=int, default=None,
                    help="leaf threshold of the tree (default: the tuned value)")
    ap.add_argument("--pm-only", action="store_true",
                    help="profiling aid: --steps PM long-range calls on the workload's particles "
                         "(mesh 2 N_side per axis); prints their mean time, not the bench line")
    ap.add_argument("--fmm-only", action="store_true",
                    help="profiling aid: bootstrap walk, then --steps FMM calls (p = 4) on the workload; "
                         "prints their mean time, not the bench line")
    ap.add_argument("--n-side", type=int, default=N_SIDE,
                    help="particles per side (default 256: the headline workload; smaller sizes "
                         "keep the spacing, split and softening, for profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "gb300":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.pm_only:
        return run_pm_only(args)
    if args.fmm_only:
        return run_fmm_only(args)
    return run_gpu(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
