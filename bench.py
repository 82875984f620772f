"""Benchmark: leapfrog steps of the Barnes-Hut tree force on one GB300.

Workload (default): Hernquist halo, N = 2^24, theta = 0.5, quadrupole
superparticles, n_leaf = 16, n_grp = 128, eps = 0.005, dt = 1/512; FP32-
relative pipeline, with the all-FP64 pipeline of the same library timed on
one step beside it.  A step is kick + drift + the whole force calculation
(root box, keys, sort, reorder, octree, moments, groups, walk, force) +
kick.  Inputs are resident in HBM and far larger than L2.

Metric: particle-particle + particle-superparticle interactions per second
(sum over i-groups of n_i * (|EPJ| + |SPJ|)), with ms/step beside it.

Under torchrun each rank steps its own replica (the single-system path has
no data-parallel split without a domain decomposition); ``value`` is the sum
over ranks, timed by the slowest rank.
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

# FP32-lane operations of one interaction as the kernels evaluate the
# formulas (FMA = 1): particle-particle and monopole superparticle 13,
# quadrupole superparticle 32; plus one MUFU reciprocal square root each.
OPS_EPJ = 13
OPS_SPJ_MONO = 13
OPS_SPJ_QUAD = 32
# The algorithmic count of the measurement plan: 13 operations per
# particle-particle interaction and about twice that, 26, per quadrupole
# superparticle (the paper's cost ratio of a quadrupole to a monopole term,
# Sect. 5.5); the roofline fraction on this count is reported beside the
# instruction count's.
# Short-range mode (algorithmic FP32 operations): a candidate pair's r^2
# and comparison, a neighbour's Wendland C6 term and sum.
OPS_SR_CAND = 7
OPS_SR_NB = 10
ALG_EPJ = 13
ALG_SPJ_MONO = 13
ALG_SPJ_QUAD = 26


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--model", default="hernquist")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--n-leaf", type=int, default=16)
    ap.add_argument("--n-grp", type=int, default=256)
    ap.add_argument("--eps", type=float, default=0.005)
    ap.add_argument("--dt", type=float, default=1.0 / 512.0)
    ap.add_argument("--mono", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ensemble", action="store_true",
                    help="the ensemble workload: 4096 Plummer clusters, N log-uniform in "
                         "[256, 65536], eps = 1/(4 N^1/3), theta 0.5 monopole, dt 1/256")
    ap.add_argument("--n-sys", type=int, default=4096)
    ap.add_argument("--theta-target", type=float, default=None,
                    help="choose the opening angle whose median force error against the GPU direct "
                         "sum on --n-sample rows meets this target (one JSON line)")
    ap.add_argument("--n-sample", type=int, default=4096)
    ap.add_argument("--sph", action="store_true",
                    help="short-range mode: SPH density (Wendland C6) of a uniform random cube with "
                         "the cutoff at 4.2 mean inter-particle distances, i-dependent cutoff")
    ap.add_argument("--suite", action="store_true",
                    help="one JSON line per workload configuration: Plummer 2^20 (10 steps), "
                         "Hernquist 2^24 at theta 0.3/0.5/0.7, clumpy 2^26; with force errors "
                         "against the FP64 direct sum on a random subsample and energy drift")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the other workload configurations measured after the headline run")
    ap.add_argument("--user-law", action="store_true",
                    help="a user interaction law compiled at run time, timed on the benchmark's lists "
                         "beside the built-in force kernel")
    ap.add_argument("--largest", action="store_true",
                    help="the clumpy mixture at the largest particle count that fits the device "
                         "(one JSON line: throughput, force error, drift, bytes per particle)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep n_leaf / n_grp as given instead of the autotuner's choice")
    return ap.parse_args()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the force kernel, from an ncu capture of this workload; each holds for the
# force-kernel source whose SHA-256 starts with the recorded prefix, and the
# bench reports null once that source has changed
FORCE_TRAFFIC = {
    "hernquist N=16777216 theta=0.5 quad n_leaf=16 n_grp=256 eps=0.005 dt=0.00195312":
        ("80cf8cab93dcebe0", 4.2531e9 + 532.69e6),
}


def force_traffic(workload: str):
    import hashlib
    rec = FORCE_TRAFFIC.get(workload)
    if rec is None:
        return None
    src = os.path.join(ROOT, "paper_1601_03138_gb300", "csrc", "force.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    return rec[1] if sha.startswith(rec[0]) else None


# Algorithmic DRAM bytes of the HBM-bound stages: per particle, and per
# octree node where the stage writes nodes (each kernel's reads and writes
# of its inputs and outputs, once).
STAGE_BYTES = {
    # root box (x, y, z read) + Morton keys (x, y, z read, key written)
    "ms_box_keys": (24 + 32, 0),
    # 8 stable LSD passes of 8 bits: pass 0 reads keys and writes (key,
    # index), passes 1-7 read and write (key, index)
    "ms_sort": (8 + 12 + 7 * 24, 0),
    # permutation and 8 FP64 fields + id gathered, written in key order,
    # FP32 hi/lo copies and the three products m x written
    "ms_permute": (4 + 64 + 4 + 64 + 4 + 32 + 24, 0),
    # sorted keys, per-position first differing level and leaf level; node
    # records written
    "ms_build": (16 + 4, 37),
    # particle positions and masses read; node sums, centres, quadrupoles
    # and their FP32 copies written
    "ms_moments": (32, 200),
}
# The coherent time-step sort: the key pass also writes each key's bucket;
# the sort is a scatter into the buckets (key and bucket read, key and
# position written) and the per-bucket sort (the same 12 bytes read and
# written again).
STAGE_BYTES_COHERENT = dict(STAGE_BYTES, ms_box_keys=(24 + 24 + 12, 0), ms_sort=(12 + 12 + 12 + 12, 0))


def stage_hbm(stages_ms, n, n_nodes, peak_gbs, coherent=False):
    """Algorithmic GB/s and fraction of the measured HBM copy bandwidth of
    the HBM-bound stages (the byte counts of the sort the call took)."""
    out = {}
    for k, (bp, bn) in (STAGE_BYTES_COHERENT if coherent else STAGE_BYTES).items():
        ms = stages_ms.get(k)
        if not ms:
            continue
        b = bp * n + bn * n_nodes
        out[k[3:]] = {"bytes": b, "gb_s": b / (ms * 1e6), "frac": b / (ms * 1e6) / peak_gbs}
    return out


def combine_ranks(t_local: float, units_local: float, world: int, device: str):
    """Whole-job numbers over ranks: the slowest rank's time and the sum of
    the units every rank processed (all_gather over the default group)."""
    if world <= 1:
        return t_local, units_local
    import torch
    tt = torch.tensor([t_local, float(units_local)], device=device, dtype=torch.float64)
    gathered = [torch.zeros_like(tt) for _ in range(world)]
    torch.distributed.all_gather(gathered, tt)
    return max(float(g[0]) for g in gathered), sum(float(g[1]) for g in gathered)


def partition_systems(sizes, world: int):
    """Contiguous ranges [a, b) of systems per rank, balanced by the tree
    cost of a system, taken as N log2 N; every system in exactly one range."""
    sizes = np.asarray(sizes, dtype=np.float64)
    cost = sizes * np.log2(np.maximum(sizes, 2.0))
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    cuts = [0]
    for r in range(1, world):
        k = int(np.searchsorted(cum, cum[-1] * r / world))
        cuts.append(min(max(k, cuts[-1]), len(sizes)))
    cuts.append(len(sizes))
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_inputs(args):
    import ics
    seed = ics.SEED_BASE + 3
    return ics.make(args.model, args.n, seed, args.eps)


def workload_name(args):
    mom = "mono" if args.mono else "quad"
    return (f"{args.model} N={args.n} theta={args.theta} {mom} n_leaf={args.n_leaf} "
            f"n_grp={args.n_grp} eps={args.eps} dt={args.dt:.6g}")


def cpu_sample(pos, mass, eps, args, seconds, built=None, seed=1):
    """The oracle as it stands on a bounded sample of the same workload:
    full tree build, then walk + force for a random subset of i-groups sized
    to about `seconds` of CPU work, the build charged in proportion to the
    particles sampled.  `built` = (tree, build seconds) reuses one build of
    the same particle set.  Returns a cpu_baseline dict."""
    import oracle
    if built is None:
        t0 = time.perf_counter()
        tree = oracle.Tree(pos, mass, eps, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp,
                           quad=not args.mono)
        t_build = time.perf_counter() - t0
    else:
        tree, t_build = built
    ng = tree.n_groups
    rng = np.random.default_rng(seed)
    order = rng.permutation(ng)
    done, inter, t_force, k = 0, 0, 0.0, 16
    gcount = tree.groups()["count"]
    while t_force < seconds and done < ng:
        sel = order[done:done + k]
        t1 = time.perf_counter()
        _, _, tot = tree.force(sel)
        t_force += time.perf_counter() - t1
        inter += tot[2]
        done += len(sel)
        k *= 2
    frac = gcount[order[:done]].sum() / len(pos)
    t_eff = t_force + t_build * frac
    return {"value": inter / t_eff, "unit": "interactions/s", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": (f"FP64 C oracle: full tree build of the same {len(pos)}-particle set "
                       f"({t_build:.1f} s, charged pro rata) + walk and force of {done} of {ng} "
                       f"random i-groups ({frac * 100:.2f}% of particles, {inter:.3e} "
                       f"interactions, {t_force:.1f} s)")}


def cpu_baseline(pos, mass, eps, args, seconds):
    """The oracle on all host cores (cpu_sample) and on one core.  The one-core
    figure walks and forces the first groups of one random order for about
    `seconds` / 2 on one thread, and the same groups again on all cores, so the
    two are comparable; the tree build is charged pro rata, its one-core time
    measured on the first 2^20 particles (a fair subsample of the same
    distribution) and scaled by N log N."""
    import oracle
    cores = oracle.get_threads()
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, mass, eps, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp,
                       quad=not args.mono)
    t_build = time.perf_counter() - t0
    main = cpu_sample(pos, mass, eps, args, seconds, built=(tree, t_build))
    n = len(pos)
    order = np.random.default_rng(7).permutation(tree.n_groups)
    gcount = tree.groups()["count"]
    oracle.set_threads(1)
    try:
        m1 = min(len(pos), 1 << 20)
        t0 = time.perf_counter()
        oracle.Tree(pos[:m1], mass[:m1], eps[:m1], theta=args.theta, n_leaf=args.n_leaf,
                    n_grp=args.n_grp, quad=not args.mono)
        t_b1 = (time.perf_counter() - t0) * (n * np.log2(max(n, 2))) / (m1 * np.log2(max(m1, 2)))
        done, inter, t1, k = 0, 0, 0.0, 4
        while t1 < seconds / 2 and done < len(order):
            sel = order[done:done + k]
            t2 = time.perf_counter()
            _, _, tot = tree.force(sel)
            t1 += time.perf_counter() - t2
            inter += tot[2]
            done += len(sel)
            k *= 2
    finally:
        oracle.set_threads(cores)
    t2 = time.perf_counter()
    tree.force(order[:done])
    tn = time.perf_counter() - t2
    frac = gcount[order[:done]].sum() / n
    main["cores_1"] = {
        "value": inter / (t1 + t_b1 * frac), "cores": 1,
        "value_all_cores_same_groups": inter / (tn + t_build * frac), "cores_all": cores,
        "sample": (f"walk and force of the same {done} random i-groups ({frac * 100:.3f}% of "
                   f"particles, {inter:.3e} interactions) on 1 core ({t1:.1f} s) and on {cores} "
                   f"cores ({tn:.2f} s); build charged pro rata: {t_build:.1f} s measured on "
                   f"{cores} cores, {t_b1:.1f} s on 1 core scaled from a build of "
                   f"{m1} particles by N log N")}
    return main


def run_reference(args, rank, world):
    if rank != 0:
        return
    pos, vel, mass, eps = make_inputs(args)
    import oracle
    # one build of the particle set, timed once and charged pro rata to
    # every sample; the samples take different random groups
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, mass, eps, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp,
                       quad=not args.mono)
    built = (tree, time.perf_counter() - t0)
    for k in range(args.warmup):
        cpu_sample(pos, mass, eps, args, 1.0, built, seed=1000 + k)
    vals = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        vals.append(cpu_sample(pos, mass, eps, args, args.cpu_seconds / max(args.steps, 1), built, seed=1 + k))
    wall = time.perf_counter() - t0
    v = statistics.median([c["value"] for c in vals])
    line = {"impl": "reference", "metric": "particle-interactions/s", "value": v,
            "unit": "interactions/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "l2": "inputs larger than L2"},
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_run(G, torch, ps, tree, dt, steps, warmup=1):
    """ms per step of `steps` graph-replayed KDK steps after `warmup`, with
    the last step's statistics."""
    stream = torch.cuda.ExternalStream(tree.ctx.stream)
    tree.calc_force_all_and_write_back(ps)
    tree.run(ps, dt, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tree.run(ps, dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, tree.stats()


def other_configs(G, torch, main_inputs, args):
    """The other workload configurations, measured in the same run (one GPU):
    Hernquist 2^24 at theta 0.3 and 0.7 on the benchmark's own particles,
    Plummer 2^20, the clumpy mixture at 2^26 and the 4096-cluster ensemble,
    each with the parameters the autotuner picks for it, timed over a few
    graph-replayed steps (interactions/s from the last step's count; no
    accuracy checks here, `--suite` has them)."""
    import ics
    out = {}

    def single(name, inputs, theta, n_leaf, n_grp, tile, dt, steps):
        ctx = G.Context(0)
        ps = G.ParticleSystem(ctx, len(inputs[0]))
        tree = G.Tree(ctx, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=True, tile_depth=tile)
        try:
            ps.set(*inputs)
            ms, st = time_run(G, torch, ps, tree, dt, steps)
            inter = st["interactions_epj"] + st["interactions_spj"]
            out[name] = {"workload": f"N={len(inputs[0])} theta={theta} quad n_leaf={n_leaf} n_grp={n_grp} "
                                     f"tile={tile} dt={dt:.6g}",
                         "value": inter / (ms / 1e3), "unit": "interactions/s", "ms_per_step": ms,
                         "steps": steps, "interactions_per_step": inter}
        finally:
            tree.close()
            ps.close()
            ctx.close()

    jobs = [("hernquist16m-theta0.3", lambda: single("hernquist16m-theta0.3", main_inputs, 0.3, 16, 256, 512,
                                                      1.0 / 512.0, 3)),
            ("hernquist16m-theta0.7", lambda: single("hernquist16m-theta0.7", main_inputs, 0.7, 16, 256, 512,
                                                      1.0 / 512.0, 5)),
            ("plummer1m", lambda: single("plummer1m", ics.make_config("plummer1m"), 0.5, 16, 128, 0,
                                         1.0 / 256.0, 10)),
            ("clumpy64m", lambda: single("clumpy64m", ics.make_config("clumpy64m"), 0.5, 16, 256, 512,
                                         1.0 / 512.0, 2))]

    def ensemble():
        cfg = ics.CONFIGS["ensemble4096"]
        pos, vel, mass, eps, off = ics.ensemble(4096, cfg["seed"])
        ctx = G.Context(0)
        ps = G.ParticleSystem(ctx, len(pos))
        tree = G.Tree(ctx, theta=cfg["theta"], n_leaf=8, n_grp=256, tile_depth=512, block=64, i_per_thread=5)
        try:
            ps.set_systems(off)
            ps.set(pos, vel, mass, eps)
            steps = 10
            ms, st = time_run(G, torch, ps, tree, cfg["dt"], steps, warmup=3)
            out["ensemble4096"] = {"workload": f"4096 Plummer clusters, N log-uniform [256, 65536] (total "
                                               f"{len(pos)}), theta 0.5 monopole, n_leaf 8, n_grp 256, "
                                               f"tile 512, block 64 x 5, dt {cfg['dt']:.6g}",
                                   "value": 4096 / (ms / 1e3), "unit": "systems*steps/s", "ms_per_step": ms,
                                   "steps": steps,
                                   "interactions_per_step": st["interactions_epj"] + st["interactions_spj"]}
        finally:
            tree.close()
            ps.close()
            ctx.close()

    jobs.append(("ensemble4096", ensemble))
    for name, job in jobs:
        try:
            job()
        except Exception as e:  # reported in the line; the headline stands on its own
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    torch.cuda.set_device(local_rank)
    pos, vel, mass, eps = make_inputs(args)
    n = len(pos)
    ctx = G.Context(local_rank)
    ctx.set_profiling(True)
    stream = torch.cuda.ExternalStream(ctx.stream)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp, quad=not args.mono)
    ps.set(pos, vel, mass, eps)
    tuned = None
    if not args.no_autotune:
        # n_grp in {64, 128, 256, 512} (and n_leaf, tile depth) by measured
        # time of the whole force calculation
        best, ms = tree.autotune(ps, n_leaf=(8, 16), n_grp=(64, 128, 256, 512),
                                 tile_depth=(256, 512), block=(64, 128, 256), i_per_thread=(2, 4, 5), repeats=1)
        tuned = {**best, "force_ms": ms}
        args.n_leaf, args.n_grp = best["n_leaf"], best["n_grp"]
    tree.calc_force_all_and_write_back(ps)
    for _ in range(args.warmup):
        tree.step(ps, args.dt)
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    per_step, inter, inter_e, inter_s, force_ms, stage = [], 0, 0, 0, [], []
    launches0 = ctx.launches
    for k in range(args.steps):
        ev[k][0].record(stream)
        tree.step(ps, args.dt)
        ev[k][1].record(stream)
        st = tree.stats()  # synchronises the stream; outside the events
        inter_e += st["interactions_epj"]
        inter_s += st["interactions_spj"]
        force_ms.append(st["ms_force"])
        stage.append(st)
    torch.cuda.synchronize()
    launches = ctx.launches - launches0
    if dist:
        torch.distributed.barrier()
    clk = clocks.stop()
    per_step = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(per_step) / 1e3
    inter = inter_e + inter_s
    t_max = t_total
    if dist:
        t_max, inter = combine_ranks(t_total, inter, world, "cuda")
    value = inter / t_max
    last = stage[-1]

    # roofline of the dominant kernel: the force kernel (FP32 ALU bound)
    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(local_rank).multi_processor_count
    f_ghz = pk.get("sm_max_mhz", 2070.0) / 1e3
    peak_ops = sm_count * 128 * f_ghz * 1e9
    ops_spj = OPS_SPJ_MONO if args.mono else OPS_SPJ_QUAD
    ops_last = last["interactions_epj"] * OPS_EPJ + last["interactions_spj"] * ops_spj
    f_s = statistics.median(force_ms) / 1e3
    achieved = ops_last / f_s
    alg_spj = ALG_SPJ_MONO if args.mono else ALG_SPJ_QUAD
    alg_last = last["interactions_epj"] * ALG_EPJ + last["interactions_spj"] * alg_spj
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_ops,
                "frac_algorithmic": alg_last / f_s / peak_ops,
                "traffic": force_traffic(workload_name(args)),
                "kernel": "k_force_f32 (quadrupole)" if not args.mono else "k_force_f32",
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {f_ghz:.3f} GHz "
                               f"(sm_max_mhz of {pk_kind} peaks), FMA = 1 op",
                "ops_per_interaction": {"epj": OPS_EPJ, "spj": ops_spj},
                "ops_per_interaction_algorithmic": {"epj": ALG_EPJ, "spj": alg_spj}}
    stages = {k: round(statistics.median([s[k] for s in stage]), 3) for k in stage[0]
              if k.startswith("ms_")}
    hbm = stage_hbm(stages, n, last["n_nodes"], pk.get("hbm_gbs", 6800.0), bool(last.get("sort_coherent")))

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hp, hv, hm, he = pin(pos), pin(vel), pin(mass), pin(eps)
        hacc = torch.zeros((n, 3), dtype=torch.float64).pin_memory().numpy()
        hpot = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        ps2 = G.ParticleSystem(ctx, n)
        ps2.set(hp, hv, hm, he)
        tree.calc_force_all_and_write_back(ps2)
        torch.cuda.synchronize()
        t_e2e, ie = [], []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            # the force calculation's inputs: positions, masses, softenings
            ps2.set(hp, None, hm, he)
            tree.calc_force_all_and_write_back(ps2)
            G.fdps_psys_get(ctx.h, ps2.h, None, None, hacc, hpot)
            s2 = tree.stats()
            t_e2e.append(time.perf_counter() - t0)
            ie.append(s2["interactions_epj"] + s2["interactions_spj"])
        ps2.close()
        # every step does the same work: the median step, with the spread
        k_med = int(np.argsort(t_e2e)[len(t_e2e) // 2])
        e2e = {"value": ie[k_med] / t_e2e[k_med], "unit": "interactions/s", "h2d_bytes_per_step": 40 * n,
               "d2h_bytes_per_step": 32 * n, "steps": args.e2e_steps,
               "ms_per_step": [round(1e3 * t, 2) for t in t_e2e],
               "what": "psys_set(pos, mass, eps) from pinned host + calcForceAllAndWriteBack + get(acc, pot) "
                       "into pinned host; median step"}

    # all-FP64 pipeline of the same library on the same particles: one step
    fp64 = None
    if not args.no_fp64:
        ps3 = G.ParticleSystem(ctx, n)
        tree64 = G.Tree(ctx, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp,
                        quad=not args.mono, fp64=True)
        ps3.set(pos, vel, mass, eps)
        tree64.calc_force_all_and_write_back(ps3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree64.step(ps3, args.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        s3 = tree64.stats()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"ms_per_step": ms64,
                "value": (s3["interactions_epj"] + s3["interactions_spj"]) / (ms64 / 1e3),
                "ms_force": s3["ms_force"], "steps": 1}
        tree64.close()
        ps3.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(pos, mass, eps, args, args.cpu_seconds)

    other = None
    if rank == 0 and world == 1 and not args.no_other:
        other = other_configs(G, torch, (pos, vel, mass, eps), args)

    if rank == 0:
        line = {"metric": "particle-interactions/s", "value": value, "unit": "interactions/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_max / args.steps,
                "ms_per_step_median": statistics.median(per_step), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": workload_name(args), "l2": "inputs larger than L2",
                           "replicas": world, "autotuned": tuned},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "fp64_variant": fp64, "stages_ms": stages, "stages_hbm": hbm,
                "sort_path": "coherent" if last.get("sort_coherent") else "radix",
                "per_step": {"interactions": inter / args.steps,
                             "interactions_epj": inter_e / args.steps,
                             "interactions_spj": inter_s / args.steps,
                             "spj_kind": "monopole" if args.mono else "quadrupole",
                             "n_nodes": last["n_nodes"], "n_groups": last["n_groups"],
                             "fp64_fallbacks": last["fp64_fallbacks"]},
                "interactions_per_s_force_kernel": (inter / args.steps) / statistics.median(
                    [f / 1e3 for f in force_ms]),
                "other_configs": other}
        print(json.dumps(line), flush=True)
    tree.close()
    ps.close()
    ctx.close()


def run_ensemble(args, rank=0, world=1, local_rank=0):
    """Systems-steps/s of the ensemble stepped by graph-captured runs, with
    per-system energy drift, beside one step of the all-FP64 pipeline.  With
    several ranks the systems are split into contiguous ranges (no exchange
    between ranks); the whole job's value is all systems' steps over the
    slowest rank's time."""
    import torch
    import ics
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    cfg = ics.CONFIGS["ensemble4096"]
    pos, vel, mass, eps, off = ics.ensemble(args.n_sys, cfg["seed"])
    n_sys_all, n_all = args.n_sys, len(pos)
    if world > 1:
        a, b = partition_systems(np.diff(off), world)[rank]
        p0, p1 = off[a], off[b]
        pos, vel, mass, eps = pos[p0:p1], vel[p0:p1], mass[p0:p1], eps[p0:p1]
        off = off[a:b + 1] - p0
    n_sys = len(off) - 1
    n = len(pos)
    dt = cfg["dt"]
    torch.cuda.set_device(local_rank)
    ctx = G.Context(local_rank)
    ctx.set_profiling(True)
    stream = torch.cuda.ExternalStream(ctx.stream)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=cfg["theta"], n_leaf=cfg["n_leaf"], n_grp=cfg["n_grp"])
    ps.set_systems(off)
    ps.set(pos, vel, mass, eps)
    tuned = None
    if not args.no_autotune:
        best, ms = tree.autotune(ps, n_leaf=(8, 16), n_grp=(32, 64, 128, 256), tile_depth=(256, 512),
                                 block=(64, 128, 256), i_per_thread=(2, 4, 5), repeats=1)
        tuned = {**best, "force_ms": ms}
    tree.calc_force_all_and_write_back(ps)
    ek0, ep0 = ps.energy_systems()
    tree.run(ps, dt, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = ctx.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tree.run(ps, dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = ctx.launches - l0
    t, systems_steps = combine_ranks(e0.elapsed_time(e1) / 1e3, n_sys * args.steps, world, "cuda")
    st = tree.stats()
    ek1, ep1 = ps.energy_systems()
    E0, E1 = ek0 + ep0, ek1 + ep1
    drift = np.abs((E1 - E0) / E0)
    fp64 = None
    if not args.no_fp64:
        ps3 = G.ParticleSystem(ctx, n)
        p64 = tuned or {"n_leaf": cfg["n_leaf"], "n_grp": cfg["n_grp"]}
        t64 = G.Tree(ctx, theta=cfg["theta"], n_leaf=p64["n_leaf"], n_grp=p64["n_grp"], fp64=True)
        ps3.set_systems(off)
        ps3.set(pos, vel, mass, eps)
        t64.calc_force_all_and_write_back(ps3)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        t64.step(ps3, dt)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1)
        fp64 = {"ms_per_step": ms64, "value": n_sys / (ms64 / 1e3), "steps": 1, "rank": rank}
        t64.close()
        ps3.close()
    inter = st["interactions_epj"] + st["interactions_spj"]
    if rank != 0:
        tree.close()
        ps.close()
        ctx.close()
        return
    line = {"metric": "systems-steps/s", "value": systems_steps / t, "unit": "systems*steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ensemble of {n_sys_all} Plummer clusters, N log-uniform "
                                   f"[256, 65536] (total {n_all}), theta {cfg['theta']} monopole, "
                                   f"dt {dt}, graph-captured steps", "l2": "inputs larger than L2",
                       "ranks": "systems split in contiguous ranges balanced by N log N"
                                if world > 1 else "one GPU",
                       "params": tuned or {"n_leaf": cfg["n_leaf"], "n_grp": cfg["n_grp"]}},
            "gpu_launches": launches, "clocks": clk,
            "interactions_per_s_estimate": inter * args.steps / t,
            "energy_drift": {"median": float(np.median(drift)), "p99": float(np.quantile(drift, 0.99)),
                             "max": float(drift.max()), "steps": args.warmup + args.steps},
            "fp64_variant": fp64, "stages_ms_last_step": {k: v for k, v in st.items() if k.startswith("ms_")}}
    print(json.dumps(line), flush=True)
    tree.close()
    ps.close()
    ctx.close()


def run_config(G, torch, name, model, n, eps, theta, quad, n_leaf, n_grp, steps, dt, n_direct,
               autotune, fp64_step, seed, tile_depth=0, extra=None):
    """One configuration: time `steps` graph-replayed KDK steps, force error of
    the first force calculation against the FP64 direct sum on n_direct random
    particles (oracle), relative energy drift over the run."""
    import ics
    import oracle
    pos, vel, mass, e = ics.make(model, n, seed, eps)
    ctx = G.Context(0)
    ctx.set_profiling(True)
    stream = torch.cuda.ExternalStream(ctx.stream)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad, tile_depth=tile_depth)
    ps.set(pos, vel, mass, e)
    tuned = None
    if autotune:
        best, ms = tree.autotune(ps, n_leaf=(8, 16), n_grp=(64, 128, 256, 512), tile_depth=(256, 512),
                                 block=(64, 128, 256), i_per_thread=(2, 4, 5), repeats=1)
        tuned = {**best, "force_ms": ms}
    tree.calc_force_all_and_write_back(ps)
    st0 = tree.stats()
    _, _, acc, pot = ps.get()
    idx = np.random.default_rng(seed).choice(n, n_direct, replace=False)
    t0 = time.perf_counter()
    ad, _ = oracle.direct(pos, mass, e, idx)
    t_direct = time.perf_counter() - t0
    err = np.linalg.norm(acc[idx] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    ek0, ep0 = ps.energy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tree.run(ps, dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    st = tree.stats()
    ek1, ep1 = ps.energy()
    inter = st0["interactions_epj"] + st0["interactions_spj"]
    line = {"config": name, "workload": f"{model} N={n} theta={theta} {'quad' if quad else 'mono'} "
                                        f"eps={eps} dt={dt:.6g}",
            "params": tuned or {"n_leaf": n_leaf, "n_grp": n_grp},
            "steps": steps, "ms_per_step": 1e3 * t / steps,
            "interactions_per_step": inter, "interactions_per_s": inter * steps / t,
            "force_ms_first_call": st0["ms_force"], "stages_ms_first_call":
                {k: round(v, 3) for k, v in st0.items() if k.startswith("ms_")},
            "force_error_vs_direct": {"n_sample": n_direct, "median": float(np.median(err)),
                                      "rms": float(np.sqrt(np.mean(err ** 2))),
                                      "p99": float(np.quantile(err, 0.99)),
                                      "oracle_direct_s": round(t_direct, 1)},
            "energy": {"E0": ek0 + ep0, "rel_drift": abs((ek1 + ep1) - (ek0 + ep0)) / abs(ek0 + ep0)},
            "n_nodes": st0["n_nodes"], "n_groups": st0["n_groups"], "fp64_fallbacks": st0["fp64_fallbacks"]}
    # the force kernel against the FP32 peak, on the algorithmic count
    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sm_count * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6
    alg = st0["interactions_epj"] * ALG_EPJ + st0["interactions_spj"] * (ALG_SPJ_QUAD if quad else ALG_SPJ_MONO)
    line["force_frac_algorithmic"] = alg / (st0["ms_force"] / 1e3) / peak_ops
    line.update(extra or {})
    tree.close()
    ps.close()
    if fp64_step:
        ps3 = G.ParticleSystem(ctx, n)
        p = line["params"]
        t64 = G.Tree(ctx, theta=theta, n_leaf=p["n_leaf"], n_grp=p["n_grp"], quad=quad, fp64=True)
        ps3.set(pos, vel, mass, e)
        t64.calc_force_all_and_write_back(ps3)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        t64.step(ps3, dt)
        a1.record(stream)
        torch.cuda.synchronize()
        line["fp64_ms_per_step"] = a0.elapsed_time(a1)
        t64.close()
        ps3.close()
    ctx.close()
    print(json.dumps(line), flush=True)


# A user's gravity law, given to the library as source text (the Force and
# Law structs of include/fdps_user_force.cuh): softened monopole terms for
# particles, monopole + traceless quadrupole for superparticles.
USER_GRAVITY_LAW = r"""
struct Force {
    float ax, ay, az, pot;
    __device__ void clear() { ax = ay = az = pot = 0.f; }
};
struct Law {
    __device__ void operator()(const Epi& i, const Epj* j, int nj, Force& f) const {
        for (int k = 0; k < nj; ++k) {
            const float dx = j[k].x - i.x, dy = j[k].y - i.y, dz = j[k].z - i.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, i.eps2)));
            const float ri = rsqrtf(r2);
            const float mri = j[k].m * ri, mri3 = mri * ri * ri;
            f.ax = fmaf(mri3, dx, f.ax);
            f.ay = fmaf(mri3, dy, f.ay);
            f.az = fmaf(mri3, dz, f.az);
            f.pot -= mri;
        }
    }
    __device__ void operator()(const Epi& i, const Spj* j, int nj, Force& f) const {
        for (int k = 0; k < nj; ++k) {
            const Spj& s = j[k];
            const float rx = i.x - s.x, ry = i.y - s.y, rz = i.z - s.z;
            const float R2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, i.eps2)));
            const float Ri = rsqrtf(R2), Ri2 = Ri * Ri, Ri3 = Ri * Ri2, Ri5 = Ri3 * Ri2;
            const float qx = fmaf(s.qxx, rx, fmaf(s.qxy, ry, s.qxz * rz));
            const float qy = fmaf(s.qxy, rx, fmaf(s.qyy, ry, s.qyz * rz));
            const float qz = fmaf(s.qxz, rx, fmaf(s.qyz, ry, s.qzz * rz));
            const float rqr = fmaf(rx, qx, fmaf(ry, qy, rz * qz));
            const float c = fmaf(2.5f * rqr * Ri5, Ri2, s.m * Ri3);
            f.ax += fmaf(qx, Ri5, -c * rx);
            f.ay += fmaf(qy, Ri5, -c * ry);
            f.az += fmaf(qz, Ri5, -c * rz);
            f.pot -= fmaf(0.5f * rqr, Ri5, s.m * Ri);
        }
    }
};
"""


def run_user_law(args):
    """A user interaction law compiled at run time (NVRTC) through the C ABI,
    run over the library's own interaction lists of the benchmark workload,
    timed beside the built-in force kernel on the same lists: ms per launch
    and interactions/s, and the FP32 roofline fraction on the measurement
    plan's algorithmic count."""
    import torch
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    pos, vel, mass, eps = make_inputs(args)
    n = len(pos)
    ctx = G.Context(0)
    ctx.set_profiling(True)
    stream = torch.cuda.ExternalStream(ctx.stream)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp, quad=not args.mono)
    law = G.UserLaw(ctx, USER_GRAVITY_LAW)
    try:
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)  # the built-in kernel on these lists
        st = tree.stats()
        tree.calc_force_all_and_write_back(ps)
        st = tree.stats()
        builtin_ms = st["ms_force"]
        out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            law.run(tree, ps, out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            law.run(tree, ps, out)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        _, _, acc, _ = ps.get()
        a_user = out[:, :3].double().cpu().numpy()
        rel = np.linalg.norm(a_user - acc, axis=1) / np.linalg.norm(acc, axis=1)
        inter = st["interactions_epj"] + st["interactions_spj"]
        pk, pk_kind = peaks()
        sm_count = torch.cuda.get_device_properties(0).multi_processor_count
        peak_ops = sm_count * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6
        alg = st["interactions_epj"] * ALG_EPJ + st["interactions_spj"] * (ALG_SPJ_MONO if args.mono else ALG_SPJ_QUAD)
        line = {"metric": "user-law interactions/s", "value": inter / (ms / 1e3), "unit": "interactions/s",
                "workload": workload_name(args), "law": "softened gravity, monopole + quadrupole "
                                                        "superparticles, one i-particle per thread (header template)",
                "ms_per_launch": ms, "launches": args.steps, "interactions": inter,
                "builtin_force_ms": builtin_ms, "user_over_builtin": ms / builtin_ms,
                "roofline": {"bound": "alu", "frac_algorithmic": alg / (ms / 1e3) / peak_ops,
                             "builtin_frac_algorithmic": alg / (builtin_ms / 1e3) / peak_ops},
                "acc_rel_vs_builtin": {"median": float(np.median(rel)), "max": float(rel.max())}}
        print(json.dumps(line), flush=True)
    finally:
        law.close()
        tree.close()
        ps.close()
        ctx.close()


def run_sph(args):
    """Short-range mode on n particles of a uniform random unit cube with
    radii h_i = 4.2 n^(-1/3) (about 310 neighbours, the paper's SPH cutoff):
    neighbour pairs per second over the whole call (tree + neighbour walk +
    pair pass), the FP32 roofline of the pair pass, and the density's mean
    against the exact mean density."""
    import torch
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    n = args.n
    rng = np.random.default_rng(1601031385)
    pos = rng.random((n, 3))
    mass = np.full(n, 1.0 / n)
    hval = 4.2 * n ** (-1.0 / 3.0)
    ctx = G.Context(0)
    ctx.set_profiling(True)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=args.n_leaf, n_grp=args.n_grp)
    ps.set(pos, np.zeros_like(pos), mass, np.full(n, 1e-3))
    h = torch.full((n,), hval, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        cnt, rho, info = tree.neighbors(ps, G.FDPS_CUTOFF_I, h)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cnt, rho, info = tree.neighbors(ps, G.FDPS_CUTOFF_I, h)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    st = tree.stats()  # stage times of the last call: ms_walk, ms_force = the pair pass
    # the pair pass against the FP32 peak: per candidate pair r^2 and the
    # comparison on plain FP32 coordinates (3 subtractions, 3 multiply-adds,
    # 1 compare), per neighbour the Wendland C6 term and its sum (q = r/H,
    # 1 - q, three squarings, three multiply-adds of the polynomial, the
    # product with the normalisation and the mass-weighted sum: 10), plus a
    # square root on the special-function unit
    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = sm_count * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6
    alg = OPS_SR_CAND * float(info[1]) + OPS_SR_NB * float(info[0])
    t_pair = st["ms_force"] / 1e3
    roofline = {"bound": "alu", "kernel": "k_short_pairs", "achieved": alg / t_pair / 1e12,
                "peak": peak_ops / 1e12, "unit": "TFLOP/s", "frac": alg / t_pair / peak_ops,
                "ops_per_candidate": OPS_SR_CAND, "ops_per_neighbour": OPS_SR_NB,
                "peak_source": f"{sm_count} SMs x 128 FP32 lanes x sm_max_mhz of {pk_kind} peaks"}
    inner = np.all((pos > hval) & (pos < 1.0 - hval), axis=1)
    line = {"metric": "SPH density neighbour pairs/s", "value": float(info[0]) / t, "unit": "pairs/s",
            "workload": f"uniform cube N={n}, h = 4.2 N^-1/3, i-dependent cutoff, Wendland C6, "
                        f"n_leaf={args.n_leaf} n_grp={args.n_grp}",
            "ms_per_call": 1e3 * t, "steps": args.steps,
            "neighbours_mean": float(info[0]) / n, "candidates_per_neighbour": float(info[1]) / float(info[0]),
            "fp64_decisions": int(info[2]),
            "density_interior_mean": float(rho[inner].mean()), "density_interior_std": float(rho[inner].std()),
            "counts_min_max": [int(cnt.min()), int(cnt.max())],
            "stages_ms_last_call": {"tree_and_groups": round(st["ms_total"] - st["ms_walk"] - st["ms_force"], 3),
                                    "walk": round(st["ms_walk"], 3), "pairs": round(st["ms_force"], 3)},
            "roofline": roofline}
    print(json.dumps(line), flush=True)
    tree.close()
    ps.close()
    ctx.close()


def run_theta_target(args):
    """The opening angle chosen for a median acceleration-error target on the
    benchmark workload: time of the direct-sum reference and of the choice,
    and the forces' error at the choice (against the GPU direct sum)."""
    import torch
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    pos, vel, mass, eps = make_inputs(args)
    n = len(pos)
    ctx = G.Context(0)
    ctx.set_profiling(True)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=args.theta, n_leaf=args.n_leaf, n_grp=args.n_grp, quad=not args.mono)
    ps.set(pos, vel, mass, eps)
    rows = (np.arange(min(args.n_sample, n), dtype=np.int64) * n) // min(args.n_sample, n)
    t0 = time.perf_counter()
    ad, _ = ps.direct(rows)
    t_direct = time.perf_counter() - t0
    t0 = time.perf_counter()
    theta, med = tree.choose_theta(ps, args.theta_target, args.n_sample)
    t_choose = time.perf_counter() - t0
    _, _, acc, _ = ps.get()
    err = np.linalg.norm(acc[rows] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    st = tree.stats()
    line = {"metric": "opening angle for a median force-error target",
            "workload": workload_name(args), "target_median": args.theta_target,
            "theta": theta, "median": med, "rms": float(np.sqrt(np.mean(err ** 2))),
            "p99": float(np.quantile(err, 0.99)), "n_sample": int(len(rows)),
            "direct_sample_s": t_direct, "direct_interactions_per_s": len(rows) * (n - 1) / t_direct,
            "choose_theta_s": t_choose, "force_ms_at_choice": st["ms_force"],
            "interactions_at_choice": st["interactions_epj"] + st["interactions_spj"]}
    print(json.dumps(line), flush=True)
    tree.close()
    ps.close()
    ctx.close()


def host_memory_available():
    """Bytes of host memory this process may still use: MemAvailable, and
    below the cgroup's limit where one is set."""
    with open("/proc/meminfo") as f:
        avail = next(int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable"))
    for lim, cur in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                     ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                      "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(lim) as f:
                v = f.read().strip()
            with open(cur) as f:
                u = int(f.read().strip())
        except (OSError, ValueError):
            continue
        if v.isdigit():
            avail = min(avail, int(v) - u)
    return avail


def run_largest(args):
    """The clumpy mixture (1000 Plummer clumps, 20 % background, eps 0.002,
    theta 0.5 quadrupole) at the largest particle count that fits the
    device: the library's device bytes per particle are measured on a 2^25
    clumpy set (every buffer at its grown size after one force calculation),
    raised by 10 % for the longer lists of a larger set, and N is the
    multiple of 2^20 that fills 80 % of the free device memory with that
    (capped so that the run's host arrays, about 150 bytes a particle at
    their peak, stay well within the available host memory).  n_leaf 16, n_grp 256, tile depth 512 (the
    autotuner's pick at 2^26); two graph-replayed steps."""
    import torch
    import ics
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    S = ics.SEED_BASE
    n0 = 1 << 25
    pos, vel, mass, e = ics.make("clumpy", n0, S + 4, 0.002)
    torch.cuda.init()
    free0, total = torch.cuda.mem_get_info(0)
    ctx = G.Context(0)
    ps = G.ParticleSystem(ctx, n0)
    tree = G.Tree(ctx, theta=0.5, n_leaf=16, n_grp=256, quad=True, tile_depth=512)
    ps.set(pos, vel, mass, e)
    tree.calc_force_all_and_write_back(ps)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    tree.close()
    ps.close()
    ctx.close()
    del pos, vel, mass, e
    bpp = (free0 - free1) / n0
    n_dev = int(0.8 * free0 / (1.1 * bpp))
    avail = host_memory_available()
    n_host = int(0.6 * avail / 300)  # the run's host arrays peak near 150 bytes a particle
    n = min(n_dev, n_host, 0x7FFFFFFF) >> 20 << 20
    extra = {"largest": {"device_bytes_per_particle_at_2^25": round(bpp, 1),
                         "device_free_gb": round(free0 / 1e9, 1), "device_total_gb": round(total / 1e9, 1),
                         "n_device_limit": n_dev, "n_host_limit": n_host,
                         "host_available_gb": round(avail / 1e9, 1)}}
    run_config(G, torch, "clumpy-largest", "clumpy", n, 0.002, 0.5, True, 16, 256, 2, 1.0 / 512.0,
               256, False, False, S + 4, tile_depth=512, extra=extra)


def run_suite(args):
    import torch
    import ics
    import paper_1601_03138_gb300 as G
    from paper_1601_03138_gb300 import build as B
    B.build()
    S = ics.SEED_BASE
    run_config(G, torch, "plummer1m", "plummer", 1 << 20, 1.0 / 64.0, 0.5, True, 16, 128, 10,
               1.0 / 256.0, 4096, False, True, S + 2)
    for th in (0.3, 0.5, 0.7):
        run_config(G, torch, f"hernquist16m-theta{th}", "hernquist", 1 << 24, 0.005, th, True, 16, 128,
                   20, 1.0 / 512.0, 1024, True, th == 0.5, S + 3)
    run_config(G, torch, "clumpy64m", "clumpy", 1 << 26, 0.002, 0.5, True, 16, 128, 2, 1.0 / 512.0,
               256, True, False, S + 4)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.ensemble:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        run_ensemble(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    if args.suite:
        if rank == 0:
            run_suite(args)
        return
    if args.sph:
        if rank == 0:
            run_sph(args)
        return
    if args.largest:
        if rank == 0:
            run_largest(args)
        return
    if args.user_law:
        if rank == 0:
            run_user_law(args)
        return
    if args.theta_target is not None:
        if rank == 0:
            run_theta_target(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
