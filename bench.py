#!/usr/bin/env python
"""Throughput benchmark of the well-balanced WCSPH hot path on GB300.

One step = one SSP-RK2 step of the whole path (two stages, each: cell keys,
radix sort, reorder, cell bounds, dummy/volume prepass, fused pair pass,
update) over the synthetic scene named by --workload, inputs resident in HBM.
Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload dam3d|slosh3d] [--precision fp64|mixed|df64]

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the host cores, on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (weak scaling): the method's single
domain is not partitioned across GPUs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (3D, 1.2M and 17.5M particles): FP64 vs mixed vs surrogate at stated error"
UNIT = "particle-steps/s"

# FP64 flops of one neighbour pair in the fused pair pass with all terms on
# (an FMA counts 2): distance 8, reciprocal square root (two Newton steps)
# 12, kernel scalars 7, velocity difference and normal component 10,
# interface potential 4, L 12, S 6, C 6, M 18 (3D), D 2, Lambda 6, shifting 16.
FLOPS_PER_PAIR_3D = 110
FLOPS_PER_PAIR_2D = 74
# per fluid particle: eigenvalue, 3x3 inverse, contractions and rates
FLOPS_EPILOGUE_3D = 260
# FP32 flops of one pair in the mixed pass: 78 for the pair terms and
# 77.5 for the Kahan-compensated updates of 31 accumulators (two
# consecutive terms share one 4-operation step after a 1-operation park:
# 2.5 each); 2D: 46 and 18 accumulators
FLOPS_PER_PAIR_MIXED_3D = 155.5
FLOPS_PER_PAIR_MIXED_2D = 91
# measured FMA throughput of this GB300 (independent FMA chains, 152 SMs at
# 1987 MHz): FP64 5.93e11 DFMA/s = 1.186 TFLOP/s; FP32 3.62e13 FFMA/s = 72.4
FP64_PEAK_TFLOPS = 1.186
FP32_PEAK_TFLOPS = 72.4
# FP32 instructions of one pair in the double-float pass, all terms on (each
# FADD, FMUL or FFMA is one operation on the FP32 pipe; two-sum 6, fast
# two-sum 3, double-float product 8, raw product 4, accumulate 11): offsets 9,
# |r|^2 31, 1/|r| 17, q/2 16 (|r|/R times R/2h), 1 - q/2 7, kernel factor
# 12, velocity differences 24, g r 12, normal velocity 39, potential terms 23,
# L 90, S 45, M 135, K 33, C 53, D 15, Lambda 45, shifting 76 (3D)
OPS_PER_PAIR_DF_3D = 682
OPS_PER_PAIR_DF_2D = 452
# FP32 instruction rate of the FP32 pipe (one FFMA counts once)
FP32_PEAK_TOPS = FP32_PEAK_TFLOPS / 2
PRECISIONS = ("fp64", "mixed", "df64")
DTYPES = {"fp64": "f64", "mixed": "f32 (Kahan-compensated sums) + f64 epilogue",
          "df64": "f32x2 (double-float sums) + f64 epilogue"}

WORKLOADS = {
    "dam3d": dict(
        make=lambda: _scenes().dam_break_3d(dx=0.0084),
        sample=lambda: _scenes().dam_break_3d(dx=0.0168),
        desc=("3D dam break: box 3.2x1.0x1.0 m, water column 1.2x1.0x0.6 m, dx=0.0084 m "
              "(1,208,207 fluid + 498,949 dummy particles in 3 layers), Wendland C2 h=1.3dx, "
              "c0=10 sqrt(gH), linear EOS, delta-SPH, shifting and TIC on, adaptive dt (CFL 0.2)"),
        sample_desc="same scene at dx=0.0168 m (1/8 replica: 153,360 fluid + 127,188 dummy)"),
    "dam3d_s": dict(
        make=lambda: _scenes().dam_break_3d(dx=0.0126),
        sample=lambda: _scenes().dam_break_3d(dx=0.0252),
        desc=("3D dam break as dam3d at dx=0.0126 m (360,240 fluid + 221,996 dummy particles): the profiling "
              "case, larger than L2"),
        sample_desc="same scene at dx=0.0252 m"),
    "slosh3d": dict(
        make=lambda: _scenes().sloshing_3d(),
        sample=lambda: _scenes().sloshing_3d(dx=0.0307),
        desc=("3D sloshing tank 4.0x2.0x2.0 m, depth 1.0 m, dx=0.00769 m (17,576,000 fluid "
              "particles + dummies), harmonic forcing A=0.01 m, T=1.5 s, delta-SPH, shifting, TIC on"),
        sample_desc="same tank at dx=0.0307 m (1/64 replica)"),
}


def _scenes():
    from paper_2608_22269_gb300 import scenes
    return scenes


def algorithmic_bytes_per_particle_step(dim: int) -> int:
    """HBM bytes the method must move per fluid particle-step (two stages):
    per stage the build reads positions and writes keys (8d+4), sorts (3
    passes x 16 B), reorders the state (2 x (16d+18+8d)), the pair pass reads
    x, U, phi, V of the particle (8(2d+2)) and writes rates (8(2d+2)), the
    update reads/writes state (2 x 8(2d+1))."""
    d = dim
    per_stage = (8 * d + 4) + 48 + 2 * (24 * d + 18) + 16 * (2 * d + 2) + 16 * (2 * d + 1)
    return 2 * per_stage


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [v.strip() for v in line.split(",")]
                if len(f) >= 8 and f[0].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][1]),
                "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int, device: str = "cuda") -> float:
    """Largest value over ranks (the slowest replica sets the job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of independent replicas: units of all ranks over
    the slowest rank's time."""
    return units_per_rank * world / seconds_max


def profile_traffic(kernel_file: str, key: str):
    """DRAM traffic per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(key)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2608_22269_gb300", "csrc", kernel_file)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if ent.get("source_sha") != sha:
        return None
    return ent.get("bytes_per_launch")


def cpu_baseline(sample_scene, budget_s=12.0, max_steps=500):
    import oracle
    st = oracle.State(sample_scene)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (steps < 2 or time.perf_counter() - t0 < budget_s):
        st.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return sample_scene.n_fluid * steps / dt, steps, dt, oracle.num_threads()


# ---------------------------------------------------------------------------
def time_path(scene, precision, args, world, local):
    """Warm up, then time args.steps steps device-side; returns the sim and
    a dict of measurements (CUDA events on the library's stream)."""
    import torch

    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(scene.params, precision=precision, water_height=scene.water_height,
                    device=local)
    sim.set_scene(scene)
    sim.step(args.warmup)
    sim.sync()
    st0 = sim.stats()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(sim.stream)
        sim.step(args.steps)       # replayed as a CUDA graph after the first step
        e1.record(sim.stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    sim.sync()
    st1 = sim.stats()
    # kernel-class timing: the same number of steps again with CUDA events
    # bracketing every kernel class (eager launches)
    sim.set_profiling(True)
    sim.profile(reset=True)
    sp0 = sim.stats()
    sim.step(args.steps)
    sim.sync()
    sp1 = sim.stats()
    prof = sim.profile(reset=True)
    sim.set_profiling(False)
    return sim, {"ms": max_over_ranks(ms, world), "st0": st0, "st1": st1, "prof": prof,
                 "sp0": sp0, "sp1": sp1, "clocks": clk.summary()}


def pair_roofline(m, dim, nf, precision, workload):
    pair_ms, pair_n = m["prof"]["pair"]
    pairs = m["sp1"]["pairs"] - m["sp0"]["pairs"]
    per_launch = pairs / max(pair_n, 1)
    avg_ms = pair_ms / max(pair_n, 1)
    unit, pipe = "TFLOP/s", "FP64"
    if precision == "mixed":
        fpp = FLOPS_PER_PAIR_MIXED_3D if dim == 3 else FLOPS_PER_PAIR_MIXED_2D
        flops = per_launch * fpp + nf * 600
        peak, kernel, src, pipe = FP32_PEAK_TFLOPS, "k_pair_mixed<%d>" % dim, "pair_mixed.cu", "FP32"
    elif precision == "df64":
        # FP32 operations of the pair terms only (the FP64 epilogue runs on the other pipe)
        fpp = OPS_PER_PAIR_DF_3D if dim == 3 else OPS_PER_PAIR_DF_2D
        flops = per_launch * fpp
        peak, kernel, src, pipe = FP32_PEAK_TOPS, "k_pair_df<%d>" % dim, "pair_df64.cu", "FP32"
        unit = "Top/s (FP32 instructions)"
    else:
        fpp = FLOPS_PER_PAIR_3D if dim == 3 else FLOPS_PER_PAIR_2D
        flops = per_launch * fpp + nf * FLOPS_EPILOGUE_3D
        peak, kernel, src = FP64_PEAK_TFLOPS, "k_pair_fp64<%d>" % dim, "pair_fp64.cu"
    achieved = flops / (avg_ms / 1e3) / 1e12
    key = "pair_%s_%s" % (precision, workload)
    total = sum(v[0] for v in m["prof"].values())
    return {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 4), "peak": peak,
            "unit": unit, "frac": round(achieved / peak, 4),
            "traffic": profile_traffic(src, key),
            "peak_source": "measured %s FMA throughput of this GB300 (profiles/fp64_alu_peak.md)" % pipe,
            "pairs_per_launch": int(per_launch), "flops_per_pair": fpp,
            "avg_launch_ms": round(avg_ms, 4), "share_of_step": round(pair_ms / max(total, 1e-9), 4)}


def natural_scales(params, water_height):
    """Natural scales of the relative error measure: accelerations by |G|,
    potential rates by C0^2 sqrt(|G| H) / h."""
    g = math.sqrt(sum(v * v for v in params["g"][: params["dim"]])) or 1.0
    H = water_height if water_height > 0 else 1.0
    h = params["h_over_dx"] * params["dx"]
    return {"dudt": g, "dphidt": params["c0"] ** 2 * math.sqrt(g * H) / h}


def scaled_err(a, b, scale):
    """max |a - b| / max(max |b|, scale)."""
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    return float(np.abs(a - b).max()) / max(float(np.abs(b).max()), scale)


def rates_diff(a, b, scene):
    """Scaled difference of the stage rates of two sims on the same state
    (particles within 1e-4 of the TIC threshold are left out: there the two
    arithmetics may legitimately take different branches)."""
    import numpy as np
    f = scene.type == 0
    sk = natural_scales(scene.params, scene.water_height)
    lam = b.get("lambda")[f]
    keep = np.abs(lam - scene.params["tic_lambda"]) > 1e-4
    return {"dudt": scaled_err(a.get("dudt")[:, f][:, keep], b.get("dudt")[:, f][:, keep], sk["dudt"]),
            "dphidt": scaled_err(a.get("dphidt")[f][keep], b.get("dphidt")[f][keep], sk["dphidt"]),
            "excluded_tic_boundary": int((~keep).sum())}


def surrogate_flops_per_stage(dim, n, nf, E, hidden=64, layers=3, send=32):
    """Dense-contraction FLOPs of one surrogate stage (2 per multiply-add), as
    the kernels run them: the node encoder (inputs padded to 16), per layer
    the per-edge first layer of the message MLP on the edge inputs (K = 16)
    and the sender's first 32 features (K = 32), and per node the receiver
    term (64 x 64), the message MLP's second layer on the sums (64 x 64) and
    the node MLP (128 -> 64 -> 64), and the decoder on fluid rows (64 -> 64
    -> 16 padded)."""
    H = hidden
    enc = 2 * n * (16 * H + H * H)
    per_layer = 2 * (E * (16 + send) * H + nf * (H * H + H * H) + n * (2 * H * H + H * H))
    dec = 2 * nf * (H * H + H * 16)
    return enc + layers * per_layer + dec


def surrogate_bytes_per_stage(n, nf, E, hidden=64, layers=3):
    """Algorithmic HBM bytes of one surrogate stage: the neighbour lists
    (written once, 4 B per entry, read by every layer), the node inputs and
    packs (state in, 16 + 32 B out per node), per layer the node states (h
    in, h' out: 2 x 128 B per node; the per-edge gathers of sender rows and
    packs are reuse served by L2, not additional algorithmic bytes) and the
    decoder (h in, outputs out, fluid rows)."""
    row = 2 * hidden
    lists = E * 4 * (1 + layers)
    inputs = n * (8 * 8 + 16 + 32)
    per_layer = n * 2 * row
    dec = nf * (row + 16)
    return lists + inputs + layers * per_layer + dec


def surrogate_path(args, local, dim=2, scene=None):
    """Surrogate rollouts with a plain FP64 re-anchoring step every 10 steps
    (the first step of the rollout is one), timed against the plain FP64
    rollout of the same scene; error = position RMS / dx against that plain
    rollout. 2D: the configs' inference case (dam break, column 0.6 x 0.3 m,
    dx = 0.00085 m, 249,218 fluid particles). 3D: the 3D dam break of the
    headline (1,208,207 fluid particles) with the network trained on its
    half-size replicas, or (scene = "slosh3d") the 17.58M-fluid sloshing tank
    with the same network. The timed rollout keeps the surrogate between
    anchors (tau = inf); the fallback rule (tau = 0.1: a window whose anchor
    error exceeds tau runs plain) is reported from a second, untimed
    rollout."""
    import numpy as np
    import torch

    from paper_2608_22269_gb300 import scenes, wbsph
    from paper_2608_22269_gb300 import surrogate as SG
    name = "surrogate_2d.npz" if dim == 2 else "surrogate_3d.npz"
    path = os.path.join(ROOT, "paper_2608_22269_gb300", "data", name)
    if not os.path.exists(path):
        return {"unavailable": f"no trained {dim}D surrogate weights in paper_2608_22269_gb300/data"}
    sur, norm = SG.load(path, dim)
    if dim == 2:
        sc = scenes.dam_break_2d(dx=0.00085, width=2.0, wall=0.6, column=(0.6, 0.3))
        desc = ("2D dam break, column 0.6x0.3 m in a 2.0 m basin, dx=0.00085 m "
                f"({sc.n_fluid:,} fluid), FP64 anchor every 10 steps, no fallback (tau = inf)")
    elif scene == "slosh3d":
        sc = scenes.sloshing_3d()
        desc = ("3D sloshing tank 4.0x2.0x2.0 m, depth 1.0 m, dx=0.00769 m "
                f"({sc.n_fluid:,} fluid), 3D network, FP64 anchor every 10 steps, no fallback (tau = inf)")
    else:
        sc = scenes.dam_break_3d(dx=0.0084)
        desc = ("3D dam break, box 3.2x1.0x1.0 m, column 1.2x1.0x0.6 m, dx=0.0084 m "
                f"({sc.n_fluid:,} fluid), FP64 anchor every 10 steps, no fallback (tau = inf)")
    K = max(args.steps, 10) if scene != "slosh3d" else 10
    warm = args.warmup if scene != "slosh3d" else 3
    inf = float("inf")

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    plain = wbsph.Sim(sc.params, water_height=sc.water_height, device=local)
    plain.set_scene(sc)
    plain.step(warm)
    plain.sync()
    t_plain = timed(lambda: (plain.step(K), plain.sync()))
    sim = wbsph.Sim(sc.params, water_height=sc.water_height, device=local)
    sim.set_scene(sc)
    sur.step(sim, warm, anchor_every=10, tau=inf)
    stats = {}
    t_sur = timed(lambda: stats.update(sur.step(sim, K, anchor_every=10, tau=inf)))
    f = sc.type == 0
    err = float(np.sqrt(((plain.get("x")[:, f] - sim.get("x")[:, f]) ** 2).sum(0).mean()) / sc.params["dx"])
    plain.close()
    # one surrogate stage alone (CUDA events in the library) and one plain
    # stage of the same state, each without the neighbour sort (the same
    # kernels for both): wall update and prepass, time step, lists, and the
    # network or the pair pass. Edges = the pairs of that plain stage (the
    # surrogate's graph is the same exact neighbour lists)
    st = sim.stats()
    n, nf = st["n"], st["n_fluid"]
    sur.predict(sim)
    sim.set_profiling(True)
    sim.profile(reset=True)
    sur.predict(sim)
    stage_ms = stage_time(sim.profile(reset=True))
    p0 = sim.stats()["pairs"]
    sim.eval_rates()
    plain_stage_ms = stage_time(sim.profile(reset=True))
    sim.set_profiling(False)
    E = int(sim.stats()["pairs"] - p0)
    flops = surrogate_flops_per_stage(dim, n, nf, E)
    peak = 1925.2
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
    except (OSError, ValueError, KeyError):
        pass
    achieved = flops / (stage_ms / 1e3) / 1e12
    sbytes = surrogate_bytes_per_stage(n, nf, E)
    hbm_peak = 6686.1
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        pass
    gbs = sbytes / (stage_ms / 1e3) / 1e9
    sim.close()
    fb_sim = wbsph.Sim(sc.params, water_height=sc.water_height, device=local)
    fb_sim.set_scene(sc)
    fb = sur.step(fb_sim, K, anchor_every=10, tau=0.1)
    fb_sim.close()
    out = {"workload": desc,
           "value": round(sc.n_fluid * K / t_sur, 1), "unit": UNIT,
           "plain_fp64_same_scene": round(sc.n_fluid * K / t_plain, 1),
           "ms_per_step": round(t_sur * 1e3 / K, 3), "steps": K,
           "anchors": stats, "error": {"pos_rms_over_dx_vs_plain": err,
                                        "max_anchor_rel_l2_dudt": stats.get("max_rel_err")},
           "stage": {"ms": round(stage_ms, 3), "plain_fp64_stage_ms": round(plain_stage_ms, 3), "edges": E,
                     "nodes": n, "network_gflop": round(flops / 1e9, 2)},
           "roofline": {"bound": "tensor", "kernel": "surrogate stage (lists, inputs and all network kernels)",
                        "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "peak_source": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"},
           "hbm": {"algorithmic_bytes_per_stage": int(sbytes), "achieved_gbs": round(gbs, 1),
                   "peak_gbs": hbm_peak, "frac": round(gbs / hbm_peak, 4),
                   "bytes_per_fluid_particle": round(sbytes / max(nf, 1), 1),
                   "note": "nothing per edge reaches memory; the per-edge gathers of sender rows (64 B) and "
                           "packs (32 B) are served by L2, and the layer is bound by the latency of its "
                           "gather, MMA and epilogue chains"},
           "with_fallback_tau_0.1": fb,
           "weights": f"paper_2608_22269_gb300/data/{name} (trained on the GPU by this library)"}
    sur.close()
    return out


def stage_time(prof):
    """Milliseconds of a stage without its neighbour sort: the prepass
    (wall update, volumes or U_max), the time step, the lists and the pair
    pass or the network (library profile classes)."""
    return sum(prof[k][0] for k in ("prepass", "other", "nlist", "pair"))


def surrogate_stage_profile(dx):
    """One surrogate stage (lists, node inputs, encoder, three message
    layers, decoder) of the committed 3D network on the 3D dam break at
    spacing dx, after one plain step and one warm stage; the second stage
    runs inside the NVTX range 'surrogate_stage' so that a profiler can take
    exactly its kernels. Returns its time from the library's CUDA events."""
    import torch

    from paper_2608_22269_gb300 import scenes, wbsph
    from paper_2608_22269_gb300 import surrogate as SG
    torch.cuda.set_device(0)
    sc = scenes.dam_break_3d(dx=dx)
    sim = wbsph.Sim(sc.params, water_height=sc.water_height)
    sim.set_scene(sc)
    sim.step(1)
    sur, _ = SG.load(os.path.join(ROOT, "paper_2608_22269_gb300", "data", "surrogate_3d.npz"), 3)
    sur.predict(sim)
    sim.sync()
    sim.set_profiling(True)
    sim.profile(reset=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("surrogate_stage")
    sur.predict(sim)
    sim.sync()
    torch.cuda.nvtx.range_pop()
    ms = stage_time(sim.profile(reset=True))
    sim.eval_rates()
    sim.sync()
    sim.profile(reset=True)
    sim.eval_rates()
    sim.sync()
    plain = stage_time(sim.profile(reset=True))
    out = {"surrogate_stage_ms": round(ms, 3), "plain_fp64_stage_ms": round(plain, 3), "dx": dx,
           "n_fluid": sc.n_fluid}
    sur.close()
    sim.close()
    return out


def precision_paths(scene, args, world, local, workload, primary=None, primary_sim=None,
                    primary_m=None, steps=None, warmup=None):
    """Every precision on one scene: value, roofline of the pair pass, HBM
    fraction, resident footprint, and the rate errors of the mixed and
    double-float paths against the FP64 path on one common state (the state
    the FP64 run reached). Returns (paths, sims); the sims stay open."""
    from paper_2608_22269_gb300 import wbsph
    prec_code = {"fp64": wbsph.FP64, "mixed": wbsph.MIXED, "df64": wbsph.DF64}
    a = argparse.Namespace(**vars(args))
    if steps is not None:
        a.steps = steps
    if warmup is not None:
        a.warmup = warmup
    dim, nf = scene.params["dim"], scene.n_fluid
    bytes_ps = algorithmic_bytes_per_particle_step(dim)
    hbm = measured_peaks().get("hbm_gbs", 6686.1)
    sims, paths = {}, {}
    for prec in PRECISIONS:
        if prec == primary:
            sims[prec], m = primary_sim, primary_m
        else:
            sims[prec], m = time_path(scene, prec_code[prec], a, world, local)
        v = nf * a.steps * world / (m["ms"] / 1e3)
        paths[prec] = {"value": round(v, 1), "ms_per_step": round(m["ms"] / a.steps, 4),
                       "steps": a.steps, "dtype": DTYPES[prec],
                       "roofline": pair_roofline(m, dim, nf, prec, workload),
                       "hbm_frac": round(v / world * bytes_ps / (hbm * 1e9), 5),
                       "resident_gb": round(m["st1"]["device_bytes"] / 1e9, 2)}
    fp64 = sims["fp64"]
    st = {k: fp64.get(k) for k in ("x", "u", "phi", "mass")}
    # reload the FP64 sim too, so that every path evaluates at the same time t = 0
    # (the forced tank's body force depends on t)
    fp64.set_particles(st["x"], st["u"], st["phi"], scene.type, scene.normal, st["mass"])
    fp64.eval_rates()
    for other in ("mixed", "df64"):
        o = sims[other]
        o.set_particles(st["x"], st["u"], st["phi"], scene.type, scene.normal, st["mass"])
        o.eval_rates()
        paths[other]["error_vs_fp64"] = rates_diff(o, fp64, scene)
    return paths, sims


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def summary_of(line) -> dict:
    """Compact per-path digest (value, ms per step, pair-pass roofline
    fraction, HBM fraction, error) placed last on the JSON line."""
    def digest(p, err=None):
        if not isinstance(p, dict) or "value" not in p:
            return {"error": str(p.get("error", p.get("unavailable", "not run")))[:160]} \
                if isinstance(p, dict) else None
        d = {"value": p["value"], "ms_per_step": p.get("ms_per_step")}
        rf = p.get("roofline") or {}
        if "frac" in rf:
            d["roofline_frac"] = rf["frac"]
            d["roofline_bound"] = rf.get("bound")
        hb = p.get("hbm_frac", (p.get("hbm") or {}).get("frac"))
        if hb is not None:
            d["hbm_frac"] = hb
        if err is not None:
            d["error"] = err
        return d

    out = {}
    head = {"value": line["value"], "ms_per_step": line["ms_per_step"],
            "roofline_frac": line["roofline"]["frac"], "hbm_frac": line["hbm"]["frac"],
            "error": "fp64 vs oracle <= 1e-12 (tests/test_gpu_fullsize.py)"}
    out[line["config"]["precision"] + "@" + line["config"]["workload_key"]] = head
    paths = line.get("paths", {})
    for prec in PRECISIONS:
        p = paths.get(prec)
        if p is not None and prec != line["config"]["precision"]:
            e = p.get("error_vs_fp64")
            out[prec + "@" + line["config"]["workload_key"]] = digest(
                p, None if e is None else {"dudt": e["dudt"], "dphidt": e["dphidt"]})
    for key in ("slosh3d",):
        sp = paths.get(key) or {}
        for prec in PRECISIONS:
            p = sp.get(prec)
            if p is not None:
                e = p.get("error_vs_fp64")
                out[prec + "@" + key] = digest(
                    p, None if e is None else {"dudt": e["dudt"], "dphidt": e["dphidt"]})
        if "error" in sp:
            out[key] = {"error": sp["error"][:160]}
    for key in ("surrogate", "surrogate_3d", "surrogate_slosh3d"):
        p = paths.get(key)
        if p is not None:
            out[key] = digest(p, (p.get("error") or {}) if isinstance(p, dict) else None)
            if isinstance(p, dict) and "plain_fp64_same_scene" in p:
                out[key]["plain_fp64_same_scene"] = p["plain_fp64_same_scene"]
                stg = p.get("stage", {})
                out[key]["stage_ms"] = stg.get("ms")
                out[key]["plain_stage_ms"] = stg.get("plain_fp64_stage_ms")
    if "cpu_baseline" in line:
        out["cpu_baseline_oracle"] = line["cpu_baseline"]["value"]
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2608_22269_gb300 import wbsph

    world, rank, local = dist_setup()
    wl = WORKLOADS[args.workload]
    t_setup = time.perf_counter()
    scene = wl["make"]()
    dim = scene.params["dim"]
    nf = scene.n_fluid
    setup_s = time.perf_counter() - t_setup
    prec_code = {"fp64": wbsph.FP64, "mixed": wbsph.MIXED, "df64": wbsph.DF64}
    primary = args.precision
    sim, m = time_path(scene, prec_code[primary], args, world, local)
    value = weak_scaling_value(nf * args.steps, world, m["ms"] / 1e3)
    roofline = pair_roofline(m, dim, nf, primary, args.workload)
    hbm = measured_peaks().get("hbm_gbs", 6686.1)
    bytes_ps = algorithmic_bytes_per_particle_step(dim)

    # ---- end to end through the C-ABI with pinned host buffers ----
    k_e2e = max(1, min(args.steps, 5))
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hx, hu, hphi = pin(sim.get("x")), pin(sim.get("u")), pin(sim.get("phi"))
    htype = pin(scene.type)
    hnormal, hmass = pin(scene.normal), pin(sim.get("mass"))
    ox = torch.empty_like(hx).pin_memory()
    ou = torch.empty_like(hu).pin_memory()
    ophi = torch.empty_like(hphi).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        sim.set_particles(hx, hu, hphi, htype, hnormal, hmass, where=wbsph.HOST)
        sim.step(1)
        sim.get("x", ox)
        sim.get("u", ou)
        sim.get("phi", ophi)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    h2d = sum(t.numel() * t.element_size() for t in (hx, hu, hphi, htype, hnormal, hmass))
    d2h = sum(t.numel() * t.element_size() for t in (ox, ou, ophi))
    e2e = {"value": round(nf * k_e2e * world / e2e_s, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": k_e2e,
           "api": "wbsph_set_particles(host) + wbsph_step(1) + wbsph_get_fields(x,u,phi -> host)"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(m["ms"] / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[primary],
        "data": "synthetic",
        "config": {"workload": wl["desc"], "precision": args.precision, "n_fluid": nf,
                   "n_total": scene.n, "dim": dim,
                   "l2": f"inputs larger than L2 ({m['st1']['device_bytes'] / 1e9:.2f} GB resident)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "unit_counted": "fluid particles x steps"},
        "roofline": roofline,
        "hbm": {"algorithmic_bytes_per_particle_step": bytes_ps,
                "achieved_gbs": round(value / world * bytes_ps / 1e9, 1), "peak_gbs": hbm,
                "frac": round(value / world * bytes_ps / (hbm * 1e9), 5)},
        "e2e": e2e,
        "gpu_launches": int(m["st1"]["launches"] - m["st0"]["launches"]),
        "clocks": m["clocks"],
        "kernel_ms": {k: round(v[0], 3) for k, v in m["prof"].items()},
        "setup_s": round(setup_s, 1),
    }
    line["config"]["workload_key"] = args.workload
    if not args.no_paths:
        # every precision on the same workload, and the errors of the mixed and
        # double-float paths at this size against the FP64 path on one state
        paths, sims = precision_paths(scene, args, world, local, args.workload, primary, sim, m)
        line["error"] = {
            "fp64_vs_oracle": "within 1e-12 (tests/test_gpu_fullsize.py samples this workload)",
            "measure": "max|a-b| / max(max|b|, natural scale) over fluid particles"}
        for k, s2 in sims.items():
            if k != primary:
                s2.close()
        if args.workload == "dam3d":
            # the metric's second point: the 17.58M-fluid sloshing tank, every precision
            try:
                big = WORKLOADS["slosh3d"]["make"]()
                sp, ssims = precision_paths(big, args, world, local, "slosh3d",
                                            steps=min(args.steps, 10), warmup=3)
                sp["workload"] = WORKLOADS["slosh3d"]["desc"]
                sp["n_fluid"], sp["n_total"] = big.n_fluid, big.n
                for s2 in ssims.values():
                    s2.close()
                del ssims, big
            except Exception as exc:  # report, do not abort the headline
                sp = {"error": f"{type(exc).__name__}: {exc}"}
            paths["slosh3d"] = sp
        if rank == 0:
            for key, sdim, ssc in (("surrogate", 2, None), ("surrogate_3d", 3, None),
                                   ("surrogate_slosh3d", 3, "slosh3d")):
                try:
                    paths[key] = surrogate_path(args, local, sdim, ssc)
                except Exception as exc:  # the plain paths above are the headline; report, do not abort
                    paths[key] = {"error": f"{type(exc).__name__}: {exc}"}
        line["paths"] = paths
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = wl["sample"]()
        v, steps, secs, cores = cpu_baseline(sample)
        line["cpu_baseline"] = {"value": round(v, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{wl['sample_desc']}, {steps} steps in {secs:.1f} s"}
    if rank == 0:
        line["summary"] = summary_of(line)   # last key: the compact digest ends the line
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    sample = wl["sample"]()
    st = oracle.State(sample)
    st.step(args.warmup)
    t0 = time.perf_counter()
    st.step(args.steps)
    secs = time.perf_counter() - t0
    v = sample.n_fluid * args.steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "precision": "fp64", "sample": wl["sample_desc"]},
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"{wl['sample_desc']}, {args.steps} timed steps"},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dam3d", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paths", action="store_true",
                    help="skip the second precision and the surrogate paths")
    ap.add_argument("--only-surrogate", action="store_true",
                    help="run only the surrogate rollout timing (profiling aid)")
    ap.add_argument("--surrogate-dim", type=int, default=2, choices=(2, 3),
                    help="with --only-surrogate: the 2D or the 3D surrogate case")
    ap.add_argument("--surrogate-stage", type=float, default=None, metavar="DX",
                    help="profiling aid: one 3D surrogate stage on the 3D dam break at spacing DX, "
                         "after a warm one, inside the NVTX range 'surrogate_stage'")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.surrogate_stage:
        print(json.dumps(surrogate_stage_profile(args.surrogate_stage)), flush=True)
    elif args.only_surrogate:
        import torch
        torch.cuda.set_device(0)
        key = "surrogate" if args.surrogate_dim == 2 else "surrogate_3d"
        print(json.dumps({key: surrogate_path(args, 0, args.surrogate_dim)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
