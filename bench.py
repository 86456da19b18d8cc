"""Benchmark: the multi-level greedy RBF mesh deformation hot path on one
GB300 (or N replicas under torchrun).

One step = the whole path for the 3D swept-wing workload: 60,000 surface
points (400 chordwise x 150 spanwise), 6,000,000 volume points, three greedy
levels (R = 1.5c, 0.4c, 0.1c), eps = 1e-5, volume reduction factor k = 4 with
D = 1c, a leading-edge ice ridge.  rbfd_create (Morton preparation of the
surface), rbfd_greedy (every level to its tolerance, about 31,000 controls)
and rbfd_deform (volume point reduction and the psi-blended update of every
volume point), as one rbfd_run_jobs call; the counters are read and the mesh
destroyed after the timed region.

value    = RBF pair evaluations with |r - r_c| < R that the kernels performed
           (list sweeps of Eq. 12, the Newton-basis update's phi values, the
           volume update of Eq. 23) over the timed steps on all ranks / max
           over ranks of the device time (CUDA events on the launching stream),
           inputs resident in HBM; L2 is flushed between steps and the volume
           (96 MB in, 72 MB out, plus the packed copies) exceeds it anyway.
           Eq. 12's own pair count for every greedy step (what a list sweep of
           each step evaluates) is reported beside it as eq12_pairs_per_step.
           The list sweep skips the warps of points whose bound shows they
           cannot hold a step's argmax (option prune, on; --no-prune turns it
           off): fewer pairs, same controls, shorter time to eps.  What it
           skipped is in sweep_pairs_skipped_per_step.
time_to_eps_ms = device time of rbfd_greedy (all levels to eps).
e2e      = the same through host (pinned) buffers: host->device copies of the
           inputs and device->host copy of the volume displacement inside the
           timed region.
roofline = the dominant kernel by device time (library profiler, CUDA events
           on the mesh's stream): its useful pair evaluations x the FP32-pipe
           operations of one plain FP32 pair (13 in 2D, 16 in 3D) over its
           launch time, against the FP32 issue rate (SMs x 128 lanes x max SM
           clock); the same with the double-float evaluation's own operation
           count beside it; per-phase times of the persistent launch; the
           volume sweep's own figures.  traffic: DRAM bytes per launch from an
           ncu capture, only while the kernel source is the one captured.
cpu_baseline = the FP64 oracle on the host cores over a bounded sample: the
           first K greedy steps of every level and a volume subset (the full
           greedy of 31,000 controls would take the oracle hours); the full
           step's oracle time is extrapolated from it and labelled so.
clocks   = SM clocks and throttle reasons sampled by nvidia-smi every 200 ms
           over the warm-up and timed steps; gpu_launches = the library's
           kernel launches in the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64] [--workload NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "wing_60ks_6mv_ridge"
CASES = (WORKLOAD,)
METRIC = "rbf_pair_evals_per_s"
UNIT = "pair-evals/s"

# FP32-pipe operations of one useful pair evaluated in plain FP32 (the
# evaluation's algorithmic unit: differences, r^2, rsqrt-based eta, phi, three
# accumulating FMAs; 2D has two coordinates and two components)
OPS_PER_PAIR_FP32 = {2: 13, 3: 16}
# FP32-pipe operations of one pair in the double-float evaluation the mixed
# mode runs, counted from csrc/common.cuh (df_add 20, df_mul 7, df_sqr 7,
# df_sqrt 12 incl. MUFU): 2D differences 2 x 20, r^2 2 x 7 + 20, sqrt 12,
# eta 7, phi 63, accumulate 2 x 27 -> 210; 3D -> 284
OPS_PER_PAIR_DF = {2: 210, 3: 284}
FP32_LANES_PER_SM = 128
# FP64 multiply-adds per SM per clock on GB300 (the nominal 1.25 TFLOP/s over
# 152 SMs at 2.07 GHz is about 4 flops, two FMAs, per SM per clock)
FP64_FMA_PER_SM_CLK = 2
CPU_BASELINE_S = 15.0  # about this much oracle time behind the cpu_baseline figure

# DRAM bytes (read + written) per launch from an ncu capture, each with the
# SHA-256 prefix of the kernel's source file when it was captured: a figure
# whose source has changed since is reported as null
DRAM_BYTES_PER_LAUNCH = {}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--engine", type=int, default=0,
                   help="0: Newton-basis start + persistent list sweep, 2: persistent list sweep, 1: launches per step")
    p.add_argument("--ctas", type=int, default=0, help="blocks of the persistent launch (0: automatic)")
    p.add_argument("--no-prune", action="store_true",
                   help="sweep every surface point every greedy step (no bound-pruned skipping)")
    p.add_argument("--no-serve", action="store_true", help="skip the serving leg (p50/p99 latency)")
    p.add_argument("--serve-requests", type=int, default=1000)
    p.add_argument("--no-local-global", action="store_true",
                   help="skip Section 5's local (ice) vs global (sinusoid) comparison over the Wendland bases")
    p.add_argument("--oracle-steps", type=int, default=0,
                   help="greedy steps per level of the oracle sample (0: sized to about 15 s)")
    return p.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms, units, dev):
    """The whole job's (time, units) from every rank's: the slowest rank's
    time and the sum of the units (the ranks are independent replicas; this
    is the only collective)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def reference_rank_works(rank):
    """The reference arm (the oracle on the host cores) runs on rank 0 alone;
    the other ranks exit without work."""
    return rank == 0


def make_case(name):
    from paper_2107_13887_gb300 import synth

    return synth.make_config(name, seed=0)


def workload_config(c):
    return {"workload": c.name, "cases": [c.name], "n_surface": int(c.n_s), "n_volume": int(c.n_v),
            "dim": int(c.dim), "levels": len(c.R), "R": list(c.R), "eps": c.eps, "k": c.k, "D": c.D}


def source_sha16(rel):
    with open(os.path.join(ROOT, "paper_2107_13887_gb300", "csrc", rel), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


# ------------------------------------------------------------ oracle sample

def oracle_sample(c, k_steps, n_vol, n_threads=None, seed=0):
    """The FP64 oracle on a bounded sample of the workload: the first
    k_steps greedy steps of every level (nc_cap = k_steps; each later level
    takes the capped level's error) and the volume update of n_vol sampled
    volume points with those levels.  Returns a dict with the useful pair
    evaluations (|r - r_c| < R, counted with a k-d tree), the brute-force pair
    evaluations (every point against every control, as the oracle forms
    them) and the seconds of oracle time."""
    import oracle
    from scipy.spatial import cKDTree

    nt = n_threads or (os.cpu_count() or 1)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(c.n_v, size=min(n_vol, c.n_v), replace=False))
    xv = np.ascontiguousarray(c.xyz_v[idx])
    dv = np.ascontiguousarray(c.d_v[idx])
    t0 = time.perf_counter()
    res = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, nc_cap=k_steps, n_threads=nt)
    t1 = time.perf_counter()
    oracle.deform(res, c.xyz_s, c.R, xv, dv, c.k, c.D, n_threads=nt)
    t2 = time.perf_counter()
    tree_s = cKDTree(c.xyz_s)
    useful, brute_greedy = 0, 0
    for l, R in enumerate(c.R):
        C = res.idx[l]
        n = len(C)
        cnt = np.array([len(v) for v in tree_s.query_ball_point(c.xyz_s[C], r=R * (1 - 1e-12))])
        # control j is in the sweeps of steps j + 1 .. n (n - j sweeps, the stopping sweep included)
        useful += int((cnt * (n - np.arange(n))).sum())
        brute_greedy += c.n_s * n * (n + 1) // 2
    Dl = oracle.support_distances(res.smax, c.k, c.D)
    brute_vol = 0
    for l, R in enumerate(c.R):
        if not Dl[l] > 0 or len(res.idx[l]) == 0:
            continue
        keep = dv.astype(np.float64) < Dl[l]
        brute_vol += int(keep.sum()) * len(res.idx[l])
        if keep.any():
            tree_c = cKDTree(c.xyz_s[res.idx[l]])
            useful += int(sum(len(v) for v in tree_c.query_ball_point(xv[keep].astype(np.float64),
                                                                      r=R * (1 - 1e-12))))
    return {"pairs_useful": useful, "brute_greedy": brute_greedy, "brute_vol": brute_vol,
            "greedy_s": t1 - t0, "vol_s": t2 - t1, "seconds": t2 - t0, "k_steps": k_steps,
            "n_vol": int(len(idx)), "cores": nt}


def oracle_extrapolate(c, sample, nc_levels):
    """Oracle time of the full step, extrapolated from the sample's brute-force
    pair rates: the greedy of Section 3 forms n_s x n pairs at a step with n
    controls (its Eq. 9 solves are not counted, so this is a lower bound), the
    volume update forms (points below D_l) x n_l pairs per level, taken here
    as every volume point."""
    rate_g = sample["brute_greedy"] / max(sample["greedy_s"], 1e-9)
    rate_v = sample["brute_vol"] / max(sample["vol_s"], 1e-9) if sample["brute_vol"] else rate_g
    pairs_g = sum(c.n_s * n * (n + 1) // 2 for n in nc_levels)
    pairs_v = sum(c.n_v * n for n in nc_levels)
    return pairs_g / rate_g + pairs_v / rate_v


def oracle_steps_for(c, budget_s=CPU_BASELINE_S, cores=None):
    """Greedy steps per level that keep the oracle sample near budget_s on
    the host cores (about 2e8 brute-force pairs per second per core)."""
    cores = cores or (os.cpu_count() or 1)
    rate = 2.0e8 * cores
    k = int(np.sqrt(2.0 * budget_s * rate / (len(c.R) * c.n_s)))
    return int(max(20, min(k, 2000)))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def count(self):
        return len(self.lines)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ roofline

def roofline_of(stats, dim, sms, sm_clock_hz, precision_mixed):
    """Roofline of the dominant kernel by device time (the library's event
    timing on the mesh's stream).  The evaluation kernels are bound by the
    FP32 pipe (neither HBM nor tensor cores): peak = SMs x 128 lanes x clock.
    Their work is the useful pairs they evaluated x the operations of one
    plain FP32 pair; the double-float operation count is given beside it."""
    peak = sms * FP32_LANES_PER_SM * sm_clock_hz
    tot = lambda key: sum(s[key] for s in stats)
    kinds = {
        # (device ms, launches, useful pairs evaluated)
        "persist": (tot("persist_ms"), tot("persist_launches"), tot("sweep_pairs_useful")),
        "newton": (tot("newton_ms"), tot("newton_launches"), tot("newton_pairs_useful")),
        "vol": (tot("vol_ms"), tot("vol_launches"), tot("vol_pairs_useful")),
        "sweep": (tot("sweep_ms"), tot("sweep_launches"), 0),
    }
    names = {"persist": f"k_greedy_persist<{dim},2,{1 if precision_mixed else 0}>",
             "newton": f"k_greedy_newton<{dim},2,{1 if precision_mixed else 0}>",
             "vol": f"k_vol_sweep<{dim},2,{2 if precision_mixed else 0}>",
             "sweep": f"k_sweep<{dim},2,{1 if precision_mixed else 0}>"}
    srcs = {"persist": "persist.cu", "newton": "newton.cu", "vol": "deform.cu", "sweep": "greedy.cu"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    ms, launches, pairs = kinds[dom]

    def fr(p, ms_, ops):
        return (p * ops / (ms_ / 1e3)) / peak if ms_ > 0 else 0.0

    achieved = pairs * OPS_PER_PAIR_FP32[dim] / (ms / 1e3) if ms > 0 else 0.0
    traffic = None
    cap = DRAM_BYTES_PER_LAUNCH.get(dom)
    if cap and cap[1] == source_sha16(srcs[dom]):
        traffic = cap[0]
    phases = [round(sum(s["persist_phase_ms"][q] for s in stats), 3) for q in range(8)]
    vol_ms, vol_pairs = kinds["vol"][0], kinds["vol"][2]
    # the persistent launch keeps two pipes busy: the double-float sweep on
    # the FP32 pipe and the rows of G in FP64 (k (k + 1) / 2 multiply-adds
    # for the step adding control k).  Its two-pipe fraction is the time each
    # part needs at its own pipe's peak, summed, over the launch's time.
    p_ms, _, p_pairs = kinds["persist"]
    fp64_fma_peak = sms * FP64_FMA_PER_SM_CLK * sm_clock_hz
    grow_fma = tot("persist_grow_fma")
    frac_pipes = None
    if precision_mixed and p_ms > 0:
        frac_pipes = (p_pairs * OPS_PER_PAIR_DF[dim] / peak + grow_fma / fp64_fma_peak) / (p_ms / 1e3)
    # a2 (the sweep and the step's decision) and a4 (the growth: y = G phi and
    # the rows of G) apart, each over the wall time of its phases in the
    # launch (block 0's work plus its wait at the phase's barrier).  In FP64
    # mode the sweep's pairs run on the FP64 pipe: its survey-unit operations
    # are set against that pipe's instruction rate.
    a2_s = (phases[0] + phases[1]) / 1e3
    a4_s = (phases[4] + phases[5] + phases[6] + phases[7]) / 1e3
    rows_s = (phases[6] + phases[7]) / 1e3
    a2_peak = peak if precision_mixed else fp64_fma_peak
    by_phase = {
        "a2_sweep": {"s": round(a2_s, 3), "pairs_useful": int(p_pairs),
                     "frac": round(p_pairs * OPS_PER_PAIR_FP32[dim] / a2_s / a2_peak, 5) if a2_s > 0 else None,
                     "frac_df_ops": round(p_pairs * OPS_PER_PAIR_DF[dim] / a2_s / peak, 5)
                     if a2_s > 0 and precision_mixed else None,
                     "peak": "FP32 issue" if precision_mixed else "FP64 instructions (152 x 2 per clock)"},
        "a4_grow": {"s": round(a4_s, 3), "g_rows_s": round(rows_s, 3), "g_rows_fp64_fma": int(grow_fma),
                    "g_rows_frac": round(grow_fma / rows_s / fp64_fma_peak, 5) if rows_s > 0 else None},
    }
    return {
        "bound": "alu", "kernel": names[dom],
        "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
        "frac": achieved / peak if peak else 0.0,
        "frac_df_ops": fr(pairs, ms, OPS_PER_PAIR_DF[dim]) if precision_mixed else None,
        "traffic": traffic,
        "traffic_unit": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu)",
        "avg_launch_ms": ms / max(1, launches), "launches": int(launches),
        "pairs_per_launch": pairs / max(1, launches),
        "kernel_ms": {k: round(v[0], 3) for k, v in kinds.items()},
        "kernel_frac": {k: round(fr(v[2], v[0], OPS_PER_PAIR_FP32[dim]), 5) for k, v in kinds.items()
                        if v[0] > 0 and v[2]},
        # block 0 of the persistent launch, summed over levels and steps:
        # [2p] work of phase p (sweep, argmax + phi column, G phi, G row), [2p+1] wait at its barrier
        "persist_phase_ms": phases,
        "persist_by_phase": by_phase,
        "persist_pipes": {"grow_fp64_fma": int(grow_fma),
                          "fp64_fma_peak_per_s": fp64_fma_peak,
                          "frac": round(frac_pipes, 5) if frac_pipes is not None else None},
        "vol_sweep": {"ms": round(vol_ms, 3), "pairs_useful": int(vol_pairs),
                      "frac": round(fr(vol_pairs, vol_ms, OPS_PER_PAIR_FP32[dim]), 5),
                      "frac_df_ops": round(fr(vol_pairs, vol_ms, OPS_PER_PAIR_DF[dim]), 5) if precision_mixed
                      else None},
        "peak_basis": (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_clock_hz / 1e9:.2f} GHz (derived from "
                       "unit counts and clocks: MEASURED_PEAKS.json has no FP32 figure); work = useful pairs x "
                       f"{OPS_PER_PAIR_FP32[dim]} FP32-pipe operations of a plain FP32 pair (frac_df_ops: x "
                       f"{OPS_PER_PAIR_DF[dim]}, the double-float pair the mixed mode evaluates)"),
    }


# ------------------------------------------------------------ GPU arm, meshes together

def run_set(args):
    """A workload of several meshes (the four uneven wings): one step =
    rbfd_create of every mesh, the greedy runs side by side (rbfd_greedy_batch)
    and the volume updates of all meshes in one work-list launch
    (rbfd_deform_worklist, autotuned on the warm-up steps, its settings
    cached); wall distances are computed on the device.  Device time by CUDA
    events on the first mesh's stream after a device-wide wait on both sides."""
    import torch

    from paper_2107_13887_gb300 import rbfd, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    rbfd.load()
    cases = synth.make_config_set(args.workload, wall_distance=False)
    outs = [np.empty((c.n_v, c.dim), np.float32) for c in cases]
    precision = rbfd.MIXED if args.precision == "mixed" else rbfd.FP64

    def step():
        ms = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, nc_cap=c.nc_cap, profile=True)
              for c in cases]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rbfd.greedy_batch(ms)
        t1 = time.perf_counter()
        tune = rbfd.deform_worklist(ms, [c.xyz_v for c in cases], None, [c.D for c in cases],
                                    [c.k for c in cases], outs)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        st = [m.stats() for m in ms]
        lv = [[len(L.idx) for L in m.levels()] for m in ms]
        for m in ms:
            m.close()
        return t1 - t0, t2 - t1, st, lv, tune

    for _ in range(args.warmup):
        step()
    g_s, d_s, pairs, stats, tunes = 0.0, 0.0, 0, [], []
    for _ in range(args.steps):
        g, d, st, lv, tune = step()
        g_s += g
        d_s += d
        pairs += sum(s["pairs_useful"] for s in st)
        stats.append(st)
        tunes.append(tune)
    tot_ms = 1e3 * (g_s + d_s)
    line = {
        "metric": METRIC, "value": pairs / (tot_ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64" if precision == rbfd.MIXED else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "meshes": [c.name for c in cases],
                   "n_surface": [int(c.n_s) for c in cases], "n_volume": [int(c.n_v) for c in cases],
                   "levels": 3, "nc_cap": cases[0].nc_cap, "precision": args.precision,
                   "timing": "host wall clock around each call with device-wide waits on both sides"},
        "greedy_batch_ms": 1e3 * g_s / args.steps,
        "worklist_deform_ms": 1e3 * d_s / args.steps,
        "worklist_launch_ms": statistics.median(t["launch_ms"] for t in tunes),
        "autotuned": {k: tunes[-1][k] for k in ("ctas_per_sm", "item_blocks", "cell_div", "cached")},
        "controls_per_level": lv,
        "time_to_eps_ms": [s["greedy_ms"] for s in stats[-1]],
        "vol_pairs_useful_per_step": sum(s["vol_pairs_useful"] for s in stats[-1]),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2107_13887_gb300 import rbfd

    rbfd.load()
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    precision = rbfd.MIXED if args.precision == "mixed" else rbfd.FP64
    c = make_case(args.workload)
    stream = torch.cuda.Stream(dev, priority=-1)

    d = dict(xyz_s=torch.from_numpy(c.xyz_s).to(dev), dS=torch.from_numpy(c.dS).to(dev),
             xyz_v=torch.from_numpy(c.xyz_v).to(dev), d_v=torch.from_numpy(c.d_v).to(dev),
             out=torch.empty((c.n_v, c.dim), dtype=torch.float32, device=dev))

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    h = dict(xyz_s=pin(c.xyz_s), dS=pin(c.dS), xyz_v=pin(c.xyz_v), d_v=pin(c.d_v),
             out=pin(np.zeros((c.n_v, c.dim), np.float32)))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def one_step(src, record):
        """rbfd_run_jobs with one job: create (the surface's spatial set-up),
        greedy, volume update.  Returns the mesh; its counters are read and it
        is destroyed after the timed region."""
        job = dict(xyz_s=src["xyz_s"], dS=src["dS"], R=c.R, eps=c.eps, precision=precision,
                   stream=stream.cuda_stream, profile=record, engine=args.engine, grid_ctas=args.ctas,
                   prune=not args.no_prune,
                   xyz_v=src["xyz_v"], d_v=src["d_v"], D=c.D, k=c.k, out=src["out"])
        ms, _ = rbfd.run_jobs([job])
        return ms[0]

    def finish(m):
        st = m.stats()
        lv = [len(L.idx) for L in m.levels()]
        m.close()
        return st, lv

    def timed(src, K, W, record):
        for _ in range(W):
            finish(one_step(src, False))
        torch.cuda.synchronize()
        tot_ms, stats, nc = 0.0, [], None
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m = one_step(src, record)
            e1.record(stream)
            torch.cuda.synchronize()
            tot_ms += e0.elapsed_time(e1)
            st, nc = finish(m)
            stats.append(st)
        return tot_ms, stats, nc

    sampler = ClockSampler(local)
    sampler.start()
    ms, stats, nc_levels = timed(d, args.steps, args.warmup, True)
    clocks = sampler.stop()
    if clocks is not None:
        clocks["sampled_over"] = "warm-up and timed steps"
    pairs = sum(s["pairs_useful"] for s in stats)
    e2e = None
    if not args.no_e2e:
        ms_e, stats_e, _ = timed(h, args.steps, 0, False)
        pairs_e = sum(s["pairs_useful"] for s in stats_e)
    if ws > 1:
        ms_all, pairs_all = aggregate_over_ranks(ms, pairs, dev)
        if not args.no_e2e:
            ms_e, pairs_e = aggregate_over_ranks(ms_e, pairs_e, dev)
    else:
        ms_all, pairs_all = ms, float(pairs)
    if not args.no_e2e:
        h2d = c.xyz_s.nbytes + c.dS.nbytes + c.xyz_v.nbytes + c.d_v.nbytes
        d2h = c.n_v * c.dim * 4
        e2e = {"value": pairs_e / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e / args.steps}
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    clock_hz = 1e6 * (clocks["sm_max_mhz"] if clocks else 2070.0)
    mixed = precision == rbfd.MIXED
    med = lambda key: statistics.median([s[key] for s in stats])
    line = {
        "metric": METRIC, "value": pairs_all / (ms_all / 1e3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2+f64" if mixed else "f64", "data": "synthetic",
        "config": dict(workload_config(c), precision=args.precision,
                       l2="flushed (256 MB write) between timed steps; the 6M-point volume exceeds L2",
                       parallelism=f"replicas{ws}",
                       engine={0: "newton+persistent", 1: "per-step launches", 2: "persistent"}[args.engine],
                       persist_ctas=int(stats[-1]["persist_ctas"]) if stats else 0,
                       prune=not args.no_prune),
        "time_to_eps_ms": med("greedy_ms"),
        "deform_ms": med("deform_ms"),
        "controls_per_level": nc_levels,
        "pairs_useful_per_step": pairs_all / args.steps / ws,
        # Eq. 12's nonzeros for every greedy step (what a list sweep of each
        # step evaluates; the Newton-basis steps evaluate one phi per point
        # instead) plus the volume update's pairs: the method's own count
        "eq12_pairs_per_step": sum(s["eq12_pairs"] + s["vol_pairs_useful"] for s in stats) / args.steps,
        "pairs_visited_per_step": sum(s["pairs_visited"] for s in stats) / args.steps,
        # what the bound-pruned sweep skipped (points x list length, counted
        # as pairs_visited counts them) and the 32-point warp steps skipped
        "sweep_pairs_skipped_per_step": sum(s["sweep_pairs_skipped"] for s in stats) / args.steps,
        "sweep_warps_skipped_per_step": sum(s["sweep_warps_skipped"] for s in stats) / args.steps,
        "roofline": roofline_of(stats, c.dim, sms, clock_hz, mixed),
        "e2e": e2e,
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        k = args.oracle_steps or oracle_steps_for(c)
        smp = oracle_sample(c, k, n_vol=20000)
        line["cpu_baseline"] = {
            "value": smp["pairs_useful"] / smp["seconds"], "unit": UNIT, "cores": smp["cores"], "kind": "oracle",
            "sample": (f"first {k} greedy steps of each of the {len(c.R)} levels (nc_cap = {k}) + the volume "
                       f"update of {smp['n_vol']} sampled volume points (FP64 oracle, OpenMP)"),
            "seconds": smp["seconds"],
            "extrapolated_full_step_s": oracle_extrapolate(c, smp, nc_levels),
            "extrapolation": "lower bound: brute-force pair rates of the sample applied to the full step's "
                             "control counts, Eq. 9 solves not counted",
        }
    if not args.no_local_global:
        line["local_vs_global"] = local_global_comparison()
    if not args.no_serve:
        line["serving"] = run_serving(n_requests=args.serve_requests)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ local vs global

def local_global_comparison(precision_names=("fp64", "mixed")):
    """Section 5's comparison of a local (ice) and a global (sinusoid)
    deformation, with the Wendland bases of Table 1: per case and basis the
    controls per level, the final error and the greedy's device time to eps.
    2D: the 4,000-point airfoil with its three ice horns against the
    sinusoid dy = 0.01 sin(15 pi x) of Section 5.1; 3D: a 4,000-point wing
    (100 x 40) with the leading-edge ridge against the sinusoid of Eq. 27,
    dy = 0.03 sin(4 pi z).  Levels R = 1c then 0.2c (2D) and 1.5c then 0.4c
    (3D), eps = 1e-5 (2D) and 1e-4 (3D).  A basis whose control system the
    precision cannot resolve reports its status instead."""
    from paper_2107_13887_gb300 import rbfd, synth

    cases = {
        "2d_ice": synth.airfoil_case(4000, 0, displacement="horns", seed=0, R=(1.0, 0.2), eps=1e-5),
        "2d_sinusoid": synth.airfoil_case(4000, 0, displacement="sinusoid", seed=0, R=(1.0, 0.2), eps=1e-5),
        "3d_ice": synth.wing_case(100, 40, 0, displacement="ridge", seed=0, R=(1.5, 0.4), eps=1e-4),
        "3d_sinusoid": synth.wing_case(100, 40, 0, displacement="sinusoid", seed=0, R=(1.5, 0.4), eps=1e-4),
    }
    out = {}
    for pname in precision_names:
        prec = rbfd.FP64 if pname == "fp64" else rbfd.MIXED
        for cname, c in cases.items():
            for bname, bid in (("C0", 0), ("C2", 2), ("C4", 4), ("C6", 6)):
                key = f"{cname}/{bname}/{pname}"
                try:
                    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=prec, basis=bid, nc_cap=c.n_s)
                    rc = m.greedy()
                    lv = m.levels()
                    st = m.stats()
                    out[key] = {"controls_per_level": [len(L.idx) for L in lv],
                                "e_max": lv[-1].e_max if lv else 0.0, "time_to_eps_ms": st["greedy_ms"],
                                "status": rbfd.STATUS_NAMES.get(rc, rc)}
                    m.close()
                except rbfd.RbfdError as exc:
                    out[key] = {"status": rbfd.STATUS_NAMES.get(exc.status, exc.status), "error": str(exc)[:160]}
    return out


# ------------------------------------------------------------ serving leg

def serving_meshes():
    """Eight meshes drawn from the 2D and 3D workload families, 20k to 10M
    volume points, each with its base ice shape: the 400-point airfoil (40k),
    the two 4,000-point / 1M airfoil cases, the 4,000-point airfoil with
    2,500 layers (10M), a 1,000-point airfoil with 20 layers (20k), and three
    swept wings of the four-wing family at coarse surfaces (1.2k, 4k and 9k
    points with 20k-ish, 2M and 9M volume points; two levels to 1e-3, so that
    one time step costs milliseconds: the full 60k-point wing to 1e-5 takes
    seconds per step).  Wall distances are computed on the device."""
    from paper_2107_13887_gb300 import synth

    return [
        synth.make_config("naca0012_400s_40kv_bump", seed=0),
        synth.make_config("naca0012_4000s_1mv_horns", seed=0),
        synth.make_config("naca0012_4000s_1mv_pitch_heave", seed=0),
        synth.airfoil_case(4000, 2500, displacement="horns", seed=3, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0,
                           wall_distance=False),
        synth.airfoil_case(1000, 20, displacement="horns", seed=1, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0),
        synth.wing_case(60, 20, 18, displacement="ridge", seed=4, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0),
        synth.wing_case(100, 40, 500, displacement="ridge", seed=5, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0,
                        wall_distance=False),
        synth.wing_case(150, 60, 1000, displacement="ridge", seed=6, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0,
                        wall_distance=False),
    ]


def run_serving(n_requests=1000, rate=50.0, slots=4, seed=0):
    """Requests with Poisson arrivals at `rate`/s, each one time step of an
    ice-growth sequence (displacement scaled up linearly with the step) on one
    of the meshes; submitted in real time to the request loop.  Returns the
    latency percentiles (submit to done) and the throughput."""
    from paper_2107_13887_gb300 import rbfd

    meshes = serving_meshes()
    srv = rbfd.Server(slots=slots)
    ids = [srv.add_mesh(c.xyz_s, c.xyz_v, c.d_v, c.R, c.eps, c.D, c.k) for c in meshes]
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    which = rng.integers(0, len(meshes), size=n_requests)
    steps = np.zeros(len(meshes), dtype=int)
    per_mesh = np.bincount(which, minlength=len(meshes))
    # warm each mesh once (resident instances, code paths) outside the measured stream
    for mid, c in zip(ids, meshes):
        srv.wait(srv.submit(mid, c.dS * 0.5), timeout_s=600.0)
    tickets = []
    t0 = time.perf_counter()
    for a, w in zip(arrivals, which):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        c = meshes[w]
        growth = 0.2 + 0.8 * (steps[w] + 1) / per_mesh[w]
        steps[w] += 1
        tickets.append(srv.submit(ids[w], c.dS * growth))
    for t in tickets:
        srv.wait(t, timeout_s=600.0)
    wall = time.perf_counter() - t0
    tot = np.array([srv.times(t)[2] for t in tickets])
    que = np.array([srv.times(t)[0] for t in tickets])
    run = np.array([srv.times(t)[1] for t in tickets])
    srv.close()
    mesh_stats = []
    for i, c in enumerate(meshes):
        sel = which == i
        mesh_stats.append({"n_surface": int(c.n_s), "n_volume": int(c.n_v), "requests": int(sel.sum()),
                         "run_ms_p50": float(np.median(run[sel])) if sel.any() else None,
                         "run_ms_max": float(run[sel].max()) if sel.any() else None,
                         "latency_ms_p99": float(np.percentile(tot[sel], 99)) if sel.any() else None})
    return {
        "requests": n_requests, "arrival_rate_per_s": rate, "slots": slots, "meshes": len(meshes),
        "volume_points": [int(c.n_v) for c in meshes],
        "latency_ms_p50": float(np.percentile(tot, 50)), "latency_ms_p99": float(np.percentile(tot, 99)),
        "queue_ms_p50": float(np.percentile(que, 50)), "queue_ms_p99": float(np.percentile(que, 99)),
        "throughput_req_per_s": n_requests / wall, "wall_s": wall, "per_mesh": mesh_stats,
    }


# ------------------------------------------------------------ reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if not reference_rank_works(rank):
        return
    c = make_case(args.workload)
    k = args.oracle_steps or oracle_steps_for(c, budget_s=CPU_BASELINE_S / 2)
    cores = cpu_cores()
    for _ in range(args.warmup):
        oracle_sample(c, max(10, k // 4), n_vol=2000, seed=1)
    tot_p, tot_s, smp = 0, 0.0, None
    for step in range(args.steps):
        smp = oracle_sample(c, k, n_vol=20000, seed=100 + step)
        tot_p += smp["pairs_useful"]
        tot_s += smp["seconds"]
    v = tot_p / tot_s
    sample = (f"each step: the first {k} greedy steps of each of the {len(c.R)} levels (nc_cap = {k}) + the volume "
              f"update of {smp['n_vol']} sampled volume points (FP64 oracle, OpenMP on {smp['cores']} threads)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(c), precision="fp64"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": smp["cores"], "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    from paper_2107_13887_gb300 import synth

    if args.impl == "reference":
        run_reference(args)
    elif args.workload in synth.CONFIG_SETS:
        run_set(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
