"""Benchmark: RBF pair-evaluations/s of the multi-level greedy RBF mesh
deformation hot path on one GB300 (or N replicas under torchrun).

One step = the whole path for the 2D airfoil workload of 4,000 surface and
1,000,000 volume points, two greedy levels (R = 1c then 0.2c), eps = 1e-5,
for both displacement cases: a global rigid pitch (5 deg) + heave (0.05c), and
a three-horn ice shape.  For each case: rbfd_create (Morton prep), rbfd_greedy
(both levels, to eps), rbfd_deform (volume point reduction + update of every
volume point), the cases side by side; the counters are read and the meshes
destroyed after the timed region.

value   = useful point/control pair evaluations (|r - r_c| < R) of all timed
          steps on all ranks / max over ranks of the device time (CUDA events on
          the library's stream), inputs resident in HBM, L2 flushed between steps.
e2e     = the same through host (pinned) buffers: host->device copies of the
          inputs and device->host copies of the results inside the timed region.
roofline = the dominant kernel class by device time, its counted FP32-pipe
          operations over that time against the FP32 issue rate, its DRAM bytes
          per launch from an ncu capture of the same workload, and the Newton
          step's latency;
cpu_baseline = the FP64 oracle on the host cores over a bounded sample;
clocks = SM clocks and throttle reasons sampled (nvidia-smi, every 200 ms) from
          the warm-up on, the same step kept running untimed until three
          samples are in; gpu_launches = the library's kernel launches in the
          timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "naca0012_4000s_1mv"
CASES = ("naca0012_4000s_1mv_pitch_heave", "naca0012_4000s_1mv_horns")
METRIC = "rbf_pair_evals_per_s"
UNIT = "pair-evals/s"

# FP32-pipe operations per useful pair of the double-float evaluation, counted
# from csrc/common.cuh (df_add 20, df_mul 7, df_sqr 7, df_sqrt 12 incl. MUFU).
# 2D: differences 2 x 20, r^2 2 x 7 + 20,
# sqrt 12, eta 7, phi 63, accumulate 2 x 27 -> 210; 3D -> 284.
OPS_PER_PAIR_DF = {2: 210, 3: 284}
CPU_BASELINE_S = 10.0  # seconds of oracle time behind the cpu_baseline figure
OPS_PER_NEWTON_TERM = 12  # df multiply-add of a basis value: TwoProduct by FMA (4), TwoSum (6), two adds
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--engine", type=int, default=0,
                   help="0: Newton-basis start + persistent list sweep, 2: persistent list sweep, 1: launches per step")
    p.add_argument("--ctas", type=int, default=0, help="blocks of the persistent launch (0: automatic)")
    p.add_argument("--no-serve", action="store_true", help="skip the serving leg (p50/p99 latency)")
    p.add_argument("--serve-requests", type=int, default=200)
    return p.parse_args()


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


def make_cases():
    from paper_2107_13887_gb300 import synth

    return [synth.make_config(n, seed=0) for n in CASES]


# ------------------------------------------------------------ useful pairs

def useful_pairs_oracle_run(case, res, Dl, sample_idx=None):
    """Useful pair evaluations (|r - r_c| < R) of the oracle's own run:
    every greedy sweep (one per added control, plus the stopping sweep) and
    the volume update of the sampled volume points."""
    from scipy.spatial import cKDTree

    total = 0
    tree_s = cKDTree(case.xyz_s)
    for l, R in enumerate(case.R):
        C = res.idx[l]
        n = len(C)
        cnt = np.array([len(v) for v in tree_s.query_ball_point(case.xyz_s[C], r=R * (1 - 1e-12))])
        # control j is present in the sweeps of steps j+1 .. n (n - j sweeps)
        total += int((cnt * (n - np.arange(n))).sum())
    xv = case.xyz_v if sample_idx is None else case.xyz_v[sample_idx]
    dv = case.d_v if sample_idx is None else case.d_v[sample_idx]
    for l, R in enumerate(case.R):
        if not Dl[l] > 0 or len(res.idx[l]) == 0:
            continue
        keep = dv.astype(np.float64) < Dl[l]
        if not keep.any():
            continue
        tree_c = cKDTree(case.xyz_s[res.idx[l]])
        total += int(sum(len(v) for v in tree_c.query_ball_point(xv[keep].astype(np.float64), r=R * (1 - 1e-12))))
    return total


def oracle_step(cases, frac, rng_seed=0, n_threads=None, count=True):
    """One CPU step with the FP64 oracle: full greedy of every case, volume
    update of a random `frac` of the volume points (all of them at frac = 1).
    Returns (useful_pairs, seconds)."""
    import oracle

    nt = n_threads or (os.cpu_count() or 1)
    rng = np.random.default_rng(rng_seed)
    pairs = 0
    secs = 0.0
    for c in cases:
        if frac >= 1.0:
            idx = np.arange(c.n_v)
        else:
            idx = np.sort(rng.choice(c.n_v, size=max(1, int(frac * c.n_v)), replace=False))
        xv = np.ascontiguousarray(c.xyz_v[idx])
        dv = np.ascontiguousarray(c.d_v[idx])
        t0 = time.perf_counter()
        res = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=nt)
        oracle.deform(res, c.xyz_s, c.R, xv, dv, c.k, c.D, n_threads=nt)
        secs += time.perf_counter() - t0
        if count:
            Dl = oracle.support_distances(res.smax, c.k, c.D)
            pairs += useful_pairs_oracle_run(c, res, Dl, idx)
    return pairs, secs


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# DRAM bytes per launch (read + written) from an ncu capture of the same
# workload, for the kernels whose code has not changed since
# (profiles/k_greedy_newton_naca0012_4000s.md: the mean of the four launches
# of one step)
DRAM_BYTES_PER_LAUNCH = {"newton": 434624}


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
    precision = rbfd.MIXED if args.precision == "mixed" else rbfd.FP64
    cases = make_cases()
    stream = torch.cuda.current_stream(dev)

    # device-resident inputs
    dcases = []
    for c in cases:
        dcases.append(dict(
            xyz_s=torch.from_numpy(c.xyz_s).to(dev), dS=torch.from_numpy(c.dS).to(dev),
            xyz_v=torch.from_numpy(c.xyz_v).to(dev), d_v=torch.from_numpy(c.d_v).to(dev),
            out=torch.empty((c.n_v, c.dim), dtype=torch.float32, device=dev)))
    # pinned host inputs for the end-to-end leg
    hcases = []
    for c in cases:
        def pin(a):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            return t.numpy()
        hcases.append(dict(xyz_s=pin(c.xyz_s), dS=pin(c.dS), xyz_v=pin(c.xyz_v), d_v=pin(c.d_v),
                           out=pin(np.zeros((c.n_v, c.dim), np.float32))))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    # each case gets its own stream so that the batch calls overlap them
    # (high priority: the library's staging streams, at the lowest, fill in behind the greedy)
    streams = [torch.cuda.Stream(dev, priority=-1) for _ in cases]

    def one_step(src, record):
        """Both cases as one library call (rbfd_run_jobs): per case, create
        (the spatial set-up of the surface), greedy and volume update, the
        cases side by side on their own host threads and streams.  Returns the
        meshes; their counters are read and they are destroyed after the timed
        region."""
        jobs = [dict(xyz_s=d["xyz_s"], dS=d["dS"], R=c.R, eps=c.eps, precision=precision, stream=s_.cuda_stream,
                     profile=record, engine=args.engine, grid_ctas=args.ctas, xyz_v=d["xyz_v"], d_v=d["d_v"],
                     D=c.D, k=c.k, out=d["out"]) for c, d, s_ in zip(cases, src, streams)]
        ms, _ = rbfd.run_jobs(jobs)
        return ms

    def finish(ms):
        stats = [m.stats() for m in ms]
        for m in ms:
            m.close()
        return sum(st["pairs_useful"] for st in stats), stats

    def timed(src, K, W, record):
        for _ in range(W):
            finish(one_step(src, False))
        torch.cuda.synchronize()
        tot_ms, tot_pairs, all_stats = 0.0, 0, []
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s_ in streams:  # the case streams start after e0
                s_.wait_event(e0)
            meshes = one_step(src, record)
            for s_ in streams:  # e1 follows the work of every case stream
                stream.wait_stream(s_)
            e1.record(stream)
            torch.cuda.synchronize()
            tot_ms += e0.elapsed_time(e1)
            p, st = finish(meshes)
            tot_pairs += p
            all_stats.extend(st)
        return tot_ms, tot_pairs, all_stats

    sampler = ClockSampler(local)
    sampler.start()
    ms, pairs, stats = timed(dcases, args.steps, args.warmup, True)
    # nvidia-smi samples every 200 ms, longer than a short timed region: the
    # same step keeps running (untimed) until three samples have been taken
    # under this load, at most 3 s
    t_stop = time.monotonic() + 3.0
    while sampler.count() < 3 and time.monotonic() < t_stop:
        finish(one_step(dcases, False))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if clocks is not None:
        clocks["sampled_over"] = "warm-up, timed steps and untimed repeats of the same step"
    e2e = None
    if not args.no_e2e:
        ms_e, pairs_e, _ = timed(hcases, args.steps, args.warmup, False)
    # aggregate over ranks: units summed, time = max
    if ws > 1:
        ms_all, pairs_all = aggregate_over_ranks(ms, pairs, dev)
        if not args.no_e2e:
            ms_e, pairs_e = aggregate_over_ranks(ms_e, pairs_e, dev)
    else:
        ms_all, pairs_all = ms, float(pairs)
    if not args.no_e2e:
        h2d = sum(c.xyz_s.nbytes + c.dS.nbytes + c.xyz_v.nbytes + c.d_v.nbytes for c in cases)
        d2h = sum(c.n_v * c.dim * 4 for c in cases)
        e2e = {"value": pairs_e / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e / args.steps}
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # roofline of the dominant kernel class (device time inside the timed region)
    sweep_pairs = sum(s["sweep_pairs_useful"] for s in stats)
    dim = cases[0].dim
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * 2.07e9  # FP32 issue slots per second at max SM clock
    # (device ms, launches, FP32-pipe operations of the work the class did)
    kinds = {
        "sweep": (sum(s["sweep_ms"] for s in stats), sum(s["sweep_launches"] for s in stats),
                  sweep_pairs * OPS_PER_PAIR_DF[dim]),
        "grow": (sum(s["grow_ms"] for s in stats), sum(s["grow_launches"] for s in stats), 0),
        "vol": (sum(s["vol_ms"] for s in stats), sum(s["vol_launches"] for s in stats),
                sum(s["vol_pairs_useful"] for s in stats) * OPS_PER_PAIR_DF[dim]),
        # the persistent list sweep runs the sweeps AND the FP64 growth; only
        # its sweep pairs are counted as work here, so its fraction is a lower bound
        "persist": (sum(s["persist_ms"] for s in stats), sum(s["persist_launches"] for s in stats),
                    0),
        # the Newton-basis launch: one double-float multiply-add (12 FP32
        # operations) per basis value read; its per-point tail and growth are
        # not counted, so the fraction is a lower bound
        "newton": (sum(s["newton_ms"] for s in stats), sum(s["newton_launches"] for s in stats),
                   sum(s["newton_terms"] for s in stats) * OPS_PER_NEWTON_TERM),
    }
    names = {"sweep": f"k_sweep<{dim},2,1>", "vol": f"k_vol_sweep<{dim},2,1>",
             "persist": f"k_greedy_persist<{dim},2,1>", "newton": f"k_greedy_newton<{dim},2,1>"}
    ev_kinds = {k: v for k, v in kinds.items() if k != "grow"}
    dom = max(ev_kinds, key=lambda k: ev_kinds[k][0])
    d_ms, d_launch, d_ops = ev_kinds[dom]
    achieved = d_ops / (d_ms / 1e3) if d_ms > 0 else 0.0
    roofline = {
        "bound": "alu", "kernel": names[dom],
        "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
        "frac": achieved / peak_ops, "traffic": DRAM_BYTES_PER_LAUNCH.get(dom),
        "traffic_unit": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu)",
        "avg_launch_ms": d_ms / max(1, d_launch), "launches": int(d_launch),
        "kernel_ms": {k: round(v[0], 3) for k, v in kinds.items()},
        "kernel_frac": {k: round(v[2] / (v[0] / 1e3) / peak_ops, 5) for k, v in kinds.items() if v[0] > 0 and v[2]},
        "persist_phase_ms": [round(sum(s["persist_phase_ms"][q] for s in stats), 3) for q in range(8)],
        # the Newton launches' device time per greedy step (the two cases run
        # side by side, so this is the latency of one case's step)
        "newton_us_per_step": round(1e3 * sum(s["newton_ms"] for s in stats)
                                    / max(1, sum(s["newton_steps"] for s in stats)), 3),
        "note": ("FP32-pipe operations: 210 (2D) / 284 (3D) per double-float pair evaluation, 12 per "
                 "double-float basis multiply-add; peak = 152 SMs x 128 FP32 lanes x 2.07 GHz. The greedy "
                 "launches are latency-bound chains of dependent steps (one grid barrier per step)"),
    }
    greedy_ms = [s["greedy_ms"] for s in stats]
    line = {
        "metric": METRIC, "value": pairs_all / (ms_all / 1e3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2+f64" if precision == rbfd.MIXED else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cases": list(CASES), "n_surface": 4000, "n_volume": 1000000,
                   "levels": 2, "R": [1.0, 0.2], "eps": 1e-5, "k": 5.0, "D": 2.0, "precision": args.precision,
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas{ws}",
                   "engine": {0: "newton+persistent", 1: "per-step launches", 2: "persistent"}[args.engine],
                   "persist_ctas": int(stats[-1]["persist_ctas"]) if stats else 0},
        "time_to_eps_ms": {"pitch_heave": statistics.median(greedy_ms[0::2]),
                           "horns": statistics.median(greedy_ms[1::2])},
        # device time of each case's volume update (after its greedy), median over the timed steps
        "deform_ms": {"pitch_heave": statistics.median([s["deform_ms"] for s in stats[0::2]]),
                      "horns": statistics.median([s["deform_ms"] for s in stats[1::2]])},
        "pairs_useful_per_step": pairs_all / args.steps / ws,
        # the second count: pairs the kernels evaluated (the useful ones plus
        # those the cell and control lists let through beyond R; the Newton
        # start counts its basis multiply-adds), per step and per second (rank 0)
        "pairs_visited_per_step": sum(s["pairs_visited"] for s in stats) / args.steps,
        "visited_per_s": sum(s["pairs_visited"] for s in stats) / (ms / 1e3),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        # the whole step (both cases, every volume point), repeated until at
        # least CPU_BASELINE_S seconds of oracle time have run
        # (the full step is the same every time: its pairs are counted once)
        p_cpu, s_cpu, reps, p_one = 0, 0.0, 0, 0
        while s_cpu < CPU_BASELINE_S and reps < 200:
            p, s_ = oracle_step(cases, 1.0, count=(reps == 0))
            p_one = p_one or p
            p_cpu += p_one
            s_cpu += s_
            reps += 1
        line["cpu_baseline"] = {"value": p_cpu / s_cpu, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"the full step (greedy of both cases + volume update of all their "
                                          f"volume points) repeated {reps} times (FP64 oracle, OpenMP)",
                                "seconds": s_cpu}
    if not args.no_serve:
        line["serving"] = run_serving(n_requests=args.serve_requests)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ serving leg

def serving_meshes():
    """Eight meshes drawn from the 2D and 3D workload families (20k to 1M
    volume points), each with its base ice shape."""
    from paper_2107_13887_gb300 import synth

    return [
        synth.make_config("naca0012_400s_40kv_bump", seed=0),
        synth.airfoil_case(1000, 100, displacement="horns", seed=1, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0),
        synth.airfoil_case(2000, 150, displacement="horns", seed=2, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0),
        synth.make_config("naca0012_4000s_1mv_horns", seed=0),
        synth.make_config("naca0012_4000s_1mv_pitch_heave", seed=0),
        synth.airfoil_case(800, 25, displacement="bump", seed=3, R=(0.5,), eps=1e-4, D=2.0, k=0.0),
        synth.wing_case(60, 20, 20, displacement="ridge", seed=4, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0),
        synth.wing_case(80, 30, 25, displacement="ridge", seed=5, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0),
    ]


def run_serving(n_requests=200, rate=50.0, slots=4, seed=0):
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
    srv.close()
    return {
        "requests": n_requests, "arrival_rate_per_s": rate, "slots": slots, "meshes": len(meshes),
        "volume_points": [int(c.n_v) for c in meshes],
        "latency_ms_p50": float(np.percentile(tot, 50)), "latency_ms_p99": float(np.percentile(tot, 99)),
        "queue_ms_p50": float(np.percentile(que, 50)), "queue_ms_p99": float(np.percentile(que, 99)),
        "throughput_req_per_s": n_requests / wall, "wall_s": wall,
    }


# ------------------------------------------------------------ reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if not reference_rank_works(rank):
        return
    cases = make_cases()
    frac = 1.0  # the whole workload each step
    cores = cpu_cores()
    for _ in range(args.warmup):
        oracle_step(cases, frac, rng_seed=1, count=False)
    tot_p, tot_s, p_one = 0, 0.0, 0
    for k in range(args.steps):
        p, s = oracle_step(cases, frac, rng_seed=100 + k, count=(k == 0))  # the same full step each time
        p_one = p_one or p
        tot_p += p_one
        tot_s += s
    v = tot_p / tot_s
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cases": list(CASES), "n_surface": 4000, "n_volume": 1000000,
                   "levels": 2, "R": [1.0, 0.2], "eps": 1e-5, "k": 5.0, "D": 2.0},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: the full workload (greedy of both cases + volume update of "
                                   "all their volume points)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
