"""The N-GPU bench path without GPUs: world_size-2 ranks over gloo on the CPU.

bench.py runs independent replicas (one mesh batch per rank, no collective on
the data path) and reduces only its result: the time is the maximum over the
ranks and the units are summed.  These tests run that reduction, and the
reference arm's rank rule (rank 0 alone works), in two processes.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys

        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import bench

        ws, r, local = bench.dist_env()
        ms, units = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
        results[rank] = (ws, r, local, ms, units, bench.reference_rank_works(r))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_reduce_time_by_max_and_units_by_sum():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert sorted(res) == [0, 1]
    for rank, (ws, r, local, ms, units, works) in res.items():
        assert (ws, r, local) == (2, rank, rank)
        assert ms == 15.0  # the slowest rank's time
        assert units == 3000.0  # every rank's units
        assert works == (rank == 0)  # the reference arm runs on rank 0 only


# ------------------------------------------------ the split of the hot path


def _split_main(rank, world, port, results):
    """One rank of the CPU emulation of the surface split: the greedy of
    Section 3 with this rank's keys limited to its Morton range of the
    surface and the per-step argmax combined by shard.allreduce_maxloc over
    gloo; the control system is solved identically on every rank (numpy).
    The volume update of this rank's Morton range of the volume points uses
    the oracle with the rank's own copy of the levels."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys

        import numpy as np
        from scipy.spatial.distance import cdist

        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle
        from paper_2107_13887_gb300 import shard, synth

        # the tie rule of the exchange: largest key, lowest index, (-1, -1) loses
        probes = [((5.0, 7), (5.0, 3)), ((2.0, 1), (3.0, 9)), ((-1.0, -1), (4.0, 2)), ((-1.0, -1), (-1.0, -1))]
        ties = [shard.allreduce_maxloc(*p[rank]) for p in probes]

        c = synth.airfoil_case(90, 4, displacement="horns", seed=4, R=(1.0, 0.25), eps=1e-4, D=2.0, k=5.0)
        mine = np.zeros(c.n_s, dtype=bool)
        mine[shard.morton_ranges(c.xyz_s, world)[rank]] = True
        phi = lambda e: np.where(e < 1.0, (1.0 - np.minimum(e, 1.0)) ** 4 * (4.0 * e + 1.0), 0.0)
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        cur = c.dS.copy()
        levels, alphas = [], []
        for l, R in enumerate(c.R):
            tau = c.eps ** ((l + 1) / len(c.R))
            C = [0]
            while True:
                a = np.linalg.solve(phi(cdist(c.xyz_s[C], c.xyz_s[C]) / R), cur[C])
                E = cur - phi(cdist(c.xyz_s, c.xyz_s[C]) / R) @ a
                key = (E**2).sum(1)
                key[C] = -1.0
                key[~mine] = -1.0
                i = int(np.argmax(key)) if (key >= 0).any() else -1
                k, i = shard.allreduce_maxloc(float(key[i]) if i >= 0 else -1.0, i)
                if i < 0 or np.sqrt(k) / S0 < tau:
                    break
                C.append(i)
            levels.append(np.array(C))
            alphas.append(a)
            cur = E
        res = oracle.GreedyResult(oracle.OK, levels, alphas,
                                  np.array([0.0] * len(c.R)), np.zeros(2), np.zeros(2), None, S0)
        res.smax = np.array([np.sqrt((t**2).sum(1)).max() for t in [c.dS, c.dS - phi(
            cdist(c.xyz_s, c.xyz_s[levels[0]]) / c.R[0]) @ alphas[0]]])
        vidx = shard.morton_ranges(c.xyz_v, world)[rank]
        vol = oracle.deform(res, c.xyz_s, c.R, c.xyz_v[vidx], c.d_v[vidx], c.k, c.D)
        # the single-rank update with the same levels, for the comparison
        full = oracle.deform(res, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D)
        results[rank] = (ties, [lv.tolist() for lv in levels], vidx.tolist(), vol.tolist(), full.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_split_matches_one_rank():
    """World size 2 over gloo: the exchange's tie rule, the surface-split
    greedy's control sequence equal to the single-rank oracle's, and the two
    ranks' volume ranges covering every point once with the single-rank
    update bit for bit."""
    import numpy as np

    import oracle
    from paper_2107_13887_gb300 import synth

    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_split_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    want_ties = [(5.0, 3), (3.0, 9), (4.0, 2), (-1.0, -1)]
    for r in range(world):
        assert [tuple(t) for t in res[r][0]] == want_ties
    c = synth.airfoil_case(90, 4, displacement="horns", seed=4, R=(1.0, 0.25), eps=1e-4, D=2.0, k=5.0)
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps)
    for r in range(world):
        assert len(res[r][1]) == ref.n_levels
        assert all(np.array_equal(np.array(a), b) for a, b in zip(res[r][1], ref.idx))
    vidx = np.concatenate([np.array(res[r][2], dtype=np.int64) for r in range(world)])
    assert np.array_equal(np.sort(vidx), np.arange(c.n_v))
    vol = np.concatenate([np.array(res[r][3]).reshape(-1, 2) for r in range(world)])
    full = np.array(res[0][4])
    assert np.array_equal(full, np.array(res[1][4]))  # the levels are the same on every rank
    assert np.array_equal(vol, full[vidx])  # each point's update is the single-rank one, bit for bit


def test_morton_ranges_cover_every_point_once_and_are_compact():
    import numpy as np

    from paper_2107_13887_gb300 import shard, synth

    c = synth.wing_case(40, 12, 6, displacement="ridge", seed=0, R=(1.5,), eps=1e-3)
    for world in (1, 2, 3, 8):
        parts = shard.morton_ranges(c.xyz_v, world)
        allv = np.concatenate(parts)
        assert np.array_equal(np.sort(allv), np.arange(c.n_v))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    # Morton halves are spatially compact: their boxes overlap far less than
    # those of two random halves of the same points
    def overlap(a, b):
        lo = np.maximum(a.min(0), b.min(0))
        hi = np.minimum(a.max(0), b.max(0))
        return float(np.prod(np.maximum(hi - lo, 0.0)))
    p0, p1 = shard.morton_ranges(c.xyz_v, 2)
    rng = np.random.default_rng(0).permutation(c.n_v)
    r0, r1 = rng[: c.n_v // 2], rng[c.n_v // 2:]
    x = c.xyz_v.astype(np.float64)
    assert overlap(x[p0], x[p1]) < 0.25 * overlap(x[r0], x[r1])
    assert shard.maxloc_pairs([1.0, 1.0, 0.5], [9, 4, 1]) == (1.0, 4)
