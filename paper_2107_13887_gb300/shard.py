"""Multi-GPU split of the hot path: one process per GPU, host side.

The method shards along its two sweeps:

* Volume update (Eq. 19 with the blending of Eq. 23, Section 4): every volume
  point is independent, so the points are split into contiguous ranges of
  their Morton order (spatially compact ranges: each GPU's cell-list sweep
  touches a compact set of control cells) and every rank deforms its range
  with its own copy of the levels (controls and weights are replicated: at
  most 32 bytes per control).  No collective is needed.
* Greedy selection (Section 3): ``rbfd_greedy_split`` sweeps E = dS - Phi_sc
  alpha (Eq. 12) over a rank's range of the Morton-ordered surface point
  blocks; each step's argmax over all ranks is one all-reduce-maxloc of a
  16-byte (key, index) pair (``allreduce_maxloc``); the control system is
  updated identically on every rank.

Serving replicates whole meshes per GPU and needs none of this.
"""
from __future__ import annotations

import numpy as np

__all__ = ["morton_order", "morton_ranges", "maxloc_pairs", "allreduce_maxloc", "greedy_split", "deform_split"]


def _spread_bits(v: np.ndarray, dim: int) -> np.ndarray:
    """Insert dim - 1 zero bits between the bits of v (uint64, up to 21 bits)."""
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    nbits = 21 if dim == 3 else 31
    for b in range(nbits):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(dim * b)
    return out


def morton_order(xyz) -> np.ndarray:
    """Stable permutation that sorts the points by their Morton (Z-order) key
    on a 2^21 (3D) or 2^31 (2D) grid over their bounding box."""
    x = np.asarray(xyz, dtype=np.float64)
    n, dim = x.shape
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    lo = x.min(0)
    ext = np.maximum(x.max(0) - lo, 1e-300)
    top = (1 << (21 if dim == 3 else 31)) - 1
    q = np.clip(np.floor((x - lo) / ext * top), 0, top).astype(np.uint64)
    key = np.zeros(n, dtype=np.uint64)
    for a in range(dim):
        key |= _spread_bits(q[:, a], dim) << np.uint64(a)
    return np.argsort(key, kind="stable")


def morton_ranges(xyz, world: int):
    """Split the points into `world` contiguous ranges of their Morton order,
    of sizes differing by at most one.  Returns one index array per rank
    (indices into xyz, in Morton order); together they hold every index once."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = morton_order(xyz)
    n = order.shape[0]
    bounds = [n * r // world for r in range(world + 1)]
    return [order[bounds[r]:bounds[r + 1]] for r in range(world)]


def maxloc_pairs(keys, idxs):
    """The combined candidate of several ranks: the largest key, the lowest
    index among equal keys (the tie rule of the single-GPU argmax); a rank
    without a candidate reports (-1, -1)."""
    best_k, best_i = -1.0, -1
    for k, i in zip(keys, idxs):
        k, i = float(k), int(i)
        if i < 0:
            continue
        if best_i < 0 or k > best_k or (k == best_k and i < best_i):
            best_k, best_i = k, i
    return best_k, best_i


def allreduce_maxloc(key: float, idx: int, group=None):
    """All-reduce-maxloc of one (key, index) pair over the ranks of `group`
    (torch.distributed, any backend): an all-gather of 16 bytes per rank and
    the same pick on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([float(key), float(idx)], dtype=torch.float64, device=dev)
    allv = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    pairs = torch.stack(allv).cpu().numpy()
    return maxloc_pairs(pairs[:, 0], pairs[:, 1].astype(np.int64))


def greedy_split(mesh, group=None, allow_not_converged: bool = True) -> int:
    """rbfd_greedy_split on this rank of `group`: the surface sweep over this
    rank's Morton range, the per-step argmax combined by allreduce_maxloc."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    return mesh.greedy_split(rank, world, lambda k, i: allreduce_maxloc(k, i, group),
                             allow_not_converged=allow_not_converged)


def deform_split(mesh, xyz_v, d_v, D: float, k: float, rank: int, world: int):
    """This rank's share of the volume update: its Morton range of the volume
    points, deformed with its own copy of the levels.  Returns (indices into
    the caller's arrays, displacements of those points)."""
    idx = morton_ranges(np.asarray(xyz_v), world)[rank]
    sub_x = np.ascontiguousarray(np.asarray(xyz_v)[idx])
    sub_d = None if d_v is None else np.ascontiguousarray(np.asarray(d_v)[idx])
    return idx, mesh.deform(sub_x, sub_d, D, k)
