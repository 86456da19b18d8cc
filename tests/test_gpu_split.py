"""The multi-GPU split of the hot path, on one GPU: two (or three) ranks run
as host threads of one process, each with its own mesh and stream.  The
ranks exchange only on the host (the per-step all-reduce-maxloc is a host
barrier here, NCCL or gloo across processes), so no kernel of one rank ever
waits for another rank's kernels.

* rbfd_greedy_split: every rank ends with the levels of the single-rank step
  engine (options.engine = 1), controls and weights bit for bit;
* the volume update split by Morton ranges of the volume points: the ranks'
  results together are the single-call update of every point, bit for bit
  in FP64 mode (each point's sum runs over the same controls in the same
  order), within 1e-5 max|dS| in mixed mode.
"""
import threading

import numpy as np
import pytest

from paper_2107_13887_gb300 import rbfd, shard, synth

pytestmark = pytest.mark.gpu


class HostExchange:
    """All-reduce-maxloc between threads: each rank posts its candidate, the
    combined one (shard.maxloc_pairs) is read by all after a barrier."""

    def __init__(self, world):
        self.world = world
        self.vals = [None] * world
        self.bar = threading.Barrier(world, timeout=120)
        self.calls = [0] * world

    def fn(self, rank):
        def maxloc(key, idx):
            self.calls[rank] += 1
            self.vals[rank] = (key, idx)
            self.bar.wait()
            out = shard.maxloc_pairs([v[0] for v in self.vals], [v[1] for v in self.vals])
            self.bar.wait()
            return out
        return maxloc


def run_split(c, world, precision, **kw):
    meshes = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, **kw) for _ in range(world)]
    ex = HostExchange(world)
    rcs, errs = [None] * world, []

    def go(r):
        try:
            rcs[r] = meshes[r].greedy_split(r, world, ex.fn(r))
        except Exception as exc:  # noqa: BLE001
            errs.append(exc)
            ex.bar.abort()

    th = [threading.Thread(target=go, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    return meshes, rcs, ex


@pytest.mark.parametrize("name,world", [("airfoil", 2), ("wing", 2), ("wing", 3), ("tiny", 3)])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_greedy_split_equals_single_rank(name, world, precision):
    c = {"airfoil": synth.airfoil_case(1500, 40, displacement="horns", seed=2, R=(1.0, 0.2), eps=1e-5, D=2.0,
                                       k=5.0),
         "wing": synth.wing_case(60, 30, 8, displacement="ridge", seed=3, R=(1.5, 0.4), eps=1e-4, D=1.0, k=4.0),
         "tiny": synth.airfoil_case(150, 4, displacement="bump", seed=1, R=(0.5,), eps=1e-4, D=2.0, k=0.0)}[name]
    one = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=1)
    one.greedy()
    want = one.levels()
    meshes, rcs, ex = run_split(c, world, precision)
    assert all(n == ex.calls[0] for n in ex.calls) and ex.calls[0] >= sum(len(L.idx) for L in want) - len(want)
    for m in meshes:
        got = m.levels()
        assert len(got) == len(want)
        for a, b in zip(got, want):
            assert np.array_equal(a.idx, b.idx)
            assert np.array_equal(a.alpha, b.alpha)
            assert a.e_max == b.e_max
    # every rank deforms its Morton range of the volume: together, the single call's update bit for bit
    full = one.deform(c.xyz_v, c.d_v, c.D, c.k)
    got = np.empty_like(full)
    seen = np.zeros(c.n_v, dtype=int)
    for r, m in enumerate(meshes):
        idx, part = shard.deform_split(m, c.xyz_v, c.d_v, c.D, c.k, r, world)
        got[idx] = part
        seen[idx] += 1
    assert (seen == 1).all()
    if precision == rbfd.FP64:
        assert np.array_equal(got, full)
    else:
        # the FP32-input sweep forms coordinates relative to each point
        # block's corner, and the blocks of a range differ from those of the
        # whole volume: agreement within the mixed-mode bar
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        assert np.abs(got.astype(np.float64) - full).max() <= 1e-5 * S0 + np.abs(full).max() * 2.0**-24
    for m in meshes + [one]:
        m.close()


def test_greedy_split_callback_failure_is_reported():
    """A maxloc callback that fails (a lost peer, a collective that timed out)
    ends the call with RBFD_ECOMM; the mesh works afterwards."""
    c = synth.airfoil_case(300, 4, displacement="bump", seed=1, R=(0.5,), eps=1e-4, D=2.0, k=0.0)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    calls = []

    def broken(key, idx):
        calls.append(key)
        if len(calls) == 3:
            raise TimeoutError("peer lost")
        return key, idx

    with pytest.raises(rbfd.RbfdError) as ei:
        m.greedy_split(0, 2, broken)
    assert ei.value.status == rbfd.ECOMM
    with pytest.raises(rbfd.RbfdError) as ei:
        m.greedy_split(2, 2, lambda k, i: (k, i))
    assert ei.value.status == rbfd.EINVAL
    # a one-rank "split" is the step engine
    m.greedy_split(0, 1, lambda k, i: (k, i))
    a = m.levels()
    ref = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=1)
    ref.greedy()
    for x, y in zip(a, ref.levels()):
        assert np.array_equal(x.idx, y.idx) and np.array_equal(x.alpha, y.alpha)
    m.close()
    ref.close()
