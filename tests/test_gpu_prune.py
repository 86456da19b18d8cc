"""The pruned list sweep (option ``prune``, on by default): a point block is
skipped in a greedy step while a bound shows that none of its points can hold
the step's argmax.  The picks and the stop test must be those of the full
sweep, so the levels (controls and weights, every bit) must equal the
unpruned run's, and the oracle's replay must accept every pick; the
skipped-work counters must show that blocks were skipped.
"""
import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth
from test_gpu_parity import NT, check_replay

pytestmark = pytest.mark.gpu


def _levels(c, **kw):
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, **kw)
    try:
        rc = m.greedy()
        return rc, m.levels(), m.stats()
    finally:
        m.close()


def _same_levels(a, b):
    assert len(a) == len(b)
    for l, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x.idx, y.idx), f"level {l}: control sequences differ"
        assert np.array_equal(x.alpha, y.alpha), f"level {l}: weights differ"
        assert x.e_max == y.e_max


def _wing():
    # the benchmark's swept wing at 1/15 of its surface: three levels, the
    # finest (R = 0.1c) local enough that most blocks are skipped per step
    return synth.wing_case(100, 40, 2, displacement="ridge", seed=0, R=(1.5, 0.4, 0.1), eps=1e-5, D=1.0, k=4.0,
                           wall_distance=False)


@pytest.mark.parametrize("precision", [rbfd.MIXED, rbfd.FP64])
def test_pruned_persistent_sweep_equals_full_sweep(precision):
    c = _wing()
    rc0, full, st0 = _levels(c, precision=precision, engine=2, prune=False, profile=True)
    rc1, pruned, st1 = _levels(c, precision=precision, engine=2, prune=True, profile=True)
    assert rc0 == rc1 == rbfd.OK
    _same_levels(full, pruned)
    assert st0["sweep_warps_skipped"] == 0 and st0["sweep_pairs_skipped"] == 0
    assert st1["sweep_warps_skipped"] > 0
    # the skipped pairs are pairs the full sweep visited
    assert st1["sweep_pairs_visited"] < st0["sweep_pairs_visited"]
    assert st1["sweep_pairs_visited"] + st1["sweep_pairs_skipped"] >= st0["sweep_pairs_visited"] * 0.999
    print(f"{'fp64' if precision == rbfd.FP64 else 'mixed'}: visited {st0['sweep_pairs_visited']:.3e} -> "
          f"{st1['sweep_pairs_visited']:.3e}, greedy {st0['greedy_ms']:.1f} -> {st1['greedy_ms']:.1f} ms")


def test_pruned_sweep_matches_the_oracle_sequence():
    # (seed 1: the oracle's closest pair of keys differs by 4e-6 relative, far
    # above FP64 rounding, so the FP64 sequence must be the oracle's exactly)
    c = synth.wing_case(60, 30, 2, displacement="ridge", seed=1, R=(1.0, 0.3, 0.1), eps=1e-5, D=1.0, k=4.0,
                        wall_distance=False)
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    assert min(ref.gap) > 1e-7
    rc, levels, st = _levels(c, precision=rbfd.FP64, engine=2, prune=True)
    assert rc == rbfd.OK and st["sweep_warps_skipped"] > 0
    assert len(levels) == len(ref.idx)
    for l, L in enumerate(levels):
        assert np.array_equal(L.idx, ref.idx[l]), f"level {l}"
    check_replay(c, levels)
    rc, levels, st = _levels(c, precision=rbfd.MIXED, engine=2, prune=True)
    assert rc == rbfd.OK and st["sweep_warps_skipped"] > 0
    check_replay(c, levels)


def test_pruned_sweep_after_newton_start_and_in_2d():
    # default engine: the Newton start hands levels to the list sweep, which
    # builds its block bounds from the lists it receives
    c = synth.airfoil_case(4000, 20, displacement="horns", seed=1, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)
    for precision in (rbfd.MIXED, rbfd.FP64):
        rc0, full, _ = _levels(c, precision=precision, prune=False)
        rc1, pruned, _ = _levels(c, precision=precision, prune=True)
        assert rc0 == rc1
        _same_levels(full, pruned)
    c = _wing()
    rc0, full, _ = _levels(c, prune=False)
    rc1, pruned, st = _levels(c, prune=True, profile=True)
    assert rc0 == rc1
    _same_levels(full, pruned)


def test_round_robin_items_do_not_prune(monkeypatch):
    # beyond the balanced item layout nothing is skipped; the result is the same
    monkeypatch.setenv("RBFD_TEST_SWEEP_ROUND_ROBIN", "1")
    c = synth.wing_case(60, 30, 2, displacement="ridge", seed=1, R=(1.0, 0.3), eps=1e-4, D=1.0, k=4.0,
                        wall_distance=False)
    rc0, a, st = _levels(c, engine=2, prune=True, profile=True)
    assert st["sweep_warps_skipped"] == 0
    monkeypatch.delenv("RBFD_TEST_SWEEP_ROUND_ROBIN")
    rc1, b, _ = _levels(c, engine=2, prune=True)
    assert rc0 == rc1
    _same_levels(a, b)
