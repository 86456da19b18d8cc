"""rbfd_greedy_warm: a time step started from the previous step's controls
and inverse factor (the serving loop's resident meshes run every step this
way).

* A displacement proportional to the previous one leaves E / S0 unchanged, so
  every level keeps its controls: no greedy step runs, and the weights are
  the previous ones scaled, as the oracle's solve of Eq. 9 on the same
  controls gives them; the volume update equals a cold run's within the
  mixed-mode bar.
* A displacement of another shape: each level starts from the previous
  controls and the greedy continues from them where they miss tau_l.  The
  oracle replays the resulting sequence: the restored prefix is given, every
  pick after it must be the oracle's argmax of Eq. 12 up to rounding, every
  level ends below tau_l with its weights solving Eq. 9.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


def _case():
    return synth.airfoil_case(1500, 20, displacement="horns", seed=4, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)


@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_warm_step_with_proportional_displacement_keeps_controls(precision):
    from test_gpu_parity import check_valid, check_volume_own

    c = _case()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision)
    m.greedy_warm()  # the first call is the plain greedy (and keeps the factors)
    first = m.levels()
    assert m.stats()["greedy_steps"] > 0
    dS2 = 1.3 * c.dS
    m.set_displacement(dS2)
    m.greedy_warm()
    st = m.stats()
    second = m.levels()
    assert st["greedy_steps"] == 0 and st["newton_steps"] == 0
    S0 = float(np.sqrt((dS2**2).sum(1)).max())
    rp = oracle.replay(c.xyz_s, dS2, c.R, [L.idx for L in first], n_threads=NT)
    for l, (a, b) in enumerate(zip(first, second)):
        assert np.array_equal(a.idx, b.idx)
        amax = np.abs(b.alpha).max()
        assert np.abs(b.alpha - 1.3 * a.alpha).max() <= 1e-6 * amax
        assert np.abs(b.alpha - rp.alpha[l]).max() <= 1e-6 * amax
        # the oracle's error after the level is below tau, as the GPU's confirm sweep found
        assert np.sqrt(rp.best_key[l][-1]) < b.tau * S0 * (1 + 1e-9)
    c2 = synth.Case(c.name, c.dim, c.xyz_s, dS2, c.xyz_v, c.d_v, c.R, c.eps, c.D, c.k)
    check_valid(c2, second, S0)
    check_volume_own(c2, m, second, precision)
    # the volume update of the warm step against a cold run on the new displacement
    cold = rbfd.Mesh(c.xyz_s, dS2, c.R, c.eps, precision=precision)
    cold.greedy()
    want = cold.deform(c.xyz_v, c.d_v, c.D, c.k).astype(np.float64)
    got = m.deform(c.xyz_v, c.d_v, c.D, c.k).astype(np.float64)
    assert np.abs(got - want).max() <= 1e-5 * S0 + np.abs(want).max() * 2.0**-23
    cold.close()
    m.close()


@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_warm_step_with_new_shape_continues_the_greedy(precision):
    from test_gpu_parity import REPLAY_SLACK, U, check_valid, check_volume_own

    c = _case()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision)
    m.greedy_warm()
    first = m.levels()
    # another ice shape on the same airfoil
    other = synth.airfoil_case(1500, 0, displacement="horns", seed=9, R=(1.0, 0.2), eps=1e-5)
    dS3 = c.dS + 0.5 * other.dS
    m.set_displacement(dS3)
    m.greedy_warm()
    third = m.levels()
    assert m.stats()["greedy_steps"] > 0  # the previous controls do not reach tau for this shape
    S0 = float(np.sqrt((dS3**2).sum(1)).max())
    c3 = synth.Case(c.name, c.dim, c.xyz_s, dS3, c.xyz_v, c.d_v, c.R, c.eps, c.D, c.k)
    check_valid(c3, third, S0)
    check_volume_own(c3, m, third, precision)
    rp = oracle.replay(c.xyz_s, dS3, c.R, [L.idx for L in third], n_threads=NT)
    for l, (a, b) in enumerate(zip(first, third)):
        k0 = len(a.idx)
        assert np.array_equal(b.idx[:k0], a.idx)  # the restored prefix
        n = np.arange(1, len(b.idx) + 1, dtype=np.float64)
        bk, pk = rp.best_key[l], rp.pick_key[l]
        dE = REPLAY_SLACK * n * U * (rp.best_scale[l] + rp.pick_scale[l])
        allow = 2.0 * np.sqrt(bk) * dE + dE * dE
        # picks after the prefix (slot k picks control k): the oracle's argmax up to rounding
        for k in range(k0, len(b.idx)):
            assert bk[k - 1] - pk[k - 1] <= allow[k - 1], f"level {l}: control {k} is not an argmax"
        assert np.sqrt(bk[-1]) < b.tau * S0 * (1 + 1e-9) + dE[-1]
    m.close()
