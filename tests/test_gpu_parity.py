"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Greedy, three checks:
* the selected control sequence equals the oracle's exactly up to the first
  step where the oracle's two largest error keys are within rounding of each
  other (relative gap below TIE); past such a near-tie both answers are
  correct and the runs interpolate different targets;
* replay (every case, split or not): the oracle follows the GPU's own
  sequence and at every step the GPU's pick must be the oracle's argmax of
  Eq. 12 up to the rounding of Eq. 12 itself, and every stop decision must
  agree with the oracle's error against tau_l up to the same rounding;
* validity: each level's weights solve Eq. 9 on the GPU's own controls, each
  level's error is below tau_l, the levels telescope.

Volume: the GPU's update against the oracle's psi-blended update with the
GPU's own controls and weights (always): 1e-10 max|dS| in FP64 mode, 1e-5
max|dS| in mixed mode; and, where the sequences agree in full, against the
oracle's own run (FP64: fp64_volume_tol, mixed: 1e-5 max|dS|).
"""
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1
TIE = 1e-7
U = 2.0**-53
# rounding of Eq. 12: two FP64 (or double-float, |error| below 2^-44 per
# operation) evaluations of E_i = dS_l,i - sum_j alpha_j phi_ij with n terms,
# summed in different orders and with weights from different (backward
# stable) solves, differ by a small multiple of n u (|dS_l,i| + sum_j
# |alpha_j| phi_ij); REPLAY_SLACK is that multiple (measured at most 0.15 on
# the benchmark inputs and the 3D wing's first 400 steps per level)
REPLAY_SLACK = 8.0
C2 = [4.0, -15.0, 20.0, -10.0, 0.0, 1.0]


def phi_np(eta):
    return np.where(eta < 1.0, np.polyval(C2, np.minimum(eta, 1.0)), 0.0)


def run_gpu(c, precision, **kw):
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, **kw)
    rc = m.greedy()
    return m, rc


def check_sequences(ref, levels, strict_full=False):
    """Element-by-element equality of the control sequences.  The first
    mismatch is allowed only at a step where the oracle's two largest keys are
    within TIE of each other (both choices are correct there); from that point
    on the runs interpolate different targets and only validity is checked.
    Returns True if every level matched in full."""
    assert len(levels) == ref.n_levels
    for l, lv in enumerate(levels):
        r_idx, g_idx, gaps = ref.idx[l], lv.idx, ref.step_gap[l]
        n = min(len(r_idx), len(g_idx))
        mism = np.nonzero(r_idx[:n] != g_idx[:n])[0]
        if mism.size:
            k = int(mism[0])
            assert gaps[k] < TIE, f"level {l}: control {k} differs ({g_idx[k]} vs {r_idx[k]}) with gap {gaps[k]:g}"
            assert not strict_full
            return False
        if len(r_idx) != len(g_idx):
            # same controls, different stopping step: the stop test sat on its threshold
            assert not strict_full, f"level {l}: {len(g_idx)} controls vs {len(r_idx)}"
            return False
    return True


def check_replay(c, levels, basis="C2"):
    """The oracle replays the GPU's own sequence (oracle.replay): every pick
    must be the oracle's argmax of Eq. 12 up to the rounding of Eq. 12 (a
    key deficit of at most 2 |E| dE + dE^2, dE = REPLAY_SLACK n u (scale of
    E at the best point + at the pick)), the greedy must have continued only
    while the oracle's largest error was above tau_l S0 and stopped a
    converged level with it below, both up to dE.  Returns the largest
    deficit relative to its allowance."""
    S0 = float(np.sqrt((c.dS**2).sum(1)).max())
    rp = oracle.replay(c.xyz_s, c.dS, c.R, [L.idx for L in levels], basis=basis, n_threads=NT)
    worst = 0.0
    for l, L in enumerate(levels):
        n = np.arange(1, len(L.idx) + 1, dtype=np.float64)
        bk, pk = rp.best_key[l], rp.pick_key[l]
        dE = REPLAY_SLACK * n * U * (rp.best_scale[l] + rp.pick_scale[l])
        allow = 2.0 * np.sqrt(bk) * dE + dE * dE
        d = (bk - pk)[:-1]
        if d.size:
            k = int(np.argmax(d - allow[:-1]))
            assert d[k] <= allow[k], (f"level {l}: control {k + 1} ({L.idx[k + 1]}) has key {pk[k]:.17g}, the "
                                      f"oracle's best is {bk[k]:.17g} (allowed deficit {allow[k]:g})")
            worst = max(worst, float((d / np.maximum(allow[:-1], 1e-300)).max()))
        tauS = L.tau * S0
        e = np.sqrt(bk)
        assert (e[:-1] + dE[:-1] >= tauS).all(), f"level {l}: the greedy went on below tau"
        if L.e_max < L.tau:
            assert e[-1] - dE[-1] < tauS, f"level {l}: stopped with the oracle's error {e[-1] / S0:g} above tau"
    return worst


def gpu_result(levels, S0):
    """The GPU's levels (controls, weights, max |dS_l|) as an oracle result,
    for the oracle's volume update on the GPU's own controls and weights."""
    L = len(levels)
    return oracle.GreedyResult(oracle.OK, [x.idx for x in levels], [x.alpha for x in levels],
                               np.array([x.smax for x in levels]), np.zeros(L), np.zeros(L), None, S0)


def volume_rounding_scale(c, levels, basis="C2"):
    """max over the volume points of sum_l psi(d / D_l) sum_j |alpha_j^(l)| phi_vj:
    two evaluations of Eq. 19 / Eq. 23 that sum in different orders differ by
    a few n u times this (dense products: small cases only)."""
    poly = POLY.get(basis, C2)
    ph = lambda e: np.where(e < 1.0, np.polyval(poly, np.minimum(e, 1.0)), 0.0)
    Dl = oracle.support_distances(np.array([L.smax for L in levels]), c.k, c.D)
    xv = c.xyz_v.astype(np.float64)
    dv = c.d_v.astype(np.float64)
    tot = np.zeros(len(xv))
    for l, L in enumerate(levels):
        if not Dl[l] > 0:
            continue
        w = psi_np(dv / Dl[l])
        tot += w * (ph(cdist(xv, c.xyz_s[L.idx]) / c.R[l]) @ np.abs(L.alpha).sum(1))
    return float(tot.max()) if len(tot) else 0.0


def check_volume_own(c, m, levels, precision, basis="C2"):
    """The GPU's volume update against the oracle's (Eq. 19, Eq. 23) on the
    GPU's own controls and weights: only the evaluation's rounding differs.
    FP64: 1e-10 max|dS|, or the rounding of the sums where the weights are so
    large (ill-conditioned control systems) that it exceeds that: 8 n u times
    the volume_rounding_scale, n the most controls of a level."""
    S0 = float(np.sqrt((c.dS**2).sum(1)).max())
    want = oracle.deform(gpu_result(levels, S0), c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D, basis=basis,
                         n_threads=NT)
    if precision == rbfd.FP64:
        nmax = max(len(L.idx) for L in levels)
        tol = max(1e-10 * S0, 8.0 * nmax * U * volume_rounding_scale(c, levels, basis))
    else:
        tol = 1e-5 * S0
    got = m.deform(c.xyz_v, c.d_v, c.D, c.k).astype(np.float64)
    assert np.abs(got - want).max() <= tol + np.abs(want).max() * 2.0**-24
    got64 = m.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k)
    err64 = np.abs(got64 - want).max()
    assert err64 <= tol, f"volume error {err64 / S0:g} S0 on the GPU's own controls"
    return err64 / S0


def check_valid(c, levels, S0):
    """Validity of any correct answer: each level's weights solve Eq. 9 on its
    own controls, the level error is below tau_l, levels telescope."""
    cur = c.dS.copy()
    L = len(c.R)
    for l, lv in enumerate(levels):
        C = lv.idx
        A = phi_np(cdist(c.xyz_s[C], c.xyz_s[C]) / c.R[l])
        res = A @ lv.alpha - cur[C]
        assert np.abs(res).max() <= 1e-9 * S0 + 1e-12 * np.abs(lv.alpha).max(), f"level {l}: Eq. 9 residual"
        E = cur - phi_np(cdist(c.xyz_s, c.xyz_s[C]) / c.R[l]) @ lv.alpha
        e = np.sqrt((E**2).sum(1)).max() / S0
        tau = c.eps ** ((l + 1) / L)
        assert e < tau * (1 + 1e-9), f"level {l}: error {e} above tau {tau}"
        assert abs(e - lv.e_max) <= 1e-6 * tau + 1e-12, f"level {l}: reported e_max {lv.e_max} vs {e}"
        cur = E


def psi_np(xi):
    xi = np.maximum(xi, 0.0)
    return np.where(xi < 1.0, 1.0 - xi, 0.0)


# cases whose FP64 volume bound against the oracle's own run exceeds
# 1e-10 max|dS| (ill-conditioned control systems; their volumes are held to
# 1e-10 max|dS| on the GPU's own weights instead)
FP64_BOUND_ABOVE_1E10 = {"wing_ridge_2lvl", "C4", "C6"}


def fp64_volume_tol(c, ref, basis_poly=None, name=None):
    """FP64 volume bound against the oracle's own run: the larger of 1e-10
    max|dS| and ten times the disagreement, at the volume points, between two
    backward-stable FP64 solves of Eq. 9 on the oracle's controls (its row
    Cholesky and LAPACK's LU).  Both are correct to about cond(Phi_cc) u; no
    solver can do better.  The bound is printed, and the cases where it
    exceeds 1e-10 max|dS| must be the ones listed in FP64_BOUND_ABOVE_1E10."""
    poly = basis_poly or C2
    ph = lambda e: np.where(e < 1.0, np.polyval(poly, np.minimum(e, 1.0)), 0.0)
    Dl = oracle.support_distances(ref.smax, c.k, c.D)
    xv = c.xyz_v.astype(np.float64)
    dv = c.d_v.astype(np.float64)
    cur = c.dS.copy()
    va = np.zeros_like(xv)
    vb = np.zeros_like(xv)
    for l, R in enumerate(c.R):
        C = ref.idx[l]
        A = ph(cdist(c.xyz_s[C], c.xyz_s[C]) / R)
        a_lu = np.linalg.solve(A, cur[C])
        w = psi_np(dv / Dl[l])[:, None] if Dl[l] > 0 else np.zeros((len(dv), 1))
        P = ph(cdist(xv, c.xyz_s[C]) / R)
        va += w * (P @ ref.alpha[l])
        vb += w * (P @ a_lu)
        cur = cur - ph(cdist(c.xyz_s, c.xyz_s[C]) / R) @ ref.alpha[l]
    tol = max(1e-10 * ref.S0, 10.0 * np.abs(va - vb).max())
    print(f"fp64_volume_tol[{name}] = {tol / ref.S0:.3g} max|dS|")
    if name is not None:
        assert (tol > 1e-10 * ref.S0) == (name in FP64_BOUND_ABOVE_1E10), f"{name}: bound {tol / ref.S0:g} S0"
    return tol


def small_cases():
    return {
        "airfoil_bump_333": synth.airfoil_case(333, 7, displacement="bump", seed=1, R=(0.5,), eps=1e-4, D=2.0, k=0.0),
        "airfoil_horns_2lvl": synth.airfoil_case(600, 9, displacement="horns", seed=2, R=(1.0, 0.2), eps=1e-5,
                                                 D=2.0, k=5.0),
        "airfoil_pitch_2lvl": synth.airfoil_case(500, 9, displacement="pitch_heave", seed=0, R=(1.0, 0.2),
                                                 eps=1e-5, D=2.0, k=5.0),
        "wing_ridge_2lvl": synth.wing_case(40, 15, 6, displacement="ridge", seed=3, R=(1.5, 0.4), eps=1e-3,
                                           D=1.0, k=4.0),
        "wing_sinusoid": synth.wing_case(30, 12, 5, displacement="sinusoid", seed=0, R=(1.5,), eps=1e-3,
                                         D=1.0, k=4.0),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_greedy_and_deform_parity(name, precision):
    c = CASES[name]
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    m, rc = run_gpu(c, precision)
    levels = m.levels()
    full = check_sequences(ref, levels)
    check_replay(c, levels)
    check_valid(c, levels, ref.S0)
    check_volume_own(c, m, levels, precision)
    for l, lv in enumerate(levels):
        # level 0 targets are the inputs; later levels' targets carry the
        # rounding of Eq. 12 (about n u sum|alpha phi|, below 1e-9 S0 here).
        # After a split at a near-tie the runs interpolate different control
        # sets and only validity (check_valid) applies to the later levels.
        if l == 0:
            assert abs(lv.smax - ref.smax[0]) <= 1e-15 * ref.S0
        elif full:
            assert abs(lv.smax - ref.smax[l]) <= 1e-9 * ref.S0
        if full and l == 0:
            amax = np.abs(ref.alpha[l]).max()
            assert np.abs(lv.alpha - ref.alpha[l]).max() <= 1e-6 * amax
    if not full:
        return
    dv_ref = oracle.deform(ref, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D, n_threads=NT)
    dv = m.deform(c.xyz_v, c.d_v, c.D, c.k)
    tol = fp64_volume_tol(c, ref, name=name) if precision == rbfd.FP64 else 1e-5 * ref.S0
    err = np.abs(dv.astype(np.float64) - dv_ref).max()
    # float32 output: add half an ulp of the largest displacement
    assert err <= tol + np.abs(dv_ref).max() * 2.0**-24, f"volume error {err / ref.S0:g} S0"
    dv64 = m.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k)
    assert np.abs(dv64 - dv_ref).max() <= tol
    st = m.stats()
    assert 0 < st["pairs_useful"] <= st["pairs_visited"]
    m.close()


# Table 1 multiplied out (C4 = (1-e)^6 (35/3 e^2 + 6 e + 1), C6 = (1-e)^8 (32 e^3 + 25 e^2 + 8 e + 1))
POLY = {
    "C0": [1.0, -2.0, 1.0],
    "C4": list(np.polymul(np.poly1d([-1.0, 1.0]) ** 6, [35.0 / 3.0, 6.0, 1.0]).coeffs),
    "C6": list(np.polymul(np.poly1d([-1.0, 1.0]) ** 8, [32.0, 25.0, 8.0, 1.0]).coeffs),
}


@pytest.mark.parametrize("basis", ["C0", "C4", "C6"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_other_wendland_bases(basis, precision):
    """Wendland C0, C4, C6 (Table 1) on an airfoil with a 2D ice horn, in both
    precisions (a mesh with C4 or C6 runs in FP64 when mixed is asked: its
    weights reach about 1e9 max|dS| here, beyond what the double-float sweeps
    resolve): sequence (up to near-ties), replay, validity, volume on the
    GPU's own weights, and against the oracle's own run where the sequences
    agree in full."""
    c = synth.airfoil_case(256, 6, displacement="bump", seed=0, R=(0.6,), eps=1e-3, D=2.0, k=0.0)
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, basis=basis, n_threads=NT)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, basis=oracle.BASIS[basis])
    m.greedy()
    levels = m.levels()
    full = check_sequences(ref, levels)
    check_replay(c, levels, basis=basis)
    check_volume_own(c, m, levels, precision, basis=basis)
    if full:
        dv_ref = oracle.deform(ref, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D, basis=basis, n_threads=NT)
        dv = m.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k)
        # against the oracle's own weights no result can be closer than two
        # backward-stable FP64 solves are to each other (fp64_volume_tol)
        tol = fp64_volume_tol(c, ref, POLY[basis], name=basis)
        if precision == rbfd.MIXED:
            tol = max(tol, 1e-5 * ref.S0)
        assert np.abs(dv - dv_ref).max() <= tol


@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_first_point_argmax_rule(precision):
    c = synth.airfoil_case(300, 5, displacement="horns", seed=5, R=(1.0, 0.2), eps=1e-4, D=2.0, k=5.0)
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, first_rule=1, n_threads=NT)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, first_point=1)
    m.greedy()
    check_sequences(ref, m.levels())


def test_naca0012_400_full_fp64_and_mixed():
    c = synth.make_config("naca0012_400s_40kv_bump")
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    dv_ref = oracle.deform(ref, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D, n_threads=NT)
    for precision in (rbfd.FP64, rbfd.MIXED):
        m, _ = run_gpu(c, precision)
        assert check_sequences(ref, m.levels(), strict_full=True)
        check_replay(c, m.levels())
        dv = m.deform(c.xyz_v, c.d_v, c.D, c.k).astype(np.float64)
        tol = fp64_volume_tol(c, ref, name=c.name) if precision == rbfd.FP64 else 1e-5 * ref.S0
        assert np.abs(dv - dv_ref).max() <= tol + np.abs(dv_ref).max() * 2.0**-24


@pytest.mark.parametrize("disp", ["horns", "pitch_heave"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_naca0012_4000_1m_full(disp, precision):
    """The 4,000-point / 1M-point airfoil configurations, both cases, both
    precisions: the control sequence must equal the oracle's in full (the
    oracle's smallest top-2 gap on these inputs, 1.8e-8, is far above the
    rounding of Eq. 12 in either precision), the replay must pass, and the
    volume must meet the FP64 (1e-10 max|dS|) or mixed (1e-5 max|dS|) bar
    against the oracle's own run."""
    c = synth.make_config(f"naca0012_4000s_1mv_{disp}")
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    m, _ = run_gpu(c, precision)
    levels = m.levels()
    assert check_sequences(ref, levels, strict_full=True)
    check_replay(c, levels)
    check_valid(c, levels, ref.S0)
    dv_ref = oracle.deform(ref, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D, n_threads=NT)
    if precision == rbfd.FP64:
        tol = fp64_volume_tol(c, ref, name=c.name)
        assert tol == 1e-10 * ref.S0
        dv = m.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k)
        assert np.abs(dv - dv_ref).max() <= tol
    else:
        dv = m.deform(c.xyz_v, c.d_v, c.D, c.k).astype(np.float64)
        assert np.abs(dv - dv_ref).max() <= 1e-5 * ref.S0 + np.abs(dv_ref).max() * 2.0**-24


def test_mixed_batched_matches_fp64_single():
    """The mixed-precision batched form (rbfd_run_jobs: both 4,000-point cases
    and the 400-point case in one call) against the plain FP64 single-request
    form (rbfd_create + rbfd_greedy + rbfd_deform_f64) on the same GPU: the
    volume displacements agree within 1e-5 max|dS|."""
    names = ["naca0012_4000s_1mv_horns", "naca0012_4000s_1mv_pitch_heave", "naca0012_400s_40kv_bump"]
    cases = [synth.make_config(n) for n in names]
    want = []
    for c in cases:
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=rbfd.FP64)
        m.greedy()
        want.append(m.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k))
        m.close()
    jobs = [dict(xyz_s=c.xyz_s, dS=c.dS, R=c.R, eps=c.eps, precision=rbfd.MIXED, xyz_v=c.xyz_v, d_v=c.d_v,
                 D=c.D, k=c.k, out=np.empty((c.n_v, c.dim), np.float32)) for c in cases]
    ms, rc = rbfd.run_jobs(jobs)
    assert rc == rbfd.OK
    for c, j, w, m in zip(cases, jobs, want, ms):
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        err = np.abs(j["out"].astype(np.float64) - w).max()
        assert err <= 1e-5 * S0 + np.abs(w).max() * 2.0**-24, f"{c.name}: {err / S0:g} max|dS|"
        m.close()


# ---------------------------------------------------------------- edge cases


def test_single_surface_point():
    xyz = np.array([[0.3, 0.1]])
    dS = np.array([[0.01, -0.02]])
    m = rbfd.Mesh(xyz, dS, [0.5], 1e-3, precision=rbfd.MIXED)
    m.greedy()
    lv = m.levels()
    assert len(lv) == 1 and lv[0].idx.tolist() == [0]
    np.testing.assert_allclose(lv[0].alpha, dS, rtol=0, atol=1e-15)
    xv = np.array([[0.3, 0.1], [0.3, 0.35], [5.0, 5.0]], dtype=np.float32)
    dv = np.array([0.0, 0.25, 7.0], dtype=np.float32)
    out = m.deform(xv, dv, D=1.0, k=0.0)
    ref = oracle.greedy(xyz, dS, [0.5], 1e-3)
    want = oracle.deform(ref, xyz, [0.5], xv, dv, 0.0, 1.0)
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-7)


def test_zero_displacement_gives_zero_levels():
    c = synth.airfoil_case(200, 4, displacement="bump", seed=0)
    m = rbfd.Mesh(c.xyz_s, np.zeros_like(c.dS), c.R, c.eps)
    m.greedy()
    assert m.num_levels() == 0
    out = m.deform(c.xyz_v, c.d_v, 2.0, 0.0)
    assert not out.any()


def test_empty_and_out_of_reach_volumes():
    c = synth.airfoil_case(200, 4, displacement="bump", seed=0)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    m.greedy()
    out = m.deform(np.zeros((0, 2), np.float32), np.zeros(0, np.float32), 2.0, 0.0)
    assert out.shape == (0, 2)
    far = np.full((1000, 2), 50.0, np.float32)
    out = m.deform(far, np.full(1000, 30.0, np.float32), 2.0, 0.0)
    assert not out.any()


def test_cap_reports_not_converged():
    c = synth.airfoil_case(300, 0, displacement="bump", seed=0, eps=1e-8)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, nc_cap=7)
    rc = m.greedy()
    assert rc == rbfd.ENOTCONV
    lv = m.levels()
    assert len(lv[0].idx) == 7
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, nc_cap=7)
    assert ref.status == oracle.ENOTCONV
    assert np.array_equal(ref.idx[0], lv[0].idx)


def test_duplicate_point_is_singular():
    c = synth.airfoil_case(64, 0, displacement="bump", seed=0)
    xyz = np.concatenate([c.xyz_s, c.xyz_s[5:6]])
    dS = np.concatenate([c.dS, c.dS[5:6] + 0.01])
    m = rbfd.Mesh(xyz, dS, c.R, 1e-12, precision=rbfd.FP64)
    with pytest.raises(rbfd.RbfdError) as ei:
        m.greedy(allow_not_converged=False)
    assert ei.value.status == rbfd.ESINGULAR


def test_invalid_arguments():
    xyz = np.zeros((4, 2))
    for kw in (dict(R=[0.0], eps=1e-3), dict(R=[1.0], eps=0.0), dict(R=[1.0], eps=2.0)):
        with pytest.raises(rbfd.RbfdError) as ei:
            rbfd.Mesh(xyz, xyz, kw["R"], kw["eps"])
        assert ei.value.status == rbfd.EINVAL
    with pytest.raises(rbfd.RbfdError):
        rbfd.Mesh(np.zeros((4, 4)), np.zeros((4, 4)), [1.0], 1e-3)


def test_deform_before_greedy_is_a_state_error():
    c = synth.airfoil_case(100, 2, displacement="bump", seed=0)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    with pytest.raises(rbfd.RbfdError) as ei:
        m.deform(c.xyz_v, c.d_v, 2.0, 0.0)
    assert ei.value.status == rbfd.ESTATE


def test_device_pointers_match_host_pointers():
    torch = pytest.importorskip("torch")
    c = synth.airfoil_case(500, 8, displacement="horns", seed=7, R=(1.0, 0.2), eps=1e-4, D=2.0, k=5.0)
    mh = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    mh.greedy()
    outh = mh.deform(c.xyz_v, c.d_v, c.D, c.k)
    dev = torch.device("cuda:0")
    md = rbfd.Mesh(torch.from_numpy(c.xyz_s).to(dev), torch.from_numpy(c.dS).to(dev), c.R, c.eps)
    md.greedy()
    for a, b in zip(mh.levels(), md.levels()):
        assert np.array_equal(a.idx, b.idx) and np.array_equal(a.alpha, b.alpha)
    outd = md.deform(torch.from_numpy(c.xyz_v).to(dev), torch.from_numpy(c.d_v).to(dev), c.D, c.k)
    assert np.array_equal(outd.cpu().numpy(), outh)


def test_repeat_greedy_is_deterministic():
    c = CASES["airfoil_horns_2lvl"]
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    m.greedy()
    a = m.levels()
    o1 = m.deform(c.xyz_v, c.d_v, c.D, c.k)
    m.greedy()
    b = m.levels()
    o2 = m.deform(c.xyz_v, c.d_v, c.D, c.k)
    for x, y in zip(a, b):
        assert np.array_equal(x.idx, y.idx) and np.array_equal(x.alpha, y.alpha)
    assert np.array_equal(o1, o2)


# ---------------------------------------------------------------- engines


@pytest.mark.parametrize("name", ["airfoil_horns_2lvl", "wing_ridge_2lvl"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_persistent_engine_matches_step_engine(name, precision):
    """The list sweep as one persistent launch per level (engine 2) and as
    separate launches per step (engine 1) run the same arithmetic: the same
    controls, on grids of any size; the default engine (Newton start, engine
    0) on those grid sizes follows the oracle up to near-ties and is valid."""
    c = CASES[name]
    a = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=2)
    a.greedy()
    b = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=1)
    b.greedy()
    for x, y in zip(a.levels(), b.levels()):
        assert np.array_equal(x.idx, y.idx)
        assert np.abs(x.alpha - y.alpha).max() <= 1e-6 * max(np.abs(y.alpha).max(), 1e-300)
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    S0 = np.sqrt((c.dS**2).sum(1)).max()
    for ctas in (1, 7, 300):
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=2, grid_ctas=ctas)
        m.greedy()
        for x, y in zip(m.levels(), b.levels()):
            assert np.array_equal(x.idx, y.idx)
        m0 = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=0, grid_ctas=ctas)
        m0.greedy()
        check_sequences(ref, m0.levels())
        check_valid(c, m0.levels(), S0)


@pytest.mark.parametrize("name", ["airfoil_horns_2lvl", "wing_ridge_2lvl"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_sweep_item_assignment_does_not_change_results(name, precision, monkeypatch):
    """The persistent sweep hands its items (chunks of the point blocks'
    control lists) out from a counter as blocks come free; on meshes with more
    point blocks than its shared-memory prefix holds it takes them round-robin
    instead (test hook: round-robin at any size).  A chunk's partial sums do
    not depend on the block that computes them and are reduced in chunk
    order, so both give the same controls and weights bit for bit."""
    c = CASES[name]
    runs = []
    for rr in ("0", "1"):
        monkeypatch.setenv("RBFD_TEST_SWEEP_ROUND_ROBIN", rr)
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=2, grid_ctas=7)
        m.greedy()
        runs.append(m.levels())
    monkeypatch.delenv("RBFD_TEST_SWEEP_ROUND_ROBIN")
    assert len(runs[0]) == len(runs[1])
    for x, y in zip(*runs):
        assert np.array_equal(x.idx, y.idx)
        assert np.array_equal(x.alpha, y.alpha)


@pytest.mark.parametrize("name", ["airfoil_horns_2lvl", "wing_ridge_2lvl", "airfoil_bump_333"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_newton_start_matches_list_sweep(name, precision, monkeypatch):
    """Engine 0 starts every level in the Newton basis (E updated by one basis
    function per step) and hands over to the list sweep; engine 2 runs the
    list sweep alone.  Both follow the oracle's controls up to near-ties (and
    agree with each other where both follow it in full); so does a forced
    hand-over after 8 Newton steps (V capped at 8 columns)."""
    c = CASES[name]
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    S0 = np.sqrt((c.dS**2).sum(1)).max()
    a = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=0)
    a.greedy()
    assert a.stats()["newton_steps"] > 0
    full_a = check_sequences(ref, a.levels())
    check_valid(c, a.levels(), S0)
    b = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=2)
    b.greedy()
    assert b.stats()["newton_steps"] == 0
    full_b = check_sequences(ref, b.levels())
    if full_a and full_b:
        for x, y in zip(a.levels(), b.levels()):
            assert np.array_equal(x.idx, y.idx)
            assert np.abs(x.alpha - y.alpha).max() <= 1e-6 * max(np.abs(y.alpha).max(), 1e-300)
    monkeypatch.setenv("RBFD_NEWTON_COLS", "8")
    h = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, engine=0)
    h.greedy()
    st = h.stats()
    assert 0 < st["newton_steps"] <= 7 * len(c.R)
    check_sequences(ref, h.levels())
    check_valid(c, h.levels(), S0)


def test_barrier_wait_bound_returns_timeout(monkeypatch):
    """A block that never arrives at the grid barrier (test hook) makes the
    other blocks' bounded waits run out: the launch ends and rbfd_greedy
    reports RBFD_ETIMEOUT; the next call on the same mesh works."""
    c = CASES["airfoil_bump_333"]
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=0, grid_ctas=8)
    monkeypatch.setenv("RBFD_TEST_BARRIER_POLLS", "2000")
    monkeypatch.setenv("RBFD_TEST_SKIP_ARRIVAL", "1")
    with pytest.raises(rbfd.RbfdError) as ei:
        m.greedy(allow_not_converged=False)
    assert ei.value.status == rbfd.ETIMEOUT
    monkeypatch.delenv("RBFD_TEST_BARRIER_POLLS")
    monkeypatch.delenv("RBFD_TEST_SKIP_ARRIVAL")
    m.greedy()
    ref = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=NT)
    check_sequences(ref, m.levels(), strict_full=True)


# ---------------------------------------------------------------- batches


def test_staged_volume_with_device_arrays_matches_plain_calls():
    """greedy_deform_batch on device tensors prepares each volume on a second
    stream while the greedy runs: the outputs equal rbfd_greedy + rbfd_deform
    bit for bit, also when a batch call reuses the meshes' buffers, and the
    volume arrays may be rewritten after the call."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    names = ["airfoil_horns_2lvl", "wing_ridge_2lvl", "airfoil_bump_333"]
    cases = [CASES[n] for n in names]
    want = []
    for c in cases:
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
        m.greedy()
        want.append(m.deform(c.xyz_v, c.d_v, c.D, c.k))
        m.close()
    for rep in range(2):
        ms = [rbfd.Mesh(t(c.xyz_s), t(c.dS), c.R, c.eps) for c in cases]
        xv = [t(c.xyz_v) for c in cases]
        dv = [t(c.d_v) for c in cases]
        outs = [torch.empty((c.n_v, c.dim), dtype=torch.float32, device=dev) for c in cases]
        rbfd.greedy_deform_batch(ms, xv, dv, [c.D for c in cases], [c.k for c in cases], outs)
        torch.cuda.synchronize()
        for x in xv:
            x.zero_()  # the call has finished with its inputs
        for w, o in zip(want, outs):
            assert np.array_equal(o.cpu().numpy(), w)
        # the same meshes deformed again by a plain call: the staged buffers are not reused
        for c, m, w in zip(cases, ms, want):
            o2 = m.deform(t(c.xyz_v), t(c.d_v), c.D, c.k)
            assert np.array_equal(o2.cpu().numpy(), w)
            m.close()


def test_run_jobs_matches_separate_calls():
    """rbfd_run_jobs (create, greedy and volume update per job, side by side,
    in one call) gives the levels and volumes of the separate calls bit for
    bit, on host arrays and on device tensors; a bad job fails alone."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    names = ["airfoil_horns_2lvl", "wing_ridge_2lvl", "airfoil_pitch_2lvl"]
    cases = [CASES[n] for n in names]
    want = []
    for c in cases:
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
        m.greedy()
        want.append((m.levels(), m.deform(c.xyz_v, c.d_v, c.D, c.k)))
        m.close()
    for on_dev in (False, True):
        conv = t if on_dev else (lambda a: a)
        jobs = [dict(xyz_s=conv(c.xyz_s), dS=conv(c.dS), R=c.R, eps=c.eps, xyz_v=conv(c.xyz_v), d_v=conv(c.d_v),
                     D=c.D, k=c.k,
                     out=(torch.empty((c.n_v, c.dim), dtype=torch.float32, device=dev) if on_dev
                          else np.empty((c.n_v, c.dim), np.float32))) for c in cases]
        ms, rc = rbfd.run_jobs(jobs)
        assert rc == 0
        for j, m, (lv, w) in zip(jobs, ms, want):
            out = j["out"].cpu().numpy() if on_dev else j["out"]
            assert np.array_equal(out, w)
            for x, y in zip(m.levels(), lv):
                assert np.array_equal(x.idx, y.idx) and np.array_equal(x.alpha, y.alpha)
            assert m.stats()["greedy_steps"] > 0
            m.close()
    # one FP64 job with the wall distances computed on the device, beside a mixed one
    c0, c1 = cases[0], cases[1]
    m0 = rbfd.Mesh(c0.xyz_s, c0.dS, c0.R, c0.eps, precision=rbfd.FP64)
    m0.greedy()
    w0 = m0.deform(c0.xyz_v, None, c0.D, c0.k)
    m0.close()
    jobs = [dict(xyz_s=c0.xyz_s, dS=c0.dS, R=c0.R, eps=c0.eps, precision=rbfd.FP64, xyz_v=c0.xyz_v, d_v=None,
                 D=c0.D, k=c0.k, out=np.empty((c0.n_v, c0.dim), np.float32)),
            dict(xyz_s=c1.xyz_s, dS=c1.dS, R=c1.R, eps=c1.eps, xyz_v=c1.xyz_v, d_v=c1.d_v, D=c1.D, k=c1.k,
                 out=np.empty((c1.n_v, c1.dim), np.float32))]
    ms, rc = rbfd.run_jobs(jobs)
    assert rc == 0 and np.array_equal(jobs[0]["out"], w0) and np.array_equal(jobs[1]["out"], want[1][1])
    for m in ms:
        m.close()
    # a job with an invalid radius: its mesh is not created, the others run
    jobs = [dict(xyz_s=c0.xyz_s, dS=c0.dS, R=c0.R, eps=c0.eps, xyz_v=c0.xyz_v, d_v=c0.d_v, D=c0.D, k=c0.k,
                 out=np.empty((c0.n_v, c0.dim), np.float32)),
            dict(xyz_s=c1.xyz_s, dS=c1.dS, R=(-1.0,), eps=c1.eps, xyz_v=c1.xyz_v, d_v=c1.d_v, D=c1.D, k=c1.k,
                 out=np.empty((c1.n_v, c1.dim), np.float32))]
    with pytest.raises(rbfd.RbfdError) as ei:
        rbfd.run_jobs(jobs)
    assert ei.value.status == rbfd.EINVAL and "mesh 1" in str(ei.value)


def test_run_jobs_device_radii_and_capped_job():
    """In rbfd_run_jobs the volume update is queued behind the greedy without a
    host wait: D_l = min(k max|dS_l|, D) (or D when k = 0) is formed on the
    device from the levels' scalars.  Every rule gives the volumes of the
    separate calls bit for bit: k > 0 with D capping some levels, k > 0 with
    no cap (D = 0), k = 0 (D at every level), and a job whose greedy stops at
    its control cap (ENOTCONV reported, its levels still used)."""
    c = CASES["airfoil_horns_2lvl"]
    c2 = CASES["airfoil_pitch_2lvl"]
    S0 = float(np.sqrt((c.dS**2).sum(1)).max())
    variants = [dict(case=c, D=c.D, k=c.k), dict(case=c, D=0.0, k=3.0),
                dict(case=c2, D=0.25, k=0.0), dict(case=c, D=3.0 * S0, k=1.5, nc_cap=7)]
    want = []
    for v in variants:
        cc = v["case"]
        m = rbfd.Mesh(cc.xyz_s, cc.dS, cc.R, cc.eps, nc_cap=v.get("nc_cap", 0))
        rc = m.greedy()
        want.append((rc, m.levels(), m.deform(cc.xyz_v, cc.d_v, v["D"], v["k"])))
        m.close()
    assert want[3][0] == rbfd.ENOTCONV
    jobs = [dict(xyz_s=v["case"].xyz_s, dS=v["case"].dS, R=v["case"].R, eps=v["case"].eps,
                 nc_cap=v.get("nc_cap", 0), xyz_v=v["case"].xyz_v, d_v=v["case"].d_v, D=v["D"], k=v["k"],
                 out=np.empty((v["case"].n_v, v["case"].dim), np.float32)) for v in variants]
    ms, rc = rbfd.run_jobs(jobs)
    assert rc == rbfd.ENOTCONV
    for j, m, (rc1, lv, w) in zip(jobs, ms, want):
        assert np.array_equal(j["out"], w)
        for x, y in zip(m.levels(), lv):
            assert np.array_equal(x.idx, y.idx) and np.array_equal(x.alpha, y.alpha)
        m.close()


def test_batch_relaunches_match_single_meshes(monkeypatch):
    """In a batch, a mesh's persistent launch ends every few steps while other
    meshes still run and is relaunched on the share of the blocks the
    finished meshes left (test hook: every 7 steps).  The relaunched level
    goes on from the state the launch left: the same controls as each mesh
    alone, the weights within the rounding of a different block count."""
    monkeypatch.setenv("RBFD_TEST_YIELD_STEPS", "7")
    names = ["airfoil_horns_2lvl", "wing_ridge_2lvl", "airfoil_pitch_2lvl"]
    cases = [CASES[n] for n in names]
    single = []
    for c in cases:
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=2)
        m.greedy()
        single.append(m.levels())
        m.close()
    ms = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, engine=2, profile=True) for c in cases]
    rbfd.greedy_batch(ms)
    launches = [m.stats()["persist_launches"] for m in ms]
    for m, lv1 in zip(ms, single):
        for x, y in zip(m.levels(), lv1):
            assert np.array_equal(x.idx, y.idx)
            assert np.abs(x.alpha - y.alpha).max() <= 1e-6 * max(np.abs(y.alpha).max(), 1e-300)
        m.close()
    # (the first meshes to finish leave the others relaunching)
    assert max(launches) > max(len(lv) for lv in single)


@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_batch_matches_single_meshes(precision):
    names = ["airfoil_horns_2lvl", "wing_ridge_2lvl", "airfoil_pitch_2lvl", "airfoil_bump_333"]
    cases = [CASES[n] for n in names]
    single = []
    for c in cases:
        m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision)
        m.greedy()
        single.append((m.levels(), m.deform(c.xyz_v, c.d_v, c.D, c.k)))
        m.close()
    ms = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision) for c in cases]
    rbfd.greedy_batch(ms)
    outs = [np.empty((c.n_v, c.dim), np.float32) for c in cases]
    rbfd.deform_batch(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                      [c.k for c in cases], outs)
    for c, m, (lv1, out1), out2 in zip(cases, ms, single, outs):
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        for x, y in zip(m.levels(), lv1):
            assert np.array_equal(x.idx, y.idx)
            assert np.abs(x.alpha - y.alpha).max() <= 1e-6 * max(np.abs(y.alpha).max(), 1e-300)
        assert np.abs(out2.astype(np.float64) - out1).max() <= 1e-5 * S0 + np.abs(out1).max() * 2.0**-24
        m.close()
    # greedy then volume update per mesh, meshes side by side: the same as
    # the two batch calls one after the other, bit for bit
    ms2 = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision) for c in cases]
    outs2 = [np.empty((c.n_v, c.dim), np.float32) for c in cases]
    rbfd.greedy_deform_batch(ms2, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                             [c.k for c in cases], outs2)
    for c, m, o1, o2 in zip(cases, ms2, outs, outs2):
        assert np.array_equal(o1, o2)
    # with the wall distances computed on the device
    outs3 = [np.empty((c.n_v, c.dim), np.float32) for c in cases]
    rbfd.greedy_deform_batch(ms2, [c.xyz_v for c in cases], None, [c.D for c in cases], [c.k for c in cases], outs3)
    for c, m, o1, o3 in zip(cases, ms2, outs, outs3):
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        assert np.abs(o3.astype(np.float64) - o1).max() <= 1e-5 * S0
        m.close()
