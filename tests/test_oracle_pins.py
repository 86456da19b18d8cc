"""Pins of the FP64 oracle against facts outside the oracle itself.

Each pin compares the oracle with something it does not share code with:
exact values of the paper's Table 1 (tests/golden/wendland_table1.txt), the
algebraically expanded polynomial of Eq. 2, library routines (numpy / scipy
Cholesky, dense solve, eigenvalues, distance matrices), and invariants the
equations imply (exact interpolation at the controls, telescoping over levels,
zero displacement where psi = 0, the dense RBF solve of Eq. 9 / Eq. 10 as the
limit of the greedy).

The same pin functions run against deliberately broken builds of the oracle
source at the end of this file, to show that each plausible mistake (a
dropped term, a wrong sign, a transposed index, a skipped blend) fails at
least one of them.
"""
import os
import shutil
from fractions import Fraction

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2107_13887_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wendland_table1.txt")

# (1 - e)^4 (4 e + 1) multiplied out: 1 - 10 e^2 + 20 e^3 - 15 e^4 + 4 e^5
C2_EXPANDED = [4.0, -15.0, 20.0, -10.0, 0.0, 1.0]


def phi_expanded(eta):
    eta = np.asarray(eta, dtype=np.float64)
    return np.where(eta < 1.0, np.polyval(C2_EXPANDED, np.minimum(eta, 1.0)), 0.0)


def psi_ref(xi):
    xi = np.maximum(np.asarray(xi, dtype=np.float64), 0.0)
    return np.where(xi < 1.0, 1.0 - xi, 0.0)


def tiny_airfoil(n=48, displacement="bump", seed=0, R=(0.5,), eps=1e-6, layers=6):
    return synth.airfoil_case(n, layers, displacement=displacement, seed=seed, R=R, eps=eps, D=2.0, k=0.0)


def tiny_airfoil_k5():
    c = tiny_airfoil(n=60, displacement="horns", R=(1.0, 0.2), eps=1e-6, layers=8)
    c.k = 5.0
    return c


def tiny_wing(seed=0, R=(1.5, 0.4), eps=1e-4):
    return synth.wing_case(16, 6, 3, displacement="ridge", seed=seed, R=R, eps=eps, D=1.0, k=4.0)


# ------------------------------------------------------------------ pins
# Each returns a list of failure strings (empty = pinned).


def pin_table1(o):
    bad = []
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        name, e, v, _ = line.split()
        eta = float(Fraction(e))
        want = float(Fraction(v))
        got = float(o.phi([eta], basis=name)[0])
        if abs(got - want) > 4e-16:
            bad.append(f"Table 1 {name} at eta={e}: {got!r} != {want!r}")
    return bad


def pin_phi_expanded(o):
    eta = np.linspace(0.0, 1.3, 1001)
    got = o.phi(eta)
    err = np.abs(got - phi_expanded(eta)).max()
    return [] if err < 1e-14 else [f"C2 differs from its expanded polynomial by {err:g}"]


def pin_phi_smoothness(o):
    # C2 (Eq. 2) is twice continuously differentiable with phi(0) = 1, phi'(0) = 0
    # and phi, phi', phi'' vanishing at eta = 1
    h = 1e-4
    f = lambda e: float(o.phi([e])[0])
    bad = []
    if abs(f(0.0) - 1.0) > 0:
        bad.append("phi(0) != 1")
    if abs((f(h) - f(0.0)) / h) > 1e-3:
        bad.append("phi'(0) != 0")
    d1 = (f(1.0) - f(1.0 - h)) / h
    d2 = (f(1.0) - 2 * f(1.0 - h) + f(1.0 - 2 * h)) / h**2
    if abs(d1) > 1e-6 or abs(d2) > 1e-3:
        bad.append(f"phi not C2 at eta=1 (d1={d1:g}, d2={d2:g})")
    return bad


def pin_psi(o):
    xi = np.array([-0.5, 0.0, 0.25, 0.5, 0.999, 1.0, 1.5, 7.0])
    err = np.abs(o.psi(xi) - psi_ref(xi)).max()
    return [] if err == 0 else [f"psi differs from Section 4 by {err:g}"]


def pin_cholesky(o):
    rng = np.random.default_rng(1)
    M = rng.standard_normal((12, 12))
    A = M @ M.T + 12 * np.eye(12)
    L = o.cholesky(A)
    bad = []
    if L is None:
        return ["SPD matrix reported not positive definite"]
    if np.abs(L - np.linalg.cholesky(A)).max() > 1e-12:
        bad.append("Cholesky factor differs from numpy.linalg.cholesky")
    B = rng.standard_normal((12, 3))
    X = o.chol_solve(L, B)
    if np.abs(X - np.linalg.solve(A, B)).max() > 1e-12:
        bad.append("Cholesky solve differs from numpy.linalg.solve")
    Aneg = A.copy()
    Aneg[5, 5] = -1.0
    if o.cholesky(Aneg) is not None:
        bad.append("indefinite matrix accepted")
    return bad


def pin_eval_dense(o):
    rng = np.random.default_rng(2)
    bad = []
    for dim in (2, 3):
        xc = rng.uniform(-1, 1, (40, dim))
        al = rng.standard_normal((40, dim))
        xp = rng.uniform(-1, 1, (70, dim))
        R = 0.9
        want = phi_expanded(cdist(xp, xc) / R) @ al
        got = o.evaluate(xc, al, xp, R)
        if np.abs(got - want).max() > 1e-12:
            bad.append(f"evaluation ({dim}D) differs from the dense product")
    return bad


def pin_spd(o):
    # Wendland's theorem: C2 (and C4, C6) are positive definite in up to 3 dimensions
    rng = np.random.default_rng(3)
    bad = []
    for dim in (2, 3):
        x = rng.uniform(0, 1, (30, dim))
        A = phi_expanded(cdist(x, x) / 0.8)
        lam = np.linalg.eigvalsh(A)
        if lam.min() <= 0:
            bad.append(f"{dim}D Phi_cc not SPD (lambda_min={lam.min():g})")
        if o.cholesky(A) is None:
            bad.append(f"{dim}D Phi_cc rejected by the oracle Cholesky")
    return bad


U = 2.0**-53  # unit roundoff of IEEE double


def _level_targets(case, res):
    """dS_l for every level, recomputed from the oracle's (C, alpha) by dense
    products, with an absolute bound on how far two summation orders of those
    products can drift apart (8 n u max_i sum_j |alpha_j| phi_ij, summed over
    the levels so far)."""
    cur = case.dS.copy()
    out, bounds = [], []
    acc = 0.0
    for l, R in enumerate(case.R):
        out.append(cur.copy())
        bounds.append(acc)
        C = res.idx[l]
        P = phi_expanded(cdist(case.xyz_s, case.xyz_s[C]) / R)
        cur = cur - P @ res.alpha[l]
        acc += 8 * max(len(C), 1) * U * ((P @ np.abs(res.alpha[l])).max() + np.abs(out[-1]).max())
    return out, cur, bounds, acc


def pin_greedy(o, case, first_rule=0):
    """alpha solves Eq. 9 on the controls, each added control is the brute-force
    argmax of Eq. 12, every level meets its tolerance, E is exact at the controls,
    and the levels telescope to dS - E_final."""
    res = o.greedy(case.xyz_s, case.dS, case.R, case.eps, first_rule=first_rule)
    bad = []
    S0 = float(np.sqrt((case.dS**2).sum(1)).max())
    if abs(res.S0 - S0) > 0:
        bad.append("S0 mismatch")
    targets, final, bounds, final_bound = _level_targets(case, res)
    L = len(case.R)
    for l, R in enumerate(case.R):
        C = list(res.idx[l])
        tgt = targets[l]
        if first_rule == 0 and C[0] != 0:
            bad.append(f"level {l}: first control {C[0]} != 0")
        if abs(res.smax[l] - np.sqrt((tgt**2).sum(1)).max()) > 1e-14 * S0 + 2 * bounds[l]:
            bad.append(f"level {l}: smax mismatch")
        # alpha against a library solve of Phi_cc alpha = dS_l(C)
        A = phi_expanded(cdist(case.xyz_s[C], case.xyz_s[C]) / R)
        a_ref = np.linalg.solve(A, tgt[C])
        scale = np.abs(a_ref).max() + S0
        if np.abs(res.alpha[l] - a_ref).max() > 1e-7 * scale:
            bad.append(f"level {l}: alpha differs from numpy.linalg.solve")
        # brute-force argmax at every step
        for k in range(1, len(C)):
            Ck = C[:k]
            Ak = phi_expanded(cdist(case.xyz_s[Ck], case.xyz_s[Ck]) / R)
            ak = np.linalg.solve(Ak, tgt[Ck])
            E = tgt - phi_expanded(cdist(case.xyz_s, case.xyz_s[Ck]) / R) @ ak
            key = (E**2).sum(1)
            key[Ck] = -1.0
            best = int(np.argmax(key))
            if best != C[k]:
                tie = abs(key[best] - key[C[k]]) <= 1e-9 * key[best]
                if not tie:
                    bad.append(f"level {l} step {k}: picked {C[k]}, brute-force argmax is {best}")
                    break
        # the level's final error is below its tolerance and ~0 at the controls
        P = phi_expanded(cdist(case.xyz_s, case.xyz_s[C]) / R)
        E = tgt - P @ res.alpha[l]
        tau = case.eps ** ((l + 1) / L)
        emax = np.sqrt((E**2).sum(1)).max() / S0
        if len(C) < case.n_s and not emax < tau:
            bad.append(f"level {l}: error {emax:g} not below tau {tau:g}")
        # two summation orders of Eq. 12 differ by at most ~ n u sum_j |alpha_j| phi_ij
        round_tol = (8 * len(C) * U * (P @ np.abs(res.alpha[l])).max() + 2 * bounds[l]) / S0
        if abs(emax - res.emax[l]) > 1e-9 * emax + round_tol:
            bad.append(f"level {l}: reported emax {res.emax[l]:g} != {emax:g}")
        if np.abs(E[C]).max() > 1e-10 * S0:
            bad.append(f"level {l}: not interpolating at the controls ({np.abs(E[C]).max():g})")
    # telescoping: dS = sum_l Phi_sc^(l) alpha^(l) + E_final
    if np.abs(final - res.E).max() > 1e-14 * S0 + final_bound:
        bad.append("levels do not telescope to dS - E_final")
    return bad


def pin_replay(o, case, seed=0):
    """Replay of a given (non-greedy, random) control sequence: at every slot
    the weights solve Eq. 9 on the controls so far (numpy.linalg.solve), the
    best key is the largest |E_i|^2 of Eq. 12 over unselected points (dense
    numpy product), the pick key is that of the given control, and the scale
    is |dS_l,i| + sum_j |alpha_j| phi_ij at both points; the next level's target
    is the replayed level's error.  Replaying the greedy's own sequence picks
    the best point at every step."""
    bad = []
    rng = np.random.default_rng(seed)
    given = [rng.permutation(case.n_s)[: min(case.n_s, 12 + 5 * l)] for l in range(len(case.R))]
    rp = o.replay(case.xyz_s, case.dS, case.R, given)
    cur = case.dS.copy()
    S0 = float(np.sqrt((case.dS**2).sum(1)).max())
    for l, R in enumerate(case.R):
        g = list(given[l])
        if abs(rp.smax[l] - np.sqrt((cur**2).sum(1)).max()) > 1e-14 * S0:
            bad.append(f"replay level {l}: smax")
        for k in range(1, len(g) + 1):
            C = g[:k]
            A = phi_expanded(cdist(case.xyz_s[C], case.xyz_s[C]) / R)
            a = np.linalg.solve(A, cur[C])
            P = phi_expanded(cdist(case.xyz_s, case.xyz_s[C]) / R)
            E = cur - P @ a
            key = (E**2).sum(1)
            key[C] = -1.0
            best = int(np.argmax(key))
            pick = g[k] if k < len(g) else best
            sc = np.sqrt((cur**2).sum(1)) + P @ np.sqrt((a**2).sum(1))
            tol = 1e-9 * key[best] + 1e-24
            if abs(rp.best_key[l][k - 1] - key[best]) > tol:
                bad.append(f"replay level {l} slot {k}: best key {rp.best_key[l][k - 1]:g} != {key[best]:g}")
                break
            if abs(rp.pick_key[l][k - 1] - key[pick]) > 1e-9 * max(key[pick], key[best]) + 1e-24:
                bad.append(f"replay level {l} slot {k}: pick key")
                break
            if abs(rp.pick_scale[l][k - 1] - sc[pick]) > 1e-9 * sc[pick]:
                bad.append(f"replay level {l} slot {k}: pick scale")
                break
            if abs(rp.best_scale[l][k - 1] - sc[best]) > 1e-9 * sc[best]:
                bad.append(f"replay level {l} slot {k}: best scale")
                break
            if k == len(g):
                if np.abs(rp.alpha[l] - a).max() > 1e-7 * (np.abs(a).max() + S0):
                    bad.append(f"replay level {l}: weights differ from numpy.linalg.solve")
                cur = cur - P @ a
    res = o.greedy(case.xyz_s, case.dS, case.R, case.eps)
    own = o.replay(case.xyz_s, case.dS, case.R, res.idx)
    for l in range(len(case.R)):
        if not np.array_equal(own.best_key[l][:-1], own.pick_key[l][:-1]):
            bad.append(f"replay of the greedy's own sequence: level {l} picks below the best key")
    return bad


def pin_dense_limit(o):
    """With eps -> 0 every surface point becomes a control and the result is
    the full RBF system of Eq. 9 / Eq. 10 solved densely."""
    case = synth.airfoil_case(20, 5, displacement="bump", seed=4, R=(1.5,), eps=1e-300)
    res = o.greedy(case.xyz_s, case.dS, case.R, case.eps)
    bad = []
    if sorted(res.idx[0].tolist()) != list(range(case.n_s)):
        return ["dense limit did not select every surface point"]
    A = phi_expanded(cdist(case.xyz_s, case.xyz_s) / 1.5)
    a_dense = np.linalg.solve(A, case.dS)
    a = np.zeros_like(a_dense)
    a[res.idx[0]] = res.alpha[0]
    if np.abs(a - a_dense).max() > 1e-8 * np.abs(a_dense).max():
        bad.append("dense limit alpha differs from the full solve of Eq. 9")
    dv = o.deform(res, case.xyz_s, case.R, case.xyz_v, case.d_v, k=0.0, D=2.0)
    want = psi_ref(case.d_v.astype(np.float64) / 2.0)[:, None] * (
        phi_expanded(cdist(case.xyz_v.astype(np.float64), case.xyz_s) / 1.5) @ a_dense
    )
    if np.abs(dv - want).max() > 1e-8 * np.abs(case.dS).max():
        bad.append("dense limit volume update differs from psi * Phi_vs alpha (Eq. 10, Eq. 23)")
    return bad


def pin_deform(o, case):
    """Eq. 19 / Eq. 23: zero where psi = 0 at every level; dS - E_final at
    volume points placed on surface points with d = 0; otherwise equal to the
    dense sum over levels of psi(d/D_l) Phi_vc alpha."""
    res = o.greedy(case.xyz_s, case.dS, case.R, case.eps)
    Dl = o.support_distances(res.smax, case.k, case.D)
    bad = []
    want_D = np.array([min(case.k * s, case.D) if case.k > 0 else case.D for s in res.smax])
    if np.abs(Dl - want_D).max() > 0:
        bad.append("support distances do not follow D_l = k max|dS_l| capped at D")
    rng = np.random.default_rng(5)
    pick = rng.choice(case.n_s, size=min(10, case.n_s), replace=False)
    xv = np.concatenate([case.xyz_v.astype(np.float64), case.xyz_s[pick]])
    dv_in = np.concatenate([case.d_v.astype(np.float64), np.zeros(len(pick))])
    far = dv_in >= Dl.max()
    out = o.deform(res, case.xyz_s, case.R, xv, dv_in, case.k, case.D)
    if np.abs(out[far]).max(initial=0.0) != 0.0:
        bad.append("points beyond every D_l moved")
    want = np.zeros_like(out)
    bound = 0.0
    for l, R in enumerate(case.R):
        w = psi_ref(dv_in / Dl[l]) if Dl[l] > 0 else np.zeros_like(dv_in)
        C = res.idx[l]
        P = phi_expanded(cdist(xv, case.xyz_s[C]) / R)
        want += w[:, None] * (P @ res.alpha[l])
        bound += 8 * max(len(C), 1) * U * (P @ np.abs(res.alpha[l])).max()
    on = out[-len(pick):]
    want_on = case.dS[pick] - res.E[pick]
    _, _, _, tele_bound = _level_targets(case, res)
    if np.abs(on - want_on).max() > 1e-14 * res.S0 + bound + tele_bound:
        bad.append("volume points on the surface (d = 0) do not move by dS - E_final")
    if np.abs(out - want).max() > 1e-14 * res.S0 + bound:
        bad.append("volume update differs from the dense sum of Eq. 19 / Eq. 23")
    return bad


def pin_wall_distance(o):
    """Brute-force nearest-surface-point distance against a k-d tree (scipy)
    and against a closed form: points on a regular polygon inscribed in the
    unit circle seen from the centre are all at distance 1."""
    from scipy.spatial import cKDTree

    bad = []
    for dim, case in ((2, tiny_airfoil(n=64, layers=8)), (3, tiny_wing())):
        d = o.wall_distance(case.xyz_s, case.xyz_v.astype(np.float64))
        want, _ = cKDTree(case.xyz_s).query(case.xyz_v.astype(np.float64))
        if np.abs(d - want).max() > 1e-12:
            bad.append(f"{dim}D wall distance differs from the k-d tree")
    t = np.linspace(0, 2 * np.pi, 17)[:-1]
    ring = np.stack([np.cos(t), np.sin(t)], axis=1)
    d = o.wall_distance(ring, np.zeros((1, 2)))
    if abs(d[0] - 1.0) > 1e-15:
        bad.append("distance from the centre of a unit ring is not 1")
    return bad


def _cart_grid_2d(nx, ny, hx=0.25, hy=0.5, shear=0.0):
    """Cartesian nx x (ny + 1) grid, row 0 the wall, x' = x + shear * y (dyadic
    values: exact in FP32)."""
    xs = np.arange(nx) * hx
    ys = np.arange(ny + 1) * hy
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    P = np.stack([X + shear * Y, Y], axis=-1)  # [i][j]
    return P[:, 0, :].copy(), P[:, 1:, :].reshape(-1, 2).copy()


def _cart_grid_3d(nx, nz, ny, shear_k=0.0):
    """Box grid: i along x, k along z (span), j along y (wall normal);
    x' = x + shear_k * z."""
    xs, zs, ys = np.arange(nx) * 0.25, np.arange(nz) * 0.5, np.arange(ny + 1) * 0.125
    Z, X, Y = np.meshgrid(zs, xs, ys, indexing="ij")  # [k][i][j]
    P = np.stack([X + shear_k * Z, Y, Z], axis=-1)
    return P[:, :, 0, :].reshape(-1, 3).copy(), P[:, :, 1:, :].reshape(-1, 3).copy()


def pin_orthogonality(o):
    """Closed forms of the orthogonality angle (mesh quality, Section 5):
    right angles on a Cartesian grid; atan(1/s) on a grid sheared by s; on a
    polar O-grid with n rays every cell is an isosceles trapezoid whose acute
    corner is 90 - 180/n degrees (this includes the cell that closes the
    ring); a node pushed through its neighbour tangles the cells around it; a
    collapsed edge gives 0."""
    bad = []
    wall, vol = _cart_grid_2d(6, 4)
    q = o.orthogonality(wall, vol, 4, periodic_i=False)
    if q.cells != 20 or np.abs(q.theta - 90.0).max() > 1e-12 or q.tangled:
        bad.append("Cartesian 2D grid is not orthogonal")
    wall, vol = _cart_grid_2d(6, 4, shear=0.5)
    q = o.orthogonality(wall, vol, 4, periodic_i=False)
    if np.abs(q.theta - np.degrees(np.arctan(2.0))).max() > 1e-12 or q.tangled:
        bad.append("sheared 2D grid angle is not atan(1/s)")
    if q.hist.sum() != q.cells or q.hist[6] != q.cells or abs(q.mean_deg - q.theta.mean()) > 1e-12:
        bad.append("histogram or mean inconsistent")
    n, r = 16, np.array([1.0, 1.5, 2.25, 3.0])
    ph = 2 * np.pi * np.arange(n) / n
    ring = np.stack([np.cos(ph), np.sin(ph)], 1)
    vol = (ring[:, None, :] * r[None, 1:, None]).reshape(-1, 2)
    q = o.orthogonality(ring * r[0], vol, 3, periodic_i=True)
    # FP32 volume coordinates move the corners by up to 2^-24 |r|: a few 1e-5 degrees here
    if q.cells != n * 3 or np.abs(q.theta - (90.0 - 180.0 / n)).max() > 1e-4 or q.tangled:
        bad.append("polar O-grid angle is not 90 - 180/n")
    wall, vol = _cart_grid_2d(5, 3)
    v = vol.reshape(5, 3, 2)
    v[2, 1, 1] = v[2, 1, 1] + 1.0  # through the node above it
    q = o.orthogonality(wall, v.reshape(-1, 2), 3, periodic_i=False)
    if q.tangled < 1:
        bad.append("a folded cell is not counted as tangled")
    wall, vol = _cart_grid_2d(5, 3)
    wd = np.zeros_like(wall)
    wd[2] = [0.25, 0.0]  # wall node 2 onto wall node 3: a zero-length edge
    q = o.orthogonality(wall, vol, 3, periodic_i=False, wall_disp=wd)
    if q.min_deg != 0.0 or q.argmin != 2 * 3 + 0:
        bad.append("collapsed edge does not give angle 0 at its cell")
    # one general quad whose only smallest corner is the last one round the cell:
    # edges (1.25, 0.25) and (0.25, -1) there, angle atan2(1.1875, 0.5625)
    q = o.orthogonality(np.array([[0.0, 0.0], [1.0, 0.0]]), np.array([[-0.25, 1.0], [1.0, 0.75]]), 1,
                        periodic_i=False)
    if abs(q.min_deg - np.degrees(np.arctan2(1.1875, 0.5625))) > 1e-12:
        bad.append("single quad: smallest corner angle wrong")
    wall, vol = _cart_grid_3d(5, 4, 3)
    q = o.orthogonality(wall, vol, 3, periodic_i=False, n_k=4)
    if q.cells != 4 * 3 * 3 or np.abs(q.theta - 90.0).max() > 1e-12 or q.tangled:
        bad.append("Cartesian 3D grid is not orthogonal or counted tangled")
    wall, vol = _cart_grid_3d(5, 4, 3, shear_k=0.25)
    q = o.orthogonality(wall, vol, 3, periodic_i=False, n_k=4)
    if np.abs(q.theta - np.degrees(np.arctan(1.0 / 0.25))).max() > 1e-12 or q.tangled:
        bad.append("sheared 3D grid angle is not atan(1/s)")
    return bad


def all_pins(o):
    bad = []
    bad += pin_table1(o)
    bad += pin_phi_expanded(o)
    bad += pin_phi_smoothness(o)
    bad += pin_psi(o)
    bad += pin_cholesky(o)
    bad += pin_eval_dense(o)
    bad += pin_spd(o)
    bad += pin_greedy(o, tiny_airfoil())
    bad += pin_greedy(o, tiny_airfoil(n=60, displacement="horns", R=(1.0, 0.2), eps=1e-6))
    bad += pin_greedy(o, tiny_wing())
    bad += pin_dense_limit(o)
    bad += pin_replay(o, tiny_airfoil(n=60, displacement="horns", R=(1.0, 0.2), eps=1e-6))
    bad += pin_replay(o, tiny_wing(), seed=1)
    bad += pin_deform(o, tiny_airfoil_k5())
    bad += pin_deform(o, tiny_wing())
    bad += pin_wall_distance(o)
    bad += pin_orthogonality(o)
    return bad


# ------------------------------------------------------------------ tests


def test_table1_exact():
    assert pin_table1(oracle) == []


def test_phi_matches_expanded_polynomial():
    assert pin_phi_expanded(oracle) == []


def test_phi_smoothness():
    assert pin_phi_smoothness(oracle) == []


def test_psi_closed_form():
    assert pin_psi(oracle) == []


def test_cholesky_and_solve_vs_numpy():
    assert pin_cholesky(oracle) == []


def test_evaluation_vs_dense_product():
    assert pin_eval_dense(oracle) == []


def test_phi_cc_spd():
    assert pin_spd(oracle) == []


@pytest.mark.parametrize("disp", ["bump", "horns", "sinusoid", "pitch_heave"])
def test_greedy_airfoil_single_level(disp):
    assert pin_greedy(oracle, tiny_airfoil(n=64, displacement=disp, eps=1e-6)) == []


def test_greedy_airfoil_two_levels():
    assert pin_greedy(oracle, tiny_airfoil(n=80, displacement="horns", R=(1.0, 0.2), eps=1e-6)) == []


def test_greedy_first_rule_argmax():
    assert pin_greedy(oracle, tiny_airfoil(n=64, displacement="bump", eps=1e-5), first_rule=1) == []


def test_greedy_wing_3d():
    assert pin_greedy(oracle, tiny_wing()) == []


def test_replay_of_given_sequences():
    assert pin_replay(oracle, tiny_airfoil(n=60, displacement="horns", R=(1.0, 0.2), eps=1e-6)) == []
    assert pin_replay(oracle, tiny_wing(), seed=1) == []


def test_dense_limit():
    assert pin_dense_limit(oracle) == []


def test_deform_airfoil():
    assert pin_deform(oracle, tiny_airfoil_k5()) == []


def test_deform_wing():
    assert pin_deform(oracle, tiny_wing()) == []


def test_wall_distance_vs_kdtree_and_closed_form():
    assert pin_wall_distance(oracle) == []


def test_orthogonality_closed_forms():
    assert pin_orthogonality(oracle) == []


def test_incremental_equals_scratch():
    # appending one Cholesky row per control is the same arithmetic as
    # refactorising from scratch, so the two solve modes agree bit for bit
    c = tiny_airfoil(n=80, displacement="horns", R=(1.0, 0.2), eps=1e-6)
    a = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, solve_mode=0)
    b = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, solve_mode=1)
    for l in range(2):
        assert np.array_equal(a.idx[l], b.idx[l])
        assert np.array_equal(a.alpha[l], b.alpha[l])


def test_zero_displacement_gives_zero_levels():
    c = tiny_airfoil()
    r = oracle.greedy(c.xyz_s, np.zeros_like(c.dS), c.R, c.eps)
    assert r.status == oracle.OK and all(len(i) == 0 for i in r.idx)
    dv = oracle.deform(r, c.xyz_s, c.R, c.xyz_v, c.d_v, c.k, c.D)
    assert not dv.any()


def test_cap_reports_not_converged():
    c = tiny_airfoil(n=64, eps=1e-8)
    r = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, nc_cap=5)
    assert r.status == oracle.ENOTCONV and len(r.idx[0]) == 5


def test_duplicate_point_is_singular():
    # two coincident surface points with different displacements make Phi_cc singular
    c = tiny_airfoil(n=32)
    xyz = np.concatenate([c.xyz_s, c.xyz_s[5:6]])
    dS = np.concatenate([c.dS, c.dS[5:6] + 0.01])
    with pytest.raises(RuntimeError, match="status 3"):
        oracle.greedy(xyz, dS, c.R, 1e-12)


def test_local_ice_controls_cluster_at_leading_edge():
    # Section 5.1: for local ice the controls gather around the leading edge,
    # for the sinusoid they spread along the chord
    ice = synth.airfoil_case(400, 0, displacement="bump", seed=0, R=(0.5,), eps=1e-4)
    r = oracle.greedy(ice.xyz_s, ice.dS, ice.R, ice.eps)
    x_ice = ice.xyz_s[r.idx[0], 0]
    sin = synth.airfoil_case(400, 0, displacement="sinusoid", seed=0, R=(0.5,), eps=1e-4)
    r = oracle.greedy(sin.xyz_s, sin.dS, sin.R, sin.eps)
    x_sin = sin.xyz_s[r.idx[0], 0]
    near_le_surface = (ice.xyz_s[:, 0] < 0.1).mean()
    assert (x_ice < 0.1).mean() > 2 * near_le_surface
    assert (x_ice < 0.1).mean() > 2 * (x_sin < 0.1).mean()
    assert all(((x_sin >= a) & (x_sin < a + 0.25)).any() for a in (0.0, 0.25, 0.5, 0.75))


def test_openmp_threads_do_not_change_results():
    c = tiny_airfoil(n=80, displacement="horns", R=(1.0, 0.2), eps=1e-6)
    a = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=1)
    b = oracle.greedy(c.xyz_s, c.dS, c.R, c.eps, n_threads=4)
    for l in range(2):
        assert np.array_equal(a.idx[l], b.idx[l]) and np.array_equal(a.alpha[l], b.alpha[l])


# ------------------------------------------------------------ mutation tests

MUTATIONS = {
    "drop (4 eta + 1) term": ("return (t2 * t2) * (4.0 * eta + 1.0);", "return (t2 * t2) * (4.0 * eta);"),
    "wrong power in C2": ("return (t2 * t2) * (4.0 * eta + 1.0);", "return (t2 * t) * (4.0 * eta + 1.0);"),
    "wrong sign in Eq. 12": ("E[i] = cur[i] - E[i];", "E[i] = cur[i] + E[i];"),
    "psi not 1 - xi": ("return 1.0 - xi;", "return 1.0 - 0.5 * xi;"),
    "argmax picks smallest": ("if (v > bestv) {", "if (bestv < 0.0 || v < bestv) {"),
    "Cholesky sign": ("s = s - Lrow[k] * Lj[k];", "s = s + Lrow[k] * Lj[k];"),
    "back substitution transposed": ("s = s - L[k * ld + i] * X[k * nrhs + r];",
                                     "s = s - L[i * ld + k] * X[k * nrhs + r];"),
    "next level ignores E": ("memcpy(cur, E, sizeof(double) * (size_t)(n_s * dim));\n    }",
                             "memcpy(cur, dS, sizeof(double) * (size_t)(n_s * dim));\n    }"),
    "support distance of level 0 only": ("double v = (k > 0.0) ? k * smax[l] : D;",
                                         "double v = (k > 0.0) ? k * smax[0] : D;"),
    "psi blend dropped": ("out[v * dim + k] = out[v * dim + k] + w * acc[k];",
                          "out[v * dim + k] = out[v * dim + k] + acc[k];"),
    "distance drops z": ("for (int k = 0; k < dim; ++k) {\n        double d = a[k] - b[k];",
                         "for (int k = 0; k < 2; ++k) {\n        double d = a[k] - b[k];"),
    "first control not point 0": ("int64_t first = 0;", "int64_t first = 1;"),
    "replay records the key before the pick's": ("pick_key[slot] = pick >= 0 ? norm2sq(E + pick * dim, dim) : -1.0;",
                                                 "pick_key[slot] = pick >= 0 ? norm2sq(E + best * dim, dim) : -1.0;"),
    "replay scale drops the weights": ("sc = sc + sqrt(norm2sq(alpha + j * dim, dim)) *",
                                       "sc = sc + 0.0 * sqrt(norm2sq(alpha + j * dim, dim)) *"),
    "wall distance skips the last point": ("for (int64_t i = 0; i < n_s; ++i) {\n            double r = dist(",
                                           "for (int64_t i = 0; i < n_s - 1; ++i) {\n            double r = dist("),
    "orthogonality drops the ring-closing cell": ("int64_t n_ci = periodic_i ? n_i : n_i - 1;",
                                                  "int64_t n_ci = n_i - 1;"),
    "orthogonality volume layer off by one": ("int64_t q = ((k * g->n_i + i) * g->n_layers + (j - 1)) * g->dim + c;",
                                              "int64_t q = ((k * g->n_i + i) * g->n_layers + j) * g->dim + c;"),
    "orthogonality ignores corner parity": ("if ((di + dk + dj) & 1) o = -o;", ""),
    "orthogonality skips one corner": ("for (int q = 0; q < 4; ++q) {\n                        sub3(P[(q + 1) % 4]",
                                       "for (int q = 0; q < 3; ++q) {\n                        sub3(P[(q + 1) % 4]"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rbfd_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new)
    p = tmp_path / "mutant.c"
    p.write_text(mutated)
    lib = oracle.build(force=True, src=str(p), out=str(tmp_path / "libmutant.so"))
    variant = oracle.load_variant(lib)
    try:
        bad = all_pins(variant)
    except Exception as exc:  # a mutant that breaks a solve outright is caught too
        bad = [repr(exc)]
    assert bad, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_every_pin():
    assert all_pins(oracle) == []
