"""The bound behind the pruned list sweep, checked on the CPU in plain FP64
(no GPU): a greedy step adds control n with weight row g = row n of the
inverse factor G = L^{-1} and Newton weight w_n (Section 3, Eq. 9 solved by
the bordered Cholesky update), so the error of Eq. 12 moves by

    E_new(x) - E_old(x) = -w_n sum_c g_c phi(|x - r_c| / R),

and for every point x in a box B,

    |E_new(x) - E_old(x)| <= |w_n| sum_c |g_c| phi(dist(r_c, B) / R).

The library keeps that sum per warp of 32 points (box of the warp) and skips
a warp while its last maximum plus the accumulated moves stays below the
largest lower bound of any warp.  This test runs the greedy in numpy on a
small wing, checks the inequality for every warp and step, and checks that
the skipping rule never skips the warp that holds the step's argmax.
"""
import numpy as np

from paper_2107_13887_gb300 import synth


def _wendland_c2(q):
    return np.where(q < 1.0, (1.0 - q) ** 4 * (4.0 * q + 1.0), 0.0)


def _morton_order(X):
    lo = X.min(0)
    ext = (X.max(0) - lo).max()
    q = np.minimum(((X - lo) / ext * 1024).astype(np.int64), 1023)

    def spread(v):
        v = v & 0x3FF
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        return v

    return np.argsort(spread(q[:, 0]) | (spread(q[:, 1]) << 1) | (spread(q[:, 2]) << 2), kind="stable")


def test_move_bound_holds_and_never_skips_the_argmax():
    c = synth.wing_case(30, 20, 2, displacement="ridge", seed=0, R=(0.3,), eps=1e-4, D=1.0, k=4.0,
                        wall_distance=False)
    X = np.asarray(c.xyz_s, np.float64)
    order = _morton_order(X)
    X = X[order]
    F = np.asarray(c.dS, np.float64)[order]
    n_s, R = len(X), 0.3
    S0 = np.sqrt((F ** 2).sum(1)).max()
    starts = np.arange(0, n_s, 32)
    n_w = len(starts)
    blo = np.minimum.reduceat(X, starts)
    bhi = np.maximum.reduceat(X, starts)
    wmax = lambda v: np.maximum.reduceat(v, starts)

    cap = 200
    G = np.zeros((cap, cap))
    w = np.zeros((cap, 3))
    ctrl = []
    E = F.copy()
    M = np.sqrt(wmax((E ** 2).sum(1)))  # every warp swept at the start
    acc = np.zeros(n_w)
    selected = np.zeros(n_s, bool)
    skipped_any = False
    for n in range(cap):
        key = (E ** 2).sum(1)
        key[selected] = -1.0
        i = int(np.argmax(key))
        if np.sqrt(key[i]) / S0 < 1e-4:
            break
        # the skipping rule on the bounds of the previous steps: the warp of
        # the argmax must be among the swept ones
        hi, lo = M + acc, M - acc
        swept = hi >= lo.max()
        assert swept[i // 32], f"step {n}: the argmax's warp would have been skipped"
        skipped_any |= not swept.all()
        cur = np.sqrt(wmax(np.where(selected, 0.0, key)))
        M[swept] = cur[swept]
        acc[swept] = 0.0
        # the selected point's warp loses its maximum: no lower bound until swept again
        acc[i // 32] = np.inf
        # bordered Cholesky update through the inverse factor
        xc = X[i]
        phi = _wendland_c2(np.linalg.norm(X[ctrl] - xc, axis=1) / R) if ctrl else np.zeros(0)
        y = G[:n, :n] @ phi
        l = np.sqrt(1.0 - y @ y)
        wn = (F[i] - y @ w[:n]) / l
        g = np.zeros(n + 1)
        g[:n] = -(y @ G[:n, :n]) / l
        g[n] = 1.0 / l
        G[n, :n + 1] = g
        w[n] = wn
        ctrl.append(i)
        selected[i] = True
        # the move of E and its bound per warp box
        C = X[ctrl]
        phis = _wendland_c2(np.linalg.norm(X[:, None, :] - C[None, :, :], axis=2) / R)  # [n_s, n + 1]
        E_new = E - np.outer(phis @ g, wn)
        d = np.maximum(np.maximum(blo[:, None, :] - C[None], C[None] - bhi[:, None, :]), 0.0)
        bound = np.linalg.norm(wn) * (_wendland_c2(np.linalg.norm(d, axis=2) / R) @ np.abs(g))  # [n_w]
        moved = wmax(np.linalg.norm(E_new - E, axis=1))
        assert (moved <= bound * (1 + 1e-12) + 1e-15 * S0).all(), f"step {n}: a move exceeds its bound"
        acc += bound
        E = E_new
    assert len(ctrl) > 20 and skipped_any  # (the rule skipped warps on this case)


def test_move_bound_sum_needs_fp64():
    """The per-warp move bound is a sum of many atomic additions in any order:
    a far warp receives small increments against a running sum that may be
    far larger.  Summed in FP32 they can vanish (each is rounded against the
    running sum), so the FP32 sum read with the kernel's 2^-8 margin can fall
    below the exact sum; summed in FP64 (each addition within 2^-53 of the
    running sum) and read rounded up to FP32 with the same margin, it cannot.
    """
    import math

    rng = np.random.default_rng(0)
    # one large increment (a near control) and a million small ones (far
    # controls, each under half an FP32 ulp of the running sum)
    inc = np.concatenate([[1.0], np.full(1_000_000, 1e-8)])
    exact = math.fsum(inc)
    s32 = np.cumsum(inc.astype(np.float32), dtype=np.float32)[-1]
    assert float(s32) * (1 + 2.0 ** -8) < exact  # the FP32 sum is no bound
    for order in (np.arange(len(inc)), rng.permutation(len(inc))):
        s64 = np.cumsum(inc[order], dtype=np.float64)[-1]
        read = np.float32(s64)  # FP32, rounded up
        if float(read) < s64:
            read = np.nextafter(read, np.float32(np.inf))
        read = float(read)
        assert read * (1 + 2.0 ** -8) >= exact
        assert abs(s64 - exact) <= len(inc) * 2.0 ** -53 * exact
    # increments of every size in random order
    inc = np.exp(rng.uniform(np.log(1e-12), np.log(1.0), 200_000))
    exact = math.fsum(inc)
    s64 = np.cumsum(inc[rng.permutation(len(inc))], dtype=np.float64)[-1]
    assert abs(s64 - exact) <= len(inc) * 2.0 ** -53 * exact
