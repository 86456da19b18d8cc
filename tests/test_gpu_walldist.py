"""Wall distance d(r) on the GPU (rbfd_wall_distance) against the oracle's
brute-force minimum, and the volume update paths that compute d on the device.

The GPU result is the minimum over the surface of the same FP64 expression the
oracle evaluates (differences, squares and sums rounded once each, in axis
order, then a correctly rounded square root), so the bar is bit-for-bit
equality, also at full size on sampled points.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


def wall_ref(xyz_s, xv):
    return oracle.wall_distance(xyz_s, np.asarray(xv, dtype=np.float64), n_threads=NT)


def assert_exact(got, want):
    got = np.asarray(got)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (f"{bad.size} of {len(want)} distances differ, first at {bad[0]}: "
                           f"{got[bad[0]]!r} vs {want[bad[0]]!r}")


def probe_points(c, rng, n_far=500, n_near=2000):
    """The case's volume points plus hard ones: the surface points themselves
    (d = 0), points a hair off the wall (1e-7 .. 1e-3 along random directions,
    where FP32 coordinates alone cannot separate neighbours) and far points."""
    dim = c.dim
    xs = c.xyz_s
    pick = rng.integers(0, len(xs), n_near)
    off = rng.normal(size=(n_near, dim))
    off /= np.linalg.norm(off, axis=1, keepdims=True)
    near = xs[pick] + off * 10.0 ** rng.uniform(-7, -3, (n_near, 1))
    far = rng.normal(size=(n_far, dim))
    far = far / np.linalg.norm(far, axis=1, keepdims=True) * rng.uniform(5, 60, (n_far, 1))
    return np.concatenate([c.xyz_v, xs, near, far]).astype(np.float32)


CASES = {
    # 333 surface points: two full blocks of 128 and a ragged block of 77
    "airfoil_333": lambda: synth.airfoil_case(333, 7, displacement="bump", seed=1, R=(0.5,), eps=1e-4, D=2.0, k=0.0),
    "airfoil_4000": lambda: synth.airfoil_case(4000, 12, displacement="horns", seed=2, R=(1.0, 0.2), eps=1e-5,
                                               D=2.0, k=5.0),
    "wing_40x15": lambda: synth.wing_case(40, 15, 6, displacement="ridge", seed=3, R=(1.5, 0.4), eps=1e-3,
                                          D=1.0, k=4.0),
    "wing_120x40": lambda: synth.wing_case(120, 40, 8, displacement="ridge", seed=4, R=(1.5, 0.4), eps=1e-3,
                                           D=1.0, k=4.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_wall_distance_bit_exact(name):
    c = CASES[name]()
    rng = np.random.default_rng(7)
    xv = probe_points(c, rng)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    got = m.wall_distance(xv)
    assert got.dtype == np.float64 and got.shape == (len(xv),)
    assert_exact(got, wall_ref(c.xyz_s, xv))
    # the surface points (rounded to FP32) lie within their rounding offset
    n0 = len(c.xyz_v)
    off = np.linalg.norm(xv[n0 : n0 + len(c.xyz_s)].astype(np.float64) - c.xyz_s, axis=1)
    assert np.all(got[n0 : n0 + len(c.xyz_s)] <= off)
    st = m.stats()
    assert st["wall_launches"] >= 1 and st["wall_pairs_search"] > 0 and st["wall_pairs_exact"] > 0


def test_wall_distance_f64_coordinates_and_device_pointers():
    import torch

    c = CASES["airfoil_333"]()
    rng = np.random.default_rng(11)
    xv64 = rng.uniform(-2.0, 3.0, (5000, 2))  # not representable in FP32
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    assert_exact(m.wall_distance(xv64), wall_ref(c.xyz_s, xv64))
    # the surface points themselves, in FP64, are at distance exactly 0
    assert not m.wall_distance(c.xyz_s).any()
    # device pointers: the same call on torch tensors
    md = rbfd.Mesh(torch.from_numpy(c.xyz_s).cuda(), torch.from_numpy(c.dS).cuda(), c.R, c.eps)
    d64 = md.wall_distance(torch.from_numpy(xv64).cuda())
    assert d64.is_cuda and d64.dtype == torch.float64
    assert_exact(d64.cpu().numpy(), wall_ref(c.xyz_s, xv64))
    xv32 = xv64.astype(np.float32)
    d32 = md.wall_distance(torch.from_numpy(xv32).cuda())
    assert_exact(d32.cpu().numpy(), wall_ref(c.xyz_s, xv32))


@pytest.mark.parametrize("n_v", [0, 1, 31, 33, 129, 4097])
def test_wall_distance_ragged_counts(n_v):
    c = CASES["wing_40x15"]()
    rng = np.random.default_rng(n_v)
    xv = rng.uniform(-1.0, 4.0, (n_v, 3)).astype(np.float32)
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    got = m.wall_distance(xv)
    assert got.shape == (n_v,)
    if n_v:
        assert_exact(got, wall_ref(c.xyz_s, xv))


def test_wall_distance_degenerate_surfaces():
    # one surface point: the plain Euclidean distance
    xs = np.array([[0.25, -0.5, 1.0]])
    m = rbfd.Mesh(xs, np.array([[0.0, 0.01, 0.0]]), [1.0], 1e-3)
    rng = np.random.default_rng(0)
    xv = rng.normal(size=(300, 3)).astype(np.float32)
    assert_exact(m.wall_distance(xv), wall_ref(xs, xv))
    # all volume points at one location, and points on a far-away plane
    c = CASES["airfoil_333"]()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    same = np.tile(np.array([[0.3, 0.02]], np.float32), (257, 1))
    plane = np.stack([np.linspace(-1e4, 1e4, 1000), np.full(1000, 3e3)], 1).astype(np.float32)
    for xv in (same, plane):
        assert_exact(m.wall_distance(xv), wall_ref(c.xyz_s, xv))


def test_wall_distance_invalid_arguments():
    c = CASES["airfoil_333"]()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    lib = rbfd.load()
    assert lib.rbfd_wall_distance(m.h, 10, None, None) == rbfd.EINVAL
    assert lib.rbfd_wall_distance(m.h, -1, None, None) == rbfd.EINVAL
    assert lib.rbfd_wall_distance(None, 0, None, None) == rbfd.EINVAL


@pytest.mark.parametrize("disp", ["horns", "pitch_heave"])
def test_wall_distance_full_size_sampled(disp):
    """4000 surface points, 1M volume points (the two-level NACA 0012
    workload): every point through the GPU, 4096 sampled points plus the first
    and last against the oracle, bit for bit."""
    c = synth.make_config(f"naca0012_4000s_1mv_{disp}")
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    got = m.wall_distance(c.xyz_v)
    rng = np.random.default_rng(5)
    sample = np.concatenate([[0, len(got) - 1], rng.choice(len(got), 4096, replace=False)])
    assert_exact(got[sample], wall_ref(c.xyz_s, c.xyz_v[sample]))
    # the generator's k-d tree distances (FP32-stored) agree to FP32 rounding
    assert np.abs(got - c.d_v.astype(np.float64)).max() <= 2.0**-23 * max(1.0, np.abs(got).max())


# ------------------------------------------------ volume update without d_v


def _ref_deform(c, ref, d):
    return oracle.deform(ref, c.xyz_s, c.R, c.xyz_v, d, c.k, c.D, n_threads=NT)


def _gpu_levels_as_reference(c, m):
    """The GPU's own controls and weights in the oracle's result type, so
    that the FP64 volume update of the oracle uses exactly them."""
    lv = m.levels()
    return oracle.GreedyResult(status=0, idx=[l.idx for l in lv], alpha=[l.alpha for l in lv],
                               smax=np.array([l.smax for l in lv]), emax=np.array([l.e_max for l in lv]),
                               gap=np.zeros(len(lv)), E=None, S0=float(np.sqrt((c.dS**2).sum(1)).max()))


@pytest.mark.parametrize("name", ["airfoil_333", "wing_40x15"])
@pytest.mark.parametrize("precision", [rbfd.FP64, rbfd.MIXED], ids=["fp64", "mixed"])
def test_deform_with_device_wall_distance(name, precision):
    """rbfd_deform with d_v = NULL equals the oracle's FP64 volume update on
    the same controls and weights fed the oracle's exact wall distances
    (FP64: 1e-10 max|dS|; mixed: 1e-5 max|dS|, the volume parity bars)."""
    c = CASES[name]()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision)
    m.greedy()
    ref = _gpu_levels_as_reference(c, m)
    d = wall_ref(c.xyz_s, c.xyz_v)
    want = _ref_deform(c, ref, d)
    got = m.deform(c.xyz_v, None, c.D, c.k).astype(np.float64)
    tol = (1e-10 if precision == rbfd.FP64 else 1e-5) * ref.S0
    assert np.abs(got - want).max() <= tol + np.abs(want).max() * 2.0**-24
    # FP64 coordinates as well
    if precision == rbfd.FP64:
        got64 = m.deform(c.xyz_v.astype(np.float64), None, c.D, c.k)
        assert np.abs(got64 - want).max() <= tol


def test_registered_volume_and_server_with_device_wall_distance():
    c = CASES["airfoil_4000"]()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    m.greedy()
    direct = m.deform(c.xyz_v, None, c.D, c.k)
    m.set_volume(c.xyz_v, None)
    reg = m.deform_volume(c.D, c.k)
    S0 = np.sqrt((c.dS**2).sum(1)).max()
    assert np.abs(reg - direct).max() <= 1e-7 * S0
    srv = rbfd.Server(slots=2)
    try:
        mid = srv.add_mesh(c.xyz_s, c.xyz_v, None, c.R, c.eps, c.D, c.k)
        t = srv.submit(mid, c.dS)
        _, out = srv.wait(t)
        # another instance, its greedy on a share of the grid: same controls,
        # weights equal up to the rounding of the growth reductions
        assert np.abs(out - direct).max() <= 1e-5 * S0
    finally:
        srv.close()
