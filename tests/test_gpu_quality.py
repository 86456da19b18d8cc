"""Mesh quality (orthogonality angle) on the GPU (rbfd_orthogonality) against
the oracle, cell by cell.

Bars: angles within 1e-4 degrees of the oracle's FP64 angles (the GPU forms
nodes and edges in FP64 like the oracle, then rounds the edges to FP32 unit
vectors: a few FP32 roundings of O(2^-24) radians each, far below 1e-5 deg,
plus atan2f and the degree conversion at a few ulp of 90); tangled decisions
equal (taken in FP64 wherever the FP32 value is within its error of zero);
the histogram equals the bins of the GPU's own angles; the mean within 1e-12
relative of the mean of the GPU angles; the minimum and argmin consistent.
"""
import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu

TOL_DEG = 1e-4


def check(wall, vol, n_layers, periodic=True, wall_disp=None, vol_disp=None, n_k=1):
    th, q = rbfd.orthogonality(wall, vol, n_layers, periodic_i=periodic, wall_disp=wall_disp, vol_disp=vol_disp,
                               n_k=n_k)
    ref = oracle.orthogonality(wall, vol, n_layers, periodic_i=periodic, wall_disp=wall_disp, vol_disp=vol_disp,
                               n_k=n_k)
    th = np.asarray(th, dtype=np.float64)
    assert q["cells"] == ref.cells == len(th)
    err = np.abs(th - ref.theta)
    assert err.max() <= TOL_DEG, f"angle error {err.max():g} deg at cell {err.argmax()}"
    assert q["tangled"] == ref.tangled
    bins = np.minimum(8, (th.astype(np.float32) * np.float32(0.1)).astype(np.int64))
    assert list(np.bincount(bins, minlength=9)) == q["hist"]
    assert abs(q["mean_deg"] - th.mean()) <= 1e-12 * max(1.0, th.mean())
    assert q["min_deg"] == th.min() and th[q["argmin"]] == th.min() and q["argmin"] == int(np.argmin(th))
    assert abs(q["min_deg"] - ref.min_deg) <= TOL_DEG
    return th, q, ref


def polar(n, radii):
    ph = 2 * np.pi * np.arange(n) / n
    ring = np.stack([np.cos(ph), np.sin(ph)], 1)
    return ring * radii[0], (ring[:, None, :] * np.asarray(radii)[None, 1:, None]).reshape(-1, 2)


def test_closed_form_grids():
    wall, vol = polar(64, [1.0, 1.1, 1.3, 1.6, 2.0])
    th, q, _ = check(wall, vol, 4)
    assert np.abs(th - (90.0 - 180.0 / 64)).max() <= TOL_DEG and q["tangled"] == 0
    # sheared Cartesian grid (dyadic coordinates, exact in FP32): atan(1/s)
    xs, ys = np.arange(9) * 0.25, np.arange(6) * 0.5
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    P = np.stack([X + 0.5 * Y, Y], -1)
    th, _, _ = check(P[:, 0], P[:, 1:].reshape(-1, 2), 5, periodic=False)
    assert np.abs(th - np.degrees(np.arctan(2.0))).max() <= TOL_DEG
    # 3D box sheared along the span
    zs = np.arange(4) * 0.5
    Z, X, Y = np.meshgrid(zs, xs, ys, indexing="ij")
    P = np.stack([X + 0.25 * Z, Y, Z], -1)
    th, q, _ = check(P[:, :, 0].reshape(-1, 3), P[:, :, 1:].reshape(-1, 3), 5, periodic=False, n_k=4)
    assert np.abs(th - np.degrees(np.arctan(4.0))).max() <= TOL_DEG and q["tangled"] == 0


def _deformed(c, precision=rbfd.MIXED):
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision)
    m.greedy()
    return m.deform(c.xyz_v, c.d_v, c.D, c.k)


@pytest.mark.parametrize("disp", ["bump", "horns", "pitch_heave"])
def test_airfoil_o_mesh_clean_and_deformed(disp):
    c = synth.airfoil_case(333, 24, displacement=disp, seed=1, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)
    check(c.xyz_s, c.xyz_v, 24)
    dv = _deformed(c)
    _, q, _ = check(c.xyz_s, c.xyz_v, 24, wall_disp=c.dS, vol_disp=dv)
    assert q["tangled"] == 0


@pytest.mark.parametrize("disp", ["ridge", "sinusoid"])
def test_wing_o_h_mesh_clean_and_deformed(disp):
    nc, ns, nl = 60, 12, 10
    c = synth.wing_case(nc, ns, nl, displacement=disp, seed=3, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0)
    check(c.xyz_s, c.xyz_v, nl, n_k=ns)
    dv = _deformed(c)
    check(c.xyz_s, c.xyz_v, nl, wall_disp=c.dS, vol_disp=dv, n_k=ns)


def test_tangled_and_degenerate_cells():
    c = synth.airfoil_case(200, 6, displacement="bump", seed=0)
    v = c.xyz_v.reshape(200, 6, 2).copy()
    v[50, 2] = v[50, 4]          # a node pushed through the layer above it
    v[120, 0] = c.xyz_s[121]     # a node dropped onto the wall: a collapsed cell
    _, q, ref = check(c.xyz_s, v.reshape(-1, 2), 6)
    assert q["tangled"] >= 2 and ref.tangled == q["tangled"]
    # 3D: a layer squashed flat (zero-volume corners exercise the FP64 orientation path)
    w = synth.wing_case(30, 6, 5, displacement="ridge", seed=1, R=(1.5,), eps=1e-3)
    vv = w.xyz_v.reshape(6, 30, 5, 3).copy()
    vv[2, 10:14, 1] = vv[2, 10:14, 0]
    vv[4, 3, 2] = vv[4, 3, 2] + np.float32(1e-9)
    check(w.xyz_s, vv.reshape(-1, 3), 5, n_k=6)


def test_full_size_airfoil_one_million_cells():
    """4000 x 250 O-mesh (1M cells) deformed by the two-level greedy: every cell
    against the oracle."""
    c = synth.make_config("naca0012_4000s_1mv_horns")
    dv = _deformed(c)
    _, q, ref = check(c.xyz_s, c.xyz_v, 250, wall_disp=c.dS, vol_disp=dv)
    assert q["cells"] == 1_000_000 and q["tangled"] == 0


def test_device_pointers_and_repeatability():
    import torch

    c = synth.airfoil_case(333, 24, displacement="horns", seed=1, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)
    dv = _deformed(c)
    th_h, q_h = rbfd.orthogonality(c.xyz_s, c.xyz_v, 24, wall_disp=c.dS, vol_disp=dv)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    th_d, q_d = rbfd.orthogonality(t(c.xyz_s), t(c.xyz_v), 24, wall_disp=t(c.dS), vol_disp=t(dv))
    assert np.array_equal(th_d.cpu().numpy(), th_h) and q_d == q_h
    th_2, q_2 = rbfd.orthogonality(c.xyz_s, c.xyz_v, 24, wall_disp=c.dS, vol_disp=dv)
    assert np.array_equal(th_2, th_h) and q_2 == q_h
    # summary only
    none, q_n = rbfd.orthogonality(c.xyz_s, c.xyz_v, 24, wall_disp=c.dS, vol_disp=dv, theta=False)
    assert none is None and q_n == q_h


def test_invalid_arguments():
    lib = rbfd.load()
    q = rbfd.rbfd_quality()
    w = np.zeros((4, 2))
    v = np.zeros((8, 2), np.float32)
    pw, pv = rbfd._ptr(w), rbfd._ptr(v)
    assert lib.rbfd_orthogonality(4, 4, 1, 2, 1, pw, None, pv, None, None, q, 0, None) == rbfd.EINVAL
    assert lib.rbfd_orthogonality(2, 1, 1, 2, 1, pw, None, pv, None, None, q, 0, None) == rbfd.EINVAL
    assert lib.rbfd_orthogonality(2, 4, 1, 0, 1, pw, None, pv, None, None, q, 0, None) == rbfd.EINVAL
    assert lib.rbfd_orthogonality(2, 4, 1, 2, 1, None, None, pv, None, None, q, 0, None) == rbfd.EINVAL
    assert lib.rbfd_orthogonality(3, 4, 1, 2, 1, pw, None, pv, None, None, q, 0, None) == rbfd.EINVAL
    # host arrays with on_device set
    assert lib.rbfd_orthogonality(2, 4, 1, 2, 1, pw, None, pv, None, None, q, 1, None) == rbfd.EINVAL
