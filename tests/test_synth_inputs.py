"""The seeded synthetic inputs that stand in for the paper's meshes: the named
workloads have the stated sizes and structure, the NACA0012 outline follows
the 4-digit thickness law, no two surface points coincide, the wall distance
is the distance to the nearest surface point, and a seed reproduces a case
exactly.  No GPU."""
import numpy as np
import pytest

from paper_2107_13887_gb300 import synth

scipy_spatial = pytest.importorskip("scipy.spatial")


def test_naca0012_outline_closed_form():
    xy, nrm, s = synth.naca0012_surface(400)
    assert xy.shape == (400, 2) and nrm.shape == (400, 2)
    # half thickness 5 t (0.2969 sqrt x - 0.1260 x - 0.3516 x^2 + 0.2843 x^3 - 0.1015 x^4), t = 0.12:
    # maximum 0.0600 near x = 0.30, zero at the leading edge, 0.00126 at the open trailing edge
    x, y = xy[:, 0], xy[:, 1]
    assert x.min() == 0.0 and abs(x.max() - 1.0) < 1e-12
    assert abs(np.abs(y).max() - 0.0600) < 2e-4
    assert abs(x[np.argmax(y)] - 0.30) < 0.02
    te = np.abs(x - 1.0) < 1e-12
    assert np.allclose(np.abs(y[te]), 0.00126, atol=1e-5)
    np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-12)
    assert s[np.argmin(x)] == 0.0 and (s[y > 0] < 0).all()


@pytest.mark.parametrize("name,n_s,n_v,dim,levels", [
    ("naca0012_400s_40kv_bump", 400, 40_000, 2, 1),
    ("naca0012_4000s_1mv_pitch_heave", 4000, 1_000_000, 2, 2),
    ("naca0012_4000s_1mv_horns", 4000, 1_000_000, 2, 2),
])
def test_named_2d_workloads(name, n_s, n_v, dim, levels):
    c = synth.make_config(name)
    assert (c.n_s, c.n_v, c.dim, c.n_levels) == (n_s, n_v, dim, levels)
    assert c.xyz_s.dtype == np.float64 and c.dS.dtype == np.float64
    assert c.xyz_v.dtype == np.float32 and c.d_v.dtype == np.float32
    assert len(np.unique(c.xyz_s, axis=0)) == n_s  # no coincident surface points
    assert np.isfinite(c.dS).all() and np.abs(c.dS).max() > 0
    # d_v is the distance to the nearest surface point (sampled)
    idx = np.random.default_rng(1).choice(n_v, 2000, replace=False)
    d, _ = scipy_spatial.cKDTree(c.xyz_s).query(c.xyz_v[idx].astype(np.float64))
    np.testing.assert_allclose(c.d_v[idx], d, rtol=1e-6, atol=1e-6)


def test_wing_workload_structure():
    c = synth.make_config("wing_60ks_6mv_ridge", n_layers=2)  # the 60k surface, two volume layers
    assert (c.n_s, c.dim, c.n_levels) == (60_000, 3, 3) and c.n_v == 120_000
    assert list(c.R) == [1.5, 0.4, 0.1] and c.eps == 1e-5 and c.D == 1.0 and c.k == 4.0
    assert len(np.unique(c.xyz_s, axis=0)) == c.n_s
    z = c.xyz_s[:, 2]
    assert abs(z.min()) < 1e-12 and abs(z.max() - 3.0) < 1e-9  # semi-span of 3 chords


def test_seed_reproduces_a_case():
    a = synth.airfoil_case(300, 5, displacement="horns", seed=7)
    b = synth.airfoil_case(300, 5, displacement="horns", seed=7)
    c = synth.airfoil_case(300, 5, displacement="horns", seed=8)
    assert np.array_equal(a.xyz_s, b.xyz_s) and np.array_equal(a.dS, b.dS)
    assert np.array_equal(a.xyz_v, b.xyz_v) and np.array_equal(a.d_v, b.d_v)
    assert not np.array_equal(a.dS, c.dS)
