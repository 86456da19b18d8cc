"""rbfd_deform_worklist: the volume updates of several meshes in one
persistent work-list launch (Section 4, Eq. 19 and Eq. 23), with the
autotuner's settings.

* Fixed settings with the level grids of cell size R_l: each mesh's result
  equals its own rbfd_deform bit for bit (the same lists, blocks and pair
  arithmetic; only the launch that runs them differs).
* Autotuned settings (cell size R_l or R_l / 2 per mesh, blocks per SM,
  blocks per item): within the mixed-mode bar of rbfd_deform, 1e-5 max|dS|
  (a finer grid changes the order of the sums); a second call with meshes of
  the same sizes takes the cached settings.
* Wall distances computed on the device (d_v = None) as in rbfd_deform.
* The four uneven wings (30k to 250k surface points) at reduced volume, the
  first K greedy steps of each level: the mixed batched form (greedy batch +
  work-list launch) against four sequential plain FP64 single runs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


def wings(n_layers=6):
    return [synth.wing_case(nc, ns, n_layers, displacement="ridge", seed=s, R=(1.5, 0.4), eps=1e-4, D=1.0, k=4.0)
            for s, (nc, ns) in enumerate([(30, 12), (60, 20), (90, 30)])]


def meshes_for(cases, precision=rbfd.MIXED):
    ms = [rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=precision, nc_cap=c.nc_cap) for c in cases]
    rbfd.greedy_batch(ms)
    return ms


def test_worklist_equals_each_mesh_deform():
    cases = wings()
    ms = meshes_for(cases)
    want = [m.deform(c.xyz_v, c.d_v, c.D, c.k) for m, c in zip(ms, cases)]
    outs = [np.full((c.n_v, 3), np.nan, np.float32) for c in cases]
    t = rbfd.deform_worklist(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                             [c.k for c in cases], outs, autotune=False, ctas_per_sm=2, item_blocks=1,
                             cell_div=[1, 1, 1])
    assert t["trials"] == 0 and t["items"] > 0
    for o, w in zip(outs, want):
        assert np.array_equal(o, w)
    # other launch shapes: the same sums
    for cps, ib in ((1, 4), (4, 2)):
        outs2 = [np.empty((c.n_v, 3), np.float32) for c in cases]
        rbfd.deform_worklist(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                             [c.k for c in cases], outs2, autotune=False, ctas_per_sm=cps, item_blocks=ib,
                             cell_div=[1, 1, 1])
        for o, w in zip(outs2, want):
            assert np.array_equal(o, w)
    for m in ms:
        m.close()


def test_worklist_autotuned_and_cached():
    cases = wings()
    ms = meshes_for(cases)
    want = [m.deform(c.xyz_v, c.d_v, c.D, c.k) for m, c in zip(ms, cases)]
    for call in range(2):
        outs = [np.empty((c.n_v, 3), np.float32) for c in cases]
        t = rbfd.deform_worklist(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                                 [c.k for c in cases], outs)
        assert t["cached"] == (call == 1)
        assert (t["trials"] > 0) == (call == 0)
        assert all(d in (1, 2) for d in t["cell_div"]) and 1 <= t["ctas_per_sm"] <= 8
        for c, o, w in zip(cases, outs, want):
            S0 = float(np.sqrt((c.dS**2).sum(1)).max())
            assert np.abs(o.astype(np.float64) - w).max() <= 1e-5 * S0 + np.abs(w).max() * 2.0**-24
        # the tuner's discarded trials leave the pair counters alone: the
        # volume pairs of one update, as rbfd_deform counts them
    # a fine grid everywhere gives the same update within the mixed bar
    outs = [np.empty((c.n_v, 3), np.float32) for c in cases]
    rbfd.deform_worklist(ms, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                         [c.k for c in cases], outs, autotune=False, cell_div=[2, 2, 2])
    for c, o, w in zip(cases, outs, want):
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        assert np.abs(o.astype(np.float64) - w).max() <= 1e-5 * S0 + np.abs(w).max() * 2.0**-24
    for m in ms:
        m.close()


def test_worklist_wall_distance_on_device_and_device_arrays():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    cases = wings()
    ms = meshes_for(cases)
    want = [m.deform(c.xyz_v, None, c.D, c.k) for m, c in zip(ms, cases)]
    outs = [np.empty((c.n_v, 3), np.float32) for c in cases]
    rbfd.deform_worklist(ms, [c.xyz_v for c in cases], None, [c.D for c in cases], [c.k for c in cases], outs,
                         autotune=False, cell_div=[1, 1, 1])
    for o, w in zip(outs, want):
        assert np.array_equal(o, w)
    # meshes made from device arrays take device volume arrays
    md = [rbfd.Mesh(torch.from_numpy(c.xyz_s).to(dev), torch.from_numpy(c.dS).to(dev), c.R, c.eps) for c in cases]
    rbfd.greedy_batch(md)
    outd = [torch.empty((c.n_v, 3), dtype=torch.float32, device=dev) for c in cases]
    rbfd.deform_worklist(md, [torch.from_numpy(c.xyz_v).to(dev) for c in cases],
                         [torch.from_numpy(c.d_v).to(dev) for c in cases], [c.D for c in cases],
                         [c.k for c in cases], outd, autotune=False, cell_div=[1, 1, 1])
    for m, c, o in zip(ms, cases, outd):
        assert np.array_equal(o.cpu().numpy(), m.deform(c.xyz_v, c.d_v, c.D, c.k))
    for m in ms + md:
        m.close()


def test_worklist_argument_errors():
    cases = wings()[:2]
    ms = meshes_for(cases)
    f = rbfd.Mesh(cases[0].xyz_s, cases[0].dS, cases[0].R, cases[0].eps, precision=rbfd.FP64)
    f.greedy()
    a2 = synth.airfoil_case(200, 4, displacement="bump", seed=0)
    m2 = rbfd.Mesh(a2.xyz_s, a2.dS, a2.R, a2.eps)
    m2.greedy()
    fresh = rbfd.Mesh(cases[1].xyz_s, cases[1].dS, cases[1].R, cases[1].eps)
    out = [np.empty((c.n_v, 3), np.float32) for c in cases]
    for bad, status in (([ms[0], f], rbfd.EINVAL), ([ms[0], fresh], rbfd.ESTATE)):
        with pytest.raises(rbfd.RbfdError) as ei:
            rbfd.deform_worklist(bad, [c.xyz_v for c in cases], [c.d_v for c in cases], [1.0, 1.0], [4.0, 4.0],
                                 out)
        assert ei.value.status == status
    with pytest.raises(rbfd.RbfdError) as ei:
        rbfd.deform_worklist([ms[0], m2], [cases[0].xyz_v, a2.xyz_v], [cases[0].d_v, a2.d_v], [1.0, 2.0],
                             [4.0, 0.0], [out[0], np.empty((a2.n_v, 2), np.float32)])
    assert ei.value.status == rbfd.EINVAL
    for m in ms + [f, m2, fresh]:
        m.close()


def test_four_uneven_wings_first_steps_against_fp64_single_runs():
    """The four-wing workload (30k, 80k, 150k, 250k surface points), volumes
    reduced to 20 layers (0.6M to 5M points), the first K = 120 greedy steps of
    each level.  Mixed batched form: the four greedy runs side by side and one
    work-list launch for the four volume updates.  Reference: four
    sequential FP64 runs (rbfd_greedy + rbfd_deform per wing).  Where the
    two control sequences agree the volume updates must agree within 1e-5
    max|dS|; a split is allowed only where the oracle's replay shows both
    sequences pick argmaxes of Eq. 12 up to rounding (a near-tie), and then
    the mixed update is held to the oracle's on its own controls and weights
    at sampled volume points.  The oracle replays the smallest wing's mixed
    sequence in any case."""
    from test_gpu_parity import check_replay, gpu_result

    K = 120
    cases = synth.make_config_set("wings4_30k_250ks_3m_25mv_ridge", n_layers=20, nc_cap=K)
    mixed = meshes_for(cases)
    outs = [np.empty((c.n_v, 3), np.float32) for c in cases]
    t = rbfd.deform_worklist(mixed, [c.xyz_v for c in cases], [c.d_v for c in cases], [c.D for c in cases],
                             [c.k for c in cases], outs)
    print("autotuned:", t)
    check_replay(cases[0], mixed[0].levels())
    for c, m, o in zip(cases, mixed, outs):
        f = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps, precision=rbfd.FP64, nc_cap=K)
        f.greedy()
        S0 = float(np.sqrt((c.dS**2).sum(1)).max())
        same = all(np.array_equal(a.idx, b.idx) for a, b in zip(m.levels(), f.levels()))
        if same:
            want = f.deform(c.xyz_v.astype(np.float64), c.d_v.astype(np.float64), c.D, c.k)
            err = np.abs(o.astype(np.float64) - want).max()
            assert err <= 1e-5 * S0 + np.abs(want).max() * 2.0**-24, f"{c.name}: {err / S0:g} max|dS|"
        else:
            print(f"{c.name}: mixed and FP64 sequences split at a near-tie")
            check_replay(c, m.levels())
            check_replay(c, f.levels())
            vi = np.random.default_rng(0).choice(c.n_v, 4000, replace=False)
            want = oracle.deform(gpu_result(m.levels(), S0), c.xyz_s, c.R, c.xyz_v[vi], c.d_v[vi], c.k, c.D,
                                 n_threads=NT)
            assert np.abs(o[vi].astype(np.float64) - want).max() <= 1e-5 * S0 + np.abs(want).max() * 2.0**-24
        f.close()
        m.close()
