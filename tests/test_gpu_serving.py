"""Time stepping and serving on the GPU: a mesh whose geometry stays resident
while the displacement changes, and the request loop (rbfd_server_*) whose
results must not depend on what else runs beside them."""
import numpy as np
import pytest

import oracle
from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu


def _airfoil(seed=2):
    return synth.airfoil_case(600, 9, displacement="horns", seed=seed, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)


def _wing(seed=3):
    return synth.wing_case(40, 15, 6, displacement="ridge", seed=seed, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0)


def _fresh(c, dS, precision=rbfd.MIXED):
    m = rbfd.Mesh(c.xyz_s, dS, c.R, c.eps, precision=precision)
    m.greedy()
    out = m.deform(c.xyz_v, c.d_v, c.D, c.k)
    lv = m.levels()
    m.close()
    return lv, out


def _close(a, b, S0):
    return np.abs(a.astype(np.float64) - b.astype(np.float64)).max() <= 1e-5 * S0 + np.abs(b).max() * 2.0**-23


def test_set_displacement_and_registered_volume_match_fresh_meshes():
    c = _airfoil()
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    m.set_volume(c.xyz_v, c.d_v)
    for step, scale in enumerate([1.0, 1.3, 0.7, 1.6]):
        dS = c.dS * scale
        m.set_displacement(dS)
        m.greedy()
        got = m.deform_volume(c.D, c.k)
        lv, want = _fresh(c, dS)
        for x, y in zip(m.levels(), lv):
            assert np.array_equal(x.idx, y.idx)
        S0 = float(np.sqrt((dS**2).sum(1)).max())
        assert _close(got, want, S0), f"time step {step}"
    # and against the oracle for one step
    ref = oracle.greedy(c.xyz_s, c.dS * 0.7, c.R, c.eps)
    m.set_displacement(c.dS * 0.7)
    m.greedy()
    for x, r in zip(m.levels(), ref.idx):
        assert np.array_equal(x.idx, r)
    m.close()


def test_server_results_same_alone_and_in_the_mix():
    a, w = _airfoil(), _wing()
    srv = rbfd.Server(slots=3)
    ia = srv.add_mesh(a.xyz_s, a.xyz_v, a.d_v, a.R, a.eps, a.D, a.k)
    iw = srv.add_mesh(w.xyz_s, w.xyz_v, w.d_v, w.R, w.eps, w.D, w.k)
    # an ice-growth sequence on each mesh, interleaved
    jobs = []
    for t in range(6):
        s = 0.5 + 0.25 * t
        jobs.append((ia, a, a.dS * s))
        jobs.append((iw, w, w.dS * s))
    tickets = [srv.submit(mid, dS) for mid, _, dS in jobs]
    results = [srv.wait(t, timeout_s=120.0) for t in tickets]
    for (mid, c, dS), t, (rc, out) in zip(jobs, tickets, results):
        assert rc in (rbfd.OK, rbfd.ENOTCONV)
        _, want = _fresh(c, dS)
        S0 = float(np.sqrt((dS**2).sum(1)).max())
        assert _close(out, want, S0)
        q, r, tot = srv.times(t)
        assert q >= 0 and r > 0 and tot >= r
    # the same request alone on an idle server
    alone = rbfd.Server(slots=1)
    j = alone.add_mesh(w.xyz_s, w.xyz_v, w.d_v, w.R, w.eps, w.D, w.k)
    rc, out_alone = alone.wait(alone.submit(j, jobs[5][2]), timeout_s=120.0)
    assert _close(out_alone, results[5][1], float(np.sqrt((jobs[5][2] ** 2).sum(1)).max()))
    alone.close()
    srv.close()


def test_server_admission_by_memory_budget():
    """With a budget that holds one instance only, requests on two meshes
    still all complete (the second mesh waits for memory, not forever)."""
    a, w = _airfoil(), _wing()
    probe = rbfd.Server(slots=2)
    probe.close()
    srv = rbfd.Server(slots=2, mem_budget_bytes=200 << 20)
    ia = srv.add_mesh(a.xyz_s, a.xyz_v, a.d_v, a.R, a.eps, a.D, a.k)
    tickets = [srv.submit(ia, a.dS * (1 + 0.1 * i)) for i in range(4)]
    for t in tickets:
        rc, out = srv.wait(t, timeout_s=120.0)
        assert rc in (rbfd.OK, rbfd.ENOTCONV) and np.isfinite(out).all()
    srv.close()


def test_server_rejects_bad_requests():
    a = _airfoil()
    srv = rbfd.Server(slots=1, max_queue=1)
    ia = srv.add_mesh(a.xyz_s, a.xyz_v, a.d_v, a.R, a.eps, a.D, a.k)
    with pytest.raises(rbfd.RbfdError):
        srv.submit(ia + 7, a.dS)
    srv.close()


def test_fused_volume_stage_same_bits_alone_and_in_the_mix():
    """Four slots with fuse_volume: the volume updates of requests whose
    greedy is done run in one work-list launch (cells of size R_l: the same
    sums as a request alone).  One slot: every request alone.  Each mesh's requests run in order
    on its own resident instance (warm starts) in both servers, so every
    result must agree bit for bit."""
    cases = [synth.wing_case(40, 15, 6, displacement="ridge", seed=s, R=(1.5, 0.4), eps=1e-3, D=1.0, k=4.0)
             for s in (3, 4, 5)] + [_airfoil(seed=2), _airfoil(seed=6)]
    results = []
    for slots in (4, 1):
        srv = rbfd.Server(slots=slots, fuse_volume=True)
        ids = [srv.add_mesh(c.xyz_s, c.xyz_v, c.d_v, c.R, c.eps, c.D, c.k) for c in cases]
        tickets = []
        for t in range(4):
            for mid, c in zip(ids, cases):
                tickets.append(srv.submit(mid, c.dS * (0.6 + 0.2 * t)))
        outs = []
        for t in tickets:
            rc, out = srv.wait(t, timeout_s=120.0)
            assert rc in (rbfd.OK, rbfd.ENOTCONV)
            outs.append(out)
        results.append(outs)
        srv.close()
    for a, b in zip(*results):
        assert np.array_equal(a, b)
