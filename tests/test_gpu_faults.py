"""Failure behaviour, injected on the host (no GPU fault, no real memory
exhaustion, nothing that traps):

* RBFD_TEST_ENOMEM_AT=N makes the N-th device allocation fail as if the
  device were out of memory: every call on the path (create, greedy, volume
  update) must return RBFD_ENOMEM with a message, leave nothing half made,
  and the library must work normally once the variable is gone;
* a queued serving request cancelled with rbfd_cancel never runs and never
  writes its output; the requests around it complete as usual;
* (the bounded grid-barrier wait and the split greedy's failing exchange are
  tested in test_gpu_parity.py and test_gpu_split.py.)
"""
import numpy as np
import pytest

from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu


def _case():
    return synth.airfoil_case(600, 9, displacement="horns", seed=2, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)


def _pipeline(c):
    m = rbfd.Mesh(c.xyz_s, c.dS, c.R, c.eps)
    try:
        m.greedy()
        return m.levels(), m.deform(c.xyz_v, None, c.D, c.k)
    finally:
        m.close()


def test_injected_out_of_memory_at_every_allocation(monkeypatch):
    c = _case()
    want_levels, want = _pipeline(c)
    failures = 0
    for n in range(1, 80):
        monkeypatch.setenv("RBFD_TEST_ENOMEM_AT", str(n))
        try:
            lv, out = _pipeline(c)
        except rbfd.RbfdError as exc:
            assert exc.status == rbfd.ENOMEM, f"allocation {n}: {exc}"
            assert "injected" in str(exc)
            failures += 1
            continue
        # the n-th allocation came after the pipeline (or was served by the
        # pool): the results are the ordinary ones
        assert np.array_equal(out, want)
        monkeypatch.delenv("RBFD_TEST_ENOMEM_AT")
    monkeypatch.delenv("RBFD_TEST_ENOMEM_AT", raising=False)
    assert failures > 0
    lv, out = _pipeline(c)  # nothing was left broken
    assert np.array_equal(out, want)
    for a, b in zip(lv, want_levels):
        assert np.array_equal(a.idx, b.idx) and np.array_equal(a.alpha, b.alpha)


def test_cancelled_request_never_runs():
    c = _case()
    srv = rbfd.Server(slots=1)
    mid = srv.add_mesh(c.xyz_s, c.xyz_v, c.d_v, c.R, c.eps, c.D, c.k)
    outs = [np.full((c.n_v, 2), np.nan, np.float32) for _ in range(8)]
    tickets = [srv.submit(mid, c.dS * (0.5 + 0.1 * i), out=o) for i, o in enumerate(outs)]
    cancelled = []
    for t in tickets[4:]:
        try:
            srv.cancel(t)
            cancelled.append(t)
        except rbfd.RbfdError as exc:  # it had started already
            assert exc.status in (rbfd.EBUSY, rbfd.ESTATE)
    assert cancelled  # (one slot: the later requests were still queued)
    for t, o in zip(tickets, outs):
        if t in cancelled:
            with pytest.raises(rbfd.RbfdError) as ei:
                srv.poll(t)  # finished with status RBFD_ECANCELED
            assert ei.value.status == rbfd.ECANCELED
            with pytest.raises(rbfd.RbfdError) as ei:
                srv.wait(t, timeout_s=60.0)
            assert ei.value.status == rbfd.ECANCELED
            assert np.isnan(o).all()  # never written
        else:
            rc, out = srv.wait(t, timeout_s=120.0)
            assert rc in (rbfd.OK, rbfd.ENOTCONV) and np.isfinite(out).all()
    with pytest.raises(rbfd.RbfdError) as ei:
        srv.cancel(tickets[0])  # finished
    assert ei.value.status == rbfd.ESTATE
    with pytest.raises(rbfd.RbfdError) as ei:
        srv.cancel(10**9)
    assert ei.value.status == rbfd.EINVAL
    srv.close()
