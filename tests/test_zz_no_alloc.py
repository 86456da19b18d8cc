"""rbfd_deform_noalloc: the volume update for callers that cannot allocate
device memory during the call (solvers with a fixed device-memory budget,
hosts that keep cudaMalloc/cudaFree off their hot path).  Its result must
match rbfd_deform's, within the tolerances the parity tests use, on two calls
in a row (the scratch array keeps the previous call's contents).

This file is collected last on purpose, and it must also pass when run alone
in a fresh process."""
import numpy as np
import pytest

from paper_2107_13887_gb300 import rbfd, synth

pytestmark = pytest.mark.gpu


def _mesh_and_volume(torch, precision):
    c = synth.airfoil_case(600, 150, displacement="horns", seed=3, R=(1.0, 0.2), eps=1e-5, D=2.0, k=5.0)
    dev = torch.device("cuda:0")
    m = rbfd.Mesh(torch.from_numpy(c.xyz_s).to(dev), torch.from_numpy(c.dS).to(dev), c.R, c.eps,
                  precision=precision)
    m.greedy()
    xv = torch.from_numpy(c.xyz_v).to(dev)
    dv = torch.from_numpy(c.d_v).to(dev)
    return c, m, xv, dv


@pytest.mark.parametrize("precision", [rbfd.MIXED, rbfd.FP64], ids=["mixed", "fp64"])
def test_noalloc_matches_deform_on_two_calls(precision):
    """Mixed mode: rbfd_deform's FP32-input sweep and this call's sweep on
    FP64-packed points agree within the mixed-mode bound, 1e-5 max|dS|.  FP64
    mode: both form the same per-point FP64 sums (only the grouping of points
    into blocks differs), held to 1e-10 max|dS|, the FP64 volume bound.  The
    second call must not change the device's free memory (nothing allocated)."""
    torch = pytest.importorskip("torch")
    c, m, xv, dv = _mesh_and_volume(torch, precision)
    assert c.n_v == 90000 and c.n_v <= 131072
    want = m.deform(xv, dv, c.D, c.k).cpu().numpy().astype(np.float64)
    S0 = float(np.sqrt((c.dS**2).sum(1)).max())
    rel = 1e-5 if precision == rbfd.MIXED else 1e-10
    tol = rel * S0 + np.abs(want).max() * 2.0**-24
    for call in range(2):
        out = torch.full((c.n_v, 2), float("nan"), dtype=torch.float32, device=xv.device)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        m.deform_noalloc(xv, dv, c.D, c.k, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call may still load kernels lazily
            assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= tol
    # a second volume of a different size reuses the same array
    half = c.n_v // 2 + 17
    want_h = m.deform(xv[:half].contiguous(), dv[:half].contiguous(), c.D, c.k).cpu().numpy().astype(np.float64)
    out = torch.empty((half, 2), dtype=torch.float32, device=xv.device)
    m.deform_noalloc(xv[:half].contiguous(), dv[:half].contiguous(), c.D, c.k, out)
    assert np.abs(out.cpu().numpy().astype(np.float64) - want_h).max() <= tol
    m.close()


def test_noalloc_rejects_oversize_and_host_memory():
    torch = pytest.importorskip("torch")
    c, m, xv, dv = _mesh_and_volume(torch, rbfd.MIXED)
    big = 131072 + 1
    xb = torch.zeros((big, 2), dtype=torch.float32, device=xv.device)
    db = torch.zeros(big, dtype=torch.float32, device=xv.device)
    ob = torch.empty((big, 2), dtype=torch.float32, device=xv.device)
    with pytest.raises(rbfd.RbfdError) as ei:
        m.deform_noalloc(xb, db, c.D, c.k, ob)
    assert ei.value.status == rbfd.EINVAL and "131072" in str(ei.value)
    with pytest.raises(rbfd.RbfdError) as ei:
        m.deform_noalloc(xv.cpu(), dv.cpu(), c.D, c.k, torch.empty((c.n_v, 2)))
    assert ei.value.status == rbfd.EINVAL
    # wrong dtype, shape or layout of out is refused before the library call
    for bad in (torch.empty((c.n_v, 2), dtype=torch.float64, device=xv.device),
                torch.empty((c.n_v - 1, 2), dtype=torch.float32, device=xv.device),
                torch.empty((2, c.n_v), dtype=torch.float32, device=xv.device).t()):
        with pytest.raises(rbfd.RbfdError) as ei:
            m.deform_noalloc(xv, dv, c.D, c.k, bad)
        assert ei.value.status == rbfd.EINVAL
    m.close()
