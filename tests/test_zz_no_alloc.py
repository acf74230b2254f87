"""The residual entry point that allocates no device memory.

It exists for callers that cannot allocate: code whose device memory is owned
by another allocator (a framework's pool holding the whole GPU), or loops that
must not call cudaMalloc/cudaFree because those calls can synchronise the
device.  It is checked through the C ABI against the ordinary entry point
(hx_rhs of an FP64 Euler context with the same periodic block), on two calls
in a row, since every call reuses the same static scratch array.  This file
is named to be collected last."""
import numpy as np
import pytest

from paper_2006_07964_gb300 import build, hx
from paper_2006_07964_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_RHS = 1e-10   # the residual tolerance of the parity tests


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_noalloc_rhs_matches_hx_rhs_twice():
    torch = pytest.importorskip("torch")
    build.build()
    hx.load()
    for dims, amp in (((30, 26, 20), 0.08), ((24, 24, 24), 0.1)):
        ni, nj, nk = dims
        L = (10.0, 10.0 * nj / ni, 10.0 * nk / ni)
        xyz = W.warped_box(dims, L, amp)
        q0 = W.conservative(1.4, *W.isentropic_vortex(1.4, xyz[0], xyz[1], L=10.0, centre=(5.0, 0.5 * L[1])))
        w = W.Workload("noalloc", [W.Block(xyz, W.periodic_faces(L), q0)], gamma=1.4, mach=0.5, viscous=False)
        ctx = hx.from_workload(w, precision="fp64")
        ref = ctx.rhs(0)
        met = torch.empty((10, nk, nj, ni), dtype=torch.float64, device="cuda")
        ctx.get_metrics(0, met)
        q = torch.tensor(q0, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(2):
            r = torch.full((5, nk, nj, ni), float("nan"), dtype=torch.float64, device="cuda")
            hx.euler_rhs_periodic_noalloc(q, met, r, gamma=1.4)
            outs.append(r.cpu().numpy())
        for r in outs:
            assert _rel(r, ref) < TOL_RHS
        assert _rel(outs[1], outs[0]) < TOL_RHS
        ctx.close()


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    hx.load()
    n = 64
    q = torch.ones((5, n, n, n), dtype=torch.float64, device="cuda")
    met = torch.ones((10, n, n, n), dtype=torch.float64, device="cuda")
    r = torch.zeros((5, n, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(hx.HxError) as ei:
        hx.euler_rhs_periodic_noalloc(q, met, r)
    assert ei.value.name == "HX_ERR_INVALID_ARG"
