"""The residual entry point that allocates no device memory.

It exists for callers that cannot allocate: code whose device memory is owned
by another allocator (a framework's pool holding the whole GPU), or loops that
must not call cudaMalloc/cudaFree because those calls can synchronise the
device.  It is checked through the C ABI against the ordinary entry point
(hx_rhs of an FP64 Euler context with the same periodic block) and against
the FP64 oracle, on two calls in a row, since every call reuses the same
static scratch array.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
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
        # and directly against the FP64 oracle's residual of the same block
        P = oracle.from_workload(w)
        P.rhs()
        assert _rel(outs[1], P.get_rhs(0)) < TOL_RHS
        ctx.close()


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    build.build()
    hx.load()
    n = 64
    q = torch.ones((5, n, n, n), dtype=torch.float64, device="cuda")
    met = torch.ones((10, n, n, n), dtype=torch.float64, device="cuda")
    r = torch.zeros((5, n, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(hx.HxError) as ei:
        hx.euler_rhs_periodic_noalloc(q, met, r)
    assert ei.value.name == "HX_ERR_INVALID_ARG"


def test_noalloc_rejects_memory_of_the_host():
    """Arrays must be memory of the current device: a host pointer is refused
    by the library before any kernel runs (called through the C ABI
    directly, past the Python wrapper's own check)."""
    pytest.importorskip("torch")
    build.build()
    lib = hx.load()
    n = 8
    host = np.zeros((10, n, n, n))
    import torch
    dev = torch.zeros((10, n, n, n), dtype=torch.float64, device="cuda")
    hp = host.ctypes.data
    dp = dev.data_ptr()
    for q, met, r in ((hp, dp, dp), (dp, hp, dp), (dp, dp, hp)):
        rc = lib.hx_euler_rhs_periodic_noalloc(n, n, n, 1.4, q, met, r, ctypes.c_void_p(0))
        assert hx.ERRORS.get(rc) == "HX_ERR_INVALID_ARG"
