"""Thin ctypes binding of libhx.so (the C ABI declared in include/hx.h).

Argument marshalling only: every step of the RK-stage path runs in the CUDA
kernels of the library.  Function names follow the C entry points; the
``Context`` class bundles them for one ``hx_ctx``.  Arrays are numpy arrays
(host memory) or CUDA tensors exposing ``data_ptr()`` (device memory, e.g.
torch); layouts are those of include/hx.h ([nf][nk][nj][ni], double).

There is no CPU fallback: if libhx.so is missing or no CUDA device is
present, the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhx.so")

HX_OK = 0
ERRORS = {
    -1: "HX_ERR_INVALID_ARG", -2: "HX_ERR_STATE", -3: "HX_ERR_TOPOLOGY", -4: "HX_ERR_BAD_GRID",
    -5: "HX_ERR_OOM", -6: "HX_ERR_CUDA", -7: "HX_ERR_NONFINITE", -8: "HX_ERR_UNPHYSICAL", -9: "HX_ERR_TIMEOUT",
    -10: "HX_ERR_BOUNDS",
}
FACE = {"periodic": 0, "interface": 1, "wall": 2, "farfield": 3}
HX_FP64, HX_MIXED = 0, 1

# Every function declared in include/hx.h (checked by the test suite).
EXPORTS = (
    "hx_config_default", "hx_create", "hx_add_block", "hx_set_face", "hx_finalize", "hx_compute_metrics",
    "hx_set_state", "hx_get_state", "hx_get_metrics", "hx_compute_dt", "hx_step", "hx_step_multi", "hx_rhs",
    "hx_get_gradients", "hx_profile_step", "hx_launches_per_step", "hx_points", "hx_device_bytes",
    "hx_last_error", "hx_destroy", "hx_euler_rhs_periodic_noalloc", "hx_tuning", "hx_step_cfl", "hx_residual",
    "hx_set_face_transform", "hx_step_local", "hx_local_dt",
)


class hx_config(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("mach", ctypes.c_double), ("reynolds", ctypes.c_double),
        ("prandtl", ctypes.c_double), ("viscous", ctypes.c_int), ("mu_law", ctypes.c_int),
        ("sutherland_s", ctypes.c_double), ("precision", ctypes.c_int), ("scheme", ctypes.c_int),
        ("mem_cap_bytes", ctypes.c_size_t), ("autotune", ctypes.c_int), ("debug_poison", ctypes.c_int),
    ]


class hx_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


class HxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "HX_ERR"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "HX_ERR")


_lib = None


def load(path=None):
    """Loads libhx.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HX_LIB") or LIB_PATH   # HX_LIB: another build (the checking one)
    if not os.path.exists(path):
        raise OSError("libhx.so is not built (%s); run paper_2006_07964_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    CTX = ctypes.c_void_p
    sig = {
        "hx_config_default": (I, [ctypes.POINTER(hx_config)]),
        "hx_create": (I, [ctypes.POINTER(CTX), ctypes.POINTER(hx_config), VP]),
        "hx_add_block": (I, [CTX, I, I, I, VP, ctypes.POINTER(I)]),
        "hx_set_face": (I, [CTX, I, I, I, I, I, P]),
        "hx_set_face_transform": (I, [CTX, I, I, ctypes.POINTER(ctypes.c_int)]),
        "hx_finalize": (I, [CTX]),
        "hx_compute_metrics": (I, [CTX]),
        "hx_set_state": (I, [CTX, I, VP, I]),
        "hx_get_state": (I, [CTX, I, VP, I]),
        "hx_get_metrics": (I, [CTX, I, VP, I]),
        "hx_compute_dt": (I, [CTX, D, P, P]),
        "hx_step": (I, [CTX, I, D]),
        "hx_step_multi": (I, [CTX, I, P]),
        "hx_rhs": (I, [CTX, I, VP, I]),
        "hx_get_gradients": (I, [CTX, I, VP, I]),
        "hx_profile_step": (I, [CTX, I, D, ctypes.POINTER(hx_kernel_stat), I, ctypes.POINTER(I)]),
        "hx_launches_per_step": (I, [CTX]),
        "hx_points": (ctypes.c_longlong, [CTX]),
        "hx_device_bytes": (ctypes.c_size_t, [CTX]),
        "hx_last_error": (ctypes.c_char_p, [CTX]),
        "hx_destroy": (None, [CTX]),
        "hx_euler_rhs_periodic_noalloc": (I, [I, I, I, D, VP, VP, VP, VP]),
        "hx_tuning": (I, [CTX, ctypes.POINTER(I), ctypes.POINTER(I), P]),
        "hx_step_cfl": (I, [CTX, I, D, I, P]),
        "hx_step_local": (I, [CTX, I, D]),
        "hx_local_dt": (I, [CTX, I, D, P, I]),
        "hx_residual": (I, [CTX, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, nvals=None):
    """(address, on_device) of a numpy array or a CUDA tensor.  A CUDA
    tensor's producers on torch's current stream of its device are waited
    for first: the library works on its own stream, which is not ordered
    after torch's."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise ValueError("device tensors must be contiguous float64")
        if nvals is not None and a.numel() != nvals:
            raise ValueError("expected %d values, got %d" % (nvals, a.numel()))
        if a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr(), int(bool(a.is_cuda))
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("host arrays must be C-contiguous float64 numpy arrays")
    if nvals is not None and a.size != nvals:
        raise ValueError("expected %d values, got %d" % (nvals, a.size))
    return a.ctypes.data, 0


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_config(**kw):
    cfg = hx_config()
    load().hx_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": HX_FP64, "mixed": HX_MIXED}[v]
        setattr(cfg, k, v)
    return cfg


class Context:
    """One hx_ctx: blocks, faces, metrics, state, steps (see include/hx.h)."""

    def __init__(self, stream=None, **cfg):
        self._lib = load()
        self.cfg = default_config(**cfg)
        h = ctypes.c_void_p()
        rc = self._lib.hx_create(ctypes.byref(h), ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0))
        if rc:
            raise HxError(rc, self._lib.hx_last_error(None).decode())
        self._h = h
        self.dims = []

    def _check(self, rc):
        if rc:
            raise HxError(rc, self._lib.hx_last_error(self._h).decode())

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.hx_destroy(h)

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- set-up
    def add_block(self, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        nk, nj, ni = xyz.shape[1:]
        bid = ctypes.c_int()
        self._check(self._lib.hx_add_block(self._h, ni, nj, nk, xyz.ctypes.data, ctypes.byref(bid)))
        self.dims.append((nk, nj, ni))
        return bid.value

    def set_face(self, block, face, kind, nbr=-1, nbr_face=-1, translate=(0.0, 0.0, 0.0), transform=None):
        """transform: axis a of `block` runs along axis |t[a]|-1 of the
        neighbour, reversed when t[a] < 0 (None: identity)."""
        kind = FACE[kind] if isinstance(kind, str) else int(kind)
        tr = np.ascontiguousarray(translate, dtype=np.float64)
        self._check(self._lib.hx_set_face(self._h, block, face, kind, nbr, nbr_face, _dp(tr)))
        if transform is not None and tuple(transform) != (1, 2, 3):
            tf = (ctypes.c_int * 3)(*[int(t) for t in transform])
            self._check(self._lib.hx_set_face_transform(self._h, block, face, tf))

    def finalize(self):
        self._check(self._lib.hx_finalize(self._h))

    def compute_metrics(self):
        self._check(self._lib.hx_compute_metrics(self._h))

    # ---- state
    def _n(self, block, nf):
        nk, nj, ni = self.dims[block]
        return nf * nk * nj * ni

    def set_state(self, block, q):
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        p, dev = _ptr(q, self._n(block, 5))
        self._check(self._lib.hx_set_state(self._h, block, p, dev))

    def _get(self, fn, block, nf, out):
        if out is None:
            out = np.empty((nf,) + self.dims[block])
        p, dev = _ptr(out, self._n(block, nf))
        self._check(fn(self._h, block, p, dev))
        return out

    def get_state(self, block, out=None):
        return self._get(self._lib.hx_get_state, block, 5, out)

    def get_metrics(self, block, out=None):
        return self._get(self._lib.hx_get_metrics, block, 10, out)

    def rhs(self, block, out=None):
        return self._get(self._lib.hx_rhs, block, 5, out)

    def get_gradients(self, block, out=None):
        return self._get(self._lib.hx_get_gradients, block, 12, out)

    # ---- time stepping
    def compute_dt(self, cfl):
        per = np.empty(len(self.dims))
        g = ctypes.c_double()
        self._check(self._lib.hx_compute_dt(self._h, float(cfl), ctypes.byref(g), _dp(per)))
        return g.value, per

    def step(self, nsteps, dt):
        if np.ndim(dt) == 0:
            self._check(self._lib.hx_step(self._h, int(nsteps), float(dt)))
        else:
            d = np.ascontiguousarray(dt, dtype=np.float64)
            if d.shape != (len(self.dims),):
                raise ValueError("one dt per block")
            self._check(self._lib.hx_step_multi(self._h, int(nsteps), _dp(d)))

    def step_cfl(self, nsteps, cfl, per_block=False):
        """nsteps RK3 steps with dt chosen on the device each step; returns
        the simulated time advanced (sum of the global dt)."""
        t = ctypes.c_double()
        self._check(self._lib.hx_step_cfl(self._h, int(nsteps), float(cfl), int(bool(per_block)), ctypes.byref(t)))
        return t.value

    def step_local(self, nsteps, cfl):
        """nsteps RK3 steps of local time stepping (each node its own dt)."""
        self._check(self._lib.hx_step_local(self._h, int(nsteps), float(cfl)))

    def local_dt(self, block, cfl):
        """Per-node local time steps of the current state, [nk][nj][ni]."""
        out = np.empty(self.dims[block])
        self._check(self._lib.hx_local_dt(self._h, block, float(cfl), _dp(out), 0))
        return out

    def residual(self):
        """RMS of R over all nodes, per conservative variable (5 values)."""
        out = np.empty(5)
        self._check(self._lib.hx_residual(self._h, _dp(out)))
        return out

    def profile_step(self, nsteps, dt):
        out = (hx_kernel_stat * 16)()
        n = ctypes.c_int()
        self._check(self._lib.hx_profile_step(self._h, int(nsteps), float(dt), out, 16, ctypes.byref(n)))
        return {out[i].name.decode(): (out[i].launches, out[i].total_ms) for i in range(n.value)}

    def tuning(self):
        """{direction: {"chosen": (tp, na), "candidates": {(tp, na): ms}}}."""
        var = (ctypes.c_int * 3)()
        shp = (ctypes.c_int * 18)()
        ms = (ctypes.c_double * 9)()
        self._check(self._lib.hx_tuning(self._h, var, shp, ms))
        out = {}
        for d, name in enumerate(("xi", "eta", "zeta")):
            cands = {}
            for v in range(3):
                key = "%dx%d" % (shp[(d * 3 + v) * 2], shp[(d * 3 + v) * 2 + 1])
                cands[key] = ms[d * 3 + v]
            out[name] = {"chosen": "%dx%d" % (shp[(d * 3 + var[d]) * 2], shp[(d * 3 + var[d]) * 2 + 1]),
                         "candidates_ms": cands}
        return out

    @property
    def launches_per_step(self):
        return self._lib.hx_launches_per_step(self._h)

    @property
    def points(self):
        return self._lib.hx_points(self._h)

    @property
    def device_bytes(self):
        return self._lib.hx_device_bytes(self._h)


def euler_rhs_periodic_noalloc(q, met, r_out, gamma=1.4, stream=None):
    """Residual of one fully periodic Euler block in FP64 without any device
    allocation (hx_euler_rhs_periodic_noalloc); q [5][nk][nj][ni], met
    [10][nk][nj][ni] and r_out [5][nk][nj][ni] are contiguous float64 CUDA
    tensors on one device, which the call makes current.  stream: a
    cudaStream_t handle, default torch's current stream of that device, so
    that the call is ordered after the tensors' producers.  For callers that
    cannot allocate device memory; see include/hx.h for the size limit and
    the shared-scratch caveat."""
    import torch
    for t in (q, met, r_out):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError("q, met and r_out must be CUDA tensors")
    if not (q.device == met.device == r_out.device):
        raise ValueError("q, met and r_out must be on one device")
    _, nk, nj, ni = q.shape
    for t, nf in ((q, 5), (met, 10), (r_out, 5)):
        if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != nf * nk * nj * ni:
            raise ValueError("expected a contiguous float64 tensor of %d values" % (nf * nk * nj * ni))
    with torch.cuda.device(q.device):
        if stream is None:
            stream = torch.cuda.current_stream(q.device).cuda_stream
        rc = load().hx_euler_rhs_periodic_noalloc(ni, nj, nk, float(gamma), q.data_ptr(), met.data_ptr(),
                                                  r_out.data_ptr(), ctypes.c_void_p(stream or 0))
    if rc:
        raise HxError(rc, "hx_euler_rhs_periodic_noalloc failed")
    return r_out


def from_workload(w, precision="fp64", stream=None, autotune=1, mem_cap_bytes=0, scheme=0, debug_poison=0):
    """Context with the blocks, faces, metrics and initial state of a
    workload from ``paper_2006_07964_gb300.workloads``."""
    ctx = Context(stream=stream, gamma=w.gamma, mach=w.mach, reynolds=w.reynolds, prandtl=w.prandtl,
                  viscous=int(w.viscous), mu_law=w.mu_law, sutherland_s=w.sutherland_s, precision=precision,
                  autotune=autotune, mem_cap_bytes=mem_cap_bytes, scheme=scheme, debug_poison=debug_poison)
    for blk in w.blocks:
        ctx.add_block(blk.xyz)
    for b, blk in enumerate(w.blocks):
        for f, face in enumerate(blk.faces):
            ctx.set_face(b, f, face.kind, face.nbr, face.nbr_face, face.translate, face.transform)
    ctx.finalize()
    ctx.compute_metrics()
    for b, blk in enumerate(w.blocks):
        ctx.set_state(b, blk.q0)
    return ctx


PROBE_PATH = os.path.join(HERE, "libhx_probe.so")
PROBE_EXPORTS = ("hx_probe_fma_peaks",)   # include/hx_probe.h


def probe_fma_peaks():
    """Measured (fp64_tflops, fp32_tflops) of the current GPU from
    libhx_probe.so (include/hx_probe.h): the FMA-chain probe the benchmark's
    ALU roofline divides by."""
    lib = ctypes.CDLL(PROBE_PATH)
    fn = lib.hx_probe_fma_peaks
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3
    f64, f32, ms = ctypes.c_double(), ctypes.c_double(), (ctypes.c_double * 2)()
    rc = fn(ctypes.byref(f64), ctypes.byref(f32), ms)
    if rc:
        raise HxError(rc, "hx_probe_fma_peaks failed")
    return f64.value, f32.value
