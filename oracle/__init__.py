"""FP64 CPU oracle of the per-RK-stage residual evaluation (test infrastructure).

This package is the independent reference the CUDA path is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library in ``paper_2006_07964_gb300`` never
does, and the two share no code.  The arithmetic lives in ``hx_oracle.c``
(plain C, IEEE double, built with ``-ffp-contract=off``); this module only
builds it with gcc and marshals arrays through ctypes.

Every function of ``hx_oracle.c`` cites the equation or section of the paper
it follows (Ye et al., "Accelerating CFD simulation with high order finite
difference method on curvilinear coordinates for modern GPU clusters").
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PERIODIC, INTERFACE, WALL, FARFIELD = 0, 1, 2, 3
KIND = {"periodic": PERIODIC, "interface": INTERFACE, "wall": WALL, "farfield": FARFIELD}

_lib = None


def build(force=False):
    """Compile hx_oracle.c into liboracle.so (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def load():
    """Loads liboracle.so (building it if needed).  HX_ORACLE_LIB names
    another build of hx_oracle.c to load instead; the mutation tests use it
    to run the pins against copies with planted mistakes."""
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(os.environ.get("HX_ORACLE_LIB") or build())
    P, I, D, VP = ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "orc_new": (VP, [P]),
        "orc_add_block": (I, [VP, I, I, I, P]),
        "orc_set_face": (I, [VP, I, I, I, I, I, P]),
        "orc_set_face_transform": (I, [VP, I, I, ctypes.POINTER(ctypes.c_int)]),
        "orc_check": (I, [VP]),
        "orc_metrics": (I, [VP]),
        "orc_get_metrics": (None, [VP, I, P, I]),
        "orc_set_state": (None, [VP, I, P]),
        "orc_get_state": (None, [VP, I, P]),
        "orc_rhs": (None, [VP]),
        "orc_get_rhs": (None, [VP, I, P]),
        "orc_get_grad": (None, [VP, I, P]),
        "orc_step": (None, [VP, I, D]),
        "orc_step_multi": (None, [VP, I, P]),
        "orc_dt": (D, [VP, D, P]),
        "orc_step_local": (None, [VP, I, D]),
        "orc_dt_local": (None, [VP, I, D, P]),
        "orc_set_threads": (None, [I]),
        "orc_max_threads": (I, []),
        "orc_free": (None, [VP]),
        "orc_op_weno": (None, [P, P, P, P]),
        "orc_op_d6": (D, [P]),
        "orc_op_mid6": (D, [P]),
        "orc_op_eq19": (D, [D, D, P]),
        "orc_op_dline": (D, [P, I, I, I, I]),
        "orc_op_eigen": (None, [VP, P, P, P, P, P]),
        "orc_op_sw_flux": (None, [VP, P, P, I, P]),
        "orc_op_point_flux": (None, [VP, P, P, P]),
        "orc_op_farfield": (None, [VP, P, P, P]),
        "orc_op_viscous_flux": (None, [VP, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    load().orc_set_threads(int(n))


def max_threads():
    return load().orc_max_threads()


class Problem:
    """A multi-block problem held by the oracle.

    Arrays use the layout of the C library boundary: coordinates
    ``[3][nk][nj][ni]``, state ``[5][nk][nj][ni]`` (rho, rho u, rho v, rho w, e),
    metrics ``[10][nk][nj][ni]`` (xi^_x, xi^_y, xi^_z, eta^_x, ..., zeta^_z, J).
    """

    def __init__(self, gamma=1.4, mach=0.5, reynolds=1.0, prandtl=0.72,
                 sutherland_s=110.4 / 288.15, viscous=False, mu_law=1, scheme=0):
        self._lib = load()
        cfg = np.array([gamma, mach, reynolds, prandtl, sutherland_s, float(viscous), float(mu_law), float(scheme)])
        self._h = self._lib.orc_new(_p(cfg))
        self.gamma = gamma
        self.dims = []

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.orc_free(h)

    def add_block(self, xyz):
        xyz = _f64(xyz)
        nk, nj, ni = xyz.shape[1:]
        b = self._lib.orc_add_block(self._h, ni, nj, nk, _p(xyz))
        if b < 0:
            raise ValueError("oracle: block needs at least 6 nodes per direction")
        self.dims.append((nk, nj, ni))
        return b

    def set_face(self, b, f, kind, nbr=-1, nbr_face=-1, translate=(0.0, 0.0, 0.0), transform=(1, 2, 3)):
        """transform: axis a of block b runs along axis |t[a]|-1 of the
        neighbour, reversed when t[a] < 0 (identity by default)."""
        kind = KIND[kind] if isinstance(kind, str) else int(kind)
        tr = _f64(translate)
        if self._lib.orc_set_face(self._h, b, f, kind, nbr, nbr_face, _p(tr)):
            raise ValueError("oracle: bad face")
        tf = (ctypes.c_int * 3)(*[int(t) for t in transform])
        if self._lib.orc_set_face_transform(self._h, b, f, tf):
            raise ValueError("oracle: bad face")

    def check(self):
        if self._lib.orc_check(self._h):
            raise ValueError("oracle: inconsistent topology")

    def metrics(self):
        rc = self._lib.orc_metrics(self._h)
        if rc:
            raise ValueError("oracle: non-positive Jacobian" if rc == -1 else "oracle: out of memory")

    def get_metrics(self, b, padded=False):
        nk, nj, ni = self.dims[b]
        shape = (10, nk + 6, nj + 6, ni + 6) if padded else (10, nk, nj, ni)
        out = np.empty(shape)
        self._lib.orc_get_metrics(self._h, b, _p(out), int(padded))
        return out

    def set_state(self, b, q):
        q = _f64(q)
        assert q.shape == (5,) + self.dims[b]
        self._lib.orc_set_state(self._h, b, _p(q))

    def get_state(self, b):
        out = np.empty((5,) + self.dims[b])
        self._lib.orc_get_state(self._h, b, _p(out))
        return out

    def rhs(self):
        self._lib.orc_rhs(self._h)

    def get_rhs(self, b):
        out = np.empty((5,) + self.dims[b])
        self._lib.orc_get_rhs(self._h, b, _p(out))
        return out

    def get_grad(self, b):
        out = np.empty((12,) + self.dims[b])
        self._lib.orc_get_grad(self._h, b, _p(out))
        return out

    def step(self, nsteps, dt):
        if np.ndim(dt) == 0:
            self._lib.orc_step(self._h, int(nsteps), float(dt))
        else:
            d = _f64(dt)
            assert d.shape == (len(self.dims),)
            self._lib.orc_step_multi(self._h, int(nsteps), _p(d))

    def step_local(self, nsteps, cfl):
        """Local time stepping: each node advances with its own time step,
        taken from the state at the start of every step."""
        self._lib.orc_step_local(self._h, int(nsteps), float(cfl))

    def dt_local(self, b, cfl):
        """Per-node local time steps of block b, [nk][nj][ni]."""
        out = np.empty(self.dims[b])
        self._lib.orc_dt_local(self._h, b, float(cfl), _p(out))
        return out

    def dt(self, cfl):
        """Returns (global dt, per-block dt) from the current state."""
        per = np.empty(len(self.dims))
        g = self._lib.orc_dt(self._h, float(cfl), _p(per))
        return g, per


def from_workload(w, scheme=0):
    """Builds an oracle Problem from a workload description (blocks, faces,
    initial state) produced by ``paper_2006_07964_gb300.workloads``;
    scheme 0 is the modified AFWENO, 1 the original one."""
    P = Problem(gamma=w.gamma, mach=w.mach, reynolds=w.reynolds, prandtl=w.prandtl,
                sutherland_s=w.sutherland_s, viscous=w.viscous, mu_law=w.mu_law, scheme=scheme)
    for blk in w.blocks:
        P.add_block(blk.xyz)
    for b, blk in enumerate(w.blocks):
        for f, face in enumerate(blk.faces):
            P.set_face(b, f, face.kind, face.nbr, face.nbr_face, face.translate, face.transform)
    P.check()
    P.metrics()
    for b, blk in enumerate(w.blocks):
        P.set_state(b, blk.q0)
    return P


# ---- single operators (pins) ------------------------------------------------

def op_weno(W):
    W = _f64(W)
    b = np.empty(3)
    l, r = ctypes.c_double(), ctypes.c_double()
    lib = load()
    lib.orc_op_weno(_p(W), _p(b), ctypes.byref(l), ctypes.byref(r))
    return b, l.value, r.value


def op_d6(f7):
    return load().orc_op_d6(_p(_f64(f7)))


def op_mid6(f6):
    return load().orc_op_mid6(_p(_f64(f6)))


def op_eq19(hp, hm, f7):
    return load().orc_op_eq19(float(hp), float(hm), _p(_f64(f7)))


def op_dline(f, p, lo, hi):
    f = _f64(f)
    return load().orc_op_dline(_p(f), int(p), len(f), int(lo), int(hi))


class Ops:
    """Gas-dependent single operators; holds a Problem for the gas constants."""

    def __init__(self, **kw):
        self.P = Problem(**kw)
        self._lib = self.P._lib

    def eigen(self, q, k):
        L, R, lam = np.empty(25), np.empty(25), np.empty(5)
        self._lib.orc_op_eigen(self.P._h, _p(_f64(q)), _p(_f64(k)), _p(L), _p(R), _p(lam))
        return L.reshape(5, 5), R.reshape(5, 5), lam

    def sw_flux(self, q, m, sign):
        F = np.empty(5)
        self._lib.orc_op_sw_flux(self.P._h, _p(_f64(q)), _p(_f64(m)), int(sign), _p(F))
        return F

    def point_flux(self, q, m):
        F = np.empty(5)
        self._lib.orc_op_point_flux(self.P._h, _p(_f64(q)), _p(_f64(m)), _p(F))
        return F

    def farfield(self, qi, nrm):
        qb = np.empty(5)
        self._lib.orc_op_farfield(self.P._h, _p(_f64(qi)), _p(_f64(nrm)), _p(qb))
        return qb

    def viscous_flux(self, q, g, m):
        fv = np.empty(5)
        self._lib.orc_op_viscous_flux(self.P._h, _p(_f64(q)), _p(_f64(g)), _p(_f64(m)), _p(fv))
        return fv
