"""Synthetic grids, topologies and initial states (seeded, analytic).

This module only builds inputs: node coordinates, face connections and the
initial conservative state.  It holds none of the discretisation; both the
CUDA library and the CPU oracle consume what it returns.

Units are the paper's nondimensionalisation (Eq. (1) and the definitions
below it): free-stream density, temperature and sound speed are 1, so
p_inf = 1/gamma, T = gamma p / rho, e = p/(gamma-1) + rho |u|^2 / 2.

Workloads (sizes as the benchmark configurations state them):
  vortex      isentropic vortex, strength 5, advected at Mach 0.5, periodic
              warped box [0,10)^3 (x_i + 0.1 L sin sin warp), Euler
  tgv         Taylor-Green vortex, Re 1600, Ma 0.1, Pr 0.71, periodic box
              [0,2pi)^3 with a 0.02 L warp, Navier-Stokes
  ogrid       8-block O-grid around a cylinder of radius 0.5 (outer radius
              20), Ma 0.2, Re 3900, wall + far field, spanwise periodic
  batch       64 independent vortex instances with edge lengths drawn from
              {24, 32, 48, 64, 96} per axis (numpy default_rng(2006_07964))
  shocktube   two Sod shock tubes back to back in a periodic box (the high
              state in the middle half along x), Euler; exercises the
              nonlinear WENO weights and the flux splitting at shocks
"""
from dataclasses import dataclass, field
import math

import numpy as np

FACE_NAMES = ("i-", "i+", "j-", "j+", "k-", "k+")
SUTHERLAND_S = 110.4 / 288.15


@dataclass
class Face:
    kind: str                 # "periodic" | "interface" | "wall" | "farfield"
    nbr: int = -1
    nbr_face: int = -1
    translate: tuple = (0.0, 0.0, 0.0)   # added to the neighbour's coordinates
    # axis a of this block runs along axis |transform[a]|-1 of the neighbour,
    # in the same direction when positive (CGNS 1-to-1 convention)
    transform: tuple = (1, 2, 3)


@dataclass
class Block:
    xyz: np.ndarray           # [3][nk][nj][ni]
    faces: list               # 6 Face objects, order i-, i+, j-, j+, k-, k+
    q0: np.ndarray = None     # [5][nk][nj][ni]

    @property
    def shape(self):
        return self.xyz.shape[1:]

    @property
    def npts(self):
        nk, nj, ni = self.shape
        return nk * nj * ni


@dataclass
class Workload:
    name: str
    blocks: list
    gamma: float = 1.4
    mach: float = 0.5
    reynolds: float = 1.0
    prandtl: float = 0.72
    viscous: bool = False
    mu_law: int = 1
    sutherland_s: float = SUTHERLAND_S
    cfl: float = 0.5
    steps: int = 10
    meta: dict = field(default_factory=dict)

    @property
    def npts(self):
        return sum(b.npts for b in self.blocks)


# ---------------------------------------------------------------------------
# state helpers
# ---------------------------------------------------------------------------

def conservative(gamma, rho, u, v, w, p):
    """(rho, rho u, rho v, rho w, e) with e = p/(gamma-1) + rho |u|^2/2."""
    rho, u, v, w, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, v, w, p)))
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def primitive(gamma, q):
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    return rho, u, v, w, p


# ---------------------------------------------------------------------------
# grids
# ---------------------------------------------------------------------------

def lattice(n, L, origin=(0.0, 0.0, 0.0)):
    """Uniform periodic lattice X_i = origin + i L/n (no duplicated end node).
    n = (ni, nj, nk); returns X, Y, Z with shape (nk, nj, ni)."""
    ni, nj, nk = n
    x = origin[0] + np.arange(ni) * (L[0] / ni)
    y = origin[1] + np.arange(nj) * (L[1] / nj)
    z = origin[2] + np.arange(nk) * (L[2] / nk)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def warped_box(n, L, amp, dims=3):
    """Periodic box with the sinusoidal warp
         x = X + a sin(2 pi Y/Ly) sin(2 pi Z/Lz)
         y = Y + a sin(2 pi X/Lx) sin(2 pi Z/Lz)
         z = Z + a sin(2 pi X/Lx) sin(2 pi Y/Ly),  a = amp * L.
    dims=2 drops the z dependence (x, y warped in-plane only), which keeps a
    short spanwise extent valid for quasi-2D refinement studies."""
    X, Y, Z = lattice(n, L)
    Lx, Ly, Lz = L
    sx, sy, sz = (np.sin(2 * np.pi * X / Lx), np.sin(2 * np.pi * Y / Ly), np.sin(2 * np.pi * Z / Lz))
    if dims == 3:
        x = X + amp * Lx * sy * sz
        y = Y + amp * Ly * sx * sz
        z = Z + amp * Lz * sx * sy
    else:
        x = X + amp * Lx * sy
        y = Y + amp * Ly * sx
        z = Z.copy()
    return np.stack([x, y, z])


def periodic_faces(L, self_index=0):
    """Six periodic self-faces of a single block; translations are +-L per axis."""
    faces = []
    for d in range(3):
        t = [0.0, 0.0, 0.0]
        t[d] = -L[d]
        faces.append(Face("periodic", self_index, 2 * d + 1, tuple(t)))
        t = [0.0, 0.0, 0.0]
        t[d] = L[d]
        faces.append(Face("periodic", self_index, 2 * d, tuple(t)))
    return faces


def split_periodic_box(xyz, L, parts):
    """Splits one periodic block into parts=(pi, pj, pk) blocks joined by
    interface faces; the outer faces stay periodic (with translations)."""
    nk, nj, ni = xyz.shape[1:]
    cuts = []
    for n, p in zip((ni, nj, nk), parts):
        edges = [round(n * t / p) for t in range(p + 1)]
        cuts.append(edges)
    pi_, pj_, pk_ = parts

    def bid(a, b, c):
        return (c % pk_) * pj_ * pi_ + (b % pj_) * pi_ + (a % pi_)

    blocks = []
    for c in range(pk_):
        for b in range(pj_):
            for a in range(pi_):
                i0, i1 = cuts[0][a], cuts[0][a + 1]
                j0, j1 = cuts[1][b], cuts[1][b + 1]
                k0, k1 = cuts[2][c], cuts[2][c + 1]
                sub = np.ascontiguousarray(xyz[:, k0:k1, j0:j1, i0:i1])
                faces = []
                idx = (a, b, c)
                for d in range(3):
                    for side in (0, 1):
                        nidx = list(idx)
                        nidx[d] += 1 if side else -1
                        wrap = nidx[d] < 0 or nidx[d] >= parts[d]
                        t = [0.0, 0.0, 0.0]
                        if wrap:
                            t[d] = L[d] if side else -L[d]
                        kind = "periodic" if wrap else "interface"
                        faces.append(Face(kind, bid(*nidx), 2 * d + (1 - side), tuple(t)))
                blocks.append(Block(sub, faces))
    return blocks


def split_state(q, parts):
    """Splits a [5][nk][nj][ni] state the same way as split_periodic_box."""
    nk, nj, ni = q.shape[1:]
    cuts = [[round(n * t / p) for t in range(p + 1)] for n, p in zip((ni, nj, nk), parts)]
    out = []
    for c in range(parts[2]):
        for b in range(parts[1]):
            for a in range(parts[0]):
                out.append(np.ascontiguousarray(q[:, cuts[2][c]:cuts[2][c + 1], cuts[1][b]:cuts[1][b + 1],
                                                  cuts[0][a]:cuts[0][a + 1]]))
    return out


def permute_axes(arr, perm):
    """Relabels the index axes of a [C][nk][nj][ni] array: old axis c
    (0 = i, 1 = j, 2 = k) becomes new axis |perm[c]|-1, reversed when
    perm[c] < 0."""
    out = np.asarray(arr)
    for c in range(3):
        if perm[c] < 0:
            out = np.flip(out, axis=3 - c)
    src = {abs(perm[c]) - 1: c for c in range(3)}
    return np.ascontiguousarray(np.transpose(out, [0] + [3 - src[e] for e in (2, 1, 0)]))


def inverse_perm(perm):
    """The signed permutation that undoes `perm`."""
    inv = [0, 0, 0]
    for c in range(3):
        e = abs(perm[c]) - 1
        inv[e] = (c + 1) if perm[c] > 0 else -(c + 1)
    return tuple(inv)


def reindex_block(blocks, b, perm):
    """Relabels the index axes of block b by the signed permutation `perm`
    (see permute_axes) and rewrites its faces and every face joined to it,
    so that the grid and the solution are unchanged.  A permutation with
    determinant -1 would turn the block left-handed (negative Jacobian)."""
    import copy
    blocks = [copy.copy(B) for B in blocks]
    for B in blocks:
        B.faces = [copy.copy(F) for F in B.faces]
    B = blocks[b]

    def new_face(f):
        c, side = f // 2, f % 2
        e = abs(perm[c]) - 1
        return 2 * e + (side if perm[c] > 0 else 1 - side)

    sig = [1 if perm[c] > 0 else -1 for c in range(3)]
    # this block's faces: new position, transform from the new axes
    faces = [None] * 6
    for f, F in enumerate(B.faces):
        c = f // 2
        G = copy.copy(F)
        if F.kind in ("periodic", "interface"):
            t = [0, 0, 0]
            for cc in range(3):
                t[abs(perm[cc]) - 1] = sig[cc] * F.transform[cc]
            G.transform = tuple(t)
        faces[new_face(f)] = G
    B.faces = faces
    B.xyz = permute_axes(B.xyz, perm)
    if B.q0 is not None:
        B.q0 = permute_axes(B.q0, perm)
    # faces that point at this block: neighbour face and target axes
    for C in blocks:
        for F in C.faces:
            if F.kind in ("periodic", "interface") and F.nbr == b:
                F.nbr_face = new_face(F.nbr_face)
                t = []
                for a in range(3):
                    c = abs(F.transform[a]) - 1
                    s = 1 if F.transform[a] > 0 else -1
                    t.append(s * sig[c] * (abs(perm[c])))
                F.transform = tuple(t)
    return blocks


# ---------------------------------------------------------------------------
# initial states
# ---------------------------------------------------------------------------

def isentropic_vortex(gamma, x, y, t=0.0, strength=5.0, u_inf=0.5, L=10.0, centre=(5.0, 5.0), Ly=None):
    """Shu's isentropic vortex (strength 5 in Shu's units rho_inf = p_inf = 1),
    mapped to the paper's units by u' = u/sqrt(gamma), p' = p/gamma,
    rho' = rho, t' = sqrt(gamma) t; advected along x at u_inf (paper units,
    u_inf = Mach number since c_inf = 1).  The exact solution at time t is the
    initial vortex moved by u_inf t, taken on the periodic image nearest to
    each node (periods L along x and Ly, default L, along y).  Returns
    (rho, u, v, w, p)."""
    Ly = L if Ly is None else Ly
    xc = centre[0] + u_inf * t
    dx = x - xc
    dx = dx - L * np.round(dx / L)
    dy = y - centre[1]
    dy = dy - Ly * np.round(dy / Ly)
    r2 = dx * dx + dy * dy
    e = np.exp(0.5 * (1.0 - r2))
    du = -strength / (2 * np.pi) * e * dy
    dv = strength / (2 * np.pi) * e * dx
    Ts = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * e * e
    rho = Ts ** (1.0 / (gamma - 1.0))
    ps = rho * Ts
    sg = math.sqrt(gamma)
    return rho, u_inf + du / sg, dv / sg, np.zeros_like(rho), ps / gamma


def taylor_green(gamma, x, y, z, mach):
    """Compressible Taylor-Green vortex: u = Ma sin x cos y cos z,
    v = -Ma cos x sin y cos z, w = 0,
    p = 1/gamma + Ma^2/16 (cos 2x + cos 2y)(cos 2z + 2), T = 1 (rho = gamma p)."""
    u = mach * np.sin(x) * np.cos(y) * np.cos(z)
    v = -mach * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = 1.0 / gamma + mach ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = gamma * p
    return rho, u, v, w, p


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def vortex(n=32, amp=0.1, steps=10, dims=3, nk=None, free_stream=False):
    """Isentropic vortex on a warped periodic [0,10)^3 box, Euler, CFL 0.5."""
    L = 10.0
    shape = (n, n, nk if nk else n)
    Ls = (L, L, L * shape[2] / n) if nk else (L, L, L)
    xyz = warped_box(shape, Ls, amp, dims=dims)
    g = 1.4
    if free_stream:
        rho = np.ones(xyz.shape[1:])
        q = conservative(g, rho, 0.5, 0.2, 0.1, 1.0 / g)
    else:
        q = conservative(g, *isentropic_vortex(g, xyz[0], xyz[1], L=L))
    blk = Block(xyz, periodic_faces(Ls), q)
    return Workload("vortex%d" % n, [blk], gamma=g, mach=0.5, viscous=False, cfl=0.5, steps=steps,
                    meta={"L": Ls, "amp": amp})


def tgv(n=128, amp=0.02, steps=200, mach=0.1, reynolds=1600.0, prandtl=0.71, mu_law=1):
    """Taylor-Green vortex on a warped periodic [0,2pi)^3 box, Navier-Stokes."""
    L = 2 * np.pi
    xyz = warped_box((n, n, n), (L, L, L), amp)
    g = 1.4
    q = conservative(g, *taylor_green(g, xyz[0], xyz[1], xyz[2], mach))
    blk = Block(xyz, periodic_faces((L, L, L)), q)
    return Workload("tgv%d" % n, [blk], gamma=g, mach=mach, reynolds=reynolds, prandtl=prandtl, viscous=True,
                    mu_law=mu_law, cfl=0.5, steps=steps, meta={"L": (L, L, L), "amp": amp})


def ogrid_radii(nr=192, r0=0.5, r1=20.0, first=1.0e-3):
    """Geometric radial distribution from r0 to r1 over nr-1 cells whose first
    cell is `first` (the growth ratio solved by bisection)."""
    ncell = nr - 1
    span = r1 - r0
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = first * (q ** ncell - 1.0) / (q - 1.0)
        if s > span:
            hi = q
        else:
            lo = q
    q = 0.5 * (lo + hi)
    r = r0 + first * (q ** np.arange(nr) - 1.0) / (q - 1.0)
    r[-1] = r1
    return r, q


def ogrid(scale=1, steps=100, mach=0.2, reynolds=3900.0, prandtl=0.71, sectors=(96, 128, 160, 192),
          layers=(64, 128), nz=32):
    """8-block O-grid around a cylinder of radius 0.5 (outer radius 20).
    i runs around the cylinder (clockwise, so that J > 0) through four sectors
    of uneven width; j runs outward through an inner and an outer layer
    (geometric stretching, first cell 1e-3 at full size); k is spanwise over
    L_z = pi, periodic.  Block (s, l) = sector s, layer l.  The initial state
    is the potential flow past the cylinder at free-stream Mach `mach` with
    the wall nodes at rest.  scale > 1 divides every count by `scale` for
    reduced-size tests."""
    sec = [max(6, s // scale) for s in sectors]
    lay = [max(6, l // scale) for l in layers]
    nz = max(6, nz // scale)
    nth = sum(sec)
    nr = sum(lay)
    r, _ = ogrid_radii(nr, first=1.0e-3 * scale)
    Lz = np.pi
    z = np.arange(nz) * (Lz / nz)
    g = 1.4
    blocks = []
    i0 = 0
    nb_s = len(sec)
    for s in range(nb_s):
        j0 = 0
        th = -2 * np.pi * (i0 + np.arange(sec[s])) / nth
        for l in range(len(lay)):
            rr = r[j0:j0 + lay[l]]
            Z, R, TH = np.meshgrid(z, rr, th, indexing="ij")
            xyz = np.stack([R * np.cos(TH), R * np.sin(TH), Z])
            bid = s * len(lay) + l
            faces = [
                Face("interface", ((s - 1) % nb_s) * len(lay) + l, 1),
                Face("interface", ((s + 1) % nb_s) * len(lay) + l, 0),
                Face("wall") if l == 0 else Face("interface", s * len(lay) + l - 1, 3),
                Face("farfield") if l == len(lay) - 1 else Face("interface", s * len(lay) + l + 1, 2),
                Face("periodic", bid, 5, (0.0, 0.0, -Lz)),
                Face("periodic", bid, 4, (0.0, 0.0, Lz)),
            ]
            # potential flow past the cylinder (radius a = 0.5): smooth and
            # non-uniform in every block; pressure by Bernoulli, density
            # isentropic; wall nodes at rest
            a2 = 0.25 / (R * R)
            ur = mach * (1.0 - a2) * np.cos(TH)
            ut = -mach * (1.0 + a2) * np.sin(TH)
            u = ur * np.cos(TH) - ut * np.sin(TH)
            v = ur * np.sin(TH) + ut * np.cos(TH)
            p = 1.0 / g + 0.5 * (mach * mach - (u * u + v * v))
            rho = (g * p) ** (1.0 / g)
            if l == 0:
                u[:, 0, :] = 0.0
                v[:, 0, :] = 0.0
            q = conservative(g, rho, u, v, 0.0, p)
            blocks.append(Block(xyz, faces, q))
            j0 += lay[l]
        i0 += sec[s]
    return Workload("ogrid" if scale == 1 else "ogrid_s%d" % scale, blocks, gamma=g, mach=mach,
                    reynolds=reynolds, prandtl=prandtl, viscous=True, mu_law=1, cfl=0.5, steps=steps,
                    meta={"sectors": sec, "layers": lay, "nz": nz})


BATCH_EDGES = (24, 32, 48, 64, 96)


def batch(count=64, seed=2006_07964, edges=BATCH_EDGES, amp=0.1, steps=10):
    """`count` independent vortex instances on warped periodic [0,10)^3 boxes
    with (ni, nj, nk) drawn i.i.d. from `edges` by default_rng(seed)."""
    rng = np.random.default_rng(seed)
    dims = rng.choice(np.asarray(edges), size=(count, 3))
    L = 10.0
    g = 1.4
    blocks = []
    for b in range(count):
        ni, nj, nk = (int(v) for v in dims[b])
        xyz = warped_box((ni, nj, nk), (L, L, L), amp)
        q = conservative(g, *isentropic_vortex(g, xyz[0], xyz[1], L=L))
        blocks.append(Block(xyz, periodic_faces((L, L, L), self_index=b), q))
    return Workload("batch%d" % count, blocks, gamma=g, mach=0.5, viscous=False, cfl=0.5, steps=steps,
                    meta={"dims": dims.tolist(), "seed": seed})


def shocktube(n=(256, 8, 8), length=2.0, amp=0.0, steps=20, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Periodic box [0, length) x [0, length n_j/n_i) x [0, length n_k/n_i):
    state `left` (rho, u, p) for x in [length/4, 3 length/4), `right`
    elsewhere (Sod's states by default), so that two Riemann problems evolve
    from x = length/4 and x = 3 length/4 until their waves meet.  amp > 0
    warps the grid as warped_box does (the discontinuity stays a plane in
    physical space)."""
    ni, nj, nk = n
    L = (length, length * nj / ni, length * nk / ni)
    xyz = warped_box(n, L, amp) if amp > 0 else np.stack(lattice(n, L))
    g = 1.4
    inside = (xyz[0] >= 0.25 * length) & (xyz[0] < 0.75 * length)
    rho = np.where(inside, left[0], right[0])
    u = np.where(inside, left[1], right[1])
    p = np.where(inside, left[2], right[2])
    q = conservative(g, rho, u, 0.0, 0.0, p)
    return Workload("shocktube%d" % ni, [Block(xyz, periodic_faces(L), q)], gamma=g, mach=0.0, viscous=False,
                    cfl=0.5, steps=steps, meta={"L": L, "left": left, "right": right})


def shock_vortex(n=(128, 64, 8), length=10.0, amp=0.04, mach_s=1.2, strength=3.0, steps=40):
    """Shock-vortex interaction in a periodic box [0, length) x [0, length
    n_j/n_i) x [0, length n_k/n_i), Euler.  Gas at rest (rho = 1, p =
    1/gamma, c = 1) holds an isentropic vortex (Shu's, at rest, strength
    `strength`) centred at x = 0.55 length, y = half the box; a normal shock
    of Mach mach_s moving along +x stands at x = 0.45 length, with the
    Rankine-Hugoniot post-shock state behind it back to x = 0.1 length, so
    that the shock runs into the vortex from the first step and both the
    shock and the vortex are bent across y (the nonlinear weights act along
    every direction of the warped grid).  amp > 0 warps the grid as
    warped_box does."""
    ni, nj, nk = n
    L = (length, length * nj / ni, length * nk / ni)
    xyz = warped_box(n, L, amp) if amp > 0 else np.stack(lattice(n, L))
    g = 1.4
    rho, u, v, w, p = isentropic_vortex(g, xyz[0], xyz[1], strength=strength, u_inf=0.0, L=L[0],
                                        centre=(0.55 * length, 0.5 * L[1]), Ly=L[1])
    # Rankine-Hugoniot: shock at speed mach_s into gas at rest (rho 1, p 1/gamma, c 1)
    m2 = mach_s * mach_s
    p2 = (1.0 / g) * (1.0 + 2.0 * g / (g + 1.0) * (m2 - 1.0))
    r2 = (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    u2 = mach_s * (1.0 - 1.0 / r2)
    behind = (xyz[0] >= 0.1 * length) & (xyz[0] < 0.45 * length)
    rho = np.where(behind, r2, rho)
    u = np.where(behind, u2, u)
    v = np.where(behind, 0.0, v)
    p = np.where(behind, p2, p)
    q = conservative(g, rho, u, v, w, p)
    return Workload("shockvortex%d" % ni, [Block(xyz, periodic_faces(L), q)], gamma=g, mach=0.0, viscous=False,
                    cfl=0.5, steps=steps, meta={"L": L, "mach_s": mach_s, "strength": strength})
