"""The FP64 sweeps' reformulations of the characteristic WENO and the
Steger-Warming face flux (csrc/hx_common.cuh: node_state, CharBasis,
weno_parts_d, sw_flux), restated step for step in numpy and checked against
the oracle's own operators (its eigenvector matrices, one-field WENO and
split flux) on random physical states.  Each reformulation is exact in real
arithmetic; these tests pin that algebra on the CPU, and the GPU parity
tests check the kernels that carry it.
  - the node basis from the direction-independent node state, with the
    projection W = L q and the back projection U = R W in vector form, the
    latter from the node's rho k (Pulliam-Chaussee pair, Sec. 4.5.1);
  - a node's own characteristic values in closed form;
  - the WENO of the modified scheme from the projected state differences
    across the stencil's faces (the projection is linear), Eqs. (13)-(17);
  - the split flux with c^2 and H from E/rho - |u|^2/2, Eq. (12)."""
import numpy as np

import oracle

GAMMA = 1.4
GM1 = GAMMA - 1.0
S2 = np.sqrt(0.5)


def _state(rng):
    rho = rng.uniform(0.5, 2.0)
    u = rng.uniform(-0.8, 0.8, 3)
    p = rng.uniform(0.3, 2.0)
    return np.array([rho, *(rho * u), p / GM1 + 0.5 * rho * u @ u])


def _unit(rng):
    k = rng.normal(size=3)
    return k / np.linalg.norm(k)


class Basis:
    """node_state + CharBasis::set_state / set_normal / project / center / back."""

    def __init__(self, q, k):
        rho = q[0]
        self.rho, self.k = rho, k
        irho = 1.0 / rho
        self.vel = q[1:4] * irho
        self.half_uu = 0.5 * self.vel @ self.vel
        p = GM1 * (q[4] - rho * self.half_uu)
        c2 = GAMMA * p * irho
        ic = 1.0 / np.sqrt(c2)
        self.c = c2 * ic
        self.a0 = 1.0 - GM1 * self.half_uu * ic * ic
        self.g = GM1 * ic * ic
        self.cir = self.c * irho * S2
        self.al = rho * ic * S2
        self.H = self.half_uu + c2 / GM1
        self.alc = self.al * self.c
        self.ki = k * irho
        self.ks = self.ki * S2
        self.acth = self.alc * (k @ self.vel)
        self.rk = rho * k

    def project(self, q):
        d = q[1:4] - self.vel * q[0]
        S = self.a0 * q[0] + self.g * (self.vel @ q[1:4]) - self.g * q[4]
        W012 = self.k * S + np.cross(d, self.ki)
        kd = self.ks @ d
        base = self.cir * (q[0] - S)
        return np.array([*W012, base + kd, base - kd])

    def center(self):
        S = self.rho * GM1 / GAMMA
        return np.array([*(self.k * S), self.c / (GAMMA * np.sqrt(2.0)), self.c / (GAMMA * np.sqrt(2.0))])

    def back(self, W):
        Wk = self.k @ W[:3]
        rC = np.cross(self.rk, W[:3])
        s, t = W[3] + W[4], W[3] - W[4]
        U0 = Wk + self.al * s
        U = [U0, *(self.vel * U0 + rC + self.alc * t * self.k)]
        U.append(self.half_uu * Wk + self.vel @ rC + self.al * s * self.H + self.acth * t)
        return np.array(U)


def weno_from_differences(d10, d21, d32, d43, w2):
    """weno_parts_d: the left value at i+1/2 and the right value at i-1/2."""
    a1, a2, a3 = d21 - d10, d32 - d21, d43 - d32
    c1, c2, c3 = 2 * d21 + a1, d21 + d32, -2 * d32 + a3
    s1, s2, s3 = [(a * (13.0 / 3.0 * a) + (c * c + 4e-6)) ** 2 for a, c in ((a1, c1), (a2, c2), (a3, c3))]
    p12, p13, p23 = s1 * s2, s1 * s3, s2 * s3
    dL, dR = 10 * p13 + 5 * p12 + p23, 10 * p13 + 5 * p23 + p12
    e1, e2 = a1 - a2, a2 - a3
    A, B = p23 * e1, p12 * e2
    left = w2 + (3 * d32 + d21) / 8 + (3 * A + 5 * B) / (8 * dL)
    right = w2 - (3 * d21 + d32) / 8 - (3 * B + 5 * A) / (8 * dR)
    return left, right


def split_flux(q, m, pos):
    """sw_flux with mmg = |m| / (2 gamma) and c^2, H from t = E/rho - |u|^2/2."""
    mm = np.linalg.norm(m)
    k = m / mm
    irho = 1.0 / q[0]
    vel = q[1:4] * irho
    uu = vel @ vel
    e = q[4] * irho
    t = e - 0.5 * uu
    c = np.sqrt(GAMMA * GM1 * t)
    th = k @ vel
    lam = np.array([th, th + c, th - c])
    lam = np.maximum(lam, 0.0) if pos else np.minimum(lam, 0.0)
    l1, l4, l5 = lam
    a = q[0] * mm / (2 * GAMMA)
    S45, D45 = l4 + l5, l4 - l5
    aM = a * (2 * GM1 * l1 + S45)
    acD = a * c * D45
    H = e + GM1 * t
    return np.array([aM, *(vel * aM + k * acD), a * (GM1 * l1 * uu + S45 * H) + th * acD])


def test_node_basis_is_the_oracles_eigenvector_pair():
    ops = oracle.Ops(gamma=GAMMA)
    rng = np.random.default_rng(21)
    for _ in range(200):
        q, k = _state(rng), _unit(rng)
        L, R, _ = ops.eigen(q, k)
        b = Basis(q, k)
        for _ in range(3):
            x = _state(rng)
            np.testing.assert_allclose(b.project(x), L @ x, rtol=1e-12, atol=1e-12 * np.abs(L @ x).max())
            W = rng.normal(size=5)
            np.testing.assert_allclose(b.back(W), R @ W, rtol=1e-12, atol=1e-12 * np.abs(R @ W).max())
        np.testing.assert_allclose(b.center(), L @ q, rtol=1e-12, atol=1e-13)


def test_weno_from_projected_face_differences():
    ops = oracle.Ops(gamma=GAMMA)
    rng = np.random.default_rng(5)
    for trial in range(200):
        q0, k = _state(rng), _unit(rng)
        # a smooth stencil, or one with a jump between two of its nodes
        Q = np.array([q0 * (1 + 0.02 * rng.normal()) for _ in range(5)])
        if trial % 2:
            Q[3:] *= rng.uniform(1.5, 3.0)
        L, _, _ = ops.eigen(Q[2], k)
        b = Basis(Q[2], k)
        dW = [b.project(Q[s + 1] - Q[s]) for s in range(4)]
        Wc = b.center()
        W = Q @ L.T   # W[s, l]: the oracle's characteristic values of the stencil
        for l in range(5):
            _, left, right = oracle.op_weno(W[:, l])
            mine = weno_from_differences(dW[0][l], dW[1][l], dW[2][l], dW[3][l], Wc[l])
            scale = max(1.0, np.abs(W[:, l]).max())
            assert abs(mine[0] - left) <= 1e-12 * scale, (trial, l, mine[0], left)
            assert abs(mine[1] - right) <= 1e-12 * scale, (trial, l, mine[1], right)


def test_split_flux_without_the_pressure():
    ops = oracle.Ops(gamma=GAMMA)
    rng = np.random.default_rng(9)
    for _ in range(300):
        q = _state(rng)
        m = rng.normal(size=3) * rng.uniform(0.2, 3.0)
        for pos, sign in ((True, 1), (False, -1)):
            ref = ops.sw_flux(q, m, sign)
            np.testing.assert_allclose(split_flux(q, m, pos), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
