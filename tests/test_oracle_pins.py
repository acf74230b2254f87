"""Pins of the oracle's single operators against what the paper and the
mathematics fix (polynomial exactness, the paper's printed coefficients,
eigen-decomposition identities, flux-splitting identities)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_data import air_viscosity_table, coefficients

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
RNG = np.random.default_rng(12345)
G = 1.4


def cons(rho, u, v, w, p, g=G):
    return np.array([rho, rho * u, rho * v, rho * w, p / (g - 1) + 0.5 * rho * (u * u + v * v + w * w)])


# ---------------------------------------------------------------- D and mid6

@pytest.mark.parametrize("deg", range(0, 7))
def test_d6_exact_up_to_degree_6(deg):
    """Sec. 2 sixth-order central scheme: exact for polynomials of degree <= 6."""
    c = RNG.normal(size=deg + 1)
    h = 0.37
    x = np.arange(-3, 4) * h
    f = np.polyval(c, x)
    exact = np.polyval(np.polyder(c), 0.0) if deg > 0 else 0.0
    assert oracle.op_d6(f) / h == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_d6_not_exact_at_degree_7():
    f = np.arange(-3, 4, dtype=float) ** 7
    assert abs(oracle.op_d6(f)) > 1.0   # truncation term of x^7 at unit spacing is -36


def test_d6_order_six_on_sine():
    errs = []
    for h in (0.2, 0.1):
        x = np.arange(-3, 4) * h + 0.3
        errs.append(abs(oracle.op_d6(np.sin(x)) / h - np.cos(0.3)))
    assert np.log2(errs[0] / errs[1]) == pytest.approx(6.0, abs=0.2)


@pytest.mark.parametrize("deg", range(0, 6))
def test_mid6_exact_up_to_degree_5(deg):
    c = RNG.normal(size=deg + 1)
    x = np.arange(-2, 4, dtype=float)
    assert oracle.op_mid6(np.polyval(c, x)) == pytest.approx(np.polyval(c, 0.5), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("p,lo,hi,deg", [(0, 1, 0, 2), (1, 1, 0, 2), (2, 1, 0, 4), (9, 0, 1, 2), (8, 0, 1, 2),
                                         (7, 0, 1, 4), (5, 1, 1, 6), (3, 0, 0, 6)])
def test_viscous_closure_exactness(p, lo, hi, deg):
    """Closure stencils of the physical-face reading (one-sided 2nd order,
    2nd-order central, 4th-order central) and the interior sixth-order
    operator are exact on polynomials of their degree."""
    n = 10
    c = RNG.normal(size=deg + 1)
    f = np.polyval(c, np.arange(n, dtype=float))
    assert oracle.op_dline(f, p, lo, hi) == pytest.approx(np.polyval(np.polyder(c), p), rel=1e-11, abs=1e-11)


# ---------------------------------------------------------------- WENO (Eqs. 13-17)

def test_weno_ideal_weights_give_fifth_order_interpolant():
    """Reading R1: with the pairing used, the linear weights reproduce the
    fifth-order interpolant (3,-20,90,60,-5)/128 at i+1/2.  Tiny data make
    beta << epsilon so the nonlinear weights equal the linear ones."""
    cf = coefficients()
    gam = cf["eq16_gamma"]
    u1, u2, u3 = cf["eq14_u1"], cf["eq14_u2"], cf["eq14_u3"]
    # interpolant implied by the paper's sub-stencils; u3 (stencil i-2..i) takes gamma_1
    ideal = {s: Fraction(0) for s in range(-2, 3)}
    for s, c in u3.items():
        ideal[s] += gam[1] * c
    for s, c in u2.items():
        ideal[s] += gam[2] * c
    for s, c in u1.items():
        ideal[s] += gam[3] * c
    assert [ideal[s] * 128 for s in range(-2, 3)] == [3, -20, 90, 60, -5]
    for _ in range(20):
        W = RNG.normal(size=5) * 1e-9
        _, left, right = oracle.op_weno(W)
        want_l = sum(float(ideal[s]) * W[s + 2] for s in range(-2, 3))
        want_r = sum(float(ideal[s]) * W[2 - s] for s in range(-2, 3))
        # weights deviate from the linear ones by O(beta/eps) ~ 1e-11
        assert abs(left - want_l) < 1e-9 * np.abs(W).max()
        assert abs(right - want_r) < 1e-9 * np.abs(W).max()


def test_weno_paper_literal_pairing_is_not_fifth_order():
    """Eq. (14) numbering with Eq. (16) weights taken literally (gamma_1 on u^(1))
    is not the fifth-order interpolant: the reason for reading R1."""
    cf = coefficients()
    gam = cf["eq16_gamma"]
    lit = {s: Fraction(0) for s in range(-2, 3)}
    for j, name in ((1, "eq14_u1"), (2, "eq14_u2"), (3, "eq14_u3")):
        for s, c in cf[name].items():
            lit[s] += gam[j] * c
    assert [lit[s] * 128 for s in range(-2, 3)] != [3, -20, 90, 60, -5]


def test_weno_beta_equals_printed_eq17():
    """The oracle's indicators equal the printed quadratic forms of Eq. (17),
    evaluated exactly in rational arithmetic on the same (binary) inputs."""
    cf = coefficients()
    for _ in range(50):
        W = RNG.normal(size=5)
        b, _, _ = oracle.op_weno(W)
        Wf = [Fraction(float(x)) for x in W]
        for j, name in enumerate(("eq17_b1", "eq17_b2", "eq17_b3")):
            exact = sum(c * Wf[k // 10] * Wf[k % 10] for k, c in cf[name].items()) / 3
            assert abs(Fraction(b[j]) - exact) <= Fraction(1, 10 ** 14) * max(abs(exact), Fraction(1, 10 ** 6))


def test_weno_beta_is_well_conditioned():
    """Smooth data around a large offset: the indicators keep their relative
    accuracy (no cancellation of the O(W^2) terms)."""
    x = np.arange(-2, 3) * 1e-3
    W = 5.0 + x + 0.5 * x * x
    b, _, _ = oracle.op_weno(W)
    Wf = [Fraction(float(v)) for v in W]
    cf = coefficients()
    for j, name in enumerate(("eq17_b1", "eq17_b2", "eq17_b3")):
        exact = sum(c * Wf[k // 10] * Wf[k % 10] for k, c in cf[name].items()) / 3
        assert abs(Fraction(b[j]) - exact) <= Fraction(1, 10 ** 12) * abs(exact)


def test_weno_exact_on_linear_data():
    for _ in range(10):
        a, s = RNG.normal(size=2)
        W = a + s * np.arange(-2, 3)
        _, left, right = oracle.op_weno(W)
        assert left == pytest.approx(a + 0.5 * s, rel=1e-13, abs=1e-13)
        assert right == pytest.approx(a - 0.5 * s, rel=1e-13, abs=1e-13)


def test_weno_picks_smooth_side_of_a_jump():
    """A jump between i and i+1: the left value at i+1/2 stays at the left state."""
    W = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    _, left, _ = oracle.op_weno(W)
    assert left == pytest.approx(1.0, abs=1e-9)
    W = np.array([1.0, 1.0, 0.0, 0.0, 0.0])   # jump between i-1 and i
    _, _, right = oracle.op_weno(W)
    assert right == pytest.approx(0.0, abs=1e-9)


def test_weno_interpolation_order_five():
    """Left value at i+1/2 of exp(x) sampled at x_i: fifth-order error."""
    errs = []
    for h in (0.1, 0.05, 0.025):
        x = (np.arange(-2, 3)) * h
        _, left, _ = oracle.op_weno(np.exp(x))
        errs.append(abs(left - np.exp(0.5 * h)))
    assert np.log2(errs[1] / errs[2]) > 4.7


# ---------------------------------------------------------------- Eq. (19)

def test_eq19_equals_eq11_with_eq18():
    """Eq. (19) coefficients follow from substituting Eq. (18) into Eq. (11) and
    differencing (Eq. 9); the oracle's combination must match on impulses."""
    cf = coefficients()
    a2, a4 = cf["eq11_a2"][0], cf["eq11_a4"][0]
    corr = {s: a2 * cf["eq18_fxx"][s] + a4 * cf["eq18_fxxxx"][s] for s in range(-2, 4)}
    # f_hat_{i+1/2} - f_hat_{i-1/2}: node offset t gets corr[t] - corr[t+1]
    deriv = {t: corr.get(t, 0) - corr.get(t + 1, 0) for t in range(-3, 4)}
    for s in (1, 2, 3):
        assert deriv[s] == cf["eq19"][s]
        assert deriv[-s] == -cf["eq19"][s]
    assert deriv[0] == 0
    for t in range(-3, 4):
        f = np.zeros(7)
        f[t + 3] = 1.0
        assert oracle.op_eq19(0.0, 0.0, f) == pytest.approx(float(deriv[t]), rel=1e-15, abs=1e-17)
    assert oracle.op_eq19(2.5, 1.0, np.zeros(7)) == 1.5


def test_mid6_difference_plus_eq19_is_d6():
    """Reading R4: the face-metric midpoint difference plus Eq. (19) on node
    metrics is the sixth-order central operator, which makes free-stream
    preservation follow from the metric identity of Eq. (7)."""
    for _ in range(10):
        m = RNG.normal(size=7)
        mp = oracle.op_mid6(m[1:7])
        mm = oracle.op_mid6(m[0:6])
        assert oracle.op_eq19(mp, mm, m) == pytest.approx(oracle.op_d6(m), rel=1e-13, abs=1e-14)


# ---------------------------------------------------------------- eigenvectors, fluxes

@pytest.fixture(scope="module")
def ops():
    return oracle.Ops(gamma=G, mach=0.2)


def _rand_state():
    return cons(RNG.uniform(0.5, 2.0), *RNG.normal(size=3), RNG.uniform(0.3, 2.0))


def test_eigen_left_times_right_is_identity(ops):
    for _ in range(20):
        k = RNG.normal(size=3)
        k /= np.linalg.norm(k)
        L, R, _ = ops.eigen(_rand_state(), k)
        assert np.abs(L @ R - np.eye(5)).max() < 1e-12


def test_eigen_reconstructs_flux_jacobian(ops):
    """R diag(lambda) L = d(k.F)/dQ, the Jacobian taken by central differences
    of the node flux of Eq. (4)."""
    for _ in range(10):
        k = RNG.normal(size=3)
        k /= np.linalg.norm(k)
        q = _rand_state()
        L, R, lam = ops.eigen(q, k)
        Jn = np.zeros((5, 5))
        h = 1e-6
        for j in range(5):
            dq = np.zeros(5)
            dq[j] = h
            Jn[:, j] = (ops.point_flux(q + dq, k) - ops.point_flux(q - dq, k)) / (2 * h)
        assert np.abs(R @ np.diag(lam) @ L - Jn).max() < 1e-7 * max(1.0, np.abs(Jn).max())


def test_steger_warming_sum_is_flux(ops):
    for _ in range(30):
        q = _rand_state()
        m = RNG.normal(size=3) * RNG.uniform(0.1, 3.0)
        Fp, Fm = ops.sw_flux(q, m, +1), ops.sw_flux(q, m, -1)
        F = ops.point_flux(q, m)
        assert np.allclose(Fp + Fm, F, rtol=1e-12, atol=1e-12 * np.abs(F).max())


def test_steger_warming_supersonic_limits(ops):
    m = np.array([0.3, -0.4, 1.2])
    k = m / np.linalg.norm(m)
    q = cons(1.3, *(3.0 * k), 1.0 / G)       # theta = 3 > c = 1
    assert np.allclose(ops.sw_flux(q, m, +1), ops.point_flux(q, m), rtol=1e-13)
    assert np.abs(ops.sw_flux(q, m, -1)).max() < 1e-13
    q = cons(1.3, *(-3.0 * k), 1.0 / G)
    assert np.abs(ops.sw_flux(q, m, +1)).max() < 1e-13


def test_steger_warming_homogeneous_in_metric(ops):
    q = _rand_state()
    m = RNG.normal(size=3)
    for s in (0.5, 3.0):
        assert np.allclose(ops.sw_flux(q, s * m, +1), s * ops.sw_flux(q, m, +1), rtol=1e-13, atol=1e-14)


def test_point_flux_mass_component(ops):
    q = cons(1.7, 0.3, -0.2, 0.5, 0.9)
    m = np.array([0.2, 0.7, -1.1])
    assert ops.point_flux(q, m)[0] == pytest.approx(1.7 * (0.2 * 0.3 - 0.7 * 0.2 - 1.1 * 0.5), rel=1e-14)


def test_farfield_keeps_free_stream(ops):
    qinf = cons(1.0, 0.2, 0.0, 0.0, 1.0 / G)
    for _ in range(10):
        n = RNG.normal(size=3)
        n /= np.linalg.norm(n)
        assert np.allclose(ops.farfield(qinf, n), qinf, rtol=1e-13, atol=1e-14)


def test_farfield_invariants(ops):
    """The boundary state carries the interior outgoing invariant and the free
    stream's incoming invariant along the normal (1D characteristics)."""
    n = np.array([0.6, 0.8, 0.0])
    qi = cons(1.1, 0.25, 0.05, 0.0, 1.05 / G)
    qb = ops.farfield(qi, n)
    rho, u, v, w = qb[0], qb[1] / qb[0], qb[2] / qb[0], qb[3] / qb[0]
    p = (G - 1) * (qb[4] - 0.5 * rho * (u * u + v * v + w * w))
    c = np.sqrt(G * p / rho)
    un = n @ [u, v, w]
    ci = np.sqrt(1.05 / 1.1)
    uni = n @ [0.25 / 1.0, 0.05, 0.0]
    assert un + 2 * c / (G - 1) == pytest.approx(uni + 2 * ci / (G - 1), rel=1e-13)
    assert un - 2 * c / (G - 1) == pytest.approx(n @ [0.2, 0, 0] - 2 / (G - 1), rel=1e-13)


# ---------------------------------------------------------------- viscous stress (Eq. (1), Eq. (6))

def _stress_rows(ops, q, g):
    """tau rows and beta from the viscous flux along the three unit metrics."""
    rows, beta = [], []
    for d in range(3):
        m = np.zeros(3)
        m[d] = 1.0
        fv = ops.viscous_flux(q, g, m)
        rows.append(fv[1:4])
        beta.append(fv[4])
    return np.array(rows), np.array(beta)


def test_viscous_stress_is_symmetric_and_traceless():
    """Eq. (1): tau_ij = mu(du_i/dx_j + du_j/dx_i - 2/3 delta_ij div u), a
    symmetric deviatoric tensor (zero trace for any velocity gradient)."""
    ops = oracle.Ops(gamma=G, mach=0.7, reynolds=13.0, viscous=True, mu_law=1)
    for _ in range(10):
        q = cons(RNG.uniform(0.5, 2.0), *RNG.normal(size=3), RNG.uniform(0.3, 2.0))
        g = RNG.normal(size=12)
        tau, _ = _stress_rows(ops, q, g)
        scale = np.abs(tau).max()
        assert np.allclose(tau, tau.T, atol=1e-14 * scale)
        assert abs(np.trace(tau)) < 1e-14 * scale
        assert scale > 1e-3


def test_viscous_stress_vanishes_for_rigid_rotation():
    """A rigid rotation (antisymmetric velocity gradient) and uniform T
    produce no stress and no heat flux."""
    ops = oracle.Ops(gamma=G, mach=0.7, reynolds=13.0, viscous=True, mu_law=1)
    q = cons(1.2, 0.3, -0.4, 0.1, 0.8)
    w = RNG.normal(size=3)
    grad_u = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    g = np.concatenate([grad_u.ravel(), np.zeros(3)])
    tau, beta = _stress_rows(ops, q, g)
    assert np.abs(tau).max() < 1e-15 and np.abs(beta).max() < 1e-15


# ---------------------------------------------------------------- Sutherland's law (reading R11)

T_INF_K = 288.15   # free-stream temperature in kelvin: the sea-level row of the table, the solver's unit


def _mu(ops, T, mach=0.7, reynolds=13.0):
    """The oracle's viscosity at temperature T (free-stream units), read
    through its viscous flux: with du/dy = 1 the only gradient,
    tau_xy = (Ma/Re) mu, the x-momentum entry of the flux along (0, 1, 0)."""
    q = cons(1.0, 0.1, -0.2, 0.05, T / G)   # rho = 1, T = gamma p / rho
    g = np.zeros(12)
    g[1] = 1.0
    fv = ops.viscous_flux(q, g, np.array([0.0, 1.0, 0.0]))
    return fv[1] / (mach / reynolds)


def test_sutherland_is_one_at_the_free_stream_temperature():
    """The Reynolds number is formed with the free-stream viscosity, so
    mu(T = 1) = 1 (Eq. (1) definitions)."""
    ops = oracle.Ops(gamma=G, mach=0.7, reynolds=13.0, viscous=True, mu_law=1)
    assert _mu(ops, 1.0) == pytest.approx(1.0, rel=1e-15)


def test_sutherland_reproduces_the_standard_atmosphere_table():
    """Reading R11 (the paper leaves mu(T) open): Sutherland's law with
    S = 110.4 K / 288.15 K.  Its values must reproduce the viscosity ratios
    the U.S. Standard Atmosphere 1976 tabulates (five significant digits, so
    1.5e-4 relative), which a wrong exponent or a wrong sign of S misses by
    percents."""
    ops = oracle.Ops(gamma=G, mach=0.7, reynolds=13.0, viscous=True, mu_law=1)
    rows = air_viscosity_table()
    ref = dict(rows)[T_INF_K]
    assert len(rows) >= 2
    for T_k, mu_k in rows:
        assert _mu(ops, T_k / T_INF_K) == pytest.approx(mu_k / ref, rel=1.5e-4), T_k


def test_constant_viscosity_law_ignores_temperature():
    ops = oracle.Ops(gamma=G, mach=0.7, reynolds=13.0, viscous=True, mu_law=0)
    for T in (0.5, 1.0, 2.5):
        assert _mu(ops, T) == pytest.approx(1.0, rel=1e-15)
