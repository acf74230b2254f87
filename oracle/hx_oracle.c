/*
 * hx_oracle.c -- plain, slow, FP64 CPU oracle of the per-Runge-Kutta-stage
 * residual evaluation and update of the multi-block curvilinear high-order
 * finite-difference Navier-Stokes method of Ye, Zhang, Wan, Yan, Sun,
 * "Accelerating CFD simulation with high order finite difference method on
 * curvilinear coordinates for modern GPU clusters" (HiResX).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library and includes none of its
 * files; the product path never calls it.
 *
 * Everything is IEEE double, built without FMA contraction or fast-math.
 * Periodic and block-interface neighbours are reached by following the face
 * connections index by index (no ghost arrays for the state); only the node
 * metrics are stored on a box padded by three layers.
 *
 * Passages followed (section / equation numbers of the paper):
 *   Eq. (1) and the definitions below it    nondimensional NS, T, e, tau, q
 *   Eqs. (2)-(5)                            curvilinear conservation form and fluxes
 *   Eq. (6)                                 stresses, work + heat terms
 *   Eqs. (7)-(8)                            conservative metrics and Jacobian
 *   Sec. 2, sixth-order central scheme      metric, Jacobian and viscous derivatives
 *   Eqs. (9)-(19)                           alternative-formulation WENO (AFWENO)
 *   Sec. 4.5.1, Figs. 10-11                 modified AFWENO: characteristic space at i
 *   Eq. (20)                                TVD Runge-Kutta 3
 *   Eq. (21), Sec. 4.5.2, Fig. 12           chain rule, viscous fluxes at points
 *   Sec. 4.5.2 (one-sided derivatives near block edges), Fig. 2 bc_phys
 *
 * Readings where the paper is silent or garbled (each is listed with its
 * reason in the design notes of the repository):
 *   R1  WENO: each sub-stencil is paired with the smoothness indicator of the
 *       same stencil; linear weights 1/16, 5/8, 5/16 go to the stencils
 *       {i-2..i}, {i-1..i+1}, {i..i+2} for the left-biased value at i+1/2
 *       (this is the pairing under which the weights reproduce the
 *       fifth-order interpolant), mirrored for the right-biased value at i-1/2.
 *   R2  the left-biased value at a face feeds F+, the right-biased one F-.
 *   R3  the conservative variables Q (without 1/J) are interpolated.
 *   R4  face metrics: sixth-order midpoint interpolation
 *       (3,-25,150,150,-25,3)/256 of the node conservative metrics.
 *   R5  metric derivatives use the same sixth-order central operator for the
 *       inner and the outer derivative; ghost coordinates come from the face
 *       neighbour (plus a translation on periodic faces) or, on physical
 *       faces, by point reflection through the boundary node.
 *   R6  characteristic basis: Pulliam-Chaussee eigenvector matrices of the
 *       flux Jacobian along the unit normal of the node metric.
 *   R7  eigenvectors are built from the node state Q_i (no averaging).
 *   R8  dt = CFL / max over nodes of sum_d (|m_d.u| + c|m_d|) J.
 *   R9  viscous one-sided closure only at physical faces, normal direction:
 *       boundary node (-3,4,-1)/2, next node 2nd-order central, third node
 *       4th-order central (1,-8,0,8,-1)/12.
 *   R10 wall: ghosts mirror rho, p and negate u; after each stage the wall
 *       node gets u = 0, e = p/(gamma-1).  Far field: 1D Riemann invariants
 *       along the outward normal of the boundary node, outgoing invariant from
 *       the node next to it, incoming from the free stream; entropy and
 *       tangential velocity upwinded by the sign of the normal velocity.
 *   R11 viscosity: mu = 1 or Sutherland T^(3/2)(1+S)/(T+S), temperatures in
 *       units of the free stream (pinned to the viscosity ratios that the
 *       U.S. Standard Atmosphere 1976 tabulates).
 *   R12 tau and q carry the factor Ma/Re; q = Ma mu/(Re Pr (gamma-1)) dT/dx_j.
 *   R13 original AFWENO (Fig. 9): the characteristic space of face i+1/2 is
 *       built from the arithmetic mean of Q_i and Q_{i+1} and the unit normal
 *       of the face metric; the left-biased value comes from the nodes
 *       i-2..i+2 and the right-biased one from i-1..i+3, each with its own
 *       smoothness indicators.
 *   R14 1:1 interfaces (Sec. 4.2, Fig. 2 bc_block) may join any face of a
 *       block to any face of another, with the index axes of the two blocks
 *       related by a signed permutation (the CGNS 1-to-1 "transform": axis a
 *       of this block runs along axis |t[a]|-1 of the neighbour, in the same
 *       direction if t[a] > 0).  The paper's figures show aligned blocks
 *       only; the state, coordinates and gradients are physical quantities,
 *       so crossing a face only maps indices.
 *   R15 local time step (Sec. 4.4 stores a time step per point and uses the
 *       viscosity for it; no formula is printed): dt_i = CFL / (lambda_c +
 *       lambda_v) with the convective radius of R8 at the node and, for
 *       Navier-Stokes, lambda_v = (Ma/Re) max(4/3, gamma/Pr) (mu/rho)
 *       sum_d (J |m_d|)^2; dt_i is taken from Q^n and held for the three
 *       stages of a step.
 * The paper gives no formulas for the physical-face rules (R9, R10), so the
 * readings themselves are not pinned to it.  The wall rule with the closure
 * next to it is pinned to closed forms of the equations it closes: the decay
 * of a shear mode between no-slip walls, and an acoustic standing wave
 * between rigid adiabatic walls, inviscid and damped.  The far-field rule is
 * pinned by its invariants (free stream is a fixed point; the outgoing and
 * incoming Riemann invariants) and by the property that defines a
 * characteristic boundary: a plane acoustic pulse leaves through it, at the
 * outflow or the inflow end, without reflection.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OF_PERIODIC = 0, OF_INTERFACE = 1, OF_WALL = 2, OF_FARFIELD = 3, OF_UNSET = -1 };

typedef struct {
    int kind, nbr, nbr_face;
    int tf[3];      /* index transform to the neighbour (reading R14)          */
    double tr[3];
} oface;

typedef struct {
    int n[3];
    double *x;      /* [3][n2][n1][n0] node coordinates, interior only          */
    oface f[6];     /* faces 0..5 = i-, i+, j-, j+, k-, k+                       */
    double *met;    /* [10][n2+6][n1+6][n0+6]: xi^_x..zeta^_z (9) and J, on [-3, n+2]^3 */
    double *q;      /* [5][n2][n1][n0] current conservative state                */
    double *qn;     /* Q^n during a step                                         */
    double *qs;     /* stage state                                               */
    double *r;      /* residual R = dQ/dt                                        */
    double *grad;   /* [12][..] (u,v,w,T)_(x,y,z), interior                     */
} oblock;

typedef struct {
    double gamma, mach, re, pr, suth;
    int viscous, mu_law;
    int scheme;     /* 0: modified AFWENO (Figs. 10-11), 1: original AFWENO (Fig. 9) */
    int nb, cap;
    oblock *b;
} oproblem;

/* ------------------------------------------------------------------------ */
/* operators                                                                 */
/* ------------------------------------------------------------------------ */

/* Sixth-order central first derivative (Sec. 2, "sixth order central scheme"),
 * unit grid spacing: D f_i = sum_{s=1..3} a_s (f_{i+s} - f_{i-s}). */
static const double D6A[4] = {0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};

static double d6(const double *f /* f[0] is the centre */) {
    double s = 0.0;
    for (int m = 1; m <= 3; ++m) s += D6A[m] * (f[m] - f[-m]);
    return s;
}

/* Derivative at node p of a line with n nodes (f[p] valid where used),
 * with the one-sided closure of reading R9 next to physical ends. */
static double dline(const double *f, int p, int n, int lo_phys, int hi_phys) {
    if (lo_phys && p <= 2) {
        if (p == 0) return (-3.0 * f[0] + 4.0 * f[1] - f[2]) / 2.0;
        if (p == 1) return (f[2] - f[0]) / 2.0;
        return (f[0] - 8.0 * f[1] + 8.0 * f[3] - f[4]) / 12.0;
    }
    if (hi_phys && p >= n - 3) {
        if (p == n - 1) return (3.0 * f[n - 1] - 4.0 * f[n - 2] + f[n - 3]) / 2.0;
        if (p == n - 2) return (f[n - 1] - f[n - 3]) / 2.0;
        return (f[n - 5] - 8.0 * f[n - 4] + 8.0 * f[n - 2] - f[n - 1]) / 12.0;
    }
    return d6(f + p);
}

/* Face value at i+1/2 from nodes i-2..i+3 (reading R4). */
static double mid6(const double *f /* f[0] = node i */) {
    return (3.0 * f[-2] - 25.0 * f[-1] + 150.0 * f[0] + 150.0 * f[1] - 25.0 * f[2] + 3.0 * f[3]) / 256.0;
}

/* Eq. (17): smoothness indicators of the three 3-node sub-stencils of the
 * 5-node stencil W[0..4] = W_{i-2..i+2}; b[0] on {i-2,i-1,i}, b[1] on
 * {i-1,i,i+1}, b[2] on {i,i+1,i+2}.  Eq. (17) defines each indicator as the
 * scaled sum of the squared L2 norms of the derivatives of the sub-stencil's
 * interpolation polynomial; that sum is written out here term by term,
 * (13/12) (second difference)^2 + (1/4) (first derivative at the node)^2,
 * which equals the printed quadratic form exactly but without its
 * cancellation (the expanded form loses ~1e-16 W^2 absolutely, a large
 * perturbation next to epsilon = 1e-6 of Eq. (15)). */
static void weno_beta(const double *W, double b[3]) {
    const double a = W[0], c = W[1], d = W[2], e = W[3], g = W[4];
    const double s1 = a - 2.0 * c + d, t1 = a - 4.0 * c + 3.0 * d;
    const double s2 = c - 2.0 * d + e, t2 = c - e;
    const double s3 = d - 2.0 * e + g, t3 = 3.0 * d - 4.0 * e + g;
    b[0] = 13.0 / 12.0 * s1 * s1 + 1.0 / 4.0 * t1 * t1;
    b[1] = 13.0 / 12.0 * s2 * s2 + 1.0 / 4.0 * t2 * t2;
    b[2] = 13.0 / 12.0 * s3 * s3 + 1.0 / 4.0 * t3 * t3;
}

static const double WENO_EPS = 1.0e-6;   /* Eq. (15) epsilon */

/* Eq. (15): normalised nonlinear weights from linear weights gam and indicators bet. */
static void weno_weights(const double gam[3], const double bet[3], double w[3]) {
    double t[3], s = 0.0;
    for (int j = 0; j < 3; ++j) {
        double den = WENO_EPS + bet[j];
        t[j] = gam[j] / (den * den);
        s += t[j];
    }
    for (int j = 0; j < 3; ++j) w[j] = t[j] / s;
}

/* Eqs. (13)-(16) with reading R1: left-biased value at i+1/2 of the stencil
 * W_{i-2..i+2}. */
static double weno_left(const double *W, const double b[3]) {
    const double u1 = 3.0 / 8.0 * W[0] - 5.0 / 4.0 * W[1] + 15.0 / 8.0 * W[2];
    const double u2 = -1.0 / 8.0 * W[1] + 3.0 / 4.0 * W[2] + 3.0 / 8.0 * W[3];
    const double u3 = 3.0 / 8.0 * W[2] + 3.0 / 4.0 * W[3] - 1.0 / 8.0 * W[4];
    const double gam[3] = {1.0 / 16.0, 5.0 / 8.0, 5.0 / 16.0};
    const double bet[3] = {b[0], b[1], b[2]};
    double w[3];
    weno_weights(gam, bet, w);
    return w[0] * u1 + w[1] * u2 + w[2] * u3;
}

/* Mirror image: right-biased value at i-1/2 of the same stencil; the
 * indicators are shared with weno_left (Fig. 10: modified AFWENO). */
static double weno_right(const double *W, const double b[3]) {
    const double u1 = 3.0 / 8.0 * W[4] - 5.0 / 4.0 * W[3] + 15.0 / 8.0 * W[2];
    const double u2 = -1.0 / 8.0 * W[3] + 3.0 / 4.0 * W[2] + 3.0 / 8.0 * W[1];
    const double u3 = 3.0 / 8.0 * W[2] + 3.0 / 4.0 * W[1] - 1.0 / 8.0 * W[0];
    const double gam[3] = {1.0 / 16.0, 5.0 / 8.0, 5.0 / 16.0};
    const double bet[3] = {b[2], b[1], b[0]};
    double w[3];
    weno_weights(gam, bet, w);
    return w[0] * u1 + w[1] * u2 + w[2] * u3;
}

/* Eq. (19): derivative at node i from the numerical fluxes at i+-1/2 and the
 * node fluxes f_{i-3..i+3} (f[0] = node i). */
static double eq19(double h_plus, double h_minus, const double *f) {
    return h_plus - h_minus + 17.0 / 256.0 * (f[1] - f[-1]) - 13.0 / 320.0 * (f[2] - f[-2])
           + 19.0 / 3840.0 * (f[3] - f[-3]);
}

/* ------------------------------------------------------------------------ */
/* gas relations (Eq. (1) definitions: T = gamma p / rho, e = p/(gamma-1) + rho|u|^2/2) */
/* ------------------------------------------------------------------------ */

typedef struct { double rho, u, v, w, p, T, c; } prim_t;

static prim_t to_prim(const oproblem *P, const double q[5]) {
    prim_t s;
    s.rho = q[0];
    s.u = q[1] / q[0];
    s.v = q[2] / q[0];
    s.w = q[3] / q[0];
    s.p = (P->gamma - 1.0) * (q[4] - 0.5 * q[0] * (s.u * s.u + s.v * s.v + s.w * s.w));
    s.T = P->gamma * s.p / s.rho;
    s.c = sqrt(s.T);   /* c^2 = gamma p / rho = T in these units */
    return s;
}

static void to_cons(const oproblem *P, double rho, double u, double v, double w, double p, double q[5]) {
    q[0] = rho;
    q[1] = rho * u;
    q[2] = rho * v;
    q[3] = rho * w;
    q[4] = p / (P->gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

/* Reading R11. */
static double viscosity(const oproblem *P, double T) {
    if (P->mu_law == 0) return 1.0;
    const double S = P->suth;
    return T * sqrt(T) * (1.0 + S) / (T + S);
}

/* Eq. (4): node flux along the conservative metric m = (xi^_x, xi^_y, xi^_z). */
static void point_flux(const oproblem *P, const double q[5], const double m[3], double f[5]) {
    prim_t s = to_prim(P, q);
    const double th = m[0] * s.u + m[1] * s.v + m[2] * s.w;
    f[0] = s.rho * th;
    f[1] = s.rho * s.u * th + m[0] * s.p;
    f[2] = s.rho * s.v * th + m[1] * s.p;
    f[3] = s.rho * s.w * th + m[2] * s.p;
    f[4] = (q[4] + s.p) * th;
}

/* Steger-Warming split flux (Sec. 2, h(u-, u+) = F+(u-) + F-(u+)) along the
 * conservative metric m; sign = +1 gives F+, -1 gives F-. */
static void sw_flux(const oproblem *P, const double q[5], const double m[3], int sign, double F[5]) {
    const double g = P->gamma;
    prim_t s = to_prim(P, q);
    const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    const double kx = m[0] / mm, ky = m[1] / mm, kz = m[2] / mm;
    const double th = kx * s.u + ky * s.v + kz * s.w;
    double l1 = th * mm, l4 = (th + s.c) * mm, l5 = (th - s.c) * mm;
    l1 = 0.5 * (l1 + sign * fabs(l1));
    l4 = 0.5 * (l4 + sign * fabs(l4));
    l5 = 0.5 * (l5 + sign * fabs(l5));
    const double a = s.rho / (2.0 * g);
    const double uu = s.u * s.u + s.v * s.v + s.w * s.w;
    const double upx = s.u + s.c * kx, upy = s.v + s.c * ky, upz = s.w + s.c * kz;
    const double umx = s.u - s.c * kx, umy = s.v - s.c * ky, umz = s.w - s.c * kz;
    F[0] = a * (2.0 * (g - 1.0) * l1 + l4 + l5);
    F[1] = a * (2.0 * (g - 1.0) * l1 * s.u + l4 * upx + l5 * umx);
    F[2] = a * (2.0 * (g - 1.0) * l1 * s.v + l4 * upy + l5 * umy);
    F[3] = a * (2.0 * (g - 1.0) * l1 * s.w + l4 * upz + l5 * umz);
    F[4] = a * ((g - 1.0) * l1 * uu + 0.5 * l4 * (upx * upx + upy * upy + upz * upz)
                + 0.5 * l5 * (umx * umx + umy * umy + umz * umz)
                + (l4 + l5) * (3.0 - g) * s.c * s.c / (2.0 * (g - 1.0)));
}

/* Reading R6: left (L) and right (R) eigenvector matrices, row-major 5x5,
 * of the Jacobian of k.F for the unit vector k at state q; lam gets the
 * eigenvalues (theta, theta, theta, theta + c, theta - c). */
static void eigen(const oproblem *P, const double q[5], const double k[3], double L[25], double R[25], double lam[5]) {
    const double g = P->gamma;
    prim_t s = to_prim(P, q);
    const double kx = k[0], ky = k[1], kz = k[2];
    const double rho = s.rho, u = s.u, v = s.v, w = s.w, c = s.c, c2 = s.c * s.c;
    const double th = kx * u + ky * v + kz * w;
    const double phi2 = 0.5 * (g - 1.0) * (u * u + v * v + w * w);
    const double al = rho / (sqrt(2.0) * c), be = 1.0 / (sqrt(2.0) * rho * c);
    const double Rm[25] = {
        kx, ky, kz, al, al,
        kx * u, ky * u - kz * rho, kz * u + ky * rho, al * (u + kx * c), al * (u - kx * c),
        kx * v + kz * rho, ky * v, kz * v - kx * rho, al * (v + ky * c), al * (v - ky * c),
        kx * w - ky * rho, ky * w + kx * rho, kz * w, al * (w + kz * c), al * (w - kz * c),
        kx * phi2 / (g - 1.0) + rho * (kz * v - ky * w), ky * phi2 / (g - 1.0) + rho * (kx * w - kz * u),
        kz * phi2 / (g - 1.0) + rho * (ky * u - kx * v),
        al * ((phi2 + c2) / (g - 1.0) + c * th), al * ((phi2 + c2) / (g - 1.0) - c * th)};
    const double Lm[25] = {
        kx * (1.0 - phi2 / c2) - (kz * v - ky * w) / rho, kx * (g - 1.0) * u / c2,
        kx * (g - 1.0) * v / c2 + kz / rho, kx * (g - 1.0) * w / c2 - ky / rho, -kx * (g - 1.0) / c2,
        ky * (1.0 - phi2 / c2) - (kx * w - kz * u) / rho, ky * (g - 1.0) * u / c2 - kz / rho,
        ky * (g - 1.0) * v / c2, ky * (g - 1.0) * w / c2 + kx / rho, -ky * (g - 1.0) / c2,
        kz * (1.0 - phi2 / c2) - (ky * u - kx * v) / rho, kz * (g - 1.0) * u / c2 + ky / rho,
        kz * (g - 1.0) * v / c2 - kx / rho, kz * (g - 1.0) * w / c2, -kz * (g - 1.0) / c2,
        be * (phi2 - c * th), be * (kx * c - (g - 1.0) * u), be * (ky * c - (g - 1.0) * v),
        be * (kz * c - (g - 1.0) * w), be * (g - 1.0),
        be * (phi2 + c * th), -be * (kx * c + (g - 1.0) * u), -be * (ky * c + (g - 1.0) * v),
        -be * (kz * c + (g - 1.0) * w), be * (g - 1.0)};
    memcpy(L, Lm, sizeof Lm);
    memcpy(R, Rm, sizeof Rm);
    lam[0] = lam[1] = lam[2] = th;
    lam[3] = th + c;
    lam[4] = th - c;
}

/* Reading R10, far field: state at a far-field node from the interior state
 * qi (node next to the boundary) and the outward unit normal nrm. */
static void farfield_state(const oproblem *P, const double qi[5], const double nrm[3], double qb[5]) {
    const double g = P->gamma;
    prim_t s = to_prim(P, qi);
    const double rinf = 1.0, pinf = 1.0 / g, cinf = 1.0;
    const double uinf[3] = {P->mach, 0.0, 0.0};
    const double ui[3] = {s.u, s.v, s.w};
    const double uni = nrm[0] * ui[0] + nrm[1] * ui[1] + nrm[2] * ui[2];
    const double unf = nrm[0] * uinf[0] + nrm[1] * uinf[1] + nrm[2] * uinf[2];
    double Rp = uni + 2.0 * s.c / (g - 1.0);     /* outgoing, from the interior  */
    double Rm = unf - 2.0 * cinf / (g - 1.0);    /* incoming, from the free stream */
    if (unf <= -cinf) Rp = unf + 2.0 * cinf / (g - 1.0);   /* supersonic inflow  */
    if (uni >= s.c) Rm = uni - 2.0 * s.c / (g - 1.0);      /* supersonic outflow */
    const double un = 0.5 * (Rp + Rm);
    const double cb = 0.25 * (g - 1.0) * (Rp - Rm);
    double ent, ut[3];
    if (un > 0.0) {
        ent = s.p / pow(s.rho, g);
        for (int m = 0; m < 3; ++m) ut[m] = ui[m] - uni * nrm[m];
    } else {
        ent = pinf / pow(rinf, g);
        for (int m = 0; m < 3; ++m) ut[m] = uinf[m] - unf * nrm[m];
    }
    const double rho = pow(cb * cb / (g * ent), 1.0 / (g - 1.0));
    const double p = rho * cb * cb / g;
    to_cons(P, rho, ut[0] + un * nrm[0], ut[1] + un * nrm[1], ut[2] + un * nrm[2], p, qb);
}

/* ------------------------------------------------------------------------ */
/* indexing and topology                                                     */
/* ------------------------------------------------------------------------ */

static size_t npts(const oblock *B) { return (size_t)B->n[0] * B->n[1] * B->n[2]; }

static size_t pidx(const oblock *B, const int id[3]) {
    return ((size_t)id[2] * B->n[1] + id[1]) * B->n[0] + id[0];
}

static size_t mpts(const oblock *B) { return (size_t)(B->n[0] + 6) * (B->n[1] + 6) * (B->n[2] + 6); }

static size_t midx(const oblock *B, const int id[3]) {
    return ((size_t)(id[2] + 3) * (B->n[1] + 6) + (id[1] + 3)) * (B->n[0] + 6) + (id[0] + 3);
}

static int is_phys(int kind) { return kind == OF_WALL || kind == OF_FARFIELD; }

/* Index in the neighbour across face f of block b of the node id, which
 * lies beyond face f (reading R14).  Layer l = 0, 1, .. beyond the face is
 * the neighbour's node at distance l from its joined face; the other
 * directions follow the transform (they may lie outside either block, for
 * the coordinates of edge and corner ghosts). */
static void across(const oproblem *P, int b, int f, const int id[3], int nid[3]) {
    const oblock *B = &P->b[b];
    const oface *F = &B->f[f];
    const oblock *N = &P->b[F->nbr];
    const int d = f / 2, side = f % 2;
    for (int a = 0; a < 3; ++a) {
        const int t = F->tf[a], p = abs(t) - 1;
        if (a == d) {
            const int l = side ? id[d] - B->n[d] : -1 - id[d];
            const int nside = F->nbr_face % 2;
            nid[p] = nside ? N->n[p] - 1 - l : l;
        } else {
            nid[p] = t > 0 ? id[a] : N->n[p] - 1 - id[a];
        }
    }
}

/* Coordinates at any index of block b within six layers of its faces
 * (reading R5).  Out-of-range directions are resolved k first, then j, then
 * i: a face neighbour supplies its node (plus the face translation), a
 * physical face reflects through its boundary node. */
static void coord_at(const oproblem *P, int b, const int id0[3], double out[3]) {
    const oblock *B = &P->b[b];
    int id[3] = {id0[0], id0[1], id0[2]};
    for (int d = 2; d >= 0; --d) {
        if (id[d] >= 0 && id[d] < B->n[d]) continue;
        const int side = id[d] < 0 ? 0 : 1;
        const oface *F = &B->f[2 * d + side];
        if (!is_phys(F->kind)) {
            int nid[3];
            across(P, b, 2 * d + side, id, nid);
            double c[3];
            coord_at(P, F->nbr, nid, c);
            for (int m = 0; m < 3; ++m) out[m] = c[m] + F->tr[m];
        } else {
            const int bn = side ? B->n[d] - 1 : 0;
            int bid[3] = {id[0], id[1], id[2]}, rid[3] = {id[0], id[1], id[2]};
            bid[d] = bn;
            rid[d] = 2 * bn - id[d];
            double xb[3], xr[3];
            coord_at(P, b, bid, xb);
            coord_at(P, b, rid, xr);
            for (int m = 0; m < 3; ++m) out[m] = 2.0 * xb[m] - xr[m];
        }
        return;
    }
    const size_t N = npts(B), p = pidx(B, id);
    for (int m = 0; m < 3; ++m) out[m] = B->x[m * N + p];
}

static void metric_at(const oblock *B, const int id[3], int dir, double m[3]) {
    const size_t M = mpts(B), p = midx(B, id);
    for (int c = 0; c < 3; ++c) m[c] = B->met[(3 * dir + c) * M + p];
}

static double jac_at(const oblock *B, const int id[3]) { return B->met[9 * mpts(B) + midx(B, id)]; }

/* Conservative state at an index that lies outside block b in at most one
 * direction d (the sweeps only read along their own line).  Qs[b] is the
 * state array of block b. */
static void state_at(const oproblem *P, double *const *Qs, int b, const int id[3], double q[5]) {
    const oblock *B = &P->b[b];
    int d = -1;
    for (int a = 0; a < 3; ++a)
        if (id[a] < 0 || id[a] >= B->n[a]) d = a;
    if (d < 0) {
        const size_t N = npts(B), p = pidx(B, id);
        for (int c = 0; c < 5; ++c) q[c] = Qs[b][c * N + p];
        return;
    }
    const int side = id[d] < 0 ? 0 : 1;
    const oface *F = &B->f[2 * d + side];
    int nid[3] = {id[0], id[1], id[2]};
    if (!is_phys(F->kind)) {
        across(P, b, 2 * d + side, id, nid);
        state_at(P, Qs, F->nbr, nid, q);
    } else if (F->kind == OF_WALL) {
        const int bn = side ? B->n[d] - 1 : 0;
        nid[d] = 2 * bn - id[d];
        state_at(P, Qs, b, nid, q);
        q[1] = -q[1];
        q[2] = -q[2];
        q[3] = -q[3];
    } else {
        const int bn = side ? B->n[d] - 1 : 0;
        int bid[3] = {id[0], id[1], id[2]};
        bid[d] = bn;
        nid[d] = side ? bn - 1 : bn + 1;
        double qi[5], m[3];
        state_at(P, Qs, b, nid, qi);
        metric_at(B, bid, d, m);
        const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        const double sg = side ? 1.0 : -1.0;
        const double nrm[3] = {sg * m[0] / mm, sg * m[1] / mm, sg * m[2] / mm};
        farfield_state(P, qi, nrm, q);
    }
}

/* Gradients (12) at an index outside block b in at most one direction that is
 * a periodic or interface face (physical faces use the one-sided closure and
 * never need ghost gradients). */
static void grad_at(const oproblem *P, int b, const int id[3], double g[12]) {
    const oblock *B = &P->b[b];
    int d = -1;
    for (int a = 0; a < 3; ++a)
        if (id[a] < 0 || id[a] >= B->n[a]) d = a;
    if (d < 0) {
        const size_t N = npts(B), p = pidx(B, id);
        for (int c = 0; c < 12; ++c) g[c] = B->grad[c * N + p];
        return;
    }
    const int side = id[d] < 0 ? 0 : 1;
    const oface *F = &B->f[2 * d + side];
    int nid[3];
    across(P, b, 2 * d + side, id, nid);
    grad_at(P, F->nbr, nid, g);
}

/* ------------------------------------------------------------------------ */
/* metrics: Eqs. (7)-(8)                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *X;   /* [3][n2+12][n1+12][n0+12] coordinates on [-6, n+5]^3 */
    int e[3];          /* extents n+12 */
} cbox;

static double cval(const cbox *C, int c, int i, int j, int k) {
    return C->X[(((size_t)c * C->e[2] + (k + 6)) * C->e[1] + (j + 6)) * C->e[0] + (i + 6)];
}

/* D along axis a of coordinate c at (i,j,k). */
static double dcoord(const cbox *C, int c, int a, int i, int j, int k) {
    double f[7];
    for (int s = -3; s <= 3; ++s) {
        int ii = i, jj = j, kk = k;
        if (a == 0) ii += s; else if (a == 1) jj += s; else kk += s;
        f[s + 3] = cval(C, c, ii, jj, kk);
    }
    return d6(f + 3);
}

/* (X_{ci, a_in} * X_cm)_{a_out} at (i,j,k): the outer D of the product of an
 * inner D and a coordinate, as each term of Eq. (7). */
static double prod_d(const cbox *C, int ci, int a_in, int cm, int a_out, int i, int j, int k) {
    double f[7];
    for (int s = -3; s <= 3; ++s) {
        int ii = i, jj = j, kk = k;
        if (a_out == 0) ii += s; else if (a_out == 1) jj += s; else kk += s;
        f[s + 3] = dcoord(C, ci, a_in, ii, jj, kk) * cval(C, cm, ii, jj, kk);
    }
    return d6(f + 3);
}

enum { XI = 0, ETA = 1, ZETA = 2, CX = 0, CY = 1, CZ = 2 };

static int block_metrics(oproblem *P, int b) {
    oblock *B = &P->b[b];
    cbox C;
    for (int d = 0; d < 3; ++d) C.e[d] = B->n[d] + 12;
    const size_t E = (size_t)C.e[0] * C.e[1] * C.e[2];
    double *X = (double *)malloc(3 * E * sizeof(double));
    if (!X) return -2;
    for (int k = -6; k < B->n[2] + 6; ++k)
        for (int j = -6; j < B->n[1] + 6; ++j)
            for (int i = -6; i < B->n[0] + 6; ++i) {
                int id[3] = {i, j, k};
                double x[3];
                coord_at(P, b, id, x);
                for (int c = 0; c < 3; ++c)
                    X[(((size_t)c * C.e[2] + (k + 6)) * C.e[1] + (j + 6)) * C.e[0] + (i + 6)] = x[c];
            }
    C.X = X;
    const size_t M = mpts(B);
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int k = -3; k < B->n[2] + 3; ++k)
        for (int j = -3; j < B->n[1] + 3; ++j)
            for (int i = -3; i < B->n[0] + 3; ++i) {
                double m[10];
                /* Eq. (7) */
                m[0] = prod_d(&C, CY, ETA, CZ, ZETA, i, j, k) - prod_d(&C, CY, ZETA, CZ, ETA, i, j, k);
                m[1] = prod_d(&C, CZ, ETA, CX, ZETA, i, j, k) - prod_d(&C, CZ, ZETA, CX, ETA, i, j, k);
                m[2] = prod_d(&C, CX, ETA, CY, ZETA, i, j, k) - prod_d(&C, CX, ZETA, CY, ETA, i, j, k);
                m[3] = prod_d(&C, CY, ZETA, CZ, XI, i, j, k) - prod_d(&C, CY, XI, CZ, ZETA, i, j, k);
                m[4] = prod_d(&C, CZ, ZETA, CX, XI, i, j, k) - prod_d(&C, CZ, XI, CX, ZETA, i, j, k);
                m[5] = prod_d(&C, CX, ZETA, CY, XI, i, j, k) - prod_d(&C, CX, XI, CY, ZETA, i, j, k);
                m[6] = prod_d(&C, CY, XI, CZ, ETA, i, j, k) - prod_d(&C, CY, ETA, CZ, XI, i, j, k);
                m[7] = prod_d(&C, CZ, XI, CX, ETA, i, j, k) - prod_d(&C, CZ, ETA, CX, XI, i, j, k);
                m[8] = prod_d(&C, CX, XI, CY, ETA, i, j, k) - prod_d(&C, CX, ETA, CY, XI, i, j, k);
                /* Eq. (8) */
                const double xx = dcoord(&C, CX, XI, i, j, k), xe = dcoord(&C, CX, ETA, i, j, k),
                             xz = dcoord(&C, CX, ZETA, i, j, k);
                const double yx = dcoord(&C, CY, XI, i, j, k), ye = dcoord(&C, CY, ETA, i, j, k),
                             yz = dcoord(&C, CY, ZETA, i, j, k);
                const double zx = dcoord(&C, CZ, XI, i, j, k), ze = dcoord(&C, CZ, ETA, i, j, k),
                             zz = dcoord(&C, CZ, ZETA, i, j, k);
                const double jinv = xx * ye * zz - xx * yz * ze + xe * yz * zx - xe * yx * zz
                                    + xz * yx * ze - xz * ye * zx;
                if (!(jinv > 0.0)) bad = 1;
                m[9] = 1.0 / jinv;
                const int id[3] = {i, j, k};
                const size_t p = midx(B, id);
                for (int c = 0; c < 10; ++c) B->met[c * M + p] = m[c];
            }
    free(X);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* right-hand side                                                           */
/* ------------------------------------------------------------------------ */

/* Inviscid contribution of direction d on one line of block b (modified
 * AFWENO, Sec. 4.5.1 and Fig. 11): A += f_x|_i of Eq. (19) per node. */
static void inviscid_line(const oproblem *P, double *const *Qs, int b, int d, const int base[3], double *A) {
    const oblock *B = &P->b[b];
    const int n = B->n[d], L = n + 6, O = 3;
    double *Q = (double *)malloc(sizeof(double) * 5 * L);
    double *Mt = (double *)malloc(sizeof(double) * 3 * L);
    double *Fp = (double *)malloc(sizeof(double) * 5 * L);   /* node fluxes               */
    double *UL = (double *)malloc(sizeof(double) * 5 * L);   /* U^L_{p+1/2} from node p    */
    double *UR = (double *)malloc(sizeof(double) * 5 * L);   /* U^R_{p-1/2} from node p    */
    double *H = (double *)malloc(sizeof(double) * 5 * L);    /* h_{f+1/2} at face f        */
    double *mc[3];
    for (int c = 0; c < 3; ++c) mc[c] = Mt + c * L;
    for (int p = -3; p < n + 3; ++p) {
        int id[3] = {base[0], base[1], base[2]};
        id[d] = p;
        double q[5], m[3];
        state_at(P, Qs, b, id, q);
        metric_at(B, id, d, m);
        for (int c = 0; c < 5; ++c) Q[c * L + p + O] = q[c];
        for (int c = 0; c < 3; ++c) mc[c][p + O] = m[c];
    }
    /* node fluxes, Eq. (4) */
    for (int p = -3; p < n + 3; ++p) {
        double q[5], m[3], f[5];
        for (int c = 0; c < 5; ++c) q[c] = Q[c * L + p + O];
        for (int c = 0; c < 3; ++c) m[c] = mc[c][p + O];
        point_flux(P, q, m, f);
        for (int c = 0; c < 5; ++c) Fp[c * L + p + O] = f[c];
    }
    if (P->scheme == 0) {
        /* modified AFWENO: characteristic space at node p gives
         * U^L_{p+1/2} and U^R_{p-1/2} from one stencil and shared indicators */
        for (int p = -1; p <= n; ++p) {
            double q[5], m[3], k[3], Le[25], Re[25], lam[5];
            for (int c = 0; c < 5; ++c) q[c] = Q[c * L + p + O];
            for (int c = 0; c < 3; ++c) m[c] = mc[c][p + O];
            const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            for (int c = 0; c < 3; ++c) k[c] = m[c] / mm;
            eigen(P, q, k, Le, Re, lam);
            double WL[5], WR[5];
            for (int l = 0; l < 5; ++l) {
                double W[5];
                for (int s = -2; s <= 2; ++s) {
                    double acc = 0.0;
                    for (int c = 0; c < 5; ++c) acc += Le[l * 5 + c] * Q[c * L + p + s + O];
                    W[s + 2] = acc;
                }
                double bt[3];
                weno_beta(W, bt);
                WL[l] = weno_left(W, bt);
                WR[l] = weno_right(W, bt);
            }
            for (int c = 0; c < 5; ++c) {
                double al = 0.0, ar = 0.0;
                for (int l = 0; l < 5; ++l) {
                    al += Re[c * 5 + l] * WL[l];
                    ar += Re[c * 5 + l] * WR[l];
                }
                UL[c * L + p + O] = al;
                UR[c * L + p + O] = ar;
            }
        }
    } else {
        /* original AFWENO (Fig. 9, reading R13): characteristic space at face
         * f+1/2 from the mean state and the face metric; two independent
         * WENO interpolations per face.  U^L of face f is kept at UL[f],
         * U^R of face f at UR[f+1], as in the modified scheme. */
        for (int f = -1; f <= n - 1; ++f) {
            double q[5], mf[3], k[3], Le[25], Re[25], lam[5];
            for (int c = 0; c < 5; ++c) q[c] = 0.5 * (Q[c * L + f + O] + Q[c * L + f + 1 + O]);
            for (int c = 0; c < 3; ++c) mf[c] = mid6(mc[c] + f + O);
            const double mm = sqrt(mf[0] * mf[0] + mf[1] * mf[1] + mf[2] * mf[2]);
            for (int c = 0; c < 3; ++c) k[c] = mf[c] / mm;
            eigen(P, q, k, Le, Re, lam);
            double WL[5], WR[5];
            for (int l = 0; l < 5; ++l) {
                double W[6];
                for (int s = -2; s <= 3; ++s) {
                    double acc = 0.0;
                    for (int c = 0; c < 5; ++c) acc += Le[l * 5 + c] * Q[c * L + f + s + O];
                    W[s + 2] = acc;
                }
                double bl[3], br[3];
                weno_beta(W, bl);       /* stencil f-2..f+2 */
                weno_beta(W + 1, br);   /* stencil f-1..f+3 */
                WL[l] = weno_left(W, bl);
                WR[l] = weno_right(W + 1, br);
            }
            for (int c = 0; c < 5; ++c) {
                double al = 0.0, ar = 0.0;
                for (int l = 0; l < 5; ++l) {
                    al += Re[c * 5 + l] * WL[l];
                    ar += Re[c * 5 + l] * WR[l];
                }
                UL[c * L + f + O] = al;
                UR[c * L + f + 1 + O] = ar;
            }
        }
    }
    /* Steger-Warming numerical flux at faces f+1/2, f = -1..n-1 */
    for (int f = -1; f <= n - 1; ++f) {
        double mf[3], ql[5], qr[5], Fpl[5], Fmr[5];
        for (int c = 0; c < 3; ++c) mf[c] = mid6(mc[c] + f + O);
        for (int c = 0; c < 5; ++c) {
            ql[c] = UL[c * L + f + O];
            qr[c] = UR[c * L + f + 1 + O];
        }
        sw_flux(P, ql, mf, +1, Fpl);
        sw_flux(P, qr, mf, -1, Fmr);
        for (int c = 0; c < 5; ++c) H[c * L + f + O] = Fpl[c] + Fmr[c];
    }
    /* Eq. (19) */
    const size_t N = npts(B);
    for (int p = 0; p < n; ++p) {
        int id[3] = {base[0], base[1], base[2]};
        id[d] = p;
        const size_t pi = pidx(B, id);
        for (int c = 0; c < 5; ++c)
            A[c * N + pi] += eq19(H[c * L + p + O], H[c * L + p - 1 + O], Fp + c * L + p + O);
    }
    free(Q); free(Mt); free(Fp); free(UL); free(UR); free(H);
}

/* Eq. (21) and Sec. 4.5.2: (u, v, w, T)_(x,y,z) at every node of block b;
 * the (xi, eta, zeta) derivatives use the sixth-order central operator, or
 * the closure of reading R9 next to physical faces. */
static void gradients(const oproblem *P, double *const *Qs, int b) {
    oblock *B = &P->b[b];
    const size_t N = npts(B);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < B->n[2]; ++k)
        for (int j = 0; j < B->n[1]; ++j)
            for (int i = 0; i < B->n[0]; ++i) {
                const int id[3] = {i, j, k};
                double dc[4][3];   /* d(phi)/d(xi, eta, zeta) for phi = u, v, w, T */
                for (int d = 0; d < 3; ++d) {
                    const int n = B->n[d], c0 = id[d];
                    const int lo = is_phys(B->f[2 * d].kind), hi = is_phys(B->f[2 * d + 1].kind);
                    double *lb = (double *)malloc(sizeof(double) * 4 * (n + 6));   /* nodes -3..n+2 */
                    for (int p = c0 - 4; p <= c0 + 4; ++p) {
                        if (p < -3 || p > n + 2 || (lo && p < 0) || (hi && p >= n)) continue;
                        int nid[3] = {i, j, k};
                        nid[d] = p;
                        double q[5];
                        state_at(P, Qs, b, nid, q);
                        prim_t st = to_prim(P, q);
                        lb[0 * (n + 6) + p + 3] = st.u;
                        lb[1 * (n + 6) + p + 3] = st.v;
                        lb[2 * (n + 6) + p + 3] = st.w;
                        lb[3 * (n + 6) + p + 3] = st.T;
                    }
                    for (int v = 0; v < 4; ++v) dc[v][d] = dline(lb + v * (n + 6) + 3, c0, n, lo, hi);
                    free(lb);
                }
                double mx[3][3];   /* mx[dir][comp] conservative metric */
                for (int d = 0; d < 3; ++d) metric_at(B, id, d, mx[d]);
                const double J = jac_at(B, id);
                const size_t p = pidx(B, id);
                for (int v = 0; v < 4; ++v)
                    for (int c = 0; c < 3; ++c)
                        B->grad[(v * 3 + c) * N + p] =
                            J * (mx[0][c] * dc[v][0] + mx[1][c] * dc[v][1] + mx[2][c] * dc[v][2]);
            }
}

/* Eqs. (5)-(6) with reading R12: viscous flux along metric m at a node with
 * primitive state s and gradients g = (u,v,w,T)_(x,y,z). */
static void viscous_flux(const oproblem *P, const prim_t *s, const double g[12], const double m[3], double fv[5]) {
    const double mu = viscosity(P, s->T);
    const double kv = P->mach / P->re * mu;
    const double kq = kv / (P->pr * (P->gamma - 1.0));
    const double ux = g[0], uy = g[1], uz = g[2], vx = g[3], vy = g[4], vz = g[5];
    const double wx = g[6], wy = g[7], wz = g[8], Tx = g[9], Ty = g[10], Tz = g[11];
    const double div = ux + vy + wz;
    const double lam = -2.0 / 3.0 * kv;
    const double txx = lam * div + 2.0 * kv * ux, tyy = lam * div + 2.0 * kv * vy, tzz = lam * div + 2.0 * kv * wz;
    const double txy = kv * (uy + vx), txz = kv * (uz + wx), tyz = kv * (vz + wy);
    const double bx = s->u * txx + s->v * txy + s->w * txz + kq * Tx;
    const double by = s->u * txy + s->v * tyy + s->w * tyz + kq * Ty;
    const double bz = s->u * txz + s->v * tyz + s->w * tzz + kq * Tz;
    fv[0] = 0.0;
    fv[1] = m[0] * txx + m[1] * txy + m[2] * txz;
    fv[2] = m[0] * txy + m[1] * tyy + m[2] * tyz;
    fv[3] = m[0] * txz + m[1] * tyz + m[2] * tzz;
    fv[4] = m[0] * bx + m[1] * by + m[2] * bz;
}

/* Fig. 12: A -= D_d(E_v,d) on one line. */
static void viscous_line(const oproblem *P, double *const *Qs, int b, int d, const int base[3], double *A) {
    const oblock *B = &P->b[b];
    const int n = B->n[d], L = n + 6, O = 3;
    const int lo = is_phys(B->f[2 * d].kind), hi = is_phys(B->f[2 * d + 1].kind);
    double *Fv = (double *)malloc(sizeof(double) * 5 * L);
    for (int p = -3; p < n + 3; ++p) {
        if ((lo && p < 0) || (hi && p >= n)) continue;
        int id[3] = {base[0], base[1], base[2]};
        id[d] = p;
        double q[5], m[3], g[12], fv[5];
        state_at(P, Qs, b, id, q);
        prim_t s = to_prim(P, q);
        grad_at(P, b, id, g);
        metric_at(B, id, d, m);
        viscous_flux(P, &s, g, m, fv);
        for (int c = 0; c < 5; ++c) Fv[c * L + p + O] = fv[c];
    }
    const size_t N = npts(B);
    for (int p = 0; p < n; ++p) {
        int id[3] = {base[0], base[1], base[2]};
        id[d] = p;
        const size_t pi = pidx(B, id);
        for (int c = 1; c < 5; ++c) A[c * N + pi] -= dline(Fv + c * L + O, p, n, lo, hi);
    }
    free(Fv);
}

/* R = dQ/dt = -J * sum_d (D_d(E_d) - D_d(E_v,d)), from Eqs. (2)-(3). */
static void rhs_all(oproblem *P, double *const *Qs) {
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        memset(B->r, 0, sizeof(double) * 5 * npts(B));
    }
    if (P->viscous)
        for (int b = 0; b < P->nb; ++b) gradients(P, Qs, b);
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        for (int d = 0; d < 3; ++d) {
            const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            const int nl = B->n[a1] * B->n[a2];
#pragma omp parallel for schedule(dynamic)
            for (int l = 0; l < nl; ++l) {
                int base[3] = {0, 0, 0};
                base[a1] = l % B->n[a1];
                base[a2] = l / B->n[a1];
                inviscid_line(P, Qs, b, d, base, B->r);
                if (P->viscous) viscous_line(P, Qs, b, d, base, B->r);
            }
        }
        const size_t N = npts(B);
        for (int k = 0; k < B->n[2]; ++k)
            for (int j = 0; j < B->n[1]; ++j)
                for (int i = 0; i < B->n[0]; ++i) {
                    const int id[3] = {i, j, k};
                    const size_t p = pidx(B, id);
                    const double J = jac_at(B, id);
                    for (int c = 0; c < 5; ++c) B->r[c * N + p] = -J * B->r[c * N + p];
                }
    }
}

/* Reading R10: node values on physical faces after an RK stage. */
static void bc_nodes(oproblem *P, double *const *Qs) {
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        const size_t N = npts(B);
        for (int f = 0; f < 6; ++f) {
            const int kind = B->f[f].kind;
            if (kind != OF_WALL) continue;
            const int d = f / 2, side = f % 2, a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            for (int t2 = 0; t2 < B->n[a2]; ++t2)
                for (int t1 = 0; t1 < B->n[a1]; ++t1) {
                    int id[3];
                    id[d] = side ? B->n[d] - 1 : 0;
                    id[a1] = t1;
                    id[a2] = t2;
                    const size_t p = pidx(B, id);
                    double q[5];
                    for (int c = 0; c < 5; ++c) q[c] = Qs[b][c * N + p];
                    prim_t s = to_prim(P, q);
                    Qs[b][1 * N + p] = 0.0;
                    Qs[b][2 * N + p] = 0.0;
                    Qs[b][3 * N + p] = 0.0;
                    Qs[b][4 * N + p] = s.p / (P->gamma - 1.0);
                }
        }
    }
    /* far-field nodes read the updated neighbouring node; walls are done first */
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        const size_t N = npts(B);
        for (int f = 0; f < 6; ++f) {
            if (B->f[f].kind != OF_FARFIELD) continue;
            const int d = f / 2, side = f % 2, a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            for (int t2 = 0; t2 < B->n[a2]; ++t2)
                for (int t1 = 0; t1 < B->n[a1]; ++t1) {
                    int id[3], in[3];
                    id[d] = side ? B->n[d] - 1 : 0;
                    id[a1] = t1;
                    id[a2] = t2;
                    in[0] = id[0]; in[1] = id[1]; in[2] = id[2];
                    in[d] = side ? id[d] - 1 : id[d] + 1;
                    double qi[5], m[3], qb[5];
                    const size_t pi = pidx(B, in), p = pidx(B, id);
                    for (int c = 0; c < 5; ++c) qi[c] = Qs[b][c * N + pi];
                    metric_at(B, id, d, m);
                    const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                    const double sg = side ? 1.0 : -1.0;
                    const double nrm[3] = {sg * m[0] / mm, sg * m[1] / mm, sg * m[2] / mm};
                    farfield_state(P, qi, nrm, qb);
                    for (int c = 0; c < 5; ++c) Qs[b][c * N + p] = qb[c];
                }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* exported API (ctypes)                                                     */
/* ------------------------------------------------------------------------ */

/* cfg = {gamma, mach, reynolds, prandtl, sutherland_s, viscous, mu_law, scheme} */
void *orc_new(const double *cfg) {
    oproblem *P = (oproblem *)calloc(1, sizeof(oproblem));
    P->gamma = cfg[0];
    P->mach = cfg[1];
    P->re = cfg[2];
    P->pr = cfg[3];
    P->suth = cfg[4];
    P->viscous = (int)cfg[5];
    P->mu_law = (int)cfg[6];
    P->scheme = (int)cfg[7];
    return P;
}

int orc_add_block(void *h, int ni, int nj, int nk, const double *xyz) {
    oproblem *P = (oproblem *)h;
    if (ni < 6 || nj < 6 || nk < 6) return -1;
    if (P->nb == P->cap) {
        P->cap = P->cap ? 2 * P->cap : 8;
        P->b = (oblock *)realloc(P->b, sizeof(oblock) * P->cap);
    }
    oblock *B = &P->b[P->nb];
    memset(B, 0, sizeof *B);
    B->n[0] = ni;
    B->n[1] = nj;
    B->n[2] = nk;
    const size_t N = npts(B);
    B->x = (double *)malloc(sizeof(double) * 3 * N);
    memcpy(B->x, xyz, sizeof(double) * 3 * N);
    for (int f = 0; f < 6; ++f) B->f[f].kind = OF_UNSET;
    B->met = (double *)calloc(10 * mpts(B), sizeof(double));
    B->q = (double *)calloc(5 * N, sizeof(double));
    B->qn = (double *)calloc(5 * N, sizeof(double));
    B->qs = (double *)calloc(5 * N, sizeof(double));
    B->r = (double *)calloc(5 * N, sizeof(double));
    B->grad = (double *)calloc(12 * N, sizeof(double));
    return P->nb++;
}

int orc_set_face(void *h, int b, int f, int kind, int nbr, int nbr_face, const double *tr) {
    oproblem *P = (oproblem *)h;
    if (b < 0 || b >= P->nb || f < 0 || f > 5) return -1;
    oface *F = &P->b[b].f[f];
    F->kind = kind;
    F->nbr = nbr;
    F->nbr_face = nbr_face;
    for (int a = 0; a < 3; ++a) F->tf[a] = a + 1;
    for (int m = 0; m < 3; ++m) F->tr[m] = tr ? tr[m] : 0.0;
    return 0;
}

/* Index transform of face f of block b (reading R14); call after
 * orc_set_face, whose default is the identity. */
int orc_set_face_transform(void *h, int b, int f, const int *tf) {
    oproblem *P = (oproblem *)h;
    if (b < 0 || b >= P->nb || f < 0 || f > 5) return -1;
    for (int a = 0; a < 3; ++a) P->b[b].f[f].tf[a] = tf[a];
    return 0;
}

/* Checks that every face is set and that each face connection is a
 * consistent 1:1 join (reading R14): the transform is a signed permutation
 * with determinant +1 (both blocks keep a right-handed index space), its
 * normal entry points to the neighbour's face with the sign that the two
 * sides imply, the neighbour's face points back with the inverse transform,
 * and the extents along the face agree. */
int orc_check(void *h) {
    oproblem *P = (oproblem *)h;
    for (int b = 0; b < P->nb; ++b)
        for (int f = 0; f < 6; ++f) {
            const oface *F = &P->b[b].f[f];
            if (F->kind == OF_UNSET) return -1;
            if (is_phys(F->kind)) continue;
            if (F->nbr < 0 || F->nbr >= P->nb || F->nbr_face < 0 || F->nbr_face > 5) return -1;
            const int d = f / 2, side = f % 2, nd = F->nbr_face / 2, nside = F->nbr_face % 2;
            int seen = 0, M[3][3] = {{0}};
            for (int a = 0; a < 3; ++a) {
                const int t = F->tf[a];
                if (t == 0 || abs(t) > 3) return -1;
                seen |= 1 << (abs(t) - 1);
                M[abs(t) - 1][a] = t > 0 ? 1 : -1;
            }
            if (seen != 7) return -1;
            const int det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                            M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                            M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            if (det != 1) return -1;
            if (abs(F->tf[d]) - 1 != nd || (F->tf[d] > 0) != (side != nside)) return -1;
            const oface *Bk = &P->b[F->nbr].f[F->nbr_face];
            if (is_phys(Bk->kind) || Bk->nbr != b || Bk->nbr_face != f) return -1;
            for (int a = 0; a < 3; ++a) {
                const int t = F->tf[a], p = abs(t) - 1;
                const int u = Bk->tf[p];
                if (abs(u) - 1 != a || (u > 0) != (t > 0)) return -1;
                if (a != d && P->b[F->nbr].n[p] != P->b[b].n[a]) return -1;
            }
        }
    return 0;
}

int orc_metrics(void *h) {
    oproblem *P = (oproblem *)h;
    int rc = 0;
    for (int b = 0; b < P->nb; ++b) {
        int r = block_metrics(P, b);
        if (r) rc = r;
    }
    return rc;
}

/* Metrics of block b: out = [10][n2+6][n1+6][n0+6] on [-3, n+2]^3 when
 * padded != 0, else [10][n2][n1][n0] interior. */
void orc_get_metrics(void *h, int b, double *out, int padded) {
    oproblem *P = (oproblem *)h;
    oblock *B = &P->b[b];
    const size_t M = mpts(B);
    if (padded) {
        memcpy(out, B->met, sizeof(double) * 10 * M);
        return;
    }
    const size_t N = npts(B);
    for (int c = 0; c < 10; ++c)
        for (int k = 0; k < B->n[2]; ++k)
            for (int j = 0; j < B->n[1]; ++j)
                for (int i = 0; i < B->n[0]; ++i) {
                    const int id[3] = {i, j, k};
                    out[c * N + pidx(B, id)] = B->met[c * M + midx(B, id)];
                }
}

void orc_set_state(void *h, int b, const double *q) {
    oproblem *P = (oproblem *)h;
    memcpy(P->b[b].q, q, sizeof(double) * 5 * npts(&P->b[b]));
}

void orc_get_state(void *h, int b, double *q) {
    oproblem *P = (oproblem *)h;
    memcpy(q, P->b[b].q, sizeof(double) * 5 * npts(&P->b[b]));
}

static double **state_ptrs(oproblem *P, int which) {
    double **Qs = (double **)malloc(sizeof(double *) * (P->nb ? P->nb : 1));
    for (int b = 0; b < P->nb; ++b) Qs[b] = which == 0 ? P->b[b].q : which == 1 ? P->b[b].qn : P->b[b].qs;
    return Qs;
}

/* R(Q) of the current state, kept per block (orc_get_rhs). */
void orc_rhs(void *h) {
    oproblem *P = (oproblem *)h;
    double **Qs = state_ptrs(P, 0);
    rhs_all(P, Qs);
    free(Qs);
}

void orc_get_rhs(void *h, int b, double *r) {
    oproblem *P = (oproblem *)h;
    memcpy(r, P->b[b].r, sizeof(double) * 5 * npts(&P->b[b]));
}

void orc_get_grad(void *h, int b, double *g) {
    oproblem *P = (oproblem *)h;
    memcpy(g, P->b[b].grad, sizeof(double) * 12 * npts(&P->b[b]));
}

/* Convective spectral radius of node id of block B (reading R8):
 * sum_d (|m_d.u| + c |m_d|) J. */
static double lambda_c(const oproblem *P, const oblock *B, const int id[3], const double q[5]) {
    prim_t s = to_prim(P, q);
    const double J = jac_at(B, id);
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {
        double m[3];
        metric_at(B, id, d, m);
        const double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        sum += (fabs(m[0] * s.u + m[1] * s.v + m[2] * s.w) + s.c * mm) * J;
    }
    return sum;
}

/* Local time step of node id (reading R15). */
static double local_dt(const oproblem *P, const oblock *B, const int id[3], const double q[5], double cfl) {
    double lam = lambda_c(P, B, id, q);
    if (P->viscous) {
        prim_t s = to_prim(P, q);
        const double J = jac_at(B, id);
        double g2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double m[3];
            metric_at(B, id, d, m);
            g2 += J * J * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        }
        const double gp = P->gamma / P->pr;
        lam += P->mach / P->re * (gp > 4.0 / 3.0 ? gp : 4.0 / 3.0) * viscosity(P, s.T) / s.rho * g2;
    }
    return cfl / lam;
}

/* Eq. (20), nsteps steps.  Time step per block (dt[b]) or, when dtl is not
 * NULL, per node: dtl[b] holds each node's local step of the state at the
 * start of the step (reading R15), refreshed every step from cfl. */
static void step_rk3(oproblem *P, int nsteps, const double *dt, double **dtl, double cfl) {
    double **Qc = state_ptrs(P, 0), **Qs = state_ptrs(P, 2);
    for (int it = 0; it < nsteps; ++it) {
        for (int b = 0; b < P->nb; ++b) memcpy(P->b[b].qn, P->b[b].q, sizeof(double) * 5 * npts(&P->b[b]));
        if (dtl) {
            for (int b = 0; b < P->nb; ++b) {
                oblock *B = &P->b[b];
                const size_t N = npts(B);
                for (int k = 0; k < B->n[2]; ++k)
                    for (int j = 0; j < B->n[1]; ++j)
                        for (int i = 0; i < B->n[0]; ++i) {
                            const int id[3] = {i, j, k};
                            const size_t pp = pidx(B, id);
                            double q[5];
                            for (int c = 0; c < 5; ++c) q[c] = B->qn[c * N + pp];
                            dtl[b][pp] = local_dt(P, B, id, q, cfl);
                        }
            }
        }
        /* stage 1: Q1 = Qn + dt R(Qn) */
        rhs_all(P, Qc);
        for (int b = 0; b < P->nb; ++b) {
            oblock *B = &P->b[b];
            const size_t N = npts(B), M5 = 5 * N;
            for (size_t t = 0; t < M5; ++t) {
                const double h = dtl ? dtl[b][t % N] : dt[b];
                B->qs[t] = B->qn[t] + h * B->r[t];
            }
        }
        bc_nodes(P, Qs);
        /* stage 2: Q2 = 3/4 Qn + 1/4 Q1 + 1/4 dt R(Q1) */
        rhs_all(P, Qs);
        for (int b = 0; b < P->nb; ++b) {
            oblock *B = &P->b[b];
            const size_t N = npts(B), M5 = 5 * N;
            for (size_t t = 0; t < M5; ++t) {
                const double h = dtl ? dtl[b][t % N] : dt[b];
                B->qs[t] = 3.0 / 4.0 * B->qn[t] + 1.0 / 4.0 * B->qs[t] + 1.0 / 4.0 * h * B->r[t];
            }
        }
        bc_nodes(P, Qs);
        /* stage 3: Q^{n+1} = 1/3 Qn + 2/3 Q2 + 2/3 dt R(Q2) */
        rhs_all(P, Qs);
        for (int b = 0; b < P->nb; ++b) {
            oblock *B = &P->b[b];
            const size_t N = npts(B), M5 = 5 * N;
            for (size_t t = 0; t < M5; ++t) {
                const double h = dtl ? dtl[b][t % N] : dt[b];
                B->q[t] = 1.0 / 3.0 * B->qn[t] + 2.0 / 3.0 * B->qs[t] + 2.0 / 3.0 * h * B->r[t];
            }
        }
        bc_nodes(P, Qc);
    }
    free(Qc);
    free(Qs);
}

/* Eq. (20) with dt[b] per block, nsteps steps. */
void orc_step_multi(void *h, int nsteps, const double *dt) {
    step_rk3((oproblem *)h, nsteps, dt, NULL, 0.0);
}

void orc_step(void *h, int nsteps, double dt) {
    oproblem *P = (oproblem *)h;
    double *d = (double *)malloc(sizeof(double) * (P->nb ? P->nb : 1));
    for (int b = 0; b < P->nb; ++b) d[b] = dt;
    orc_step_multi(h, nsteps, d);
    free(d);
}

/* Local time stepping (reading R15): nsteps steps, each node with its own
 * time step from the state at the start of the step. */
void orc_step_local(void *h, int nsteps, double cfl) {
    oproblem *P = (oproblem *)h;
    double **dtl = (double **)malloc(sizeof(double *) * (P->nb ? P->nb : 1));
    for (int b = 0; b < P->nb; ++b) dtl[b] = (double *)malloc(sizeof(double) * npts(&P->b[b]));
    step_rk3(P, nsteps, NULL, dtl, cfl);
    for (int b = 0; b < P->nb; ++b) free(dtl[b]);
    free(dtl);
}

/* Local time steps (reading R15) of the current state of block b,
 * [nk][nj][ni]. */
void orc_dt_local(void *h, int b, double cfl, double *out) {
    oproblem *P = (oproblem *)h;
    oblock *B = &P->b[b];
    const size_t N = npts(B);
    for (int k = 0; k < B->n[2]; ++k)
        for (int j = 0; j < B->n[1]; ++j)
            for (int i = 0; i < B->n[0]; ++i) {
                const int id[3] = {i, j, k};
                const size_t pp = pidx(B, id);
                double q[5];
                for (int c = 0; c < 5; ++c) q[c] = B->q[c * N + pp];
                out[pp] = local_dt(P, B, id, q, cfl);
            }
}

/* Reading R8: dt_out[b] = cfl / max over nodes of block b of
 * sum_d (|m_d.u| + c |m_d|) J.  Returns the minimum over blocks. */
double orc_dt(void *h, double cfl, double *dt_out) {
    oproblem *P = (oproblem *)h;
    double dmin = INFINITY;
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        const size_t N = npts(B);
        double smax = 0.0;
        for (int k = 0; k < B->n[2]; ++k)
            for (int j = 0; j < B->n[1]; ++j)
                for (int i = 0; i < B->n[0]; ++i) {
                    const int id[3] = {i, j, k};
                    const size_t pp = pidx(B, id);
                    double q[5];
                    for (int c = 0; c < 5; ++c) q[c] = B->q[c * N + pp];
                    const double sum = lambda_c(P, B, id, q);
                    if (sum > smax) smax = sum;
                }
        const double dt = cfl / smax;
        if (dt_out) dt_out[b] = dt;
        if (dt < dmin) dmin = dt;
    }
    return dmin;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_free(void *h) {
    oproblem *P = (oproblem *)h;
    if (!P) return;
    for (int b = 0; b < P->nb; ++b) {
        oblock *B = &P->b[b];
        free(B->x); free(B->met); free(B->q); free(B->qn); free(B->qs); free(B->r); free(B->grad);
    }
    free(P->b);
    free(P);
}

/* ---- single operators, exported for the pins in the test suite -------- */

void orc_op_weno(const double *W, double *beta3, double *left, double *right) {
    double b[3];
    weno_beta(W, b);
    for (int j = 0; j < 3; ++j) beta3[j] = b[j];
    *left = weno_left(W, b);
    *right = weno_right(W, b);
}

double orc_op_d6(const double *f7) { return d6(f7 + 3); }

double orc_op_mid6(const double *f6) { return mid6(f6 + 2); }

double orc_op_eq19(double hp, double hm, const double *f7) { return eq19(hp, hm, f7 + 3); }

double orc_op_dline(const double *f, int p, int n, int lo, int hi) { return dline(f, p, n, lo, hi); }

void orc_op_eigen(void *h, const double *q, const double *k, double *L, double *R, double *lam) {
    eigen((oproblem *)h, q, k, L, R, lam);
}

void orc_op_sw_flux(void *h, const double *q, const double *m, int sign, double *F) {
    sw_flux((oproblem *)h, q, m, sign, F);
}

void orc_op_point_flux(void *h, const double *q, const double *m, double *f) { point_flux((oproblem *)h, q, m, f); }

void orc_op_farfield(void *h, const double *qi, const double *nrm, double *qb) {
    farfield_state((oproblem *)h, qi, nrm, qb);
}

void orc_op_viscous_flux(void *h, const double *q, const double *g, const double *m, double *fv) {
    oproblem *P = (oproblem *)h;
    prim_t s = to_prim(P, q);
    viscous_flux(P, &s, g, m, fv);
}
