// hx_common.cuh -- device layout, block table and the per-node arithmetic of
// the RK-stage residual (Ye et al., HiResX), templated on the working real
// type R (double for the FP64 form, float for the mixed form).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hx {

// ---------------------------------------------------------------------------
// layout
// ---------------------------------------------------------------------------
// Every block-resident field lives in one arena per buffer: field f of block
// b, node (i, j, k) is element  f * fstride + base_b + i + j * sj_b + k * sk_b.
// State-like fields carry G = 3 ghost layers per face (the reach of the
// six-point stencils of Eqs. (18)-(19)); node coordinates carry GC = 6 (inner
// and outer derivative of Eq. (7)).  Rows are padded so that i = 0 of every
// row sits at an 8-element boundary.
constexpr int G = 3;
constexpr int GC = 6;
constexpr int XOFF = 8;

struct DevBlock {
    int n[3];         // interior nodes per direction
    int sj, sk;       // element strides of the state layout (si = 1)
    long long base;   // element index of node (0, 0, 0) in the state layout
    int phys;         // bit f: face f is a physical face (wall or far field)
    int wall;         // bit f: face f is a wall
    int ff;           // bit f: face f is a far field
    int nbr[6];       // block joined across face f (periodic / interface), -1 on physical faces
    // index transform of face f (1:1 interface, Sec. 4.2): axis a of this
    // block runs along axis |tf[f][a]|-1 of the neighbour, reversed when
    // negative (the CGNS 1-to-1 convention); identity for aligned blocks
    signed char tf[6][3];
    double dt;        // time step of this block
    long long lim;    // elements per field of the layout (checking builds: node offsets must be below)
    unsigned* flags;  // device error word (checking builds record FLAG_BOUNDS there), or null
};

struct Gas {
    double gamma, mach, re, pr, suth;
    int viscous, mu_law;
};

struct Tile {          // origin of a sweep tile (node indices)
    int b, i0, j0, k0;
};

struct Brick {         // box [i0, i0+ni) x [j0, j0+nj) x [k0, k0+nk) of block b
    int b, i0, j0, k0, ni, nj, nk, pad;
};

struct HaloItem {      // one ghost node: dst <- f(src, aux)
    int dst, src, aux, mode;
};

struct NodeItem {      // a node on a physical face: block, indices, face direction and side
    int b, i, j, k, dir, side, pad0, pad1;
};

enum : int { FLAG_NONFINITE = 1, FLAG_BAD_GRID = 2, FLAG_UNPHYSICAL = 4, FLAG_BOUNDS = 8 };

// The RK3 stage combination (Eq. (20)) fused into the last sweep:
// Q_out = ca Q^n + cb Q^(k) + cc dt R, R = -J A, in FP64.
struct RKArgs {
    const double* Qn;     // Q^n (read at the node only)
    const double* Qk;     // stage input Q^(k), FP64
    const double* metd;   // FP64 metrics; field 9 is J
    double* Qout;         // stage output, FP64
    float* Qfout;         // FP32 copy of the stage output (mixed form) or null
    const float* Aref;    // mixed form: the FP32 divergence of the rest state (rounding only), or null
    const double* dtl;    // local time stepping: the time step of every node (field layout), or null
    double ca, cb, cc, gm1;
    float ccf;            // -cc in FP32 (the mixed form's FP32 increment)
    float* primout;       // mixed Navier-Stokes, a stage whose output feeds the next: the FP32
                          // (u, v, w, T) of the output at the node, so that the next stage's
                          // prep fills only the ghosts; or null
    unsigned* flags;
};

// L2 prefetch hint for one global address: no register result, nothing to
// wait for.  The address must lie inside a device allocation.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// Non-finite test on the exponent bits (integer pipe, not the FP64 unit).
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}

// Exact FP32 -> FP64 widening and FP64 -> FP32 narrowing (IEEE 754
// round-to-nearest-even) on the integer pipe.  GB300 executes the
// conversion instructions on its FP64 unit, whose rate is 1/64 of FP32;
// a point-parallel kernel with ten FP64 FMAs per node is held by it.  Both
// follow the binary formats bit by bit (sign, exponent rebias by 896,
// mantissa shift by 29), subnormals and non-finite values included.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned s = b & 0x80000000u, em = b & 0x7fffffffu;
    if (em >= 0x00800000u && em < 0x7f800000u)   // normal
        return __hiloint2double((int)(s | ((em >> 3) + (896u << 20))), (int)(em << 29));
    if (em == 0u) return __hiloint2double((int)s, 0);
    if (em >= 0x7f800000u)   // infinity, or a quiet NaN
        return __hiloint2double((int)(s | (em == 0x7f800000u ? 0x7ff00000u : 0x7ff80000u)), 0);
    // subnormal em * 2^-149: the leading bit n becomes the implicit one
    const int n = 31 - __clz(em);
    const unsigned long long m = ((unsigned long long)em << (52 - n)) & 0x000fffffffffffffULL;
    return __longlong_as_double((long long)(((unsigned long long)s << 32) |
                                            ((unsigned long long)(n + 874) << 52) | m));
}

__device__ __forceinline__ float narrow_f64_rn(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned s = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) return __uint_as_float(s | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
    const int fe = e - 896;   // biased FP32 exponent
    if (fe >= 0xff) return __uint_as_float(s | 0x7f800000u);
    if (fe > 0) {   // normal: keep 23 mantissa bits, round the other 29 to nearest, ties to even
        const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        const unsigned r = (((unsigned)fe << 23) | mant) + ((rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u);
        return __uint_as_float(s | r);   // a carry moves into the exponent (up to infinity)
    }
    if (e == 0) return __uint_as_float(s);   // zero, or an FP64 subnormal
    // FP32 subnormal (or zero) result: the 53-bit significand times 2^(e - 926)
    const unsigned long long m = ((((unsigned long long)(hi & 0xfffffu)) << 32) | lo) | (1ULL << 52);
    const int sh = 926 - e;   // >= 30
    if (sh >= 64) return __uint_as_float(s);
    const unsigned long long q = m >> sh, rem = m & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
    return __uint_as_float(s | (unsigned)(q + ((rem > half || (rem == half && (q & 1ULL))) ? 1ULL : 0ULL)));
}

// HaloItem.mode: bits 0-3 kind, bits 4-5 direction, bit 6 side (1 = + face),
// bits 8.. translation index (coordinates).
enum : int { HM_COPY = 0, HM_WALL = 1, HM_FARFIELD = 2, HM_TRANSLATE = 3, HM_REFLECT = 4 };

// A node offset into a field of block B's layout.  Checking builds
// (HX_BOUNDS) verify it lies inside the field; an offset outside records
// FLAG_BOUNDS and is replaced by 0 (a padding element), so the access stays
// inside the buffer and the host reports HX_ERR_BOUNDS.  No trap.
__host__ __device__ inline long long hx_chk(const DevBlock& B, long long e) {
#if defined(HX_BOUNDS) && defined(__CUDA_ARCH__)
    if (e < 0 || e >= B.lim) {
        if (B.flags) atomicOr(B.flags, (unsigned)FLAG_BOUNDS);
        return 0;
    }
#else
    (void)B;
#endif
    return e;
}

__host__ __device__ inline long long node_index(const DevBlock& B, int i, int j, int k) {
    return hx_chk(B, B.base + i + (long long)j * B.sj + (long long)k * B.sk);
}

// Index in the neighbour N (extents nN) across face f of block B of the
// index id of B, which lies beyond face f: layer l = 0, 1, .. beyond the
// face is N's node at distance l from its joined face; the other directions
// follow the face transform (they may lie outside either block, for the
// coordinates of edge and corner ghosts).
__host__ __device__ inline void across_face(const DevBlock& B, const int nN[3], int f, const int id[3], int out[3]) {
    const int d = f >> 1, side = f & 1;
    int v[3], p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int t = B.tf[f][a];
        p[a] = (t < 0 ? -t : t) - 1;
        if (a == d) {
            const int l = side ? id[d] - B.n[d] : -1 - id[d];
            const int nside = t > 0 ? 1 - side : side;
            v[a] = nside ? nN[p[a]] - 1 - l : l;
        } else {
            v[a] = t > 0 ? id[a] : nN[p[a]] - 1 - id[a];
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) out[q] = p[0] == q ? v[0] : (p[1] == q ? v[1] : v[2]);
}

// The face ghost of N that a node (indices id, at distance s from face f
// of its block) fills: the inverse of across_face.  tf is the face's
// transform, read from the block table where the push needs it.
__device__ __forceinline__ void ghost_across(const signed char* tf, const DevBlock& N, int f, int s,
                                             const int id[3], int out[3]) {
    const int d = f >> 1, side = f & 1;
    int v[3], p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int t = tf[a];
        p[a] = (t < 0 ? -t : t) - 1;
        if (a == d) {
            const int nside = t > 0 ? 1 - side : side;
            v[a] = nside ? N.n[p[a]] + s : -1 - s;
        } else {
            v[a] = t > 0 ? id[a] : N.n[p[a]] - 1 - id[a];
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) out[q] = p[0] == q ? v[0] : (p[1] == q ? v[1] : v[2]);
}

// Halo by push: node id of block B sends its values `vals` (nf fields) to
// the face ghosts they fill in the blocks joined across its faces (nodes
// within G of a periodic or interface face), and, with `mirror`, to B's own
// wall-mirror ghosts (nodes 1..G from a wall; fields 1..3, the momentum,
// negated).  Each ghost has exactly one sender, so no synchronisation is
// needed; the ghosts are ready for the next kernel on the stream.
template <class T>
__device__ __forceinline__ void push_ghosts(const DevBlock* __restrict__ blocks, const DevBlock& B, int bidx,
                                            const int id[3], T* arr, long long fs, int nf, const T* vals, bool mirror) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, side = f & 1;
        const int s = side ? B.n[d] - 1 - id[d] : id[d];
        int t[3] = {id[0], id[1], id[2]};
        if (B.nbr[f] >= 0) {
            if (s < G) {
                const DevBlock& N = blocks[B.nbr[f]];
                ghost_across(blocks[bidx].tf[f], N, f, s, id, t);
                const long long e = node_index(N, t[0], t[1], t[2]);
                for (int c = 0; c < nf; ++c) arr[c * fs + e] = vals[c];
            }
        } else if (mirror && ((B.wall >> f) & 1) && s >= 1 && s <= G) {
            t[d] = side ? B.n[d] - 1 + s : -s;
            const long long e = node_index(B, t[0], t[1], t[2]);
            for (int c = 0; c < nf; ++c) arr[c * fs + e] = (c >= 1 && c <= 3) ? -vals[c] : vals[c];
        }
    }
}


// ---------------------------------------------------------------------------
// small math wrappers
// ---------------------------------------------------------------------------
// FP64: IEEE division and square root, CUDA's double rsqrt.  FP32 (mixed
// form, 1e-5 error budget): the approximate hardware reciprocal and
// reciprocal square root.
__device__ __forceinline__ double hsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float hsqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double hrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float hrcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double hrsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float hrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double habs(double x) { return fabs(x); }
__device__ __forceinline__ float habs(float x) { return fabsf(x); }
__device__ __forceinline__ double hmax0(double x) { return fmax(x, 0.0); }
__device__ __forceinline__ float hmax0(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ double hmin0(double x) { return fmin(x, 0.0); }
__device__ __forceinline__ float hmin0(float x) { return fminf(x, 0.0f); }

template <class R>
struct GasR {   // gas constants in the working precision (built on the host)
    R gamma, gm1, inv_2gamma, two_gm1, mach_re, kq_fac, suth, one_p_suth, inv_gm1, g_gm1;
    R gm1_over_g, inv_g_sqrt2;   // (gamma-1)/gamma and 1/(gamma sqrt 2): a node's own characteristic values
    int mu_law;
    __host__ __device__ void init(const Gas& g) {
        gamma = R(g.gamma);
        gm1_over_g = R((g.gamma - 1.0) / g.gamma);
        inv_g_sqrt2 = R(0.70710678118654752440 / g.gamma);
        gm1 = R(g.gamma - 1.0);
        inv_2gamma = R(1.0 / (2.0 * g.gamma));
        two_gm1 = R(2.0 * (g.gamma - 1.0));
        mach_re = R(g.mach / g.re);
        kq_fac = R(1.0 / (g.pr * (g.gamma - 1.0)));
        suth = R(g.suth);
        one_p_suth = R(1.0 + g.suth);
        inv_gm1 = R(1.0 / (g.gamma - 1.0));
        g_gm1 = R(g.gamma * (g.gamma - 1.0));
        mu_law = g.mu_law;
    }
};

// Sixth-order central first derivative (Sec. 2), unit spacing, from the six
// neighbours fm3..fp3.
template <class R>
__device__ __forceinline__ R d6(R fm3, R fm2, R fm1, R fp1, R fp2, R fp3) {
    return R(0.75) * (fp1 - fm1) + R(-0.15) * (fp2 - fm2) + R(1.0 / 60.0) * (fp3 - fm3);
}

// Face value at i+1/2 from nodes i-2..i+3 (sixth-order midpoint formula).
template <class R>
__device__ __forceinline__ R mid6(R fm2, R fm1, R f0, R fp1, R fp2, R fp3) {
    return (R(3.0) * (fm2 + fp3) - R(25.0) * (fm1 + fp2) + R(150.0) * (f0 + fp1)) * R(1.0 / 256.0);
}

// Primitives (u, v, w, T) of a conservative state (T = gamma p / rho); the
// one formula every kernel of the mixed form uses, so that results do not
// depend on which kernel formed them.  The FP64 form forms them only in
// k_prep, from the node state (node_state below).
template <class R>
__device__ __forceinline__ void primitives(const GasR<R>& gs, const R q[5], R pv[4]) {
    const R irho = hrcp(q[0]);
    pv[0] = q[1] * irho;
    pv[1] = q[2] * irho;
    pv[2] = q[3] * irho;
    const R p = gs.gm1 * (q[4] - R(0.5) * (q[1] * pv[0] + q[2] * pv[1] + q[3] * pv[2]));
    pv[3] = gs.gamma * p * irho;
}

// Viscosity: mu = 1, or Sutherland T^(3/2) (1+S)/(T+S).
template <class R>
__device__ __forceinline__ R viscosity(const GasR<R>& g, R T) {
    if (g.mu_law == 0) return R(1);
    return T * hsqrt(T) * g.one_p_suth / (T + g.suth);
}

// ---------------------------------------------------------------------------
// WENO5 interpolation of the modified AFWENO (Eqs. (13)-(17), Figs. 10-11):
// from the 5-node stencil W[-2..2] of node i, the left-biased value at i+1/2
// and the right-biased value at i-1/2, sharing the smoothness indicators.
// Each sub-stencil is paired with its own indicator; linear weights 1/16,
// 5/8, 5/16 for the stencils {i-2..i}, {i-1..i+1}, {i..i+2} (left value),
// mirrored for the right value.
// ---------------------------------------------------------------------------
//
// FP64 runs at 1/64 of the FP32 rate here, so the FP64 form is written for
// the fewest FP64 instructions; in exact arithmetic it gives the same values:
//   - a_k are the second differences and c_k the remaining Eq. (17) terms,
//     both from the first differences;
//   - s_k = 4 (eps + beta_k) = 4 eps + (13/3) a_k^2 + c_k^2 (a common factor
//     of the s_k cancels in the normalised weights), and gamma/s^2 scaled by
//     16 s1^2 s2^2 s3^2 gives the unnormalised weights (p23, 10 p13, 5 p12)
//     of the left value and (p12, 10 p13, 5 p23) of the right one,
//     p_jk = s_j^2 s_k^2;
//   - since the weights sum to one, each value is the central candidate plus
//     weighted differences of the outer candidates, which are third
//     differences: uL1 - uL2 = 3 e1 / 8, uL3 - uL2 = e2 / 8 with
//     e1 = a1 - a2 = w0 - 3w1 + 3w2 - w3, e2 = a2 - a3 (mirrored for the right
//     value), so left = uL2 + (3 p23 e1 + 5 p12 e2) / (8 dL) and
//     right = uR2 - (3 p12 e2 + 5 p23 e1) / (8 dR).
struct WenoParts {   // one field: value = u2 + n / (8 d) for each side
    double nL, nR, dL, dR, uL2, uR2;
};

// From the first differences d10 .. d43 of the stencil values and the
// central value w2 (the only places the values enter).
__device__ __forceinline__ WenoParts weno_parts_d(double d10, double d21, double d32, double d43, double w2) {
    const double eps4 = 4.0e-6;
    const double a1 = d21 - d10, a2 = d32 - d21, a3 = d43 - d32;
    const double c1 = fma(2.0, d21, a1), c2 = d21 + d32, c3 = fma(-2.0, d32, a3);
    const double k = 13.0 / 3.0;
    double s1 = fma(a1, k * a1, fma(c1, c1, eps4));
    double s2 = fma(a2, k * a2, fma(c2, c2, eps4));
    double s3 = fma(a3, k * a3, fma(c3, c3, eps4));
    s1 *= s1;
    s2 *= s2;
    s3 *= s3;
    const double p12 = s1 * s2, p13 = s1 * s3, p23 = s2 * s3;
    WenoParts r;
    r.dL = fma(10.0, p13, fma(5.0, p12, p23));
    r.dR = fma(10.0, p13, fma(5.0, p23, p12));
    const double e1 = a1 - a2, e2 = a2 - a3;
    const double A = p23 * e1, B = p12 * e2;
    r.nL = fma(3.0, A, 5.0 * B);
    r.nR = -fma(3.0, B, 5.0 * A);
    r.uL2 = fma(0.125, fma(3.0, d32, d21), w2);    // (-w1 + 6 w2 + 3 w3) / 8
    r.uR2 = fma(-0.125, fma(3.0, d21, d32), w2);   // (-w3 + 6 w2 + 3 w1) / 8
    return r;
}

__device__ __forceinline__ WenoParts weno_parts(double w0, double w1, double w2, double w3, double w4) {
    return weno_parts_d(w1 - w0, w2 - w1, w3 - w2, w4 - w3, w2);
}

__device__ __forceinline__ void weno_pair(double w0, double w1, double w2, double w3, double w4,
                                          double& left, double& right) {
    const WenoParts r = weno_parts(w0, w1, w2, w3, w4);
    const double inv = 0.125 / (r.dL * r.dR);   // one division for both values
    left = fma(r.nL, r.dR * inv, r.uL2);
    right = fma(r.nR, r.dL * inv, r.uR2);
}

// num / D[l] for N positive FP64 values with one division: each D[l] is
// brought to [1, 2) by its binary exponent (integer pipe; the WENO
// denominators lie far inside the exponent range), the reciprocals come from
// one division of their product and the prefix products, and each is scaled
// back by its exponent.
template <int N>
__device__ __forceinline__ void batch_recip(const double (&D)[N], double num, double (&inv)[N]) {
    double m[N], P[N];
    int ex[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
        const long long b = __double_as_longlong(D[l]);
        ex[l] = (int)(b >> 52) & 0x7ff;
        m[l] = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
        P[l] = l == 0 ? m[0] : P[l - 1] * m[l];
    }
    double I = num / P[N - 1];
#pragma unroll
    for (int l = N - 1; l > 0; --l) {
        inv[l] = I * P[l - 1];
        I *= m[l];
    }
    inv[0] = I;
#pragma unroll
    for (int l = 0; l < N; ++l)
        inv[l] = __longlong_as_double(__double_as_longlong(inv[l]) - ((long long)(ex[l] - 1023) << 52));
}

// The five characteristic fields of a node with one FP64 division, from
// the differences dW[s][l] of the stencil's characteristic values across
// its faces s = 0..3 (i-3/2 .. i+3/2) and the node's own values Wc[l].
// The projection is linear, so dW is the projection of the differences of
// the conservative state: formed once per face, shared by the four
// stencils that contain the face.
__device__ __forceinline__ void weno_pair5_d(const double (&dW)[4][5], const double (&Wc)[5], double (&WL)[5],
                                             double (&WR)[5]) {
    WenoParts r[5];
    double D[5], inv[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        r[l] = weno_parts_d(dW[0][l], dW[1][l], dW[2][l], dW[3][l], Wc[l]);
        D[l] = r[l].dL * r[l].dR;
    }
    batch_recip<5>(D, 0.125, inv);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        WL[l] = fma(r[l].nL, r[l].dR * inv[l], r[l].uL2);
        WR[l] = fma(r[l].nR, r[l].dL * inv[l], r[l].uR2);
    }
}

// FP32: the same algebra as the FP64 form with one hardware reciprocal per
// side (dL, dR >= 4e-21 from eps, and below FP32's range limit for
// indicators up to about 4e9, far beyond any physical state in these units).
__device__ __forceinline__ void weno_pair(float w0, float w1, float w2, float w3, float w4, float& left,
                                          float& right) {
    const float eps4 = 4.0e-6f;
    const float d10 = w1 - w0, d21 = w2 - w1, d32 = w3 - w2, d43 = w4 - w3;
    const float a1 = d21 - d10, a2 = d32 - d21, a3 = d43 - d32;
    const float c1 = fmaf(2.0f, d21, a1), c2 = d21 + d32, c3 = fmaf(-2.0f, d32, a3);
    const float k = 13.0f / 3.0f;
    float s1 = fmaf(a1, k * a1, fmaf(c1, c1, eps4));
    float s2 = fmaf(a2, k * a2, fmaf(c2, c2, eps4));
    float s3 = fmaf(a3, k * a3, fmaf(c3, c3, eps4));
    s1 *= s1;
    s2 *= s2;
    s3 *= s3;
    const float p12 = s1 * s2, p13 = s1 * s3, p23 = s2 * s3;
    const float t13 = 10.0f * p13;
    const float dL = fmaf(5.0f, p12, p23) + t13, dR = fmaf(5.0f, p23, p12) + t13;
    const float e1 = a1 - a2, e2 = a2 - a3;
    const float A = p23 * e1, B = p12 * e2;
    const float uL2 = fmaf(0.125f, fmaf(3.0f, d32, d21), w2);
    const float uR2 = fmaf(-0.125f, fmaf(3.0f, d21, d32), w2);
    // the 1/8 of the correction folded into the weights' constants
    const float nL = fmaf(0.375f, A, 0.625f * B), nR = fmaf(0.375f, B, 0.625f * A);
    left = fmaf(nL, __fdividef(1.0f, dL), uL2);
    right = fmaf(-nR, __fdividef(1.0f, dR), uR2);
}

// FP32: each field on its own (hardware reciprocals are cheap).
__device__ __forceinline__ void weno_pair5(const float (&W)[5][5], float (&WL)[5], float (&WR)[5]) {
#pragma unroll
    for (int l = 0; l < 5; ++l) weno_pair(W[0][l], W[1][l], W[2][l], W[3][l], W[4][l], WL[l], WR[l]);
}

// One WENO5 value with its own indicators (original AFWENO, Fig. 9): the
// left-biased value at i+1/2 (LEFT) or the right-biased value at i-1/2 of
// the stencil W[-2..2] of node i, in the form of the pair above:
// value = u2 + n / (8 d).
template <class R>
struct WenoSide {
    R n, d, u2;
};

template <class R, bool LEFT>
__device__ __forceinline__ WenoSide<R> weno_side(R w0, R w1, R w2, R w3, R w4) {
    const R eps4 = R(4.0e-6);
    const R d10 = w1 - w0, d21 = w2 - w1, d32 = w3 - w2, d43 = w4 - w3;
    const R a1 = d21 - d10, a2 = d32 - d21, a3 = d43 - d32;
    const R c1 = R(2) * d21 + a1, c2 = d21 + d32, c3 = R(-2) * d32 + a3;
    const R k = R(13.0 / 3.0);
    R s1 = a1 * (k * a1) + (c1 * c1 + eps4);
    R s2 = a2 * (k * a2) + (c2 * c2 + eps4);
    R s3 = a3 * (k * a3) + (c3 * c3 + eps4);
    s1 *= s1;
    s2 *= s2;
    s3 *= s3;
    const R p12 = s1 * s2, p13 = s1 * s3, p23 = s2 * s3;
    const R e1 = a1 - a2, e2 = a2 - a3;
    WenoSide<R> r;
    if (LEFT) {
        r.d = R(10) * p13 + (R(5) * p12 + p23);
        r.n = R(3) * (p23 * e1) + R(5) * (p12 * e2);
        r.u2 = R(0.125) * (R(3) * d32 + d21) + w2;
    } else {
        r.d = R(10) * p13 + (R(5) * p23 + p12);
        r.n = -(R(3) * (p12 * e2) + R(5) * (p23 * e1));
        r.u2 = R(-0.125) * (R(3) * d21 + d32) + w2;
    }
    return r;
}

// The ten values of a face (five fields, each side with its own stencil:
// left from nodes i-2..i+2, right from i-1..i+3): one FP64 division, or two
// hardware reciprocals per field in FP32.  W[s][l]: nodes s = 0..5.
__device__ __forceinline__ void weno_face10(const double (&W)[6][5], double (&WL)[5], double (&WR)[5]) {
    WenoSide<double> L[5], Rt[5];
    double D[10], inv[10];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        L[l] = weno_side<double, true>(W[0][l], W[1][l], W[2][l], W[3][l], W[4][l]);
        Rt[l] = weno_side<double, false>(W[1][l], W[2][l], W[3][l], W[4][l], W[5][l]);
        D[l] = L[l].d;
        D[5 + l] = Rt[l].d;
    }
    batch_recip<10>(D, 0.125, inv);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        WL[l] = fma(L[l].n, inv[l], L[l].u2);
        WR[l] = fma(Rt[l].n, inv[5 + l], Rt[l].u2);
    }
}

__device__ __forceinline__ void weno_face10(const float (&W)[6][5], float (&WL)[5], float (&WR)[5]) {
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const WenoSide<float> L = weno_side<float, true>(W[0][l], W[1][l], W[2][l], W[3][l], W[4][l]);
        const WenoSide<float> Rt = weno_side<float, false>(W[1][l], W[2][l], W[3][l], W[4][l], W[5][l]);
        WL[l] = fmaf(L.n, __fdividef(0.125f, L.d), L.u2);
        WR[l] = fmaf(Rt.n, __fdividef(0.125f, Rt.d), Rt.u2);
    }
}

// ---------------------------------------------------------------------------
// Characteristic basis at a node: Pulliam-Chaussee eigenvectors of the
// Jacobian of k.F for the unit normal k of the node metric.  The projection
// W = L Q and back projection U = R W are written in vector form:
//   d = (Q_1 - u Q_0, Q_2 - v Q_0, Q_3 - w Q_0) / rho,
//   S = (1 - phi2/c^2) Q_0 + (gamma-1)/c^2 (u Q_1 + v Q_2 + w Q_3 - Q_4),
//   (W_0, W_1, W_2) = k S + d x k,
//   W_3,4 = (c/rho (Q_0 - S) +- k.d) / sqrt(2),
// and with C = k x (W_0, W_1, W_2), s = W_3 + W_4, t = W_3 - W_4, Wk = k.(W_0, W_1, W_2):
//   U_0 = Wk + al s,  U_m = u_m Wk + rho C_m + al (s u_m + k_m c t)  (m = 1..3),
//   U_4 = |u|^2/2 Wk + rho u.C + al (s H + c theta t),  al = rho/(sqrt(2) c),
// which is the matrix pair L = T_k^-1, R = T_k entry by entry.
// ---------------------------------------------------------------------------
// The direction-independent part of a node's basis: 1/rho, the velocity,
// |u|^2/2, p, c, a0 = 1 - phi2/c^2, g = (gamma-1)/c^2, c/(sqrt(2) rho),
// rho/(sqrt(2) c) and H.  The FP64 form forms it once per node and stage
// (k_prep, NodeState::NF fields of a node-state array) and its three sweeps
// read it, instead of each sweep dividing and taking the square root again.
template <class R>
struct NodeState {
    static constexpr int NF = 12;
    R irho, u, v, w, half_uu, p, c, a0, g, cir, al, H;
};

// Returns c^2 = gamma p / rho, the temperature of the primitives.
template <class R>
__device__ __forceinline__ R node_state(const GasR<R>& gs, const R q[5], NodeState<R>& s) {
    const R rho = q[0];
    s.irho = hrcp(rho);
    s.u = q[1] * s.irho;
    s.v = q[2] * s.irho;
    s.w = q[3] * s.irho;
    s.half_uu = R(0.5) * (s.u * s.u + s.v * s.v + s.w * s.w);
    s.p = gs.gm1 * (q[4] - rho * s.half_uu);
    const R c2 = gs.gamma * s.p * s.irho;
    const R ic = hrsqrt(c2);
    s.c = c2 * ic;
    const R phi2 = gs.gm1 * s.half_uu;
    const R ic2 = ic * ic;
    s.a0 = R(1) - phi2 * ic2;
    s.g = gs.gm1 * ic2;
    s.cir = s.c * s.irho * R(0.70710678118654752440);
    s.al = rho * ic * R(0.70710678118654752440);
    s.H = s.half_uu + c2 * gs.inv_gm1;
    return c2;
}

// FP64: per-node products are hoisted out of the five stencil projections
// (the FP64 pipe is the bound; registers are not).
template <class R>
struct CharBasis {
    R kx, ky, kz, u, v, w, rho, irho, p, c, a0, g, gu, gv, gw, cir, kxi, kyi, kzi, kxs, kys, kzs, al, alc, acth,
        half_uu, H, rkx, rky, rkz;
    __device__ __forceinline__ void set_state(R rho_, const NodeState<R>& s) {
        rho = rho_;
        irho = s.irho;
        u = s.u;
        v = s.v;
        w = s.w;
        half_uu = s.half_uu;
        p = s.p;
        c = s.c;
        a0 = s.a0;
        g = s.g;
        cir = s.cir;
        al = s.al;
        H = s.H;
        gu = g * u;
        gv = g * v;
        gw = g * w;
        alc = al * c;
    }
    // the state part (the node flux needs only this) ...
    __device__ __forceinline__ void init_state(const GasR<R>& gs, const R q[5]) {
        NodeState<R> s;
        node_state(gs, q, s);
        set_state(q[0], s);
    }
    // ... or read from a node-state array (field stride fs) at the node
    __device__ __forceinline__ void load_state(const R* __restrict__ ns, long long fs, R rho_) {
        NodeState<R> s;
        s.irho = ns[0];
        s.u = ns[fs];
        s.v = ns[2 * fs];
        s.w = ns[3 * fs];
        s.half_uu = ns[4 * fs];
        s.p = ns[5 * fs];
        s.c = ns[6 * fs];
        s.a0 = ns[7 * fs];
        s.g = ns[8 * fs];
        s.cir = ns[9 * fs];
        s.al = ns[10 * fs];
        s.H = ns[11 * fs];
        set_state(rho_, s);
    }
    // ... and the unit normal k.  The projection works on rho d = (Q_m - u_m
    // Q_0); 1/rho and 1/sqrt(2) go into the normal once per node.
    __device__ __forceinline__ void set_normal(R kx_, R ky_, R kz_) {
        kx = kx_;
        ky = ky_;
        kz = kz_;
        kxi = kx * irho;
        kyi = ky * irho;
        kzi = kz * irho;
        kxs = kxi * R(0.70710678118654752440);
        kys = kyi * R(0.70710678118654752440);
        kzs = kzi * R(0.70710678118654752440);
        acth = alc * (kx * u + ky * v + kz * w);
        rkx = rho * kx;
        rky = rho * ky;
        rkz = rho * kz;
    }
    __device__ __forceinline__ void init(const GasR<R>& gs, const R q[5], R mx, R my, R mz) {
        init_state(gs, q);
        const R imm = hrsqrt(mx * mx + my * my + mz * mz);
        set_normal(mx * imm, my * imm, mz * imm);
    }
    // W = L q of the node's own state q: there d = 0 and
    // S = rho - p/c^2 = rho (gamma-1)/gamma, so W_0..2 = k rho (gamma-1)/gamma
    // and W_3 = W_4 = c/(gamma sqrt 2) (equal to project() up to rounding).
    __device__ __forceinline__ void center(const GasR<R>& gs, R W[5]) const {
        const R S = rho * gs.gm1_over_g;
        W[0] = kx * S;
        W[1] = ky * S;
        W[2] = kz * S;
        W[3] = W[4] = c * gs.inv_g_sqrt2;
    }
    // W = L q
    __device__ __forceinline__ void project(R q0, R q1, R q2, R q3, R q4, R W[5]) const {
        const R d1 = q1 - u * q0, d2 = q2 - v * q0, d3 = q3 - w * q0;
        const R S = a0 * q0 + gu * q1 + gv * q2 + gw * q3 - g * q4;
        W[0] = kx * S + (d2 * kzi - d3 * kyi);
        W[1] = ky * S + (d3 * kxi - d1 * kzi);
        W[2] = kz * S + (d1 * kyi - d2 * kxi);
        const R kd = kxs * d1 + kys * d2 + kzs * d3;
        const R base = cir * (q0 - S);
        W[3] = base + kd;
        W[4] = base - kd;
    }
    // U = R W, with rho C = (rho k) x (W_0, W_1, W_2) from the node's rho k
    __device__ __forceinline__ void back(const R W[5], R U[5]) const {
        const R Wk = kx * W[0] + ky * W[1] + kz * W[2];
        const R rCx = rky * W[2] - rkz * W[1], rCy = rkz * W[0] - rkx * W[2], rCz = rkx * W[1] - rky * W[0];
        const R s = W[3] + W[4], t = W[3] - W[4];
        const R as = al * s, act = alc * t;
        U[0] = Wk + as;
        U[1] = u * U[0] + (rCx + act * kx);
        U[2] = v * U[0] + (rCy + act * ky);
        U[3] = w * U[0] + (rCz + act * kz);
        U[4] = half_uu * Wk + (u * rCx + v * rCy + w * rCz) + as * H + acth * t;
    }
};

// FP32 (mixed form): the same basis with fewer per-node members, which keeps
// the sweep kernels within their register budget; FP32 arithmetic is cheap.
template <>
struct CharBasis<float> {
    using R = float;
    R kx, ky, kz, u, v, w, rho, irho, p, c, a0, g, cir, al, half_uu, H, cth;
    __device__ __forceinline__ void init_state(const GasR<R>& gs, const R q[5]) {
        irho = hrcp(q[0]);
        rho = q[0];
        u = q[1] * irho;
        v = q[2] * irho;
        w = q[3] * irho;
        half_uu = R(0.5) * (u * u + v * v + w * w);
        p = gs.gm1 * (q[4] - rho * half_uu);
        const R c2 = gs.gamma * p * irho;
        const R ic = hrsqrt(c2);
        c = c2 * ic;
        const R phi2 = gs.gm1 * half_uu;
        const R ic2 = ic * ic;
        a0 = R(1) - phi2 * ic2;
        g = gs.gm1 * ic2;
        cir = c * irho * R(0.70710678118654752440);
        al = rho * ic * R(0.70710678118654752440);
        H = half_uu + c2 * gs.inv_gm1;
    }
    __device__ __forceinline__ void set_normal(R kx_, R ky_, R kz_) {
        kx = kx_;
        ky = ky_;
        kz = kz_;
        cth = c * (kx * u + ky * v + kz * w);
    }
    __device__ __forceinline__ void init(const GasR<R>& gs, const R q[5], R mx, R my, R mz) {
        init_state(gs, q);
        const R imm = hrsqrt(mx * mx + my * my + mz * mz);
        set_normal(mx * imm, my * imm, mz * imm);
    }
    // W = L q of the node's own state (as CharBasis<double>::center)
    __device__ __forceinline__ void center(const GasR<R>& gs, R W[5]) const {
        const R S = rho * gs.gm1_over_g;
        W[0] = kx * S;
        W[1] = ky * S;
        W[2] = kz * S;
        W[3] = W[4] = c * gs.inv_g_sqrt2;
    }
    // W = L q
    __device__ __forceinline__ void project(R q0, R q1, R q2, R q3, R q4, R W[5]) const {
        const R d1 = (q1 - u * q0) * irho, d2 = (q2 - v * q0) * irho, d3 = (q3 - w * q0) * irho;
        const R S = a0 * q0 + g * (u * q1 + v * q2 + w * q3 - q4);
        W[0] = kx * S + (d2 * kz - d3 * ky);
        W[1] = ky * S + (d3 * kx - d1 * kz);
        W[2] = kz * S + (d1 * ky - d2 * kx);
        const R kd = (kx * d1 + ky * d2 + kz * d3) * R(0.70710678118654752440);
        const R base = cir * (q0 - S);
        W[3] = base + kd;
        W[4] = base - kd;
    }
    // U = R W
    __device__ __forceinline__ void back(const R W[5], R U[5]) const {
        const R Wk = kx * W[0] + ky * W[1] + kz * W[2];
        const R Cx = ky * W[2] - kz * W[1], Cy = kz * W[0] - kx * W[2], Cz = kx * W[1] - ky * W[0];
        const R s = W[3] + W[4], t = W[3] - W[4];
        const R as = al * s, act = al * c * t;
        U[0] = Wk + as;
        U[1] = u * U[0] + (rho * Cx + act * kx);
        U[2] = v * U[0] + (rho * Cy + act * ky);
        U[3] = w * U[0] + (rho * Cz + act * kz);
        U[4] = half_uu * Wk + rho * (u * Cx + v * Cy + w * Cz) + as * H + al * cth * t;
    }
};

// Node flux along the conservative metric m, Eq. (4).
template <class R>
__device__ __forceinline__ void point_flux(const GasR<R>& gs, const R q[5], R mx, R my, R mz, R f[5]) {
    const R irho = hrcp(q[0]);
    const R u = q[1] * irho, v = q[2] * irho, w = q[3] * irho;
    const R p = gs.gm1 * (q[4] - R(0.5) * (q[1] * u + q[2] * v + q[3] * w));
    const R th = mx * u + my * v + mz * w;
    f[0] = q[0] * th;
    f[1] = q[1] * th + mx * p;
    f[2] = q[2] * th + my * p;
    f[3] = q[3] * th + mz * p;
    f[4] = (q[4] + p) * th;
}

// Positive or negative part of x on the integer pipe (sign-bit mask), so
// that the split of the eigenvalues costs no floating-point instruction.
__device__ __forceinline__ double hpos(double x) {
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(b & ~(b >> 63));
}
__device__ __forceinline__ double hneg(double x) {
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(b & (b >> 63));
}
__device__ __forceinline__ float hpos(float x) {
    const int b = __float_as_int(x);
    return __int_as_float(b & ~(b >> 31));
}
__device__ __forceinline__ float hneg(float x) {
    const int b = __float_as_int(x);
    return __int_as_float(b & (b >> 31));
}

// Steger-Warming split flux along metric (kx, ky, kz) * |m|, with mmg =
// |m| / (2 gamma); POS selects F+.
//   F = rho |m| / (2 gamma) [M, u M + c kx D, v M + c ky D, w M + c kz D,
//                            (gamma-1) l1 |u|^2 + (l4+l5) H + c theta D]
//   with l = lambda^+- of (theta, theta + c, theta - c) (the factor |m| > 0
//   commutes with the split), M = 2(gamma-1) l1 + l4 + l5, D = l4 - l5 and
//   H = |u|^2/2 + c^2/(gamma-1): the energy row's (|u|^2+c^2)/2 and
//   (3-gamma) c^2 / (2 (gamma-1)) terms of (l4+l5) sum to H.
template <class R, bool POS>
__device__ __forceinline__ void sw_flux(const GasR<R>& gs, const R q[5], R irho, R kx, R ky, R kz, R mmg, R F[5]) {
    const R u = q[1] * irho, v = q[2] * irho, w = q[3] * irho;
    const R uu = u * u + v * v + w * w;
    // t = E/rho - |u|^2/2 = p / ((gamma-1) rho): c^2 = gamma (gamma-1) t and
    // H = E/rho + (gamma-1) t, without forming p
    const R e = q[4] * irho;
    const R t = e - R(0.5) * uu;
    const R c2 = gs.g_gm1 * t;
    const R c = c2 * hrsqrt(c2);
    const R th = kx * u + ky * v + kz * w;
    R l1 = th, l4 = th + c, l5 = th - c;
    if (POS) {
        l1 = hpos(l1);
        l4 = hpos(l4);
        l5 = hpos(l5);
    } else {
        l1 = hneg(l1);
        l4 = hneg(l4);
        l5 = hneg(l5);
    }
    const R a = q[0] * mmg;
    const R S45 = l4 + l5, D45 = l4 - l5;
    const R aM = a * (gs.two_gm1 * l1 + S45);
    const R acD = a * (c * D45);
    const R H = e + gs.gm1 * t;
    F[0] = aM;
    F[1] = u * aM + kx * acD;
    F[2] = v * aM + ky * acD;
    F[3] = w * aM + kz * acD;
    F[4] = a * (gs.gm1 * l1 * uu + S45 * H) + th * acD;
}

// h = F+(ql) + F-(qr) of a face along (kx, ky, kz) * mm.  In FP64 the two
// densities share one division: 1/rho_l = rho_r / (rho_l rho_r) and
// 1/rho_r = rho_l / (rho_l rho_r).
template <class R>
__device__ __forceinline__ void face_flux(const GasR<R>& gs, const R ql[5], const R qr[5], R kx, R ky, R kz, R mm,
                                          R h[5]) {
    R il, ir;
    if (sizeof(R) == 8) {
        const R inv = hrcp(ql[0] * qr[0]);
        il = qr[0] * inv;
        ir = ql[0] * inv;
    } else {
        il = hrcp(ql[0]);
        ir = hrcp(qr[0]);
    }
    const R mmg = mm * gs.inv_2gamma;   // |m| / (2 gamma), shared by the two sides
    R Fp[5], Fm[5];
    sw_flux<R, true>(gs, ql, il, kx, ky, kz, mmg, Fp);
    sw_flux<R, false>(gs, qr, ir, kx, ky, kz, mmg, Fm);
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = Fp[k] + Fm[k];
}

// Stress tensor and work + heat-flux vector at a node, Eqs. (5)-(6) and the
// definitions under Eq. (1): S = (tau_xx, tau_yy, tau_zz, tau_xy, tau_xz,
// tau_yz, beta_x, beta_y, beta_z) from g = (u,v,w,T)_(x,y,z) / sc, row-major
// (S is linear in the gradients, so a common factor sc of all twelve, the
// Jacobian of the chain rule, enters through the viscosity once).  The
// viscous flux of a direction with metric m is then (m.tau_x., m.tau_y.,
// m.tau_z., m.beta): the direction-independent part is formed once per node.
template <class R>
__device__ __forceinline__ void stress(const GasR<R>& gs, R u, R v, R w, R T, const R g[12], R sc, R S[9]) {
    const R kv = gs.mach_re * viscosity(gs, T) * sc;
    const R kq = kv * gs.kq_fac;
    const R div = g[0] + g[4] + g[8];
    const R lam = R(-2.0 / 3.0) * kv * div;
    const R txx = lam + R(2) * kv * g[0], tyy = lam + R(2) * kv * g[4], tzz = lam + R(2) * kv * g[8];
    const R txy = kv * (g[1] + g[3]), txz = kv * (g[2] + g[6]), tyz = kv * (g[5] + g[7]);
    S[0] = txx;
    S[1] = tyy;
    S[2] = tzz;
    S[3] = txy;
    S[4] = txz;
    S[5] = tyz;
    S[6] = u * txx + v * txy + w * txz + kq * g[9];
    S[7] = u * txy + v * tyy + w * tyz + kq * g[10];
    S[8] = u * txz + v * tyz + w * tzz + kq * g[11];
}

// Derivative at node p of a line of n nodes from values f(-4..4) around it,
// with the one-sided closure next to physical ends (boundary node
// (-3,4,-1)/2, then 2nd-order central, then 4th-order central).
template <class R, class F>
__device__ __forceinline__ R dline(const F& f, int p, int n, bool lo, bool hi) {
    if (lo && p <= 2) {
        if (p == 0) return (R(-3) * f(0) + R(4) * f(1) - f(2)) * R(0.5);
        if (p == 1) return (f(1) - f(-1)) * R(0.5);
        return (f(-2) - R(8) * f(-1) + R(8) * f(1) - f(2)) * R(1.0 / 12.0);
    }
    if (hi && p >= n - 3) {
        if (p == n - 1) return (R(3) * f(0) - R(4) * f(-1) + f(-2)) * R(0.5);
        if (p == n - 2) return (f(1) - f(-1)) * R(0.5);
        return (f(-2) - R(8) * f(-1) + R(8) * f(1) - f(2)) * R(1.0 / 12.0);
    }
    return d6<R>(f(-3), f(-2), f(-1), f(1), f(2), f(3));
}

}  // namespace hx
