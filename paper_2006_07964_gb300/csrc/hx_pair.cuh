// hx_pair.cuh -- two FP32 values in one register pair, with the packed FP32
// arithmetic of sm_100-class GPUs (add / sub / mul / fma .f32x2: one
// instruction for both lanes, each rounded as its scalar counterpart).
//
// The mixed form's stencil kernels are bound by instruction issue, not by
// the FP32 pipe; computing two grid lines per thread with packed
// instructions halves the FP32 instruction count and, with 64-bit shared
// memory accesses, the loads and stores and the index arithmetic per node.
#pragma once
#include <cuda_runtime.h>

#include "hx_common.cuh"

namespace hx {

struct P2 {
    float2 v;
};

__device__ __forceinline__ P2 pk(float a) { return P2{make_float2(a, a)}; }
__device__ __forceinline__ P2 pk(float a, float b) { return P2{make_float2(a, b)}; }

__device__ __forceinline__ unsigned long long pbits(P2 a) {
    return (unsigned long long)__float_as_uint(a.v.x) | ((unsigned long long)__float_as_uint(a.v.y) << 32);
}
__device__ __forceinline__ P2 pfrom(unsigned long long b) {
    return P2{make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)))};
}

__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pbits(a)), "l"(pbits(b)));
    return pfrom(d);
}
__device__ __forceinline__ P2 operator-(P2 a) { return P2{make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ P2 pfma(P2 a, P2 b, P2 c) { return P2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ P2 operator*(float s, P2 a) { return pk(s) * a; }

// per lane (no packed form): the hardware reciprocal and reciprocal square
// root of the scalar FP32 path, and the integer-pipe sign splits
__device__ __forceinline__ P2 prcp(P2 a) { return pk(__fdividef(1.0f, a.v.x), __fdividef(1.0f, a.v.y)); }
__device__ __forceinline__ P2 prsqrt(P2 a) { return pk(rsqrtf(a.v.x), rsqrtf(a.v.y)); }
__device__ __forceinline__ P2 ppos(P2 a) { return pk(hpos(a.v.x), hpos(a.v.y)); }
__device__ __forceinline__ P2 pneg(P2 a) { return pk(hneg(a.v.x), hneg(a.v.y)); }

// 64-bit shared / global accesses of a pair stored in two consecutive floats
__device__ __forceinline__ P2 ld2(const float* p) { return P2{*reinterpret_cast<const float2*>(p)}; }
__device__ __forceinline__ void st2(float* p, P2 a) { *reinterpret_cast<float2*>(p) = a.v; }

// Sixth-order central first derivative and midpoint value (Sec. 2), as the
// scalar d6 / mid6 of hx_common.cuh.
__device__ __forceinline__ P2 d6p(P2 fm3, P2 fm2, P2 fm1, P2 fp1, P2 fp2, P2 fp3) {
    return pfma(pk(0.75f), fp1 - fm1, pfma(pk(-0.15f), fp2 - fm2, pk(1.0f / 60.0f) * (fp3 - fm3)));
}
__device__ __forceinline__ P2 mid6p(P2 fm2, P2 fm1, P2 f0, P2 fp1, P2 fp2, P2 fp3) {
    return pfma(pk(3.0f / 256.0f), fm2 + fp3, pfma(pk(-25.0f / 256.0f), fm1 + fp2, pk(150.0f / 256.0f) * (f0 + fp1)));
}

// WENO5 pair of the modified AFWENO for one characteristic field of two
// lines: the FP32 weno_pair of hx_common.cuh (same algebra: product-form
// weights, the central candidate plus weighted third differences), packed.
__device__ __forceinline__ void weno_pair_p(P2 w0, P2 w1, P2 w2, P2 w3, P2 w4, P2& left, P2& right) {
    const P2 d10 = w1 - w0, d21 = w2 - w1, d32 = w3 - w2, d43 = w4 - w3;
    const P2 a1 = d21 - d10, a2 = d32 - d21, a3 = d43 - d32;
    const P2 c1 = pfma(pk(2.0f), d21, a1), c2 = d21 + d32, c3 = pfma(pk(-2.0f), d32, a3);
    const P2 k = pk(13.0f / 3.0f), eps4 = pk(4.0e-6f);
    P2 s1 = pfma(a1, k * a1, pfma(c1, c1, eps4));
    P2 s2 = pfma(a2, k * a2, pfma(c2, c2, eps4));
    P2 s3 = pfma(a3, k * a3, pfma(c3, c3, eps4));
    s1 = s1 * s1;
    s2 = s2 * s2;
    s3 = s3 * s3;
    const P2 p12 = s1 * s2, p13 = s1 * s3, p23 = s2 * s3;
    const P2 t13 = pk(10.0f) * p13;
    const P2 dL = pfma(pk(5.0f), p12, p23) + t13, dR = pfma(pk(5.0f), p23, p12) + t13;
    const P2 e1 = a1 - a2, e2 = a2 - a3;
    const P2 A = p23 * e1, B = p12 * e2;
    const P2 uL2 = pfma(pk(0.125f), pfma(pk(3.0f), d32, d21), w2);
    const P2 uR2 = pfma(pk(-0.125f), pfma(pk(3.0f), d21, d32), w2);
    const P2 nL = pfma(pk(0.375f), A, pk(0.625f) * B), nR = pfma(pk(0.375f), B, pk(0.625f) * A);
    left = pfma(nL, prcp(dL), uL2);
    right = pfma(-nR, prcp(dR), uR2);
}

// Characteristic basis of the node state, packed: the members and formulas
// of CharBasis<float> (Pulliam-Chaussee eigenvectors along the unit normal
// of the node metric, projection W = L q and back projection U = R W in
// vector form).
struct CharBasisP {
    P2 kx, ky, kz, u, v, w, rho, irho, p, c, a0, g, cir, al, half_uu, H, cth;
    __device__ __forceinline__ void init_state(const GasR<float>& gs, const P2 q[5]) {
        irho = prcp(q[0]);
        rho = q[0];
        u = q[1] * irho;
        v = q[2] * irho;
        w = q[3] * irho;
        half_uu = pk(0.5f) * pfma(u, u, pfma(v, v, w * w));
        p = pk(gs.gm1) * (q[4] - rho * half_uu);
        const P2 c2 = pk(gs.gamma) * p * irho;
        const P2 ic = prsqrt(c2);
        c = c2 * ic;
        const P2 ic2 = ic * ic;
        a0 = pk(1.0f) - pk(gs.gm1) * half_uu * ic2;
        g = pk(gs.gm1) * ic2;
        cir = c * irho * pk(0.70710678118654752440f);
        al = rho * ic * pk(0.70710678118654752440f);
        H = pfma(c2, pk(gs.inv_gm1), half_uu);
    }
    __device__ __forceinline__ void init(const GasR<float>& gs, const P2 q[5], P2 mx, P2 my, P2 mz) {
        init_state(gs, q);
        const P2 imm = prsqrt(pfma(mx, mx, pfma(my, my, mz * mz)));
        kx = mx * imm;
        ky = my * imm;
        kz = mz * imm;
        cth = c * pfma(kx, u, pfma(ky, v, kz * w));
    }
    // W = L q of the node's own state (as CharBasis<double>::center)
    __device__ __forceinline__ void center(const GasR<float>& gs, P2 W[5]) const {
        const P2 S = rho * pk(gs.gm1_over_g);
        W[0] = kx * S;
        W[1] = ky * S;
        W[2] = kz * S;
        W[3] = W[4] = c * pk(gs.inv_g_sqrt2);
    }
    // W = L q
    __device__ __forceinline__ void project(P2 q0, P2 q1, P2 q2, P2 q3, P2 q4, P2 W[5]) const {
        const P2 d1 = (q1 - u * q0) * irho, d2 = (q2 - v * q0) * irho, d3 = (q3 - w * q0) * irho;
        const P2 S = pfma(a0, q0, g * (pfma(u, q1, pfma(v, q2, w * q3)) - q4));
        W[0] = pfma(kx, S, d2 * kz - d3 * ky);
        W[1] = pfma(ky, S, d3 * kx - d1 * kz);
        W[2] = pfma(kz, S, d1 * ky - d2 * kx);
        const P2 kd = pfma(kx, d1, pfma(ky, d2, kz * d3)) * pk(0.70710678118654752440f);
        const P2 base = cir * (q0 - S);
        W[3] = base + kd;
        W[4] = base - kd;
    }
    // U = R W
    __device__ __forceinline__ void back(const P2 W[5], P2 U[5]) const {
        const P2 Wk = pfma(kx, W[0], pfma(ky, W[1], kz * W[2]));
        const P2 Cx = ky * W[2] - kz * W[1], Cy = kz * W[0] - kx * W[2], Cz = kx * W[1] - ky * W[0];
        const P2 s = W[3] + W[4], t = W[3] - W[4];
        const P2 as = al * s, act = al * c * t;
        U[0] = Wk + as;
        U[1] = pfma(u, U[0], pfma(rho, Cx, act * kx));
        U[2] = pfma(v, U[0], pfma(rho, Cy, act * ky));
        U[3] = pfma(w, U[0], pfma(rho, Cz, act * kz));
        U[4] = pfma(half_uu, Wk, pfma(rho, pfma(u, Cx, pfma(v, Cy, w * Cz)), pfma(as, H, al * cth * t)));
    }
};

// Steger-Warming split flux along (kx, ky, kz) * mm, POS selects F+: the
// scalar sw_flux of hx_common.cuh, packed.
template <bool POS>
__device__ __forceinline__ void sw_flux_p(const GasR<float>& gs, const P2 q[5], P2 kx, P2 ky, P2 kz, P2 mm, P2 F[5]) {
    const P2 irho = prcp(q[0]);
    const P2 u = q[1] * irho, v = q[2] * irho, w = q[3] * irho;
    const P2 uu = pfma(u, u, pfma(v, v, w * w));
    const P2 p = pk(gs.gm1) * (q[4] - pk(0.5f) * q[0] * uu);
    const P2 c2 = pk(gs.gamma) * p * irho;
    const P2 c = c2 * prsqrt(c2);
    const P2 th = pfma(kx, u, pfma(ky, v, kz * w));
    P2 l1 = th, l4 = th + c, l5 = th - c;
    if (POS) {
        l1 = ppos(l1);
        l4 = ppos(l4);
        l5 = ppos(l5);
    } else {
        l1 = pneg(l1);
        l4 = pneg(l4);
        l5 = pneg(l5);
    }
    const P2 a = q[0] * mm * pk(gs.inv_2gamma);
    const P2 S45 = l4 + l5, D45 = l4 - l5;
    const P2 aM = a * pfma(pk(gs.two_gm1), l1, S45);
    const P2 acD = a * (c * D45);
    const P2 H = pfma(pk(0.5f), uu, c2 * pk(gs.inv_gm1));
    F[0] = aM;
    F[1] = pfma(u, aM, kx * acD);
    F[2] = pfma(v, aM, ky * acD);
    F[3] = pfma(w, aM, kz * acD);
    F[4] = pfma(a, pfma(pk(gs.gm1) * l1, uu, S45 * H), th * acD);
}

// Derivative at node p of two lines of n nodes from values f(-3..3) around
// it, with the one-sided closure next to physical ends: the scalar dline of
// hx_common.cuh, packed (both lines share p, n and the ends).
template <class F>
__device__ __forceinline__ P2 dline_p(const F& f, int p, int n, bool lo, bool hi) {
    if (lo && p <= 2) {
        if (p == 0) return (pfma(pk(-3.0f), f(0), pfma(pk(4.0f), f(1), -f(2)))) * pk(0.5f);
        if (p == 1) return (f(1) - f(-1)) * pk(0.5f);
        return (f(-2) - pk(8.0f) * f(-1) + pk(8.0f) * f(1) - f(2)) * pk(1.0f / 12.0f);
    }
    if (hi && p >= n - 3) {
        if (p == n - 1) return pfma(pk(3.0f), f(0), pfma(pk(-4.0f), f(-1), f(-2))) * pk(0.5f);
        if (p == n - 2) return (f(1) - f(-1)) * pk(0.5f);
        return (f(-2) - pk(8.0f) * f(-1) + pk(8.0f) * f(1) - f(2)) * pk(1.0f / 12.0f);
    }
    return d6p(f(-3), f(-2), f(-1), f(1), f(2), f(3));
}

}  // namespace hx
