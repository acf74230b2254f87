// k_flux2.cuh -- the fused per-direction flux kernel of the mixed form
// (FP32 stencil arithmetic), two grid lines per thread.
//
// It computes what k_flux<float, ...> computes (the modified AFWENO of
// Sec. 4.5.1, Figs. 10-11, Steger-Warming face fluxes, Eq. (19), the
// viscous node flux of Eqs. (5)-(6) and its central derivative, accumulated
// into A; the stage's RK update follows in k_rk_stage), with the same ring
// of chunks in shared memory, but every thread owns a pair of adjacent
// lines and works on both with the packed FP32 instructions of hx_pair.cuh:
// the arithmetic, the shared-memory accesses (64-bit) and the index
// arithmetic are issued once for two nodes.  GB300 executes the scalar
// sweeps at the issue limit with the FP32 pipe a third busy; the packed form
// trades issue slots for pipe cycles.
//
// Shared memory: each field plane is [slot][line]; a pair (lines 2a, 2a+1)
// is one 8-byte word.  Along eta and zeta the lanes of a warp run across
// the pairs (consecutive i: 64-bit global accesses); along xi they run along
// the ring (consecutive i again), and the pair index is swizzled by the row
// so that a half-warp's 64-bit accesses fall on distinct banks.
#pragma once
#include "hx_pair.cuh"

namespace hx {

template <int DIR, int TP, int NP>
struct Flux2Layout {
    static constexpr int NA = 2 * NP;                     // lines per CTA
    static constexpr int RING = TP >= 8 ? 2 * TP : 16;    // >= TP + 8 live nodes, power of two
    static constexpr int RS = NP;                         // pairs per ring row
    static constexpr int PL = RING * RS * 2;              // floats per field plane
    // fields per ring slot: Q 5, metric 3, node flux 5, U^L (then h) 5, U^R 5, viscous node flux 4
    static constexpr int NF_INV = 23, NF_VISC = 27;
    static_assert((NP & (NP - 1)) == 0 && (TP & (TP - 1)) == 0, "power-of-two chunk and pair count");
    // float offset of (node p >= -4 RING, pair a2) within a plane.  Along xi
    // a half-warp reads 16 consecutive rows of one pair: the pair index is
    // XORed with the row's bits above the 16 / NP rows that share a bank
    // group, so that the 16 accesses fall on distinct banks.
    __device__ static __forceinline__ int idx(int p, int a2) {
        const int row = (p + 4 * RING) & (RING - 1);
        if (DIR == 0) return (row * RS + (a2 ^ ((row / (16 / NP)) & (NP - 1)))) * 2;
        return (row * RS + a2) * 2;
    }
    // item it (>= 0) of a step over X nodes of NP pairs -> (node, pair)
    __device__ static __forceinline__ void split(int it, int X, int& p, int& a2) {
        const unsigned u = (unsigned)it;
        if (DIR == 0) {
            if (X == TP) {
                p = (int)(u % TP);
                a2 = (int)(u / TP);
            } else {
                p = (int)(u % (unsigned)X);
                a2 = (int)(u / (unsigned)X);
            }
        } else {
            a2 = (int)(u % NP);
            p = (int)(u / NP);
        }
    }
    static constexpr size_t smem_bytes(bool visc) { return 4 * (size_t)PL * (visc ? NF_VISC : NF_INV); }
};

// The two lines' values of field f at node offset e: adjacent along i
// (eta and zeta sweeps, one 64-bit load) or one row apart (xi sweep).
template <int DIR>
__device__ __forceinline__ P2 gld2(const float* __restrict__ a, long long e, long long sa) {
    if (DIR == 0) return pk(a[e], a[e + sa]);
    return ld2(a + e);
}

// Resident CTAs per SM that the register allocation must allow: 16 warps
// per SM (128 registers), which the shared memory of the 128-line-node
// tiles also allows.
template <int NT>
constexpr int flux2_min_ctas() {
    return 2048 / 4 / NT;
}

template <int DIR, int TP, int NP, bool VISC>
__global__ void __launch_bounds__(TP * NP, flux2_min_ctas<TP * NP>())
k_flux2(const DevBlock* __restrict__ blocks, const Tile* __restrict__ tiles, int ntiles, const float* __restrict__ Q,
        const float* __restrict__ met, long long fs, const float* __restrict__ stress, float* __restrict__ A,
        int accumulate, GasR<float> gs) {
    using LY = Flux2Layout<DIR, TP, NP>;
    constexpr int PL = LY::PL;
    constexpr int NT = TP * NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sQ = reinterpret_cast<float*>(smem_raw);   // 5 planes
    float* sM = sQ + 5 * PL;                           // 3
    float* sF = sM + 3 * PL;                           // 5
    float* sUL = sF + 5 * PL;                          // 5 (U^L at the + face, then h)
    float* sUR = sUL + 5 * PL;                         // 5 (U^R at the - face)
    float* sFv = sUR + 5 * PL;                         // 4 (VISC)
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const DevBlock B = blocks[T.b];
        const int n = B.n[DIR];
        const int a0 = DIR == 0 ? T.j0 : T.i0;
        const int na = DIR == 0 ? B.n[1] : B.n[0];
        const long long sd = DIR == 0 ? 1 : (DIR == 1 ? B.sj : B.sk);
        const long long sa = DIR == 0 ? B.sj : 1;   // between the two lines of a pair
        const long long e0 = node_index(B, T.i0, T.j0, T.k0);
        const bool lo = (B.phys >> (2 * DIR)) & 1, hi = (B.phys >> (2 * DIR + 1)) & 1;

        for (int c = 0; c * TP - 2 < n; ++c) {
            const int base = c * TP;
            // ---- load nodes base+3 .. base+TP+2 (first chunk also -3 .. 2)
            {
                const int first = c == 0 ? -3 : base + 3, cnt = c == 0 ? TP + 6 : TP;
                for (int it = tid; it < cnt * NP; it += NT) {
                    int p, a2;
                    LY::split(it, cnt, p, a2);
                    p += first;
                    if (a0 + 2 * a2 >= na || p > n + 2) continue;
                    const long long e = hx_chk(B, e0 + p * sd + 2 * a2 * sa);
                    const int s = LY::idx(p, a2);
#pragma unroll
                    for (int f = 0; f < 5; ++f) st2(sQ + f * PL + s, gld2<DIR>(Q + f * fs, e, sa));
#pragma unroll
                    for (int f = 0; f < 3; ++f) st2(sM + f * PL + s, gld2<DIR>(met + (3 * DIR + f) * fs, e, sa));
                }
            }
            // ---- L2 prefetches: this chunk's accumulator and the next chunk's
            // state, metric and stress (as k_flux<float>)
            {
                int tq = tid;
                long long fq = fs;
                asm volatile("" : "+r"(tq), "+l"(fq));
                int p, a2;
                LY::split(tq, TP, p, a2);
                const bool line = a0 + 2 * a2 < na;
                const int po = base - 2 + p;
                if (accumulate && line && po >= 0 && po < n) {
                    const long long e = hx_chk(B, e0 + po * sd + 2 * a2 * sa);
#pragma unroll
                    for (int l = 0; l < (DIR == 0 ? 2 : 1); ++l) {
#pragma unroll
                        for (int k = 0; k < 5; ++k) prefetch_l2(A + k * fq + e + l * sa);
                    }
                }
                const int pl = base + TP + 3 + p;
                if (line && pl <= n + 2) {
                    const long long e = hx_chk(B, e0 + pl * sd + 2 * a2 * sa);
#pragma unroll
                    for (int l = 0; l < (DIR == 0 ? 2 : 1); ++l) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) prefetch_l2(Q + f * fq + e + l * sa);
#pragma unroll
                        for (int f = 0; f < 3; ++f) prefetch_l2(met + (3 * DIR + f) * fq + e + l * sa);
                    }
                }
                const int pn = base + TP + 1 + p;
                if (VISC && line && pn <= n + 2 && !(hi && pn >= n)) {
                    const long long e = hx_chk(B, e0 + pn * sd + 2 * a2 * sa);
#pragma unroll
                    for (int l = 0; l < (DIR == 0 ? 2 : 1); ++l) {
#pragma unroll
                        for (int f = 0; f < 9; ++f) prefetch_l2(stress + f * fq + e + l * sa);
                    }
                }
            }
            __syncthreads();
            // ---- node work at base+1 .. base+TP (first chunk also -3 .. 0)
            {
                const int first = c == 0 ? -3 : base + 1, cnt = c == 0 ? TP + 4 : TP;
                for (int it = tid; it < cnt * NP; it += NT) {
                    int p, a2;
                    LY::split(it, cnt, p, a2);
                    p += first;
                    if (a0 + 2 * a2 >= na || p > n + 2) continue;
                    const int s0 = LY::idx(p, a2);
                    const bool vnode = VISC && !((lo && p < 0) || (hi && p >= n));
                    P2 S[9];
                    if (vnode) {   // issued first; consumed after the WENO
                        const long long e = hx_chk(B, e0 + p * sd + 2 * a2 * sa);
#pragma unroll
                        for (int f = 0; f < 9; ++f) S[f] = gld2<DIR>(stress + f * fs, e, sa);
                    }
                    P2 q[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f) q[f] = ld2(sQ + f * PL + s0);
                    const P2 mx = ld2(sM + s0), my = ld2(sM + PL + s0), mz = ld2(sM + 2 * PL + s0);
                    CharBasisP cb;
                    cb.init(gs, q, mx, my, mz);
                    {   // node flux along the un-normalised metric, Eq. (4)
                        const P2 th = pfma(mx, cb.u, pfma(my, cb.v, mz * cb.w));
                        st2(sF + s0, q[0] * th);
                        st2(sF + PL + s0, pfma(q[1], th, mx * cb.p));
                        st2(sF + 2 * PL + s0, pfma(q[2], th, my * cb.p));
                        st2(sF + 3 * PL + s0, pfma(q[3], th, mz * cb.p));
                        st2(sF + 4 * PL + s0, (q[4] + cb.p) * th);
                    }
                    auto put_fv = [&]() {   // viscous node flux m.(tau, beta)
                        if (!vnode) return;
                        st2(sFv + s0, pfma(mx, S[0], pfma(my, S[3], mz * S[4])));
                        st2(sFv + PL + s0, pfma(mx, S[3], pfma(my, S[1], mz * S[5])));
                        st2(sFv + 2 * PL + s0, pfma(mx, S[4], pfma(my, S[5], mz * S[2])));
                        st2(sFv + 3 * PL + s0, pfma(mx, S[6], pfma(my, S[7], mz * S[8])));
                    };
                    if (p < -1 || p > n) {   // WENO only where a face needs it
                        put_fv();
                        continue;
                    }
                    P2 W[5][5];
#pragma unroll
                    for (int s = -2; s <= 2; ++s) {
                        if (s == 0) {   // the node's own state: closed form
                            cb.center(gs, W[2]);
                            continue;
                        }
                        const int si = LY::idx(p + s, a2);
                        cb.project(ld2(sQ + si), ld2(sQ + PL + si), ld2(sQ + 2 * PL + si), ld2(sQ + 3 * PL + si),
                                   ld2(sQ + 4 * PL + si), W[s + 2]);
                    }
                    P2 WL[5], WR[5];
#pragma unroll
                    for (int l = 0; l < 5; ++l) weno_pair_p(W[0][l], W[1][l], W[2][l], W[3][l], W[4][l], WL[l], WR[l]);
                    P2 U[5];
                    cb.back(WL, U);
#pragma unroll
                    for (int f = 0; f < 5; ++f) st2(sUL + f * PL + s0, U[f]);
                    cb.back(WR, U);
#pragma unroll
                    for (int f = 0; f < 5; ++f) st2(sUR + f * PL + s0, U[f]);
                    put_fv();
                }
            }
            __syncthreads();
            // ---- faces base .. base+TP-1 (first chunk also -1): h in place of U^L
            {
                const int first = c == 0 ? -1 : base, cnt = c == 0 ? TP + 1 : TP;
                for (int it = tid; it < cnt * NP; it += NT) {
                    int f, a2;
                    LY::split(it, cnt, f, a2);
                    f += first;
                    if (a0 + 2 * a2 >= na || f > n - 1) continue;
                    const int uf = LY::idx(f, a2), ur = LY::idx(f + 1, a2);
                    P2 mf[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float* m = sM + k * PL;
                        mf[k] = mid6p(ld2(m + LY::idx(f - 2, a2)), ld2(m + LY::idx(f - 1, a2)), ld2(m + uf),
                                      ld2(m + ur), ld2(m + LY::idx(f + 2, a2)), ld2(m + LY::idx(f + 3, a2)));
                    }
                    const P2 mm2 = pfma(mf[0], mf[0], pfma(mf[1], mf[1], mf[2] * mf[2]));
                    const P2 imm = prsqrt(mm2);
                    const P2 mm = mm2 * imm, kx = mf[0] * imm, ky = mf[1] * imm, kz = mf[2] * imm;
                    P2 ql[5], qr[5], Fp[5], Fm[5];
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        ql[k] = ld2(sUL + k * PL + uf);
                        qr[k] = ld2(sUR + k * PL + ur);
                    }
                    sw_flux_p<true>(gs, ql, kx, ky, kz, mm, Fp);
                    sw_flux_p<false>(gs, qr, kx, ky, kz, mm, Fm);
#pragma unroll
                    for (int k = 0; k < 5; ++k) st2(sUL + k * PL + uf, Fp[k] + Fm[k]);
                }
            }
            __syncthreads();
            // ---- outputs base-2 .. base+TP-3: Eq. (19) minus the viscous derivative
            for (int it = tid; it < TP * NP; it += NT) {
                int p, a2;
                LY::split(it, TP, p, a2);
                p += base - 2;
                if (a0 + 2 * a2 >= na || p < 0 || p >= n) continue;
                const bool two = a0 + 2 * a2 + 1 < na;   // the pair's second line lies in the block
                const long long e = hx_chk(B, e0 + p * sd + 2 * a2 * sa);
                P2 acc[5];
                if (accumulate) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc[k] = gld2<DIR>(A + k * fs, e, sa);
                }
                P2 dv[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float* F = sF + k * PL;
                    auto fl = [&](int s) { return ld2(F + LY::idx(p + s, a2)); };
                    P2 div = ld2(sUL + k * PL + LY::idx(p, a2)) - ld2(sUL + k * PL + LY::idx(p - 1, a2));
                    div = pfma(pk(17.0f / 256.0f), fl(1) - fl(-1), div);
                    div = pfma(pk(-13.0f / 320.0f), fl(2) - fl(-2), div);
                    div = pfma(pk(19.0f / 3840.0f), fl(3) - fl(-3), div);
                    if (VISC && k > 0) {
                        const float* Fv = sFv + (k - 1) * PL;
                        auto fv = [&](int s) { return ld2(Fv + LY::idx(p + s, a2)); };
                        div = div - dline_p(fv, p, n, lo, hi);
                    }
                    dv[k] = accumulate ? acc[k] + div : div;
                }
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if (DIR == 0) {
                        A[k * fs + e] = dv[k].v.x;
                        if (two) A[k * fs + e + sa] = dv[k].v.y;
                    } else if (two) {
                        st2(A + k * fs + e, dv[k]);
                    } else {
                        A[k * fs + e] = dv[k].v.x;
                    }
                }
            }
            // no barrier here: the next chunk's loads touch only state and
            // metric slots, and its node step comes after the next barrier
        }
        __syncthreads();   // before the next line group reuses the ring
    }
}

}  // namespace hx
