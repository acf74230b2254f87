// k_flux.cuh -- fused per-direction flux kernel of the RK-stage residual.
//
// One launch handles one computational direction d (xi, eta or zeta) for all
// blocks.  A CTA takes sweep tiles of TP nodes along d times NA lines across
// (persistent: it strides over the tile list) and does, in shared memory:
//   A  stage the state Q and the metric of d on nodes -3 .. TP+2 of the tile;
//   B  at nodes -1 .. TP: characteristic projection of the 5-node stencil at
//      the node (modified AFWENO, Sec. 4.5.1, Figs. 10-11), WENO5 left value
//      at the node's + face and right value at its - face (Eqs. (13)-(17)),
//      back projection;
//   C  node fluxes (Eq. (4)) on nodes -3 .. TP+2, and for Navier-Stokes the
//      node viscous fluxes of d (Eqs. (5)-(6)) from the gradients;
//   D  at faces -1/2 .. TP-1/2: sixth-order midpoint metric and the
//      Steger-Warming numerical flux h = F+(U^L) + F-(U^R) (Eq. (12));
//   E  Eq. (19) at the TP output nodes minus the sixth-order central
//      derivative of the viscous flux (Fig. 12), accumulated into A.
// Phases B..E replace the split_flux / sum_split_flux / phys_flux / cflux_df
// and vflux_flux / vflux_df kernel chains of Figs. 11-12: the intermediates
// never leave shared memory.
#pragma once
#include "hx_common.cuh"

namespace hx {

template <int DIR, int TP, int NA>
struct FluxLayout {
    static constexpr int NP = TP + 6;   // nodes -3 .. TP+2
    static constexpr int NU = TP + 2;   // nodes -1 .. TP
    // DIR 0 sweeps the contiguous i: lanes run along the sweep, planes are
    // [line][node] with one pad element; DIR 1, 2: lanes run across (i).
    static constexpr int SP = DIR == 0 ? NA * (NP + 1) : NP * NA;
    static constexpr int SU = DIR == 0 ? NA * (NU + 1) : NU * NA;
    __device__ static __forceinline__ int pidx(int p, int a) {   // p in [-3, TP+2]
        return DIR == 0 ? a * (NP + 1) + (p + 3) : (p + 3) * NA + a;
    }
    __device__ static __forceinline__ int uidx(int p, int a) {   // p in [-1, TP]
        return DIR == 0 ? a * (NU + 1) + (p + 1) : (p + 1) * NA + a;
    }
    __device__ static __forceinline__ void split(int it, int X, int& p, int& a) {
        if (DIR == 0) {
            p = it % X;
            a = it / X;
        } else {
            a = it % NA;
            p = it / NA;
        }
    }
    template <class R, bool VISC>
    static constexpr size_t smem_bytes() {
        return sizeof(R) * (size_t)(8 * SP + 10 * SU + (VISC ? 4 * SP : 0));
    }
};

template <class R, int DIR, int TP, int NA, bool VISC>
__global__ void __launch_bounds__(TP * NA)
k_flux(const DevBlock* __restrict__ blocks, const Tile* __restrict__ tiles, int ntiles,
       const R* __restrict__ Q, const R* __restrict__ met, long long fs, const R* __restrict__ prim,
       const R* __restrict__ grad, R* __restrict__ A, int accumulate, Gas gas) {
    using LY = FluxLayout<DIR, TP, NA>;
    constexpr int NP = LY::NP, NU = LY::NU, SP = LY::SP, SU = LY::SU;
    constexpr int NT = TP * NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sQ = reinterpret_cast<R*>(smem_raw);   // state, then node fluxes
    R* sM = sQ + 5 * SP;                       // metric of DIR
    R* sUL = sM + 3 * SP;                      // U^L at + faces, then h
    R* sUR = sUL + 5 * SU;                     // U^R at - faces
    R* sFv = sUR + 5 * SU;                     // viscous node fluxes (VISC)

    GasR<R> gs;
    gs.init(gas);
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const DevBlock B = blocks[T.b];
        const int n = B.n[DIR];
        const int p0 = DIR == 0 ? T.i0 : (DIR == 1 ? T.j0 : T.k0);
        const int a0 = DIR == 0 ? T.j0 : T.i0;
        const int na = DIR == 0 ? B.n[1] : B.n[0];
        const long long sd = DIR == 0 ? 1 : (DIR == 1 ? B.sj : B.sk);
        const long long sa = DIR == 0 ? B.sj : 1;
        const long long e0 = node_index(B, T.i0, T.j0, T.k0);
        const bool lo = (B.phys >> (2 * DIR)) & 1, hi = (B.phys >> (2 * DIR + 1)) & 1;

        // ---- A: stage state and metric of DIR on nodes -3 .. TP+2
        for (int it = tid; it < NP * NA; it += NT) {
            int p, a;
            LY::split(it, NP, p, a);
            p -= 3;
            if (a0 + a >= na || p0 + p > n + 2) continue;
            const long long e = e0 + p * sd + a * sa;
            const int s = LY::pidx(p, a);
#pragma unroll
            for (int c = 0; c < 5; ++c) sQ[c * SP + s] = Q[c * fs + e];
#pragma unroll
            for (int c = 0; c < 3; ++c) sM[c * SP + s] = met[(3 * DIR + c) * fs + e];
        }
        __syncthreads();

        // ---- B: characteristic WENO at nodes -1 .. TP
        for (int it = tid; it < NU * NA; it += NT) {
            int p, a;
            LY::split(it, NU, p, a);
            p -= 1;
            if (a0 + a >= na || p0 + p > n) continue;
            const int s0 = LY::pidx(p, a);
            R q[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) q[c] = sQ[c * SP + s0];
            CharBasis<R> cb;
            cb.init(gs, q, sM[s0], sM[SP + s0], sM[2 * SP + s0]);
            R W[5][5];
#pragma unroll
            for (int s = -2; s <= 2; ++s) {
                const int si = LY::pidx(p + s, a);
                cb.project(sQ[si], sQ[SP + si], sQ[2 * SP + si], sQ[3 * SP + si], sQ[4 * SP + si], W[s + 2]);
            }
            R WL[5], WR[5];
#pragma unroll
            for (int l = 0; l < 5; ++l) weno_pair(W[0][l], W[1][l], W[2][l], W[3][l], W[4][l], WL[l], WR[l]);
            R U[5];
            const int ui = LY::uidx(p, a);
            cb.back(WL, U);
#pragma unroll
            for (int c = 0; c < 5; ++c) sUL[c * SU + ui] = U[c];
            cb.back(WR, U);
#pragma unroll
            for (int c = 0; c < 5; ++c) sUR[c * SU + ui] = U[c];
        }
        __syncthreads();

        // ---- C: node fluxes (in place over the state) and viscous node fluxes
        for (int it = tid; it < NP * NA; it += NT) {
            int p, a;
            LY::split(it, NP, p, a);
            p -= 3;
            if (a0 + a >= na || p0 + p > n + 2) continue;
            const int s = LY::pidx(p, a);
            const R mx = sM[s], my = sM[SP + s], mz = sM[2 * SP + s];
            R q[5], f[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) q[c] = sQ[c * SP + s];
            point_flux(gs, q, mx, my, mz, f);
#pragma unroll
            for (int c = 0; c < 5; ++c) sQ[c * SP + s] = f[c];
            if (VISC) {
                const int pa = p0 + p;
                if ((lo && pa < 0) || (hi && pa >= n)) continue;
                const long long e = e0 + p * sd + a * sa;
                R g[12];
#pragma unroll
                for (int c = 0; c < 12; ++c) g[c] = grad[c * fs + e];
                R fv[4];
                viscous_flux(gs, prim[e], prim[fs + e], prim[2 * fs + e], prim[3 * fs + e], g, mx, my, mz, fv);
#pragma unroll
                for (int c = 0; c < 4; ++c) sFv[c * SP + s] = fv[c];
            }
        }
        // ---- D: Steger-Warming numerical flux at faces -1/2 .. TP-1/2
        for (int it = tid; it < (TP + 1) * NA; it += NT) {
            int f, a;
            LY::split(it, TP + 1, f, a);
            f -= 1;
            if (a0 + a >= na || p0 + f > n - 1) continue;
            R mf[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const R* m = sM + c * SP;
                mf[c] = mid6<R>(m[LY::pidx(f - 2, a)], m[LY::pidx(f - 1, a)], m[LY::pidx(f, a)],
                                m[LY::pidx(f + 1, a)], m[LY::pidx(f + 2, a)], m[LY::pidx(f + 3, a)]);
            }
            const R mm = hsqrt(mf[0] * mf[0] + mf[1] * mf[1] + mf[2] * mf[2]);
            const R imm = hrcp(mm);
            const R kx = mf[0] * imm, ky = mf[1] * imm, kz = mf[2] * imm;
            const int uf = LY::uidx(f, a), ur = LY::uidx(f + 1, a);
            R ql[5], qr[5], Fp[5], Fm[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                ql[c] = sUL[c * SU + uf];
                qr[c] = sUR[c * SU + ur];
            }
            sw_flux<R, true>(gs, ql, kx, ky, kz, mm, Fp);
            sw_flux<R, false>(gs, qr, kx, ky, kz, mm, Fm);
#pragma unroll
            for (int c = 0; c < 5; ++c) sUL[c * SU + uf] = Fp[c] + Fm[c];
        }
        __syncthreads();

        // ---- E: Eq. (19) minus the viscous derivative, accumulated into A
        for (int it = tid; it < TP * NA; it += NT) {
            int p, a;
            LY::split(it, TP, p, a);
            if (a0 + a >= na || p0 + p >= n) continue;
            const long long e = e0 + p * sd + a * sa;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const R* F = sQ + c * SP;
                R div = sUL[c * SU + LY::uidx(p, a)] - sUL[c * SU + LY::uidx(p - 1, a)] +
                        R(17.0 / 256.0) * (F[LY::pidx(p + 1, a)] - F[LY::pidx(p - 1, a)]) -
                        R(13.0 / 320.0) * (F[LY::pidx(p + 2, a)] - F[LY::pidx(p - 2, a)]) +
                        R(19.0 / 3840.0) * (F[LY::pidx(p + 3, a)] - F[LY::pidx(p - 3, a)]);
                if (VISC && c > 0) {
                    const R* Fv = sFv + (c - 1) * SP;
                    auto fv = [&](int s) { return Fv[LY::pidx(p + s, a)]; };
                    div -= dline<R>(fv, p0 + p, n, lo, hi);
                }
                A[c * fs + e] = accumulate ? A[c * fs + e] + div : div;
            }
        }
        __syncthreads();
    }
}

}  // namespace hx
