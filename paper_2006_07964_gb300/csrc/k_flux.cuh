// k_flux.cuh -- fused per-direction flux kernel of the RK-stage residual.
//
// One launch handles one computational direction d (xi, eta or zeta) for all
// blocks.  A CTA owns NA adjacent lines of the sweep (persistent: it strides
// over a list of line groups) and marches along them in chunks of TP nodes,
// keeping a ring of RING nodes per line in shared memory.  Every node's
// work is done once; per chunk c (nodes c*TP ..):
//   load  state and metric of d at nodes c*TP+3 .. c*TP+TP+2 (FP64: the
//         state only) and, for the modified scheme, the state difference
//         across the face before each; FP32: L2 prefetch hints for this
//         chunk's output step and the next chunk's load and node steps;
//   node  at nodes c*TP+1 .. c*TP+TP: characteristic projection of the
//         5-node stencil at the node (modified AFWENO, Sec. 4.5.1,
//         Figs. 10-11; the projection is linear, so the WENO's first
//         differences are the projected state differences of the stencil's
//         four faces), WENO5 left value at the node's + face and right
//         value at its - face (Eqs. (13)-(17)), back projection; the node
//         flux (Eq. (4)) and, for Navier-Stokes, the node viscous flux of d
//         from the node's stress tensor and heat flux (Eqs. (5)-(6));
//         FP64 reads the node's basis state (k_prep) and unit normal;
//   face  at faces c*TP .. c*TP+TP-1: sixth-order midpoint metric and the
//         Steger-Warming numerical flux h = F+(U^L) + F-(U^R) (Eq. (12));
//   out   at nodes c*TP-2 .. c*TP+TP-3 (two behind, so that every input is
//         ready): Eq. (19) minus the sixth-order central derivative of the
//         viscous flux, accumulated into A.
// This replaces the split_flux / sum_split_flux / phys_flux / cflux_df and
// vflux_flux / vflux_df chains of Figs. 11-12; the intermediates never leave
// shared memory and no node is computed twice.
#pragma once
#include "hx_common.cuh"

namespace hx {

template <int DIR, int TP, int NA>
struct FluxLayout {
    static constexpr int RING = TP >= 8 ? 2 * TP : 16;   // >= TP + 6 live nodes, power of two
    // DIR 0 sweeps the contiguous i: lanes run along the sweep and planes are
    // [line][slot]; a warp spans two lines of 16 nodes when TP = 16, so odd
    // lines swap the two halves of their ring (slot ^ RING/2) and the two
    // half-warps fall on complementary banks.  DIR 1, 2: lanes run across
    // (i), planes [slot][line].
    static constexpr int PLANE = RING * NA;
    // fields per ring slot: Q 5, metric 3, node flux 5, U^L (then h) 5, U^R 5, viscous node flux 4;
    // with stored normals (NRM) the metric and the normals are read at the
    // node and face that use them, not staged: 3 fields fewer; the modified
    // scheme (DQ) adds the state difference Q_(p+1) - Q_p across face p+1/2: 5
    static constexpr int NF_INV = 23, NF_VISC = 27;
    static_assert((NA & (NA - 1)) == 0 && (TP & (TP - 1)) == 0 && (RING & (RING - 1)) == 0,
                  "power-of-two line count, chunk and ring");
    // Slot of node p: (p mod RING); DIR 0 rotates odd lines by RING/2 (the
    // XOR of the top slot bit, written as an add inside the mask).  The line
    // base has no bits in common with the slot, so each index is an add and
    // one three-input logic operation.
    __device__ static __forceinline__ int idx(int p, int a) {
        if (DIR == 0) return (a * RING) | ((p + 4 * RING + (a & 1) * (RING / 2)) & (RING - 1));
        return ((p + 4 * RING) * NA + a) & (RING * NA - 1);
    }
    // Item it (>= 0) of a step over X nodes of NA lines -> (node, line).
    // Along xi, X is TP (a power of two) after the first chunk: a shift
    // then, an integer division only in the first chunk.
    __device__ static __forceinline__ void split(int it, int X, int& p, int& a) {
        const unsigned u = (unsigned)it;
        if (DIR == 0) {
            if (X == TP) {
                p = (int)(u % TP);
                a = (int)(u / TP);
            } else {
                p = (int)(u % (unsigned)X);
                a = (int)(u / (unsigned)X);
            }
        } else {
            a = (int)(u % NA);
            p = (int)(u / NA);
        }
    }
    template <class R, bool VISC, bool NRM, bool DQ>
    static constexpr size_t smem_bytes() {
        return sizeof(R) * (size_t)PLANE * ((VISC ? NF_VISC : NF_INV) - (NRM ? 3 : 0) + (DQ ? 5 : 0));
    }
};

// RK (last sweep of the FP64 form only): instead of storing A, finish
// R = -J (A + div) and the RK3 stage combination at each output node
// (Eq. (20)), with the wall-node values and the non-finite / non-physical
// flags.  The mixed form ends its stages in k_rk_stage instead.
// SCH 0: modified AFWENO (characteristic space at the node, Figs. 10-11);
// SCH 1: original AFWENO (characteristic space at the face from the mean
// state and the face metric, two independent WENOs per face, Fig. 9).
// NRM (FP64 with the stored unit normals of k_normals and the node state of
// k_prep): the node basis and the face metric are read from them instead of
// formed from the metric and the state.
// Resident CTAs per SM that the register allocation must allow.  FP64: two
// of 256 threads (128 registers) or three of 128, so that the FP64 pipe
// always has a second CTA's warps (four of 128 spill at 128 registers and
// measured 1.3 % slower).  FP32 Navier-Stokes with 128 threads:
// seven (72 registers), which is what its shared memory allows; left free,
// the allocation drifts between 72 and 80 registers (six CTAs) with small
// code changes.  Other FP32 sweeps: no target (0); the compiler's own
// allocation measured as fast as a 64-register target and faster than an
// explicit 85-register one, and Euler sweeps keep 56-64 registers.
template <class R, int NT, bool VISC, bool NRM>
constexpr int flux_min_ctas() {
    return sizeof(R) == 8 ? (NT >= 256 ? 2 : 3) : (VISC && NT < 256 ? 7 : 0);
}

template <class R, int DIR, int TP, int NA, bool VISC, bool RK, int SCH, bool NRM>
__global__ void __launch_bounds__(TP * NA, flux_min_ctas<R, TP * NA, VISC, NRM>())
k_flux(const DevBlock* __restrict__ blocks, const Tile* __restrict__ tiles, int ntiles,
       const R* __restrict__ Q, const R* __restrict__ met, const R* __restrict__ nrm,
       const R* __restrict__ nst, long long fs, const R* __restrict__ stress, R* __restrict__ A, int accumulate,
       GasR<R> gs, RKArgs rk) {
    using LY = FluxLayout<DIR, TP, NA>;
    constexpr int PL = LY::PLANE;
    constexpr int NT = TP * NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(!NRM || sizeof(R) == 8, "stored normals are the FP64 form's");
    R* sQ = reinterpret_cast<R*>(smem_raw);   // 5 planes
    R* sM = sQ + 5 * PL;                       // 3 (not NRM)
    R* sF = sM + (NRM ? 0 : 3) * PL;           // 5
    R* sUL = sF + 5 * PL;                      // 5 (U^L at the + face, then h)
    R* sUR = sUL + 5 * PL;                     // 5 (U^R at the - face)
    R* sFv = sUR + 5 * PL;                     // 4 (VISC)
    R* sD = sFv + (VISC ? 4 : 0) * PL;         // 5 (SCH 0): Q_(p+1) - Q_p at slot p
    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile T = tiles[t];
        const DevBlock B = blocks[T.b];
        const int n = B.n[DIR];
        const int a0 = DIR == 0 ? T.j0 : T.i0;
        const int na = DIR == 0 ? B.n[1] : B.n[0];
        const long long sd = DIR == 0 ? 1 : (DIR == 1 ? B.sj : B.sk);
        const long long sa = DIR == 0 ? B.sj : 1;
        const long long e0 = node_index(B, T.i0, T.j0, T.k0);   // node 0 of line 0 (sweep index 0)
        const bool lo = (B.phys >> (2 * DIR)) & 1, hi = (B.phys >> (2 * DIR + 1)) & 1;

        for (int c = 0; c * TP - 2 < n; ++c) {
            const int base = c * TP;
            // ---- load nodes base+3 .. base+TP+2 (first chunk also -3 .. 2)
            {
                const int first = c == 0 ? -3 : base + 3, cnt = c == 0 ? TP + 6 : TP;
                for (int it = tid; it < cnt * NA; it += NT) {
                    int p, a;
                    LY::split(it, cnt, p, a);
                    p += first;
                    if (a0 + a >= na || p > n + 2) continue;
                    const long long e = hx_chk(B, e0 + p * sd + a * sa);
                    const int s = LY::idx(p, a);
                    R qp[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f) {
                        qp[f] = Q[f * fs + e];
                        sQ[f * PL + s] = qp[f];
                    }
                    if (SCH == 0 && p > -3) {   // the face p-1/2 (its left node from global memory)
                        const long long em = hx_chk(B, e - sd);
                        const int sl = LY::idx(p - 1, a);
#pragma unroll
                        for (int f = 0; f < 5; ++f) sD[f * PL + sl] = qp[f] - Q[f * fs + em];
                    }
                    if (!NRM) {
#pragma unroll
                        for (int f = 0; f < 3; ++f) sM[f * PL + s] = met[(3 * DIR + f) * fs + e];
                    }
                }
            }
            // ---- L2 prefetches (FP32 sweeps; each thread owns one node of
            // every step): what this chunk's output step reads from global
            // memory (the accumulator), and what the next chunk's load and
            // node steps read (state, metric, stress).  Issued now, they arrive
            // while the stencil phases run (measured on the 128^3 Taylor-Green
            // sweeps: eta 0.124 -> 0.116 ms).
            if (sizeof(R) == 4) {
                // Opaque copies of the thread index and the field stride, so
                // that none of this address arithmetic is shared with the
                // other steps or hoisted out of the chunk loop, where it
                // would hold registers through the stencil phases.
                int tq = tid;
                long long fq = fs;
                asm volatile("" : "+r"(tq), "+l"(fq));
                int p, a;
                LY::split(tq, TP, p, a);
                const bool line = a0 + a < na;
                const int po = base - 2 + p;   // this chunk's output node
                if (accumulate && line && po >= 0 && po < n) {
                    const long long e = hx_chk(B, e0 + po * sd + a * sa);
#pragma unroll
                    for (int k = 0; k < 5; ++k) prefetch_l2(A + k * fq + e);
                }
                const int pl = base + TP + 3 + p;   // the next chunk's load node
                if (line && pl <= n + 2) {
                    const long long e = hx_chk(B, e0 + pl * sd + a * sa);
#pragma unroll
                    for (int f = 0; f < 5; ++f) prefetch_l2(Q + f * fq + e);
#pragma unroll
                    for (int f = 0; f < 3; ++f) prefetch_l2(met + (3 * DIR + f) * fq + e);
                }
                const int pn = base + TP + 1 + p;   // the next chunk's node step
                if (VISC && line && pn <= n + 2 && !(hi && pn >= n)) {
                    const long long e = hx_chk(B, e0 + pn * sd + a * sa);
#pragma unroll
                    for (int f = 0; f < 9; ++f) prefetch_l2(stress + f * fq + e);
                }
            }
            __syncthreads();
            // ---- node work at base+1 .. base+TP (first chunk also -3 .. 0)
            {
                const int first = c == 0 ? -3 : base + 1, cnt = c == 0 ? TP + 4 : TP;
                for (int it = tid; it < cnt * NA; it += NT) {
                    int p, a;
                    LY::split(it, cnt, p, a);
                    p += first;
                    if (a0 + a >= na || p > n + 2) continue;
                    const int s0 = LY::idx(p, a);
                    const bool vnode = VISC && !((lo && p < 0) || (hi && p >= n));
                    const long long e = hx_chk(B, e0 + p * sd + a * sa);
                    R S[9];
                    if (vnode) {   // issued first; consumed after the node flux
#pragma unroll
                        for (int f = 0; f < 9; ++f) S[f] = stress[f * fs + e];
                    }
                    R q[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f) q[f] = sQ[f * PL + s0];
                    R mx, my, mz;
                    if (NRM) {
                        mx = met[(3 * DIR) * fs + e];
                        my = met[(3 * DIR + 1) * fs + e];
                        mz = met[(3 * DIR + 2) * fs + e];
                    } else {
                        mx = sM[s0];
                        my = sM[PL + s0];
                        mz = sM[2 * PL + s0];
                    }
                    CharBasis<R> cb;
                    if constexpr (NRM)
                        cb.load_state(nst + e, fs, q[0]);
                    else
                        cb.init(gs, q, mx, my, mz);
                    // node flux along the un-normalised metric, Eq. (4)
                    {
                        const R th = mx * cb.u + my * cb.v + mz * cb.w;
                        sF[s0] = q[0] * th;
                        sF[PL + s0] = q[1] * th + mx * cb.p;
                        sF[2 * PL + s0] = q[2] * th + my * cb.p;
                        sF[3 * PL + s0] = q[3] * th + mz * cb.p;
                        sF[4 * PL + s0] = (q[4] + cb.p) * th;
                    }
                    // viscous node flux m.(tau, beta); FP32 writes it after the WENO
                    // of the node, so that the stress loads have arrived by then
                    auto put_fv = [&]() {
                        if (!vnode) return;
                        sFv[s0] = mx * S[0] + my * S[3] + mz * S[4];
                        sFv[PL + s0] = mx * S[3] + my * S[1] + mz * S[5];
                        sFv[2 * PL + s0] = mx * S[4] + my * S[5] + mz * S[2];
                        sFv[3 * PL + s0] = mx * S[6] + my * S[7] + mz * S[8];
                    };
                    constexpr bool LATE_FV = sizeof(R) == 4;
                    if (!LATE_FV) put_fv();
                    if (SCH == 1 || p < -1 || p > n) {   // WENO only where a face needs it
                        if (LATE_FV) put_fv();
                        continue;
                    }
                    if constexpr (SCH == 0) {
                        if (NRM) {   // node normal (defined on nodes -1 .. n)
                            const R* nr = nrm + 7 * DIR * fs + e;
                            cb.set_normal(nr[0], nr[fs], nr[2 * fs]);
                        }
                        // the stencil's characteristic differences across faces
                        // p-3/2 .. p+3/2, and the node's own values in closed form
                        R dW[4][5], Wc[5];
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            const int si = LY::idx(p - 2 + s, a);
                            cb.project(sD[si], sD[PL + si], sD[2 * PL + si], sD[3 * PL + si], sD[4 * PL + si], dW[s]);
                        }
                        cb.center(gs, Wc);
                        R WL[5], WR[5];
                        weno_pair5_d(dW, Wc, WL, WR);
                        R U[5];
                        cb.back(WL, U);
#pragma unroll
                        for (int f = 0; f < 5; ++f) sUL[f * PL + s0] = U[f];
                        cb.back(WR, U);
#pragma unroll
                        for (int f = 0; f < 5; ++f) sUR[f * PL + s0] = U[f];
                    }
                    if (LATE_FV) put_fv();
                }
            }
            __syncthreads();
            // ---- faces base .. base+TP-1 (first chunk also -1): h in place of U^L
            {
                const int first = c == 0 ? -1 : base, cnt = c == 0 ? TP + 1 : TP;
                for (int it = tid; it < cnt * NA; it += NT) {
                    int f, a;
                    LY::split(it, cnt, f, a);
                    f += first;
                    if (a0 + a >= na || f > n - 1) continue;
                    const int uf = LY::idx(f, a), ur = LY::idx(f + 1, a);
                    R kx, ky, kz, mm;
                    if (NRM) {   // + face normal and |m| of node f (defined on nodes -1 .. n-1)
                        const R* nr = nrm + (7 * DIR + 3) * fs + hx_chk(B, e0 + f * sd + a * sa);
                        kx = nr[0];
                        ky = nr[fs];
                        kz = nr[2 * fs];
                        mm = nr[3 * fs];
                    } else {
                        R mf[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const R* m = sM + k * PL;
                            mf[k] = mid6<R>(m[LY::idx(f - 2, a)], m[LY::idx(f - 1, a)], m[LY::idx(f, a)],
                                            m[LY::idx(f + 1, a)], m[LY::idx(f + 2, a)], m[LY::idx(f + 3, a)]);
                        }
                        const R mm2 = mf[0] * mf[0] + mf[1] * mf[1] + mf[2] * mf[2];
                        const R imm = hrsqrt(mm2);
                        mm = mm2 * imm;
                        kx = mf[0] * imm;
                        ky = mf[1] * imm;
                        kz = mf[2] * imm;
                    }
                    R ql[5], qr[5];
                    if (SCH == 0) {
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            ql[k] = sUL[k * PL + uf];
                            qr[k] = sUR[k * PL + ur];
                        }
                    } else {
                        R qm[5];
#pragma unroll
                        for (int k = 0; k < 5; ++k) qm[k] = R(0.5) * (sQ[k * PL + uf] + sQ[k * PL + ur]);
                        CharBasis<R> cb;
                        cb.init_state(gs, qm);
                        cb.set_normal(kx, ky, kz);
                        R W[6][5];
#pragma unroll
                        for (int s = -2; s <= 3; ++s) {
                            const int si = LY::idx(f + s, a);
                            cb.project(sQ[si], sQ[PL + si], sQ[2 * PL + si], sQ[3 * PL + si], sQ[4 * PL + si],
                                       W[s + 2]);
                        }
                        R WL[5], WR[5];
                        weno_face10(W, WL, WR);
                        cb.back(WL, ql);
                        cb.back(WR, qr);
                    }
                    R h[5];
                    face_flux(gs, ql, qr, kx, ky, kz, mm, h);
#pragma unroll
                    for (int k = 0; k < 5; ++k) sUL[k * PL + uf] = h[k];
                }
            }
            __syncthreads();
            // ---- outputs base-2 .. base+TP-3: Eq. (19) minus the viscous derivative
            for (int it = tid; it < TP * NA; it += NT) {
                int p, a;
                LY::split(it, TP, p, a);
                p += base - 2;
                if (a0 + a >= na || p < 0 || p >= n) continue;
                const long long e = hx_chk(B, e0 + p * sd + a * sa);
                const int sp = LY::idx(p, a), sm1 = LY::idx(p - 1, a);
                const int s1 = LY::idx(p + 1, a), s2 = LY::idx(p + 2, a), s3 = LY::idx(p + 3, a);
                const int t1 = LY::idx(p - 1, a), t2 = LY::idx(p - 2, a), t3 = LY::idx(p - 3, a);
                // The accumulator is loaded first, so that it arrives while the
                // differences below are formed from shared memory.  The fused
                // RK sweep's other inputs are loaded where they are used:
                // hoisting them too costs registers (80 instead of 72 in FP32,
                // one CTA less per SM) and measured slower.
                R acc[5];
                if (accumulate) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) acc[k] = A[k * fs + e];
                }
                R dv[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const R* F = sF + k * PL;
                    R div = sUL[k * PL + sp] - sUL[k * PL + sm1] + R(17.0 / 256.0) * (F[s1] - F[t1]) -
                            R(13.0 / 320.0) * (F[s2] - F[t2]) + R(19.0 / 3840.0) * (F[s3] - F[t3]);
                    if (VISC && k > 0) {
                        const R* Fv = sFv + (k - 1) * PL;
                        auto fv = [&](int s) { return Fv[LY::idx(p + s, a)]; };
                        div -= dline<R>(fv, p, n, lo, hi);
                    }
                    dv[k] = accumulate ? acc[k] + div : div;
                }
                if (!RK) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) A[k * fs + e] = dv[k];
                } else {
                    static_assert(!RK || sizeof(R) == 8, "the fused RK stage is the FP64 form's");
                    double qo[5];
                    const double f = -rk.cc * (rk.dtl ? rk.dtl[e] : B.dt) * rk.metd[9 * fs + e];
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        double v = rk.ca * rk.Qn[k * fs + e] + f * (double)dv[k];
                        if (rk.cb != 0.0) v += rk.cb * rk.Qk[k * fs + e];
                        qo[k] = v;
                    }
                    if (B.wall) {   // node indices of this output (line groups start at sweep index 0)
                        const int ni_ = DIR == 0 ? p : T.i0 + a;
                        const int nj_ = DIR == 1 ? p : (DIR == 0 ? T.j0 + a : T.j0);
                        const int nk_ = DIR == 2 ? p : T.k0;
                        const bool on = ((B.wall & 1) && ni_ == 0) || ((B.wall & 2) && ni_ == B.n[0] - 1) ||
                                        ((B.wall & 4) && nj_ == 0) || ((B.wall & 8) && nj_ == B.n[1] - 1) ||
                                        ((B.wall & 16) && nk_ == 0) || ((B.wall & 32) && nk_ == B.n[2] - 1);
                        if (on) {
                            const double pw = rk.gm1 * (qo[4] - 0.5 * (qo[1] * qo[1] + qo[2] * qo[2] + qo[3] * qo[3]) / qo[0]);
                            qo[1] = qo[2] = qo[3] = 0.0;
                            qo[4] = pw / rk.gm1;
                        }
                    }
                    bool bad = false;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        bad = bad || nonfinite_bits(qo[k]);
                        rk.Qout[k * fs + e] = qo[k];
                    }
                    if (!bad &&
                        !(qo[0] > 0.0 && qo[4] * qo[0] - 0.5 * (qo[1] * qo[1] + qo[2] * qo[2] + qo[3] * qo[3]) > 0.0))
                        atomicOr(rk.flags, (unsigned)FLAG_UNPHYSICAL);
                    if (bad) atomicOr(rk.flags, (unsigned)FLAG_NONFINITE);
                }
            }
            // no barrier here: the next chunk's loads touch only state and
            // metric slots, and its node step comes after the next barrier
        }
        __syncthreads();   // before the next line group reuses the ring
    }
}

}  // namespace hx
