// k_misc.cu -- point-parallel kernels of the RK stage and of set-up:
// layout packing, halo gathers, conservative metrics (Eqs. (7)-(8)),
// primitives, chain-rule gradients and the node stress tensor (Eq. (21),
// Eqs. (5)-(6)), physical-face node values and the CFL time step.  The RK3
// combination (Eq. (20)) is fused into the last flux sweep.
#include "kernels.h"

namespace hx {

namespace {

constexpr int kThreads = 256;   // brick kernels: 32 x 8 threads

inline int grid_for(long long work, int per_cta = kThreads) {
    long long g = (work + per_cta - 1) / per_cta;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

__device__ __forceinline__ void brick_node(const Brick& br, int& i, int& j, int& k, bool& ok) {
    const int ti = threadIdx.x & 31, tj = threadIdx.x >> 5;
    i = br.i0 + ti;
    j = br.j0 + tj;
    k = br.k0;
    ok = ti < br.ni && tj < br.nj;
}

// ---------------------------------------------------------------- packing
template <class T>
__global__ void k_unpack(const double* __restrict__ src, T* __restrict__ dst, long long fs, DevBlock B, int nf) {
    const long long N = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nf;
         t += (long long)gridDim.x * blockDim.x) {
        const long long f = t / N, r = t - f * N;
        const int i = (int)(r % B.n[0]);
        const long long r2 = r / B.n[0];
        const int j = (int)(r2 % B.n[1]), k = (int)(r2 / B.n[1]);
        dst[f * fs + node_index(B, i, j, k)] = (T)src[t];
    }
}

__global__ void k_unpack2(const double* __restrict__ src, double* __restrict__ d64, float* __restrict__ d32,
                          long long fs, DevBlock B, int nf) {
    const long long N = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nf;
         t += (long long)gridDim.x * blockDim.x) {
        const long long f = t / N, r = t - f * N;
        const int i = (int)(r % B.n[0]);
        const long long r2 = r / B.n[0];
        const int j = (int)(r2 % B.n[1]), k = (int)(r2 / B.n[1]);
        const long long e = f * fs + node_index(B, i, j, k);
        d64[e] = src[t];
        if (d32) d32[e] = (float)src[t];
    }
}

template <class T>
__global__ void k_pack(const T* __restrict__ src, long long fs, DevBlock B, int nf, double* __restrict__ dst) {
    const long long N = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nf;
         t += (long long)gridDim.x * blockDim.x) {
        const long long f = t / N, r = t - f * N;
        const int i = (int)(r % B.n[0]);
        const long long r2 = r / B.n[0];
        const int j = (int)(r2 % B.n[1]), k = (int)(r2 / B.n[1]);
        dst[t] = (double)src[f * fs + node_index(B, i, j, k)];
    }
}

// Fills fields [f0, f0 + nf) of an arena with per-field values v[f].
template <class T>
__global__ void k_fill_fields(T* p, long long fs, int nf, const double* __restrict__ v) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < fs * nf;
         t += (long long)gridDim.x * blockDim.x)
        p[t] = (T)v[t / fs];
}

template <class T>
__global__ void k_fill(T* p, long long n, T v) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        p[t] = v;
}

__global__ void k_cast(const double* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

// ---------------------------------------------------------------- far field
// State on a far-field node from the interior state qi (node next to the
// boundary) and the outward unit normal n: 1D Riemann invariants along n,
// outgoing R+ = u_n + 2c/(gamma-1) from the interior, incoming
// R- = u_n - 2c/(gamma-1) from the free stream (rho = 1, u = (Ma, 0, 0),
// p = 1/gamma, c = 1); entropy and tangential velocity from the upwind side.
template <class R>
__device__ void farfield_state(const GasR<R>& gs, R mach, const R qi[5], R nx, R ny, R nz, R qb[5]) {
    const R g = gs.gamma, gm1 = gs.gm1;
    const R irho = R(1) / qi[0];
    const R u = qi[1] * irho, v = qi[2] * irho, w = qi[3] * irho;
    const R p = gm1 * (qi[4] - R(0.5) * qi[0] * (u * u + v * v + w * w));
    const R c = hsqrt(g * p * irho);
    const R uni = nx * u + ny * v + nz * w;
    const R unf = nx * mach;
    R Rp = uni + R(2) * c / gm1;
    R Rm = unf - R(2) / gm1;
    if (unf <= R(-1)) Rp = unf + R(2) / gm1;
    if (uni >= c) Rm = uni - R(2) * c / gm1;
    const R un = R(0.5) * (Rp + Rm);
    const R cb = R(0.25) * gm1 * (Rp - Rm);
    R ent, tx, ty, tz;
    if (un > R(0)) {
        ent = p / pow(qi[0], g);
        tx = u - uni * nx;
        ty = v - uni * ny;
        tz = w - uni * nz;
    } else {
        ent = (R(1) / g) / pow(R(1), g);
        tx = mach - unf * nx;
        ty = -unf * ny;
        tz = -unf * nz;
    }
    const R rho = pow(cb * cb / (g * ent), R(1) / gm1);
    const R pb = rho * cb * cb / g;
    const R ub = tx + un * nx, vb = ty + un * ny, wb = tz + un * nz;
    qb[0] = rho;
    qb[1] = rho * ub;
    qb[2] = rho * vb;
    qb[3] = rho * wb;
    qb[4] = pb / gm1 + R(0.5) * rho * (ub * ub + vb * vb + wb * wb);
}

// ---------------------------------------------------------------- halo
// Far-field faces after an RK stage: the boundary node gets the state of
// the 1D characteristic rule from the updated node next to it (FP64), and
// its FP32 copy in the mixed form.  Wall nodes are handled in the sweep.
__global__ void k_bc_farfield(const NodeItem* __restrict__ items, int n, const DevBlock* __restrict__ blocks,
                              double* Q, float* Qf, float* primf, const double* __restrict__ met, long long fs,
                              Gas gas) {
    GasR<double> gs;
    gs.init(gas);
    GasR<float> gsf;
    gsf.init(gas);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const NodeItem it = items[t];
        const DevBlock& B = blocks[it.b];
        const int d = it.dir, side = it.side;
        int in[3] = {it.i, it.j, it.k};
        in[d] += side ? -1 : 1;
        const long long e = node_index(B, it.i, it.j, it.k), ei = node_index(B, in[0], in[1], in[2]);
        double m[3], qi[5], qb[5];
        for (int c = 0; c < 3; ++c) m[c] = met[(3 * d + c) * fs + e];
        const double im = (side ? 1.0 : -1.0) / sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        for (int c = 0; c < 5; ++c) qi[c] = Q[c * fs + ei];
        farfield_state(gs, gas.mach, qi, m[0] * im, m[1] * im, m[2] * im, qb);
        float qf[5];
        for (int c = 0; c < 5; ++c) {
            Q[c * fs + e] = qb[c];
            qf[c] = (float)qb[c];
            if (Qf) Qf[c * fs + e] = qf[c];
        }
        if (Qf && primf) {   // the node's FP32 primitives, when the next stage's prep skips the interior
            float pv[4];
            primitives(gsf, qf, pv);
            for (int c = 0; c < 4; ++c) primf[c * fs + e] = pv[c];
        }
    }
}

// Start of a stage: the ghost nodes of the stencil state and, for
// Navier-Stokes, the primitives of every node the stress tensor reads, in
// one pass over the bricks of the interior and of the six ghost slabs.  A
// ghost takes the node of the joined block (periodic / interface), the
// mirrored node (wall: rho, p even, velocity odd) or the far-field state of
// the node next to the boundary; its primitives follow from its state.
// The FP64 form also stores each node's basis state (NodeState), which its
// three sweeps read instead of forming it each.
// Register targets: FP32 eight CTAs of 256 threads per SM (32 registers;
// 0.039 -> 0.0375 ms at 128^3), FP64 the compiler's default.
template <class R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 8 : 0)
k_prep(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, R* Q, long long fs,
       const R* __restrict__ met, R* prim, R* nst, Gas gas) {
    GasR<R> gs;
    gs.init(gas);
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const DevBlock& B = blocks[br.b];
        const int id[3] = {i, j, k};
        int d = -1;
        for (int a = 0; a < 3; ++a)
            if (id[a] < 0 || id[a] >= B.n[a]) d = a;
        const long long e = node_index(B, i, j, k);
        R q[5];
        bool need_prim = prim != nullptr;
        if (d < 0) {
            for (int c = 0; c < 5; ++c) q[c] = Q[c * fs + e];
        } else {
            const int side = id[d] < 0 ? 0 : 1, f = 2 * d + side;
            int src[3] = {i, j, k};
            if (B.nbr[f] >= 0) {   // periodic / interface: the joined block's node
                const DevBlock& N = blocks[B.nbr[f]];
                across_face(B, N.n, f, id, src);
                const long long es = node_index(N, src[0], src[1], src[2]);
                for (int c = 0; c < 5; ++c) q[c] = Q[c * fs + es];
            } else if ((B.wall >> f) & 1) {   // wall mirror through the boundary node
                src[d] = side ? 2 * (B.n[d] - 1) - id[d] : -id[d];
                const long long es = node_index(B, src[0], src[1], src[2]);
                for (int c = 0; c < 5; ++c) q[c] = Q[c * fs + es];
                q[1] = -q[1];
                q[2] = -q[2];
                q[3] = -q[3];
                need_prim = false;   // physical faces use one-sided viscous derivatives
            } else {   // far field from the node next to the boundary node
                int bn[3] = {i, j, k};
                bn[d] = side ? B.n[d] - 1 : 0;
                src[d] = side ? B.n[d] - 2 : 1;
                const long long es = node_index(B, src[0], src[1], src[2]);
                const long long eb = node_index(B, bn[0], bn[1], bn[2]);
                R m[3], qi[5];
                for (int c = 0; c < 3; ++c) m[c] = met[(3 * d + c) * fs + eb];
                const R im = (side ? R(1) : R(-1)) / hsqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                for (int c = 0; c < 5; ++c) qi[c] = Q[c * fs + es];
                farfield_state(gs, R(gas.mach), qi, m[0] * im, m[1] * im, m[2] * im, q);
                need_prim = false;
            }
            for (int c = 0; c < 5; ++c) Q[c * fs + e] = q[c];
        }
        if constexpr (sizeof(R) == 8) {
            if (nst) {   // every node a sweep visits, physical-face ghosts included
                NodeState<R> ns;
                const R c2 = node_state(gs, q, ns);
                const R v[NodeState<R>::NF] = {ns.irho, ns.u, ns.v, ns.w, ns.half_uu, ns.p,
                                               ns.c, ns.a0, ns.g, ns.cir, ns.al, ns.H};
#pragma unroll
                for (int c = 0; c < NodeState<R>::NF; ++c) nst[c * fs + e] = v[c];
                if (need_prim) {   // (u, v, w, T = c^2) from the same evaluation
                    const R pv[4] = {ns.u, ns.v, ns.w, c2};
#pragma unroll
                    for (int c = 0; c < 4; ++c) prim[c * fs + e] = pv[c];
                }
                continue;
            }
        }
        if (need_prim) {
            R pv[4];
            primitives(gs, q, pv);
            for (int c = 0; c < 4; ++c) prim[c * fs + e] = pv[c];
        }
    }
}

// Node coordinates: translated copy from the joined face, or point
// reflection through the boundary node on physical faces.
__global__ void k_halo_coords(const HaloItem* __restrict__ items, int n, double* X, long long fs,
                              const double* __restrict__ tr) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const HaloItem h = items[t];
        const int kind = h.mode & 15;
        if (kind == HM_TRANSLATE) {
            const int id = h.mode >> 8;
            for (int c = 0; c < 3; ++c) X[c * fs + h.dst] = X[c * fs + h.src] + tr[3 * id + c];
        } else {
            for (int c = 0; c < 3; ++c) X[c * fs + h.dst] = 2.0 * X[c * fs + h.aux] - X[c * fs + h.src];
        }
    }
}

// ---------------------------------------------------------------- metrics
struct CoordView {
    const double* X;
    long long fs;
    DevBlock B;
    __device__ __forceinline__ double x(int c, int i, int j, int k) const {
        return X[c * fs + node_index(B, i, j, k)];
    }
    // sixth-order derivative of coordinate c along axis a at (i, j, k)
    __device__ __forceinline__ double dx(int c, int a, int i, int j, int k) const {
        const long long st = a == 0 ? 1 : (a == 1 ? B.sj : B.sk);
        const long long e = node_index(B, i, j, k);
        const double* p = X + c * fs;
        auto f = [&](int s) { return p[hx_chk(B, e + s * st)]; };
        return d6<double>(f(-3), f(-2), f(-1), f(1), f(2), f(3));
    }
    // outer derivative along ao of (d x_ci / d a_in) * x_cm
    __device__ __forceinline__ double prod_d(int ci, int ain, int cm, int ao, int i, int j, int k) const {
        double f[7];
#pragma unroll
        for (int s = -3; s <= 3; ++s) {
            if (s == 0) continue;
            const int ii = i + (ao == 0 ? s : 0), jj = j + (ao == 1 ? s : 0), kk = k + (ao == 2 ? s : 0);
            f[s + 3] = dx(ci, ain, ii, jj, kk) * x(cm, ii, jj, kk);
        }
        return d6<double>(f[0], f[1], f[2], f[4], f[5], f[6]);
    }
};

// Eq. (7): the nine conservative metrics, and Eq. (8): J^-1, on every node
// of the bricks (interior and three ghost layers).
__global__ void __launch_bounds__(kThreads)
k_metrics(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ cblocks,
          const double* __restrict__ X, long long fsc, const DevBlock* __restrict__ blocks, double* met,
          long long fs, unsigned* flags) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const CoordView C{X, fsc, cblocks[br.b]};
        enum { XI = 0, ETA = 1, ZETA = 2, CX = 0, CY = 1, CZ = 2 };
        double m[10];
        m[0] = C.prod_d(CY, ETA, CZ, ZETA, i, j, k) - C.prod_d(CY, ZETA, CZ, ETA, i, j, k);
        m[1] = C.prod_d(CZ, ETA, CX, ZETA, i, j, k) - C.prod_d(CZ, ZETA, CX, ETA, i, j, k);
        m[2] = C.prod_d(CX, ETA, CY, ZETA, i, j, k) - C.prod_d(CX, ZETA, CY, ETA, i, j, k);
        m[3] = C.prod_d(CY, ZETA, CZ, XI, i, j, k) - C.prod_d(CY, XI, CZ, ZETA, i, j, k);
        m[4] = C.prod_d(CZ, ZETA, CX, XI, i, j, k) - C.prod_d(CZ, XI, CX, ZETA, i, j, k);
        m[5] = C.prod_d(CX, ZETA, CY, XI, i, j, k) - C.prod_d(CX, XI, CY, ZETA, i, j, k);
        m[6] = C.prod_d(CY, XI, CZ, ETA, i, j, k) - C.prod_d(CY, ETA, CZ, XI, i, j, k);
        m[7] = C.prod_d(CZ, XI, CX, ETA, i, j, k) - C.prod_d(CZ, ETA, CX, XI, i, j, k);
        m[8] = C.prod_d(CX, XI, CY, ETA, i, j, k) - C.prod_d(CX, ETA, CY, XI, i, j, k);
        const double xx = C.dx(CX, XI, i, j, k), xe = C.dx(CX, ETA, i, j, k), xz = C.dx(CX, ZETA, i, j, k);
        const double yx = C.dx(CY, XI, i, j, k), ye = C.dx(CY, ETA, i, j, k), yz = C.dx(CY, ZETA, i, j, k);
        const double zx = C.dx(CZ, XI, i, j, k), ze = C.dx(CZ, ETA, i, j, k), zz = C.dx(CZ, ZETA, i, j, k);
        const double jinv =
            xx * ye * zz - xx * yz * ze + xe * yz * zx - xe * yx * zz + xz * yx * ze - xz * ye * zx;
        if (!(jinv > 0.0)) atomicOr(flags, (unsigned)FLAG_BAD_GRID);
        m[9] = 1.0 / jinv;
        const long long e = node_index(blocks[br.b], i, j, k);
        for (int c = 0; c < 10; ++c) met[c * fs + e] = m[c];
    }
}

// Unit normals of the sweeps (FP64 form; static grid data, formed once).
// For each direction d, on the lines of the interior: the node normal
// m_d/|m_d| at nodes -1..n (the nodes whose characteristic basis a sweep
// forms) and, for faces -1/2 .. n-1/2 (stored at the node below), the unit
// normal and norm of the sixth-order midpoint metric.  Fields 7d + 0..2:
// node normal; 7d + 3..5: face normal; 7d + 6: face |m|.  The formulas are
// the sweep kernel's own.
__global__ void __launch_bounds__(kThreads)
k_normals(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks,
          const double* __restrict__ met, long long fs, double* __restrict__ nrm) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const DevBlock& B = blocks[br.b];
        const int id[3] = {i, j, k};
        const long long e = node_index(B, i, j, k);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bool line = id[d] >= -1 && id[d] <= B.n[d];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (a != d && (id[a] < 0 || id[a] >= B.n[a])) line = false;
            if (!line) continue;
            const long long st = d == 0 ? 1 : (d == 1 ? B.sj : B.sk);
            const double* m = met + 3 * d * fs + e;   // e is checked; the stencil offsets below are too
            const double mx = m[0], my = m[fs], mz = m[2 * fs];
            const double imm = hrsqrt(mx * mx + my * my + mz * mz);
            double* o = nrm + 7 * d * fs + e;
            o[0] = mx * imm;
            o[fs] = my * imm;
            o[2 * fs] = mz * imm;
            if (id[d] <= B.n[d] - 1) {
                double mf[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double* q = met + (3 * d + c) * fs;
                    auto f = [&](int s) { return q[hx_chk(B, e + s * st)]; };
                    mf[c] = mid6<double>(f(-2), f(-1), f(0), f(1), f(2), f(3));
                }
                const double mm2 = mf[0] * mf[0] + mf[1] * mf[1] + mf[2] * mf[2];
                const double im = hrsqrt(mm2);
                o[3 * fs] = mf[0] * im;
                o[4 * fs] = mf[1] * im;
                o[5 * fs] = mf[2] * im;
                o[6 * fs] = mm2 * im;
            }
        }
    }
}

// Checking aid: NaN into every node of the bricks outside its block's
// interior (the ghost shell), for nf fields.
template <class T>
__global__ void __launch_bounds__(kThreads)
k_poison(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, T* p, long long fs, int nf) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const DevBlock& B = blocks[br.b];
        if (i >= 0 && i < B.n[0] && j >= 0 && j < B.n[1] && k >= 0 && k < B.n[2]) continue;
        const long long e = node_index(B, i, j, k);
        for (int f = 0; f < nf; ++f) p[f * fs + e] = T(NAN);
    }
}

// ---------------------------------------------------------------- primitives
template <class R>
__global__ void __launch_bounds__(kThreads)
k_prim(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, const R* __restrict__ Q,
       long long fs, R* __restrict__ prim, Gas gas) {
    GasR<R> gs;
    gs.init(gas);
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const long long e = node_index(blocks[br.b], i, j, k);
        R q[5], pv[4];
        for (int c = 0; c < 5; ++c) q[c] = Q[c * fs + e];
        primitives(gs, q, pv);
        for (int c = 0; c < 4; ++c) prim[c * fs + e] = pv[c];
    }
}

// Eq. (21): (u, v, w, T)_(x, y, z) = J * sum_d m^_d (.)_(xi_d), derivatives
// by the sixth-order operator or the physical-face closure.  STRESS: write
// the node stress tensor and work + heat-flux vector (9 fields) that every
// direction's viscous flux projects; otherwise the 12 gradients.
//
// Column tiles: a CTA owns a 32 x 8 (i, j) tile of a block and marches it
// along k over a segment of `nk` planes (the brick's extent along k).  Each
// thread keeps the primitives of its own column at k-3..k+3 in registers
// (the k derivative); each plane k is staged in shared memory with three
// halo nodes along i and j (the i and j derivatives; corners are never
// read).  A node's primitives are read about twice from global memory
// (own column once, halos of the neighbouring tiles) instead of 19 times.
// Register target: two CTAs per SM (128 registers).
constexpr int kColX = 32, kColY = 8;

template <class R, bool STRESS>
__global__ void __launch_bounds__(kThreads, 2)
k_grad(const Brick* __restrict__ cols, int nb, const DevBlock* __restrict__ blocks, const R* __restrict__ prim,
       const R* __restrict__ met, long long fs, R* __restrict__ out, GasR<R> gs) {
    __shared__ R sp[4][kColY + 6][kColX + 6];
    const int ti = threadIdx.x & 31, tj = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = cols[t];
        const DevBlock B = blocks[br.b];
        const int i = br.i0 + ti, j = br.j0 + tj;
        const bool own = ti < br.ni && tj < br.nj;
        bool lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = (B.phys >> (2 * a)) & 1;
            hi[a] = (B.phys >> (2 * a + 1)) & 1;
        }
        // this thread's halo node of each plane, if any: three nodes beyond
        // the tile along i (tile rows) or along j (tile columns)
        const int hxn = 6 * br.nj, hyn = 6 * br.ni;
        const int h = threadIdx.x;
        int hx_ = 0, hy_ = 0;
        const bool halo = h < hxn + hyn;
        if (h < hxn) {
            hy_ = h / 6;
            const int r = h - 6 * hy_;
            hx_ = r < 3 ? r - 3 : br.ni + r - 3;
        } else if (halo) {
            const int u = h - hxn;
            hx_ = u % br.ni;
            const int r = u / br.ni;
            hy_ = r < 3 ? r - 3 : br.nj + r - 3;
        }
        const long long hoff = hx_ + (long long)hy_ * B.sj - (long long)ti - (long long)tj * B.sj;
        // whether this column lies within G of a joined i or j face, and
        // whether the block has joined k faces: only such nodes push halo
        const bool near_ij = (B.nbr[0] >= 0 && i < G) || (B.nbr[1] >= 0 && i >= B.n[0] - G) ||
                             (B.nbr[2] >= 0 && j < G) || (B.nbr[3] >= 0 && j >= B.n[1] - G);
        const bool nbrk = B.nbr[4] >= 0 || B.nbr[5] >= 0;
        // loads of plane k issued one plane ahead (own column at k + 3, the
        // halo node and the metrics at k), so that they arrive while plane
        // k - 1 is computed
        R qv[7][4], nq[4], nh[4], nm[10];
        auto fetch = [&](int k) {
            const long long e = node_index(B, i, j, k);
            if (own) {
                const long long e3 = hx_chk(B, e + 3 * (long long)B.sk);
#pragma unroll
                for (int v = 0; v < 4; ++v) nq[v] = prim[v * fs + e3];
#pragma unroll
                for (int c = 0; c < 10; ++c) nm[c] = met[c * fs + e];
            }
            if (halo) {
                const long long eh = hx_chk(B, e + hoff);
#pragma unroll
                for (int v = 0; v < 4; ++v) nh[v] = prim[v * fs + eh];
            }
        };
        if (own) {   // own column at k0-3 .. k0+2 (slots 1..6; the loop shifts first)
#pragma unroll
            for (int s = 1; s < 7; ++s) {
                const long long e = node_index(B, i, j, br.k0 - 4 + s);
#pragma unroll
                for (int v = 0; v < 4; ++v) qv[s][v] = prim[v * fs + e];
            }
        }
        // FP32 loads a plane ahead; FP64, bound by its FP64 pipe, loads the
        // plane at the top of its step and keeps the registers for two CTAs
        constexpr bool AHEAD = sizeof(R) == 4;
        if (AHEAD) fetch(br.k0);
        for (int kk = 0; kk < br.nk; ++kk) {
            const int k = br.k0 + kk;
            if (!AHEAD) fetch(k);
            R m[10];
#pragma unroll
            for (int s = 0; s < 6; ++s)
#pragma unroll
                for (int v = 0; v < 4; ++v) qv[s][v] = qv[s + 1][v];
#pragma unroll
            for (int v = 0; v < 4; ++v) qv[6][v] = nq[v];
#pragma unroll
            for (int c = 0; c < 10; ++c) m[c] = nm[c];
            __syncthreads();   // the previous plane's readers are done
            if (own) {
#pragma unroll
                for (int v = 0; v < 4; ++v) sp[v][tj + 3][ti + 3] = qv[3][v];
            }
            if (halo) {
#pragma unroll
                for (int v = 0; v < 4; ++v) sp[v][hy_ + 3][hx_ + 3] = nh[v];
            }
            __syncthreads();
            if (AHEAD && kk + 1 < br.nk) fetch(k + 1);
            if (!own) continue;
            const long long e = node_index(B, i, j, k);
            R dc[4][3];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                auto fi = [&](int s) { return sp[v][tj + 3][ti + 3 + s]; };
                auto fj = [&](int s) { return sp[v][tj + 3 + s][ti + 3]; };
                auto fk = [&](int s) { return qv[3 + s][v]; };
                dc[v][0] = dline<R>(fi, i, B.n[0], lo[0], hi[0]);
                dc[v][1] = dline<R>(fj, j, B.n[1], lo[1], hi[1]);
                dc[v][2] = dline<R>(fk, k, B.n[2], lo[2], hi[2]);
            }
            const R J = m[9];
            R g[12];   // the gradients / J
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    g[v * 3 + c] = m[c] * dc[v][0] + m[3 + c] * dc[v][1] + m[6 + c] * dc[v][2];
            if (STRESS) {
                R S[9];
                stress(gs, qv[3][0], qv[3][1], qv[3][2], qv[3][3], g, J, S);
#pragma unroll
                for (int c = 0; c < 9; ++c) out[c * fs + e] = S[c];
                // the stress halo of the sweeps, from nodes within G of a joined face
                if (near_ij || (nbrk && (k < G || k >= B.n[2] - G))) {
                    const int id[3] = {i, j, k};
                    push_ghosts<R>(blocks, B, br.b, id, out, fs, 9, S, false);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) out[c * fs + e] = J * g[c];
            }
        }
    }
}

// The RK3 stage of the mixed form (Eq. (20)) as a streaming pass after the
// three sweeps: R = -J (A - A_ref) in FP32, the increment -cc dt J A in FP32
// (the precision A has) and its combination with Q^n and Q^(k) in FP64, the
// wall-node values, the FP32 copy of the output (rounded to nearest) and,
// for a stage whose output feeds the next, its FP32 primitives; the
// non-finite / non-physical flags.  The same arithmetic as the FP32 sweep's
// fused epilogue (k_flux with RK), which the FP64 form keeps: separated, the
// stage's FP64 work and its memory traffic overlap in a point-parallel
// kernel instead of trailing the stencil phases of the zeta sweep, and the
// format conversions run on the integer pipe (widen_f32, narrow_f64_rn), so
// that the FP64 unit does only the ten FMAs of the combination.
// Each thread owns two i-adjacent nodes of a 32 x 8 brick (an aligned
// 8-byte pair of every FP32 field, a 16-byte pair of every FP64 one), so the
// stage's loads and stores are vector accesses.
constexpr int kRkThreads = 128;

__global__ void __launch_bounds__(kRkThreads, 6)
k_rk_stage(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, const float* __restrict__ A,
           const float* __restrict__ metf, long long fs, GasR<float> gs, RKArgs rk) {
    const int ti = 2 * (threadIdx.x & 15), tj = threadIdx.x >> 4;
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        if (ti >= br.ni || tj >= br.nj) continue;
        const bool two = ti + 1 < br.ni;   // the pair's second node lies in the brick
        const int i = br.i0 + ti, j = br.j0 + tj, k = br.k0;
        const DevBlock& B = blocks[br.b];
        const long long e = node_index(B, i, j, k);   // even: i is even and rows start on 8-element boundaries
        float2 dv[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            dv[c] = *reinterpret_cast<const float2*>(A + c * fs + e);
            if (rk.Aref) {
                const float2 r = *reinterpret_cast<const float2*>(rk.Aref + c * fs + e);
                dv[c].x -= r.x;
                dv[c].y -= r.y;
            }
        }
        const float2 J = *reinterpret_cast<const float2*>(metf + 9 * fs + e);
        double qo[2][5];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const float fr = rk.ccf * narrow_f64_rn(rk.dtl ? rk.dtl[e + l] : B.dt) * (l ? J.y : J.x);
#pragma unroll
            for (int c = 0; c < 5; ++c) qo[l][c] = widen_f32(fr * (l ? dv[c].y : dv[c].x));
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const double2 qn = *reinterpret_cast<const double2*>(rk.Qn + c * fs + e);
            if (rk.cb != 0.0) {
                const double2 qk = *reinterpret_cast<const double2*>(rk.Qk + c * fs + e);
                qo[0][c] = fma(rk.ca, qn.x, fma(rk.cb, qk.x, qo[0][c]));
                qo[1][c] = fma(rk.ca, qn.y, fma(rk.cb, qk.y, qo[1][c]));
            } else {
                qo[0][c] = fma(rk.ca, qn.x, qo[0][c]);
                qo[1][c] = fma(rk.ca, qn.y, qo[1][c]);
            }
        }
        if (B.wall) {
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const int il = i + l;
                const bool on = ((B.wall & 1) && il == 0) || ((B.wall & 2) && il == B.n[0] - 1) ||
                                ((B.wall & 4) && j == 0) || ((B.wall & 8) && j == B.n[1] - 1) ||
                                ((B.wall & 16) && k == 0) || ((B.wall & 32) && k == B.n[2] - 1);
                if (on) {
                    double* q = qo[l];
                    const double pw = rk.gm1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
                    q[1] = q[2] = q[3] = 0.0;
                    q[4] = pw / rk.gm1;
                }
            }
        }
        float qv[2][5];
        bool bad = false, unphys = false;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (l == 1 && !two) break;
            bool b = false;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                b = b || nonfinite_bits(qo[l][c]);
                qv[l][c] = narrow_f64_rn(qo[l][c]);
            }
            const float* v = qv[l];
            unphys = unphys || (!b && !(v[0] > 0.0f && v[4] * v[0] - 0.5f * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) > 0.0f));
            bad = bad || b;
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            if (two) {
                *reinterpret_cast<double2*>(rk.Qout + c * fs + e) = make_double2(qo[0][c], qo[1][c]);
                *reinterpret_cast<float2*>(rk.Qfout + c * fs + e) = make_float2(qv[0][c], qv[1][c]);
            } else {
                rk.Qout[c * fs + e] = qo[0][c];
                rk.Qfout[c * fs + e] = qv[0][c];
            }
        }
        if (rk.primout) {   // the next stage's primitives, from the FP32 copy as in k_prep
            float pv[2][4];
            primitives(gs, qv[0], pv[0]);
            if (two) primitives(gs, qv[1], pv[1]);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (two)
                    *reinterpret_cast<float2*>(rk.primout + c * fs + e) = make_float2(pv[0][c], pv[1][c]);
                else
                    rk.primout[c * fs + e] = pv[0][c];
            }
        }
        if (unphys) atomicOr(rk.flags, (unsigned)FLAG_UNPHYSICAL);
        if (bad) atomicOr(rk.flags, (unsigned)FLAG_NONFINITE);
    }
}

// Residual R = -J A of one block, packed [5][nk][nj][ni].
template <class R>
__global__ void k_rhs_out(DevBlock B, const R* __restrict__ A, const float* __restrict__ Aref,
                          const double* __restrict__ met, long long fs, double* __restrict__ out) {
    const long long N = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * 5;
         t += (long long)gridDim.x * blockDim.x) {
        const long long f = t / N, r = t - f * N;
        const int i = (int)(r % B.n[0]);
        const long long r2 = r / B.n[0];
        const int j = (int)(r2 % B.n[1]), k = (int)(r2 / B.n[1]);
        const long long e = node_index(B, i, j, k);
        const R a = Aref ? A[f * fs + e] - (R)Aref[f * fs + e] : A[f * fs + e];
        out[t] = -met[9 * fs + e] * (double)a;
    }
}

// ---------------------------------------------------------------- CFL
// Per block: max over nodes of sum_d (|m_d . u| + c |m_d|) J, as the bits of
// a non-negative double (monotone under unsigned comparison).
__global__ void __launch_bounds__(kThreads)
k_dt(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, const double* __restrict__ Q,
     const double* __restrict__ met, long long fs, Gas gas, unsigned long long* bmax) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        double s = 0.0;
        if (ok) {
            const DevBlock B = blocks[br.b];
            const long long e = node_index(B, i, j, k);
            const double irho = 1.0 / Q[e];
            const double u = Q[fs + e] * irho, v = Q[2 * fs + e] * irho, w = Q[3 * fs + e] * irho;
            const double p = (gas.gamma - 1.0) * (Q[4 * fs + e] - 0.5 * Q[e] * (u * u + v * v + w * w));
            const double c = sqrt(gas.gamma * p * irho);
            const double J = met[9 * fs + e];
            for (int d = 0; d < 3; ++d) {
                const double mx = met[(3 * d) * fs + e], my = met[(3 * d + 1) * fs + e],
                             mz = met[(3 * d + 2) * fs + e];
                s += (fabs(mx * u + my * v + mz * w) + c * sqrt(mx * mx + my * my + mz * mz)) * J;
            }
        }
        unsigned long long bits = __double_as_longlong(s);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = other > bits ? other : bits;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&bmax[br.b], bits);
    }
}

// Local time step of every interior node (local time stepping): CFL over
// the node's convective spectral radius (as in k_dt) plus, for
// Navier-Stokes, the viscous one (Ma/Re) max(4/3, gamma/Pr) (mu/rho)
// sum_d (J |m_d|)^2; from the FP64 state, CFL read from device memory.
__global__ void __launch_bounds__(kThreads)
k_dt_local(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks,
           const double* __restrict__ Q, const double* __restrict__ met, long long fs, Gas gas,
           const double* __restrict__ cfl, double* __restrict__ dtl) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        if (!ok) continue;
        const DevBlock& B = blocks[br.b];
        const long long e = node_index(B, i, j, k);
        const double irho = 1.0 / Q[e];
        const double u = Q[fs + e] * irho, v = Q[2 * fs + e] * irho, w = Q[3 * fs + e] * irho;
        const double p = (gas.gamma - 1.0) * (Q[4 * fs + e] - 0.5 * Q[e] * (u * u + v * v + w * w));
        const double T = gas.gamma * p * irho;
        const double c = sqrt(T);
        const double J = met[9 * fs + e];
        double lam = 0.0, g2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double mx = met[(3 * d) * fs + e], my = met[(3 * d + 1) * fs + e], mz = met[(3 * d + 2) * fs + e];
            const double m2 = mx * mx + my * my + mz * mz;
            lam += (fabs(mx * u + my * v + mz * w) + c * sqrt(m2)) * J;
            g2 += J * J * m2;
        }
        if (gas.viscous) {
            const double mu = gas.mu_law == 0 ? 1.0 : T * sqrt(T) * (1.0 + gas.suth) / (T + gas.suth);
            lam += gas.mach / gas.re * fmax(gas.gamma / gas.pr, 4.0 / 3.0) * mu * irho * g2;
        }
        dtl[e] = cfl[0] / lam;
    }
}

// dt of every block from the per-block maxima of k_dt: cfl / max (global
// minimum when per_block == 0), written into the block table; the global dt
// is added to the simulated-time accumulator.
__global__ void k_setdt(DevBlock* blocks, int nb, const unsigned long long* __restrict__ bmax,
                        const double* __restrict__ cfl, int per_block, double* time_acc, unsigned* flags) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double gmax = 0.0;
    for (int b = 0; b < nb; ++b) gmax = fmax(gmax, __longlong_as_double((long long)bmax[b]));
    if (!(gmax > 0.0) || nonfinite_bits(gmax)) {
        atomicOr(flags, (unsigned)FLAG_NONFINITE);
        return;
    }
    for (int b = 0; b < nb; ++b) {
        const double m = per_block ? __longlong_as_double((long long)bmax[b]) : gmax;
        blocks[b].dt = cfl[0] / m;
    }
    time_acc[0] += cfl[0] / gmax;
}

// Sum over nodes of R^2 per conservative variable, R = -J (A - Aref),
// warp-reduced then accumulated in FP64.
template <class R>
__global__ void __launch_bounds__(kThreads)
k_residual(const Brick* __restrict__ bricks, int nb, const DevBlock* __restrict__ blocks, const R* __restrict__ A,
           const float* __restrict__ Aref, const double* __restrict__ met, long long fs, double* sums) {
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const Brick br = bricks[t];
        int i, j, k;
        bool ok;
        brick_node(br, i, j, k, ok);
        double r2[5] = {0, 0, 0, 0, 0};
        if (ok) {
            const long long e = node_index(blocks[br.b], i, j, k);
            const double J = met[9 * fs + e];
            for (int c = 0; c < 5; ++c) {
                const R a = Aref ? A[c * fs + e] - (R)Aref[c * fs + e] : A[c * fs + e];
                const double r = -J * (double)a;
                r2[c] = r * r;
            }
        }
        for (int c = 0; c < 5; ++c) {
            double v = r2[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&sums[c], v);
        }
    }
}

}  // namespace

// ====================================================================== launchers

cudaError_t launch_setdt(DevBlock* blocks, int nb, const unsigned long long* bmax, const double* cfl, int per_block,
                         double* time_acc, unsigned* flags, cudaStream_t s) {
    k_setdt<<<1, 32, 0, s>>>(blocks, nb, bmax, cfl, per_block, time_acc, flags);
    return cudaGetLastError();
}

cudaError_t launch_residual(const Brick* bricks, int nb, const DevBlock* blocks, const void* A, const float* Aref,
                            bool fp64, const double* met, long long fs, double* sums, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const int g = grid_for((long long)nb * kThreads);
    if (fp64)
        k_residual<double><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const double*)A, nullptr, met, fs, sums);
    else
        k_residual<float><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const float*)A, Aref, met, fs, sums);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const double* src, void* dst, bool fp64, long long fs, DevBlock B, int nf,
                          cudaStream_t s) {
    const long long n = (long long)B.n[0] * B.n[1] * B.n[2] * nf;
    if (fp64)
        k_unpack<double><<<grid_for(n), kThreads, 0, s>>>(src, (double*)dst, fs, B, nf);
    else
        k_unpack<float><<<grid_for(n), kThreads, 0, s>>>(src, (float*)dst, fs, B, nf);
    return cudaGetLastError();
}

cudaError_t launch_unpack2(const double* src, double* d64, float* d32, long long fs, DevBlock B, int nf,
                           cudaStream_t s) {
    const long long n = (long long)B.n[0] * B.n[1] * B.n[2] * nf;
    k_unpack2<<<grid_for(n), kThreads, 0, s>>>(src, d64, d32, fs, B, nf);
    return cudaGetLastError();
}

cudaError_t launch_pack(const void* src, bool fp64, long long fs, DevBlock B, int nf, double* dst,
                        cudaStream_t s) {
    const long long n = (long long)B.n[0] * B.n[1] * B.n[2] * nf;
    if (fp64)
        k_pack<double><<<grid_for(n), kThreads, 0, s>>>((const double*)src, fs, B, nf, dst);
    else
        k_pack<float><<<grid_for(n), kThreads, 0, s>>>((const float*)src, fs, B, nf, dst);
    return cudaGetLastError();
}

cudaError_t launch_fill(void* p, bool fp64, long long n, double v, cudaStream_t s) {
    if (fp64)
        k_fill<double><<<grid_for(n), kThreads, 0, s>>>((double*)p, n, v);
    else
        k_fill<float><<<grid_for(n), kThreads, 0, s>>>((float*)p, n, (float)v);
    return cudaGetLastError();
}

cudaError_t launch_fill_fields(void* p, bool fp64, long long fs, int nf, const double* v, cudaStream_t s) {
    if (fp64)
        k_fill_fields<double><<<grid_for(fs * nf), kThreads, 0, s>>>((double*)p, fs, nf, v);
    else
        k_fill_fields<float><<<grid_for(fs * nf), kThreads, 0, s>>>((float*)p, fs, nf, v);
    return cudaGetLastError();
}

cudaError_t launch_cast(const double* src, float* dst, long long n, cudaStream_t s) {
    k_cast<<<grid_for(n), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_halo_coords(const HaloItem* items, int n, double* X, long long fs, const double* tr,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_halo_coords<<<grid_for(n), kThreads, 0, s>>>(items, n, X, fs, tr);
    return cudaGetLastError();
}

cudaError_t launch_bc_farfield(const NodeItem* items, int n, const DevBlock* blocks, double* Q, float* Qf,
                               float* primf, const double* met, long long fs, Gas gas, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_bc_farfield<<<grid_for(n), kThreads, 0, s>>>(items, n, blocks, Q, Qf, primf, met, fs, gas);
    return cudaGetLastError();
}

cudaError_t launch_prep(const Brick* bricks, int nb, const DevBlock* blocks, void* Q, bool fp64, long long fs,
                        const void* met, void* prim, double* nst, Gas gas, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    if (nst && !fp64) return cudaErrorInvalidValue;
    const int g = grid_for((long long)nb * kThreads);
    if (fp64)
        k_prep<double><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (double*)Q, fs, (const double*)met, (double*)prim,
                                              nst, gas);
    else
        k_prep<float><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (float*)Q, fs, (const float*)met, (float*)prim,
                                             nullptr, gas);
    return cudaGetLastError();
}

cudaError_t launch_metrics(const Brick* bricks, int nb, const DevBlock* cblocks, const double* X, long long fsc,
                           const DevBlock* blocks, double* met, long long fs, unsigned* flags, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_metrics<<<grid_for((long long)nb * kThreads), kThreads, 0, s>>>(bricks, nb, cblocks, X, fsc, blocks, met, fs,
                                                                      flags);
    return cudaGetLastError();
}

cudaError_t launch_normals(const Brick* bricks, int nb, const DevBlock* blocks, const double* met, long long fs,
                           double* nrm, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_normals<<<grid_for((long long)nb * kThreads), kThreads, 0, s>>>(bricks, nb, blocks, met, fs, nrm);
    return cudaGetLastError();
}

cudaError_t launch_poison(const Brick* bricks, int nb, const DevBlock* blocks, void* p, bool fp64, long long fs,
                          int nf, cudaStream_t s) {
    if (nb <= 0 || !p) return cudaSuccess;
    const int g = grid_for((long long)nb * kThreads);
    if (fp64)
        k_poison<double><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (double*)p, fs, nf);
    else
        k_poison<float><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (float*)p, fs, nf);
    return cudaGetLastError();
}

cudaError_t launch_prim(const Brick* bricks, int nb, const DevBlock* blocks, const void* Q, bool fp64,
                        long long fs, void* prim, Gas gas, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const int g = grid_for((long long)nb * kThreads);
    if (fp64)
        k_prim<double><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const double*)Q, fs, (double*)prim, gas);
    else
        k_prim<float><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const float*)Q, fs, (float*)prim, gas);
    return cudaGetLastError();
}

cudaError_t launch_grad(const Brick* bricks, int nb, const DevBlock* blocks, const void* prim, const void* met,
                        bool fp64, long long fs, void* out, bool stress_mode, Gas gas, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    const int g = grid_for((long long)nb * kThreads);
    if (fp64) {
        GasR<double> gs;
        gs.init(gas);
        if (stress_mode)
            k_grad<double, true><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const double*)prim,
                                                         (const double*)met, fs, (double*)out, gs);
        else
            k_grad<double, false><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const double*)prim,
                                                          (const double*)met, fs, (double*)out, gs);
    } else {
        GasR<float> gs;
        gs.init(gas);
        if (stress_mode)
            k_grad<float, true><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const float*)prim, (const float*)met,
                                                        fs, (float*)out, gs);
        else
            k_grad<float, false><<<g, kThreads, 0, s>>>(bricks, nb, blocks, (const float*)prim, (const float*)met,
                                                         fs, (float*)out, gs);
    }
    return cudaGetLastError();
}

cudaError_t launch_rk_stage(const Brick* bricks, int nb, const DevBlock* blocks, const float* A, const float* metf,
                            long long fs, Gas gas, const RKArgs& rk, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    GasR<float> gs;
    gs.init(gas);
    k_rk_stage<<<grid_for((long long)nb * kRkThreads, kRkThreads), kRkThreads, 0, s>>>(bricks, nb, blocks, A, metf,
                                                                                          fs, gs, rk);
    return cudaGetLastError();
}

cudaError_t launch_dt_local(const Brick* bricks, int nb, const DevBlock* blocks, const double* Q, const double* met,
                            long long fs, Gas gas, const double* cfl, double* dtl, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_dt_local<<<grid_for((long long)nb * kThreads), kThreads, 0, s>>>(bricks, nb, blocks, Q, met, fs, gas, cfl, dtl);
    return cudaGetLastError();
}

cudaError_t launch_dt(const Brick* bricks, int nb, const DevBlock* blocks, const double* Q, const double* met,
                      long long fs, Gas gas, unsigned long long* bmax, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    k_dt<<<grid_for((long long)nb * kThreads), kThreads, 0, s>>>(bricks, nb, blocks, Q, met, fs, gas, bmax);
    return cudaGetLastError();
}

cudaError_t launch_rhs_out(DevBlock B, const void* A, const float* Aref, bool fp64, const double* met, long long fs,
                           double* out, cudaStream_t s) {
    const long long n = (long long)B.n[0] * B.n[1] * B.n[2] * 5;
    if (fp64)
        k_rhs_out<double><<<grid_for(n), kThreads, 0, s>>>(B, (const double*)A, nullptr, met, fs, out);
    else
        k_rhs_out<float><<<grid_for(n), kThreads, 0, s>>>(B, (const float*)A, Aref, met, fs, out);
    return cudaGetLastError();
}

}  // namespace hx
