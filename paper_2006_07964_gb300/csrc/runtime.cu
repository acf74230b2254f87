// runtime.cu -- host runtime behind the C ABI of include/hx.h: block table,
// buffer plan, halo and tile work lists, metrics set-up, CUDA-graph RK step,
// tile-shape autotuner, profiling and error handling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hx.h"
#include "kernels.h"

using namespace hx;

namespace {

thread_local std::string g_create_error;

struct HostFace {
    int kind = -1, nbr = -1, nbr_face = -1;
    int tf[3] = {1, 2, 3};     // index transform to the neighbour (identity: aligned blocks)
    double tr[3] = {0, 0, 0};
};

struct HostBlock {
    int n[3];
    std::vector<double> xyz;   // [3][nk][nj][ni], released after the metrics
    HostFace f[6];
    DevBlock dev{};            // state layout (3 ghost layers)
    DevBlock cdev{};           // coordinate layout (6 ghost layers)
    long long npts() const { return (long long)n[0] * n[1] * n[2]; }
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

enum Kind { K_PREP, K_GRAD, K_FLUX0, K_FLUX1, K_FLUX2, K_FLUX2RK, K_BC, K_RK, K_COUNT };
const char* kKindName[K_COUNT] = {"prep", "stress", "flux_xi", "flux_eta", "flux_zeta", "flux_zeta_rk",
                                  "bc_farfield", "rk_stage"};

// Process-wide autotune cache: (precision, dir, viscous, shape class) -> variant.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, long long, int, int>, int> g_tune;

}  // namespace

struct hx_ctx {
    hx_config cfg{};
    Gas gas{};
    int device = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<HostBlock> blocks;
    bool finalized = false, metrics_done = false;
    std::string err;

    long long fs = 0, fsc = 0;
    size_t bytes = 0;
    std::vector<void*> allocs;

    double *met = nullptr, *Qn = nullptr, *Qa = nullptr, *Qb = nullptr, *stage = nullptr;
    double* nrm = nullptr;     // FP64 form: unit normals of the sweeps (k_normals), 21 fields
    double* nst = nullptr;     // FP64 form: node state of the sweeps (k_prep), NodeState<double>::NF fields
    float *metf = nullptr;
    float* Aref = nullptr;   // mixed form: FP32 divergence of the rest state (pure rounding)
    float* Qf[3] = {nullptr, nullptr, nullptr};   // mixed form: FP32 copies of Qn, Qa, Qb
    void *A = nullptr, *prim = nullptr, *grad = nullptr;
    DevBlock* d_blocks = nullptr;
    Tile* d_tiles[3][kFluxVariants] = {};
    int ntiles[3][kFluxVariants] = {};
    Brick *d_int = nullptr, *d_prim = nullptr;
    int n_int = 0, n_prim = 0;
    Brick* d_col = nullptr;     // gradient / stress kernel: 32 x 8 (i, j) tiles over segments along k
    int n_col = 0;
    Brick* d_shell = nullptr;   // debug_poison: bricks over every block's padded box
    int n_shell = 0;
    NodeItem* d_bc = nullptr;       // far-field boundary nodes
    int n_bc = 0;
    Brick *d_ghost = nullptr, *d_prep = nullptr;   // ghost slabs; interior + ghost slabs
    int n_ghost = 0, n_prep = 0;
    unsigned* d_flags = nullptr;
    unsigned long long* d_bmax = nullptr;
    long long max_block_pts = 0;

    int variant[3] = {0, 0, 0};
    int grid[3] = {1, 1, 1};
    int grid_rk = 1;   // zeta sweep with the fused RK stage (FP64 form)
    int grid_z = 1;    // zeta sweep of a mixed-form stage (tuned as such)
    double tune_ms[3][kFluxVariants] = {{-1, -1, -1}, {-1, -1, -1}, {-1, -1, -1}};
    bool tuned = false;

    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec_cfl[2] = {nullptr, nullptr};   // step with on-device dt: global / per block
    cudaGraphExec_t gexec_lts = nullptr;   // step with local time stepping
    double* dtl = nullptr;                 // local time step of every node (allocated on first use)
    double* d_scal = nullptr;   // [0] cfl, [1] simulated-time accumulator, [2..6] residual sums
    std::vector<double> dt_dev;   // dt currently in the device block table
    int launches_per_step = 0;

    bool fp64() const { return cfg.precision == HX_FP64; }
    size_t rsize() const { return fp64() ? 8 : 4; }
};

namespace {

int fail(hx_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(hx_ctx* c, cudaError_t e, const char* where) {
    return fail(c, HX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HX_CK(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);      \
    } while (0)

int dalloc(hx_ctx* ctx, void** p, size_t bytes) {
    if (ctx->cfg.mem_cap_bytes && ctx->bytes + bytes > ctx->cfg.mem_cap_bytes)
        return fail(ctx, HX_ERR_OOM, "device memory cap exceeded");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, HX_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->bytes += bytes;
    ctx->allocs.push_back(*p);
    return HX_OK;
}

template <class T>
int upload(hx_ctx* ctx, T** dptr, const std::vector<T>& v) {
    int rc = dalloc(ctx, (void**)dptr, v.size() * sizeof(T));
    if (rc) return rc;
    if (!v.empty()) HX_CK(cudaMemcpyAsync(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return HX_OK;
}

void dfree(hx_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    ctx->allocs.erase(std::remove(ctx->allocs.begin(), ctx->allocs.end(), p), ctx->allocs.end());
    ctx->bytes -= bytes;
}

bool is_phys(int kind) { return kind == HX_FACE_WALL || kind == HX_FACE_FARFIELD; }

// Index of node (t[0], t[1], t[2]) in a layout.
long long nidx(const DevBlock& B, const int t[3]) { return node_index(B, t[0], t[1], t[2]); }

// Bricks (32 x 8 x 1) covering the box [lo, hi) of block b.
void add_bricks(std::vector<Brick>& out, int b, const int lo[3], const int hi[3]) {
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; j += 8)
            for (int i = lo[0]; i < hi[0]; i += 32)
                out.push_back(Brick{b, i, j, k, std::min(32, hi[0] - i), std::min(8, hi[1] - j), 1, 0});
}

// Coordinate ghost items of pass m: the ghost nodes (within GC of the
// block) that lie outside it in exactly m directions.  Each resolves its
// highest out-of-range direction d: across a periodic or interface face it
// copies the neighbour's node (plus the face translation), which lies
// outside the neighbour in m-1 directions; on a physical face it reflects
// through the boundary node (m-1 again).  Pass m therefore reads only what
// passes < m wrote, and edges and corners resolve k first, then j, then i.
void coord_halo_items(const hx_ctx* ctx, int m, std::vector<HaloItem>& out) {
    for (int b = 0; b < (int)ctx->blocks.size(); ++b) {
        const HostBlock& H = ctx->blocks[b];
        auto in = [&](int a, int x) { return x >= 0 && x < H.n[a]; };
        for (int k = -GC; k < H.n[2] + GC; ++k)
            for (int j = -GC; j < H.n[1] + GC; ++j) {
                const int cjk = !in(1, j) + !in(2, k);
                if (cjk > m || cjk < m - 1) continue;
                for (int i = -GC; i < H.n[0] + GC; ++i) {
                    if (cjk == m && !in(0, i)) continue;
                    if (cjk == m - 1 && in(0, i)) {
                        i = H.n[0] - 1;   // skip the interior run
                        continue;
                    }
                    const int g[3] = {i, j, k};
                    int d = 2;
                    while (in(d, g[d])) --d;
                    const int side = g[d] < 0 ? 0 : 1, f = 2 * d + side;
                    const HostFace& F = H.f[f];
                    HaloItem it{};
                    it.dst = (int)nidx(H.cdev, g);
                    if (!is_phys(F.kind)) {
                        const HostBlock& N = ctx->blocks[F.nbr];
                        int src[3];
                        across_face(H.dev, N.n, f, g, src);
                        it.src = (int)nidx(N.cdev, src);
                        it.mode = HM_TRANSLATE | ((b * 6 + f) << 8);
                    } else {
                        const int bnd = side ? H.n[d] - 1 : 0;
                        int bn[3] = {i, j, k}, src[3] = {i, j, k};
                        bn[d] = bnd;
                        src[d] = 2 * bnd - g[d];
                        it.src = (int)nidx(H.cdev, src);
                        it.aux = (int)nidx(H.cdev, bn);
                        it.mode = HM_REFLECT;
                    }
                    out.push_back(it);
                }
            }
    }
}

// Line groups of the sweep kernel of direction d: NA adjacent lines each,
// origin at sweep index 0 (the kernel marches the whole line).
void make_tiles(const hx_ctx* ctx, int d, FluxShape sh, std::vector<Tile>& out) {
    for (int b = 0; b < (int)ctx->blocks.size(); ++b) {
        const HostBlock& H = ctx->blocks[b];
        const int ni = H.n[0], nj = H.n[1], nk = H.n[2];
        if (d == 0) {
            for (int k = 0; k < nk; ++k)
                for (int j = 0; j < nj; j += sh.na) out.push_back(Tile{b, 0, j, k});
        } else if (d == 1) {
            for (int k = 0; k < nk; ++k)
                for (int i = 0; i < ni; i += sh.na) out.push_back(Tile{b, i, 0, k});
        } else {
            for (int j = 0; j < nj; ++j)
                for (int i = 0; i < ni; i += sh.na) out.push_back(Tile{b, i, j, 0});
        }
    }
}

// State the stencil kernels read in stage buffer slot `slot` (0 = Q^n,
// 1 = Q^(1), 2 = Q^(2)): the FP64 buffer itself, or its FP32 copy.
void* stencil_state(const hx_ctx* ctx, int slot) {
    double* q64[3] = {ctx->Qn, ctx->Qa, ctx->Qb};
    return ctx->fp64() ? (void*)q64[slot] : (void*)ctx->Qf[slot];
}
const void* stencil_met(const hx_ctx* ctx) { return ctx->fp64() ? (const void*)ctx->met : (const void*)ctx->metf; }

// Per-launch event timing (hx_profile_step).
struct Prof {
    bool on = false;
    cudaStream_t s = nullptr;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    int cur = -1;
    cudaEvent_t start_ev = nullptr;
    void begin(int kind) {
        if (!on) return;
        nvtxRangePushA(kKindName[kind]);
        Rec r{kind, nullptr, nullptr};
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end() {
        if (!on) return;
        cudaEventRecord(recs.back().b, s);
        nvtxRangePop();
    }
};

// NVTX range over an entry point (visible to nsys / ncu range filters).
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

// The residual of one stage from stage slot `in`: the ghosts of the
// stencil state and the primitives (prep), the node stress tensor (pushing
// its halo), then the three flux sweeps.  rk == null: A holds the
// accumulated divergence.  With rk, the zeta sweep finishes R = -J A and
// the RK3 stage into rk->Qout.
// prim_interior = false: the primitives of the interior nodes are already
// in place (the previous stage's epilogue wrote them), and the prep fills
// the ghosts only.
int enqueue_rhs(hx_ctx* ctx, int in, const RKArgs* rk, Prof* pf, bool prep = true, bool prim_interior = true) {
    cudaStream_t s = ctx->stream;
    const bool f64 = ctx->fp64();
    const bool visc = ctx->cfg.viscous != 0;
    void* Qs = stencil_state(ctx, in);
    const void* M = stencil_met(ctx);
    if (prep && ctx->cfg.debug_poison) {   // checking aid: every ghost NaN before the halo fill
        HX_CK(launch_poison(ctx->d_shell, ctx->n_shell, ctx->d_blocks, Qs, f64, ctx->fs, 5, s));
        HX_CK(launch_poison(ctx->d_shell, ctx->n_shell, ctx->d_blocks, ctx->A, f64, ctx->fs, 5, s));
        if (visc) {
            HX_CK(launch_poison(ctx->d_shell, ctx->n_shell, ctx->d_blocks, ctx->prim, f64, ctx->fs, 4, s));
            HX_CK(launch_poison(ctx->d_shell, ctx->n_shell, ctx->d_blocks, ctx->grad, f64, ctx->fs, 12, s));
        }
        if (f64)
            HX_CK(launch_poison(ctx->d_shell, ctx->n_shell, ctx->d_blocks, ctx->nst, true, ctx->fs,
                                NodeState<double>::NF, s));
    }
    if (prep) {
        if (pf) pf->begin(K_PREP);
        // the FP64 form's node state covers the interior and the ghosts
        double* nst = f64 ? ctx->nst : nullptr;
        if (visc && prim_interior)
            HX_CK(launch_prep(ctx->d_prep, ctx->n_prep, ctx->d_blocks, Qs, f64, ctx->fs, M, ctx->prim, nst, ctx->gas,
                              s));
        else if (visc)
            HX_CK(launch_prep(ctx->d_ghost, ctx->n_ghost, ctx->d_blocks, Qs, f64, ctx->fs, M, ctx->prim, nullptr,
                              ctx->gas, s));
        else if (nst)
            HX_CK(launch_prep(ctx->d_prep, ctx->n_prep, ctx->d_blocks, Qs, f64, ctx->fs, M, nullptr, nst, ctx->gas, s));
        else
            HX_CK(launch_prep(ctx->d_ghost, ctx->n_ghost, ctx->d_blocks, Qs, f64, ctx->fs, M, nullptr, nullptr,
                              ctx->gas, s));
        if (pf) pf->end();
    }
    if (visc) {
        if (pf) pf->begin(K_GRAD);
        HX_CK(launch_grad(ctx->d_col, ctx->n_col, ctx->d_blocks, ctx->prim, M, f64, ctx->fs, ctx->grad, true,
                          ctx->gas, s));
        if (pf) pf->end();
    }
    for (int d = 0; d < 3; ++d) {
        const int v = ctx->variant[d];
        FluxArgs a{};
        a.blocks = ctx->d_blocks;
        a.tiles = ctx->d_tiles[d][v];
        a.ntiles = ctx->ntiles[d][v];
        a.Q = Qs;
        a.met = M;
        a.nrm = ctx->nrm;
        a.nst = ctx->nst;
        a.fs = ctx->fs;
        a.stress = ctx->grad;
        a.A = ctx->A;
        a.accumulate = d > 0;
        a.gas = ctx->gas;
        a.grid = ctx->grid[d];
        a.scheme = ctx->cfg.scheme;
        // FP64: the zeta sweep finishes the stage; mixed: a streaming
        // kernel does, after the three sweeps (k_rk_stage)
        const bool fuse = d == 2 && rk && f64;
        if (d == 2 && rk && !f64) a.grid = ctx->grid_z;
        if (fuse) {
            a.fuse_rk = 1;
            a.rk = *rk;
            a.grid = ctx->grid_rk;
        }
        if (pf) pf->begin(fuse ? K_FLUX2RK : K_FLUX0 + d);
        HX_CK(launch_flux(f64, d, v, visc, a, s));
        if (pf) pf->end();
    }
    if (rk && !f64) {
        if (pf) pf->begin(K_RK);
        HX_CK(launch_rk_stage(ctx->d_int, ctx->n_int, ctx->d_blocks, (const float*)ctx->A, (const float*)M, ctx->fs,
                              ctx->gas, *rk, s));
        if (pf) pf->end();
    }
    return HX_OK;
}

int enqueue_step(hx_ctx* ctx, Prof* pf, const double* dtl = nullptr) {
    static const double co[3][3] = {{1.0, 0.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
    static const int in_slot[3] = {0, 1, 2}, out_slot[3] = {1, 2, 0};
    double* q64[3] = {ctx->Qn, ctx->Qa, ctx->Qb};
    cudaStream_t s = ctx->stream;
    // Mixed Navier-Stokes: stages 1 and 2 write the primitives of their
    // output in their epilogue, and stages 2 and 3 skip the interior prep.
    const bool fuse_prim = !ctx->fp64() && ctx->cfg.viscous != 0;
    for (int st = 0; st < 3; ++st) {
        RKArgs rk{};
        rk.Qn = ctx->Qn;
        rk.Qk = q64[in_slot[st]];
        rk.metd = ctx->met;
        rk.Qout = q64[out_slot[st]];
        rk.Qfout = ctx->fp64() ? nullptr : ctx->Qf[out_slot[st]];
        rk.Aref = ctx->Aref;
        rk.dtl = dtl;
        rk.ca = co[st][0];
        rk.cb = co[st][1];
        rk.cc = co[st][2];
        rk.ccf = (float)-co[st][2];
        rk.gm1 = ctx->gas.gamma - 1.0;
        rk.flags = ctx->d_flags;
        rk.primout = fuse_prim && st < 2 ? (float*)ctx->prim : nullptr;
        int rc = enqueue_rhs(ctx, in_slot[st], &rk, pf, true, !(fuse_prim && st > 0));
        if (rc) return rc;
        if (ctx->n_bc) {
            if (pf) pf->begin(K_BC);
            HX_CK(launch_bc_farfield(ctx->d_bc, ctx->n_bc, ctx->d_blocks, rk.Qout, rk.Qfout, rk.primout, ctx->met,
                                     ctx->fs, ctx->gas, s));
            if (pf) pf->end();
        }
    }
    return HX_OK;
}

int set_device(hx_ctx* ctx) {
    HX_CK(cudaSetDevice(ctx->device));
    return HX_OK;
}

int upload_dt(hx_ctx* ctx, const std::vector<double>& dt) {
    if (dt == ctx->dt_dev) return HX_OK;
    for (size_t b = 0; b < ctx->blocks.size(); ++b) ctx->blocks[b].dev.dt = dt[b];
    std::vector<DevBlock> tab;
    for (auto& H : ctx->blocks) tab.push_back(H.dev);
    HX_CK(cudaMemcpyAsync(ctx->d_blocks, tab.data(), tab.size() * sizeof(DevBlock), cudaMemcpyHostToDevice,
                          ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    ctx->dt_dev = dt;
    return HX_OK;
}

// Times the tile-shape variants of each flux direction once per shape class
// and keeps the fastest (process-wide cache).
int autotune(hx_ctx* ctx) {
    if (ctx->tuned) return HX_OK;
    const bool f64 = ctx->fp64(), visc = ctx->cfg.viscous != 0;
    long long tot = 0;
    int nmin[3] = {1 << 30, 1 << 30, 1 << 30};
    for (auto& H : ctx->blocks) {
        tot += H.npts();
        for (int d = 0; d < 3; ++d) nmin[d] = std::min(nmin[d], H.n[d]);
    }
    long long cls = 1;
    while (cls < tot) cls <<= 1;
    if (f64 && ctx->cfg.autotune)   // the node state of the state the FP64 sweeps are timed on
        HX_CK(launch_prep(ctx->d_prep, ctx->n_prep, ctx->d_blocks, stencil_state(ctx, 0), true, ctx->fs,
                          stencil_met(ctx), visc ? ctx->prim : nullptr, ctx->nst, ctx->gas, ctx->stream));
    for (int d = 0; d < 3; ++d) {
        auto key = std::make_tuple((int)f64 + 2 * ctx->cfg.scheme, d, (int)visc, cls, nmin[d], (int)ctx->blocks.size());
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                ctx->variant[d] = it->second;
                continue;
            }
        }
        int best = -1;
        float best_ms = 1e30f;
        if (ctx->cfg.autotune) {
            cudaEvent_t e0, e1;
            HX_CK(cudaEventCreate(&e0));
            HX_CK(cudaEventCreate(&e1));
            // zeta: the FP64 form's steps run the sweep with the fused RK
            // stage, so that is the one timed (stage-2 coefficients, output
            // into the stage buffer Q^(2), which holds nothing between steps);
            // the mixed form's zeta sweep accumulates like eta
            const bool rk = d == 2 && f64;
            for (int v = 0; v < kFluxVariants; ++v) {
                const int cps = flux_ctas_per_sm(f64, d, v, visc, rk, ctx->cfg.scheme);
                if (cps <= 0) continue;
                FluxArgs a{};
                a.blocks = ctx->d_blocks;
                a.tiles = ctx->d_tiles[d][v];
                a.ntiles = ctx->ntiles[d][v];
                a.Q = stencil_state(ctx, 0);
                a.met = stencil_met(ctx);
                a.nrm = ctx->nrm;
                a.nst = ctx->nst;
                a.fs = ctx->fs;
                a.stress = ctx->grad;
                a.A = ctx->A;
                a.accumulate = d > 0;
                a.gas = ctx->gas;
                a.scheme = ctx->cfg.scheme;
                a.grid = (int)std::min<long long>(a.ntiles, (long long)cps * ctx->num_sms);
                if (rk) {
                    a.fuse_rk = 1;
                    a.rk.Qn = ctx->Qn;
                    a.rk.Qk = ctx->Qn;
                    a.rk.metd = ctx->met;
                    a.rk.Qout = ctx->Qb;
                    a.rk.Qfout = nullptr;
                    a.rk.Aref = ctx->Aref;
                    a.rk.ca = 0.75;
                    a.rk.cb = 0.25;
                    a.rk.cc = 0.25;
                    a.rk.ccf = -0.25f;
                    a.rk.gm1 = ctx->gas.gamma - 1.0;
                    a.rk.flags = ctx->d_flags;
                }
                HX_CK(launch_flux(f64, d, v, visc, a, ctx->stream));   // warm-up
                HX_CK(cudaEventRecord(e0, ctx->stream));
                const int reps = 3;
                for (int r = 0; r < reps; ++r) HX_CK(launch_flux(f64, d, v, visc, a, ctx->stream));
                HX_CK(cudaEventRecord(e1, ctx->stream));
                HX_CK(cudaEventSynchronize(e1));
                float ms = 0;
                HX_CK(cudaEventElapsedTime(&ms, e0, e1));
                ctx->tune_ms[d][v] = ms / reps;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = v;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
        } else {   // the 128-thread tile (16 x 8 along xi, 8 x 16 across), else the first that launches
            const int order[kFluxVariants] = {2, 0, 1};
            for (int o = 0; o < kFluxVariants && best < 0; ++o)
                if (flux_ctas_per_sm(f64, d, order[o], visc, false, ctx->cfg.scheme) > 0) best = order[o];
        }
        if (best < 0) return fail(ctx, HX_ERR_CUDA, "no flux kernel variant can launch on this device");
        ctx->variant[d] = best;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best;
    }
    for (int d = 0; d < 3; ++d) {
        const int cps = std::max(1, flux_ctas_per_sm(f64, d, ctx->variant[d], visc, false, ctx->cfg.scheme));
        ctx->grid[d] = (int)std::max<long long>(
            1, std::min<long long>(ctx->ntiles[d][ctx->variant[d]], (long long)cps * ctx->num_sms));
    }
    {   // the zeta sweep with the fused RK stage (attributes set here, before any capture)
        const int cps = flux_ctas_per_sm(f64, 2, ctx->variant[2], visc, true, ctx->cfg.scheme);
        if (cps <= 0) return fail(ctx, HX_ERR_CUDA, "the fused zeta sweep cannot launch on this device");
        ctx->grid_rk = (int)std::max<long long>(
            1, std::min<long long>(ctx->ntiles[2][ctx->variant[2]], (long long)cps * ctx->num_sms));
        ctx->grid_z = ctx->grid[2];
    }
    ctx->tuned = true;
    return HX_OK;
}

// One RK step whose dt comes from the state on the device: the CFL maxima
// (k_dt), dt into the block table (k_setdt), then the three stages.
int enqueue_cfl_step(hx_ctx* ctx, int per_block) {
    const int nb = (int)ctx->blocks.size();
    HX_CK(cudaMemsetAsync(ctx->d_bmax, 0, nb * sizeof(unsigned long long), ctx->stream));
    HX_CK(launch_dt(ctx->d_int, ctx->n_int, ctx->d_blocks, ctx->Qn, ctx->met, ctx->fs, ctx->gas, ctx->d_bmax,
                    ctx->stream));
    HX_CK(launch_setdt(ctx->d_blocks, nb, ctx->d_bmax, ctx->d_scal, per_block, ctx->d_scal + 1, ctx->d_flags,
                       ctx->stream));
    return enqueue_step(ctx, nullptr);
}

// One step of local time stepping: every node's time step from Q^n (CFL in
// d_scal[0]), then the three stages with it.
int enqueue_lts_step(hx_ctx* ctx) {
    HX_CK(launch_dt_local(ctx->d_int, ctx->n_int, ctx->d_blocks, ctx->Qn, ctx->met, ctx->fs, ctx->gas, ctx->d_scal,
                          ctx->dtl, ctx->stream));
    return enqueue_step(ctx, nullptr, ctx->dtl);
}

// cfl_mode < 0: fixed dt; 0 / 1: on-device global / per-block dt; 2: local time stepping.
int capture(hx_ctx* ctx, cudaGraphExec_t* out, int cfl_mode) {
    cudaGraph_t g = nullptr;
    HX_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = cfl_mode < 0 ? enqueue_step(ctx, nullptr) : cfl_mode == 2 ? enqueue_lts_step(ctx) : enqueue_cfl_step(ctx, cfl_mode);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    return HX_OK;
}

int ensure_graph(hx_ctx* ctx) {
    if (ctx->gexec) return HX_OK;
    cudaGraph_t g = nullptr;
    HX_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(ctx, nullptr);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->gexec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    return HX_OK;
}

int read_flags(hx_ctx* ctx) {
    unsigned flags = 0;
    HX_CK(cudaMemcpyAsync(&flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    if (flags & FLAG_BOUNDS) return fail(ctx, HX_ERR_BOUNDS, "a node offset outside its field (checking build)");
    if (flags & FLAG_NONFINITE) return fail(ctx, HX_ERR_NONFINITE, "non-finite state after a step");
    if (flags & FLAG_UNPHYSICAL) return fail(ctx, HX_ERR_UNPHYSICAL, "non-positive density or pressure after a step");
    return HX_OK;
}

// Mixed form only.  On a uniform state the discrete operator is exactly zero
// (the metric identity of Eq. (7) with the sixth-order operators), but its
// FP32 evaluation is not: the O(1) pressure flux times FP32-rounded metrics
// leaves a residual of ~1e-7 relative.  That residual is evaluated once, for
// the fluid at rest at free-stream density and pressure, with the same
// kernels and metrics (every ghost filled with the same state), and the
// stage subtracts it.
int compute_ref_residual(hx_ctx* ctx) {
    if (ctx->fp64()) return HX_OK;
    int rc = autotune(ctx);
    if (rc) return rc;
    const double g = ctx->gas.gamma;
    const double qref[5] = {1.0, 0.0, 0.0, 0.0, (1.0 / g) / (g - 1.0)};
    double* dq = nullptr;
    if ((rc = dalloc(ctx, (void**)&dq, sizeof qref))) return rc;
    HX_CK(cudaMemcpyAsync(dq, qref, sizeof qref, cudaMemcpyHostToDevice, ctx->stream));
    HX_CK(launch_fill_fields(ctx->Qf[0], false, ctx->fs, 5, dq, ctx->stream));
    if (ctx->cfg.viscous)
        HX_CK(launch_prim(ctx->d_prim, ctx->n_prim, ctx->d_blocks, ctx->Qf[0], false, ctx->fs, ctx->prim, ctx->gas,
                          ctx->stream));
    if ((rc = enqueue_rhs(ctx, 0, nullptr, nullptr, false))) return rc;
    HX_CK(cudaMemcpyAsync(ctx->Aref, ctx->A, 5 * (size_t)ctx->fs * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, dq, sizeof qref);
    return HX_OK;
}

int check_ready(hx_ctx* ctx) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (!ctx->finalized || !ctx->metrics_done) return fail(ctx, HX_ERR_STATE, "call hx_finalize and hx_compute_metrics first");
    return set_device(ctx);
}

int step_common(hx_ctx* ctx, int nsteps, const std::vector<double>& dt) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (nsteps < 0) return fail(ctx, HX_ERR_INVALID_ARG, "nsteps < 0");
    for (double v : dt)
        if (!(v > 0.0) || !std::isfinite(v)) return fail(ctx, HX_ERR_INVALID_ARG, "dt must be positive and finite");
    if ((rc = upload_dt(ctx, dt))) return rc;
    if ((rc = autotune(ctx))) return rc;
    if ((rc = ensure_graph(ctx))) return rc;
    HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    for (int i = 0; i < nsteps; ++i) HX_CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    return read_flags(ctx);
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

int hx_config_default(hx_config* cfg) {
    if (!cfg) return HX_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->gamma = 1.4;
    cfg->mach = 0.5;
    cfg->reynolds = 1.0;
    cfg->prandtl = 0.72;
    cfg->viscous = 0;
    cfg->mu_law = 1;
    cfg->sutherland_s = 110.4 / 288.15;
    cfg->precision = HX_FP64;
    cfg->scheme = 0;
    cfg->mem_cap_bytes = 0;
    cfg->autotune = 1;
    return HX_OK;
}

int hx_create(hx_ctx** out, const hx_config* cfg, void* cuda_stream) {
    if (!out || !cfg) {
        g_create_error = "null argument";
        return HX_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!(cfg->gamma > 1.0) || (cfg->viscous && (!(cfg->reynolds > 0) || !(cfg->prandtl > 0))) ||
        (cfg->precision != HX_FP64 && cfg->precision != HX_MIXED) || (cfg->scheme != 0 && cfg->scheme != 1) ||
        (cfg->mu_law != 0 && cfg->mu_law != 1)) {
        g_create_error = "invalid configuration (gamma > 1, Re, Pr > 0, precision, scheme 0/1, mu_law 0/1)";
        return HX_ERR_INVALID_ARG;
    }
    int dev = 0, ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return HX_ERR_CUDA;
    }
    cudaGetDevice(&dev);
    hx_ctx* ctx = new hx_ctx();
    ctx->cfg = *cfg;
    ctx->device = dev;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    ctx->gas = Gas{cfg->gamma, cfg->mach, cfg->reynolds, cfg->prandtl, cfg->sutherland_s, cfg->viscous, cfg->mu_law};
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            delete ctx;
            return HX_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return HX_OK;
}

int hx_add_block(hx_ctx* ctx, int ni, int nj, int nk, const double* xyz, int* block_id) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (ctx->finalized) return fail(ctx, HX_ERR_STATE, "hx_add_block after hx_finalize");
    if (!xyz || ni < 6 || nj < 6 || nk < 6) return fail(ctx, HX_ERR_INVALID_ARG, "block needs >= 6 nodes per direction");
    HostBlock H;
    H.n[0] = ni;
    H.n[1] = nj;
    H.n[2] = nk;
    H.xyz.assign(xyz, xyz + 3 * H.npts());
    ctx->blocks.push_back(std::move(H));
    if (block_id) *block_id = (int)ctx->blocks.size() - 1;
    return HX_OK;
}

int hx_set_face(hx_ctx* ctx, int block, int face, int kind, int nbr_block, int nbr_face, const double translate[3]) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (ctx->finalized) return fail(ctx, HX_ERR_STATE, "hx_set_face after hx_finalize");
    if (block < 0 || block >= (int)ctx->blocks.size() || face < 0 || face > 5 || kind < HX_FACE_PERIODIC ||
        kind > HX_FACE_FARFIELD)
        return fail(ctx, HX_ERR_INVALID_ARG, "bad block, face or kind");
    HostFace& F = ctx->blocks[block].f[face];
    F.kind = kind;
    F.nbr = nbr_block;
    F.nbr_face = nbr_face;
    for (int a = 0; a < 3; ++a) F.tf[a] = a + 1;
    for (int m = 0; m < 3; ++m) F.tr[m] = translate ? translate[m] : 0.0;
    return HX_OK;
}

int hx_set_face_transform(hx_ctx* ctx, int block, int face, const int transform[3]) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (ctx->finalized) return fail(ctx, HX_ERR_STATE, "hx_set_face_transform after hx_finalize");
    if (block < 0 || block >= (int)ctx->blocks.size() || face < 0 || face > 5 || !transform)
        return fail(ctx, HX_ERR_INVALID_ARG, "bad block, face or transform");
    for (int a = 0; a < 3; ++a)
        if (transform[a] == 0 || transform[a] < -3 || transform[a] > 3)
            return fail(ctx, HX_ERR_INVALID_ARG, "transform entries must be +-1, +-2 or +-3");
    for (int a = 0; a < 3; ++a) ctx->blocks[block].f[face].tf[a] = transform[a];
    return HX_OK;
}

int hx_finalize(hx_ctx* ctx) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (ctx->finalized) return fail(ctx, HX_ERR_STATE, "hx_finalize called twice");
    if (ctx->blocks.empty()) return fail(ctx, HX_ERR_TOPOLOGY, "no blocks");
    int rc = set_device(ctx);
    if (rc) return rc;
    const int nb = (int)ctx->blocks.size();
    // ---- topology
    for (int b = 0; b < nb; ++b)
        for (int f = 0; f < 6; ++f) {
            const HostFace& F = ctx->blocks[b].f[f];
            char msg[160];
            if (F.kind < 0) {
                std::snprintf(msg, sizeof msg, "block %d face %d not set", b, f);
                return fail(ctx, HX_ERR_TOPOLOGY, msg);
            }
            const int d = f / 2, side = f % 2;
            if (is_phys(F.kind)) {
                if (ctx->blocks[b].n[d] <= GC) {
                    std::snprintf(msg, sizeof msg, "block %d face %d: a physical face needs more than %d nodes "
                                  "across", b, f, GC);
                    return fail(ctx, HX_ERR_TOPOLOGY, msg);
                }
                continue;
            }
            if (F.nbr < 0 || F.nbr >= nb || F.nbr_face < 0 || F.nbr_face > 5) {
                std::snprintf(msg, sizeof msg, "block %d face %d: bad neighbour block or face", b, f);
                return fail(ctx, HX_ERR_TOPOLOGY, msg);
            }
            // the transform: a rotation of the index axes (signed permutation,
            // determinant +1) whose normal entry reaches the neighbour's face
            // from the correct side
            int used = 0, M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int a = 0; a < 3; ++a) {
                const int t = F.tf[a], p = std::abs(t) - 1;
                used |= 1 << p;
                M[p][a] = t > 0 ? 1 : -1;
            }
            const int det = used != 7 ? 0
                            : M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                                  M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                                  M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            const int nside = F.nbr_face % 2;
            if (det != 1 || std::abs(F.tf[d]) - 1 != F.nbr_face / 2 || (F.tf[d] > 0) != (side != nside)) {
                std::snprintf(msg, sizeof msg, "block %d face %d: the transform is not a rotation that joins "
                              "face %d of block %d", b, f, F.nbr_face, F.nbr);
                return fail(ctx, HX_ERR_TOPOLOGY, msg);
            }
            const HostBlock &H = ctx->blocks[b], &N = ctx->blocks[F.nbr];
            const HostFace& back = N.f[F.nbr_face];
            if (is_phys(back.kind) || back.nbr != b || back.nbr_face != f) {
                std::snprintf(msg, sizeof msg, "block %d face %d: neighbour face does not point back", b, f);
                return fail(ctx, HX_ERR_TOPOLOGY, msg);
            }
            for (int a = 0; a < 3; ++a) {
                const int t = F.tf[a], p = std::abs(t) - 1, u = back.tf[p];
                if (std::abs(u) - 1 != a || (u > 0) != (t > 0)) {
                    std::snprintf(msg, sizeof msg, "block %d face %d: the neighbour's transform is not the inverse",
                                  b, f);
                    return fail(ctx, HX_ERR_TOPOLOGY, msg);
                }
                if (a != d && H.n[a] != N.n[p]) {
                    std::snprintf(msg, sizeof msg, "block %d face %d: extents across differ from the neighbour", b, f);
                    return fail(ctx, HX_ERR_TOPOLOGY, msg);
                }
            }
        }
    // ---- layouts
    long long off = 0, offc = 0;
    for (auto& H : ctx->blocks) {
        const long long sj = round_up(XOFF + H.n[0] + G, 8), sk = sj * (H.n[1] + 2 * G);
        H.dev.n[0] = H.n[0];
        H.dev.n[1] = H.n[1];
        H.dev.n[2] = H.n[2];
        H.dev.sj = (int)sj;
        H.dev.sk = (int)sk;
        H.dev.base = off + XOFF + G * sj + G * sk;
        off = round_up(off + sk * (H.n[2] + 2 * G), 32);
        const long long sjc = round_up(XOFF + H.n[0] + GC, 8), skc = sjc * (H.n[1] + 2 * GC);
        H.cdev = H.dev;
        H.cdev.sj = (int)sjc;
        H.cdev.sk = (int)skc;
        H.cdev.base = offc + XOFF + GC * sjc + GC * skc;
        offc = round_up(offc + skc * (H.n[2] + 2 * GC), 32);
        H.dev.phys = H.dev.wall = H.dev.ff = 0;
        for (int f = 0; f < 6; ++f) {
            if (is_phys(H.f[f].kind)) H.dev.phys |= 1 << f;
            if (H.f[f].kind == HX_FACE_WALL) H.dev.wall |= 1 << f;
            if (H.f[f].kind == HX_FACE_FARFIELD) H.dev.ff |= 1 << f;
            H.dev.nbr[f] = is_phys(H.f[f].kind) ? -1 : H.f[f].nbr;
            for (int a = 0; a < 3; ++a) H.dev.tf[f][a] = (signed char)(is_phys(H.f[f].kind) ? a + 1 : H.f[f].tf[a]);
        }
        H.dev.dt = 0.0;
        ctx->max_block_pts = std::max(ctx->max_block_pts, H.npts());
    }
    ctx->fs = round_up(off, 64);
    ctx->fsc = round_up(offc, 64);
    if (ctx->fsc >= (1LL << 31)) return fail(ctx, HX_ERR_INVALID_ARG, "grid too large for 32-bit node offsets");
    // ---- buffers
    const size_t fs = (size_t)ctx->fs, r = ctx->rsize();
    const bool visc = ctx->cfg.viscous != 0;
    if ((rc = dalloc(ctx, (void**)&ctx->met, 10 * fs * 8))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->Qn, 5 * fs * 8))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->Qa, 5 * fs * 8))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->Qb, 5 * fs * 8))) return rc;
    if ((rc = dalloc(ctx, &ctx->A, 5 * fs * r))) return rc;
    if (visc) {
        if ((rc = dalloc(ctx, &ctx->prim, 4 * fs * r))) return rc;
        if ((rc = dalloc(ctx, &ctx->grad, 12 * fs * r))) return rc;
    }
    if (ctx->fp64()) {
        if ((rc = dalloc(ctx, (void**)&ctx->nrm, 21 * fs * 8))) return rc;
        HX_CK(launch_fill(ctx->nrm, true, 21 * ctx->fs, 0.0, ctx->stream));
        if ((rc = dalloc(ctx, (void**)&ctx->nst, NodeState<double>::NF * fs * 8))) return rc;
        HX_CK(launch_fill(ctx->nst, true, NodeState<double>::NF * ctx->fs, 1.0, ctx->stream));
    } else {
        for (int q = 0; q < 3; ++q)
            if ((rc = dalloc(ctx, (void**)&ctx->Qf[q], 5 * fs * 4))) return rc;
        if ((rc = dalloc(ctx, (void**)&ctx->metf, 10 * fs * 4))) return rc;
        if ((rc = dalloc(ctx, (void**)&ctx->Aref, 5 * fs * 4))) return rc;
    }
    if ((rc = dalloc(ctx, (void**)&ctx->stage, (size_t)ctx->max_block_pts * 12 * 8))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->d_flags, sizeof(unsigned)))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->d_bmax, nb * sizeof(unsigned long long)))) return rc;
    if ((rc = dalloc(ctx, (void**)&ctx->d_scal, 8 * sizeof(double)))) return rc;
    // state-like buffers start at a benign uniform value so that never-read
    // padding holds finite numbers
    HX_CK(launch_fill(ctx->met, true, 10 * ctx->fs, 1.0, ctx->stream));
    HX_CK(launch_fill(ctx->Qn, true, 5 * ctx->fs, 1.0, ctx->stream));
    HX_CK(launch_fill(ctx->Qa, true, 5 * ctx->fs, 1.0, ctx->stream));
    HX_CK(launch_fill(ctx->Qb, true, 5 * ctx->fs, 1.0, ctx->stream));
    HX_CK(launch_fill(ctx->A, ctx->fp64(), 5 * ctx->fs, 0.0, ctx->stream));
    if (visc) {
        HX_CK(launch_fill(ctx->prim, ctx->fp64(), 4 * ctx->fs, 1.0, ctx->stream));
        HX_CK(launch_fill(ctx->grad, ctx->fp64(), 12 * ctx->fs, 0.0, ctx->stream));
    }
    if (!ctx->fp64()) {
        for (int q = 0; q < 3; ++q) HX_CK(launch_fill(ctx->Qf[q], false, 5 * ctx->fs, 1.0, ctx->stream));
        HX_CK(launch_fill(ctx->metf, false, 10 * ctx->fs, 1.0, ctx->stream));
    }
    // ---- work lists
    std::vector<DevBlock> tab;
    for (auto& H : ctx->blocks) {
        H.dev.lim = ctx->fs;
        H.dev.flags = ctx->d_flags;
        H.cdev.lim = ctx->fsc;
        H.cdev.flags = ctx->d_flags;
        tab.push_back(H.dev);
    }
    if ((rc = upload(ctx, &ctx->d_blocks, tab))) return rc;
    ctx->dt_dev.assign(nb, 0.0);
    for (int d = 0; d < 3; ++d)
        for (int v = 0; v < kFluxVariants; ++v) {
            std::vector<Tile> t;
            make_tiles(ctx, d, flux_shape(d, v), t);
            ctx->ntiles[d][v] = (int)t.size();
            if ((rc = upload(ctx, &ctx->d_tiles[d][v], t))) return rc;
        }
    std::vector<Brick> bi, bp, bg;
    for (int b = 0; b < nb; ++b) {
        const HostBlock& H = ctx->blocks[b];
        const int lo[3] = {0, 0, 0}, hi[3] = {H.n[0], H.n[1], H.n[2]};
        add_bricks(bi, b, lo, hi);
        for (int f = 0; f < 6; ++f) {   // face ghost slabs (no edges or corners)
            const int d = f / 2;
            int l2[3] = {0, 0, 0}, h2[3] = {H.n[0], H.n[1], H.n[2]};
            if (f % 2) {
                l2[d] = H.n[d];
                h2[d] = H.n[d] + G;
            } else {
                l2[d] = -G;
                h2[d] = 0;
            }
            add_bricks(bg, b, l2, h2);
        }
    }
    {   // column tiles: segments along k short enough that the launch has
        // about 16 CTAs per SM, at least 8 planes each
        long long cols = 0;
        for (auto& H : ctx->blocks) cols += (long long)((H.n[0] + 31) / 32) * ((H.n[1] + 7) / 8);
        const long long want = 16LL * ctx->num_sms;
        const int segs = (int)std::max<long long>(1, (want + cols - 1) / cols);
        std::vector<Brick> bc;
        for (int b = 0; b < nb; ++b) {
            const HostBlock& H = ctx->blocks[b];
            const int kc = std::max(8, (H.n[2] + segs - 1) / segs);
            for (int k = 0; k < H.n[2]; k += kc)
                for (int j = 0; j < H.n[1]; j += 8)
                    for (int i = 0; i < H.n[0]; i += 32)
                        bc.push_back(Brick{b, i, j, k, std::min(32, H.n[0] - i), std::min(8, H.n[1] - j),
                                           std::min(kc, H.n[2] - k), 0});
        }
        ctx->n_col = (int)bc.size();
        if ((rc = upload(ctx, &ctx->d_col, bc))) return rc;
    }
    bp = bi;
    bp.insert(bp.end(), bg.begin(), bg.end());
    ctx->n_int = (int)bi.size();
    ctx->n_prim = (int)bp.size();
    ctx->n_prep = (int)bp.size();
    ctx->n_ghost = (int)bg.size();
    if ((rc = upload(ctx, &ctx->d_int, bi))) return rc;
    if ((rc = upload(ctx, &ctx->d_prim, bp))) return rc;
    ctx->d_prep = ctx->d_prim;
    if ((rc = upload(ctx, &ctx->d_ghost, bg))) return rc;
    if (ctx->cfg.debug_poison) {
        std::vector<Brick> sh;
        for (int b = 0; b < nb; ++b) {
            const HostBlock& H = ctx->blocks[b];
            const int lo[3] = {-G, -G, -G}, hi[3] = {H.n[0] + G, H.n[1] + G, H.n[2] + G};
            add_bricks(sh, b, lo, hi);
        }
        ctx->n_shell = (int)sh.size();
        if ((rc = upload(ctx, &ctx->d_shell, sh))) return rc;
    }
    std::vector<NodeItem> bc;
    for (int b = 0; b < nb; ++b) {
        const HostBlock& H = ctx->blocks[b];
        for (int f = 0; f < 6; ++f) {
            if (H.f[f].kind != HX_FACE_FARFIELD) continue;
            const int d = f / 2, side = f % 2, a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            for (int t2 = 0; t2 < H.n[a2]; ++t2)
                for (int t1 = 0; t1 < H.n[a1]; ++t1) {
                    int id[3];
                    id[d] = side ? H.n[d] - 1 : 0;
                    id[a1] = t1;
                    id[a2] = t2;
                    bc.push_back(NodeItem{b, id[0], id[1], id[2], d, side, 0, 0});
                }
        }
    }
    ctx->n_bc = (int)bc.size();
    if ((rc = upload(ctx, &ctx->d_bc, bc))) return rc;
    HX_CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches_per_step = 3 * (1 + (visc ? 1 : 0) + 3 + (ctx->fp64() ? 0 : 1) + (ctx->n_bc ? 1 : 0) +
                                  (ctx->cfg.debug_poison ? (visc ? 4 : 2) : 0));
    ctx->finalized = true;
    return HX_OK;
}

int hx_compute_metrics(hx_ctx* ctx) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    NvtxScope range("hx_compute_metrics");
    if (!ctx->finalized) return fail(ctx, HX_ERR_STATE, "call hx_finalize first");
    int rc = set_device(ctx);
    if (rc) return rc;
    const size_t cbytes = 3 * (size_t)ctx->fsc * 8;
    double* X = nullptr;
    if ((rc = dalloc(ctx, (void**)&X, cbytes))) return rc;
    HX_CK(launch_fill(X, true, 3 * ctx->fsc, 0.0, ctx->stream));
    std::vector<DevBlock> ctab;
    for (auto& H : ctx->blocks) {
        if (H.xyz.empty()) return fail(ctx, HX_ERR_STATE, "metrics already computed");
        HX_CK(cudaMemcpyAsync(ctx->stage, H.xyz.data(), H.xyz.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        HX_CK(launch_unpack(ctx->stage, X, true, ctx->fsc, H.cdev, 3, ctx->stream));
        ctab.push_back(H.cdev);
    }
    // ghost coordinates, direction by direction (edges and corners included)
    std::vector<double> tr(6 * ctx->blocks.size() * 3);
    for (size_t b = 0; b < ctx->blocks.size(); ++b)
        for (int f = 0; f < 6; ++f)
            for (int m = 0; m < 3; ++m) tr[(b * 6 + f) * 3 + m] = ctx->blocks[b].f[f].tr[m];
    double* dtr = nullptr;
    DevBlock* dc = nullptr;
    if ((rc = upload(ctx, &dtr, tr))) return rc;
    if ((rc = upload(ctx, &dc, ctab))) return rc;
    std::vector<std::pair<void*, size_t>> tmp;
    for (int m = 1; m <= 3; ++m) {
        std::vector<HaloItem> items;
        coord_halo_items(ctx, m, items);
        for (const HaloItem& it : items)
            if (it.dst < 0 || it.dst >= ctx->fsc || it.src < 0 || it.src >= ctx->fsc || it.aux < 0 ||
                it.aux >= ctx->fsc)
                return fail(ctx, HX_ERR_TOPOLOGY, "a ghost coordinate outside the coordinate layout");
        HaloItem* di = nullptr;
        if ((rc = upload(ctx, &di, items))) return rc;
        tmp.emplace_back((void*)di, items.size() * sizeof(HaloItem));
        HX_CK(launch_halo_coords(di, (int)items.size(), X, ctx->fsc, dtr, ctx->stream));
    }
    std::vector<Brick> bm;
    for (int b = 0; b < (int)ctx->blocks.size(); ++b) {
        const HostBlock& H = ctx->blocks[b];
        const int lo[3] = {-G, -G, -G}, hi[3] = {H.n[0] + G, H.n[1] + G, H.n[2] + G};
        add_bricks(bm, b, lo, hi);
    }
    Brick* dbm = nullptr;
    if ((rc = upload(ctx, &dbm, bm))) return rc;
    HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    HX_CK(launch_metrics(dbm, (int)bm.size(), dc, X, ctx->fsc, ctx->d_blocks, ctx->met, ctx->fs, ctx->d_flags,
                         ctx->stream));
    if (ctx->fp64())
        HX_CK(launch_normals(dbm, (int)bm.size(), ctx->d_blocks, ctx->met, ctx->fs, ctx->nrm, ctx->stream));
    else
        HX_CK(launch_cast(ctx->met, ctx->metf, 10 * ctx->fs, ctx->stream));
    unsigned flags = 0;
    HX_CK(cudaMemcpyAsync(&flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, X, cbytes);
    dfree(ctx, dtr, tr.size() * 8);
    dfree(ctx, dc, ctab.size() * sizeof(DevBlock));
    dfree(ctx, dbm, bm.size() * sizeof(Brick));
    for (auto& t : tmp) dfree(ctx, t.first, t.second);
    if (flags & FLAG_BOUNDS) return fail(ctx, HX_ERR_BOUNDS, "a node offset outside its field (checking build)");
    if (flags & FLAG_BAD_GRID) return fail(ctx, HX_ERR_BAD_GRID, "non-positive Jacobian (J^-1 <= 0) at some node");
    for (auto& H : ctx->blocks) std::vector<double>().swap(H.xyz);
    ctx->metrics_done = true;
    if ((rc = compute_ref_residual(ctx))) return rc;
    return HX_OK;
}

int hx_set_state(hx_ctx* ctx, int block, const double* q, int on_device) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (block < 0 || block >= (int)ctx->blocks.size() || !q) return fail(ctx, HX_ERR_INVALID_ARG, "bad block or pointer");
    const HostBlock& H = ctx->blocks[block];
    const double* src = q;
    if (!on_device) {
        HX_CK(cudaMemcpyAsync(ctx->stage, q, 5 * H.npts() * 8, cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->stage;
    }
    HX_CK(launch_unpack2(src, ctx->Qn, ctx->Qf[0], ctx->fs, H.dev, 5, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    return HX_OK;
}

static int get_field(hx_ctx* ctx, int block, const void* buf, bool fp64, int nf, double* out, int on_device) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (block < 0 || block >= (int)ctx->blocks.size() || !out) return fail(ctx, HX_ERR_INVALID_ARG, "bad block or pointer");
    const HostBlock& H = ctx->blocks[block];
    double* dst = on_device ? out : ctx->stage;
    HX_CK(launch_pack(buf, fp64, ctx->fs, H.dev, nf, dst, ctx->stream));
    if (!on_device) HX_CK(cudaMemcpyAsync(out, ctx->stage, nf * H.npts() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    return HX_OK;
}

int hx_get_state(hx_ctx* ctx, int block, double* q_out, int on_device) {
    return get_field(ctx, block, ctx ? ctx->Qn : nullptr, true, 5, q_out, on_device);
}

int hx_get_metrics(hx_ctx* ctx, int block, double* m_out, int on_device) {
    return get_field(ctx, block, ctx ? ctx->met : nullptr, true, 10, m_out, on_device);
}

int hx_get_gradients(hx_ctx* ctx, int block, double* g_out, int on_device) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!ctx->cfg.viscous) return fail(ctx, HX_ERR_STATE, "gradients exist only for Navier-Stokes");
    // the step keeps only the node stress tensor; the 12 gradients of the
    // current state are formed here (they overwrite it until the next stage)
    const bool f64 = ctx->fp64();
    void* Qs = stencil_state(ctx, 0);
    const void* M = stencil_met(ctx);
    HX_CK(launch_prep(ctx->d_prep, ctx->n_prep, ctx->d_blocks, Qs, f64, ctx->fs, M, ctx->prim, f64 ? ctx->nst : nullptr,
                      ctx->gas, ctx->stream));
    HX_CK(launch_grad(ctx->d_col, ctx->n_col, ctx->d_blocks, ctx->prim, M, f64, ctx->fs, ctx->grad, false, ctx->gas,
                      ctx->stream));
    return get_field(ctx, block, ctx->grad, f64, 12, g_out, on_device);
}

int hx_compute_dt(hx_ctx* ctx, double cfl, double* dt_global, double* dt_per_block) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!(cfl > 0)) return fail(ctx, HX_ERR_INVALID_ARG, "cfl must be positive");
    const int nb = (int)ctx->blocks.size();
    HX_CK(cudaMemsetAsync(ctx->d_bmax, 0, nb * sizeof(unsigned long long), ctx->stream));
    HX_CK(launch_dt(ctx->d_int, ctx->n_int, ctx->d_blocks, ctx->Qn, ctx->met, ctx->fs, ctx->gas, ctx->d_bmax,
                    ctx->stream));
    std::vector<unsigned long long> bits(nb);
    HX_CK(cudaMemcpyAsync(bits.data(), ctx->d_bmax, nb * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    double gmin = INFINITY;
    for (int b = 0; b < nb; ++b) {
        double smax;
        std::memcpy(&smax, &bits[b], 8);
        if (!(smax > 0) || !std::isfinite(smax)) return fail(ctx, HX_ERR_NONFINITE, "invalid wave speed in the state");
        const double dt = cfl / smax;
        if (dt_per_block) dt_per_block[b] = dt;
        gmin = std::min(gmin, dt);
    }
    if (dt_global) *dt_global = gmin;
    return HX_OK;
}

int hx_step(hx_ctx* ctx, int nsteps, double dt) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    NvtxScope range("hx_step");
    return step_common(ctx, nsteps, std::vector<double>(ctx->blocks.size(), dt));
}

int hx_step_multi(hx_ctx* ctx, int nsteps, const double* dt_per_block) {
    if (!ctx || !dt_per_block) return HX_ERR_INVALID_ARG;
    NvtxScope range("hx_step_multi");
    return step_common(ctx, nsteps, std::vector<double>(dt_per_block, dt_per_block + ctx->blocks.size()));
}

int hx_step_cfl(hx_ctx* ctx, int nsteps, double cfl, int per_block, double* time_advanced) {
    NvtxScope range("hx_step_cfl");
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (nsteps < 0 || !(cfl > 0) || !std::isfinite(cfl)) return fail(ctx, HX_ERR_INVALID_ARG, "bad nsteps or cfl");
    per_block = per_block ? 1 : 0;
    if ((rc = autotune(ctx))) return rc;
    if (!ctx->gexec_cfl[per_block] && (rc = capture(ctx, &ctx->gexec_cfl[per_block], per_block))) return rc;
    const double init[2] = {cfl, 0.0};
    HX_CK(cudaMemcpyAsync(ctx->d_scal, init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    for (int i = 0; i < nsteps; ++i) HX_CK(cudaGraphLaunch(ctx->gexec_cfl[per_block], ctx->stream));
    double t = 0.0;
    HX_CK(cudaMemcpyAsync(&t, ctx->d_scal + 1, sizeof t, cudaMemcpyDeviceToHost, ctx->stream));
    rc = read_flags(ctx);
    ctx->dt_dev.assign(ctx->blocks.size(), -1.0);   // the table now holds device-chosen dt
    if (time_advanced) *time_advanced = t;
    return rc;
}

static int ensure_dtl(hx_ctx* ctx) {
    if (ctx->dtl) return HX_OK;
    int rc = dalloc(ctx, (void**)&ctx->dtl, (size_t)ctx->fs * 8);
    if (rc) return rc;
    HX_CK(launch_fill(ctx->dtl, true, ctx->fs, 0.0, ctx->stream));
    return HX_OK;
}

int hx_step_local(hx_ctx* ctx, int nsteps, double cfl) {
    NvtxScope range("hx_step_local");
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (nsteps < 0 || !(cfl > 0) || !std::isfinite(cfl)) return fail(ctx, HX_ERR_INVALID_ARG, "bad nsteps or cfl");
    if ((rc = autotune(ctx))) return rc;
    if ((rc = ensure_dtl(ctx))) return rc;
    if (!ctx->gexec_lts && (rc = capture(ctx, &ctx->gexec_lts, 2))) return rc;
    HX_CK(cudaMemcpyAsync(ctx->d_scal, &cfl, sizeof cfl, cudaMemcpyHostToDevice, ctx->stream));
    HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    for (int i = 0; i < nsteps; ++i) HX_CK(cudaGraphLaunch(ctx->gexec_lts, ctx->stream));
    return read_flags(ctx);
}

int hx_local_dt(hx_ctx* ctx, int block, double cfl, double* dt_out, int on_device) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!(cfl > 0) || !std::isfinite(cfl)) return fail(ctx, HX_ERR_INVALID_ARG, "bad cfl");
    if ((rc = ensure_dtl(ctx))) return rc;
    HX_CK(cudaMemcpyAsync(ctx->d_scal, &cfl, sizeof cfl, cudaMemcpyHostToDevice, ctx->stream));
    HX_CK(launch_dt_local(ctx->d_int, ctx->n_int, ctx->d_blocks, ctx->Qn, ctx->met, ctx->fs, ctx->gas, ctx->d_scal,
                          ctx->dtl, ctx->stream));
    return get_field(ctx, block, ctx->dtl, true, 1, dt_out, on_device);
}

int hx_residual(hx_ctx* ctx, double* rms) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!rms) return fail(ctx, HX_ERR_INVALID_ARG, "null output");
    if ((rc = autotune(ctx))) return rc;
    if ((rc = enqueue_rhs(ctx, 0, nullptr, nullptr))) return rc;
    HX_CK(cudaMemsetAsync(ctx->d_scal + 2, 0, 5 * sizeof(double), ctx->stream));
    HX_CK(launch_residual(ctx->d_int, ctx->n_int, ctx->d_blocks, ctx->A, ctx->Aref, ctx->fp64(), ctx->met, ctx->fs,
                          ctx->d_scal + 2, ctx->stream));
    double sums[5];
    HX_CK(cudaMemcpyAsync(sums, ctx->d_scal + 2, sizeof sums, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    const double n = (double)hx_points(ctx);
    for (int c = 0; c < 5; ++c) rms[c] = std::sqrt(sums[c] / n);
    return HX_OK;
}

int hx_rhs(hx_ctx* ctx, int block, double* r_out, int on_device) {
    NvtxScope range("hx_rhs");
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (block < 0 || block >= (int)ctx->blocks.size() || !r_out) return fail(ctx, HX_ERR_INVALID_ARG, "bad block or pointer");
    if ((rc = autotune(ctx))) return rc;
    if ((rc = enqueue_rhs(ctx, 0, nullptr, nullptr))) return rc;
    const HostBlock& H = ctx->blocks[block];
    double* dst = on_device ? r_out : ctx->stage;
    HX_CK(launch_rhs_out(H.dev, ctx->A, ctx->Aref, ctx->fp64(), ctx->met, ctx->fs, dst, ctx->stream));
    if (!on_device) HX_CK(cudaMemcpyAsync(r_out, ctx->stage, 5 * H.npts() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HX_CK(cudaStreamSynchronize(ctx->stream));
    return HX_OK;
}

int hx_profile_step(hx_ctx* ctx, int nsteps, double dt, hx_kernel_stat* out, int max_kinds, int* n_kinds) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!(dt > 0) || nsteps < 0) return fail(ctx, HX_ERR_INVALID_ARG, "bad dt or nsteps");
    if ((rc = upload_dt(ctx, std::vector<double>(ctx->blocks.size(), dt)))) return rc;
    if ((rc = autotune(ctx))) return rc;
    HX_CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    Prof pf;
    pf.on = true;
    pf.s = ctx->stream;
    for (int i = 0; i < nsteps; ++i)
        if ((rc = enqueue_step(ctx, &pf))) return rc;
    HX_CK(cudaStreamSynchronize(ctx->stream));
    double tot[K_COUNT] = {};
    int cnt[K_COUNT] = {};
    for (auto& r : pf.recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        tot[r.kind] += ms;
        cnt[r.kind] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    int k = 0;
    for (int i = 0; i < K_COUNT && k < max_kinds; ++i) {
        if (!cnt[i]) continue;
        if (out) {
            std::memset(&out[k], 0, sizeof(hx_kernel_stat));
            std::snprintf(out[k].name, sizeof out[k].name, "%s", kKindName[i]);
            out[k].launches = cnt[i];
            out[k].total_ms = tot[i];
        }
        ++k;
    }
    if (n_kinds) *n_kinds = k;
    return read_flags(ctx);
}

int hx_launches_per_step(const hx_ctx* ctx) { return ctx ? ctx->launches_per_step : 0; }

int hx_tuning(const hx_ctx* ctx, int* variant, int* tile_shape, double* ms) {
    if (!ctx) return HX_ERR_INVALID_ARG;
    if (!ctx->tuned) return HX_ERR_STATE;
    for (int d = 0; d < 3; ++d) {
        if (variant) variant[d] = ctx->variant[d];
        for (int v = 0; v < kFluxVariants; ++v) {
            if (tile_shape) {
                const FluxShape sh = flux_shape(d, v);
                tile_shape[(d * kFluxVariants + v) * 2] = sh.tp;
                tile_shape[(d * kFluxVariants + v) * 2 + 1] = sh.na;
            }
            if (ms) ms[d * kFluxVariants + v] = ctx->tune_ms[d][v];
        }
    }
    return HX_OK;
}

long long hx_points(const hx_ctx* ctx) {
    long long n = 0;
    if (ctx)
        for (auto& H : ctx->blocks) n += H.npts();
    return n;
}

size_t hx_device_bytes(const hx_ctx* ctx) { return ctx ? ctx->bytes : 0; }

const char* hx_last_error(const hx_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void hx_destroy(hx_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    for (auto& g : ctx->gexec_cfl)
        if (g) cudaGraphExecDestroy(g);
    if (ctx->gexec_lts) cudaGraphExecDestroy(ctx->gexec_lts);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
