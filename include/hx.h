/*
 * hx.h -- C ABI of the GB300 (sm_103a) library for the per-Runge-Kutta-stage
 * residual evaluation and update of a multi-block curvilinear high-order
 * finite-difference compressible Navier-Stokes solver, after Ye, Zhang, Wan,
 * Yan, Sun, "Accelerating CFD simulation with high order finite difference
 * method on curvilinear coordinates for modern GPU clusters" (HiResX).
 *
 * Method (section / equation of the paper):
 *   - nondimensional Navier-Stokes in curvilinear form, Eqs. (1)-(6);
 *   - conservative metrics and Jacobian, Eqs. (7)-(8), sixth-order central
 *     differences (Sec. 2);
 *   - inviscid fluxes by the modified alternative-formulation WENO5
 *     (characteristic space at the node, shared smoothness indicators,
 *     Sec. 4.5.1, Figs. 10-11) with Steger-Warming splitting, Eqs. (9)-(19);
 *   - viscous fluxes at nodes from chain-rule gradients, Eq. (21), and their
 *     sixth-order central divergence (Sec. 4.5.2, Fig. 12);
 *   - R = -J * sum_d d/d(xi_d)(E_d - E_v,d), Eqs. (2)-(3);
 *   - TVD Runge-Kutta 3, Eq. (20);
 *   - on-device block-interface and physical-boundary halo fill (Fig. 2:
 *     bc_block, bc_phys; Sec. 4.1: blocks of one process exchanged on the GPU).
 *
 * Conventions for every entry point:
 *   - returns HX_OK (0) on success or a negative HX_ERR_* code; the message
 *     of the last failure of a context is available from hx_last_error();
 *   - arrays are C-contiguous double precision in the layouts stated below,
 *     i fastest: a block field is [nk][nj][ni];
 *   - the library copies every input; callers keep ownership of their
 *     buffers and may free them when the call returns;
 *   - pointers flagged "on_device" are CUDA device pointers on the device
 *     current when hx_create was called (e.g. torch tensors); otherwise they
 *     are host pointers (pinned memory makes the copies faster);
 *   - calls on one context are not thread-safe; work is issued on the
 *     context's stream and every call returns after that stream is idle.
 * There is no CPU fallback: without a CUDA device hx_create fails with
 * HX_ERR_CUDA.
 */
#ifndef HX_H
#define HX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HX_OK = 0,
    HX_ERR_INVALID_ARG = -1,  /* bad pointer, index, size or value              */
    HX_ERR_STATE = -2,        /* call out of order (e.g. step before metrics)    */
    HX_ERR_TOPOLOGY = -3,     /* unset face, unmatched or inconsistent neighbour */
    HX_ERR_BAD_GRID = -4,     /* a node has J^-1 <= 0 (Eq. (8))                  */
    HX_ERR_OOM = -5,          /* device allocation failed or cap exceeded        */
    HX_ERR_CUDA = -6,         /* a CUDA runtime call failed                      */
    HX_ERR_NONFINITE = -7,    /* a step produced a non-finite state              */
    HX_ERR_UNPHYSICAL = -8,   /* non-positive density or pressure after a step   */
    HX_ERR_TIMEOUT = -9,      /* reserved: a bounded device wait gave up         */
    HX_ERR_BOUNDS = -10       /* checking builds (HX_BOUNDS) only: a kernel computed
                                 a node offset outside its field                  */
};

/* Face kinds (Sec. 4.2: connecting faces and physical faces). */
enum {
    HX_FACE_PERIODIC = 0,   /* joined to a face of the same or another block, coordinates translated */
    HX_FACE_INTERFACE = 1,  /* 1:1 block interface, node-disjoint continuation                       */
    HX_FACE_WALL = 2,       /* no-slip adiabatic wall on the boundary nodes                          */
    HX_FACE_FARFIELD = 3    /* characteristic far field (1D Riemann invariants)                      */
};

enum { HX_FP64 = 0, HX_MIXED = 1 };

typedef struct {
    double gamma;         /* specific heat ratio (1.4)                                 */
    double mach;          /* free-stream Mach number Ma (free stream along +x)         */
    double reynolds;      /* free-stream Reynolds number Re                             */
    double prandtl;       /* Prandtl number Pr                                          */
    int viscous;          /* 0: Euler, 1: Navier-Stokes                                 */
    int mu_law;           /* 0: mu = 1, 1: Sutherland mu = T^1.5 (1+S)/(T+S)            */
    double sutherland_s;  /* S of Sutherland's law (110.4/288.15)                       */
    int precision;        /* HX_FP64, or HX_MIXED: FP32 stencil state, fluxes, WENO and
                             accumulation; FP64 metrics and FP64 state.  The RK stage
                             forms its increment -c dt J A in FP32 (the precision of A)
                             and combines it with Q^n and Q^(k) in FP64 (Eq. (20)); its
                             FP32 copy of the new state rounds to nearest             */
    int scheme;           /* 0: modified AFWENO (characteristic space at the node, shared
                             indicators, Figs. 10-11); 1: the original AFWENO
                             (characteristic space at the face, two WENOs per face,
                             Fig. 9), kept to measure the modification              */
    size_t mem_cap_bytes; /* 0: no cap; else hx_finalize fails with HX_ERR_OOM above it */
    int autotune;         /* 1: time the tile-shape candidates once per shape class
                             (process-wide cache); 0: take the 128-thread tiles
                             (16 x 8 along xi, 8 x 16 across), reproducible for
                             profiling                                               */
    int debug_poison;     /* 1 (checking only, slower): before every stage the ghost
                             nodes of the stencil state, primitives, node stress,
                             accumulator and (FP64) the sweeps' node state are set
                             to NaN, so that a ghost the halo fill misses turns the
                             result non-finite; 0: off                              */
} hx_config;

typedef struct hx_ctx hx_ctx;

/* Per-kernel-family timing of hx_profile_step. */
typedef struct {
    char name[32];
    int launches;         /* launches in the profiled steps              */
    double total_ms;      /* summed CUDA-event durations                 */
} hx_kernel_stat;

/* Fills cfg with gamma 1.4, Ma 0.5, Re 1, Pr 0.72, Euler, Sutherland S,
 * FP64, modified AFWENO, no cap, autotune on. */
int hx_config_default(hx_config* cfg);

/* Creates a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t to issue all work on, or NULL for a stream the context
 * creates and owns. */
int hx_create(hx_ctx** out, const hx_config* cfg, void* cuda_stream);

/* Adds a block of ni x nj x nk nodes (each >= 6).  xyz is a host array
 * [3][nk][nj][ni] of node coordinates (x, y, z), copied.  The block id is
 * written to *block_id (ids are 0, 1, 2, ... in call order). */
int hx_add_block(hx_ctx* ctx, int ni, int nj, int nk, const double* xyz, int* block_id);

/* Sets face `face` (0..5 = i-, i+, j-, j+, k-, k+) of `block`.  For
 * PERIODIC and INTERFACE faces (the 1:1 block interfaces of Sec. 4.2 and
 * Fig. 2, bc_block), nbr_block/nbr_face name the joined face; translate (may
 * be NULL = 0) is added to the neighbour's coordinates to give this block's
 * ghost coordinates.  The index transform is reset to the identity (axis a
 * runs along axis a of the neighbour), which joins i+ to i-, j+ to j- and
 * k+ to k- of aligned blocks; other pairings need hx_set_face_transform.
 * A WALL or FARFIELD face needs more than 6 nodes across (the ghost
 * coordinates reflect through it); the neighbour arguments are ignored.
 * Checked at hx_finalize (HX_ERR_TOPOLOGY). */
int hx_set_face(hx_ctx* ctx, int block, int face, int kind, int nbr_block, int nbr_face,
                const double translate[3]);

/* Index transform of a PERIODIC or INTERFACE face, set after hx_set_face:
 * axis a (0 = i, 1 = j, 2 = k) of `block` runs along axis
 * |transform[a]| - 1 of the neighbour, in the same direction when
 * transform[a] > 0 and reversed when < 0 (the CGNS 1-to-1 convention).
 * Layer l beyond the face is the neighbour's node at distance l from its
 * joined face.  hx_finalize requires a rotation (a signed permutation with
 * determinant +1: both blocks keep a right-handed index space), a normal
 * entry that reaches nbr_face from the correct side, a neighbour face that
 * points back with the inverse transform, and equal extents along the
 * face.  The paper's interfaces are 1:1 but it shows aligned blocks only;
 * the state, coordinates and gradients are physical quantities, so the
 * transform maps indices and nothing else.  Entries outside +-1..+-3:
 * HX_ERR_INVALID_ARG; after hx_finalize: HX_ERR_STATE. */
int hx_set_face_transform(hx_ctx* ctx, int block, int face, const int transform[3]);

/* Validates the topology (HX_ERR_TOPOLOGY), plans device buffers and work
 * lists and allocates them (HX_ERR_OOM). */
int hx_finalize(hx_ctx* ctx);

/* Conservative metrics (Eq. (7)) and Jacobian (Eq. (8)) on every node and on
 * three ghost layers, in FP64.  Fails with HX_ERR_BAD_GRID if any J^-1 <= 0. */
int hx_compute_metrics(hx_ctx* ctx);

/* Sets the conservative state (rho, rho u, rho v, rho w, e) of `block` from
 * q [5][nk][nj][ni]. */
int hx_set_state(hx_ctx* ctx, int block, const double* q, int on_device);

/* Copies the conservative state of `block` into q_out [5][nk][nj][ni]. */
int hx_get_state(hx_ctx* ctx, int block, double* q_out, int on_device);

/* Copies the node metrics of `block` into m_out [10][nk][nj][ni]:
 * xi^_x, xi^_y, xi^_z, eta^_x, ..., zeta^_z (metric / J) and J. */
int hx_get_metrics(hx_ctx* ctx, int block, double* m_out, int on_device);

/* Time step from the current state:
 *   dt_b = cfl / max over the nodes of block b of sum_d (|m_d.u| + c |m_d|) J.
 * dt_global (may be NULL) gets min_b dt_b; dt_per_block (may be NULL) gets
 * one value per block. */
int hx_compute_dt(hx_ctx* ctx, double cfl, double* dt_global, double* dt_per_block);

/* Advances every block nsteps TVD-RK3 steps (Eq. (20)) with time step dt.
 * The step is captured once in a CUDA graph and replayed.  Returns
 * HX_ERR_NONFINITE if a non-finite value appeared. */
int hx_step(hx_ctx* ctx, int nsteps, double dt);

/* As hx_step with one time step per block (independent instances). */
int hx_step_multi(hx_ctx* ctx, int nsteps, const double* dt_per_block);

/* Advances every block nsteps TVD-RK3 steps with the time step chosen on
 * the device at the start of every step from the current state (the CFL
 * reduction of hx_compute_dt; Sec. 4.5.3 reduces the time step on the GPU
 * as well): dt = cfl / max over all nodes (per_block = 0), or per block
 * (per_block = 1, independent instances).  No host round trip per step; the
 * step and its dt reduction are one CUDA graph.  *time_advanced (may be
 * NULL) gets the sum of the global dt over the steps. */
int hx_step_cfl(hx_ctx* ctx, int nsteps, double cfl, int per_block, double* time_advanced);

/* Local time stepping (Sec. 4.4 keeps a time step per grid point; for
 * pseudo-time marching to a steady state): nsteps TVD-RK3 steps in which
 * every node advances with its own time step, taken on the device from the
 * state at the start of each step and held for its three stages:
 * dt_i = cfl / (lambda_c + lambda_v), lambda_c = sum_d (|m_d.u| + c |m_d|) J
 * as in hx_compute_dt, and for Navier-Stokes lambda_v = (Ma/Re)
 * max(4/3, gamma/Pr) (mu/rho) sum_d (J |m_d|)^2.  The paper prints no
 * formula; this is the library's reading.  Time is not consistent across
 * nodes, so the result is a steady state's approach, not a transient.
 * One CUDA graph per step; allocates one FP64 field on first use
 * (HX_ERR_OOM).  Errors: HX_ERR_INVALID_ARG (nsteps < 0, cfl not positive),
 * HX_ERR_NONFINITE / HX_ERR_UNPHYSICAL as hx_step. */
int hx_step_local(hx_ctx* ctx, int nsteps, double cfl);

/* The local time steps of hx_step_local for the current state of `block`,
 * written to dt_out [nk][nj][ni] (host, or device when on_device != 0). */
int hx_local_dt(hx_ctx* ctx, int block, double cfl, double* dt_out, int on_device);

/* Root-mean-square residual of the current state over all nodes of all
 * blocks, per conservative variable: rms[c] = sqrt(sum R_c^2 / N)
 * (Fig. 2 calc_res; reduced on the device, Sec. 4.5.3).  rms has 5 entries. */
int hx_residual(hx_ctx* ctx, double* rms);

/* Evaluates R(Q) = dQ/dt of the current state without advancing it and
 * copies block `block`'s residual into r_out [5][nk][nj][ni]. */
int hx_rhs(hx_ctx* ctx, int block, double* r_out, int on_device);

/* Navier-Stokes only: forms the 12 node gradients (u, v, w, T)_(x, y, z) of
 * the current state (Eq. (21)) and copies block `block`'s into
 * g_out [12][nk][nj][ni]. */
int hx_get_gradients(hx_ctx* ctx, int block, double* g_out, int on_device);

/* Runs nsteps steps launch by launch (no graph) with CUDA events around each
 * kernel on the context's stream and reports per-family totals in
 * out[0..*n_kinds-1] (at most max_kinds).  The state advances as in hx_step. */
int hx_profile_step(hx_ctx* ctx, int nsteps, double dt, hx_kernel_stat* out, int max_kinds, int* n_kinds);

/* The tile shapes the autotuner chose, after the first hx_step, hx_rhs or
 * hx_profile_step (HX_ERR_STATE before).  variant[3] (may be NULL): chosen
 * shape per direction (xi, eta, zeta); tile_shape[3][3][2] (may be NULL):
 * (nodes per chunk along the sweep, lines per CTA) of each candidate;
 * ms[3][3] (may be NULL): measured time of one launch per candidate, -1 where
 * a candidate was not timed (cached choice, autotune off, or cannot launch). */
int hx_tuning(const hx_ctx* ctx, int* variant, int* tile_shape, double* ms);

/* Kernel launches one RK step makes (all stages). */
int hx_launches_per_step(const hx_ctx* ctx);

/* Total interior nodes over all blocks. */
long long hx_points(const hx_ctx* ctx);

/* Device bytes held by the context. */
size_t hx_device_bytes(const hx_ctx* ctx);

/* Residual R(Q) = dQ/dt of one block that is periodic on all six faces,
 * Euler (inviscid terms only), FP64, computed without allocating any device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate -- code whose device memory is owned by another
 * allocator (for example a framework's memory pool holding the whole GPU),
 * or loops that must not call cudaMalloc/cudaFree because those calls can
 * synchronise the device and take unbounded time.
 *   q      device [5][nk][nj][ni] conservative state (rho, rho u, rho v, rho w, e)
 *   met    device [10][nk][nj][ni] node metrics and J, as hx_get_metrics
 *          returns them for that periodic block
 *   r_out  device [5][nk][nj][ni], written
 * q, met and r_out must be memory of the current device (device or managed
 * allocations); host memory or another GPU's memory is rejected with
 * HX_ERR_INVALID_ARG.
 * The result equals hx_rhs of an FP64 Euler context holding that block with
 * periodic faces, up to rounding.  All intermediates live in one static
 * device array of 32 MiB that the library holds on every GPU it is loaded
 * on until the process exits; a block whose padded fields do not fit (about
 * 48^3 nodes and above) is rejected with HX_ERR_INVALID_ARG, as are extents
 * below 6 and null pointers.  The first call on a device looks up that
 * array's device address (a one-time set-up); make that first call before
 * any stream capture.  Every call reuses the same array, so calls that
 * overlap on the GPU (different streams or threads) race and corrupt each
 * other's results; serialise them.  Work runs on cuda_stream (NULL = legacy
 * default stream) and the call returns after that stream is idle.
 * Returns HX_OK, HX_ERR_INVALID_ARG or HX_ERR_CUDA. */
int hx_euler_rhs_periodic_noalloc(int ni, int nj, int nk, double gamma, const double* q, const double* met,
                                  double* r_out, void* cuda_stream);

/* Message of the last failure on ctx (or of the last hx_create failure when
 * ctx is NULL).  Valid until the next call on ctx. */
const char* hx_last_error(const hx_ctx* ctx);

/* Releases every device and host resource of ctx (NULL is allowed). */
void hx_destroy(hx_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HX_H */
