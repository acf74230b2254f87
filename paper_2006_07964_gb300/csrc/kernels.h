// kernels.h -- host-side launchers of the device kernels (one per kernel
// family); the runtime calls only these.
#pragma once
#include <cuda_runtime.h>

#include "hx_common.cuh"

namespace hx {

// ---- fused per-direction flux kernel (k_flux.cuh) ------------------------
struct FluxArgs {
    const DevBlock* blocks;
    const Tile* tiles;
    int ntiles;
    const void* Q;      // R, 5 fields
    const void* met;    // R, 10 fields
    long long fs;       // field stride (elements)
    const void* stress; // R, 9 fields (tau_xx, tau_yy, tau_zz, tau_xy, tau_xz, tau_yz, beta), Navier-Stokes only
    void* A;            // R, 5 fields, accumulated divergence
    const void* nrm;    // FP64 form: the sweep normals (k_normals, 21 fields), or null
    const void* nst;    // FP64 form with nrm: the node state (k_prep, NodeState<double>::NF fields)
    int accumulate;
    Gas gas;
    int grid;           // CTAs of the persistent launch
    int fuse_rk;        // zeta sweep only: finish R and the RK3 stage instead of storing A
    int scheme;         // 0 modified AFWENO, 1 original AFWENO
    RKArgs rk;
};

struct FluxShape {
    int tp, na;         // nodes along the sweep, lines across
};

constexpr int kFluxVariants = 3;
FluxShape flux_shape(int dir, int variant);
// CTAs per SM the variant can keep resident (0 if it cannot launch); also
// sets the kernel's shared-memory opt-in.
int flux_ctas_per_sm(bool fp64, int dir, int variant, bool visc, bool rk = false, int scheme = 0);
cudaError_t launch_flux(bool fp64, int dir, int variant, bool visc, const FluxArgs& a, cudaStream_t s);

// ---- everything else (k_misc.cu) ----------------------------------------
// Unpack a host-layout array [nf][nk][nj][ni] (double) into the padded layout.
cudaError_t launch_unpack(const double* src, void* dst, bool dst_fp64, long long fs, DevBlock B, int nf,
                          cudaStream_t s);
// Same for a second, FP32 copy (nullable).
cudaError_t launch_unpack2(const double* src, double* dst64, float* dst32, long long fs, DevBlock B, int nf,
                           cudaStream_t s);
cudaError_t launch_pack(const void* src, bool src_fp64, long long fs, DevBlock B, int nf, double* dst,
                        cudaStream_t s);
cudaError_t launch_halo_coords(const HaloItem* items, int n, double* X, long long fs, const double* tr,
                               cudaStream_t s);
cudaError_t launch_metrics(const Brick* bricks, int nb, const DevBlock* cblocks, const double* X, long long fsc,
                           const DevBlock* blocks, double* met, long long fs, unsigned* flags, cudaStream_t s);
cudaError_t launch_cast(const double* src, float* dst, long long n, cudaStream_t s);
cudaError_t launch_normals(const Brick* bricks, int nb, const DevBlock* blocks, const double* met, long long fs,
                           double* nrm, cudaStream_t s);
cudaError_t launch_prim(const Brick* bricks, int nb, const DevBlock* blocks, const void* Q, bool fp64,
                        long long fs, void* prim, Gas gas, cudaStream_t s);
// Gradients (u,v,w,T)_(x,y,z) (12 fields, stress_mode = false) or the node
// stress tensor and work + heat-flux vector (9 fields, stress_mode = true),
// over column bricks (at most 32 x 8 nodes in (i, j), any extent along k).
cudaError_t launch_grad(const Brick* bricks, int nb, const DevBlock* blocks, const void* prim, const void* met,
                        bool fp64, long long fs, void* out, bool stress_mode, Gas gas, cudaStream_t s);
// Checking aid: NaN into the ghost shell of nf fields (bricks cover the padded box).
cudaError_t launch_poison(const Brick* bricks, int nb, const DevBlock* blocks, void* p, bool fp64, long long fs,
                          int nf, cudaStream_t s);
// Mixed form: the RK3 stage (Eq. (20)) of the interior bricks from the
// accumulated FP32 divergence A (rk.Qfout must be set).
cudaError_t launch_rk_stage(const Brick* bricks, int nb, const DevBlock* blocks, const float* A, const float* metf,
                            long long fs, Gas gas, const RKArgs& rk, cudaStream_t s);
// Far-field boundary nodes after a stage.
cudaError_t launch_bc_farfield(const NodeItem* items, int n, const DevBlock* blocks, double* Q, float* Qf,
                               float* primf, const double* met, long long fs, Gas gas, cudaStream_t s);
// Ghosts of the stencil state, (prim != null) primitives and (FP64, nst !=
// null) the node state of the sweeps over the bricks of the interior and the
// ghost slabs.
cudaError_t launch_prep(const Brick* bricks, int nb, const DevBlock* blocks, void* Q, bool fp64, long long fs,
                        const void* met, void* prim, double* nst, Gas gas, cudaStream_t s);
cudaError_t launch_dt(const Brick* bricks, int nb, const DevBlock* blocks, const double* Q, const double* met,
                      long long fs, Gas gas, unsigned long long* bmax, cudaStream_t s);
cudaError_t launch_rhs_out(DevBlock B, const void* A, const float* Aref, bool fp64, const double* met, long long fs,
                           double* out, cudaStream_t s);
// Fills nf fields (field stride fs) with the per-field values v[0..nf) (device array).
cudaError_t launch_fill_fields(void* p, bool fp64, long long fs, int nf, const double* v, cudaStream_t s);
cudaError_t launch_fill(void* p, bool fp64, long long n, double v, cudaStream_t s);
// dt = cfl / max wave speed per block (or the global minimum) into the block table.
// Local time step of every interior node into dtl (field layout), CFL read from *cfl.
cudaError_t launch_dt_local(const Brick* bricks, int nb, const DevBlock* blocks, const double* Q, const double* met,
                            long long fs, Gas gas, const double* cfl, double* dtl, cudaStream_t s);
cudaError_t launch_setdt(DevBlock* blocks, int nb, const unsigned long long* bmax, const double* cfl, int per_block,
                         double* time_acc, unsigned* flags, cudaStream_t s);
// sums[c] += sum over nodes of R_c^2 (R = -J (A - Aref)).
cudaError_t launch_residual(const Brick* bricks, int nb, const DevBlock* blocks, const void* A, const float* Aref,
                            bool fp64, const double* met, long long fs, double* sums, cudaStream_t s);

}  // namespace hx
