// k_flux_inst.cuh -- instantiates the flux kernel for one working precision
// (HX_FLUX_R) and one direction (HX_FLUX_DIR) in its own translation unit,
// so the heavy instantiations compile in parallel.
#include "k_flux.cuh"
#include "kernels.h"

#define HX_CAT3_(a, b, c) a##b##c
#define HX_CAT3(a, b, c) HX_CAT3_(a, b, c)

namespace hx {

// Candidate (nodes per chunk, lines per CTA): xi (32,8) (16,16) (16,8);
// eta and zeta (8,32) (16,16) (8,16).
constexpr int flux_tp(int dir, int v) { return dir == 0 ? (v == 0 ? 32 : 16) : (v == 1 ? 16 : 8); }
constexpr int flux_na(int dir, int v) { return dir == 0 ? (v == 0 ? 8 : v == 1 ? 16 : 8) : (v == 0 ? 32 : 16); }

namespace {

template <class R, int DIR, int V, bool VISC, bool RK = false>
struct FluxInst {
    static constexpr int TP = flux_tp(DIR, V), NA = flux_na(DIR, V);
    static constexpr size_t smem = FluxLayout<DIR, TP, NA>::template smem_bytes<R, VISC>();
    static int ctas() {
        cudaFuncSetAttribute(k_flux<R, DIR, TP, NA, VISC, RK>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        auto kern = k_flux<R, DIR, TP, NA, VISC, RK>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TP * NA, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    }
    static cudaError_t run(const FluxArgs& a, cudaStream_t s) {
        GasR<R> gs;
        gs.init(a.gas);
        k_flux<R, DIR, TP, NA, VISC, RK><<<a.grid, TP * NA, smem, s>>>(
            a.blocks, a.tiles, a.ntiles, (const R*)a.Q, (const R*)a.met, a.fs, (const R*)a.stress, (R*)a.A,
            a.accumulate, gs, a.rk);
        return cudaGetLastError();
    }
};

}  // namespace

int HX_CAT3(flux_ctas_, HX_FLUX_NAME, HX_FLUX_DIR)(int v, bool visc, bool rk) {
    using R = HX_FLUX_R;
    constexpr int D = HX_FLUX_DIR;
    if (rk && D == 2) {
        switch (v * 2 + (visc ? 1 : 0)) {
            case 0: return FluxInst<R, D, 0, false, D == 2>::ctas();
            case 1: return FluxInst<R, D, 0, true, D == 2>::ctas();
            case 2: return FluxInst<R, D, 1, false, D == 2>::ctas();
            case 3: return FluxInst<R, D, 1, true, D == 2>::ctas();
            case 4: return FluxInst<R, D, 2, false, D == 2>::ctas();
            case 5: return FluxInst<R, D, 2, true, D == 2>::ctas();
        }
        return 0;
    }
    switch (v * 2 + (visc ? 1 : 0)) {
        case 0: return FluxInst<R, D, 0, false>::ctas();
        case 1: return FluxInst<R, D, 0, true>::ctas();
        case 2: return FluxInst<R, D, 1, false>::ctas();
        case 3: return FluxInst<R, D, 1, true>::ctas();
        case 4: return FluxInst<R, D, 2, false>::ctas();
        case 5: return FluxInst<R, D, 2, true>::ctas();
    }
    return 0;
}

cudaError_t HX_CAT3(flux_run_, HX_FLUX_NAME, HX_FLUX_DIR)(int v, bool visc, const FluxArgs& a, cudaStream_t s) {
    using R = HX_FLUX_R;
    constexpr int D = HX_FLUX_DIR;
    if (a.fuse_rk && D == 2) {
        switch (v * 2 + (visc ? 1 : 0)) {
            case 0: return FluxInst<R, D, 0, false, D == 2>::run(a, s);
            case 1: return FluxInst<R, D, 0, true, D == 2>::run(a, s);
            case 2: return FluxInst<R, D, 1, false, D == 2>::run(a, s);
            case 3: return FluxInst<R, D, 1, true, D == 2>::run(a, s);
            case 4: return FluxInst<R, D, 2, false, D == 2>::run(a, s);
            case 5: return FluxInst<R, D, 2, true, D == 2>::run(a, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (v * 2 + (visc ? 1 : 0)) {
        case 0: return FluxInst<R, D, 0, false>::run(a, s);
        case 1: return FluxInst<R, D, 0, true>::run(a, s);
        case 2: return FluxInst<R, D, 1, false>::run(a, s);
        case 3: return FluxInst<R, D, 1, true>::run(a, s);
        case 4: return FluxInst<R, D, 2, false>::run(a, s);
        case 5: return FluxInst<R, D, 2, true>::run(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hx
