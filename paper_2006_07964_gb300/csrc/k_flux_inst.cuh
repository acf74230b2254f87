// k_flux_inst.cuh -- instantiates the flux kernel for one working precision
// (HX_FLUX_R) and one direction (HX_FLUX_DIR) in its own translation unit,
// so the heavy instantiations compile in parallel.
#include <type_traits>

#include "k_flux.cuh"
#include "k_flux2.cuh"
#include "kernels.h"

#define HX_CAT3_(a, b, c) a##b##c
#define HX_CAT3(a, b, c) HX_CAT3_(a, b, c)

namespace hx {

// Candidate (nodes per chunk, lines per CTA): xi (32,8) (8,8) (16,8);
// eta and zeta (8,32) (8,8) (8,16).
constexpr int flux_tp(int dir, int v) { return dir == 0 ? (v == 0 ? 32 : v == 1 ? 8 : 16) : 8; }
constexpr int flux_na(int dir, int v) { return v == 1 ? 8 : dir == 0 ? 8 : (v == 0 ? 32 : 16); }

namespace {

// The mixed form's sweeps of the modified scheme (FP32, SCH 0) run the
// two-lines-per-thread kernel of k_flux2.cuh (TP x NA/2 threads); the FP64
// form and the original scheme run k_flux.  Only the FP64 form fuses the RK
// stage into its zeta sweep.  FP64 contexts read the sweeps' stored unit
// normals and the node state of k_prep (NRM); a call without them (the
// allocation-free Euler residual) runs the FP64 Euler sweep that forms both.
template <class R, int DIR, int V, bool VISC, bool RK = false, int SCH = 0>
struct FluxInst {
    static constexpr int TP = flux_tp(DIR, V), NA = flux_na(DIR, V);
    static constexpr bool PAIR = std::is_same<R, float>::value && SCH == 0;
    static constexpr bool F64 = std::is_same<R, double>::value;
    static constexpr bool PLAIN64 = F64 && !VISC && !RK && SCH == 0;   // FP64 without stored normals exists
    static_assert(!RK || F64, "the fused RK stage is the FP64 form's");
    static constexpr int NT = PAIR ? TP * NA / 2 : TP * NA;
    static constexpr size_t smem = PAIR ? Flux2Layout<DIR, TP, NA / 2>::smem_bytes(VISC)
                                        : FluxLayout<DIR, TP, NA>::template smem_bytes<R, VISC, F64, SCH == 0>();
    static constexpr size_t smem_plain = FluxLayout<DIR, TP, NA>::template smem_bytes<R, VISC, false, SCH == 0>();
    static auto kernel() {
        if constexpr (PAIR)
            return k_flux2<DIR, TP, NA / 2, VISC>;
        else
            return k_flux<R, DIR, TP, NA, VISC, RK, SCH, F64>;
    }
    static bool opt_in(const void* kern, size_t bytes) {
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }
    static int ctas() {
        auto kern = kernel();
        if constexpr (PLAIN64) {
            if (!opt_in((const void*)k_flux<R, DIR, TP, NA, VISC, RK, SCH, false>, smem_plain)) return 0;
        }
        if (!opt_in((const void*)kern, smem)) return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    }
    static cudaError_t run(const FluxArgs& a, cudaStream_t s) {
        GasR<R> gs;
        gs.init(a.gas);
        if constexpr (PAIR) {
            k_flux2<DIR, TP, NA / 2, VISC><<<a.grid, NT, smem, s>>>(
                a.blocks, a.tiles, a.ntiles, (const float*)a.Q, (const float*)a.met, a.fs, (const float*)a.stress,
                (float*)a.A, a.accumulate, gs);
        } else if constexpr (F64) {
            if (a.nrm) {
                if (!a.nst) return cudaErrorInvalidValue;   // the node state comes with the normals
                k_flux<R, DIR, TP, NA, VISC, RK, SCH, true><<<a.grid, NT, smem, s>>>(
                    a.blocks, a.tiles, a.ntiles, (const R*)a.Q, (const R*)a.met, (const R*)a.nrm, (const R*)a.nst,
                    a.fs, (const R*)a.stress, (R*)a.A, a.accumulate, gs, a.rk);
            } else if constexpr (PLAIN64) {
                k_flux<R, DIR, TP, NA, VISC, RK, SCH, false><<<a.grid, NT, smem_plain, s>>>(
                    a.blocks, a.tiles, a.ntiles, (const R*)a.Q, (const R*)a.met, nullptr, nullptr, a.fs,
                    (const R*)a.stress, (R*)a.A, a.accumulate, gs, a.rk);
            } else {
                return cudaErrorInvalidValue;   // FP64 sweeps other than the Euler one need the stored normals
            }
        } else {
            k_flux<R, DIR, TP, NA, VISC, RK, SCH, false><<<a.grid, NT, smem, s>>>(
                a.blocks, a.tiles, a.ntiles, (const R*)a.Q, (const R*)a.met, nullptr, nullptr, a.fs,
                (const R*)a.stress, (R*)a.A, a.accumulate, gs, a.rk);
        }
        return cudaGetLastError();
    }
};

}  // namespace

namespace {

template <int SCH, class F>
auto pick(int v, bool visc, bool rk, F&& f) {
    using R = HX_FLUX_R;
    constexpr int D = HX_FLUX_DIR;
    constexpr bool CanRK = D == 2 && std::is_same<R, double>::value;   // the mixed form ends its stages in k_rk_stage
    const int key = v * 4 + (visc ? 2 : 0) + (rk && CanRK ? 1 : 0);
    switch (key) {
        case 0: return f(FluxInst<R, D, 0, false, false, SCH>{});
        case 1: return f(FluxInst<R, D, 0, false, CanRK, SCH>{});
        case 2: return f(FluxInst<R, D, 0, true, false, SCH>{});
        case 3: return f(FluxInst<R, D, 0, true, CanRK, SCH>{});
        case 4: return f(FluxInst<R, D, 1, false, false, SCH>{});
        case 5: return f(FluxInst<R, D, 1, false, CanRK, SCH>{});
        case 6: return f(FluxInst<R, D, 1, true, false, SCH>{});
        case 7: return f(FluxInst<R, D, 1, true, CanRK, SCH>{});
        case 8: return f(FluxInst<R, D, 2, false, false, SCH>{});
        case 9: return f(FluxInst<R, D, 2, false, CanRK, SCH>{});
        case 10: return f(FluxInst<R, D, 2, true, false, SCH>{});
        default: return f(FluxInst<R, D, 2, true, CanRK, SCH>{});
    }
}

}  // namespace

int HX_CAT3(flux_ctas_, HX_FLUX_NAME, HX_FLUX_DIR)(int v, bool visc, bool rk, int scheme) {
    if (v < 0 || v > 2) return 0;
    auto f = [](auto inst) { return decltype(inst)::ctas(); };
    return scheme ? pick<1>(v, visc, rk, f) : pick<0>(v, visc, rk, f);
}

cudaError_t HX_CAT3(flux_run_, HX_FLUX_NAME, HX_FLUX_DIR)(int v, bool visc, const FluxArgs& a, cudaStream_t s) {
    if (v < 0 || v > 2) return cudaErrorInvalidValue;
    auto f = [&](auto inst) { return decltype(inst)::run(a, s); };
    return a.scheme ? pick<1>(v, visc, a.fuse_rk != 0, f) : pick<0>(v, visc, a.fuse_rk != 0, f);
}

}  // namespace hx
