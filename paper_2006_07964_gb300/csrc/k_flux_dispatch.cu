// k_flux_dispatch.cu -- selects the flux instantiation for a precision,
// direction, tile-shape variant and Euler / Navier-Stokes.
#include "k_flux.cuh"
#include "kernels.h"

namespace hx {

int flux_ctas_f64_d0(int, bool, bool, int);
int flux_ctas_f64_d1(int, bool, bool, int);
int flux_ctas_f64_d2(int, bool, bool, int);
int flux_ctas_f32_d0(int, bool, bool, int);
int flux_ctas_f32_d1(int, bool, bool, int);
int flux_ctas_f32_d2(int, bool, bool, int);
cudaError_t flux_run_f64_d0(int, bool, const FluxArgs&, cudaStream_t);
cudaError_t flux_run_f64_d1(int, bool, const FluxArgs&, cudaStream_t);
cudaError_t flux_run_f64_d2(int, bool, const FluxArgs&, cudaStream_t);
cudaError_t flux_run_f32_d0(int, bool, const FluxArgs&, cudaStream_t);
cudaError_t flux_run_f32_d1(int, bool, const FluxArgs&, cudaStream_t);
cudaError_t flux_run_f32_d2(int, bool, const FluxArgs&, cudaStream_t);

FluxShape flux_shape(int dir, int v) {
    if (dir == 0) return v == 0 ? FluxShape{32, 8} : v == 1 ? FluxShape{8, 8} : FluxShape{16, 8};
    return v == 0 ? FluxShape{8, 32} : v == 1 ? FluxShape{8, 8} : FluxShape{8, 16};
}

int flux_ctas_per_sm(bool fp64, int dir, int v, bool visc, bool rk, int scheme) {
    if (fp64)
        return dir == 0 ? flux_ctas_f64_d0(v, visc, rk, scheme) : dir == 1 ? flux_ctas_f64_d1(v, visc, rk, scheme)
                                                                         : flux_ctas_f64_d2(v, visc, rk, scheme);
    return dir == 0 ? flux_ctas_f32_d0(v, visc, rk, scheme) : dir == 1 ? flux_ctas_f32_d1(v, visc, rk, scheme)
                                                                     : flux_ctas_f32_d2(v, visc, rk, scheme);
}

cudaError_t launch_flux(bool fp64, int dir, int v, bool visc, const FluxArgs& a, cudaStream_t s) {
    if (a.ntiles <= 0) return cudaSuccess;
    if (fp64)
        return dir == 0 ? flux_run_f64_d0(v, visc, a, s) : dir == 1 ? flux_run_f64_d1(v, visc, a, s)
                                                                  : flux_run_f64_d2(v, visc, a, s);
    return dir == 0 ? flux_run_f32_d0(v, visc, a, s) : dir == 1 ? flux_run_f32_d1(v, visc, a, s)
                                                              : flux_run_f32_d2(v, visc, a, s);
}

}  // namespace hx
