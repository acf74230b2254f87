// alu_peaks.cu -- measured FP64 and FP32 fused-multiply-add throughput of
// the current GPU, the denominators of the benchmark's ALU roofline (the
// FP64 form of the residual path is bound by the FP64 pipe; the mixed
// form's stencil arithmetic runs on the FP32 pipe).
//
// Each thread advances CH independent FMA chains x <- x * a + b (|a| < 1,
// so the values stay bounded and never denormal); the grid fills every SM
// at full occupancy.  Throughput = 2 flops per FMA x FMAs / CUDA-event time
// of one launch after a warm-up launch.
#include <cuda_runtime.h>

#include "hx_probe.h"

namespace {

constexpr int CH = 8;        // independent chains per thread
constexpr int UNROLL = 16;   // FMAs per chain per loop trip
constexpr int NT = 256;

template <class T>
__global__ void __launch_bounds__(NT) k_fma_chains(T* out, int trips, T a, T b) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = T(1e-3) * (T)threadIdx.x + T(c);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    // never true for these inputs; keeps the chains live
    if (s == T(-12345.0)) out[blockIdx.x * NT + threadIdx.x] = s;
}

template <class T>
int time_fma(int grid, int trips, double* tflops, double* ms_out) {
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)grid * NT) != cudaSuccess) return HX_PROBE_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999), b = T(1e-4);
    k_fma_chains<T><<<grid, NT>>>(out, trips / 8 + 1, a, b);   // warm-up
    cudaEventRecord(e0);
    k_fma_chains<T><<<grid, NT>>>(out, trips, a, b);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return HX_PROBE_ERR_CUDA;
    const double flops = 2.0 * CH * UNROLL * (double)trips * (double)grid * NT;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return HX_PROBE_OK;
}

}  // namespace

extern "C" int hx_probe_fma_peaks(double* fp64_tflops, double* fp32_tflops, double* ms) {
    if (!fp64_tflops || !fp32_tflops) return HX_PROBE_ERR_INVALID_ARG;
    int dev = 0, sms = 0, per_sm64 = 0, per_sm32 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm64, k_fma_chains<double>, NT, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_fma_chains<float>, NT, 0) != cudaSuccess ||
        sms <= 0 || per_sm64 <= 0 || per_sm32 <= 0) {
        cudaGetLastError();
        return HX_PROBE_ERR_CUDA;
    }
    // about 0.1 s per launch at the GB300's nominal rates (1.25 and 80 TFLOP/s)
    const double th64 = (double)sms * per_sm64 * NT, th32 = (double)sms * per_sm32 * NT;
    const int trips64 = (int)(1.25e11 * 0.1 / (th64 * 2.0 * CH * UNROLL)) + 1;
    const int trips32 = (int)(8.0e12 * 0.1 / (th32 * 2.0 * CH * UNROLL)) + 1;
    double m[2] = {0, 0};
    int rc = time_fma<double>(sms * per_sm64, trips64, fp64_tflops, &m[0]);
    if (rc) return rc;
    rc = time_fma<float>(sms * per_sm32, trips32, fp32_tflops, &m[1]);
    if (rc) return rc;
    if (ms) {
        ms[0] = m[0];
        ms[1] = m[1];
    }
    return HX_PROBE_OK;
}
