// noalloc.cu -- the inviscid residual of one fully periodic block computed
// without any device allocation: every intermediate (ghost-padded copies of
// the state and metrics, the tile list, the flux accumulator) lives in one
// file-scope static device array.  For callers whose device memory is owned
// by another allocator (a framework's pool holding the whole GPU) or whose
// loop must not call cudaMalloc/cudaFree (those calls can synchronise the
// device and their latency is unbounded).
#include <mutex>
#include <vector>

#include "hx.h"
#include "kernels.h"

using namespace hx;

namespace {

// 32 MiB, enough for a block of about 48^3 nodes; every GPU that loads the library
// keeps this array until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// In host code g_scratch names a host-side stand-in, not device memory: the
// device address is looked up once per device with cudaGetSymbolAddress,
// together with the device's SM count (the persistent grids' size).
std::mutex g_mu;
std::vector<void*> g_addr;
std::vector<int> g_sms;

constexpr int kNA = 8, kVariant = 1;   // flux variant 1: 8 nodes per chunk x 8 lines, every direction

long long rup(long long v, long long m) { return (v + m - 1) / m * m; }

// Line groups of the three sweeps (kNA lines each, sweep origin 0).
__global__ void k_na_setup(DevBlock B, DevBlock* dB, Tile* tiles, int n0, int n1, int n2, int ni, int nj, int nk) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *dB = B;
    const int gi = (ni + kNA - 1) / kNA, gj = (nj + kNA - 1) / kNA;
    if (t < n0) {   // xi sweep: groups of j lines at each k
        tiles[t] = Tile{0, 0, (t % gj) * kNA, t / gj};
    } else if (t < n0 + n1) {   // eta sweep: groups of i lines at each k
        const int u = t - n0;
        tiles[t] = Tile{0, (u % gi) * kNA, 0, u / gi};
    } else if (t < n0 + n1 + n2) {   // zeta sweep: groups of i lines at each j
        const int u = t - n0 - n1;
        tiles[t] = Tile{0, (u % gi) * kNA, u / gi, 0};
    }
}

// Ghost-padded copies of the state (5) and the nine metrics, periodic wrap.
__global__ void k_na_pack(DevBlock B, long long fs, const double* __restrict__ q, const double* __restrict__ met,
                          double* Qp, double* Mp) {
    const int ni = B.n[0], nj = B.n[1], nk = B.n[2];
    const long long np = (long long)(ni + 2 * G) * (nj + 2 * G) * (nk + 2 * G);
    const long long N = (long long)ni * nj * nk;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < np;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % (ni + 2 * G)) - G;
        const long long r = t / (ni + 2 * G);
        const int j = (int)(r % (nj + 2 * G)) - G, k = (int)(r / (nj + 2 * G)) - G;
        const int is = (i + ni) % ni, js = (j + nj) % nj, ks = (k + nk) % nk;
        const long long s = ((long long)ks * nj + js) * ni + is;
        const long long e = node_index(B, i, j, k);
        for (int c = 0; c < 5; ++c) Qp[c * fs + e] = q[c * N + s];
        for (int c = 0; c < 9; ++c) Mp[c * fs + e] = met[c * N + s];
    }
}

__global__ void k_na_out(DevBlock B, long long fs, const double* __restrict__ A, const double* __restrict__ met,
                         double* __restrict__ r) {
    const long long N = (long long)B.n[0] * B.n[1] * B.n[2];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % B.n[0]);
        const long long rr = t / B.n[0];
        const int j = (int)(rr % B.n[1]), k = (int)(rr / B.n[1]);
        const long long e = node_index(B, i, j, k);
        const double J = met[9 * N + t];
        for (int c = 0; c < 5; ++c) r[c * N + t] = -J * A[c * fs + e];
    }
}

int scratch_address(int dev, void** out, int* sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_addr.size() <= dev) {
        g_addr.resize(dev + 1, nullptr);
        g_sms.resize(dev + 1, 0);
    }
    if (!g_addr[dev]) {
        void* p = nullptr;
        int n = 0;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return HX_ERR_CUDA;
        }
        g_addr[dev] = p;
        g_sms[dev] = n;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return HX_OK;
}

// A caller's array must be device (or managed) memory of the current
// device: a pointer to another GPU's memory, or to host memory, would be
// dereferenced by the kernels without peer access.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int hx_euler_rhs_periodic_noalloc(int ni, int nj, int nk, double gamma, const double* q,
                                             const double* met, double* r_out, void* cuda_stream) {
    if (ni < 6 || nj < 6 || nk < 6 || !q || !met || !r_out || !(gamma > 1.0)) return HX_ERR_INVALID_ARG;
    // layout of one padded block (three ghost layers) and the work lists
    DevBlock B{};
    B.n[0] = ni;
    B.n[1] = nj;
    B.n[2] = nk;
    const long long sj = rup(XOFF + ni + G, 8), sk = sj * (nj + 2 * G);
    B.sj = (int)sj;
    B.sk = (int)sk;
    B.base = XOFF + G * sj + G * sk;
    const long long fs = rup(sk * (nk + 2 * G), 64);
    B.lim = fs;
    B.flags = nullptr;
    const int n0 = nk * ((nj + kNA - 1) / kNA);
    const int n1 = nk * ((ni + kNA - 1) / kNA);
    const int n2 = nj * ((ni + kNA - 1) / kNA);
    const size_t off_tiles = 256;
    const size_t off_q = rup(off_tiles + sizeof(Tile) * (size_t)(n0 + n1 + n2), 256);
    const size_t off_m = off_q + 5 * (size_t)fs * 8;
    const size_t off_a = off_m + 9 * (size_t)fs * 8;
    const size_t need = off_a + 5 * (size_t)fs * 8;
    if (need > kScratchBytes) return HX_ERR_INVALID_ARG;   // grid larger than the static scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HX_ERR_CUDA;
    if (!on_device(q, dev) || !on_device(met, dev) || !on_device(r_out, dev)) return HX_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    int sms = 0;
    int rc = scratch_address(dev, (void**)&base, &sms);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DevBlock* dB = (DevBlock*)base;
    Tile* tiles = (Tile*)(base + off_tiles);
    double* Qp = (double*)(base + off_q);
    double* Mp = (double*)(base + off_m);
    double* A = (double*)(base + off_a);

    const int nt = n0 + n1 + n2;
    k_na_setup<<<(nt + 255) / 256, 256, 0, s>>>(B, dB, tiles, n0, n1, n2, ni, nj, nk);
    k_na_pack<<<1024, 256, 0, s>>>(B, fs, q, met, Qp, Mp);
    const Tile* td[3] = {tiles, tiles + n0, tiles + n0 + n1};
    const int nd[3] = {n0, n1, n2};
    for (int d = 0; d < 3; ++d) {
        FluxArgs a{};
        a.blocks = dB;
        a.tiles = td[d];
        a.ntiles = nd[d];
        a.Q = Qp;
        a.met = Mp;
        a.fs = fs;
        a.stress = nullptr;
        a.A = A;
        a.accumulate = d > 0;   // the xi sweep overwrites what the last call left
        a.gas = Gas{gamma, 0.0, 1.0, 1.0, 0.0, 0, 0};
        // sets the kernel's shared-memory opt-in (no allocation) and sizes the grid
        const int cps = flux_ctas_per_sm(true, d, kVariant, false);
        if (cps <= 0) return HX_ERR_CUDA;
        a.grid = nd[d] < sms * cps ? nd[d] : sms * cps;
        if (launch_flux(true, d, kVariant, false, a, s) != cudaSuccess) return HX_ERR_CUDA;
    }
    k_na_out<<<1024, 256, 0, s>>>(B, fs, A, met, r_out);
    if (cudaGetLastError() != cudaSuccess) return HX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HX_ERR_CUDA;
    return HX_OK;
}
