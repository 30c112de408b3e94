// lbm_noalloc.cu -- lbm_reduce_fields_noalloc: the FP64 diagnostics reduction
// for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a host
// framework that owns every byte of device memory through its own pool (a raw
// cudaMalloc would bypass the pool and can fail or fragment it), or in a
// latency-critical loop where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable. Such a caller hands in device buffers it
// already owns (the fields and the 14-value result) and nothing else is
// allocated: the per-block partial sums live in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
#include <cmath>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerBlock = 8192;                 // cells one block reduces
constexpr int kMaxBlocks = 2048;                     // blocks the scratch array holds
constexpr long long kMaxCells = (long long)kCellsPerBlock * kMaxBlocks;   // 16,777,216
constexpr int kQ = lbm::kDiagQuantities;

// Per-block partial sums of the last call (2048 x 14 doubles = 229 KB per GPU;
// each device holds its own copy). Every call overwrites the slots of the blocks
// it launches before reading them, so nothing needs clearing; two calls in
// flight at once on the same device share this array and race.
static __device__ __align__(256) double g_partials[kMaxBlocks * kQ];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};   // device address of g_partials, per device

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Quantities in the order of the context diagnostics: 0 sum phi, 1 sum rho,
// 2 kinetic energy, 3 max |u|, 4 sum phi x, 5 sum phi y, 6 sum (1-phi) x,
// 7 sum (1-phi) y, 8 sum P over phi > 1-1e-3, 9 cells there, 10 sum P over
// phi < 1e-3, 11 cells there, 12 non-finite cells, 13 sum (1 - phi).
__global__ void __launch_bounds__(kThreads) reduce_fields_blocks(const double* __restrict__ f,
                                                                 int nx, long long n,
                                                                 double* __restrict__ partials) {
    const double* phi = f;
    const double* ux = f + n;
    const double* uy = f + 2 * n;
    const double* rho = f + 3 * n;
    const double* P = f + 4 * n;
    double acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
    const long long begin = (long long)blockIdx.x * kCellsPerBlock;
    const long long end = begin + kCellsPerBlock < n ? begin + kCellsPerBlock : n;
    for (long long c = begin + threadIdx.x; c < end; c += kThreads) {
        const double p = phi[c], u = ux[c], v = uy[c], r = rho[c], Pl = P[c];
        const double x = double(c % nx), y = double(c / nx);
        const double uu = u * u + v * v;
        const bool fin = isfinite(p) && isfinite(u) && isfinite(v) && isfinite(r) && isfinite(Pl);
        acc[0] += p;
        acc[1] += r;
        acc[2] += 0.5 * r * uu;
        acc[3] = fmax(acc[3], sqrt(uu));
        acc[4] += p * x;
        acc[5] += p * y;
        acc[6] += (1.0 - p) * x;
        acc[7] += (1.0 - p) * y;
        if (p > 1.0 - 1e-3) { acc[8] += Pl; acc[9] += 1.0; }
        if (p < 1e-3) { acc[10] += Pl; acc[11] += 1.0; }
        if (!fin) acc[12] += 1.0;
        acc[13] += 1.0 - p;
    }
    __shared__ double red[kQ][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const double v = (q == 3) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kQ) {
        const int q = threadIdx.x;
        double v = red[q][0];
        for (int k = 1; k < kThreads / 32; ++k) v = (q == 3) ? fmax(v, red[q][k]) : v + red[q][k];
        partials[blockIdx.x * kQ + q] = v;
    }
}

// One block adds the partials of this call's blocks: thread t takes blocks t,
// t + 256, ..., then a fixed shuffle / shared-memory tree combines the threads.
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) reduce_fields_final(const double* __restrict__ partials,
                                                                     int nblocks, double* __restrict__ out) {
    const int t = threadIdx.x;
    double acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
    for (int b = t; b < nblocks; b += kFinalThreads)
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const double x = partials[b * kQ + q];
            acc[q] = (q == 3) ? fmax(acc[q], x) : acc[q] + x;
        }
    __shared__ double red[kQ][kFinalThreads / 32];
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const double v = (q == 3) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (t < kQ) {
        double v = red[t][0];
        for (int w = 1; w < kFinalThreads / 32; ++w) v = (t == 3) ? fmax(v, red[t][w]) : v + red[t][w];
        out[t] = v;
    }
}

// Device address of g_partials on the current device, looked up once per device
// and kept for the life of the process (a cudaDeviceReset after the first call
// would leave it stale; the header says so).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_reduce_fields_noalloc(const double* fields_device, int nx, int ny,
                                                void* cuda_stream, double* out_device) {
    if (!fields_device || !out_device || nx < 1 || ny < 1) return LBM_EINVAL;
    const long long n = (long long)nx * ny;
    if (n > kMaxCells) return LBM_EINVAL;   // beyond the fixed scratch array
    double* partials = nullptr;
    if (scratch_address(&partials) != cudaSuccess) return LBM_ECUDA;
    const int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    reduce_fields_blocks<<<nblocks, kThreads, 0, s>>>(fields_device, nx, n, partials);
    reduce_fields_final<<<1, kFinalThreads, 0, s>>>(partials, nblocks, out_device);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
