// Allocation-free RTA conductivity (phx_kappa_rta_noalloc).
//
// Some callers cannot allocate device memory when they call in: a host framework whose
// caching allocator already owns nearly all of the GPU's memory, or a time-critical loop
// in which cudaMalloc/cudaFree (which can synchronise the whole device) are not allowed.
// This entry point serves them.  It needs no context (creating one allocates) and calls no
// allocator: its only scratch is the file-scope device array below, which every GPU that
// loads the library holds until the process exits.
//
// Scratch: one row of 9 partial sums per CTA (kMaxBlocks rows).  Each CTA reduces a fixed
// slice of kModesPerBlock modes and writes its row unconditionally, and a second kernel sums
// the rows in a fixed order into the caller's kappa buffer, so nothing in the array has to
// start at zero and the result does not depend on scheduling.  The array is shared by all
// calls on a device and keeps the last call's contents: calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.
#include <mutex>

#include "common.h"

namespace {

constexpr int kMaxBlocks = 2048;
constexpr int kModesPerBlock = 2048;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 2048 x 9 doubles = 144 KiB per device.
static __device__ __align__(256) double g_kappa_partials[kMaxBlocks * 9];

__device__ __forceinline__ double heat_capacity(double f, double T, int classic) {
    if (!(f > 0.0)) return 0.0;
    if (classic) return phx::kKbEvK;
    const double x = phx::kHbarEvPs * f * phx::kTwoPi / (phx::kKbEvK * T);
    const double em = expm1(x);
    return phx::kKbEvK * x * x * (1.0 / em) * (1.0 + 1.0 / em);
}

__global__ void __launch_bounds__(kThreads)
kappa_partials_kernel(int count, const double* __restrict__ freq, const double* __restrict__ vel,
                      const double* __restrict__ vv, const double* __restrict__ g, double T, double f_min,
                      int classic, double* __restrict__ partials) {
    double t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int begin = blockIdx.x * kModesPerBlock;
    const int end = min(begin + kModesPerBlock, count);
    for (int i = begin + threadIdx.x; i < end; i += blockDim.x) {
        const double f = freq[i], gi = g[i];
        if (!(f >= f_min) || !(gi > 0.0)) continue;
        const double w = heat_capacity(f, T, classic) / gi;
        if (vv) {
            for (int k = 0; k < 9; ++k) t[k] += w * vv[(int64_t)i * 9 + k];
        } else {
            const double* v = vel + (int64_t)i * 3;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) t[3 * a + b] += w * v[a] * v[b];
        }
    }
    __shared__ double red[9][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double v = t[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[threadIdx.x][w];
        partials[blockIdx.x * 9 + threadIdx.x] = v;
    }
}

__global__ void kappa_final_kernel(int n_blocks, const double* __restrict__ partials, double scale,
                                   double* __restrict__ kappa) {
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int b = 0; b < n_blocks; ++b) v += partials[b * 9 + threadIdx.x];
        kappa[threadIdx.x] = v * scale;
    }
}

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_kappa_partials);
        if (e != cudaSuccess) return e;
        g_partials_ptr[dev] = (double*)p;
    }
    *out = g_partials_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" phx_status phx_kappa_rta_noalloc(const phx_cell* cell, int32_t nq, int32_t n, const double* freq_thz,
                                           const double* vel, const double* vv, const double* gamma_full,
                                           double temperature, double f_min_thz, int32_t is_classic,
                                           double* kappa_dev, void* stream) {
    if (!cell || nq <= 0 || n <= 0 || !freq_thz || (!vel && !vv) || !gamma_full || !kappa_dev)
        return PHX_ERR_INVALID;
    if (!(temperature > 0.0)) return PHX_ERR_INVALID;
    const int64_t count = (int64_t)nq * n;
    if (count > (int64_t)kMaxBlocks * kModesPerBlock) return PHX_ERR_UNSUPPORTED;
    const double* L = cell->lattice;
    const double vol = fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                            L[2] * (L[3] * L[7] - L[4] * L[6]));
    if (!(vol > 0.0)) return PHX_ERR_INVALID;
    double* partials = nullptr;
    if (scratch_for_current_device(&partials) != cudaSuccess) {
        cudaGetLastError();
        return PHX_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((count + kModesPerBlock - 1) / kModesPerBlock);
    kappa_partials_kernel<<<blocks, kThreads, 0, s>>>((int)count, freq_thz, vel, vv, gamma_full, temperature,
                                                      f_min_thz, is_classic, partials);
    if (cudaGetLastError() != cudaSuccess) return PHX_ERR_CUDA;
    const double scale = phx::kEvPsAKToWmK / ((double)nq * vol);
    kappa_final_kernel<<<1, 32, 0, s>>>(blocks, partials, scale, kappa_dev);
    if (cudaGetLastError() != cudaSuccess) return PHX_ERR_CUDA;
    return PHX_OK;
}
