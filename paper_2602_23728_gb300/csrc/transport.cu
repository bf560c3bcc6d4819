// Occupations, linewidth unfolding and the RTA conductivity in FP64 (paper Sec. "Phonon
// Populations and Heat Capacity", Eqs. (bose), (heatcap); Sec. "Boltzmann Transport
// Equation", Eq. (rta); Sec. "Overview of New Capabilities": irreducible results mapped
// back onto the full grid).
#include "common.h"

namespace {

__device__ __forceinline__ void occ(double f, double T, int classic, double* nB, double* c) {
    if (!(f > 0.0)) { *nB = 0.0; *c = 0.0; return; }
    const double x = phx::kHbarEvPs * f * phx::kTwoPi / (phx::kKbEvK * T);
    if (classic) { *nB = 1.0 / x; *c = phx::kKbEvK; return; }
    const double em = expm1(x);
    *nB = 1.0 / em;
    // k_B x^2 e^x / (e^x - 1)^2 = k_B x^2 (1/em + 1/em^2)
    *c = phx::kKbEvK * x * x * (1.0 / em) * (1.0 + 1.0 / em);
}

__global__ void occupations_kernel(const double* __restrict__ freq, int count, double T, int classic,
                                   double* __restrict__ nB, double* __restrict__ cV) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        double a, b;
        occ(freq[i], T, classic, &a, &b);
        if (nB) nB[i] = a;
        if (cV) cV[i] = b;
    }
}

// One CTA per full-mesh point k: degenerate-average the irreducible row of k's orbit.
__global__ void unfold_kernel(int n, const double* __restrict__ freq_full, const int32_t* __restrict__ irr_q,
                              const double* __restrict__ g_irr, const int32_t* __restrict__ full_to_irr,
                              double* __restrict__ g_full) {
    const int k = blockIdx.x;
    const int s = full_to_irr[k];
    const double* f = freq_full + (int64_t)irr_q[s] * n;
    const double* g = g_irr + (int64_t)s * n;
    for (int mu = threadIdx.x; mu < n; mu += blockDim.x) {
        double fm = 0.0;
        for (int i = 0; i < n; ++i) fm = fmax(fm, fabs(f[i]));
        const double tol = phx::kDegenerateRelTol * fmax(fm, 1e-30);
        // groups anchored at their lowest member (frequencies ascend within a q)
        int lo = 0;
        while (true) {
            int hi = lo + 1;
            while (hi < n && f[hi] - f[lo] < tol) ++hi;
            if (mu < hi) {
                double acc = 0.0;
                for (int i = lo; i < hi; ++i) acc += g[i];
                g_full[(int64_t)k * n + mu] = acc / (hi - lo);
                break;
            }
            lo = hi;
        }
    }
}

__global__ void kappa_kernel(int count, const double* __restrict__ freq, const double* __restrict__ vel,
                             const double* __restrict__ vv, const double* __restrict__ g, double T,
                             double f_min, int classic, double* __restrict__ acc9) {
    double t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double f = freq[i], gi = g[i];
        if (!(f >= f_min) || !(gi > 0.0)) continue;
        double nb, c;
        occ(f, T, classic, &nb, &c);
        const double w = c / gi;
        if (vv) {
            for (int k = 0; k < 9; ++k) t[k] += w * vv[(int64_t)i * 9 + k];
        } else {
            const double* v = vel + (int64_t)i * 3;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) t[3 * a + b] += w * v[a] * v[b];
        }
    }
    __shared__ double red[9][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double v = t[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        atomicAdd(&acc9[threadIdx.x], v);
    }
}

__global__ void scale9_kernel(const double* __restrict__ acc, double scale, double* __restrict__ out) {
    if (threadIdx.x < 9) out[threadIdx.x] = acc[threadIdx.x] * scale;
}

}  // namespace

cudaError_t phx_launch_scale9(const double* acc, double scale, double* out, cudaStream_t s) {
    scale9_kernel<<<1, 32, 0, s>>>(acc, scale, out);
    return cudaGetLastError();
}

cudaError_t phx_launch_occupations(const double* freq, int count, double T, int is_classic,
                                   double* nB, double* cV, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int blocks = (count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096;
    occupations_kernel<<<blocks, 256, 0, s>>>(freq, count, T, is_classic, nB, cV);
    return cudaGetLastError();
}

cudaError_t phx_launch_unfold(int n_irr, int nq, int n, const double* freq_full, const int32_t* irr_q,
                              const double* gamma_irr, const int32_t* full_to_irr,
                              double* gamma_full, cudaStream_t s) {
    (void)n_irr;
    if (nq <= 0) return cudaSuccess;
    unfold_kernel<<<nq, 128, 0, s>>>(n, freq_full, irr_q, gamma_irr, full_to_irr, gamma_full);
    return cudaGetLastError();
}

cudaError_t phx_launch_kappa(int nq, int n, const double* freq, const double* vel,
                             const double* vv, const double* gamma_full, double T, double f_min,
                             int is_classic, double* acc9, cudaStream_t s) {
    const int count = nq * n;
    if (count <= 0) return cudaSuccess;
    int blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    kappa_kernel<<<blocks, 256, 0, s>>>(count, freq, vel, vv, gamma_full, T, f_min, is_classic, acc9);
    return cudaGetLastError();
}
