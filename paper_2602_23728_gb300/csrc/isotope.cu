// Isotope / mass-variance scattering (paper Sec. "Isotopic Scattering", Eq. (isotope), after
// Tamura): for every band s of the irreducible q,
//   gamma_iso = pi / (2 N_q) w_s^2 sum_{q' s'} delta(w_s - w_{q's'}) sum_i g_i |<e_i(q s)|e_i(q' s')>|^2
// with <e_i|e'_i> = sum_alpha conj(e[3i+alpha]) e'[3i+alpha] and delta(w) = g(f)/(2 pi) (the
// broadening and window of the three-phonon path).  One CTA per (irreducible q, band s); its
// threads walk the (q', s') pairs with s' fastest (coalesced eigenvector columns) and skip the
// pairs outside the window before touching the eigenvectors.  FP64 throughout.
#include <cmath>
#include <vector>

#include "common.h"

namespace {

constexpr int kIsoThreads = 256;

__global__ void __launch_bounds__(kIsoThreads)
isotope_kernel(const double* __restrict__ freq, const double2* __restrict__ evec, const int32_t* __restrict__ irr,
               const double* __restrict__ g_atom, int nq, int n, int shape, double sigma, double lim, double f_min,
               double* __restrict__ gamma) {
    extern __shared__ double2 es[];          // e(q s) column, n entries
    __shared__ double red[kIsoThreads / 32];
    const int si = blockIdx.x / n, s = blockIdx.x % n;
    const int iq = irr[si];
    const int64_t nn = (int64_t)n * n;
    const double f = freq[(int64_t)iq * n + s];
    for (int k = threadIdx.x; k < n; k += blockDim.x) es[k] = evec[(int64_t)iq * nn + (int64_t)k * n + s];
    __syncthreads();
    const int na = n / 3;
    double acc = 0.0;
    if (f >= f_min) {
        const int64_t pairs = (int64_t)nq * n;
        for (int64_t t = threadIdx.x; t < pairs; t += blockDim.x) {
            const int qp = (int)(t / n), sp = (int)(t % n);
            const double fp = freq[(int64_t)qp * n + sp];
            const double df = f - fp;
            if (!(fabs(df) < lim) || fp < f_min) continue;
            double gw;
            if (shape == PHX_GAUSS) {
                gw = exp(-(df * df) / (sigma * sigma)) / (sqrt(phx::kPi) * sigma);
            } else {
                const double h = 0.5 * sigma;
                gw = h / (phx::kPi * (df * df + h * h));
            }
            const double2* ep = evec + (int64_t)qp * nn + sp;
            double a = 0.0;
            for (int i = 0; i < na; ++i) {
                double re = 0.0, im = 0.0;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    const double2 x = es[3 * i + al], y = ep[(int64_t)(3 * i + al) * n];
                    re += x.x * y.x + x.y * y.y;      // conj(x) y
                    im += x.x * y.y - x.y * y.x;
                }
                a += g_atom[i] * (re * re + im * im);
            }
            acc += a * gw;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kIsoThreads / 32; ++w) tot += red[w];
        const double w = phx::kTwoPi * f;
        // delta(w) = g(f) / (2 pi)
        gamma[(int64_t)si * n + s] = f >= f_min ? phx::kPi / (2.0 * nq) * w * w * tot / phx::kTwoPi : 0.0;
    }
}

}  // namespace

extern "C" phx_status phx_gamma_isotope(phx_ctx* ctx, int32_t nq, int32_t n, const double* freq_thz,
                                        const double* evec, const int32_t* irr_q, int32_t n_irr,
                                        const double* g_atom, phx_broadening br, double f_min_thz, double* gamma,
                                        int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (n_irr == 0) return PHX_OK;
    if (nq <= 0 || n <= 0 || n % 3 != 0 || n_irr < 0 || !freq_thz || !evec || !irr_q || !g_atom || !gamma)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: bad argument");
    if (!(br.sigma_thz > 0.0) || !(br.window > 0.0) || !(f_min_thz > 0.0) || !std::isfinite(f_min_thz))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: sigma, window and f_min must be > 0");
    if (br.shape != PHX_GAUSS && br.shape != PHX_LORENTZ)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: unknown broadening shape %d", br.shape);
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: bad mem flag %d", mem);
    const int na = n / 3;
    for (int i = 0; i < na; ++i)
        if (!(g_atom[i] >= 0.0) || !std::isfinite(g_atom[i]))
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: g[%d] must be finite and >= 0", i);
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> irr_h(n_irr);
    if (mem == PHX_MEM_HOST) {
        for (int i = 0; i < n_irr; ++i) irr_h[i] = irr_q[i];
    } else {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(irr_h.data(), irr_q, (size_t)n_irr * 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    for (int i = 0; i < n_irr; ++i)
        if (irr_h[i] < 0 || irr_h[i] >= nq)
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_isotope: irr_q[%d]=%d outside the mesh", i, irr_h[i]);
    const double *d_f = nullptr, *d_e = nullptr;
    const int32_t* d_irr = nullptr;
    PHX_TRY(phx_stage_in(ctx, "iso.f", freq_thz, (size_t)nq * n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "iso.e", evec, (size_t)nq * n * n * 2, mem, s, &d_e));
    PHX_TRY(phx_stage_in(ctx, "iso.irr", irr_q, (size_t)n_irr, mem, s, &d_irr));
    double* d_g = (double*)phx_ws(ctx, "iso.g", (size_t)na * 8);
    double* o_g = nullptr;
    PHX_TRY(phx_stage_out_buf(ctx, "iso.og", gamma, (size_t)n_irr * n, mem, &o_g));
    if (!d_g) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_g, g_atom, (size_t)na * 8, cudaMemcpyHostToDevice, s));
    const size_t smem = (size_t)n * sizeof(double2);
    if (smem > 48 * 1024) {
        if (smem > 200 * 1024)
            return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_gamma_isotope: n = %d modes exceeds shared memory", n);
        PHX_CUDA_CHECK(ctx, cudaFuncSetAttribute(isotope_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    isotope_kernel<<<(unsigned)((int64_t)n_irr * n), kIsoThreads, smem, s>>>(
        d_f, (const double2*)d_e, d_irr, d_g, nq, n, br.shape, br.sigma_thz, br.window * br.sigma_thz, f_min_thz,
        o_g);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 1;
    if (mem == PHX_MEM_HOST) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma, o_g, (size_t)n_irr * n * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    return PHX_OK;
}
