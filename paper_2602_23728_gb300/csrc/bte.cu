// Iterative solution of the linearised BTE (paper Sec. "Boltzmann Transport Equation":
// Eqs. (gamma1), (invBTE), (kappa_general), (rta), (sc_iter)).
//
// One linewidth contraction (FP64 or tensor-core path) accumulates, next to Gamma0 = gamma,
// the off-diagonal matrix Gamma1 of every band of the time-reversal representatives of the
// mesh, columns folded onto the same representatives (mean free paths are odd under time
// reversal).  Gamma1 stays resident in HBM (FP64 for the FP64 path, FP32 for the tensor-core
// precisions) and each iteration
//     lambda^(k+1) = (v - Gamma1 lambda^(k)) / Gamma0
// is one pass over it: an HBM-bound matrix x (R x 3) product, rows split across CTAs, the
// mean-free-path columns staged through shared memory in chunks.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace {

constexpr int kStepThreads = 256;
constexpr int kStepRowsPerWarp = 4;
constexpr int kStepRows = (kStepThreads / 32) * kStepRowsPerWarp;   // rows per CTA
constexpr int kStepChunk = 1024;                                    // columns staged per pass
constexpr int kLdAlign = 128;                                       // row stride multiple (elements)

// 16-byte vector loads: streamed (evict-first) from the matrix, plain from shared memory
__device__ __forceinline__ void ld_stream(const float* p, float (&x)[4]) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld_stream(const double* p, double (&x)[2]) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
}
__device__ __forceinline__ void ld_shared(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld_shared(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
}

// Row data of the unknowns (row r = s * n + nu of representative s): velocity planes, the
// kappa weight (multiplicity x heat capacity), 1/Gamma0 on live rows (0 elsewhere) and the
// RTA start lambda^(0) = v / Gamma0.
__global__ void sc_rows_kernel(int R, int n, const int32_t* __restrict__ reps, const int32_t* __restrict__ tr_code,
                               const double* __restrict__ freq, const double* __restrict__ vel,
                               const double* __restrict__ cV, const double* __restrict__ g0, double f_min, int64_t ld,
                               double* __restrict__ vr, double* __restrict__ wc, double* __restrict__ ig,
                               double* __restrict__ F) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const int q = reps[r / n], nu = r % n;
        const int64_t m = (int64_t)q * n + nu;
        const bool paired = tr_code[q] != 0;          // q != -q: two mesh points share this row
        const bool live = paired && g0[r] > 0.0 && freq[m] >= f_min;
        const double inv = live ? 1.0 / g0[r] : 0.0;
        wc[r] = paired ? 2.0 * cV[m] : cV[m];
        ig[r] = inv;
        for (int a = 0; a < 3; ++a) {
            const double v = vel[m * 3 + a];
            vr[a * ld + r] = v;
            F[a * ld + r] = inv * v;
        }
    }
}

// Fout = (v - G F) / Gamma0 on the rows of this CTA.  Each warp owns kStepRowsPerWarp rows;
// lane l reads 16-byte vectors of a row (4 FP32 or 2 FP64 entries) at columns
// c0 + V (l + 32 k), partial sums per chunk in T, across chunks in FP64.
template <typename T>
__global__ void __launch_bounds__(kStepThreads) sc_step_kernel(const T* __restrict__ G, int64_t ld, int R,
                                                               const double* __restrict__ F,
                                                               const double* __restrict__ vr,
                                                               const double* __restrict__ ig,
                                                               double* __restrict__ Fout) {
    constexpr int V = 16 / sizeof(T);
    __shared__ __align__(16) T sF[3][kStepChunk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * kStepRows + warp * kStepRowsPerWarp;
    const int nr = max(0, min(kStepRowsPerWarp, R - r0));
    double acc[kStepRowsPerWarp][3];
#pragma unroll
    for (int r = 0; r < kStepRowsPerWarp; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
    for (int64_t c0 = 0; c0 < ld; c0 += kStepChunk) {
        const int cn = (int)(ld - c0 < kStepChunk ? ld - c0 : (int64_t)kStepChunk);
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * cn; i += kStepThreads) {
            const int a = i / cn, c = i % cn;
            sF[a][c] = (T)F[a * ld + c0 + c];
        }
        __syncthreads();
        if (nr == 0) continue;
        T part[kStepRowsPerWarp][3];
#pragma unroll
        for (int r = 0; r < kStepRowsPerWarp; ++r) part[r][0] = part[r][1] = part[r][2] = (T)0;
#pragma unroll 2
        for (int c = V * lane; c < cn; c += 32 * V) {
            T fx[V], fy[V], fz[V];
            ld_shared(&sF[0][c], fx);
            ld_shared(&sF[1][c], fy);
            ld_shared(&sF[2][c], fz);
#pragma unroll
            for (int r = 0; r < kStepRowsPerWarp; ++r) {
                if (r >= nr) break;
                T g[V];
                ld_stream(G + (int64_t)(r0 + r) * ld + c0 + c, g);
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    part[r][0] += g[u] * fx[u];
                    part[r][1] += g[u] * fy[u];
                    part[r][2] += g[u] * fz[u];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kStepRowsPerWarp; ++r) {
            acc[r][0] += (double)part[r][0];
            acc[r][1] += (double)part[r][1];
            acc[r][2] += (double)part[r][2];
        }
    }
#pragma unroll
    for (int r = 0; r < kStepRowsPerWarp; ++r) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = acc[r][a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            acc[r][a] = x;
        }
    }
    if (lane < 3 * kStepRowsPerWarp) {
        const int r = lane / 3, a = lane % 3;
        if (r < nr) {
            const int row = r0 + r;
            double s = 0.0;
#pragma unroll
            for (int rr = 0; rr < kStepRowsPerWarp; ++rr)
#pragma unroll
                for (int aa = 0; aa < 3; ++aa)
                    if (rr == r && aa == a) s = acc[rr][aa];
            Fout[a * ld + row] = ig[row] * (vr[a * ld + row] - s);
        }
    }
}

// Matrix-free step: Fout = (v - y) / Gamma0 with y = Gamma1 F accumulated by a contraction pass
__global__ void sc_update_kernel(int R, int64_t ld, const double* __restrict__ y, const double* __restrict__ vr,
                                 const double* __restrict__ ig, double* __restrict__ Fout) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) Fout[a * ld + r] = ig[r] * (vr[a * ld + r] - y[a * ld + r]);
}

// acc9[a][b] += sum_r wc[r] v[r][a] F[r][b]  (Eq. kappa_general before the 1/(N_q V) factor)
__global__ void sc_kappa_kernel(int R, int64_t ld, const double* __restrict__ wc, const double* __restrict__ vr,
                                const double* __restrict__ F, double* __restrict__ acc9) {
    double t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const double w = wc[r];
        const double v[3] = {vr[r], vr[ld + r], vr[2 * ld + r]};
        const double f[3] = {F[r], F[ld + r], F[2 * ld + r]};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) t[3 * a + b] += w * v[a] * f[b];
    }
    __shared__ double red[9][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double x = t[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x][w];
        atomicAdd(&acc9[threadIdx.x], x);
    }
}

// Plane layout [3][ld] -> rows [R][3]
__global__ void sc_planes_to_rows(int R, int64_t ld, const double* __restrict__ F, double* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) out[(int64_t)r * 3 + a] = F[a * ld + r];
}

// Padded matrix [R][ld] of T -> dense [R][R] doubles
template <typename T>
__global__ void sc_matrix_out(int R, int64_t ld, const T* __restrict__ G, double* __restrict__ out) {
    const int64_t total = (int64_t)R * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)G[(i / R) * ld + i % R];
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

}  // namespace

phx_status phx_kappa_sc(phx_ctx* ctx, const phx_cell* cell, const phx_fc3* fc3, const double* freq_thz,
                        const double* evec, const double* vel, double temperature, phx_broadening br,
                        double f_min_thz, int32_t prec, int32_t max_iter, double tol, double* kappa_hist,
                        int32_t* n_iter, int32_t* converged, double* gamma0, double* mfp, double* gamma1,
                        int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!cell || !fc3 || fc3->ctx != ctx || !freq_thz || !evec || !vel || !kappa_hist || !n_iter)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: null argument or foreign fc3 handle");
    if (!(temperature > 0.0) || !std::isfinite(temperature) || !(br.sigma_thz > 0.0) || !(br.window > 0.0) ||
        !(f_min_thz > 0.0) || !std::isfinite(f_min_thz))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: T, sigma, window and f_min must be finite and > 0");
    if (br.shape != PHX_GAUSS && br.shape != PHX_LORENTZ)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: unknown broadening shape %d", br.shape);
    if (prec != PHX_FP64 && prec != PHX_TF32 && prec != PHX_BF16X3)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: unknown precision %d", prec);
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: bad mem flag %d", mem);
    if (max_iter < 0 || !(tol >= 0.0) || !std::isfinite(tol))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: max_iter >= 0 and a finite tol >= 0 required");
    const int n = fc3->n, nq = fc3->nq;
    if (nq < 2)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                             "phx_kappa_sc: a 1x1x1 mesh has no mean free paths (q = -q carries lambda = 0)");
    const double* L = cell->lattice;
    const double vol = std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                                 L[2] * (L[3] * L[7] - L[4] * L[6]));
    if (!(vol > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: zero cell volume");
    if (cell->n_atoms * 3 != n)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: cell has %d atoms, fc3 handle %d modes", cell->n_atoms,
                             n);

    // time-reversal representatives (smallest index of {q, -q}, ascending) and column codes
    const int m1 = fc3->mesh[0], m2 = fc3->mesh[1], m3 = fc3->mesh[2];
    auto neg_of = [&](int q) {
        const int k1 = q / (m2 * m3), k2 = (q / m3) % m2, k3 = q % m3;
        return (((m1 - k1) % m1) * m2 + (m2 - k2) % m2) * m3 + (m3 - k3) % m3;
    };
    std::vector<int32_t> reps, code(nq, 0), pos(nq, -1);
    for (int q = 0; q < nq; ++q)
        if (q <= neg_of(q)) {
            pos[q] = (int)reps.size();
            reps.push_back(q);
        }
    for (int q = 0; q < nq; ++q) {
        const int neg = neg_of(q);
        code[q] = neg == q ? 0 : q < neg ? pos[q] + 1 : -(pos[neg] + 1);
    }
    const int n_tr = (int)reps.size();
    const int64_t R = (int64_t)n_tr * n;
    const int64_t ld = (R + kLdAlign - 1) / kLdAlign * kLdAlign;
    const size_t esz = prec == PHX_FP64 ? 8 : 4;
    const size_t mat_bytes = (size_t)R * ld * esz;
    cudaSetDevice(ctx->device);
    // Gamma1 is held densely: it must fit in the device memory still free, less room for the
    // contraction's own workspace (operands of one q' tile, a few GB to ~25 GB at 192 modes)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
    const size_t reserve = (size_t)32 << 30;
    const size_t have = ctx->ws.count("sc.G1") ? ctx->ws["sc.G1"].second : 0;   // reused in place
    const size_t avail = free_b + have > reserve ? free_b + have - reserve : 0;
    const bool fits = R <= INT32_MAX / 4 && mat_bytes <= avail;
    // matrix-free form: every iteration applies Gamma1 to the current mean free paths inside a
    // contraction pass (tensor-core precisions), so nothing of order R^2 is stored
    const bool mfree = ctx->opt_sc_mfree == 1 || (ctx->opt_sc_mfree == 0 && !fits);
    if (!mfree && !fits)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                             "phx_kappa_sc: Gamma1 of %lld rows needs %.1f GB (%.1f GB of device memory available)",
                             (long long)R, mat_bytes / 1e9, avail / 1e9);
    if (mfree && prec == PHX_FP64)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                             "phx_kappa_sc: the matrix-free iteration runs on the tensor-core precisions (Gamma1 "
                             "of %lld rows: %.1f GB, %.1f GB available)", (long long)R, mat_bytes / 1e9, avail / 1e9);
    if (mfree && gamma1)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_sc: the gamma1 output needs the dense Gamma1");
    if (mfree && R > INT32_MAX / 4)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_kappa_sc: %lld unknowns", (long long)R);

    cudaStream_t s = as_stream(stream);
    const int64_t n2 = (int64_t)n * n;
    const double *d_f = nullptr, *d_e = nullptr, *d_v = nullptr;
    PHX_TRY(phx_stage_in(ctx, "sc.f", freq_thz, (size_t)nq * n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "sc.e", evec, (size_t)nq * n2 * 2, mem, s, &d_e));
    PHX_TRY(phx_stage_in(ctx, "sc.v", vel, (size_t)nq * n * 3, mem, s, &d_v));
    int32_t* d_reps = (int32_t*)phx_ws(ctx, "sc.reps", (size_t)n_tr * 4);
    int32_t* d_code = (int32_t*)phx_ws(ctx, "sc.code", (size_t)nq * 4);
    double* nB = (double*)phx_ws(ctx, "sc.nB", (size_t)nq * n * 8);
    double* cV = (double*)phx_ws(ctx, "sc.cV", (size_t)nq * n * 8);
    double* gacc = (double*)phx_ws(ctx, "sc.gacc", (size_t)R * 8);
    double* g0 = (double*)phx_ws(ctx, "sc.g0", (size_t)R * 8);
    double* vr = (double*)phx_ws(ctx, "sc.vr", (size_t)3 * ld * 8);
    double* wc = (double*)phx_ws(ctx, "sc.wc", (size_t)R * 8);
    double* ig = (double*)phx_ws(ctx, "sc.ig", (size_t)R * 8);
    double* Fa = (double*)phx_ws(ctx, "sc.Fa", (size_t)3 * ld * 8);
    double* Fb = (double*)phx_ws(ctx, "sc.Fb", (size_t)3 * ld * 8);
    double* acc9 = (double*)phx_ws(ctx, "sc.acc9", 9 * 8);
    void* mat = mfree ? nullptr : phx_ws(ctx, "sc.G1", mat_bytes);
    double* yl = mfree ? (double*)phx_ws(ctx, "sc.y", (size_t)3 * ld * 8) : nullptr;
    double* gacc2 = mfree ? (double*)phx_ws(ctx, "sc.gacc2", (size_t)R * 8) : nullptr;
    if (!d_reps || !d_code || !nB || !cV || !gacc || !g0 || !vr || !wc || !ig || !Fa || !Fb || !acc9 ||
        (!mfree && !mat) || (mfree && (!yl || !gacc2)))
        return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_reps, reps.data(), (size_t)n_tr * 4, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_code, code.data(), (size_t)nq * 4, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, phx_launch_occupations(d_f, nq * n, temperature, 0, nB, cV, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(gacc, 0, (size_t)R * 8, s));
    if (!mfree) PHX_CUDA_CHECK(ctx, cudaMemsetAsync(mat, 0, mat_bytes, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(vr, 0, (size_t)3 * ld * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(Fa, 0, (size_t)3 * ld * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(Fb, 0, (size_t)3 * ld * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));
    ctx->launches += 1;

    GammaParams gp{};
    gp.n = n;
    gp.mesh[0] = m1; gp.mesh[1] = m2; gp.mesh[2] = m3;
    gp.nq = nq;
    gp.T = temperature;
    gp.shape = br.shape;
    gp.sigma = br.sigma_thz;
    gp.window = br.window;
    gp.f_min = f_min_thz;
    const double conv = phx::kEvA2AmuToPs2;
    const double pref = phx::kPi * phx::kHbarEvPs * conv * conv * conv / (8.0 * nq);
    G1Target tgt{mat, ld, d_code, pref};
    if (prec == PHX_FP64)
        PHX_TRY(phx_gamma_fp64(ctx, fc3, d_f, d_e, nB, reps.data(), n_tr, gp, gacc, nullptr, s, &tgt));
    else   // matrix-free: the first pass gives Gamma0 only
        PHX_TRY(phx_gamma_tc(ctx, fc3, d_f, d_e, nB, reps.data(), n_tr, gp, prec, gacc, nullptr, s, mfree ? nullptr : &tgt));
    PHX_CUDA_CHECK(ctx, phx_launch_finalize((int)R, n, d_reps, d_f, gacc, nullptr, pref, 0.0, f_min_thz, g0, nullptr, s));
    const int rblocks = (int)std::min<int64_t>((R + 255) / 256, 4096);
    sc_rows_kernel<<<rblocks, 256, 0, s>>>((int)R, n, d_reps, d_code, d_f, d_v, cV, g0, f_min_thz, ld, vr, wc, ig, Fa);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 2;

    const double kconv = phx::kEvPsAKToWmK / ((double)nq * vol);
    const int kblocks = (int)std::min<int64_t>((R + 255) / 256, 1024);
    const int sblocks = (int)((R + kStepRows - 1) / kStepRows);
    double h[9];
    auto kappa_of = [&](const double* F, double* out) -> phx_status {
        PHX_CUDA_CHECK(ctx, cudaMemsetAsync(acc9, 0, 72, s));
        sc_kappa_kernel<<<kblocks, 256, 0, s>>>((int)R, ld, wc, vr, F, acc9);
        PHX_CUDA_CHECK(ctx, cudaGetLastError());
        ctx->launches += 1;
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(h, acc9, 72, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        for (int k = 0; k < 9; ++k) {
            out[k] = h[k] * kconv;
            if (!std::isfinite(out[k]))
                return phx_set_error(ctx, PHX_ERR_NUMERIC, "phx_kappa_sc: non-finite kappa (the iteration diverged)");
        }
        return PHX_OK;
    };
    PHX_TRY(kappa_of(Fa, kappa_hist));
    {
        int32_t st = 0;
        PHX_CUDA_CHECK(ctx, cudaMemcpy(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost));
        if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_kappa_sc: a device wait gave up (status %d)", st);
    }
    double* Fcur = Fa;
    double* Fnext = Fb;
    int done = 0;
    int conv_flag = 0;
    for (int it = 1; it <= max_iter; ++it) {
        if (mfree) {
            // y = Gamma1 F from one contraction pass (Gamma0 recomputed into a scratch row)
            PHX_CUDA_CHECK(ctx, cudaMemsetAsync(yl, 0, (size_t)3 * ld * 8, s));
            PHX_CUDA_CHECK(ctx, cudaMemsetAsync(gacc2, 0, (size_t)R * 8, s));
            G1Target app{nullptr, ld, d_code, pref, Fcur, yl};
            PHX_TRY(phx_gamma_tc(ctx, fc3, d_f, d_e, nB, reps.data(), n_tr, gp, prec, gacc2, nullptr, s, &app));
            sc_update_kernel<<<rblocks, 256, 0, s>>>((int)R, ld, yl, vr, ig, Fnext);
            PHX_CUDA_CHECK(ctx, cudaGetLastError());
            ctx->launches += 1;
            int32_t st = 0;
            PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
            PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
            if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_kappa_sc: a device wait gave up (status %d)", st);
        } else {
            const int pf = phx_prof_begin(ctx, s);
            if (prec == PHX_FP64)
                sc_step_kernel<double><<<sblocks, kStepThreads, 0, s>>>((const double*)mat, ld, (int)R, Fcur, vr, ig, Fnext);
            else
                sc_step_kernel<float><<<sblocks, kStepThreads, 0, s>>>((const float*)mat, ld, (int)R, Fcur, vr, ig, Fnext);
            PHX_CUDA_CHECK(ctx, cudaGetLastError());
            phx_prof_end(ctx, pf, s, PHX_K_SC_STEP, 6.0 * (double)R * R, (double)R * ld * esz);
            ctx->launches += 1;
        }
        std::swap(Fcur, Fnext);
        double* kk = kappa_hist + 9 * it;
        PHX_TRY(kappa_of(Fcur, kk));
        done = it;
        const double t_old = (kk[-9] + kk[-5] + kk[-1]) / 3.0, t_new = (kk[0] + kk[4] + kk[8]) / 3.0;
        if (std::fabs(t_new - t_old) < tol * std::fabs(t_old)) {
            conv_flag = 1;
            break;
        }
    }
    *n_iter = done;
    if (converged) *converged = conv_flag;

    if (gamma0) {
        if (mem == PHX_MEM_HOST)
            PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma0, g0, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
        else
            PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma0, g0, (size_t)R * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (mfp) {
        double* o = nullptr;
        PHX_TRY(phx_stage_out_buf(ctx, "sc.mfp", mfp, (size_t)R * 3, mem, &o));
        sc_planes_to_rows<<<rblocks, 256, 0, s>>>((int)R, ld, Fcur, o);
        PHX_CUDA_CHECK(ctx, cudaGetLastError());
        ctx->launches += 1;
        if (mem == PHX_MEM_HOST) PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(mfp, o, (size_t)R * 24, cudaMemcpyDeviceToHost, s));
    }
    if (gamma1) {
        double* o = nullptr;
        PHX_TRY(phx_stage_out_buf(ctx, "sc.g1out", gamma1, (size_t)R * R, mem, &o));
        const int mb = (int)std::min<int64_t>((R * R + 255) / 256, 8192);
        if (prec == PHX_FP64)
            sc_matrix_out<double><<<mb, 256, 0, s>>>((int)R, ld, (const double*)mat, o);
        else
            sc_matrix_out<float><<<mb, 256, 0, s>>>((int)R, ld, (const float*)mat, o);
        PHX_CUDA_CHECK(ctx, cudaGetLastError());
        ctx->launches += 1;
        if (mem == PHX_MEM_HOST)
            PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma1, o, (size_t)R * R * 8, cudaMemcpyDeviceToHost, s));
    }
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    return PHX_OK;
}
