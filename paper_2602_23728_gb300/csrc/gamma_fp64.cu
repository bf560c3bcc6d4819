// Three-phonon linewidths, FP64 path on the CUDA cores (paper Sec. "Three-Phonon
// Scattering": Eqs. (phi3_proj), (gamma), (broadening), (lifetime); Sec. "Computational
// Implementation": projection as tensor products, min_frequency selection).
//
// For an irreducible q and the modes nu of q, with q'' = -(q + q') and d = R' - R'' folded
// into the mesh (exp(-i q'.d) only depends on d modulo the mesh):
//   S3  W_q[d][nu][b][c] = sum_{entries with (d,b,c)} Phi3/sqrt(mmm) exp(+i q.R'') e_q[a][nu]
//   S4  M_q(q')[nu][b][c] = sum_d exp(-i q'.d) W_q[d][nu][b][c]                (GEMM over d)
//   S5  X[nu][b][nu''] = sum_c M[nu][b][c] e_q''[c][nu'']                      (GEMM over c)
//       V[nu][nu'][nu''] = sum_b e_q'[b][nu'] X[nu][b][nu'']                   (GEMM over b)
//   S6  gamma[nu] += |V|^2 [(1+n'+n'') g(f-f'-f'') + 2(n'-n'') g(f+f'-f'')] / (2 pi w w' w'')
// which is Phi(q nu, q' nu', q'' nu'') = sum phi exp(-i q'.R') exp(-i q''.R'') e e e / sqrt(mmm)
// regrouped: exp(-i q'.R') exp(+i (q+q').R'') = exp(+i q.R'') exp(-i q'.(R'-R'')).
#include "common.h"
#include "gamma_common.cuh"

namespace {

// S3: one thread per (segment, nu); segments (d, b, c) are contiguous runs of the sorted COO.
__global__ void fold_kernel(const int32_t* __restrict__ seg_key, const int64_t* __restrict__ seg_start,
                            const int32_t* __restrict__ ent_a, const int32_t* __restrict__ ent_r2,
                            const double* __restrict__ ent_w, int64_t n_seg, double qa, double qb,
                            double qc, const double2* __restrict__ eq, int n, int nu0, int n_nu,
                            double2* __restrict__ W) {
    const int64_t total = n_seg * n_nu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t % n_seg;
        const int nl = (int)(t / n_seg);
        const int nu = nu0 + nl;
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t k = seg_start[s]; k < seg_start[s + 1]; ++k) {
            const double x = 2.0 * (qa * ent_r2[3 * k] + qb * ent_r2[3 * k + 1] + qc * ent_r2[3 * k + 2]);
            double sn, cs;
            sincospi(x, &sn, &cs);                           // exp(+i pi x)
            const double2 e = eq[(int64_t)ent_a[k] * n + nu];
            const double w = ent_w[k];
            acc.x += w * (cs * e.x - sn * e.y);
            acc.y += w * (cs * e.y + sn * e.x);
        }
        const int d = seg_key[3 * s], b = seg_key[3 * s + 1], c = seg_key[3 * s + 2];
        W[(((int64_t)d * n_nu + nl) * n + b) * n + c] = acc;
    }
}

// P[q'][d] = exp(-2 pi i k'.d / mesh) for every mesh point and folded difference.
__global__ void phase_kernel(const int32_t* __restrict__ d_int, int n_d, int m1, int m2, int m3,
                             double2* __restrict__ P) {
    const int nq = m1 * m2 * m3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nq * n_d; t += gridDim.x * blockDim.x) {
        const int qp = t / n_d, d = t % n_d;
        const int k1 = qp / (m2 * m3), k2 = (qp / m3) % m2, k3 = qp % m3;
        // reduce each product mod the mesh so the argument stays exact
        const int a1 = (k1 * d_int[3 * d]) % m1, a2 = (k2 * d_int[3 * d + 1]) % m2,
                  a3 = (k3 * d_int[3 * d + 2]) % m3;
        const double x = 2.0 * ((double)a1 / m1 + (double)a2 / m2 + (double)a3 / m3);
        double s, c;
        sincospi(x, &s, &c);
        P[t] = make_double2(c, -s);
    }
}

// q'' = -(q + q') folded into the mesh, for every q'.
__global__ void third_index_kernel(int iq, int m1, int m2, int m3, int32_t* __restrict__ qpp) {
    const int nq = m1 * m2 * m3;
    for (int qp = blockIdx.x * blockDim.x + threadIdx.x; qp < nq; qp += gridDim.x * blockDim.x)
        qpp[qp] = phx_third_index(iq, qp, m1, m2, m3);
}

// S6 for one tile of q': one CTA per (q' in tile, nu), sum over (nu', nu'').
__global__ void __launch_bounds__(256)
epilogue_fp64_kernel(const double2* __restrict__ V, int t0, int iq, int n, int nu0, int n_nu,
                     const double* __restrict__ freq, const double* __restrict__ nB,
                     const int32_t* __restrict__ qpp, GammaParams gp, double* __restrict__ gacc,
                     double* __restrict__ wacc) {
    const int b = blockIdx.x / n_nu, nl = blockIdx.x % n_nu;
    const int qp = t0 + b;
    const int q2 = qpp[qp];
    const double f0 = freq[(int64_t)iq * n + nu0 + nl];
    const double2* v = V + ((int64_t)b * n_nu + nl) * n * n;
    double g = 0.0, w = 0.0;
    if (f0 >= gp.f_min) {
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int j1 = t / n, j2 = t % n;
            const double f1 = freq[(int64_t)qp * n + j1], f2 = freq[(int64_t)q2 * n + j2];
            const double wt = phx_pair_weight(f0, f1, f2, nB[(int64_t)qp * n + j1],
                                              nB[(int64_t)q2 * n + j2], gp);
            if (wt != 0.0) {
                const double2 x = v[t];
                g += (x.x * x.x + x.y * x.y) * wt;
                w += wt;
            }
        }
    }
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        g += __shfl_xor_sync(0xffffffffu, g, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = g; red[1][threadIdx.x >> 5] = w; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sg = 0.0, sw = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { sg += red[0][k]; sw += red[1][k]; }
        atomicAdd(&gacc[nu0 + nl], sg);
        if (wacc) atomicAdd(&wacc[nu0 + nl], sw);
    }
}

// Off-diagonal scattering rows (Eq. gamma1) of the same tile: CTA (q' in tile, nu) adds, for
// every element (nu', nu'') with weight w = |V|^2 x pair weight, w f'/f to column (q', nu') and
// w f''/f to column (q'', nu'') of row (q, nu), folded onto the time-reversal representatives.
__global__ void __launch_bounds__(256)
g1_fp64_kernel(const double2* __restrict__ V, int t0, int iq, int n, int nu0, int n_nu,
               const double* __restrict__ freq, const double* __restrict__ nB, const int32_t* __restrict__ qpp,
               GammaParams gp, double* __restrict__ g1, int64_t ld, int64_t row0,
               const int32_t* __restrict__ tr_code, double scale) {
    const int b = blockIdx.x / n_nu, nl = blockIdx.x % n_nu;
    const int qp = t0 + b;
    const int q2 = qpp[qp];
    const double f0 = freq[(int64_t)iq * n + nu0 + nl];
    if (!(f0 >= gp.f_min)) return;
    const double2* v = V + ((int64_t)b * n_nu + nl) * n * n;
    double* row = g1 + (row0 + nl) * ld;
    const int c1 = tr_code[qp], c2 = tr_code[q2];
    // column (q', nu'): sum over nu''
    if (c1 != 0)
        for (int j1 = threadIdx.x; j1 < n; j1 += blockDim.x) {
            const double f1 = freq[(int64_t)qp * n + j1], n1 = nB[(int64_t)qp * n + j1];
            double acc = 0.0;
            for (int j2 = 0; j2 < n; ++j2) {
                const double wt = phx_pair_weight(f0, f1, freq[(int64_t)q2 * n + j2], n1, nB[(int64_t)q2 * n + j2], gp);
                if (wt != 0.0) {
                    const double2 x = v[(int64_t)j1 * n + j2];
                    acc += (x.x * x.x + x.y * x.y) * wt;
                }
            }
            if (acc != 0.0)
                atomicAdd(&row[(int64_t)(abs(c1) - 1) * n + j1], (c1 > 0 ? 1.0 : -1.0) * scale * acc * f1 / f0);
        }
    // column (q'', nu''): sum over nu'
    if (c2 != 0)
        for (int j2 = threadIdx.x; j2 < n; j2 += blockDim.x) {
            const double f2 = freq[(int64_t)q2 * n + j2], n2 = nB[(int64_t)q2 * n + j2];
            double acc = 0.0;
            for (int j1 = 0; j1 < n; ++j1) {
                const double wt = phx_pair_weight(f0, freq[(int64_t)qp * n + j1], f2, nB[(int64_t)qp * n + j1], n2, gp);
                if (wt != 0.0) {
                    const double2 x = v[(int64_t)j1 * n + j2];
                    acc += (x.x * x.x + x.y * x.y) * wt;
                }
            }
            if (acc != 0.0)
                atomicAdd(&row[(int64_t)(abs(c2) - 1) * n + j2], (c2 > 0 ? 1.0 : -1.0) * scale * acc * f2 / f0);
        }
}

}  // namespace

cudaError_t phx_launch_third_index(int iq, const int* mesh, int32_t* qpp, cudaStream_t s) {
    const int nq = mesh[0] * mesh[1] * mesh[2];
    third_index_kernel<<<(nq + 255) / 256, 256, 0, s>>>(iq, mesh[0], mesh[1], mesh[2], qpp);
    return cudaGetLastError();
}

cudaError_t phx_launch_phases(const phx_fc3* f, double* P, cudaStream_t s) {
    const int total = f->nq * f->n_d;
    int blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    phase_kernel<<<blocks, 256, 0, s>>>(f->d_int, f->n_d, f->mesh[0], f->mesh[1], f->mesh[2], (double2*)P);
    return cudaGetLastError();
}

// FP64 path for one call.  gacc/wacc: [n_irr][n] device accumulators (zeroed by the caller).
phx_status phx_gamma_fp64(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                          const double* nB, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                          double* gacc, double* wacc, cudaStream_t s, const G1Target* g1t) {
    const int n = f->n, nq = f->nq;
    const int64_t n2 = (int64_t)n * n, n3 = n2 * n;
    // nu chunk and q' tile sized so that W and the three per-tile buffers stay within ~1.5 GB
    int n_nu = n;
    while (n_nu > 1 && (int64_t)f->n_d * n_nu * n2 * 16 > (int64_t)1 << 30) n_nu = (n_nu + 1) / 2;
    const int64_t R = (int64_t)n_nu * n2;
    int Q = (int)std::max<int64_t>(1, std::min<int64_t>(nq, ((int64_t)1 << 28) / (R * 16)));
    if ((int64_t)Q * n_nu > 65535) Q = std::max(1, 65535 / n_nu);

    double* P = (double*)phx_ws(ctx, "f64.P", (size_t)nq * f->n_d * 16);
    double* W = (double*)phx_ws(ctx, "f64.W", (size_t)f->n_d * R * 16);
    double* M = (double*)phx_ws(ctx, "f64.M", (size_t)Q * R * 16);
    double* X = (double*)phx_ws(ctx, "f64.X", (size_t)Q * R * 16);
    double* V = (double*)phx_ws(ctx, "f64.V", (size_t)Q * R * 16);
    int32_t* qpp = (int32_t*)phx_ws(ctx, "f64.qpp", (size_t)nq * 4);
    int32_t* ident = (int32_t*)phx_ws(ctx, "f64.ident", (size_t)nq * 4);
    if (!P || !W || !M || !X || !V || !qpp || !ident) return PHX_ERR_NOMEM;
    {
        std::vector<int32_t> id(nq);
        for (int i = 0; i < nq; ++i) id[i] = i;
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(ident, id.data(), nq * 4, cudaMemcpyHostToDevice, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    PHX_CUDA_CHECK(ctx, phx_launch_phases(f, P, s));
    ctx->launches += 1;

    for (int si = 0; si < n_irr; ++si) {
        const int iq = irr_host[si];
        int k1 = iq / (f->mesh[1] * f->mesh[2]), k2 = (iq / f->mesh[2]) % f->mesh[1], k3 = iq % f->mesh[2];
        const double qa = (double)k1 / f->mesh[0], qb = (double)k2 / f->mesh[1], qc = (double)k3 / f->mesh[2];
        PHX_CUDA_CHECK(ctx, phx_launch_third_index(iq, f->mesh, qpp, s));
        ctx->launches += 1;
        const double2* eq = (const double2*)evec + (int64_t)iq * n2;
        for (int nu0 = 0; nu0 < n; nu0 += n_nu) {
            const int nn_nu = std::min(n_nu, n - nu0);
            const int64_t Rc = (int64_t)nn_nu * n2;
            PHX_CUDA_CHECK(ctx, cudaMemsetAsync(W, 0, (size_t)f->n_d * Rc * 16, s));
            {
                const int64_t total = f->n_seg * nn_nu;
                int blocks = (int)std::min<int64_t>((total + 255) / 256, 65535);
                const int pf = phx_prof_begin(ctx, s);
                fold_kernel<<<blocks, 256, 0, s>>>(f->seg_key, f->seg_start, f->ent_a, f->ent_r2, f->ent_w,
                                                   f->n_seg, qa, qb, qc, eq, n, nu0, nn_nu, (double2*)W);
                PHX_CUDA_CHECK(ctx, cudaGetLastError());
                phx_prof_end(ctx, pf, s, PHX_K_FOLD, 8.0 * (double)f->nnz * nn_nu, 0.0);
                ctx->launches += 2;
            }
            for (int t0 = 0; t0 < nq; t0 += Q) {
                const int Qt = std::min(Q, nq - t0);
                ZgemmBatch a{};
                // S4: M[Qt x Rc] = P[t0:t0+Qt][n_d] * W[n_d][Rc]
                a.A = P + (int64_t)t0 * f->n_d * 2; a.B = W; a.C = M;
                a.divA = a.divB = 1; a.lda = f->n_d; a.ldb = (int)Rc; a.ldc = (int)Rc;
                const int pg = phx_prof_begin(ctx, s);
                PHX_CUDA_CHECK(ctx, phx_launch_zgemm(Qt, (int)Rc, f->n_d, 1, a, s));
                // S5a: X_b[(nu,b) x nu''] = M_b[(nu,b) x c] * E_{q''}[c x nu'']
                ZgemmBatch g1{};
                g1.A = M; g1.strideA = Rc; g1.divA = 1;
                g1.B = evec; g1.idxB = qpp + t0; g1.strideB = n2; g1.divB = 1;
                g1.C = X; g1.strideC = Rc;
                g1.lda = n; g1.ldb = n; g1.ldc = n;
                PHX_CUDA_CHECK(ctx, phx_launch_zgemm(nn_nu * n, n, n, Qt, g1, s));
                // S5b: V_{b,nu}[nu' x nu''] = E_{q'}^T[nu' x b] * X_{b,nu}[b x nu'']
                ZgemmBatch g2{};
                g2.A = evec; g2.idxA = ident + t0; g2.divA = nn_nu; g2.strideA = n2; g2.transA = 1;
                g2.B = X; g2.strideB = n2; g2.divB = 1;
                g2.C = V; g2.strideC = n2;
                g2.lda = n; g2.ldb = n; g2.ldc = n;
                PHX_CUDA_CHECK(ctx, phx_launch_zgemm(n, n, n, Qt * nn_nu, g2, s));
                phx_prof_end(ctx, pg, s, PHX_K_FP64_GEMM,
                             8.0 * (double)Qt * Rc * ((double)f->n_d + 2.0 * n), 0.0);
                const int pe = phx_prof_begin(ctx, s);
                // S6
                epilogue_fp64_kernel<<<Qt * nn_nu, 256, 0, s>>>((const double2*)V, t0, iq, n, nu0, nn_nu, freq,
                                                                nB, qpp, gp, gacc + (int64_t)si * n,
                                                                wacc ? wacc + (int64_t)si * n : nullptr);
                PHX_CUDA_CHECK(ctx, cudaGetLastError());
                if (g1t) {
                    g1_fp64_kernel<<<Qt * nn_nu, 256, 0, s>>>((const double2*)V, t0, iq, n, nu0, nn_nu, freq, nB, qpp,
                                                              gp, (double*)g1t->mat, g1t->ld, (int64_t)si * n + nu0,
                                                              g1t->tr_code, g1t->scale);
                    PHX_CUDA_CHECK(ctx, cudaGetLastError());
                    ctx->launches += 1;
                }
                phx_prof_end(ctx, pe, s, PHX_K_FP64_EPI, 0.0, 16.0 * (double)Qt * Rc);
                ctx->launches += 4;
            }
        }
    }
    return PHX_OK;
}
