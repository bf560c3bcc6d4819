// FP64 eigensolver for one large real-symmetric dynamical matrix: the Gamma point of a big
// (disordered) cell, Eq. (eigenvalue) of the paper (Sec. "Interatomic Force Constants": the
// real-space problem D eta = omega^2 eta for Gamma-only and amorphous systems).
//
// The batched one-CTA-per-matrix Jacobi solver holds a matrix in shared memory; a 3000 x 3000
// matrix (72 MB) is solved instead in four device phases, all in FP64:
//
//  1. dynmat_gamma_kernel   D = (D + D^T)/2 with D_{ia,jb} = sum_R Phi2(0i, Rj)_{ab}/sqrt(m_i m_j)
//  2. Householder tridiagonalisation, one reflector H_k = I - beta v v^T per step k, two
//     launches per step (symv p = beta A22 v; rank-2 update A22 -= v w^T + w v^T with
//     w = p - (beta p.v / 2) v).  The reflector vector stays in row k of the matrix.
//  3. bisection on Sturm counts (one thread per eigenvalue index) for the tridiagonal T, then
//     inverse iteration (one thread per cluster of eigenvalues closer than 1e-7 ||T||; later
//     members of a cluster are Gram-Schmidt orthogonalised against earlier ones).
//  4. back-transformation Z = H_0 H_1 ... Z_T in a single launch: every CTA owns a strip of
//     four columns and applies all reflectors to it in reverse order.
//
// The output follows the batched solver's conventions: ascending frequencies in THz (signed
// for negative eigenvalues) and columns with the largest-modulus component positive.
#include <cfloat>

#include "common.h"

namespace {

constexpr int kSymvWarps = 8;          // rows per CTA in the symv kernel (one warp per row)
constexpr int kUpdRows = 8;            // rows per CTA in the rank-2 update
constexpr int kStripCols = 4;          // back-transformation columns per CTA
constexpr double kClusterRel = 1e-7;   // eigenvalues closer than this x ||T|| share a thread
constexpr int kInvitIters = 3;

__device__ double block_sum_256(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
    __syncthreads();
    return t;
}

// thread per atom pair (i, j): symmetrised 3x3 block of D at Gamma (images summed)
__global__ void dynmat_gamma_kernel(int na, const double* __restrict__ blk_val,
                                    const int32_t* __restrict__ pair_start, const double* __restrict__ masses,
                                    double* __restrict__ A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)na * na) return;
    const int i = (int)(p / na), j = (int)(p % na);
    const int64_t n = 3 * (int64_t)na;
    double s[9];
    for (int t = 0; t < 9; ++t) s[t] = 0.0;
    for (int b = pair_start[p]; b < pair_start[p + 1]; ++b)
        for (int t = 0; t < 9; ++t) s[t] += blk_val[9 * (int64_t)b + t];
    const int64_t pt = (int64_t)j * na + i;
    for (int b = pair_start[pt]; b < pair_start[pt + 1]; ++b)
        for (int al = 0; al < 3; ++al)
            for (int be = 0; be < 3; ++be) s[3 * al + be] += blk_val[9 * (int64_t)b + 3 * be + al];
    const double sc = 0.5 / sqrt(masses[i] * masses[j]);
    for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) A[(3 * i + al) * n + 3 * j + be] = s[3 * al + be] * sc;
}

// Step k: reflector from x = A[k][k+1..n-1] and p = beta A22 v.  Every CTA recomputes the norm
// of x (it reads A only); CTA 0 records d[k], e[k], beta[k], v0[k].
__global__ void __launch_bounds__(kSymvWarps * 32)
tridiag_symv_kernel(const double* __restrict__ A, int n, int k, double* __restrict__ p, double* __restrict__ d,
                    double* __restrict__ e, double* __restrict__ bet, double* __restrict__ v0s) {
    __shared__ double red[32];
    const int m = n - k - 1;
    const double* x = A + (int64_t)k * n + k + 1;
    double s = 0.0;
    for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) s += x[c] * x[c];
    s = block_sum_256(s, red);
    const double x0 = x[0];
    double alpha, beta, v0;
    if (s == 0.0) {
        alpha = x0; beta = 0.0; v0 = 0.0;
    } else {
        const double nrm = sqrt(x0 * x0 + s);
        alpha = x0 >= 0.0 ? -nrm : nrm;
        v0 = x0 - alpha;
        beta = 2.0 / (v0 * v0 + s);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d[k] = A[(int64_t)k * n + k];
        e[k] = alpha;
        bet[k] = beta;
        v0s[k] = v0;
    }
    if (beta == 0.0) return;          // H = I: the update kernel skips this step
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kSymvWarps + (threadIdx.x >> 5);
    if (r >= m) return;
    const double* row = A + (int64_t)(k + 1 + r) * n + k + 1;
    double acc = lane == 0 ? row[0] * v0 : 0.0;
    for (int c = (lane == 0 ? 32 : lane); c < m; c += 32) acc += row[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) p[r] = beta * acc;
}

// A22 -= v w^T + w v^T, w = p - K v, K = beta (p.v)/2 (every CTA recomputes p.v)
__global__ void __launch_bounds__(256)
tridiag_update_kernel(double* __restrict__ A, int n, int k, const double* __restrict__ p,
                      const double* __restrict__ bet, const double* __restrict__ v0s) {
    __shared__ double red[32];
    const double beta = bet[k];
    if (beta == 0.0) return;
    const int m = n - k - 1;
    const double* x = A + (int64_t)k * n + k + 1;
    const double v0 = v0s[k];
    double s = 0.0;
    for (int c = threadIdx.x; c < m; c += blockDim.x) s += p[c] * (c == 0 ? v0 : x[c]);
    s = block_sum_256(s, red);
    const double K = 0.5 * beta * s;
    const int r0 = blockIdx.x * kUpdRows;
    for (int rr = 0; rr < kUpdRows; ++rr) {
        const int r = r0 + rr;
        if (r >= m) break;
        const double vr = r == 0 ? v0 : x[r];
        const double wr = p[r] - K * vr;
        double* row = A + (int64_t)(k + 1 + r) * n + k + 1;
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
            const double vc = c == 0 ? v0 : x[c];
            const double wc = p[c] - K * vc;
            row[c] -= vr * wc + wr * vc;
        }
    }
}

__global__ void tridiag_finish_kernel(const double* __restrict__ A, int n, double* __restrict__ d,
                                      double* __restrict__ e) {
    d[n - 1] = A[(int64_t)(n - 1) * n + n - 1];
}

__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x, double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int cnt = q < 0.0;
    for (int i = 1; i < n; ++i) {
        q = d[i] - x - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

// e2 = e^2, Gershgorin bounds, ||T|| and pivmin (one CTA)
__global__ void tridiag_bounds_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                                      double* __restrict__ e2, double* __restrict__ info) {
    __shared__ double slo[256], shi[256], se[256];
    double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i < n - 1 ? fabs(e[i]) : 0.0;
        lo = fmin(lo, d[i] - el - er);
        hi = fmax(hi, d[i] + el + er);
        if (i < n - 1) { e2[i] = e[i] * e[i]; emax = fmax(emax, e2[i]); }
    }
    slo[threadIdx.x] = lo; shi[threadIdx.x] = hi; se[threadIdx.x] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < blockDim.x; ++t) { lo = fmin(lo, slo[t]); hi = fmax(hi, shi[t]); emax = fmax(emax, se[t]); }
        const double tn = fmax(fabs(lo), fabs(hi));
        const double pad = 2.0 * DBL_EPSILON * tn * n + 2.0 * DBL_MIN;
        info[0] = lo - pad;
        info[1] = hi + pad;
        info[2] = tn;
        info[3] = DBL_MIN * fmax(1.0, emax);
    }
}

__global__ void bisect_kernel(const double* __restrict__ d, const double* __restrict__ e2, int n,
                              const double* __restrict__ info, double* __restrict__ lam) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double lo = info[0], hi = info[1];
    const double pivmin = info[3];
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin || mid == lo || mid == hi) break;
        if (sturm_count(d, e2, n, mid, pivmin) > m) hi = mid; else lo = mid;
    }
    lam[m] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double start_value(uint64_t seed) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// Inverse iteration with the LU factorisation (partial pivoting) of T - lambda I.  Work arrays
// are interleaved by thread: element i of thread t sits at [i * n + t].
__global__ void invit_kernel(const double* __restrict__ d, const double* __restrict__ e, const double* __restrict__ lam,
                             const double* __restrict__ info, int n, double* __restrict__ Z,
                             double* __restrict__ wdl, double* __restrict__ wdd, double* __restrict__ wdu,
                             double* __restrict__ wdu2, uint8_t* __restrict__ wpiv, int32_t* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double tn = info[2];
    const double ctol = kClusterRel * fmax(tn, DBL_MIN);
    if (t > 0 && lam[t] - lam[t - 1] < ctol) return;           // not the first member of a cluster
    int tend = t + 1;
    while (tend < n && lam[tend] - lam[tend - 1] < ctol) ++tend;
    const double eps3 = 10.0 * DBL_EPSILON * fmax(tn, DBL_MIN);
    const int64_t N = n;
#define W(a, i) a[(int64_t)(i) * N + t]
    double lprev = 0.0;
    for (int j = t; j < tend; ++j) {
        double lj = lam[j];
        if (j > t && lj - lprev < eps3) lj = lprev + eps3;
        lprev = lj;
        // ---- factor T - lj I
        for (int i = 0; i < n; ++i) {
            W(wdd, i) = d[i] - lj;
            if (i < n - 1) { W(wdl, i) = e[i]; W(wdu, i) = e[i]; }
            W(wdu2, i) = 0.0;
        }
        for (int i = 0; i < n - 1; ++i) {
            const double di = W(wdd, i), li = W(wdl, i);
            if (fabs(di) >= fabs(li)) {
                W(wpiv, i) = 0;
                const double piv = di != 0.0 ? di : eps3;
                if (di == 0.0) W(wdd, i) = eps3;
                const double f = li / piv;
                W(wdl, i) = f;
                W(wdd, i + 1) -= f * W(wdu, i);
            } else {
                W(wpiv, i) = 1;
                const double f = di / li;
                W(wdd, i) = li;
                W(wdl, i) = f;
                const double tmp = W(wdu, i);
                W(wdu, i) = W(wdd, i + 1);
                W(wdd, i + 1) = tmp - f * W(wdd, i + 1);
                if (i < n - 2) {
                    W(wdu2, i) = W(wdu, i + 1);
                    W(wdu, i + 1) = -f * W(wdu, i + 1);
                }
            }
        }
        if (W(wdd, n - 1) == 0.0) W(wdd, n - 1) = eps3;
        for (int i = 0; i < n; ++i) if (fabs(W(wdd, i)) < eps3 * 1e-3) W(wdd, i) = copysign(eps3, W(wdd, i));
        // ---- start vector in column j of Z
        for (int i = 0; i < n; ++i) Z[(int64_t)i * N + j] = start_value(((uint64_t)j << 32) ^ (uint64_t)i);
        for (int it = 0; it < kInvitIters; ++it) {
            // solve L U x = b in place (column j of Z)
            for (int i = 0; i < n - 1; ++i) {
                double* bi = &Z[(int64_t)i * N + j];
                double* bn = &Z[(int64_t)(i + 1) * N + j];
                if (W(wpiv, i) == 0) {
                    *bn -= W(wdl, i) * *bi;
                } else {
                    const double tmp = *bi;
                    *bi = *bn;
                    *bn = tmp - W(wdl, i) * *bi;
                }
            }
            double xn1 = Z[(int64_t)(n - 1) * N + j] / W(wdd, n - 1);
            Z[(int64_t)(n - 1) * N + j] = xn1;
            double xn2 = 0.0;
            if (n > 1) {
                xn2 = (Z[(int64_t)(n - 2) * N + j] - W(wdu, n - 2) * xn1) / W(wdd, n - 2);
                Z[(int64_t)(n - 2) * N + j] = xn2;
            }
            for (int i = n - 3; i >= 0; --i) {
                const double xi = (Z[(int64_t)i * N + j] - W(wdu, i) * xn2 - W(wdu2, i) * xn1) / W(wdd, i);
                Z[(int64_t)i * N + j] = xi;
                xn1 = xn2;
                xn2 = xi;
            }
            // scale, orthogonalise against the earlier members of the cluster, normalise
            double amax = 0.0;
            for (int i = 0; i < n; ++i) amax = fmax(amax, fabs(Z[(int64_t)i * N + j]));
            const double sc = amax > 0.0 ? 1.0 / amax : 1.0;
            for (int i = 0; i < n; ++i) Z[(int64_t)i * N + j] *= sc;
            for (int jj = t; jj < j; ++jj) {
                double c = 0.0;
                for (int i = 0; i < n; ++i) c += Z[(int64_t)i * N + jj] * Z[(int64_t)i * N + j];
                for (int i = 0; i < n; ++i) Z[(int64_t)i * N + j] -= c * Z[(int64_t)i * N + jj];
            }
            double nr = 0.0;
            for (int i = 0; i < n; ++i) nr += Z[(int64_t)i * N + j] * Z[(int64_t)i * N + j];
            nr = sqrt(nr);
            if (!(nr > 0.0) || !isfinite(nr)) { atomicExch(status, (int)PHX_ERR_NUMERIC); nr = 1.0; }
            for (int i = 0; i < n; ++i) Z[(int64_t)i * N + j] /= nr;
        }
    }
#undef W
}

// Z <- H_0 H_1 ... H_{n-2} Z.  CTA = 4 columns x 32 row groups; reflectors in reverse order.
__global__ void __launch_bounds__(128)
backtransform_kernel(const double* __restrict__ A, const double* __restrict__ bet, const double* __restrict__ v0s,
                     int n, double* __restrict__ Z) {
    __shared__ double red[32][kStripCols];
    const int c = threadIdx.x & (kStripCols - 1), rg = threadIdx.x >> 2;
    const int col = blockIdx.x * kStripCols + c;
    const bool live = col < n;
    const int64_t N = n;
    for (int k = n - 2; k >= 0; --k) {
        const double beta = bet[k];
        if (beta == 0.0) continue;
        const double* x = A + (int64_t)k * N + k + 1;     // u[k+1] = v0, u[k+1+r] = x[r] (r >= 1)
        const double v0 = v0s[k];
        const int m = n - k - 1;
        double s = 0.0;
        if (live)
            for (int r = rg; r < m; r += 32) s += (r == 0 ? v0 : x[r]) * Z[(int64_t)(k + 1 + r) * N + col];
        red[rg][c] = s;
        __syncthreads();
        double tot = 0.0;
        for (int g = 0; g < 32; ++g) tot += red[g][c];
        tot *= beta;
        if (live)
            for (int r = rg; r < m; r += 32) Z[(int64_t)(k + 1 + r) * N + col] -= tot * (r == 0 ? v0 : x[r]);
        __syncthreads();
    }
}

// sign of each column: largest-modulus component positive (first index on ties); frequencies
__global__ void gauge_kernel(const double* __restrict__ Z, const double* __restrict__ lam, int n,
                             double* __restrict__ sgn, double* __restrict__ freq, int32_t* __restrict__ status) {
    __shared__ double sb[256];
    __shared__ int si[256];
    const int col = blockIdx.x;
    double best = -1.0;
    int bi = 0;
    bool finite = true;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = Z[(int64_t)i * n + col];
        finite = finite && isfinite(v);
        const double a = fabs(v);
        if (a > best) { best = a; bi = i; }
    }
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < blockDim.x; ++t)
            if (sb[t] > best || (sb[t] == best && si[t] < bi)) { best = sb[t]; bi = si[t]; }
        sgn[col] = Z[(int64_t)bi * n + col] < 0.0 ? -1.0 : 1.0;
        const double w2 = lam[col] * phx::kEvA2AmuToPs2;
        freq[col] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / phx::kTwoPi;
    }
    if (!finite) atomicExch(status, (int)PHX_ERR_NUMERIC);
}

__global__ void write_evec_kernel(const double* __restrict__ Z, const double* __restrict__ sgn, int n,
                                  double2* __restrict__ evec) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x)
        evec[t] = make_double2(Z[t] * sgn[t % n], 0.0);
}

}  // namespace

// D (n x n) built from the pair CSR, solved, written to freq[n] and evec[n][n] (complex,
// imaginary parts zero).  Enqueued on s; errors of the eigensolver land in the status word.
phx_status phx_eigh_gamma_large(phx_ctx* ctx, int na, const double* blk_val, const int32_t* pair_start,
                                const double* masses, double* freq, double* evec, cudaStream_t s) {
    const int n = 3 * na;
    const int64_t nn = (int64_t)n * n;
    double* A = (double*)phx_ws(ctx, "el.A", nn * 8);
    double* Z = (double*)phx_ws(ctx, "el.Z", nn * 8);
    double* vecs = (double*)phx_ws(ctx, "el.vec", (size_t)n * 10 * 8 + 64);
    double* wrk = (double*)phx_ws(ctx, "el.work", nn * 4 * 8);
    uint8_t* piv = (uint8_t*)phx_ws(ctx, "el.piv", nn);
    if (!A || !Z || !vecs || !wrk || !piv) return PHX_ERR_NOMEM;
    double *p = vecs, *d = vecs + n, *e = vecs + 2 * n, *bet = vecs + 3 * n, *v0s = vecs + 4 * n,
           *e2 = vecs + 5 * n, *lam = vecs + 6 * n, *sgn = vecs + 7 * n, *info = vecs + 8 * n;
    int32_t* status = (int32_t*)ctx->status_word;
    const int ps = phx_prof_begin(ctx, s);
    const int64_t npair = (int64_t)na * na;
    dynmat_gamma_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, s>>>(na, blk_val, pair_start, masses, A);
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(e, 0, (size_t)n * 8, s));
    for (int k = 0; k + 1 < n; ++k) {
        const int m = n - k - 1;
        tridiag_symv_kernel<<<(m + kSymvWarps - 1) / kSymvWarps, kSymvWarps * 32, 0, s>>>(A, n, k, p, d, e, bet, v0s);
        if (m > 1) tridiag_update_kernel<<<(m + kUpdRows - 1) / kUpdRows, 256, 0, s>>>(A, n, k, p, bet, v0s);
    }
    tridiag_finish_kernel<<<1, 1, 0, s>>>(A, n, d, e);
    tridiag_bounds_kernel<<<1, 256, 0, s>>>(d, e, n, e2, info);
    bisect_kernel<<<(n + 127) / 128, 128, 0, s>>>(d, e2, n, info, lam);
    invit_kernel<<<(n + 63) / 64, 64, 0, s>>>(d, e, lam, info, n, Z, wrk, wrk + nn, wrk + 2 * nn, wrk + 3 * nn, piv,
                                              status);
    backtransform_kernel<<<(n + kStripCols - 1) / kStripCols, 128, 0, s>>>(A, bet, v0s, n, Z);
    gauge_kernel<<<n, 256, 0, s>>>(Z, lam, n, sgn, freq, status);
    write_evec_kernel<<<4 * ctx->sm_count, 256, 0, s>>>(Z, sgn, n, (double2*)evec);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    // reduction (4/3 n^3) + back-transformation (2 n^3) flops; matrix traffic ~ (8 + 12) n^3 / 3 bytes
    phx_prof_end(ctx, ps, s, PHX_K_EIGEN, (10.0 / 3.0) * (double)n * n * n, 8.0 * (double)n * n * n);
    ctx->launches += 2 * (int64_t)(n - 1) + 8;
    return PHX_OK;
}
