// FP64 eigensolver for one large real-symmetric dynamical matrix: the Gamma point of a big
// (disordered) cell, Eq. (eigenvalue) of the paper (Sec. "Interatomic Force Constants": the
// real-space problem D eta = omega^2 eta for Gamma-only and amorphous systems).
//
// The batched one-CTA-per-matrix Jacobi solver holds a matrix in shared memory; a 3000 x 3000
// matrix (72 MB) is solved instead in four device phases, all in FP64:
//
//  1. dynmat_gamma_kernel   D = (D + D^T)/2 with D_{ia,jb} = sum_R Phi2(0i, Rj)_{ab}/sqrt(m_i m_j)
//  2. Householder tridiagonalisation, one reflector H_k = I - beta v v^T per step k: the
//     rank-2 update A22 -= v w^T + w v^T (w = p - (beta p.v / 2) v) of step k and the product
//     p' = beta' A22' v' of step k + 1 share one launch and one pass over the trailing block.
//     Reflector vectors are kept in a separate matrix V (row k holds v_k).
//  3. multisection on Sturm counts (a group of lanes per eigenvalue index) for the tridiagonal T,
//     then inverse iteration (one thread per cluster of eigenvalues closer than 1e-7 ||T||;
//     later members of a cluster are Gram-Schmidt orthogonalised against earlier ones).
//  4. back-transformation Z = H_0 H_1 ... Z_T in a single launch: every CTA owns a strip of
//     four columns and applies all reflectors to it in reverse order.
//
// The output follows the batched solver's conventions: ascending frequencies in THz (signed
// for negative eigenvalues) and columns with the largest-modulus component positive.
#include <algorithm>
#include <cfloat>
#include <cstdlib>

#include "common.h"

namespace {

constexpr int kSymvWarps = 8;          // rows per CTA in the symv kernel (one warp per row)
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

// Reflector of step k from x = row k of the (updated) matrix, columns k+1..n-1:
// alpha = -sign(x0) |x|, v = x - alpha e1, beta = 2 / v.v (beta = 0 when x[1..] = 0).
struct Reflector { double alpha, beta, v0; };
__device__ __forceinline__ Reflector make_reflector(double x0, double tail2) {
    Reflector r;
    if (tail2 == 0.0) { r.alpha = x0; r.beta = 0.0; r.v0 = 0.0; return r; }
    const double nrm = sqrt(x0 * x0 + tail2);
    r.alpha = x0 >= 0.0 ? -nrm : nrm;
    r.v0 = x0 - r.alpha;
    r.beta = 2.0 / (r.v0 * r.v0 + tail2);
    return r;
}

// Step 0: reflector from row 0 (stored in V row 0) and p_0 = beta A22 v (one warp per row).
__global__ void __launch_bounds__(kSymvWarps * 32)
tridiag_first_kernel(const double* __restrict__ A, int n, double* __restrict__ V, double* __restrict__ p,
                     double* __restrict__ d, double* __restrict__ e, double* __restrict__ bet, double* __restrict__ v0s) {
    __shared__ double red[32];
    const int m = n - 1;
    const double* x = A + 1;
    double s = 0.0;
    for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) s += x[c] * x[c];
    s = block_sum_256(s, red);
    const Reflector rf = make_reflector(x[0], s);
    if (blockIdx.x == 0) {
        for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) V[1 + c] = x[c];
        if (threadIdx.x == 0) { d[0] = A[0]; e[0] = rf.alpha; bet[0] = rf.beta; v0s[0] = rf.v0; }
    }
    if (rf.beta == 0.0) return;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kSymvWarps + (threadIdx.x >> 5);
    if (r >= m) return;
    const double* row = A + (int64_t)(1 + r) * n + 1;
    double acc = lane == 0 ? row[0] * rf.v0 : 0.0;
    for (int c = (lane == 0 ? 32 : lane); c < m; c += 32) acc += row[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) p[r] = rf.beta * acc;
}

// Step k (k = 0 .. n-3), fused with the product of step k + 1.  On the trailing block A22
// (rows/columns k+1 .. n-1, size m):
//   A22 <- A22 - v w^T - w v^T,  w = p - K v,  K = beta (p.v) / 2          (update of step k)
// Its first row (row k+1) is not written back: every CTA recomputes it from the untouched
// original, takes the reflector of step k+1 from it (stored in V row k+1) and, for the rows it
// owns, forms p' = beta' A22' v' from the freshly updated values (one pass over A22).
// Shared memory: v (step k), w, v' (step k+1), m doubles each.
__global__ void __launch_bounds__(kSymvWarps * 32)
tridiag_step_kernel(double* __restrict__ A, int n, int k, double* __restrict__ V, const double* __restrict__ p,
                    double* __restrict__ pn, double* __restrict__ d, double* __restrict__ e, double* __restrict__ bet,
                    double* __restrict__ v0s) {
    extern __shared__ double sh[];
    __shared__ double red[32];
    const int m = n - k - 1;
    double* sv = sh;            // v_k[c], c in [0, m)
    double* sw = sh + m;        // w_k[c]
    double* sn = sh + 2 * m;    // v_{k+1}[c'], c' in [0, m - 1)
    const int64_t N = n;
    const double beta = bet[k];
    const double* vrow = V + (int64_t)k * N + k + 1;
    for (int c = threadIdx.x; c < m; c += blockDim.x) sv[c] = c == 0 ? v0s[k] : vrow[c];
    __syncthreads();
    double pv = 0.0;
    if (beta != 0.0)
        for (int c = threadIdx.x; c < m; c += blockDim.x) pv += p[c] * sv[c];
    pv = block_sum_256(pv, red);
    const double K = 0.5 * beta * pv;
    for (int c = threadIdx.x; c < m; c += blockDim.x) sw[c] = beta != 0.0 ? p[c] - K * sv[c] : 0.0;
    __syncthreads();
    // updated row k+1 (r = 0): u[c] = A[k+1][k+1+c] - v0 w[c] - w[0] v[c]; x' = u[1..m)
    const double* row0 = A + (int64_t)(k + 1) * N + k + 1;
    const double v_0 = sv[0], w_0 = sw[0];
    double tail = 0.0;
    for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) {
        const double u = row0[c] - v_0 * sw[c] - w_0 * sv[c];
        sn[c - 1] = u;
        if (c >= 2) tail += u * u;
    }
    tail = block_sum_256(tail, red);          // (its syncs also publish sn)
    const double x0n = m > 1 ? sn[0] : 0.0;
    const Reflector rf = m > 1 ? make_reflector(x0n, tail) : Reflector{0.0, 0.0, 0.0};
    __syncthreads();
    if (threadIdx.x == 0) sn[0] = rf.v0;
    __syncthreads();
    if (blockIdx.x == 0) {
        double* vn = V + (int64_t)(k + 1) * N + k + 2;
        for (int c = 1 + threadIdx.x; c < m - 1; c += blockDim.x) vn[c] = sn[c];
        if (threadIdx.x == 0) {
            d[k + 1] = row0[0] - 2.0 * v_0 * w_0;
            e[k + 1] = rf.alpha;
            bet[k + 1] = rf.beta;
            v0s[k + 1] = rf.v0;
        }
    }
    // rows r >= 1 of A22: update, write back, and accumulate p' (rows k+2.. of step k+1)
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kSymvWarps + (threadIdx.x >> 5) + 1;
    if (r >= m) return;
    double* row = A + (int64_t)(k + 1 + r) * N + k + 1;
    const double vr = sv[r], wr = sw[r];
    double acc = 0.0;
    for (int c = lane; c < m; c += 32) {
        const double a = row[c] - vr * sw[c] - wr * sv[c];
        if (beta != 0.0) row[c] = a;
        if (c >= 1) acc += a * sn[c - 1];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) pn[r - 1] = rf.beta * acc;
}

__global__ void tridiag_finish_kernel(const double* __restrict__ A, int n, double* __restrict__ d,
                                      double* __restrict__ e) {
    d[n - 1] = A[(int64_t)(n - 1) * n + n - 1];
}

// Number of eigenvalues of T below x: sign changes of the leading principal minors
// p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1, p_0 = d_0 - x), i.e. the count of
// negative ratios p_i / p_{i-1} of the LDL^T pivots, without a division per step.  The pair
// (p_{i-1}, p_i) is rescaled by 2^-/+512 when |p_i| leaves [2^-512, 2^512); an exact zero
// minor is replaced by -pivmin x the previous one (a tiny negative pivot, as in the ratio
// form).
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x, double pivmin) {
    double pm = 1.0;               // p_{i-1}
    double pc = d[0] - x;          // p_i
    if (fabs(pc) < pivmin) pc = -pivmin;
    int cnt = pc < 0.0;
    for (int i = 1; i < n; ++i) {
        double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
        if (pn == 0.0) pn = -pivmin * pc;
        cnt += (__double_as_longlong(pn) ^ __double_as_longlong(pc)) < 0;   // sign change
        pm = pc;
        pc = pn;
        const int ex = (int)((__double_as_longlong(pc) >> 52) & 0x7ff);
        if (ex > 1023 + 512) { pc = ldexp(pc, -512); pm = ldexp(pm, -512); }
        else if (ex < 1023 - 512) { pc = ldexp(pc, 512); pm = ldexp(pm, 512); }
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

// G lanes per eigenvalue index m (multisection): each round evaluates the Sturm count at the
// G - 1 interior points of [lo, hi] splitting it into G equal parts and keeps the part holding
// the (m+1)-th eigenvalue: log2(G) bits per round.
template <int G>
__global__ void bisect_kernel(const double* __restrict__ d, const double* __restrict__ e2, int n,
                              const double* __restrict__ info, double* __restrict__ lam) {
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sub = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const int m = gid < n ? gid : n - 1;               // the warp stays converged: spare groups repeat n-1
    double lo = info[0], hi = info[1];
    const double pivmin = info[3];
    bool done = false;
    for (int round = 0; round < 128; ++round) {
        done = done || (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin);
        const double step = (hi - lo) / G;
        const double x = lo + step * (sub + 1);
        const int cnt = (done || sub == G - 1) ? n + 1 : sturm_count(d, e2, n, x, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, cnt > m);
        if (__all_sync(0xffffffffu, done)) break;
        const unsigned grp = (above >> (lane - sub)) & (G == 32 ? 0xffffffffu : ((1u << G) - 1));
        const int k = __ffs(grp) - 1;                  // first split point above the eigenvalue
        if (!done) {
            const double nlo = k == 0 ? lo : lo + step * k;
            const double nhi = k == G - 1 ? hi : lo + step * (k + 1);
            if (nlo == lo && nhi == hi) done = true;
            lo = nlo;
            hi = nhi;
        }
    }
    if (sub == 0 && gid < n) lam[m] = 0.5 * (lo + hi);
}

template <int G>
void launch_bisect(const double* d, const double* e2, int n, const double* info, double* lam, cudaStream_t s) {
    bisect_kernel<G><<<(unsigned)(((int64_t)n * G + 255) / 256), 256, 0, s>>>(d, e2, n, info, lam);
}

__device__ __forceinline__ double start_value(uint64_t seed) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// Inverse iteration with the LU factorisation (partial pivoting) of T - lambda I.  Work arrays
// are interleaved by thread (element i of thread t at [i * n + t]) and written once per
// factorisation; the recurrences carry their running values in registers, so no step waits
// on a store of the previous one.  The reciprocal pivots are stored.
__global__ void invit_kernel(const double* __restrict__ d, const double* __restrict__ e, const double* __restrict__ lam,
                             const double* __restrict__ info, int n, double* __restrict__ Z,
                             double* __restrict__ wdl, double* __restrict__ wri, double* __restrict__ wdu,
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
#define ZC(i) Z[(int64_t)(i) * N + j]
    auto safe = [&](double p) { return fabs(p) < eps3 * 1e-3 ? copysign(eps3, p) : p; };
    double lprev = 0.0;
    for (int j = t; j < tend; ++j) {
        double lj = lam[j];
        if (j > t && lj - lprev < eps3) lj = lprev + eps3;
        lprev = lj;
        // ---- factor T - lj I: row i holds (dd_i, uu_i, u2_i) after elimination
        double dcur = d[0] - lj;                  // current diagonal of row i
        double ucur = n > 1 ? e[0] : 0.0;         // current first superdiagonal of row i
        for (int i = 0; i < n - 1; ++i) {
            const double li = e[i];               // subdiagonal below row i (never modified)
            const double dnext = d[i + 1] - lj;
            const double unext = i + 1 < n - 1 ? e[i + 1] : 0.0;
            if (fabs(dcur) >= fabs(li)) {
                const double piv = safe(dcur);
                const double f = li / piv;
                W(wpiv, i) = 0;
                W(wdl, i) = f;
                W(wri, i) = 1.0 / piv;
                W(wdu, i) = ucur;
                W(wdu2, i) = 0.0;
                dcur = dnext - f * ucur;
                ucur = unext;
            } else {
                const double f = dcur / li;
                W(wpiv, i) = 1;
                W(wdl, i) = f;
                W(wri, i) = 1.0 / li;
                W(wdu, i) = dnext;
                W(wdu2, i) = unext;
                dcur = ucur - f * dnext;
                ucur = -f * unext;
            }
        }
        W(wri, n - 1) = 1.0 / safe(dcur);
        // ---- start vector in column j of Z
        for (int i = 0; i < n; ++i) ZC(i) = start_value(((uint64_t)j << 32) ^ (uint64_t)i);
        for (int it = 0; it < kInvitIters; ++it) {
            // forward: y = L^-1 P b, in place (b[i + 1] is read before y[i] is written)
            double cur = ZC(0);
            for (int i = 0; i < n - 1; ++i) {
                const double nxt = ZC(i + 1);
                const double f = W(wdl, i);
                if (W(wpiv, i) == 0) {
                    ZC(i) = cur;
                    cur = nxt - f * cur;
                } else {
                    ZC(i) = nxt;
                    cur = cur - f * nxt;
                }
            }
            ZC(n - 1) = cur;
            // backward: x_i = (y_i - u_i x_{i+1} - u2_i x_{i+2}) / dd_i
            double x1 = cur * W(wri, n - 1), x2 = 0.0;
            ZC(n - 1) = x1;
            for (int i = n - 2; i >= 0; --i) {
                const double xi = (ZC(i) - W(wdu, i) * x1 - W(wdu2, i) * x2) * W(wri, i);
                ZC(i) = xi;
                x2 = x1;
                x1 = xi;
            }
            // scale, orthogonalise against the earlier members of the cluster, normalise
            double amax = 0.0;
            for (int i = 0; i < n; ++i) amax = fmax(amax, fabs(ZC(i)));
            const double sc = amax > 0.0 ? 1.0 / amax : 1.0;
            for (int i = 0; i < n; ++i) ZC(i) *= sc;
            for (int jj = t; jj < j; ++jj) {
                double c = 0.0;
                for (int i = 0; i < n; ++i) c += Z[(int64_t)i * N + jj] * ZC(i);
                for (int i = 0; i < n; ++i) ZC(i) -= c * Z[(int64_t)i * N + jj];
            }
            double nr = 0.0;
            for (int i = 0; i < n; ++i) nr += ZC(i) * ZC(i);
            nr = sqrt(nr);
            if (!(nr > 0.0) || !isfinite(nr)) { atomicExch(status, (int)PHX_ERR_NUMERIC); nr = 1.0; }
            const double inr = 1.0 / nr;
            for (int i = 0; i < n; ++i) ZC(i) *= inr;
        }
    }
#undef ZC
#undef W
}

// Z <- H_0 H_1 ... H_{n-2} Z.  CTA = 4 columns x 32 row groups; reflectors in reverse order.
__global__ void __launch_bounds__(128)
backtransform_kernel(const double* __restrict__ V, const double* __restrict__ bet, const double* __restrict__ v0s,
                     int n, double* __restrict__ Z) {
    __shared__ double red[32][kStripCols];
    const int c = threadIdx.x & (kStripCols - 1), rg = threadIdx.x >> 2;
    const int col = blockIdx.x * kStripCols + c;
    const bool live = col < n;
    const int64_t N = n;
    for (int k = n - 2; k >= 0; --k) {
        const double beta = bet[k];
        if (beta == 0.0) continue;
        const double* x = V + (int64_t)k * N + k + 1;     // u[k+1] = v0, u[k+1+r] = x[r] (r >= 1)
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
    double* V = (double*)phx_ws(ctx, "el.Vr", nn * 8);
    double* Z = (double*)phx_ws(ctx, "el.Z", nn * 8);
    double* vecs = (double*)phx_ws(ctx, "el.vec", (size_t)n * 11 * 8 + 64);
    double* wrk = (double*)phx_ws(ctx, "el.work", nn * 4 * 8);
    uint8_t* piv = (uint8_t*)phx_ws(ctx, "el.piv", nn);
    if (!A || !V || !Z || !vecs || !wrk || !piv) return PHX_ERR_NOMEM;
    double *p = vecs, *d = vecs + n, *e = vecs + 2 * n, *bet = vecs + 3 * n, *v0s = vecs + 4 * n,
           *e2 = vecs + 5 * n, *lam = vecs + 6 * n, *sgn = vecs + 7 * n, *p2 = vecs + 8 * n, *info = vecs + 9 * n;
    int32_t* status = (int32_t*)ctx->status_word;
    const double nd = (double)n;
    int ps = phx_prof_begin(ctx, s);
    const int64_t npair = (int64_t)na * na;
    dynmat_gamma_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, s>>>(na, blk_val, pair_start, masses, A);
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(e, 0, (size_t)n * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(bet, 0, (size_t)n * 8, s));
    if (n > 1) {
        tridiag_first_kernel<<<(n - 1 + kSymvWarps - 1) / kSymvWarps, kSymvWarps * 32, 0, s>>>(A, n, V, p, d, e, bet,
                                                                                              v0s);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(tridiag_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 8192 * 8);
            attr = true;
        }
        for (int k = 0; k + 2 < n; ++k) {
            const int m = n - k - 1;
            double* pin = (k & 1) ? p2 : p;
            double* pout = (k & 1) ? p : p2;
            const int blocks = std::max(1, (m - 1 + kSymvWarps - 1) / kSymvWarps);
            tridiag_step_kernel<<<blocks, kSymvWarps * 32, (size_t)3 * m * 8, s>>>(A, n, k, V, pin, pout, d, e, bet,
                                                                                 v0s);
        }
    }
    tridiag_finish_kernel<<<1, 1, 0, s>>>(A, n, d, e);
    // Householder reduction: 4/3 n^3 flops; the trailing matrix read three times per step
    phx_prof_end(ctx, ps, s, PHX_K_EIG_TRIDIAG, (4.0 / 3.0) * nd * nd * nd, 8.0 * nd * nd * nd);
    ps = phx_prof_begin(ctx, s);
    tridiag_bounds_kernel<<<1, 256, 0, s>>>(d, e, n, e2, info);
    // lanes per eigenvalue: 8 by default (PHX_SECT_LANES = 2, 4, 8, 16 or 32 to tune)
    static const int lanes = [] {
        const char* v = std::getenv("PHX_SECT_LANES");
        const int g = v ? std::atoi(v) : 8;
        return (g == 2 || g == 4 || g == 16 || g == 32) ? g : 8;
    }();
    if (lanes == 2) launch_bisect<2>(d, e2, n, info, lam, s);
    else if (lanes == 16) launch_bisect<16>(d, e2, n, info, lam, s);
    else if (lanes == 32) launch_bisect<32>(d, e2, n, info, lam, s);
    else if (lanes == 4) launch_bisect<4>(d, e2, n, info, lam, s);
    else launch_bisect<8>(d, e2, n, info, lam, s);
    phx_prof_end(ctx, ps, s, PHX_K_EIG_BISECT, 0.0, 0.0);
    ps = phx_prof_begin(ctx, s);
    invit_kernel<<<(n + 31) / 32, 32, 0, s>>>(d, e, lam, info, n, Z, wrk, wrk + nn, wrk + 2 * nn, wrk + 3 * nn, piv,
                                              status);
    phx_prof_end(ctx, ps, s, PHX_K_EIG_VECTORS, 0.0, 0.0);
    ps = phx_prof_begin(ctx, s);
    backtransform_kernel<<<(n + kStripCols - 1) / kStripCols, 128, 0, s>>>(V, bet, v0s, n, Z);
    gauge_kernel<<<n, 256, 0, s>>>(Z, lam, n, sgn, freq, status);
    write_evec_kernel<<<4 * ctx->sm_count, 256, 0, s>>>(Z, sgn, n, (double2*)evec);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    // back-transformation: 2 n^3 flops, Z read twice and written once per reflector
    phx_prof_end(ctx, ps, s, PHX_K_EIG_BACK, 2.0 * nd * nd * nd, 12.0 * nd * nd * nd);
    ctx->launches += (int64_t)n + 8;
    return PHX_OK;
}
