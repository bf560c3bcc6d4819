// Learned linewidths: descriptor kernel and a small MLP ensemble trained and evaluated with
// the library's own kernels (no counterpart in the paper; the descriptors restate its
// quantities: w, |v| (Eq. groupvel), the weighted two-phonon phase space of Eqs. (gamma) and
// (broadening) with |Phi|^2 -> 1, and n_B (Eq. bose)).
//
//  features_kernel   per irreducible mode: sum over q' and partner bands of the occupation /
//                    smearing weight without V3 (FP32, ALU bound)
//  gemm_f32_kernel   C = op(A) op(B) (+ bias, SiLU), batched over ensemble members; the
//                    forward, weight-gradient and input-gradient products of every layer
//  small kernels     input transform, loss and its gradient, SiLU backward, bias gradient,
//                    Adam, ensemble mean/std
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"
#include "gamma_common.cuh"
#include "tc_ptx.cuh"

namespace {

// ---------------------------------------------------------------- descriptors

// Block (s, chunk of q'): every thread takes one q' and loops over (nu, nu', nu''); the
// per-band sums are reduced in shared memory and added once per block.
__global__ void __launch_bounds__(256)
features_kernel(const double* __restrict__ freq, const double* __restrict__ nB, const int32_t* __restrict__ irr,
                int n, int m1, int m2, int m3, float sigma, float window, int shape, float f_min,
                double* __restrict__ wsum) {
    __shared__ float red[192];
    const int nq = m1 * m2 * m3;
    const int s = blockIdx.y;
    const int iq = irr[s];
    for (int j = threadIdx.x; j < n; j += blockDim.x) red[j] = 0.f;
    __syncthreads();
    const float lim = window * sigma;
    const int qp = blockIdx.x * blockDim.x + threadIdx.x;
    if (qp < nq) {
        const int q2 = phx_third_index(iq, qp, m1, m2, m3);
        for (int nu = 0; nu < n; ++nu) {
            const float f0 = (float)freq[(int64_t)iq * n + nu];
            if (!(f0 >= f_min)) continue;
            float acc = 0.f;
            for (int j1 = 0; j1 < n; ++j1) {
                const float f1 = (float)freq[(int64_t)qp * n + j1];
                if (!(f1 >= f_min)) continue;
                const float n1 = (float)nB[(int64_t)qp * n + j1];
                for (int j2 = 0; j2 < n; ++j2) {
                    const float f2 = (float)freq[(int64_t)q2 * n + j2];
                    if (!(f2 >= f_min)) continue;
                    const float x = f0 - f1 - f2, y = f0 + f1 - f2;
                    float gd = 0.f, ga = 0.f;
                    if (fabsf(x) < lim)
                        gd = shape == PHX_GAUSS ? __expf(-(x / sigma) * (x / sigma)) * (0.56418958354775628f / sigma)
                                                : (0.5f * sigma) / (3.14159265358979f * (x * x + 0.25f * sigma * sigma));
                    if (fabsf(y) < lim)
                        ga = shape == PHX_GAUSS ? __expf(-(y / sigma) * (y / sigma)) * (0.56418958354775628f / sigma)
                                                : (0.5f * sigma) / (3.14159265358979f * (y * y + 0.25f * sigma * sigma));
                    if (gd == 0.f && ga == 0.f) continue;
                    const float n2 = (float)nB[(int64_t)q2 * n + j2];
                    acc += ((1.f + n1 + n2) * gd + 2.f * (n1 - n2) * ga) / (f1 * f2);
                }
            }
            if (acc != 0.f) atomicAdd(&red[nu], acc);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        if (red[j] != 0.f) atomicAdd(&wsum[(int64_t)s * n + j], (double)red[j]);
}

// features[s][nu] = (w rad/ps, |v| A/ps, WP2 ps^4, n_B)
__global__ void features_finish_kernel(const double* __restrict__ freq, const double* __restrict__ vel,
                                       const double* __restrict__ nB, const int32_t* __restrict__ irr, int n_irr,
                                       int n, int nq, double f_min, const double* __restrict__ wsum,
                                       double* __restrict__ out) {
    const int total = n_irr * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int s = t / n, nu = t % n;
        const int64_t m = (int64_t)irr[s] * n + nu;
        const double f0 = freq[m];
        const double w = f0 * phx::kTwoPi;
        const double* v = vel + m * 3;
        const bool ok = f0 >= f_min;
        // WP2 = (1/N_q) sum [..] / (2 pi w0 w1 w2) with the f1 f2 of the sum already divided out
        const double tp4 = phx::kTwoPi * phx::kTwoPi * phx::kTwoPi * phx::kTwoPi;
        out[(int64_t)t * 4 + 0] = w;
        out[(int64_t)t * 4 + 1] = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        out[(int64_t)t * 4 + 2] = ok ? wsum[t] / (tp4 * f0) / nq : 0.0;
        out[(int64_t)t * 4 + 3] = nB[m];
    }
}

// ---------------------------------------------------------------- MLP kernels

constexpr int TM = 64, TN = 64, TK = 16;

// C_e[M x N] = op(A_e) op(B_e) (+ bias_e, then optional SiLU; the pre-activation goes to Z_e).
// op(A) = A [M x K] (lda) or A^T with A stored [K x M]; op(B) = B [K x N] or B^T with B [N x K].
// Batched over ensemble members e (blockIdx.z) with element strides sA, sB, sC (0 = shared).
__global__ void __launch_bounds__(256)
gemm_f32_kernel(int M, int N, int K, const float* __restrict__ A, int lda, int64_t sA, int tA,
                const float* __restrict__ B, int ldb, int64_t sB, int tB, float* __restrict__ C, int ldc,
                int64_t sC, const float* __restrict__ bias, int64_t sBias, int act, float* __restrict__ Z,
                int accumulate) {
    __shared__ float As[TK][TM + 1], Bs[TK][TN + 1];
    const int e = blockIdx.z;
    A += e * sA;
    B += e * sB;
    C += e * sC;
    if (Z) Z += e * sC;
    if (bias) bias += e * sBias;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int i = threadIdx.x; i < TM * TK; i += 256) {
            int m, k;
            if (tA) { k = i / TM; m = i % TM; } else { m = i / TK; k = i % TK; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < M && gk < K) v = tA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[k][m] = v;
        }
        for (int i = threadIdx.x; i < TK * TN; i += 256) {
            int k, nn;
            if (tB) { nn = i / TK; k = i % TK; } else { k = i / TN; nn = i % TN; }
            const int gn = n0 + nn, gk = k0 + k;
            float v = 0.f;
            if (gn < N && gk < K) v = tB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            Bs[k][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float z = acc[i][j] + (bias ? bias[gn] : 0.f);
            if (accumulate) z += C[(int64_t)gm * ldc + gn];
            if (Z) Z[(int64_t)gm * ldc + gn] = z;
            C[(int64_t)gm * ldc + gn] = act ? z / (1.f + __expf(-z)) : z;
        }
    }
}

// The same product on the tensor cores (tcgen05, kind::f16 in BF16x3: hi.hi + hi.lo + lo.hi,
// FP32 accumulation in tensor memory), for the layers of width >= 16.  One CTA of 128
// threads per 128-row tile of C (and per 128 columns, blockIdx.x) and member: K runs in chunks
// of 64; for each chunk the threads read op(A) and op(B) from global memory (any
// transposition; coalesced along whichever index is contiguous), split every value into bf16
// hi and lo and write the 128-byte-swizzled K-major layout the MMA reads (within a 1024-byte
// group of eight 128-byte rows, the 16-byte unit u of row r sits at unit u ^ (r % 8)); thread 0
// issues the chunk's 4 K steps x 3 MMAs and commits, and the next chunk's writes wait for that
// commit.  The epilogue reads the accumulator lane by lane (row = lane) and applies bias,
// SiLU and the pre-activation output as gemm_f32_kernel does.  Every wait is bounded.
constexpr int kMlpTcK = 64;                                   // K elements per chunk (128 bytes of bf16)
constexpr uint32_t kMlpTcTile = 128 * 128;                    // bytes of one 128-row operand plane
constexpr size_t kMlpTcSmem = 4 * (size_t)kMlpTcTile + 1024;  // A hi/lo, B hi/lo, alignment

__device__ __forceinline__ uint32_t sw128_off(int r, int u) { return (uint32_t)(r * 128 + ((u ^ (r & 7)) << 4)); }

template <bool TA, bool TB>
__global__ void __launch_bounds__(128)
gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A, int lda, int64_t sA, const float* __restrict__ B,
               int ldb, int64_t sB, float* __restrict__ C, int ldc, int64_t sC, const float* __restrict__ bias,
               int64_t sBias, int act, float* __restrict__ Z, int accumulate, int ksplit, int32_t* status,
               unsigned long long wait_ns) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sAh = smem;
    uint8_t* sAl = sAh + kMlpTcTile;
    uint8_t* sBh = sAl + kMlpTcTile;
    uint8_t* sBl = sBh + kMlpTcTile;
    const int e = blockIdx.z, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    A += e * sA;
    B += e * sB;
    C += e * sC;
    if (Z) Z += e * sC;
    if (bias) bias += e * sBias;
    const int n_ntiles = (N + 127) / 128;
    const int m0 = blockIdx.y * 128, n0 = (blockIdx.x % n_ntiles) * 128, split = blockIdx.x / n_ntiles;
    const int nt = min(128, N - n0), nmma = (nt + 15) & ~15;   // columns of this tile, MMA width
    // K range of this split (whole chunks)
    const int n_chunks_all = (K + kMlpTcK - 1) / kMlpTcK;
    const int per = (n_chunks_all + ksplit - 1) / ksplit;
    const int c_begin = split * per, c_end = min(n_chunks_all, c_begin + per);
    const int n_chunks = max(0, c_end - c_begin);
    if (t == 0) {
        tc::mbar_init(&mma_bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 128);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t id = tc::idesc(128, nmma, 1u);
    // This thread's share of a chunk: 8 units (8 K elements each) of A and of B.  Row-major
    // operands: 8 threads per row read its 64 contiguous k; transposed ones: thread t takes
    // row t (the contiguous index runs across the warp) and all 8 units.
    auto a_row = [&](int i) { return TA ? t : i * 16 + (t >> 3); };
    auto a_unit = [&](int i) { return TA ? i : (t & 7); };
    auto b_row = [&](int i) { return TB ? i * 16 + (t >> 3) : t; };
    auto b_unit = [&](int i) { return TB ? (t & 7) : i; };
    float va[8][8], vb[8][8];
    auto load = [&](int ch) {          // global -> registers, every load issued before any use
        const int k0 = ch * kMlpTcK;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = a_row(i), kb = k0 + 8 * a_unit(i);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = kb + j;
                va[i][j] = (m0 + r < M && k < K) ? (TA ? A[(int64_t)k * lda + m0 + r] : A[(int64_t)(m0 + r) * lda + k]) : 0.f;
            }
            const int rb = b_row(i), kc = k0 + 8 * b_unit(i);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = kc + j;
                vb[i][j] = (rb < nt && k < K) ? (TB ? B[(int64_t)(n0 + rb) * ldb + k] : B[(int64_t)k * ldb + n0 + rb]) : 0.f;
            }
        }
    };
    auto put = [&](uint8_t* hi, uint8_t* lo, int r, int u, const float* v) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tc::split_bf16x2(v[2 * j], v[2 * j + 1], &h[j], &l[j]);
        *reinterpret_cast<uint4*>(hi + sw128_off(r, u)) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + sw128_off(r, u)) = make_uint4(l[0], l[1], l[2], l[3]);
    };
    bool ok = true;
    if (n_chunks > 0) load(c_begin);
    for (int q = 0; q < n_chunks; ++q) {
        if (q > 0) {    // the previous chunk's MMAs have read the operands
            ok = tc::mbar_wait(&mma_bar, (q - 1) & 1, &abort_flag, wait_ns);
            if (!ok) { abort_flag = 1; atomicExch(status, (int)PHX_ERR_TIMEOUT); }
            if (__syncthreads_or(!ok)) break;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            put(sAh, sAl, a_row(i), a_unit(i), va[i]);
            if (b_row(i) < nmma) put(sBh, sBl, b_row(i), b_unit(i), vb[i]);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (t == 0) {
            tc::tc_fence_after();
            const uint64_t ah = tc::sdesc_sw128(tc::smem_u32(sAh)), al = tc::sdesc_sw128(tc::smem_u32(sAl));
            const uint64_t bh = tc::sdesc_sw128(tc::smem_u32(sBh)), bl = tc::sdesc_sw128(tc::smem_u32(sBl));
#pragma unroll
            for (int kk = 0; kk < kMlpTcK / 16; ++kk) {
                const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
                const uint64_t o = (uint64_t)(2 * kk);          // 32 bytes per K step, in 16-byte units
                tc::mma_f16(tmem, ah + o, bh + o, id, acc);
                tc::mma_f16(tmem, ah + o, bl + o, id, 1u);
                tc::mma_f16(tmem, al + o, bh + o, id, 1u);
            }
            tc::mma_commit(&mma_bar);
        }
        if (q + 1 < n_chunks) load(c_begin + q + 1);   // in flight while the MMAs run
    }
    if (ok && n_chunks > 0) {
        ok = tc::mbar_wait(&mma_bar, (n_chunks - 1) & 1, &abort_flag, wait_ns);
        if (!ok) { abort_flag = 1; atomicExch(status, (int)PHX_ERR_TIMEOUT); }
    }
    ok = __syncthreads_and(ok) != 0;
    tc::tc_fence_after();
    if (ok && n_chunks > 0) {
        // epilogue: warp w holds rows 32w .. 32w + 31 of the tile in its tensor-memory lanes;
        // K splits add their partial products (the caller zeroed C; no bias, activation or Z)
        const int gm = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < nmma; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c0, v);
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int gn = n0 + c0 + j;
                if (c0 + j >= nt) break;
                if (ksplit > 1) {
                    atomicAdd(&C[(int64_t)gm * ldc + gn], v[j]);
                    continue;
                }
                float z = v[j] + (bias ? bias[gn] : 0.f);
                if (accumulate) z += C[(int64_t)gm * ldc + gn];
                if (Z) Z[(int64_t)gm * ldc + gn] = z;
                C[(int64_t)gm * ldc + gn] = act ? z / (1.f + __expf(-z)) : z;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 128);
    }
}

// x_in = (log(max(x, floor)) - mu) / sd per feature column.
__global__ void input_kernel(const double* __restrict__ X, int M, int F, const float* __restrict__ mu,
                             const float* __restrict__ sd, float* __restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * F; t += gridDim.x * blockDim.x) {
        const int f = t % F;
        const double v = fmax(X[t], 1e-12);
        out[t] = (float)((log(v) - mu[f]) / sd[f]);
    }
}

// column min / max of log(max(x, 1e-12)) over the first M rows (one block per column), rounded
// outward to float so that every row of the set lies inside its own range
__global__ void range_kernel(const double* __restrict__ X, int M, int F, float* __restrict__ lo,
                             float* __restrict__ hi) {
    __shared__ double s1[256], s2[256];
    const int f = blockIdx.x;
    double a = INFINITY, b = -INFINITY;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const double v = log(fmax(X[(int64_t)i * F + f], 1e-12));
        a = fmin(a, v);
        b = fmax(b, v);
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] = fmin(s1[threadIdx.x], s1[threadIdx.x + o]);
            s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lo[f] = __double2float_rd(s1[0]);
        hi[f] = __double2float_ru(s2[0]);
    }
}

// outside[r] = 1 when some input of row r lies outside the range of the training inputs (log scale)
__global__ void outside_kernel(const double* __restrict__ X, int M, int F, const float* __restrict__ lo,
                               const float* __restrict__ hi, int32_t* __restrict__ outside) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x) {
        int o = 0;
        for (int f = 0; f < F; ++f) {
            const double v = log(fmax(X[(int64_t)r * F + f], 1e-12));
            if (v < (double)lo[f] || v > (double)hi[f]) o = 1;
        }
        outside[r] = o;
    }
}

// column mean / std of log(max(x, floor)) (one block per column); std floored at 1e-6
__global__ void moments_kernel(const double* __restrict__ X, int M, int F, int take_log, float* __restrict__ mu,
                               float* __restrict__ sd) {
    __shared__ double s1[256], s2[256];
    const int f = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double v = X[(int64_t)i * F + f];
        if (take_log) v = log(fmax(v, 1e-12));
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / M;
        const double var = fmax(s2[0] / M - m * m, 0.0);
        mu[f] = (float)m;
        sd[f] = (float)fmax(sqrt(var), 1e-6);
    }
}

// y_std = (log(gamma) - mu) / sd
__global__ void target_kernel(const double* __restrict__ y, int M, const float* __restrict__ mu,
                              const float* __restrict__ sd, float* __restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M; t += gridDim.x * blockDim.x)
        out[t] = (float)((log(fmax(y[t], 1e-300)) - mu[0]) / sd[0]);
}

// dZ = dA * silu'(Z)
__global__ void silu_back_kernel(float* __restrict__ d, const float* __restrict__ Z, int64_t count) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[t];
        const float s = 1.f / (1.f + __expf(-z));
        d[t] *= s * (1.f + z * (1.f - s));
    }
}

// db_e[j] = sum_i dZ_e[i][j]
__global__ void bias_grad_kernel(const float* __restrict__ dZ, int M, int N, int64_t sZ, float* __restrict__ db,
                                 int64_t sDb) {
    const int e = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int i = 0; i < M; ++i) a += dZ[e * sZ + (int64_t)i * N + j];
        db[e * sDb + j] = a;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps,
                            const int* __restrict__ step) {
    // bias corrections of step t (a device counter, so one captured epoch serves every step)
    const float tt = (float)(*step);
    const float c1 = 1.f - powf(b1, tt), c2 = 1.f - powf(b2, tt);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.f - b1) * gt;
        const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    }
}

__global__ void step_kernel(int* step) { *step += 1; }

// dY = 2 (Yhat - y) / M for every member (member stride L), loss[e] += sum (Yhat - y)^2 / M
__global__ void loss_grad_all_kernel(const float* __restrict__ yhat, const float* __restrict__ y, int M, int E,
                                     int64_t L, float* __restrict__ dy, double* __restrict__ loss) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * E; t += gridDim.x * blockDim.x) {
        const int e = t / M, i = t % M;
        const float r = yhat[e * L + i] - y[i];
        dy[e * L + i] = 2.f * r / M;
        if (loss) atomicAdd(&loss[e], (double)(r * r) / M);
    }
}

// As loss_grad_all_kernel with the last M - Mt rows held out: gradient 2 r / Mt on the first Mt
// rows, 0 on the rest, whose mean squared error goes to vloss[e].
__global__ void loss_grad_split_kernel(const float* __restrict__ yhat, const float* __restrict__ y, int Mt, int M,
                                       int E, int64_t L, float* __restrict__ dy, double* __restrict__ vloss) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * E; t += gridDim.x * blockDim.x) {
        const int e = t / M, i = t % M;
        const float r = yhat[e * L + i] - y[i];
        if (i < Mt) {
            dy[e * L + i] = 2.f * r / Mt;
        } else {
            dy[e * L + i] = 0.f;
            atomicAdd(&vloss[e], (double)(r * r) / (M - Mt));
        }
    }
}

// ensemble statistics of log gamma (de-standardised): mean and std over members
__global__ void ensemble_kernel(const float* __restrict__ yhat, int M, int E, const float* __restrict__ mu,
                                const float* __restrict__ sd, double* __restrict__ mean, double* __restrict__ stdv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int e = 0; e < E; ++e) {
            const double v = (double)yhat[(int64_t)e * M + i] * sd[0] + mu[0];
            a += v;
            b += v * v;
        }
        a /= E;
        mean[i] = a;
        if (stdv) stdv[i] = sqrt(fmax(b / E - a * a, 0.0));
    }
}

// counter-based initialisation: splitmix64 of (seed, member, index) -> U(-a, a)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Linewidths from the ensemble's log prediction: one block per group of n rows (one
// irreducible q-point).  gamma = exp(mean) (x WP2 for the residual target) on rows whose mode
// is at or above f_min, 0 below; score = the largest ensemble spread over the group's live rows.
__global__ void __launch_bounds__(256) reconstruct_kernel(int n, const double* __restrict__ mean,
                                                          const double* __restrict__ stdv,
                                                          const double* __restrict__ wp2,
                                                          const double* __restrict__ freq, double f_min,
                                                          const int32_t* __restrict__ outside,
                                                          double* __restrict__ gamma, double* __restrict__ score) {
    __shared__ double red[8];
    const int64_t r0 = (int64_t)blockIdx.x * n;
    double mx = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t r = r0 + j;
        const bool live = freq[r] >= f_min;
        double g = 0.0;
        if (live) {
            g = exp(mean[r]);
            if (wp2) g *= wp2[r];
            if (stdv) mx = fmax(mx, stdv[r]);
            if (outside && outside[r]) mx = INFINITY;
        }
        gamma[r] = g;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0 && score) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
        score[blockIdx.x] = v;
    }
}

__global__ void init_kernel(float* __restrict__ p, int64_t count, uint64_t seed, float a) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = splitmix64(seed ^ splitmix64((uint64_t)t));
        const float u = (float)((r >> 11) * (1.0 / 9007199254740992.0));
        p[t] = a * (2.f * u - 1.f);
    }
}

}  // namespace

// ---------------------------------------------------------------- model object

struct phx_mlp {
    phx_ctx* ctx = nullptr;
    int n_in = 4, width = 128, depth = 3, E = 4;
    uint64_t seed = 0;
    // per member parameter block: [W0 (in x w), b0 (w), W1 (w x w), b1, ..., Wd (w x 1), bd (1)]
    std::vector<int64_t> w_off, b_off, w_rows, w_cols;
    int64_t n_par = 0;                         // per member
    float *par = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    float *mu = nullptr, *sd = nullptr;        // input (n_in) and target (1) standardisation
    float *ymu = nullptr, *ysd = nullptr;
    float *xlo = nullptr, *xhi = nullptr;      // range of the log inputs of the last training rows
    int64_t cap = 0;                           // activation buffers capacity (rows)
    float *act = nullptr, *pre = nullptr;      // [depth+2][E][rows][width]
    float *xin = nullptr, *ystd = nullptr, *dbuf0 = nullptr, *dbuf1 = nullptr;
    double* loss = nullptr;
    double* vloss = nullptr;                   // held-out loss per member (early stopping)
    float* best = nullptr;                     // parameters at the best held-out loss
    int* step = nullptr;                       // Adam step counter (device)
};

namespace {

phx_status mlp_reserve(phx_mlp* m, int64_t rows) {
    if (rows <= m->cap) return PHX_OK;
    cudaFree(m->act); cudaFree(m->pre); cudaFree(m->xin); cudaFree(m->ystd); cudaFree(m->dbuf0); cudaFree(m->dbuf1);
    const int64_t layer = (int64_t)m->E * rows * m->width;
    bool ok = cudaMalloc(&m->act, sizeof(float) * layer * (m->depth + 2)) == cudaSuccess &&
              cudaMalloc(&m->pre, sizeof(float) * layer * (m->depth + 2)) == cudaSuccess &&
              cudaMalloc(&m->xin, sizeof(float) * rows * m->n_in) == cudaSuccess &&
              cudaMalloc(&m->ystd, sizeof(float) * rows) == cudaSuccess &&
              cudaMalloc(&m->dbuf0, sizeof(float) * layer) == cudaSuccess &&
              cudaMalloc(&m->dbuf1, sizeof(float) * layer) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        m->cap = 0;
        return phx_set_error(m->ctx, PHX_ERR_NOMEM, "mlp: activation buffers");
    }
    m->cap = rows;
    return PHX_OK;
}

template <bool TA, bool TB>
cudaError_t launch_gemm_tc(dim3 grid, int M, int N, int K, const float* A, int lda, int64_t sA, const float* B,
                           int ldb, int64_t sB, float* C, int ldc, int64_t sC, const float* bias, int64_t sBias,
                           int act, float* Z, int accumulate, int ksplit, const phx_ctx* ctx, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(gemm_tc_kernel<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpTcSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gemm_tc_kernel<TA, TB><<<grid, 128, kMlpTcSmem, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, sBias, act,
                                                        Z, accumulate, ksplit, (int32_t*)ctx->status_word,
                                                        ctx->opt_wait_ns);
    return cudaGetLastError();
}

// C = op(A) op(B) (+ bias, SiLU): on the tensor cores when both the output width and K are at
// least 16 on a Blackwell device (the hidden layers and their gradients), else FP32 SIMT tiles
// (the input layer of n_in features, the one-column output layer).  `zeroed`: C holds zeros
// and no bias, activation or accumulation is asked for, so K may be split over CTAs whose
// partial products are added atomically (the weight gradients, whose K is the batch).
cudaError_t gemm(const phx_ctx* ctx, int M, int N, int K, const float* A, int lda, int64_t sA, int tA, const float* B,
                 int ldb, int64_t sB, int tB, float* C, int ldc, int64_t sC, const float* bias, int64_t sBias, int act,
                 float* Z, int E, int accumulate, cudaStream_t s, bool zeroed = false) {
    if (ctx->cc_major == 10 && N >= 16 && K >= 16 && M >= 16) {
        const int tiles = ((N + 127) / 128) * ((M + 127) / 128) * E;
        const int chunks = (K + kMlpTcK - 1) / kMlpTcK;
        const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
        int ksplit = zeroed && !bias && !act && !Z && !accumulate ? std::min(chunks, std::max(1, sms / tiles)) : 1;
        ksplit = (chunks + ((chunks + ksplit - 1) / ksplit) - 1) / ((chunks + ksplit - 1) / ksplit);   // no empty split
        dim3 grid(((N + 127) / 128) * ksplit, (M + 127) / 128, E);
        if (tA && tB) return launch_gemm_tc<true, true>(grid, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, sBias, act, Z, accumulate, ksplit, ctx, s);
        if (tA) return launch_gemm_tc<true, false>(grid, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, sBias, act, Z, accumulate, ksplit, ctx, s);
        if (tB) return launch_gemm_tc<false, true>(grid, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, sBias, act, Z, accumulate, ksplit, ctx, s);
        return launch_gemm_tc<false, false>(grid, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, sBias, act, Z, accumulate, ksplit, ctx, s);
    }
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, E);
    gemm_f32_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, tA, B, ldb, sB, tB, C, ldc, sC, bias, sBias, act, Z,
                                         accumulate);
    return cudaGetLastError();
}

// layer l: input width in_l, output width out_l
int in_w(const phx_mlp* m, int l) { return l == 0 ? m->n_in : m->width; }
int out_w(const phx_mlp* m, int l) { return l == m->depth ? 1 : m->width; }

}  // namespace

// Forward pass of every member on rows of xin: act[l + 1] = layer-l output, pre[l + 1] its
// pre-activation (act[0] is unused: layer 0 reads xin).
static phx_status mlp_forward(phx_mlp* m, int rows, cudaStream_t s) {
    const int64_t L = (int64_t)rows * m->width;
    const int64_t layer = (int64_t)m->E * L;
    for (int l = 0; l <= m->depth; ++l) {
        const float* in = l == 0 ? m->xin : m->act + (int64_t)l * layer;
        const int64_t s_in = l == 0 ? 0 : L;
        float* out = m->act + (int64_t)(l + 1) * layer;
        float* z = m->pre + (int64_t)(l + 1) * layer;
        const int ow = out_w(m, l);
        PHX_CUDA_CHECK(m->ctx, gemm(m->ctx, rows, ow, in_w(m, l), in, in_w(m, l), s_in, 0, m->par + m->w_off[l], ow, m->n_par,
                                    0, out, ow, L, m->par + m->b_off[l], m->n_par, l < m->depth ? 1 : 0, z, m->E, 0,
                                    s));
    }
    return PHX_OK;
}

// Backward pass for loss gradient dy [E][rows] (in dbuf); fills m->grad.
static phx_status mlp_backward(phx_mlp* m, int rows, cudaStream_t s) {
    const int64_t L = (int64_t)rows * m->width;
    const int64_t layer = (int64_t)m->E * L;
    float* d = m->dbuf0;    // gradient w.r.t. the output of layer l (post-activation)
    float* dn = m->dbuf1;
    // the weight gradients of the hidden layers are summed over K splits into a zeroed buffer
    PHX_CUDA_CHECK(m->ctx, cudaMemsetAsync(m->grad, 0, sizeof(float) * m->n_par * m->E, s));
    for (int l = m->depth; l >= 0; --l) {
        const int iw = in_w(m, l), ow = out_w(m, l);
        if (l < m->depth) {
            const int64_t cnt = (int64_t)m->E * rows * ow;
            silu_back_kernel<<<(int)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, s>>>(
                d, m->pre + (int64_t)(l + 1) * layer, cnt);
            PHX_CUDA_CHECK(m->ctx, cudaGetLastError());
        }
        // d is [E][rows][ow] with member stride L
        const float* in = l == 0 ? m->xin : m->act + (int64_t)l * layer;
        const int64_t s_in = l == 0 ? 0 : L;
        // dW = in^T d : [iw x ow]
        PHX_CUDA_CHECK(m->ctx, gemm(m->ctx, iw, ow, rows, in, iw, s_in, 1, d, ow, L, 0, m->grad + m->w_off[l], ow, m->n_par,
                                    nullptr, 0, 0, nullptr, m->E, 0, s, true));
        bias_grad_kernel<<<dim3((ow + 127) / 128, m->E), 128, 0, s>>>(d, rows, ow, L, m->grad + m->b_off[l], m->n_par);
        PHX_CUDA_CHECK(m->ctx, cudaGetLastError());
        if (l > 0) {
            // d_in = d W^T : [rows x iw]
            PHX_CUDA_CHECK(m->ctx, gemm(m->ctx, rows, iw, ow, d, ow, L, 0, m->par + m->w_off[l], ow, m->n_par, 1, dn, iw, L,
                                        nullptr, 0, 0, nullptr, m->E, 0, s));
            std::swap(d, dn);
        }
    }
    return PHX_OK;
}

extern "C" {

phx_status phx_mlp_create(phx_ctx* ctx, int32_t n_in, int32_t width, int32_t depth, int32_t ensemble, uint64_t seed,
                          phx_mlp** out) {
    if (!ctx || !out) return PHX_ERR_INVALID;
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || width < 1 || width > 1024 || depth < 1 || depth > 16 || ensemble < 1 || ensemble > 64)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_mlp_create: sizes out of range");
    cudaSetDevice(ctx->device);
    phx_mlp* m = new phx_mlp();
    m->ctx = ctx; m->n_in = n_in; m->width = width; m->depth = depth; m->E = ensemble; m->seed = seed;
    int64_t off = 0;
    for (int l = 0; l <= depth; ++l) {
        const int iw = in_w(m, l), ow = out_w(m, l);
        m->w_off.push_back(off); m->w_rows.push_back(iw); m->w_cols.push_back(ow);
        off += (int64_t)iw * ow;
        m->b_off.push_back(off);
        off += ow;
    }
    m->n_par = off;
    const size_t pb = sizeof(float) * off * ensemble;
    bool ok = cudaMalloc(&m->par, pb) == cudaSuccess && cudaMalloc(&m->grad, pb) == cudaSuccess &&
              cudaMalloc(&m->m1, pb) == cudaSuccess && cudaMalloc(&m->m2, pb) == cudaSuccess &&
              cudaMalloc(&m->mu, sizeof(float) * 64) == cudaSuccess && cudaMalloc(&m->sd, sizeof(float) * 64) == cudaSuccess &&
              cudaMalloc(&m->ymu, sizeof(float)) == cudaSuccess && cudaMalloc(&m->ysd, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->xlo, sizeof(float) * 64) == cudaSuccess &&
              cudaMalloc(&m->xhi, sizeof(float) * 64) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(double) * ensemble) == cudaSuccess &&
              cudaMalloc(&m->vloss, sizeof(double) * ensemble) == cudaSuccess &&
              cudaMalloc(&m->best, pb) == cudaSuccess &&
              cudaMalloc(&m->step, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        delete m;
        return phx_set_error(ctx, PHX_ERR_NOMEM, "phx_mlp_create: allocation failed");
    }
    cudaMemset(m->par, 0, pb);
    // weights U(-sqrt(6/fan_in)/.., ..) per layer and member (SiLU: He-style scale), biases 0
    for (int e = 0; e < ensemble; ++e)
        for (int l = 0; l <= depth; ++l) {
            const int64_t cnt = m->w_rows[l] * m->w_cols[l];
            const float a = sqrtf(6.f / (float)m->w_rows[l]);
            init_kernel<<<(int)((cnt + 255) / 256), 256>>>(m->par + e * off + m->w_off[l], cnt,
                                                        seed * 1000003ull + (uint64_t)(e * 131 + l), a);
        }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete m;
        return phx_set_error(ctx, PHX_ERR_CUDA, "phx_mlp_create: init failed");
    }
    float one = 1.f, zero = 0.f;
    for (int f = 0; f < 64; ++f) { cudaMemcpy(m->mu + f, &zero, 4, cudaMemcpyHostToDevice); cudaMemcpy(m->sd + f, &one, 4, cudaMemcpyHostToDevice); }
    // no training rows yet: every input is inside
    const float big = 3.0e38f, nbig = -3.0e38f;
    for (int f = 0; f < 64; ++f) {
        cudaMemcpy(m->xlo + f, &nbig, 4, cudaMemcpyHostToDevice);
        cudaMemcpy(m->xhi + f, &big, 4, cudaMemcpyHostToDevice);
    }
    cudaMemcpy(m->ymu, &zero, 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->ysd, &one, 4, cudaMemcpyHostToDevice);
    *out = m;
    return PHX_OK;
}

void phx_mlp_destroy(phx_mlp* m) {
    if (!m) return;
    cudaFree(m->par); cudaFree(m->grad); cudaFree(m->m1); cudaFree(m->m2);
    cudaFree(m->mu); cudaFree(m->sd); cudaFree(m->ymu); cudaFree(m->ysd); cudaFree(m->loss); cudaFree(m->step);
    cudaFree(m->xlo); cudaFree(m->xhi);
    cudaFree(m->vloss); cudaFree(m->best);
    cudaFree(m->act); cudaFree(m->pre); cudaFree(m->xin); cudaFree(m->ystd); cudaFree(m->dbuf0); cudaFree(m->dbuf1);
    delete m;
}

int64_t phx_mlp_num_params(const phx_mlp* m) { return m ? m->n_par : -1; }

phx_status phx_mlp_get_params(phx_mlp* m, float* host_params, float* host_norm) {
    if (!m || !host_params) return PHX_ERR_INVALID;
    PHX_CUDA_CHECK(m->ctx, cudaMemcpy(host_params, m->par, sizeof(float) * m->n_par * m->E, cudaMemcpyDeviceToHost));
    if (host_norm) {
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(host_norm, m->mu, sizeof(float) * m->n_in, cudaMemcpyDeviceToHost));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(host_norm + m->n_in, m->sd, sizeof(float) * m->n_in, cudaMemcpyDeviceToHost));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(host_norm + 2 * m->n_in, m->ymu, sizeof(float), cudaMemcpyDeviceToHost));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(host_norm + 2 * m->n_in + 1, m->ysd, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return PHX_OK;
}

phx_status phx_mlp_set_params(phx_mlp* m, const float* host_params, const float* host_norm) {
    if (!m || !host_params) return PHX_ERR_INVALID;
    PHX_CUDA_CHECK(m->ctx, cudaMemcpy(m->par, host_params, sizeof(float) * m->n_par * m->E, cudaMemcpyHostToDevice));
    if (host_norm) {
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(m->mu, host_norm, sizeof(float) * m->n_in, cudaMemcpyHostToDevice));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(m->sd, host_norm + m->n_in, sizeof(float) * m->n_in, cudaMemcpyHostToDevice));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(m->ymu, host_norm + 2 * m->n_in, sizeof(float), cudaMemcpyHostToDevice));
        PHX_CUDA_CHECK(m->ctx, cudaMemcpy(m->ysd, host_norm + 2 * m->n_in + 1, sizeof(float), cudaMemcpyHostToDevice));
    }
    return PHX_OK;
}

// Loss and gradient of every member on one batch (no update): loss[E] host, grad host
// [E][n_par] (may be NULL).  X [rows][n_in] and y [rows] are device memory (raw features and
// linewidths; the stored normalisation is applied).
phx_status phx_mlp_loss_grad(phx_mlp* m, const double* X, const double* y, int32_t rows, double* loss, float* grad,
                             void* stream) {
    if (!m || !X || !y || rows <= 0) return PHX_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    PHX_TRY(mlp_reserve(m, rows));
    input_kernel<<<256, 256, 0, s>>>(X, rows, m->n_in, m->mu, m->sd, m->xin);
    target_kernel<<<64, 256, 0, s>>>(y, rows, m->ymu, m->ysd, m->ystd);
    PHX_TRY(mlp_forward(m, rows, s));
    const int64_t L = (int64_t)rows * m->width;
    const int64_t layer = (int64_t)m->E * L;
    const float* yhat = m->act + (int64_t)(m->depth + 1) * layer;
    // outputs are [E][rows] with member stride L: compact them into dbuf0 as dy
    PHX_CUDA_CHECK(m->ctx, cudaMemsetAsync(m->loss, 0, sizeof(double) * m->E, s));
    loss_grad_all_kernel<<<64, 256, 0, s>>>(yhat, m->ystd, rows, m->E, L, m->dbuf0, m->loss);
    PHX_CUDA_CHECK(m->ctx, cudaGetLastError());
    PHX_TRY(mlp_backward(m, rows, s));
    if (loss) PHX_CUDA_CHECK(m->ctx, cudaMemcpyAsync(loss, m->loss, sizeof(double) * m->E, cudaMemcpyDeviceToHost, s));
    if (grad) PHX_CUDA_CHECK(m->ctx, cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->n_par * m->E, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(m->ctx, cudaStreamSynchronize(s));
    return PHX_OK;
}

}  // extern "C"

// Full-batch Adam training of every member on the first rows - n_val rows of (X, log y): sets
// the input/target standardisation from them, then runs epochs.  With n_val > 0 the last n_val
// rows are held out: their loss is evaluated every epoch, checked every check_every epochs,
// and training stops once it has not improved by 0.1 % for `patience` checks in a row; the
// parameters at the best check are restored.  Final training losses to loss[E] (host, may be
// NULL), epochs run to *epochs_run (may be NULL).
static phx_status mlp_train_impl(phx_mlp* m, const double* X, const double* y, int32_t rows, int32_t n_val,
                                 int32_t epochs, double lr, int32_t check_every, int32_t patience, double* loss,
                                 int32_t* epochs_run, void* stream) {
    phx_ctx* ctx = m->ctx;
    const int rows_tr = rows - n_val;
    cudaStream_t user = (cudaStream_t)stream;
    PHX_TRY(mlp_reserve(m, rows));
    if (!ctx->cap_stream) {
        PHX_CUDA_CHECK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        PHX_CUDA_CHECK(ctx, cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDefault));
        PHX_CUDA_CHECK(ctx, cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDefault));
    }
    cudaStream_t s = ctx->cap_stream;
    PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_in, user));
    PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s, ctx->ev_in, 0));
    moments_kernel<<<m->n_in, 256, 0, s>>>(X, rows_tr, m->n_in, 1, m->mu, m->sd);
    moments_kernel<<<1, 256, 0, s>>>(y, rows_tr, 1, 1, m->ymu, m->ysd);
    range_kernel<<<m->n_in, 256, 0, s>>>(X, rows_tr, m->n_in, m->xlo, m->xhi);
    input_kernel<<<256, 256, 0, s>>>(X, rows, m->n_in, m->mu, m->sd, m->xin);
    target_kernel<<<64, 256, 0, s>>>(y, rows, m->ymu, m->ysd, m->ystd);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    const int64_t np_all = m->n_par * m->E;
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(m->m1, 0, sizeof(float) * np_all, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(m->m2, 0, sizeof(float) * np_all, s));
    const int one = 1;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(m->step, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    const int64_t L = (int64_t)rows * m->width;
    const int64_t layer = (int64_t)m->E * L;
    const float* yhat = m->act + (int64_t)(m->depth + 1) * layer;
    // one epoch (forward, loss gradient, backward, Adam, step counter) as a graph; held-out rows
    // run forward with a zero gradient (their rows add nothing to the weight gradients)
    cudaGraphExec_t exec = nullptr;
    int done = 0;
    if (epochs > 0) {
        PHX_CUDA_CHECK(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        phx_status st = mlp_forward(m, rows, s);
        if (st == PHX_OK) {
            if (n_val > 0) {
                cudaMemsetAsync(m->vloss, 0, sizeof(double) * m->E, s);
                loss_grad_split_kernel<<<64, 256, 0, s>>>(yhat, m->ystd, rows_tr, rows, m->E, L, m->dbuf0, m->vloss);
            } else {
                loss_grad_all_kernel<<<64, 256, 0, s>>>(yhat, m->ystd, rows, m->E, L, m->dbuf0, nullptr);
            }
            if (cudaGetLastError() != cudaSuccess) st = PHX_ERR_CUDA;
        }
        if (st == PHX_OK) st = mlp_backward(m, rows, s);
        if (st == PHX_OK) {
            adam_kernel<<<(int)std::min<int64_t>((np_all + 255) / 256, 4096), 256, 0, s>>>(
                m->par, m->grad, m->m1, m->m2, np_all, (float)lr, 0.9f, 0.999f, 1e-8f, m->step);
            step_kernel<<<1, 1, 0, s>>>(m->step);
            if (cudaGetLastError() != cudaSuccess) st = PHX_ERR_CUDA;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (st != PHX_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return phx_set_error(ctx, st != PHX_OK ? st : PHX_ERR_CUDA, "phx_mlp_train: epoch capture failed");
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return phx_set_error(ctx, PHX_ERR_CUDA, "phx_mlp_train: instantiate failed");
        double best = 1e300;
        int bad = 0;
        bool have_best = false;
        std::vector<double> vl(m->E);
        for (int ep = 0; ep < epochs; ++ep) {
            const cudaError_t el = cudaGraphLaunch(exec, s);
            if (el != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return phx_set_error(ctx, PHX_ERR_CUDA, "phx_mlp_train: %s", cudaGetErrorString(el));
            }
            done = ep + 1;
            if (n_val > 0 && check_every > 0 && done % check_every == 0) {
                // held-out loss of the parameters before this epoch's update (the forward pass
                // of the epoch ran on them)
                PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(vl.data(), m->vloss, sizeof(double) * m->E, cudaMemcpyDeviceToHost, s));
                PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
                double mean = 0.0;
                for (double v : vl) mean += v / m->E;
                if (mean < best * (1.0 - 1e-3)) {
                    best = mean;
                    bad = 0;
                    have_best = true;
                    // the loss was taken on the parameters before this epoch's update; the copy
                    // kept is one Adam step later
                    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(m->best, m->par, sizeof(float) * np_all,
                                                        cudaMemcpyDeviceToDevice, s));
                } else if (++bad >= patience) {
                    break;
                }
            }
        }
        if (have_best)
            PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(m->par, m->best, sizeof(float) * np_all, cudaMemcpyDeviceToDevice, s));
        ctx->launches += (int64_t)done * (6 + 4 * (m->depth + 1));
    }
    if (epochs_run) *epochs_run = done;
    // final loss with the trained parameters (training rows)
    PHX_TRY(mlp_forward(m, rows, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(m->loss, 0, sizeof(double) * m->E, s));
    loss_grad_all_kernel<<<64, 256, 0, s>>>(yhat, m->ystd, rows_tr, m->E, L, m->dbuf0, m->loss);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    if (exec) {
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        cudaGraphExecDestroy(exec);
    }
    PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_out, s));
    PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(user, ctx->ev_out, 0));
    if (loss) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(loss, m->loss, sizeof(double) * m->E, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    return PHX_OK;
}

extern "C" {

phx_status phx_mlp_train(phx_mlp* m, const double* X, const double* y, int32_t rows, int32_t epochs, double lr,
                         double* loss, void* stream) {
    if (!m || !X || !y || rows <= 0 || epochs < 0 || !(lr > 0.0)) return PHX_ERR_INVALID;
    return mlp_train_impl(m, X, y, rows, 0, epochs, lr, 0, 0, loss, nullptr, stream);
}

phx_status phx_mlp_train_es(phx_mlp* m, const double* X, const double* y, int32_t rows, int32_t n_val,
                            int32_t max_epochs, double lr, int32_t check_every, int32_t patience, double* loss,
                            int32_t* epochs_run, void* stream) {
    if (!m) return PHX_ERR_INVALID;
    if (!X || !y || rows <= 0 || n_val < 1 || n_val >= rows || max_epochs < 0 || !(lr > 0.0) || check_every < 1 ||
        patience < 1)
        return phx_set_error(m->ctx, PHX_ERR_INVALID, "phx_mlp_train_es: bad argument");
    return mlp_train_impl(m, X, y, rows, n_val, max_epochs, lr, check_every, patience, loss, epochs_run, stream);
}

// Ensemble prediction of log(gamma): mean[rows] and std[rows] (device, std may be NULL).
phx_status phx_mlp_predict(phx_mlp* m, const double* X, int32_t rows, double* mean, double* stdv, void* stream) {
    if (!m || !X || !mean || rows <= 0) return PHX_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    PHX_TRY(mlp_reserve(m, rows));
    input_kernel<<<256, 256, 0, s>>>(X, rows, m->n_in, m->mu, m->sd, m->xin);
    PHX_TRY(mlp_forward(m, rows, s));
    const int64_t L = (int64_t)rows * m->width;
    const int64_t layer = (int64_t)m->E * L;
    const float* yhat = m->act + (int64_t)(m->depth + 1) * layer;
    // member outputs are L apart: gather through a strided view (compact into dbuf0 first)
    for (int e = 0; e < m->E; ++e)
        PHX_CUDA_CHECK(m->ctx, cudaMemcpyAsync(m->dbuf0 + (int64_t)e * rows, yhat + e * L, sizeof(float) * rows,
                                               cudaMemcpyDeviceToDevice, s));
    ensemble_kernel<<<(rows + 255) / 256, 256, 0, s>>>(m->dbuf0, rows, m->E, m->ymu, m->ysd, mean, stdv);
    PHX_CUDA_CHECK(m->ctx, cudaGetLastError());
    m->ctx->launches += 2 + (m->depth + 1);
    return PHX_OK;
}

phx_status phx_mlp_outside(phx_mlp* m, const double* X, int32_t rows, int32_t* outside, void* stream) {
    if (!m || !X || !outside || rows <= 0) return PHX_ERR_INVALID;
    cudaSetDevice(m->ctx->device);
    outside_kernel<<<(int)std::min<int64_t>((rows + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(
        X, rows, m->n_in, m->xlo, m->xhi, outside);
    PHX_CUDA_CHECK(m->ctx, cudaGetLastError());
    m->ctx->launches += 1;
    return PHX_OK;
}

phx_status phx_mlp_reconstruct(phx_ctx* ctx, int32_t n_groups, int32_t n, const double* mean, const double* stdv,
                               const double* wp2, const double* freq_thz, double f_min_thz, const int32_t* outside,
                               double* gamma, double* score, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (n_groups <= 0 || n <= 0 || !mean || !freq_thz || !gamma)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_mlp_reconstruct: bad argument");
    if (score && !stdv) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_mlp_reconstruct: score needs stdv");
    cudaSetDevice(ctx->device);
    reconstruct_kernel<<<n_groups, 256, 0, (cudaStream_t)stream>>>(n, mean, stdv, wp2, freq_thz, f_min_thz, outside,
                                                                   gamma, score);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 1;
    return PHX_OK;
}

// Descriptors of every band of the irreducible q-points on a mesh (see the file header):
// out[n_irr][n][4] = (w rad/ps, |v| A/ps, WP2 ps^4, n_B).  freq, vel over the full mesh.
phx_status phx_features(phx_ctx* ctx, const int32_t mesh[3], int32_t n, const double* freq_thz, const double* vel,
                        const int32_t* irr_q, int32_t n_irr, double temperature, phx_broadening br, double f_min_thz,
                        double* features, void* stream) {
    if (!ctx || !mesh || !freq_thz || !vel || !irr_q || !features || n <= 0 || n_irr <= 0)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_features: bad argument");
    if (!(temperature > 0.0) || !(br.sigma_thz > 0.0) || !(br.window > 0.0) || !(f_min_thz > 0.0))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_features: T, sigma, window and f_min must be > 0");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int nq = mesh[0] * mesh[1] * mesh[2];
    double* nB = (double*)phx_ws(ctx, "s.nB", (size_t)nq * n * 8);
    double* wsum = (double*)phx_ws(ctx, "s.wsum", (size_t)n_irr * n * 8);
    if (!nB || !wsum) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, phx_launch_occupations(freq_thz, nq * n, temperature, 0, nB, nullptr, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(wsum, 0, (size_t)n_irr * n * 8, s));
    if (n > 192) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_features: n = %d > 192", n);
    if (n_irr > 65535) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_features: n_irr > 65535");
    features_kernel<<<dim3((nq + 255) / 256, n_irr), 256, 0, s>>>(freq_thz, nB, irr_q, n, mesh[0], mesh[1], mesh[2],
                                                                  (float)br.sigma_thz, (float)br.window, br.shape,
                                                                  (float)f_min_thz, wsum);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    features_finish_kernel<<<(n_irr * n + 255) / 256, 256, 0, s>>>(freq_thz, vel, nB, irr_q, n_irr, n, nq, f_min_thz,
                                                                  wsum, features);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 3;
    return PHX_OK;
}

}  // extern "C"
