// Batched complex GEMM on the CUDA cores (row-major): C_b = opA(A_b) * B_b with per-batch
// addressing from ZgemmBatch, FP64 inputs and output.  The products and sums run in FP64 (the
// arithmetic of the FP64 reference path) or, with p.fp32, in FP32 (operands rounded once when
// staged; GB300's FP32 pipe is tens of times wider than its FP64 one).  64x64 output tile per
// CTA, K staged 8 at a time through shared memory, each of the 256 threads accumulating a 4x4
// block of outputs strided by 16 (coalesced stores).
#include "common.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 8;

template <typename C2>      // double2 or float2: the precision of the products and sums
__global__ void __launch_bounds__(256)
zgemm_kernel(int M, int N, int K, ZgemmBatch p) {
    using R = decltype(C2{}.x);
    __shared__ C2 As[BK][BM + 1];
    __shared__ C2 Bs[BK][BN + 1];
    const int b = blockIdx.z;
    if (p.skip && p.skip[b / p.skip_div]) return;
    const int64_t ia = p.idxA ? (int64_t)p.idxA[b / p.divA] : (int64_t)(b / p.divA);
    const int64_t ib = p.idxB ? (int64_t)p.idxB[b / p.divB] : (int64_t)(b / p.divB);
    const double2* A = (const double2*)p.A + ia * p.strideA;
    const double2* B = (const double2*)p.B + ib * p.strideB + (int64_t)(b % p.divB) * p.strideB_inner;
    double2* C = (double2*)p.C + (int64_t)b * p.strideC;

    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    C2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = C2{R(0), R(0)};

    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int m, k;
            if (p.transA) { k = e / BM; m = e % BM; } else { m = e / BK; k = e % BK; }
            const int gm = m0 + m, gk = k0 + k;
            double2 v = make_double2(0.0, 0.0);
            if (gm < M && gk < K)
                v = p.transA ? A[(int64_t)gk * p.lda + gm] : A[(int64_t)gm * p.lda + gk];
            As[k][m] = C2{R(v.x), R(v.y)};
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int k = e / BN, n = e % BN;
            const int gn = n0 + n, gk = k0 + k;
            const double2 v = (gn < N && gk < K) ? B[(int64_t)gk * p.ldb + gn] : make_double2(0.0, 0.0);
            Bs[k][n] = C2{R(v.x), R(v.y)};
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            C2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, bb[j].x, fma(-a[i].y, bb[j].y, acc[i][j].x));
                    acc[i][j].y = fma(a[i].x, bb[j].y, fma(a[i].y, bb[j].x, acc[i][j].y));
                }
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
            if (gn < N) C[(int64_t)gm * p.ldc + gn] = make_double2((double)acc[i][j].x, (double)acc[i][j].y);
        }
    }
}

}  // namespace

cudaError_t phx_launch_zgemm(int M, int N, int K, int batch, const ZgemmBatch& p, cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535) return cudaErrorInvalidValue;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    if (p.fp32)
        zgemm_kernel<float2><<<grid, 256, 0, s>>>(M, N, K, p);
    else
        zgemm_kernel<double2><<<grid, 256, 0, s>>>(M, N, K, p);
    return cudaGetLastError();
}
