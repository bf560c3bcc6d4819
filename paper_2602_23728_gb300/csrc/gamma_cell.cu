// Gamma-only three-phonon linewidths of a large (disordered) cell: paper Sec. "Three-Phonon
// Scattering", Eq. (phi3_proj) at q = q' = q'' = 0 with the real eigenvectors of Eq.
// (eigenvalue), Eq. (gamma) with N_q = 1 and the broadening of Eq. (broadening) (Lorentzian or
// Gaussian, terms outside the window dropped).
//
// Phi(a, b, c) = sum_ijk F[i][j][k] e_a[i] e_b[j] e_c[k], F = Phi3 / sqrt(m m m), is symmetric in
// (a, b, c) because Phi3 is a third derivative (the COO is symmetrised when the handle is made),
// so every unordered triple a <= b <= c is evaluated once and credited to the three linewidths
// it enters.  With K = Phi^2 / ((2 pi)^4 f_a f_b f_c) and the three shared deltas
//     D1 = g(f_a + f_b - f_c),  D2 = g(f_a - f_b + f_c),  D3 = g(-f_a + f_b + f_c)
//     S_a = (1 + n_b + n_c) D3 + (n_b - n_c)(D1 - D2)
//     S_b = (1 + n_a + n_c) D2 + (n_a - n_c)(D1 - D3)
//     S_c = (1 + n_a + n_b) D1 + (n_a - n_b)(D2 - D3)
// the ordered-pair sum of Eq. (gamma) regroups into
//     gamma_a += 2 K S_a (halved if b = c),  gamma_b += 2 K S_b (if b != a),
//     gamma_c += 2 K S_c (halved if a = b; only if c != b).
//
// For each chunk of consecutive modes a that have any in-window triple:
//   w_kernel          W_a[j][k] = sum_i F[i][j][k] e_a[i]   (sparse, 3x3 atom-pair blocks)
//   xform_kernel      X_a[j][c] = sum_k W_a[j][k] E[k][c]    (CUDA cores; c >= c_base(chunk))
//   transpose_kernel  X_a -> XT_a[c][j] in the K-major operand layout (BF16 hi/lo, TF32, FP64)
//   sym_tc_kernel     Phi[b][c] = sum_j ET[b][j] XT_a[c][j] on the tcgen05 tensor cores, 128 x 128
//                     tiles, over the (b-tile, c-tile) pairs of a whose frequency ranges admit
//                     an in-window triple; role weights and the three reductions fused into the
//                     epilogue (sym_fp64_kernel: the same on FP64 CUDA cores).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kTile = 128;                 // output tile edge (b and c)
constexpr int kEpiThreads = 256;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kChunkBytes = 128;
constexpr int kTileBytes = kTile * kChunkBytes;     // one 128-row x 128-byte operand box
constexpr int kMaxStages = 8;
constexpr size_t kSmemDyn = 232448 - 8192;

enum { P_BF16X3 = 0, P_TF32 = 1, P_FP64 = 2 };

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- table kernels

// Re(evec) into two row-major tables of pitch pe (zero beyond n); flags non-real input.
__global__ void real_tables_kernel(const double2* __restrict__ evec, int n, int pe, double* __restrict__ e64,
                                   float* __restrict__ e32, int32_t* __restrict__ status) {
    const int64_t total = (int64_t)n * pe;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / pe), c = (int)(t % pe);
        double v = 0.0;
        if (c < n) {
            const double2 z = evec[(int64_t)k * n + c];
            v = z.x;
            if (z.y != 0.0) atomicExch(status, (int)PHX_ERR_INVALID);
        }
        e64[t] = v;
        if (e32) e32[t] = (float)v;
    }
}

// per-mode table (f, n_B, 1/f or 0 below f_min) for padded index range [0, pe)
__global__ void mode_table_kernel(const double* __restrict__ freq, const double* __restrict__ nB, int n, int pe,
                                  double f_min, float4* __restrict__ t32, double* __restrict__ t64) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= pe) return;
    double f = 0.0, o = 0.0, inv = 0.0;
    if (b < n) {
        f = freq[b];
        if (f >= f_min) { o = nB[b]; inv = 1.0 / f; } else { f = 0.0; }
    }
    t32[b] = make_float4((float)f, (float)o, (float)inv, 0.0f);
    t64[3 * b] = f;
    t64[3 * b + 1] = o;
    t64[3 * b + 2] = inv;
}

// W[asub][seg][la] = sum over the entries of seg of F * e_{a}[i], a = chunk_a[asub * LA + la]
template <typename T, int LA>
__global__ void w_kernel(const int64_t* __restrict__ seg_start, const int32_t* __restrict__ ent_i,
                         const double* __restrict__ ent_w, int64_t n_seg, const double* __restrict__ e64, int pe,
                         const int32_t* __restrict__ chunk_a, int L, int n_asub, T* __restrict__ W) {
    const int64_t total = (int64_t)n_asub * n_seg * LA;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int la = (int)(t % LA);
        const int64_t rest = t / LA;
        const int64_t seg = rest % n_seg;
        const int al = (int)(rest / n_seg) * LA + la;
        double acc = 0.0;
        if (al < L) {
            const int a = chunk_a[al];
            for (int64_t e = seg_start[seg]; e < seg_start[seg + 1]; ++e) acc += ent_w[e] * e64[(int64_t)ent_i[e] * pe + a];
        }
        W[t] = (T)acc;
    }
}

// X[al][j][cc] = sum_{k in nbr(J)} W_a[j][k] E[k][c_base + cc].  A CTA covers NC x 256 columns
// (thread t: columns t, t + 256, ...), LA modes and the atom rows J in [blockIdx.y * tj, ...);
// W of the current J is staged in shared memory and read as LA-wide vectors, each value
// feeding NC columns.
template <typename T, int LA, int NC>
__global__ void __launch_bounds__(256)
xform_kernel(const T* __restrict__ E, int pe, const T* __restrict__ W, int64_t n_seg,
             const int32_t* __restrict__ nbr_start, const int32_t* __restrict__ nbr_atom, int na, int n, int c_base,
             int ncc, int tj, int L, T* __restrict__ X) {
    static_assert(LA % 4 == 0, "LA must be a multiple of 4");
    extern __shared__ __align__(16) uint8_t xs_raw[];
    T* Ws = (T*)xs_raw;
    int cc[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) cc[u] = blockIdx.x * (256 * NC) + u * 256 + threadIdx.x;
    const int asub = blockIdx.z;
    const T* Wsub = W + (int64_t)asub * n_seg * LA;
    const int J0 = blockIdx.y * tj, J1 = min(na, J0 + tj);
    for (int J = J0; J < J1; ++J) {
        const int s0 = nbr_start[J], ns = nbr_start[J + 1] - s0;
        const T* src = Wsub + (int64_t)s0 * 9 * LA;
        for (int t = threadIdx.x; t < ns * 9 * LA; t += 256) Ws[t] = src[t];
        __syncthreads();
        T acc[NC][LA][3];
#pragma unroll
        for (int u = 0; u < NC; ++u)
#pragma unroll
            for (int la = 0; la < LA; ++la) acc[u][la][0] = acc[u][la][1] = acc[u][la][2] = T(0);
        // E rows of the next neighbour are loaded while the current one is consumed
        T en[NC][3];
        {
            const int64_t k0 = (int64_t)(3 * nbr_atom[s0]) * pe + c_base;
#pragma unroll
            for (int u = 0; u < NC; ++u)
#pragma unroll
                for (int g = 0; g < 3; ++g) en[u][g] = (ns > 0 && cc[u] < ncc) ? E[k0 + g * pe + cc[u]] : T(0);
        }
        for (int s = 0; s < ns; ++s) {
            T e[NC][3];
#pragma unroll
            for (int u = 0; u < NC; ++u)
#pragma unroll
                for (int g = 0; g < 3; ++g) e[u][g] = en[u][g];
            if (s + 1 < ns) {
                const int64_t k1 = (int64_t)(3 * nbr_atom[s0 + s + 1]) * pe + c_base;
#pragma unroll
                for (int u = 0; u < NC; ++u)
#pragma unroll
                    for (int g = 0; g < 3; ++g) en[u][g] = cc[u] < ncc ? E[k1 + g * pe + cc[u]] : T(0);
            }
            const T* w = Ws + s * 9 * LA;
#pragma unroll
            for (int g = 0; g < 3; ++g)
#pragma unroll
                for (int be = 0; be < 3; ++be)
#pragma unroll
                    for (int l4 = 0; l4 < LA; l4 += 4) {
                        T wv[4];
                        if (sizeof(T) == 4) {
                            const float4 q = *reinterpret_cast<const float4*>(w + (g * 3 + be) * LA + l4);
                            wv[0] = (T)q.x; wv[1] = (T)q.y; wv[2] = (T)q.z; wv[3] = (T)q.w;
                        } else {
                            const double2 q0 = *reinterpret_cast<const double2*>(w + (g * 3 + be) * LA + l4);
                            const double2 q1 = *reinterpret_cast<const double2*>(w + (g * 3 + be) * LA + l4 + 2);
                            wv[0] = (T)q0.x; wv[1] = (T)q0.y; wv[2] = (T)q1.x; wv[3] = (T)q1.y;
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int u = 0; u < NC; ++u) acc[u][l4 + i][be] += e[u][g] * wv[i];
                    }
        }
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            if (cc[u] >= ncc) continue;
#pragma unroll
            for (int la = 0; la < LA; ++la) {
                const int al = asub * LA + la;
                if (al < L)
#pragma unroll
                    for (int be = 0; be < 3; ++be) X[((int64_t)al * n + 3 * J + be) * ncc + cc[u]] = acc[u][la][be];
            }
        }
        __syncthreads();
    }
}

// out[z][r][j] = in[z][j][r] (rows r < R_out, j < K_out; zero outside in's R x C), in the
// operand format of PREC.  32 x 32 tiles through shared memory.
template <typename Tin, int PREC>
__global__ void transpose_kernel(const Tin* __restrict__ in, int64_t in_zstride, int in_pitch, int rows_in,
                                 int cols_in, void* __restrict__ out_hi, void* __restrict__ out_lo,
                                 int64_t out_zstride, int out_pitch, int rows_out) {
    __shared__ Tin tile[32][33];
    const int z = blockIdx.z;
    const int j0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;         // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        const int j = j0 + yy, r = r0 + tx;
        Tin v = Tin(0);
        if (j < rows_in && r < cols_in) v = in[(int64_t)z * in_zstride + (int64_t)j * in_pitch + r];
        tile[yy][tx] = v;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int r = r0 + yy, j = j0 + tx;
        if (r >= rows_out || j >= out_pitch) continue;
        const double v = (double)tile[tx][yy];
        const int64_t idx = (int64_t)z * out_zstride + (int64_t)r * out_pitch + j;
        if (PREC == P_BF16X3) {
            __nv_bfloat16 h, l;
            tc::split_bf16((float)v, &h, &l);
            ((__nv_bfloat16*)out_hi)[idx] = h;
            ((__nv_bfloat16*)out_lo)[idx] = l;
        } else if (PREC == P_TF32) {
            ((float*)out_hi)[idx] = tc::round_tf32((float)v);
        } else {
            ((double*)out_hi)[idx] = v;
        }
    }
}

// ---------------------------------------------------------------- role weights

template <typename T>
__device__ __forceinline__ T broad(T x, T lim, T p1, int shape) {
    // unnormalised g: Gauss exp(-x^2/s^2) (p1 = -1/s^2), Lorentz 1/(x^2 + h^2) (p1 = h^2)
    const T ax = x < T(0) ? -x : x;
    if (!(ax < lim)) return T(0);
    if (shape == PHX_GAUSS) return sizeof(T) == 4 ? (T)__expf((float)(p1 * x * x)) : (T)exp((double)(p1 * x * x));
    return T(1) / (x * x + p1);
}

// Contributions of one element (a <= b <= c enforced by the masks) to gamma_a, gamma_b, gamma_c.
template <typename T>
__device__ __forceinline__ void role_weights(T v, T fa, T na_, T ia, T fb, T nb, T ib, T fc, T nc, T ic, bool valid,
                                             bool a_eq_b, bool b_eq_c, T lim, T p1, int shape, T& ga, T& gb,
                                             T& gc) {
    const T K = valid ? v * v * ia * ib * ic : T(0);
    const T d1 = broad<T>(fa + fb - fc, lim, p1, shape);
    const T d2 = broad<T>(fa - fb + fc, lim, p1, shape);
    const T d3 = broad<T>(fb + fc - fa, lim, p1, shape);
    const T sa = (T(1) + nb + nc) * d3 + (nb - nc) * (d1 - d2);
    const T sb = (T(1) + na_ + nc) * d2 + (na_ - nc) * (d1 - d3);
    const T sc = (T(1) + na_ + nb) * d1 + (na_ - nb) * (d2 - d3);
    ga += K * (b_eq_c ? T(0.5) : T(1)) * sa;
    gb += a_eq_b ? T(0) : K * sb;
    gc = b_eq_c ? T(0) : K * (a_eq_b ? T(0.5) : T(1)) * sc;
}

// ---------------------------------------------------------------- tensor-core GEMM

struct SymArgs {
    CUtensorMap a_map[2];
    CUtensorMap b_map[2];
    const int4* items;          // (a_local, b-tile, c-tile, 0)
    int n_items;
    int nk;                     // K chunks of 128 bytes
    int stages;
    int ncc;                    // B rows per a_local
    int c_base;
    uint32_t tmem_cols;
    int32_t* status;
    const int32_t* chunk_a;
    const float4* tab;          // (f, n_B, 1/f, 0) per padded mode
    int n;
    float lim, p1;
    int shape;
    double* gacc;
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) sym_tc_kernel(const __grid_constant__ SymArgs args) {
    constexpr int kPlanes = PREC == P_BF16X3 ? 2 : 1;
    constexpr uint32_t kFmt = PREC == P_BF16X3 ? 1u : 2u;
    constexpr uint32_t kStageBytes = kPlanes * 2 * kTileBytes;          // A and B boxes per plane
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = args.nk, stages = args.stages;
    const int it0 = (int)((int64_t)args.n_items * blockIdx.x / gridDim.x);
    const int it1 = (int)((int64_t)args.n_items * (blockIdx.x + 1) / gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) { tc::mbar_init(&full_bar[s], 1); tc::mbar_init(&empty_bar[s], 1); }
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&tfull_bar[a], 1); tc::mbar_init(&tempty_bar[a], kEpiThreads); }
        tc::mbar_init(&drain_bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0)
        for (int pl = 0; pl < kPlanes; ++pl) { tc::prefetch_tmap(&args.a_map[pl]); tc::prefetch_tmap(&args.b_map[pl]); }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, args.tmem_cols);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool pending[kMaxStages];
            uint32_t pend_phase[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) { pending[s] = false; pend_phase[s] = 0; }
            const int kel = kChunkBytes / (PREC == P_BF16X3 ? 2 : 4);
            for (int it = it0; it < it1 && !abort_flag; ++it) {
                const int4 w = args.items[it];
                const int arow = w.y * kTile;
                const int brow = w.x * args.ncc + w.z * kTile - args.c_base;
                for (int kc = 0; kc < nk; ++kc) {
                    if (!tc::mbar_wait(&empty_bar[stage], phase ^ 1, &abort_flag)) {
                        abort_flag = 1;
                        atomicExch(args.status, (int)PHX_ERR_TIMEOUT);
                        break;
                    }
                    pending[stage] = false;
                    uint8_t* st = smem + (size_t)stage * kStageBytes;
                    tc::mbar_expect_tx(&full_bar[stage], kStageBytes);
                    for (int pl = 0; pl < kPlanes; ++pl) {
                        tc::tma_load_2d(st + pl * kTileBytes, &args.a_map[pl], &full_bar[stage], kc * kel, arow);
                        tc::tma_load_2d(st + (kPlanes + pl) * kTileBytes, &args.b_map[pl], &full_bar[stage], kc * kel,
                                        brow);
                    }
                    pending[stage] = true;
                    pend_phase[stage] = phase;
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
            }
            if (abort_flag) {
                for (int s = 0; s < stages; ++s)
                    if (pending[s]) {
                        const uint64_t t0 = tc::global_ns();
                        while (!tc::mbar_try_wait(&full_bar[s], pend_phase[s]) &&
                               tc::global_ns() - t0 < tc::kWaitLimitNs) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id = tc::idesc(kTile, kTile, kFmt);
            const uint32_t base = tc::smem_u32(smem);
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            for (int it = it0; ok && it < it1; ++it) {
                if (!tc::mbar_wait(&tempty_bar[acc], acc_phase ^ 1, &abort_flag)) {
                    abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); break;
                }
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kTile);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!tc::mbar_wait(&full_bar[stage], phase, &abort_flag)) {
                        abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); ok = false; break;
                    }
                    tc::tc_fence_after();
                    const uint32_t sa = base + (uint32_t)stage * kStageBytes;
                    const uint32_t sb = sa + kPlanes * kTileBytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t ko = (uint32_t)k * 32;
                        const uint32_t accf = (kc | k) ? 1u : 0u;
                        if (PREC == P_BF16X3) {
                            const uint64_t ah = tc::sdesc_sw128(sa + ko), al = tc::sdesc_sw128(sa + kTileBytes + ko);
                            const uint64_t bh = tc::sdesc_sw128(sb + ko), bl = tc::sdesc_sw128(sb + kTileBytes + ko);
                            tc::mma_f16(d_tmem, ah, bh, id, accf);
                            tc::mma_f16(d_tmem, ah, bl, id, 1u);
                            tc::mma_f16(d_tmem, al, bh, id, 1u);
                        } else {
                            tc::mma_tf32(d_tmem, tc::sdesc_sw128(sa + ko), tc::sdesc_sw128(sb + ko), id, accf);
                        }
                    }
                    tc::mma_commit(&empty_bar[stage]);
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                tc::mma_commit(&tfull_bar[acc]);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1;
            }
            tc::mma_commit(&drain_bar);
            const uint64_t t0 = tc::global_ns();
            while (!tc::mbar_try_wait(&drain_bar, 0) && tc::global_ns() - t0 < tc::kWaitLimitNs) {
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        const int lgrp = warp & 3, half = (warp - 2) >> 2;
        int acc = 0;
        uint32_t acc_phase = 0;
        const float lim = args.lim, p1 = args.p1;
        for (int it = it0; it < it1; ++it) {
            const bool ok = tc::mbar_wait(&tfull_bar[acc], acc_phase, &abort_flag);
            if (!ok) { abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); }
            epi_sync();
            if (abort_flag) break;
            tc::tc_fence_after();
            const int4 w = args.items[it];
            const int a = args.chunk_a[w.x];
            const int b = w.y * kTile + lgrp * 32 + lane;
            const float4 ta = args.tab[a], tb = args.tab[b];
            const uint32_t taddr = tmem_base + ((uint32_t)(lgrp * 32) << 16) + (uint32_t)(acc * kTile);
            float ga = 0.f, gb = 0.f;
            for (int j0 = half * 16; j0 < kTile; j0 += 32) {
                float v[16];
                tc::tmem_ld16(taddr + j0, v);
                const int c0 = w.z * kTile + j0;
                float gc[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    const float4 tcv = args.tab[c];
                    const bool valid = b < args.n && c < args.n && b >= a && c >= b;
                    role_weights<float>(v[i], ta.x, ta.y, ta.z, tb.x, tb.y, tb.z, tcv.x, tcv.y, tcv.z, valid, a == b,
                                        b == c, lim, p1, args.shape, ga, gb, gc[i]);
                }
                // column sums over the warp's 32 rows: recursive halving, lane l ends with column
                // ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 + ((l >> 2) & 1) * 2 + ((l >> 1) & 1)
#pragma unroll
                for (int s = 8, off = 16; s >= 1; s >>= 1, off >>= 1) {
                    const bool up = (lane & off) != 0;
#pragma unroll
                    for (int i = 0; i < s; ++i) {
                        const float send = up ? gc[i] : gc[i + s];
                        const float keep = up ? gc[i + s] : gc[i];
                        gc[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    }
                }
                gc[0] += __shfl_xor_sync(0xffffffffu, gc[0], 1);
                if ((lane & 1) == 0) {
                    const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                    const int c = c0 + col;
                    if (gc[0] != 0.f && c < args.n) atomicAdd(&args.gacc[c], (double)gc[0]);
                }
            }
            if (gb != 0.f && b < args.n) atomicAdd(&args.gacc[b], (double)gb);
            for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
            if (lane == 0 && ga != 0.f) atomicAdd(&args.gacc[a], (double)ga);
            tc::tc_fence_before();
            tc::mbar_arrive(&tempty_bar[acc]);
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, args.tmem_cols);
    }
}

// ---------------------------------------------------------------- FP64 CUDA-core GEMM

// One CTA per item: 128 x 128 tile, 256 threads x (8 x 8) outputs, K in steps of 16.
__global__ void __launch_bounds__(256)
sym_fp64_kernel(const double* __restrict__ ET, const double* __restrict__ XT, int kpad, int ncc, int c_base,
                const int4* __restrict__ items, const int32_t* __restrict__ chunk_a, const double* __restrict__ tab,
                int n, double lim, double p1, int shape, double* __restrict__ gacc) {
    __shared__ double As[16][kTile + 1], Bs[16][kTile + 1];
    __shared__ double rowacc[kTile], colacc[kTile], aacc;
    const int4 w = items[blockIdx.x];
    const int a = chunk_a[w.x];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double* Ab = ET + (int64_t)w.y * kTile * kpad;
    const double* Bb = XT + ((int64_t)w.x * ncc + (int64_t)w.z * kTile - c_base) * kpad;
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < kpad; k0 += 16) {
        for (int t = threadIdx.x; t < kTile * 16; t += 256) {
            const int r = t >> 4, k = t & 15;
            As[k][r] = Ab[(int64_t)r * kpad + k0 + k];
            Bs[k][r] = Bb[(int64_t)r * kpad + k0 + k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double ar[8], br[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) { ar[i] = As[k][ty + 16 * i]; br[i] = Bs[k][tx + 16 * i]; }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fma(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < kTile; t += 256) { rowacc[t] = 0.0; colacc[t] = 0.0; }
    if (threadIdx.x == 0) aacc = 0.0;
    __syncthreads();
    const double fa = tab[3 * a], na_ = tab[3 * a + 1], ia = tab[3 * a + 2];
    double ga = 0.0, colp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) colp[j] = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int b = w.y * kTile + ty + 16 * i;
        const double fb = tab[3 * b], nb = tab[3 * b + 1], ib = tab[3 * b + 2];
        double gb = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = w.z * kTile + tx + 16 * j;
            const bool valid = b < n && c < n && b >= a && c >= b;
            double gc = 0.0;
            role_weights<double>(acc[i][j], fa, na_, ia, fb, nb, ib, tab[3 * c], tab[3 * c + 1], tab[3 * c + 2], valid,
                                 a == b, b == c, lim, p1, shape, ga, gb, gc);
            colp[j] += gc;
        }
        if (gb != 0.0) atomicAdd(&rowacc[ty + 16 * i], gb);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (colp[j] != 0.0) atomicAdd(&colacc[tx + 16 * j], colp[j]);
    if (ga != 0.0) atomicAdd(&aacc, ga);
    __syncthreads();
    for (int t = threadIdx.x; t < kTile; t += 256) {
        const int b = w.y * kTile + t, c = w.z * kTile + t;
        if (rowacc[t] != 0.0 && b < n) atomicAdd(&gacc[b], rowacc[t]);
        if (colacc[t] != 0.0 && c < n) atomicAdd(&gacc[c], colacc[t]);
    }
    if (threadIdx.x == 0 && aacc != 0.0) atomicAdd(&gacc[a], aacc);
}

__global__ void finalize_cell_kernel(const double* __restrict__ freq, const double* __restrict__ gacc, int n,
                                     double scale, double f_min, double* __restrict__ gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gamma[i] = freq[i] >= f_min ? scale * gacc[i] : 0.0;
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

// 2D map over a row-major [rows][kr] operand plane; box = 128-byte K chunk x 128 rows.
bool make_map(CUtensorMap* m, const void* base, int prec, int64_t rows, int kr) {
    const int esz = prec == P_BF16X3 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)kr, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kr * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / esz), (cuuint32_t)kTile};
    cuuint32_t es[2] = {1, 1};
    return g_encode(m, prec == P_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Chunk {
    int a_begin, a_end;        // range in the work list
    int c_base;                // first column (multiple of 128)
    int item_begin, item_end;  // range in the item list
};

// Tiles of each mode a that can hold an in-window triple a <= b <= c: interval test of
// f_a + f_b - f_c, f_a - f_b + f_c and -f_a + f_b + f_c over the tile's frequency ranges.
void plan_tiles(const std::vector<double>& f, double f_min, double lim, std::vector<int>& work_a,
                std::vector<int4>& items, std::vector<int>& item_start, std::vector<int>& c_lo) {
    const int n = (int)f.size();
    const int nt = (n + kTile - 1) / kTile;
    std::vector<double> lo(nt, 1e300), hi(nt, -1e300);
    for (int i = 0; i < n; ++i)
        if (f[i] >= f_min) { lo[i / kTile] = std::min(lo[i / kTile], f[i]); hi[i / kTile] = std::max(hi[i / kTile], f[i]); }
    auto hits = [&](double x0, double x1) { return x1 > -lim && x0 < lim; };
    for (int a = 0; a < n; ++a) {
        if (!(f[a] >= f_min)) continue;
        const double fa = f[a];
        const int first = (int)items.size();
        int clo = n;
        for (int bt = a / kTile; bt < nt; ++bt) {
            if (lo[bt] > hi[bt]) continue;
            for (int ct = bt; ct < nt; ++ct) {
                if (lo[ct] > hi[ct]) continue;
                const bool keep = hits(fa + lo[bt] - hi[ct], fa + hi[bt] - lo[ct]) ||
                                  hits(fa - hi[bt] + lo[ct], fa - lo[bt] + hi[ct]) ||
                                  hits(-fa + lo[bt] + lo[ct], -fa + hi[bt] + hi[ct]);
                if (!keep) continue;
                items.push_back(make_int4((int)work_a.size(), bt, ct, 0));   // a_local fixed up per chunk
                clo = std::min(clo, ct * kTile);
            }
        }
        if ((int)items.size() > first) {
            work_a.push_back(a);
            item_start.push_back(first);
            c_lo.push_back(clo);
        }
    }
    item_start.push_back((int)items.size());
}

}  // namespace

// ---------------------------------------------------------------- entry point

extern "C" phx_status phx_gamma_cell(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz, const double* evec,
                                     double temperature, phx_broadening br, double f_min_thz, int32_t prec,
                                     double* gamma, int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!fc3 || fc3->ctx != ctx) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: bad fc3 handle");
    if (!freq_thz || !evec || !gamma) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: null argument");
    if (!fc3->g0_ready)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: fc3 handle was not made for a 1x1x1 mesh");
    if (!(temperature > 0.0) || !(br.sigma_thz > 0.0) || !(br.window > 0.0) || !(f_min_thz > 0.0) ||
        !std::isfinite(f_min_thz) || !std::isfinite(temperature) || !std::isfinite(br.sigma_thz))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: T, sigma, window and f_min must be finite and > 0");
    if (br.shape != PHX_GAUSS && br.shape != PHX_LORENTZ)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: unknown broadening shape %d", br.shape);
    if (prec != PHX_FP64 && prec != PHX_TF32 && prec != PHX_BF16X3)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: unknown precision %d", prec);
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: bad mem flag %d", mem);
    const int P = prec == PHX_FP64 ? P_FP64 : prec == PHX_TF32 ? P_TF32 : P_BF16X3;
    if (P != P_FP64 && (ctx->cc_major != 10 || !get_encoder()))
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_gamma_cell: tensor-core path needs sm_100-family TMA");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = fc3->n, na = n / 3;
    const int pe = round_up(n, kTile);                       // padded mode index range
    const int kel = P == P_BF16X3 ? 64 : P == P_TF32 ? 32 : 16;
    const int kpad = round_up(n, kel);                      // padded K (atom components)
    const int nk = kpad * (P == P_BF16X3 ? 2 : 4) / kChunkBytes;

    const double *d_f = nullptr, *d_e = nullptr;
    PHX_TRY(phx_stage_in(ctx, "gc.f", freq_thz, (size_t)n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "gc.e", evec, (size_t)n * n * 2, mem, s, &d_e));
    double* o_g = nullptr;
    PHX_TRY(phx_stage_out_buf(ctx, "gc.og", gamma, (size_t)n, mem, &o_g));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));

    // tables: Re(E) (FP64 and FP32, pitch pe), occupations, per-mode table
    double* e64 = (double*)phx_ws(ctx, "gc.e64", (size_t)n * pe * 8);
    float* e32 = P == P_FP64 ? nullptr : (float*)phx_ws(ctx, "gc.e32", (size_t)n * pe * 4);
    double* nB = (double*)phx_ws(ctx, "gc.nB", (size_t)n * 8);
    float4* t32 = (float4*)phx_ws(ctx, "gc.t32", (size_t)pe * 16);
    double* t64 = (double*)phx_ws(ctx, "gc.t64", (size_t)pe * 24);
    double* gacc = (double*)phx_ws(ctx, "gc.gacc", (size_t)n * 8);
    if (!e64 || (P != P_FP64 && !e32) || !nB || !t32 || !t64 || !gacc) return PHX_ERR_NOMEM;
    real_tables_kernel<<<4 * ctx->sm_count, 256, 0, s>>>((const double2*)d_e, n, pe, e64, e32,
                                                         (int32_t*)ctx->status_word);
    PHX_CUDA_CHECK(ctx, phx_launch_occupations(d_f, n, temperature, 0, nB, nullptr, s));
    mode_table_kernel<<<(pe + 255) / 256, 256, 0, s>>>(d_f, nB, n, pe, f_min_thz, t32, t64);
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(gacc, 0, (size_t)n * 8, s));
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 3;

    // host plan from the frequencies (the only device -> host transfer before the GEMMs)
    std::vector<double> fh(n);
    int32_t st = 0;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(fh.data(), d_f, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    if (st != 0) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: eigenvectors must be real (Gamma point)");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(fh[i])) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_cell: frequency %d not finite", i);
    const double lim = br.window * br.sigma_thz;
    std::vector<int> work_a, item_start, c_lo;
    std::vector<int4> items;
    plan_tiles(fh, f_min_thz, lim, work_a, items, item_start, c_lo);

    const double conv = phx::kEvA2AmuToPs2;
    const double pref = phx::kPi * phx::kHbarEvPs * conv * conv * conv / 8.0;
    const double two_pi4 = std::pow(phx::kTwoPi, 4);
    double norm, p1;
    if (br.shape == PHX_GAUSS) {
        norm = 1.0 / (std::sqrt(phx::kPi) * br.sigma_thz);
        p1 = -1.0 / (br.sigma_thz * br.sigma_thz);
    } else {
        const double h = 0.5 * br.sigma_thz;
        norm = h / phx::kPi;
        p1 = h * h;
    }
    const double scale = pref * 2.0 * norm / two_pi4;

    if (!work_a.empty()) {
        // operand ET[b][j] (rows padded to pe)
        const int esz = P == P_BF16X3 ? 2 : P == P_TF32 ? 4 : 8;
        void* et_hi = phx_ws(ctx, "gc.et.hi", (size_t)pe * kpad * esz);
        void* et_lo = P == P_BF16X3 ? phx_ws(ctx, "gc.et.lo", (size_t)pe * kpad * esz) : nullptr;
        if (!et_hi || (P == P_BF16X3 && !et_lo)) return PHX_ERR_NOMEM;
        {
            dim3 grid((kpad + 31) / 32, (pe + 31) / 32, 1), block(32, 8);
            if (P == P_BF16X3)
                transpose_kernel<double, P_BF16X3><<<grid, block, 0, s>>>(e64, 0, pe, n, n, et_hi, et_lo, 0, kpad, pe);
            else if (P == P_TF32)
                transpose_kernel<double, P_TF32><<<grid, block, 0, s>>>(e64, 0, pe, n, n, et_hi, nullptr, 0, kpad, pe);
            else
                transpose_kernel<double, P_FP64><<<grid, block, 0, s>>>(e64, 0, pe, n, n, et_hi, nullptr, 0, kpad, pe);
            ctx->launches += 1;
        }
        // FP32 product shape: LA modes per CTA x NC columns per thread (PHX_XFORM = "16x1", "16x2",
        // "8x2" or "8x4" to tune; default 16x1)
        static const int xcfg = [] {
            const char* v = std::getenv("PHX_XFORM");
            if (!v) return 161;
            if (!std::strcmp(v, "16x2")) return 162;
            if (!std::strcmp(v, "8x2")) return 82;
            if (!std::strcmp(v, "8x4")) return 84;
            return 161;
        }();
        // chunks of consecutive work modes, sized to ~6 GB of X + XT
        const int LA = P == P_FP64 ? 8 : xcfg / 10;
        const size_t xbytes = P == P_FP64 ? 8 : 4;
        const size_t per_a = (size_t)n * pe * xbytes + (size_t)pe * kpad * (P == P_FP64 ? 8 : 4);
        int L = (int)std::min<size_t>(128, ((size_t)6 << 30) / per_a);
        L = std::max(LA, L / LA * LA);
        std::vector<int32_t> chunk_a_all(work_a.begin(), work_a.end());
        int32_t* d_chunk_a = (int32_t*)phx_ws(ctx, "gc.ca", chunk_a_all.size() * 4);
        int4* d_items = (int4*)phx_ws(ctx, "gc.items", std::max<size_t>(1, items.size()) * 16);
        if (!d_chunk_a || !d_items) return PHX_ERR_NOMEM;
        // a_local of each item relative to its chunk start
        std::vector<int4> items_loc(items);
        std::vector<Chunk> chunks;
        for (int w0 = 0; w0 < (int)work_a.size(); w0 += L) {
            Chunk ch;
            ch.a_begin = w0;
            ch.a_end = std::min((int)work_a.size(), w0 + L);
            int cb = pe;
            for (int w = ch.a_begin; w < ch.a_end; ++w) cb = std::min(cb, c_lo[w]);
            ch.c_base = cb;
            ch.item_begin = item_start[ch.a_begin];
            ch.item_end = item_start[ch.a_end];
            for (int it = ch.item_begin; it < ch.item_end; ++it) items_loc[it].x -= w0;
            chunks.push_back(ch);
        }
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_chunk_a, chunk_a_all.data(), chunk_a_all.size() * 4,
                                            cudaMemcpyHostToDevice, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_items, items_loc.data(), items_loc.size() * 16, cudaMemcpyHostToDevice, s));
        int ncc_max = 0;
        for (const Chunk& ch : chunks) ncc_max = std::max(ncc_max, pe - ch.c_base);
        const int n_asub_max = (L + LA - 1) / LA;
        const int64_t n_seg = (int64_t)fc3->g0_slots * 9;
        void* Wb = phx_ws(ctx, "gc.W", (size_t)n_asub_max * n_seg * LA * xbytes);
        void* Xb = phx_ws(ctx, "gc.X", (size_t)L * n * ncc_max * xbytes);
        void* xt_hi = phx_ws(ctx, "gc.xt.hi", (size_t)L * ncc_max * kpad * esz);
        void* xt_lo = P == P_BF16X3 ? phx_ws(ctx, "gc.xt.lo", (size_t)L * ncc_max * kpad * esz) : nullptr;
        if (!Wb || !Xb || !xt_hi || (P == P_BF16X3 && !xt_lo)) return PHX_ERR_NOMEM;
        const size_t xs_smem = (size_t)fc3->g0_max_slots * 9 * LA * xbytes;
        if (xs_smem > kSmemDyn)
            return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_gamma_cell: %d neighbour atoms per atom exceed shared memory",
                                 fc3->g0_max_slots);
        static bool attr_done = false;
        if (!attr_done) {
            cudaFuncSetAttribute(xform_kernel<float, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(xform_kernel<float, 16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(xform_kernel<float, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(xform_kernel<float, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(xform_kernel<double, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(sym_tc_kernel<P_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            cudaFuncSetAttribute(sym_tc_kernel<P_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDyn);
            attr_done = true;
        }
        const int planes = P == P_BF16X3 ? 2 : 1;
        const size_t stage_bytes = (size_t)planes * 2 * kTileBytes;
        const int stages = (int)std::min<size_t>(kMaxStages, (kSmemDyn - 1024) / stage_bytes);

        for (const Chunk& ch : chunks) {
            const int Lc = ch.a_end - ch.a_begin;
            const int n_asub = (Lc + LA - 1) / LA;
            const int ncc = pe - ch.c_base;
            // ---- W and X = W E (CUDA cores)
            int ps = phx_prof_begin(ctx, s);
            const int64_t wtot = (int64_t)n_asub * n_seg * LA;
            const unsigned wblocks = (unsigned)std::min<int64_t>((wtot + 255) / 256, 64 * ctx->sm_count);
            const int tj = 4;
            const int xnc = xcfg % 10;
            const int ncol = P == P_FP64 ? 256 : 256 * xnc;     // columns per CTA (NC x 256)
            dim3 xgrid((ncc + ncol - 1) / ncol, (na + tj - 1) / tj, n_asub);
            if (P == P_FP64) {
                w_kernel<double, 8><<<wblocks, 256, 0, s>>>(fc3->g0_seg_start, fc3->g0_ent_i, fc3->g0_ent_w, n_seg, e64,
                                                            pe, d_chunk_a + ch.a_begin, Lc, n_asub, (double*)Wb);
                xform_kernel<double, 8, 1><<<xgrid, 256, xs_smem, s>>>(e64, pe, (const double*)Wb, n_seg, fc3->g0_nbr_start,
                                                                    fc3->g0_nbr_atom, na, n, ch.c_base, ncc, tj, Lc,
                                                                    (double*)Xb);
            } else {
                const int* ns_ = fc3->g0_nbr_start;
                const int* na_ = fc3->g0_nbr_atom;
                if (LA == 16)
                    w_kernel<float, 16><<<wblocks, 256, 0, s>>>(fc3->g0_seg_start, fc3->g0_ent_i, fc3->g0_ent_w, n_seg,
                                                                e64, pe, d_chunk_a + ch.a_begin, Lc, n_asub, (float*)Wb);
                else
                    w_kernel<float, 8><<<wblocks, 256, 0, s>>>(fc3->g0_seg_start, fc3->g0_ent_i, fc3->g0_ent_w, n_seg,
                                                               e64, pe, d_chunk_a + ch.a_begin, Lc, n_asub, (float*)Wb);
                const float* Wf = (const float*)Wb;
                float* Xf = (float*)Xb;
                if (xcfg == 162)
                    xform_kernel<float, 16, 2><<<xgrid, 256, xs_smem, s>>>(e32, pe, Wf, n_seg, ns_, na_, na, n, ch.c_base,
                                                                          ncc, tj, Lc, Xf);
                else if (xcfg == 82)
                    xform_kernel<float, 8, 2><<<xgrid, 256, xs_smem, s>>>(e32, pe, Wf, n_seg, ns_, na_, na, n, ch.c_base,
                                                                         ncc, tj, Lc, Xf);
                else if (xcfg == 84)
                    xform_kernel<float, 8, 4><<<xgrid, 256, xs_smem, s>>>(e32, pe, Wf, n_seg, ns_, na_, na, n, ch.c_base,
                                                                         ncc, tj, Lc, Xf);
                else
                    xform_kernel<float, 16, 1><<<xgrid, 256, xs_smem, s>>>(e32, pe, Wf, n_seg, ns_, na_, na, n, ch.c_base,
                                                                          ncc, tj, Lc, Xf);
            }
            PHX_CUDA_CHECK(ctx, cudaGetLastError());
            // algorithmic work of X = W E: 2 x (3 x slots) x n_cols per mode
            phx_prof_end(ctx, ps, s, PHX_K_CELL_SPARSE, 2.0 * Lc * (double)fc3->g0_slots * 9.0 * ncc,
                         (double)Lc * n * ncc * xbytes);
            // ---- XT_a[c][j]
            ps = phx_prof_begin(ctx, s);
            {
                dim3 grid((kpad + 31) / 32, (ncc + 31) / 32, Lc), block(32, 8);
                const int64_t izs = (int64_t)n * ncc, ozs = (int64_t)ncc * kpad;
                if (P == P_BF16X3)
                    transpose_kernel<float, P_BF16X3><<<grid, block, 0, s>>>((const float*)Xb, izs, ncc, n, ncc, xt_hi,
                                                                            xt_lo, ozs, kpad, ncc);
                else if (P == P_TF32)
                    transpose_kernel<float, P_TF32><<<grid, block, 0, s>>>((const float*)Xb, izs, ncc, n, ncc, xt_hi,
                                                                          nullptr, ozs, kpad, ncc);
                else
                    transpose_kernel<double, P_FP64><<<grid, block, 0, s>>>((const double*)Xb, izs, ncc, n, ncc, xt_hi,
                                                                           nullptr, ozs, kpad, ncc);
            }
            PHX_CUDA_CHECK(ctx, cudaGetLastError());
            phx_prof_end(ctx, ps, s, PHX_K_CELL_TRANSPOSE, 0.0,
                         (double)Lc * ncc * ((double)n * xbytes + (double)kpad * esz * planes));
            // ---- tiles
            const int nit = ch.item_end - ch.item_begin;
            if (nit == 0) continue;
            ps = phx_prof_begin(ctx, s);
            if (P == P_FP64) {
                sym_fp64_kernel<<<nit, 256, 0, s>>>((const double*)et_hi, (const double*)xt_hi, kpad, ncc, ch.c_base,
                                                    d_items + ch.item_begin, d_chunk_a + ch.a_begin, t64, n, lim, p1,
                                                    br.shape, gacc);
            } else {
                SymArgs a{};
                if (!make_map(&a.a_map[0], et_hi, P, pe, kpad) ||
                    (P == P_BF16X3 && !make_map(&a.a_map[1], et_lo, P, pe, kpad)) ||
                    !make_map(&a.b_map[0], xt_hi, P, (int64_t)Lc * ncc, kpad) ||
                    (P == P_BF16X3 && !make_map(&a.b_map[1], xt_lo, P, (int64_t)Lc * ncc, kpad)))
                    return phx_set_error(ctx, PHX_ERR_CUDA, "phx_gamma_cell: tensor map encoding failed");
                if (P != P_BF16X3) { a.a_map[1] = a.a_map[0]; a.b_map[1] = a.b_map[0]; }
                a.items = d_items + ch.item_begin;
                a.n_items = nit;
                a.nk = nk;
                a.stages = stages;
                a.ncc = ncc;
                a.c_base = ch.c_base;
                a.tmem_cols = 2 * kTile;
                a.status = (int32_t*)ctx->status_word;
                a.chunk_a = d_chunk_a + ch.a_begin;
                a.tab = t32;
                a.n = n;
                a.lim = (float)lim;
                a.p1 = (float)p1;
                a.shape = br.shape;
                a.gacc = gacc;
                const unsigned grid = (unsigned)std::min(nit, ctx->sm_count);
                const size_t smem = 1024 + (size_t)stages * stage_bytes;
                if (P == P_BF16X3) sym_tc_kernel<P_BF16X3><<<grid, kThreads, smem, s>>>(a);
                else sym_tc_kernel<P_TF32><<<grid, kThreads, smem, s>>>(a);
            }
            PHX_CUDA_CHECK(ctx, cudaGetLastError());
            phx_prof_end(ctx, ps, s, PHX_K_CELL_GEMM, 2.0 * kTile * kTile * (double)n * nit,
                         (double)nit * 2.0 * kTile * kpad * esz * planes);
            ctx->launches += 4;
        }
    }
    finalize_cell_kernel<<<(n + 255) / 256, 256, 0, s>>>(d_f, gacc, n, scale, f_min_thz, o_g);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 1;
    if (mem == PHX_MEM_HOST) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma, o_g, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_gamma_cell: kernel reported status %d", st);
    }
    return PHX_OK;
}

// ---------------------------------------------------------------- handle preparation

// Symmetrise F over the permutations of (i, j, k) (mean over each orbit; images summed) and
// group the entries by (J, slot of K, gamma, beta).  Host work: two sorts of the nnz entries.
phx_status phx_fc3_prepare_cell(phx_ctx* ctx, const phx_cell* cell, const phx_ifc3* fc3, phx_fc3* h) {
    const int n = h->n, na = n / 3;
    const int64_t nnz = fc3->nnz;
    struct KV { int64_t key; double w; };
    std::vector<KV> kv;
    kv.reserve((size_t)nnz);
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t* e = fc3->idx + 9 * k;
        int x = e[0], y = e[1], z = e[2];
        const double w = fc3->val[k] / std::sqrt(cell->masses[x / 3] * cell->masses[y / 3] * cell->masses[z / 3]);
        if (x > y) std::swap(x, y);
        if (y > z) std::swap(y, z);
        if (x > y) std::swap(x, y);
        kv.push_back({((int64_t)x * n + y) * n + z, w});
    }
    std::sort(kv.begin(), kv.end(), [](const KV& a, const KV& b) { return a.key < b.key; });
    struct Ent { int32_t i, j, k; double w; };
    std::vector<Ent> ents;
    ents.reserve((size_t)nnz + 16);
    for (size_t p = 0; p < kv.size();) {
        size_t q = p;
        double sum = 0.0;
        while (q < kv.size() && kv[q].key == kv[p].key) sum += kv[q++].w;
        const int64_t key = kv[p].key;
        const int x = (int)(key / ((int64_t)n * n)), y = (int)((key / n) % n), z = (int)(key % n);
        p = q;
        if (sum == 0.0) continue;
        int perm[6][3] = {{x, y, z}, {x, z, y}, {y, x, z}, {y, z, x}, {z, x, y}, {z, y, x}};
        int n_orb = 0;
        int orb[6][3];
        for (auto& t : perm) {
            bool seen = false;
            for (int o = 0; o < n_orb; ++o) seen = seen || (orb[o][0] == t[0] && orb[o][1] == t[1] && orb[o][2] == t[2]);
            if (!seen) { orb[n_orb][0] = t[0]; orb[n_orb][1] = t[1]; orb[n_orb][2] = t[2]; ++n_orb; }
        }
        for (int o = 0; o < n_orb; ++o) ents.push_back({orb[o][0], orb[o][1], orb[o][2], sum / n_orb});
    }
    // neighbour slots: atoms K paired with row atom J
    std::vector<int64_t> pairs;
    pairs.reserve(ents.size());
    for (const Ent& e : ents) pairs.push_back((int64_t)(e.j / 3) * na + e.k / 3);
    std::sort(pairs.begin(), pairs.end());
    pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
    std::vector<int32_t> nbr_start(na + 1, 0), nbr_atom(pairs.size());
    for (size_t s = 0; s < pairs.size(); ++s) {
        nbr_start[pairs[s] / na + 1] += 1;
        nbr_atom[s] = (int32_t)(pairs[s] % na);
    }
    int max_slots = 0;
    for (int J = 0; J < na; ++J) {
        max_slots = std::max(max_slots, nbr_start[J + 1]);
        nbr_start[J + 1] += nbr_start[J];
    }
    const int64_t n_seg = (int64_t)pairs.size() * 9;
    std::vector<int64_t> seg_start(n_seg + 1, 0);
    std::vector<int32_t> seg_of(ents.size());
    for (size_t t = 0; t < ents.size(); ++t) {
        const Ent& e = ents[t];
        const int J = e.j / 3, K = e.k / 3;
        const int32_t* lo = nbr_atom.data() + nbr_start[J];
        const int32_t* hi = nbr_atom.data() + nbr_start[J + 1];
        const int slot = (int)(std::lower_bound(lo, hi, K) - nbr_atom.data());
        seg_of[t] = slot * 9 + (e.k % 3) * 3 + (e.j % 3);
        seg_start[seg_of[t] + 1] += 1;
    }
    for (int64_t g = 0; g < n_seg; ++g) seg_start[g + 1] += seg_start[g];
    std::vector<int64_t> fill(seg_start.begin(), seg_start.end() - 1);
    std::vector<int32_t> ent_i(ents.size());
    std::vector<double> ent_w(ents.size());
    for (size_t t = 0; t < ents.size(); ++t) {
        const int64_t pos = fill[seg_of[t]]++;
        ent_i[pos] = ents[t].i;
        ent_w[pos] = ents[t].w;
    }
    auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
        if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        return bytes == 0 || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    const bool ok = up((void**)&h->g0_nbr_start, nbr_start.data(), nbr_start.size() * 4) &&
                    up((void**)&h->g0_nbr_atom, nbr_atom.data(), nbr_atom.size() * 4) &&
                    up((void**)&h->g0_seg_start, seg_start.data(), seg_start.size() * 8) &&
                    up((void**)&h->g0_ent_i, ent_i.data(), ent_i.size() * 4) &&
                    up((void**)&h->g0_ent_w, ent_w.data(), ent_w.size() * 8);
    if (!ok) {
        cudaGetLastError();
        return phx_set_error(ctx, PHX_ERR_NOMEM, "phx_fc3_create: device upload of the Gamma-only tables failed");
    }
    h->g0_slots = (int)pairs.size();
    h->g0_max_slots = max_slots;
    h->g0_nnz = (int64_t)ents.size();
    h->g0_ready = true;
    return PHX_OK;
}
