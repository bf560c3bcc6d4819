// Three-phonon linewidths on the tcgen05 tensor cores (paper Sec. "Three-Phonon Scattering",
// Eqs. (phi3_proj), (gamma), (broadening); Sec. "Computational Implementation": the
// projection done as tensor products).  Same regrouping as the FP64 path:
//
//   S3  W_q[(nu,b,c)][d]        = sum phi/sqrt(mmm) exp(+i q.R'') e_q[a][nu]      (fold kernel)
//   S4  M_q'[(nu,b)][c]         = sum_d W[(nu,b,c)][d] exp(-i q'.d)               (GEMM, K = d)
//   S5  X_q'[(nu,nu'')][b]      = sum_c M[(nu,b)][c] e_q''[c][nu'']               (GEMM, K = c)
//       V_q'[(nu,nu'')][nu']    = sum_b X[(nu,nu'')][b] e_q'[b][nu']              (GEMM, K = b)
//   S6  gamma[nu] += sum |V|^2 w(f, f', f'')   fused into the epilogue of the last GEMM
//
// Every complex product is one real GEMM on the "real embedding": an operand row holds
// [Re(0..Kc) | Im(0..Kc)] (each half zero-padded to Kcp = 32-multiple), and the B table of
// a complex matrix E (K x modes) has rows [Re outputs (np rows) | Im outputs (np rows)]:
//     B[j][k] = Re E(k,j), B[j][Kcp+k] = -Im E(k,j), B[np+j][k] = Im E(k,j), B[np+j][Kcp+k] = Re E(k,j)
// so D = A B^T holds [Re | Im] of the complex product.  Precisions: BF16x3 (x = hi + lo in
// bf16, product hi*hi + hi*lo + lo*hi, FP32 accumulate in tensor memory) or TF32 (one pass).
//
// GEMM kernel: warp 0 issues TMA loads of 128-row x 128-byte A chunks (128B swizzle) into a
// ring of stages; warp 1 owns tensor memory and issues tcgen05.mma (M = 128, N = the padded
// output width of a column group) into one of two accumulators; the epilogue warps (24 / 16
// for the operand-writing GEMMs, 8 for the weighting GEMM) read the accumulator back with
// tcgen05.ld while the next tile accumulates.  The B operand of a problem stays resident in
// shared memory when it fits, else it is streamed with A.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <mutex>

#include "common.h"
#include "gamma_common.cuh"
#include "tc_ptx.cuh"

namespace {

// Epilogue warps (a multiple of 4: the TMEM lane group of a warp is its index mod 4), as
// measured best per mode: the Fourier GEMM's operand stores 24, the e_q'' GEMM 16, the
// register-heavy weighting epilogues EPI_G / EPI_GT 8.
template <int EPI> constexpr int epi_warps() { return EPI == 0 ? 24 : EPI == 1 ? 16 : 8; }
template <int EPI> constexpr int kernel_threads() { return 64 + 32 * epi_warps<EPI>(); }
constexpr int kMaxStages = 8;
constexpr int kBoxRows = 128;                  // rows of an A tile (= MMA M)
constexpr int kChunkBytes = 128;               // bytes of K per chunk (one swizzle row)
constexpr int kStageBytesPerPlane = kBoxRows * kChunkBytes;
constexpr int kMaxNp = 192;                    // padded modes (or q' slots) per output half
constexpr size_t kSmemLimit = 232448;          // 227 KB opt-in

// EPI_GT: EPI_G for up to kMaxT temperatures; EPI_GS: EPI_G plus the off-diagonal scattering
// rows of Eq. (gamma1)
// EPI_GL: EPI_GS's rows applied to mean free paths instead of stored (matrix-free iteration)
enum { EPI_M = 0, EPI_X = 1, EPI_G = 2, EPI_GT = 3, EPI_GS = 4, EPI_GL = 5 };
constexpr int kMaxT = 4;
enum { P_BF16X3 = 0, P_TF32 = 1 };

struct TcArgs {
    CUtensorMap a_map[2];       // A operand planes (hi, lo) or (fp32)
    CUtensorMap b_map[2];       // B operand planes
    int rows;                   // valid rows per problem
    int tiles;                  // ceil(rows / 128)
    int n_problems;             // problems (one B operand each); work items = n_problems * tiles
    int np;                     // B table half height: rows [Re outputs (np) | Im outputs (np)] per index
    int mg;                     // output modes per column group (multiple of 8); accumulator = 2 mg columns
    int n_groups;               // column groups (mg * n_groups = np)
    int nk;                     // K chunks (128 bytes each)
    int stages;
    int n_acc;                  // 1 or 2 accumulators in tensor memory
    int a_rows_per_problem;     // A row offset between problems
    const int32_t* b_idx;       // per problem: B table index (row offset b_idx[p] * 2 np)
    int b_base;                 // used when b_idx == nullptr
    uint32_t tmem_cols;
    int32_t* status;
    // ---- epilogue parameters
    void* out_hi;               // EPI_M / EPI_X: destination operand planes
    void* out_lo;
    int out_rows_per_slot;      // rows of the destination per problem / q' slot
    int out_kr;                 // destination row length (elements)
    int out_kcp;                // destination imaginary-half offset
    int n;                      // modes
    int nq_slots;               // EPI_M: valid q' slots in this tile
    // EPI_G
    const double* freq;
    const double* nB;
    int iq, nu0, m1, m2, m3;
    const int32_t* qp1;         // per problem: mesh index of q'
    int pair;                   // nonzero: each q' stands for its exchange pair (q', q'')
    float sigma, window, f_min;
    int shape;
    double* gacc;               // [n] for this irreducible q (offset applied)
    double* wacc;               // may be null
    // EPI_GT: n_t temperatures; nB holds n_t tables of nq * n, gacc n_t rows t_stride apart
    int n_t;
    int64_t nb_stride;
    int64_t t_stride;
    // EPI_GS: off-diagonal rows folded onto time-reversal representatives (see G1Target)
    float* g1;
    int64_t g1_rows;
    int64_t g1_ld;
    int64_t g1_row0;            // row of (this q, band nu0)
    const int32_t* tr_code;
    double g1_scale;
    // EPI_GL: y[a][r] += sum_c Gamma1[r][c] lam[a][c] (planes [3][g1_ld], FP64)
    const double* lam;
    double* ylam;
    unsigned long long wait_ns; // bound of every barrier wait
    int starve;                 // test hook: the producer issues nothing (waits then run out)
};

template <int PREC>
__device__ __forceinline__ void store_operand(void* hi, void* lo, int64_t idx, float v) {
    if (PREC == P_BF16X3) {
        __nv_bfloat16 h, l;
        tc::split_bf16(v, &h, &l);
        ((__nv_bfloat16*)hi)[idx] = h;
        ((__nv_bfloat16*)lo)[idx] = l;
    } else {
        ((float*)hi)[idx] = tc::round_tf32(v);
    }
}

// Two adjacent elements (idx even): one 4-byte (bf16 planes) or 8-byte (tf32) store per plane.
template <int PREC>
__device__ __forceinline__ void store_operand2(void* hi, void* lo, int64_t idx, float a0, float a1) {
    if (PREC == P_BF16X3) {
        __nv_bfloat16 h0, l0, h1, l1;
        tc::split_bf16(a0, &h0, &l0);
        tc::split_bf16(a1, &h1, &l1);
        __nv_bfloat162 H, L;
        H.x = h0; H.y = h1;
        L.x = l0; L.y = l1;
        *reinterpret_cast<__nv_bfloat162*>((__nv_bfloat16*)hi + idx) = H;
        *reinterpret_cast<__nv_bfloat162*>((__nv_bfloat16*)lo + idx) = L;
    } else {
        *reinterpret_cast<float2*>((float*)hi + idx) = make_float2(tc::round_tf32(a0), tc::round_tf32(a1));
    }
}

__device__ __forceinline__ void epi_barrier(int threads) { asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory"); }

// Epilogue barrier that also returns whether any participating thread passed pred = true, so
// that every epilogue thread takes the same decision (a shared flag read after a plain barrier
// can change between two threads' reads when another role sets it).
__device__ __forceinline__ bool epi_barrier_any(int threads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(threads)
        : "memory");
    return r != 0;
}

template <int PREC, int EPI, bool kStreamB>
__global__ void __launch_bounds__(kernel_threads<EPI>(), 1) tc_gemm_kernel(const __grid_constant__ TcArgs args) {
    constexpr int kEpiThreads = 32 * epi_warps<EPI>();
    constexpr int kEpiParts = epi_warps<EPI>() / 4;          // warps per TMEM lane group
    constexpr int kPlanes = (PREC == P_BF16X3) ? 2 : 1;
    constexpr uint32_t kFmt = (PREC == P_BF16X3) ? 1u : 2u;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t bfull_bar, bempty_bar, tfull_bar[2], tempty_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_slot;
    __shared__ volatile int abort_flag;
    __shared__ float s_f1[kMaxNp], s_n1[kMaxNp], s_if1[kMaxNp];
    __shared__ float s_n1t[EPI == EPI_GT ? kMaxT * kMaxNp : 1];
    __shared__ float s_rows[EPI == EPI_GS ? 2 : 1][4][32];   // EPI_GS: part-1 row sums per lane group
    __shared__ float s_lam[EPI == EPI_GL ? 3 : 1][EPI == EPI_GL ? kMaxNp : 1];   // EPI_GL: signed f' lambda'

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int np = args.np, mg = args.mg, NA = 2 * mg, nk = args.nk, stages = args.stages;
    // Resident B: [plane][kc][NA rows][128 B] once per problem.  Streamed B: every stage holds
    // the A chunk planes followed by the B chunk planes (NA rows each).
    const uint32_t b_bytes_plane = kStreamB ? 0u : (uint32_t)nk * NA * kChunkBytes;
    const uint32_t stage_b_plane = kStreamB ? (uint32_t)NA * kChunkBytes : 0u;
    const uint32_t stage_bytes = kPlanes * (kStageBytesPerPlane + stage_b_plane);
    uint8_t* b_smem = smem;
    uint8_t* a_smem = smem + kPlanes * b_bytes_plane;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Persistent CTAs over a flat list of (problem, tile) items, problem-major; each CTA takes
    // one contiguous, balanced range so it switches problem (and reloads B) rarely.
    const int per_p = args.tiles * args.n_groups;                  // items per problem (group innermost)
    const int64_t n_items = (int64_t)args.n_problems * per_p;
    const int item_begin = (int)(n_items * blockIdx.x / gridDim.x);
    const int item_end = (int)(n_items * (blockIdx.x + 1) / gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) { tc::mbar_init(&full_bar[s], 1); tc::mbar_init(&empty_bar[s], 1); }
        tc::mbar_init(&bfull_bar, 1);
        tc::mbar_init(&bempty_bar, 1);
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&tfull_bar[a], 1); tc::mbar_init(&tempty_bar[a], kEpiThreads); }
        tc::mbar_init(&drain_bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        for (int pl = 0; pl < kPlanes; ++pl) { tc::prefetch_tmap(&args.a_map[pl]); tc::prefetch_tmap(&args.b_map[pl]); }
    }
    if (warp == 1) tc::tmem_alloc(&tmem_base_slot, args.tmem_cols);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = tmem_base_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0 && !args.starve) {
            int stage = 0;
            uint32_t phase = 0;
            bool pending[kMaxStages];
            uint32_t pend_phase[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) { pending[s] = false; pend_phase[s] = 0; }
            const int kelems = kChunkBytes / (PREC == P_BF16X3 ? 2 : 4);
            int cur_p = -1, n_loaded = 0;
            for (int it = item_begin; it < item_end && !abort_flag; ++it) {
                const int p = it / per_p, tile = (it % per_p) / args.n_groups, g = it % args.n_groups;
                const int brow = (args.b_idx ? args.b_idx[p] : args.b_base) * (2 * np) + g * mg;
                if (!kStreamB && p != cur_p) {
                    // a new problem: wait until the MMAs using the previous B have completed
                    if (n_loaded > 0 && !tc::mbar_wait(&bempty_bar, (n_loaded - 1) & 1, &abort_flag, args.wait_ns)) {
                        abort_flag = 1;
                        atomicExch(args.status, (int)PHX_ERR_TIMEOUT);
                        break;
                    }
                    tc::mbar_expect_tx(&bfull_bar, kPlanes * b_bytes_plane);
                    for (int pl = 0; pl < kPlanes; ++pl)
                        for (int kc = 0; kc < nk; ++kc)
                            for (int half = 0; half < 2; ++half)
                                tc::tma_load_2d(b_smem + pl * b_bytes_plane + ((size_t)kc * NA + half * mg) * kChunkBytes,
                                                &args.b_map[pl], &bfull_bar, kc * kelems, brow + half * np);
                    ++n_loaded;
                    cur_p = p;
                }
                const int arow = p * args.a_rows_per_problem + tile * kBoxRows;
                for (int kc = 0; kc < nk; ++kc) {
                    if (!tc::mbar_wait(&empty_bar[stage], phase ^ 1, &abort_flag, args.wait_ns)) {
                        abort_flag = 1;
                        atomicExch(args.status, (int)PHX_ERR_TIMEOUT);
                        break;
                    }
                    pending[stage] = false;
                    uint8_t* st_base = a_smem + (size_t)stage * stage_bytes;
                    tc::mbar_expect_tx(&full_bar[stage], stage_bytes);
                    for (int pl = 0; pl < kPlanes; ++pl)
                        tc::tma_load_2d(st_base + (size_t)pl * kStageBytesPerPlane, &args.a_map[pl], &full_bar[stage],
                                        kc * kelems, arow);
                    if (kStreamB) {
                        uint8_t* sb = st_base + (size_t)kPlanes * kStageBytesPerPlane;
                        for (int pl = 0; pl < kPlanes; ++pl)
                            for (int half = 0; half < 2; ++half)
                                tc::tma_load_2d(sb + (size_t)pl * stage_b_plane + (size_t)half * mg * kChunkBytes,
                                                &args.b_map[pl], &full_bar[stage], kc * kelems, brow + half * np);
                    }
                    pending[stage] = true;
                    pend_phase[stage] = phase;
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
            }
            if (abort_flag) {
                // let loads already issued land before the CTA retires (bounded)
                for (int s = 0; s < stages; ++s)
                    if (pending[s]) {
                        const uint64_t t0 = tc::global_ns();
                        while (!tc::mbar_try_wait(&full_bar[s], pend_phase[s]) &&
                               tc::global_ns() - t0 < args.wait_ns) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_full = tc::idesc(128, NA, kFmt);
            bool ok = true;
            int stage = 0, acc = 0;
            uint32_t phase = 0, acc_phase = 0;
            const uint32_t b_base = tc::smem_u32(b_smem);
            const uint32_t a_base = tc::smem_u32(a_smem);
            int cur_p = -1, n_bloads = 0;
            for (int it = item_begin; ok && it < item_end; ++it) {
                const int p = it / per_p;
                if (!kStreamB && p != cur_p) {
                    if (cur_p >= 0) tc::mma_commit(&bempty_bar);       // B free once these MMAs finish
                    if (!tc::mbar_wait(&bfull_bar, n_bloads & 1, &abort_flag, args.wait_ns)) {
                        abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); break;
                    }
                    tc::tc_fence_after();
                    ++n_bloads;
                    cur_p = p;
                }
                if (!tc::mbar_wait(&tempty_bar[acc], acc_phase ^ 1, &abort_flag, args.wait_ns)) {
                    abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); break;
                }
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * NA);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!tc::mbar_wait(&full_bar[stage], phase, &abort_flag, args.wait_ns)) {
                        abort_flag = 1; atomicExch(args.status, (int)PHX_ERR_TIMEOUT); ok = false; break;
                    }
                    tc::tc_fence_after();
                    const uint32_t st_a = a_base + (uint32_t)stage * stage_bytes;
                    const uint32_t st_b = kStreamB ? st_a + kPlanes * kStageBytesPerPlane
                                                   : b_base + (uint32_t)kc * NA * kChunkBytes;
                    const uint32_t b_lo = kStreamB ? stage_b_plane : b_bytes_plane;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {                      // 4 x 32 bytes per chunk
                        const uint32_t koff = (uint32_t)k * 32;
                        const uint32_t acc_flag = (kc | k) ? 1u : 0u;
                        if (PREC == P_BF16X3) {
                            const uint64_t ah = tc::sdesc_sw128(st_a + koff);
                            const uint64_t al = tc::sdesc_sw128(st_a + kStageBytesPerPlane + koff);
                            const uint64_t bh = tc::sdesc_sw128(st_b + koff);
                            const uint64_t bl = tc::sdesc_sw128(st_b + b_lo + koff);
                            tc::mma_f16(d_tmem, ah, bh, id_full, acc_flag);
                            tc::mma_f16(d_tmem, ah, bl, id_full, 1u);
                            tc::mma_f16(d_tmem, al, bh, id_full, 1u);
                        } else {
                            tc::mma_tf32(d_tmem, tc::sdesc_sw128(st_a + koff), tc::sdesc_sw128(st_b + koff), id_full,
                                         acc_flag);
                        }
                    }
                    tc::mma_commit(&empty_bar[stage]);
                    if (++stage == stages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                tc::mma_commit(&tfull_bar[acc]);
                if (args.n_acc == 2) { acc ^= 1; if (acc == 0) acc_phase ^= 1; } else { acc_phase ^= 1; }
            }
            // every MMA of this thread has completed once drain_bar flips
            tc::mma_commit(&drain_bar);
            const uint64_t t0 = tc::global_ns();
            while (!tc::mbar_try_wait(&drain_bar, 0) && tc::global_ns() - t0 < args.wait_ns) {
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        // kEpiParts warps per tensor-memory lane group; warp part h handles the 16-column
        // chunks with (chunk index % kEpiParts) == h.
        const int et = threadIdx.x - 64;                  // 0..255
        const int lgrp = warp & 3;                        // tensor-memory lane group of this warp
        const int half = (warp - 2) >> 2;                 // part index (0 .. kEpiParts - 1)
        constexpr int kStride = 16 * kEpiParts;
        int q1 = 0, q2 = 0, cur_p = -1;
        // element weight cA (1+n'+n'') g(f-f'-f'') + cB (n'-n'') (g(f+f'-f'') - [pk] g(f+f''-f')):
        // (1, 2, no) for one ordered q' term; with exchange pairs (2, 2, yes) for q' != q'' (both
        // orderings) and (1, 1, yes) for q' = q'' (its (nu', nu'') sum already holds both)
        float cA = 1.f, cB = 2.f;
        bool pk = false;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int it = item_begin; it < item_end; ++it) {
            const int p = it / per_p, tile = (it % per_p) / args.n_groups, g = it % args.n_groups;
            const int m0 = g * mg;                        // first output mode of this column group
            const bool ok = tc::mbar_wait(&tfull_bar[acc], acc_phase, &abort_flag, args.wait_ns);
            if (!ok) {
                abort_flag = 1;
                atomicExch(args.status, (int)PHX_ERR_TIMEOUT);
            }
            if (epi_barrier_any(kEpiThreads, !ok || abort_flag != 0)) break;   // one decision for all
            if ((EPI == EPI_G || EPI == EPI_GT || EPI == EPI_GS || EPI == EPI_GL) && p != cur_p) {
                // partner tables of this problem's q' (the previous tile is done: barrier above)
                q1 = args.qp1[p];
                q2 = phx_third_index(args.iq, q1, args.m1, args.m2, args.m3);
                pk = args.pair != 0;
                cA = pk && q1 != q2 ? 2.f : 1.f;
                cB = pk && q1 == q2 ? 1.f : 2.f;
                for (int j = et; j < np; j += kEpiThreads) {
                    const bool v = j < args.n;
                    const float f1 = v ? (float)args.freq[(int64_t)q1 * args.n + j] : 0.0f;
                    s_f1[j] = f1;
                    s_n1[j] = v ? (float)args.nB[(int64_t)q1 * args.n + j] : 0.0f;
                    s_if1[j] = (v && f1 >= args.f_min) ? 1.0f / f1 : 0.0f;   // 0 masks padding and soft partners
                    if (EPI == EPI_GT)
                        for (int t = 0; t < kMaxT; ++t)
                            s_n1t[t * kMaxNp + j] =
                                (v && t < args.n_t) ? (float)args.nB[t * args.nb_stride + (int64_t)q1 * args.n + j] : 0.0f;
                    if (EPI == EPI_GL) {
                        // column (q', nu'): f' lambda signed by the time-reversal code of q'
                        const int cq = args.tr_code[q1];
                        const int64_t col = (int64_t)(abs(cq) - 1) * args.n + j;
                        const bool use = v && cq != 0 && col < args.g1_ld;
                        const double fs = cq > 0 ? (double)f1 : -(double)f1;
                        for (int a = 0; a < 3; ++a) s_lam[a][j] = use ? (float)(fs * args.lam[a * args.g1_ld + col]) : 0.0f;
                    }
                }
                epi_barrier(kEpiThreads);
                cur_p = p;
            }
            tc::tc_fence_after();
            const int row = tile * kBoxRows + lgrp * 32 + lane;
            const bool valid = row < args.rows;
            const uint32_t taddr = tmem_base + ((uint32_t)(lgrp * 32) << 16) + (uint32_t)(acc * NA);
            float v[16];
            if (EPI == EPI_M && (args.n & 1) == 0 && (mg & 15) == 0) {
                // row (nu, b, c) of W -> M_slot[(nu, b)][c] (re) and [(nu, b)][Kcp + c] (im).  With n
                // even, lanes (2l, 2l+1) hold rows c, c+1 of the same (nu, b): the pair exchanges one
                // value per two columns and stores two adjacent elements at once.  With mg a
                // multiple of 16 a 16-column chunk lies wholly in the Re or the Im half, so the
                // destination advances by a fixed stride per column pair.
                const int nb = row / args.n, ce = (row % args.n) & ~1;
                const bool odd = lane & 1;
                // 32-bit offsets (a tile of M is far below 2^31 elements per plane); a pair is one
                // 32-bit word of each bf16 plane, split in one packed conversion
                const uint32_t slot_stride = (uint32_t)args.out_rows_per_slot * (uint32_t)args.out_kr;
                const uint32_t row_off = (uint32_t)nb * (uint32_t)args.out_kr + (uint32_t)ce;
                for (int j0 = half * 16; j0 < NA; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    const bool re = j0 < mg;
                    const int s0 = m0 + (re ? j0 : j0 - mg) + (odd ? 1 : 0);   // slot of this lane's first pair
                    const int n_ok = valid ? args.nq_slots - s0 : 0;            // pairs with slot < nq_slots
                    uint32_t idx = (uint32_t)s0 * slot_stride + row_off + (re ? 0u : (uint32_t)args.out_kcp);
                    if (PREC == P_BF16X3) {
                        uint32_t* hw = reinterpret_cast<uint32_t*>(args.out_hi);
                        uint32_t* lw = reinterpret_cast<uint32_t*>(args.out_lo);
                        uint32_t w = idx >> 1;                                   // idx is even
                        // warp-uniform choice: both branches shuffle with the full mask
                        if (__all_sync(0xffffffffu, n_ok >= 16)) {
#pragma unroll
                            for (int i = 0; i < 16; i += 2) {
                                const float recv = __shfl_xor_sync(0xffffffffu, odd ? v[i] : v[i + 1], 1);
                                uint32_t h, l;
                                tc::split_bf16x2(odd ? recv : v[i], odd ? v[i + 1] : recv, &h, &l);
                                hw[w] = h;
                                lw[w] = l;
                                w += slot_stride;                                // two slots = slot_stride words
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; i += 2) {
                                const float recv = __shfl_xor_sync(0xffffffffu, odd ? v[i] : v[i + 1], 1);
                                uint32_t h, l;
                                tc::split_bf16x2(odd ? recv : v[i], odd ? v[i + 1] : recv, &h, &l);
                                if (i < n_ok) { hw[w] = h; lw[w] = l; }
                                w += slot_stride;
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const float recv = __shfl_xor_sync(0xffffffffu, odd ? v[i] : v[i + 1], 1);
                            const float a0 = odd ? recv : v[i], a1 = odd ? v[i + 1] : recv;
                            if (i < n_ok) store_operand2<PREC>(args.out_hi, args.out_lo, idx, a0, a1);
                            idx += 2 * slot_stride;
                        }
                    }
                }
            } else if (EPI == EPI_M && (args.n & 1) == 0) {
                // as above for any mg (a chunk may straddle the Re/Im halves)
                const int nb = row / args.n, ce = (row % args.n) & ~1;
                const bool odd = lane & 1;
                for (int j0 = half * 16; j0 < NA; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float recv = __shfl_xor_sync(0xffffffffu, odd ? v[i] : v[i + 1], 1);
                        const int j = j0 + i + (odd ? 1 : 0);
                        const float a0 = odd ? recv : v[i], a1 = odd ? v[i + 1] : recv;
                        const int slot = m0 + (j < mg ? j : j - mg);
                        if (!valid || slot >= args.nq_slots) continue;
                        const int64_t idx = ((int64_t)slot * args.out_rows_per_slot + nb) * args.out_kr +
                                            (j < mg ? 0 : args.out_kcp) + ce;
                        store_operand2<PREC>(args.out_hi, args.out_lo, idx, a0, a1);
                    }
                }
            } else if (EPI == EPI_M) {
                // row (nu, b, c) of W -> M_slot[(nu, b)][c] (re) and [(nu, b)][Kcp + c] (im)
                const int nb = row / args.n, c = row % args.n;
                for (int j0 = half * 16; j0 < NA; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    if (valid) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int j = j0 + i;
                            const int slot = m0 + (j < mg ? j : j - mg);
                            if (slot >= args.nq_slots) continue;
                            const int64_t idx = ((int64_t)slot * args.out_rows_per_slot + nb) * args.out_kr +
                                                (j < mg ? 0 : args.out_kcp) + c;
                            store_operand<PREC>(args.out_hi, args.out_lo, idx, v[i]);
                        }
                    }
                }
            } else if (EPI == EPI_X && (args.n & 1) == 0 && (mg & 15) == 0) {
                // row (nu, b) -> X[(nu, nu'')][b] (re) and [(nu, nu'')][Kcp + b] (im); paired stores
                // of rows b, b+1 as in EPI_M
                // (mg is a multiple of 16 on this path: a chunk lies in one half, fixed stride)
                const int nu = row / args.n, be = (row % args.n) & ~1;
                const bool odd = lane & 1;
                const int64_t base = (int64_t)p * args.out_rows_per_slot + (int64_t)nu * args.n;
                for (int j0 = half * 16; j0 < NA; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    const bool re = j0 < mg;
                    const int mode0 = m0 + (re ? j0 : j0 - mg) + (odd ? 1 : 0);
                    const int n_ok = valid ? args.n - mode0 : 0;
                    int64_t idx = (base + mode0) * args.out_kr + (re ? 0 : args.out_kcp) + be;
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float recv = __shfl_xor_sync(0xffffffffu, odd ? v[i] : v[i + 1], 1);
                        const float a0 = odd ? recv : v[i], a1 = odd ? v[i + 1] : recv;
                        if (i < n_ok) store_operand2<PREC>(args.out_hi, args.out_lo, idx, a0, a1);
                        idx += 2 * args.out_kr;
                    }
                }
            } else if (EPI == EPI_X) {
                // row (nu, b) -> X[(nu, nu'')][b] (re) and [(nu, nu'')][Kcp + b] (im)
                const int nu = row / args.n, b = row % args.n;
                const int64_t base = (int64_t)p * args.out_rows_per_slot + (int64_t)nu * args.n;
                for (int j0 = half * 16; j0 < NA; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    if (valid) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int j = j0 + i;
                            const int mode = m0 + (j < mg ? j : j - mg);
                            if (mode >= args.n) continue;
                            const int64_t idx = (base + mode) * args.out_kr + (j < mg ? 0 : args.out_kcp) + b;
                            store_operand<PREC>(args.out_hi, args.out_lo, idx, v[i]);
                        }
                    }
                }
            } else if (EPI == EPI_GT) {
                // EPI_G for n_t temperatures: the deltas and |V|^2 are shared, only the
                // occupations change (Sec. "Performance Optimization": multi-temperature split)
                const int nu = row / args.n, n2i = row % args.n;
                float f0 = 0.f, f2 = 0.f, nn2[kMaxT];
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) nn2[t] = 0.f;
                if (valid) {
                    f0 = (float)args.freq[(int64_t)args.iq * args.n + args.nu0 + nu];
                    f2 = (float)args.freq[(int64_t)q2 * args.n + n2i];
#pragma unroll
                    for (int t = 0; t < kMaxT; ++t)
                        if (t < args.n_t) nn2[t] = (float)args.nB[t * args.nb_stride + (int64_t)q2 * args.n + n2i];
                }
                const bool live = valid && f0 >= args.f_min && f2 >= args.f_min;
                const float inv_f02 = live ? 1.0f / (1558.5454565440389f * f0 * f2) : 0.0f;
                const float d02 = f0 - f2, s02 = f0 + f2, lim = args.window * args.sigma;
                const bool gauss = args.shape == PHX_GAUSS;
                const float a = -1.f / (args.sigma * args.sigma), h2 = 0.25f * args.sigma * args.sigma;
                const float norm = gauss ? 0.56418958354775628f / args.sigma : 0.5f * args.sigma / 3.14159265358979f;
                float gs[kMaxT];
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) gs[t] = 0.f;
                float vi[16];
                for (int j0 = half * 16; j0 < mg; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    tc::tmem_ld16(taddr + mg + j0, vi);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int j = m0 + j0 + i;
                        const float if1 = s_if1[j], f1 = s_f1[j];
                        const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                        const float gd = fabsf(x) < lim ? (gauss ? __expf(a * x * x) : __frcp_rn(x * x + h2)) : 0.f;
                        const float ga = fabsf(y) < lim ? (gauss ? __expf(a * y * y) : __frcp_rn(y * y + h2)) : 0.f;
                        const float gb = pk && fabsf(z) < lim ? (gauss ? __expf(a * z * z) : __frcp_rn(z * z + h2)) : 0.f;
                        const float v2 = fmaf(v[i], v[i], vi[i] * vi[i]) * if1;
                        const float gad = cB * (ga - gb), gdd = cA * gd;
#pragma unroll
                        for (int t = 0; t < kMaxT; ++t) {
                            const float n1 = s_n1t[t * kMaxNp + j];
                            gs[t] = fmaf(v2, (1.f + nn2[t] + n1) * gdd + (n1 - nn2[t]) * gad, gs[t]);
                        }
                    }
                }
                const int key = valid ? nu : -1 - lane;
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) {
                    if (t >= args.n_t) break;
                    double dg = (double)(gs[t] * norm * inv_f02);
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const double og = __shfl_down_sync(0xffffffffu, dg, off);
                        const int ok2 = __shfl_down_sync(0xffffffffu, key, off);
                        if (lane + off < 32 && ok2 == key) dg += og;
                    }
                    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
                    if (valid && (lane == 0 || prev != key) && dg != 0.0)
                        atomicAdd(&args.gacc[t * args.t_stride + args.nu0 + nu], dg);
                }
            } else if (EPI == EPI_GL) {
                // EPI_GS's element weight e, applied instead of stored: e adds to the linewidth of
                // (q, nu) and (scale / f) e (f' lambda(q', nu') + f'' lambda(q'', nu'')), signed by
                // the time-reversal codes, to y of row (q, nu); segmented sums over the rows of
                // each band in the warp, the first lane of a segment adds them
                const int nu = row / args.n, n2i = row % args.n;
                float f0 = 0.f, f2 = 0.f, nn2 = 0.f;
                double f0d = 1.0, f2d = 0.0;
                if (valid) {
                    f0d = args.freq[(int64_t)args.iq * args.n + args.nu0 + nu];
                    f0 = (float)f0d;
                    f2d = args.freq[(int64_t)q2 * args.n + n2i];
                    f2 = (float)f2d;
                    nn2 = (float)args.nB[(int64_t)q2 * args.n + n2i];
                }
                const bool live = valid && f0 >= args.f_min && f2 >= args.f_min;
                const bool gauss = args.shape == PHX_GAUSS;
                const float a = -1.f / (args.sigma * args.sigma), h2 = 0.25f * args.sigma * args.sigma;
                const float norm = gauss ? 0.56418958354775628f / args.sigma : 0.5f * args.sigma / 3.14159265358979f;
                const float rowfac = live ? norm / (1558.5454565440389f * f0 * f2) : 0.0f;
                const float d02 = f0 - f2, s02 = f0 + f2, lim = args.window * args.sigma;
                const float one_n2 = 1.f + nn2;
                const int key = valid ? nu : -1 - lane;
                float l2[3] = {0.f, 0.f, 0.f};
                {
                    const int cq = args.tr_code[q2];
                    const int64_t col = (int64_t)(abs(cq) - 1) * args.n + n2i;
                    if (live && cq != 0 && col < args.g1_ld) {
                        const double fs = cq > 0 ? f2d : -f2d;
                        for (int c = 0; c < 3; ++c) l2[c] = (float)(fs * args.lam[c * args.g1_ld + col]);
                    }
                }
                unsigned seg = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int off = 1 << k;
                    const int k2 = __shfl_down_sync(0xffffffffu, key, off);
                    if (lane + off < 32 && k2 == key) seg |= 1u << k;
                }
                const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
                const bool head = lane == 0 || prev_key != key;
                float gs = 0.f, y0 = 0.f, y1 = 0.f, y2 = 0.f;
                float vi[16];
                for (int j0 = half * 16; j0 < mg; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    tc::tmem_ld16(taddr + mg + j0, vi);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int j = m0 + j0 + i;
                        const float f1 = s_f1[j], n1 = s_n1[j], if1 = s_if1[j];
                        const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                        const float gd = fabsf(x) < lim ? (gauss ? __expf(a * x * x) : __frcp_rn(x * x + h2)) : 0.f;
                        const float ga = fabsf(y) < lim ? (gauss ? __expf(a * y * y) : __frcp_rn(y * y + h2)) : 0.f;
                        const float gb = pk && fabsf(z) < lim ? (gauss ? __expf(a * z * z) : __frcp_rn(z * z + h2)) : 0.f;
                        const float w = (cA * (one_n2 + n1) * gd + cB * (n1 - nn2) * (ga - gb)) * (if1 * rowfac);
                        const float e = fmaf(v[i], v[i], vi[i] * vi[i]) * w;
                        gs += e;
                        y0 = fmaf(e, s_lam[0][j], y0);
                        y1 = fmaf(e, s_lam[1][j], y1);
                        y2 = fmaf(e, s_lam[2][j], y2);
                    }
                }
                double dg = (double)gs;
                double dy[3] = {(double)fmaf(gs, l2[0], y0), (double)fmaf(gs, l2[1], y1), (double)fmaf(gs, l2[2], y2)};
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const double og = __shfl_down_sync(0xffffffffu, dg, 1 << k);
                    const double o0 = __shfl_down_sync(0xffffffffu, dy[0], 1 << k);
                    const double o1 = __shfl_down_sync(0xffffffffu, dy[1], 1 << k);
                    const double o2 = __shfl_down_sync(0xffffffffu, dy[2], 1 << k);
                    if (seg & (1u << k)) { dg += og; dy[0] += o0; dy[1] += o1; dy[2] += o2; }
                }
                if (valid && head) {
                    if (dg != 0.0) atomicAdd(&args.gacc[args.nu0 + nu], dg);
                    const int64_t grow = args.g1_row0 + nu;
                    if (grow < args.g1_rows) {
                        const double rs = args.g1_scale / f0d;
                        for (int c = 0; c < 3; ++c)
                            if (dy[c] != 0.0) atomicAdd(&args.ylam[c * args.g1_ld + grow], rs * dy[c]);
                    }
                }
            } else if (EPI == EPI_GS) {
                // EPI_G with the per-element weight e = |V|^2 x (decay + absorption weight) x the
                // row factors kept: e adds to the linewidth of (q, nu) and, scaled by f'/f and
                // f''/f, to the off-diagonal columns (q', nu') and (q'', nu'') of its row.  Column
                // sums run over the rows of one band nu (a warp holds 32 rows (nu, nu'')) and go
                // to Gamma1 from registers; the two warps of a lane group add their row sums
                // through a shared slot and a pairwise barrier.  No CTA-wide barrier per tile.
                static_assert(EPI != EPI_GS || kEpiParts == 2, "EPI_GS pairs the two warps of a lane group");
                const int nu = row / args.n, n2i = row % args.n;
                float f0 = 0.f, f2 = 0.f, nn2 = 0.f;
                double f0d = 1.0;
                if (valid) {
                    f0d = args.freq[(int64_t)args.iq * args.n + args.nu0 + nu];
                    f0 = (float)f0d;
                    f2 = (float)args.freq[(int64_t)q2 * args.n + n2i];
                    nn2 = (float)args.nB[(int64_t)q2 * args.n + n2i];
                }
                const bool live = valid && f0 >= args.f_min && f2 >= args.f_min;
                const bool gauss = args.shape == PHX_GAUSS;
                const float a = -1.f / (args.sigma * args.sigma), h2 = 0.25f * args.sigma * args.sigma;
                const float norm = gauss ? 0.56418958354775628f / args.sigma : 0.5f * args.sigma / 3.14159265358979f;
                const float rowfac = live ? norm / (1558.5454565440389f * f0 * f2) : 0.0f;
                const float d02 = f0 - f2, s02 = f0 + f2, lim = args.window * args.sigma;
                const float one_n2 = 1.f + nn2;
                const int key = valid ? nu : -1 - lane;
                const bool vec4 = (args.n & 3) == 0;       // groups of four adjacent entries stay in one row
                const int c1 = args.tr_code[q1], c2 = args.tr_code[q2];
                const double rs = args.g1_scale / f0d;     // Gamma1 scale over f of this row's band
                const int64_t grow = (args.g1_row0 + nu) * args.g1_ld;
                const bool row_ok = valid && args.g1_row0 + nu < args.g1_rows;
                // all lanes take part in every shuffle and vote below (none sits behind a condition)
                const int key0 = __shfl_sync(0xffffffffu, key, 0);
                const bool uniform = __all_sync(0xffffffffu, valid && key == key0);
                unsigned seg = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int off = 1 << k;
                    const int k2 = __shfl_down_sync(0xffffffffu, key, off);
                    if (lane + off < 32 && k2 == key) seg |= 1u << k;
                }
                const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
                const bool head = lane == 0 || prev_key != key;
                float gs = 0.f;
                float vi[16], e[16];
                for (int j0 = half * 16; j0 < mg; j0 += kStride) {
                    tc::tmem_ld16(taddr + j0, v);
                    tc::tmem_ld16(taddr + mg + j0, vi);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int j = m0 + j0 + i;
                        const float f1 = s_f1[j], n1 = s_n1[j], if1 = s_if1[j];
                        const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                        const float gd = fabsf(x) < lim ? (gauss ? __expf(a * x * x) : __frcp_rn(x * x + h2)) : 0.f;
                        const float ga = fabsf(y) < lim ? (gauss ? __expf(a * y * y) : __frcp_rn(y * y + h2)) : 0.f;
                        const float gb = pk && fabsf(z) < lim ? (gauss ? __expf(a * z * z) : __frcp_rn(z * z + h2)) : 0.f;
                        const float w = (cA * (one_n2 + n1) * gd + cB * (n1 - nn2) * (ga - gb)) * (if1 * rowfac);
                        e[i] = fmaf(v[i], v[i], vi[i] * vi[i]) * w;
                        gs += e[i];
                    }
                    if (uniform && vec4) {
                        // one band across the warp: a halving exchange leaves lane l with the warp
                        // sum of column l >> 1; lanes 8k then gather columns 4k .. 4k+3 and add
                        // them to Gamma1 with one 16-byte reduction
                        float a8[8], a4[4], a2[2];
                        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            a8[k] = (b4 ? e[k + 8] : e[k]) + __shfl_xor_sync(0xffffffffu, b4 ? e[k] : e[k + 8], 16);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            a4[k] = (b3 ? a8[k + 4] : a8[k]) + __shfl_xor_sync(0xffffffffu, b3 ? a8[k] : a8[k + 4], 8);
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            a2[k] = (b2 ? a4[k + 2] : a4[k]) + __shfl_xor_sync(0xffffffffu, b2 ? a4[k] : a4[k + 2], 4);
                        float a1 = (b1 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? a2[0] : a2[1], 2);
                        a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
                        const int src = lane & ~7;
                        const float g1v = __shfl_sync(0xffffffffu, a1, src + 2);
                        const float g2v = __shfl_sync(0xffffffffu, a1, src + 4);
                        const float g3v = __shfl_sync(0xffffffffu, a1, src + 6);
                        const int col = m0 + j0 + 4 * (lane >> 3);
                        if ((lane & 7) == 0 && row_ok && c1 != 0 && col < args.n &&
                            (a1 != 0.f || g1v != 0.f || g2v != 0.f || g3v != 0.f)) {
                            const int64_t gc = (int64_t)(abs(c1) - 1) * args.n + col;
                            if (gc + 3 < args.g1_ld) {
                                const double r = c1 > 0 ? rs : -rs;
                                const double* f1 = args.freq + (int64_t)q1 * args.n + col;
                                atomicAdd(reinterpret_cast<float4*>(args.g1 + grow + gc),
                                          make_float4((float)(r * f1[0] * a1), (float)(r * f1[1] * g1v),
                                                      (float)(r * f1[2] * g2v), (float)(r * f1[3] * g3v)));
                            } else {
                                atomicExch(args.status, (int)PHX_ERR_INVALID);   // bounds self-check
                            }
                        }
                    } else {
                        // segmented sums over the rows of each band in the warp; the first lane of
                        // a segment adds it to Gamma1
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            float c = e[i];
#pragma unroll
                            for (int k = 0; k < 5; ++k) {
                                const float o = __shfl_down_sync(0xffffffffu, c, 1 << k);
                                if (seg & (1u << k)) c += o;
                            }
                            const int col = m0 + j0 + i;
                            if (row_ok && head && c != 0.f && c1 != 0 && col < args.n) {
                                const int64_t gc = (int64_t)(abs(c1) - 1) * args.n + col;
                                if (gc < args.g1_ld)
                                    atomicAdd(args.g1 + grow + gc,
                                              (float)((c1 > 0 ? rs : -rs) * args.freq[(int64_t)q1 * args.n + col] * c));
                                else
                                    atomicExch(args.status, (int)PHX_ERR_INVALID);
                            }
                        }
                    }
                }
                // linewidth: segmented sums of this part's row sums
                double dg = (double)gs;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const double og = __shfl_down_sync(0xffffffffu, dg, 1 << k);
                    if (seg & (1u << k)) dg += og;
                }
                if (valid && head && dg != 0.0) atomicAdd(&args.gacc[args.nu0 + nu], dg);
                // column (q'', nu''): this row's sum over nu', the two parts added through a
                // double-buffered slot (the pairwise barrier orders the write before the read and
                // the read before the slot's reuse two items later)
                const int buf = (it - item_begin) & 1;
                if (half == 1) s_rows[buf][lgrp][lane] = gs;
                asm volatile("bar.sync %0, 64;" ::"r"(2 + lgrp) : "memory");
                if (half == 0) {
                    const float tot = gs + s_rows[buf][lgrp][lane];
                    if (vec4) {
                        const float t1 = __shfl_down_sync(0xffffffffu, tot, 1);
                        const float t2 = __shfl_down_sync(0xffffffffu, tot, 2);
                        const float t3 = __shfl_down_sync(0xffffffffu, tot, 3);
                        if ((lane & 3) == 0 && row_ok && c2 != 0 && (tot != 0.f || t1 != 0.f || t2 != 0.f || t3 != 0.f)) {
                            const int64_t gc = (int64_t)(abs(c2) - 1) * args.n + n2i;
                            if (gc + 3 < args.g1_ld) {
                                const double r = c2 > 0 ? rs : -rs;
                                const double* f2p = args.freq + (int64_t)q2 * args.n + n2i;
                                atomicAdd(reinterpret_cast<float4*>(args.g1 + grow + gc),
                                          make_float4((float)(r * f2p[0] * tot), (float)(r * f2p[1] * t1),
                                                      (float)(r * f2p[2] * t2), (float)(r * f2p[3] * t3)));
                            } else {
                                atomicExch(args.status, (int)PHX_ERR_INVALID);
                            }
                        }
                    } else if (row_ok && c2 != 0 && tot != 0.f) {
                        const int64_t gc = (int64_t)(abs(c2) - 1) * args.n + n2i;
                        if (gc < args.g1_ld)
                            atomicAdd(args.g1 + grow + gc,
                                      (float)((c2 > 0 ? rs : -rs) * args.freq[(int64_t)q2 * args.n + n2i] * tot));
                        else
                            atomicExch(args.status, (int)PHX_ERR_INVALID);
                    }
                }
            } else {
                // row (nu, nu'') holds V[nu'] = [Re | Im]; weight and reduce over nu'
                const int nu = row / args.n, n2i = row % args.n;
                float f0 = 0.f, f2 = 0.f, nn2 = 0.f;
                if (valid) {
                    f0 = (float)args.freq[(int64_t)args.iq * args.n + args.nu0 + nu];
                    f2 = (float)args.freq[(int64_t)q2 * args.n + n2i];
                    nn2 = (float)args.nB[(int64_t)q2 * args.n + n2i];
                }
                const bool live = valid && f0 >= args.f_min && f2 >= args.f_min;
                // w = [...] / (2 pi)^4 / (f0 f1 f2): delta(w) = g(f)/(2 pi) and 1/(w0 w1 w2)
                const float inv_f02 = live ? 1.0f / (1558.5454565440389f * f0 * f2) : 0.0f;
                const float d02 = f0 - f2, s02 = f0 + f2, lim = args.window * args.sigma;
                const float one_n2 = 1.f + nn2;
                float gs = 0.f, ws = 0.f;
                float vi[16];
                if (args.shape == PHX_GAUSS) {
                    const float a = -1.f / (args.sigma * args.sigma), norm = 0.56418958354775628f / args.sigma;
                    for (int j0 = half * 16; j0 < mg; j0 += kStride) {
                        tc::tmem_ld16(taddr + j0, v);
                        tc::tmem_ld16(taddr + mg + j0, vi);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int j = m0 + j0 + i;
                            const float f1 = s_f1[j], n1 = s_n1[j], if1 = s_if1[j];
                            const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                            const float gd = fabsf(x) < lim ? __expf(a * x * x) : 0.f;
                            const float ga = fabsf(y) < lim ? __expf(a * y * y) : 0.f;
                            const float gb = pk && fabsf(z) < lim ? __expf(a * z * z) : 0.f;
                            const float w = (cA * (one_n2 + n1) * gd + cB * (n1 - nn2) * (ga - gb)) * if1;
                            gs = fmaf(fmaf(v[i], v[i], vi[i] * vi[i]), w, gs);
                            ws += w;
                        }
                    }
                    gs *= norm;
                    ws *= norm;
                } else {
                    const float h = 0.5f * args.sigma, h2 = h * h, norm = h / 3.14159265358979f;
                    for (int j0 = half * 16; j0 < mg; j0 += kStride) {
                        tc::tmem_ld16(taddr + j0, v);
                        tc::tmem_ld16(taddr + mg + j0, vi);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int j = m0 + j0 + i;
                            const float f1 = s_f1[j], n1 = s_n1[j], if1 = s_if1[j];
                            const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                            const float gd = fabsf(x) < lim ? __frcp_rn(x * x + h2) : 0.f;
                            const float ga = fabsf(y) < lim ? __frcp_rn(y * y + h2) : 0.f;
                            const float gb = pk && fabsf(z) < lim ? __frcp_rn(z * z + h2) : 0.f;
                            const float w = (cA * (one_n2 + n1) * gd + cB * (n1 - nn2) * (ga - gb)) * if1;
                            gs = fmaf(fmaf(v[i], v[i], vi[i] * vi[i]), w, gs);
                            ws += w;
                        }
                    }
                    gs *= norm;
                    ws *= norm;
                }
                gs *= inv_f02;
                ws *= inv_f02;
                // rows of equal nu are contiguous: segmented suffix sums over the warp, then the
                // first lane of each segment adds its segment into the FP64 accumulator
                const int key = valid ? nu : -1 - lane;
                double dg = (double)gs, dw = (double)ws;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const double og = __shfl_down_sync(0xffffffffu, dg, off);
                    const double ow = __shfl_down_sync(0xffffffffu, dw, off);
                    const int ok2 = __shfl_down_sync(0xffffffffu, key, off);
                    if (lane + off < 32 && ok2 == key) { dg += og; dw += ow; }
                }
                const int prev = __shfl_up_sync(0xffffffffu, key, 1);
                if (valid && (lane == 0 || prev != key)) {
                    if (dg != 0.0) atomicAdd(&args.gacc[args.nu0 + nu], dg);
                    if (args.wacc && dw != 0.0) atomicAdd(&args.wacc[args.nu0 + nu], dw);
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&tempty_bar[acc]);
            if (args.n_acc == 2) { acc ^= 1; if (acc == 0) acc_phase ^= 1; } else { acc_phase ^= 1; }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, args.tmem_cols);
    }
}

#include "chain_tc.cuh"

// ---------------------------------------------------------------- operand preparation kernels

// Eigenvector row table of every mesh point for the chained kernel: row (q, j) = [Re e_q(k, j)
// (k < kcp) | Im e_q(k, j)], zero for k >= n.
template <int PREC>
__global__ void prep_evec_rows(const double2* __restrict__ evec, int nq, int n, int kcp, void* hi, void* lo) {
    const int kr = 2 * kcp;
    const int64_t total = (int64_t)nq * n * kr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(t % kr);
        const int64_t row = t / kr;
        const int j = (int)(row % n);
        const int64_t q = row / n;
        const int k = kk < kcp ? kk : kk - kcp;
        float val = 0.f;
        if (k < n) {
            const double2 e = evec[(q * n + k) * n + j];
            val = (float)(kk < kcp ? e.x : e.y);
        }
        store_operand<PREC>(hi, lo, t, val);
    }
}

// B tables of the eigenvectors of every mesh point: rows [Re out (np) | Im out (np)], K =
// [Re e(c) (Kcp) | Im e(c) (Kcp)] (see the header comment for the signs).
template <int PREC>
__global__ void prep_evec_tables(const double2* __restrict__ evec, int nq, int n, int np, int kcp, void* hi,
                                 void* lo) {
    const int N = 2 * np, kr = 2 * kcp;
    const int64_t total = (int64_t)nq * N * kr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(t % kr);
        const int j = (int)((t / kr) % N);
        const int q = (int)(t / ((int64_t)kr * N));
        const int mode = j < np ? j : j - np;
        const int k = kk < kcp ? kk : kk - kcp;
        float val = 0.f;
        if (mode < n && k < n) {
            const double2 e = evec[((int64_t)q * n + k) * n + mode];
            const bool re_out = j < np, re_in = kk < kcp;
            val = (float)(re_out ? (re_in ? e.x : -e.y) : (re_in ? e.y : e.x));
        }
        store_operand<PREC>(hi, lo, t, val);
    }
}

// The q' of one irreducible q in increasing mesh order with their q'' = -(q + q') mod G.  With
// `pair`, only the q' with q' <= q'' are listed: V3 is symmetric under the exchange of the two
// partners (Eq. (phi3_proj) sums over all three modes alike), so one evaluation of an
// unordered pair {q', q''} serves both terms of the q' sum; there are (nq + n_self) / 2 of
// them, n_self counting the q' = q''.  One block.
__global__ void pair_list_kernel(int iq, int m1, int m2, int m3, int pair, int32_t* __restrict__ qp,
                                 int32_t* __restrict__ qpp) {
    __shared__ int s_warp[32];
    __shared__ int s_base;
    const int nq = m1 * m2 * m3, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nq; c0 += blockDim.x) {
        const int q1 = c0 + threadIdx.x;
        const int q2 = q1 < nq ? phx_third_index(iq, q1, m1, m2, m3) : 0;
        const bool take = q1 < nq && (!pair || q1 <= q2);
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        int before = s_base;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        if (take) {
            const int pos = before + __popc(bal & ((1u << lane) - 1u));
            qp[pos] = q1;
            qpp[pos] = q2;
        }
        __syncthreads();
        if (threadIdx.x == 0) for (int w = 0; w < nw; ++w) s_base += s_warp[w];
        __syncthreads();
    }
}

// Length of pair_list_kernel's list (host side).
int pair_count(int iq, const int* mesh, bool pair) {
    const int nq = mesh[0] * mesh[1] * mesh[2];
    if (!pair) return nq;
    const int k[3] = {iq / (mesh[1] * mesh[2]), (iq / mesh[2]) % mesh[1], iq % mesh[2]};
    int n_self = 1;
    for (int d = 0; d < 3; ++d)     // solutions of 2 k' = -k (mod m): one for odd m, two or none for even m
        n_self *= (mesh[d] & 1) ? 1 : ((k[d] & 1) ? 0 : 2);
    return (nq + n_self) / 2;
}

// B tables of the Fourier phases exp(-i q'.d) for the listed q', tiles of Qb list entries
// (tile t, slot s: entry t * Qb + s; slots past the list or past Qb are zero).
template <int PREC>
__global__ void prep_phase_tables(const int32_t* __restrict__ d_int, int n_d, int m1, int m2, int m3,
                                  const int32_t* __restrict__ qlist, int count, int Qb, int n_tiles, int qp_np,
                                  int kcp, void* hi, void* lo) {
    const int N = 2 * qp_np, kr = 2 * kcp;
    const int64_t total = (int64_t)n_tiles * N * kr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = (int)(t % kr);
        const int j = (int)((t / kr) % N);
        const int tile = (int)(t / ((int64_t)kr * N));
        const int slot = j < qp_np ? j : j - qp_np;
        const int d = kk < kcp ? kk : kk - kcp;
        const int pos = tile * Qb + slot;
        float val = 0.f;
        if (slot < Qb && pos < count && d < n_d) {
            const int qp = qlist[pos];
            const int k1 = qp / (m2 * m3), k2 = (qp / m3) % m2, k3 = qp % m3;
            const int a1 = (k1 * d_int[3 * d]) % m1, a2 = (k2 * d_int[3 * d + 1]) % m2, a3 = (k3 * d_int[3 * d + 2]) % m3;
            double s, c;
            sincospi(2.0 * ((double)a1 / m1 + (double)a2 / m2 + (double)a3 / m3), &s, &c);
            // E(d, slot) = exp(-i theta) = c - i s
            const double er = c, ei = -s;
            const bool re_out = j < qp_np, re_in = kk < kcp;
            val = (float)(re_out ? (re_in ? er : -ei) : (re_in ? ei : er));
        }
        store_operand<PREC>(hi, lo, t, val);
    }
}

// S3, part 1: per COO entry the q-dependent factor phi/sqrt(mmm) * exp(+2 pi i q.R'') and the
// eigenvectors of q, both rounded to FP32 once per q (FP64 is the narrowest pipe on GB300).
__global__ void fold_phase_kernel(const int32_t* __restrict__ ent_src, const int32_t* __restrict__ ent_r2,
                                  const double* __restrict__ ent_w, int64_t nnz, double qa, double qb, double qc,
                                  float2* __restrict__ wph, const double2* __restrict__ eq, int nn,
                                  float2* __restrict__ eqf) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz + nn; k += (int64_t)gridDim.x * blockDim.x) {
        if (k < nnz) {
            const int64_t o = ent_src[k];              // wph in the (b, c)-grouped order of the entries
            const double x = 2.0 * (qa * ent_r2[3 * o] + qb * ent_r2[3 * o + 1] + qc * ent_r2[3 * o + 2]);
            double sn, cs;
            sincospi(x, &sn, &cs);
            wph[k] = make_float2((float)(ent_w[o] * cs), (float)(ent_w[o] * sn));
        } else {
            const double2 e = eq[k - nnz];
            eqf[k - nnz] = make_float2((float)e.x, (float)e.y);
        }
    }
}

// Eight consecutive elements (idx a multiple of 8): one 16-byte store per plane (bf16 planes)
// or two (tf32).
template <int PREC>
__device__ __forceinline__ void store_operand8(void* hi, void* lo, int64_t idx, const float* v) {
    if (PREC == P_BF16X3) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tc::split_bf16x2(v[2 * j], v[2 * j + 1], &h[j], &l[j]);
        *reinterpret_cast<uint4*>((__nv_bfloat16*)hi + idx) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>((__nv_bfloat16*)lo + idx) = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
        float4* o = reinterpret_cast<float4*>((float*)hi + idx);
        o[0] = make_float4(tc::round_tf32(v[0]), tc::round_tf32(v[1]), tc::round_tf32(v[2]), tc::round_tf32(v[3]));
        o[1] = make_float4(tc::round_tf32(v[4]), tc::round_tf32(v[5]), tc::round_tf32(v[6]), tc::round_tf32(v[7]));
    }
}

// S3, part 2: the DFT's A operand for one q, row (nu, b, c) with K = [Re W(d) | Im W(d)],
// W_nu(b, c; d) = sum over the COO entries (a, b, c) of lattice difference d of w_k e_q(a, nu).
// One warp per (b, c) pair and block of 32 bands (lane = band nu).  The pair's entries are
// contiguous and ordered by d: the lanes read them 32 at a time, (a, d, w) are broadcast by
// shuffles, and each run of equal d sums w e_q(a, nu) (a coalesced read of e_q's row a) in
// registers and writes it once into the warp's shared-memory tile (rows padded to 65 words:
// conflict-free row writes).  A chunk of 32 d is then stored transposed, eight lanes per row,
// so that every store instruction writes whole 128-byte lines, with the d that no run wrote
// selected as zero.  The next pair's bounds and
// first batch are read while the current one is summed.  Chunks without any entry are
// skipped: they are zero for every q, and the operand is cleared once per job.  When e_q fits
// beside the tiles (n <= 96: 16 warps, one CTA per SM) the CTA first copies it to shared
// memory; otherwise (8 warps, three CTAs per SM) it is read through the caches.
constexpr int kFoldPitch = 65;
constexpr size_t kFoldTile = 32 * kFoldPitch * sizeof(float);      // per warp
constexpr size_t kFoldSmemMax = 220 * 1024;

template <int PREC>
__global__ void __launch_bounds__(512) fold_tc_kernel(const int64_t* __restrict__ bc_start,
                                                      const int2* __restrict__ ent_ad,
                                                      const float2* __restrict__ wph,
                                                      const float2* __restrict__ eqf_g, int n, int nu0,
                                                      int nnu, int kcp, int eq_smem, void* hi, void* lo) {
    extern __shared__ float s_fold[];
    const int lane = threadIdx.x & 31;
    float* tile = s_fold + (threadIdx.x >> 5) * 32 * kFoldPitch;
    const float2* eqf = eqf_g;
    if (eq_smem) {
        float2* s_eq = reinterpret_cast<float2*>(s_fold + (blockDim.x >> 5) * 32 * kFoldPitch);
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s_eq[i] = eqf_g[i];
        __syncthreads();
        eqf = s_eq;
    }
    const int nn = n * n, kr = 2 * kcp;
    const int64_t items = (int64_t)nn * ((nnu + 31) / 32);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int2 none = make_int2(0, -1);
    // store lanes: row group lane >> 3, part (lane >> 2) & 1 (Re, Im), 8-element chunk lane & 3
    const int st_row = lane >> 3, st_part = (lane >> 2) & 1, st_chunk = (lane & 3) * 8;
    int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    // bounds of item it (a) and it + warps (b); first batch of item it
    int64_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    int2 ad = none;
    float2 w = make_float2(0.f, 0.f);
    if (it < items) {
        const int bc = (int)(it % nn);
        a0 = bc_start[bc]; a1 = bc_start[bc + 1];
        if (lane < a1 - a0) { ad = ent_ad[a0 + lane]; w = wph[a0 + lane]; }
    }
    if (it + warps < items) {
        const int bc = (int)((it + warps) % nn);
        b0 = bc_start[bc]; b1 = bc_start[bc + 1];
    }
    for (; it < items; it += warps) {
        // in flight while this item is summed: the next item's first batch, the bounds after it
        int2 nad = none;
        float2 nw = make_float2(0.f, 0.f);
        if (it + warps < items && lane < b1 - b0) { nad = ent_ad[b0 + lane]; nw = wph[b0 + lane]; }
        int64_t c0 = 0, c1 = 0;
        if (it + 2 * warps < items) {
            const int bc = (int)((it + 2 * warps) % nn);
            c0 = bc_start[bc]; c1 = bc_start[bc + 1];
        }
        if (a1 > a0) {
            const int bc = (int)(it % nn);
            const int band0 = (int)(it / nn) * 32;         // first band of the block
            const int nl = band0 + lane;
            const float2* erow = eqf + (nu0 + (nl < nnu ? nl : 0));
            int64_t jb = a0, j = a0;                       // first entry of the batch, next entry
            for (int dc = 0; dc < kcp && j < a1; dc += 32) {
                // runs of equal d (entries are ordered by d): each run's sum goes to the tile once,
                // and the mask of written d zero-selects the rest when the chunk is stored
                uint32_t mask = 0;
                while (j < a1) {
                    int t = (int)(j - jb);
                    const int d = __shfl_sync(0xffffffffu, ad.y, t);
                    if (d >= dc + 32) break;
                    float sr = 0.f, si = 0.f;
                    do {
                        const int a = __shfl_sync(0xffffffffu, ad.x, t);
                        const float wx = __shfl_sync(0xffffffffu, w.x, t), wy = __shfl_sync(0xffffffffu, w.y, t);
                        const float2 e = erow[(int64_t)a * n];
                        sr += wx * e.x - wy * e.y;
                        si += wx * e.y + wy * e.x;
                        if (++j - jb == 32 && j < a1) {
                            jb = j;
                            ad = lane < a1 - jb ? ent_ad[jb + lane] : none;
                            w = lane < a1 - jb ? wph[jb + lane] : make_float2(0.f, 0.f);
                        }
                        t = (int)(j - jb);
                    } while (j < a1 && __shfl_sync(0xffffffffu, ad.y, t) == d);
                    tile[lane * kFoldPitch + (d - dc)] = sr;
                    tile[lane * kFoldPitch + 32 + (d - dc)] = si;
                    mask |= 1u << (d - dc);
                }
                if (mask == 0) continue;
                __syncwarp();
#pragma unroll 2
                for (int g = 0; g < 32; g += 4) {
                    const int r = g + st_row;
                    if (band0 + r < nnu) {
                        const float* src = tile + r * kFoldPitch + st_part * 32 + st_chunk;
                        float v[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) v[k] = ((mask >> (st_chunk + k)) & 1u) ? src[k] : 0.f;
                        store_operand8<PREC>(hi, lo, ((int64_t)(band0 + r) * nn + bc) * kr + st_part * kcp + dc + st_chunk, v);
                    }
                }
                __syncwarp();
            }
        }
        a0 = b0; a1 = b1; b0 = c0; b1 = c1;
        ad = nad; w = nw;
    }
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

// 2D map over a row-major [rows][kr] operand plane, box = 128-byte K chunk x box_rows.
bool make_map(CUtensorMap* m, const void* base, int prec, int64_t rows, int kr, int box_rows) {
    const int esz = prec == P_BF16X3 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)kr, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kr * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / esz), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, prec == P_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Operand {
    void* hi = nullptr;
    void* lo = nullptr;
    int64_t rows = 0;
    int kr = 0;
};

size_t smem_bytes(int prec, bool stream_b, int nk, int mg, int stages) {
    const int planes = prec == P_BF16X3 ? 2 : 1;
    const size_t b_bytes = stream_b ? 0 : (size_t)planes * nk * 2 * mg * kChunkBytes;
    const size_t stage = (size_t)planes * (kStageBytesPerPlane + (stream_b ? 2 * (size_t)mg * kChunkBytes : 0));
    return 1024 + b_bytes + (size_t)stages * stage;
}

template <int PREC, int EPI, bool STREAM>
cudaError_t launch_gemm(phx_ctx* ctx, TcArgs& a, int n_problems, int ctas, cudaStream_t s) {
    const size_t smem = smem_bytes(PREC, STREAM, a.nk, a.mg, a.stages);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<PREC, EPI, STREAM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kSmemLimit - 8192));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    (void)ctx;
    a.n_problems = n_problems;
    const int64_t items = (int64_t)n_problems * a.tiles * a.n_groups;
    dim3 grid((unsigned)std::min<int64_t>(items, ctas), 1);
    tc_gemm_kernel<PREC, EPI, STREAM><<<grid, kernel_threads<EPI>(), smem, s>>>(a);
    return cudaGetLastError();
}

template <int PREC, int MODE>
cudaError_t launch_chain(ChainArgs& a, size_t smem, int ctas, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(chain_kernel<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kSmemLimit - 8192));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n_items <= 0) return cudaSuccess;
    dim3 grid((unsigned)std::min(a.n_items, ctas), 1);
    chain_kernel<PREC, MODE><<<grid, kChainThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_chain_mode(ChainArgs& a, int mode, size_t smem, int ctas, cudaStream_t s) {
    if (mode == CHAIN_GT) return launch_chain<PREC, CHAIN_GT>(a, smem, ctas, s);
    if (mode == CHAIN_GS) return launch_chain<PREC, CHAIN_GS>(a, smem, ctas, s);
    if (mode == CHAIN_GL) return launch_chain<PREC, CHAIN_GL>(a, smem, ctas, s);
    return launch_chain<PREC, CHAIN_G>(a, smem, ctas, s);
}

template <int PREC, int EPI>
cudaError_t launch_gemm_any(phx_ctx* ctx, TcArgs& a, bool stream_b, int n_problems, int ctas, cudaStream_t s) {
    return stream_b ? launch_gemm<PREC, EPI, true>(ctx, a, n_problems, ctas, s)
                    : launch_gemm<PREC, EPI, false>(ctx, a, n_problems, ctas, s);
}

// Shared-memory plan: as many stages as fit next to a resident B (stream_b = false) or with B
// streamed in every stage; at least 2 stages or the plan fails.
bool plan_stages(int prec, bool stream_b, int nk, int mg, int* stages) {
    const size_t avail = kSmemLimit - 8192;   // static shared memory headroom
    if (smem_bytes(prec, stream_b, nk, mg, 2) > avail) return false;
    int st = 2;
    while (st < kMaxStages && smem_bytes(prec, stream_b, nk, mg, st + 1) <= avail) ++st;
    *stages = st;
    return true;
}

uint32_t tmem_cols_for(int N, int n_acc) {
    uint32_t need = (uint32_t)(N * n_acc), c = 32;
    while (c < need) c <<= 1;
    return c;
}

// ---------------------------------------------------------------- plan / prepare / enqueue

// Shapes of one tensor-core linewidth job (pure arithmetic; no device work).
struct TcPlan {
    int prec = P_BF16X3;
    int n = 0, nq = 0;
    int kcp = 0, kr = 0, nk = 0;            // eigenvector contractions: K layout
    int np = 0, mg = 0, n_groups = 1, st_e = 0;
    bool stream_b = false;
    int kcp_d = 0, kr_d = 0, nk_d = 0, st_d = 0;   // Fourier GEMM
    int n_nu = 0, Q = 0, qp_np = 0, n_tiles_q = 0;
    int64_t rows_w = 0, rows_a = 0;
    // chained eigenvector contractions (chain_kernel) instead of the e_q'' and e_q' GEMMs
    bool chain = false;
    int c_ra = 0, c_rb3 = 0, c_stages = 0;
    size_t c_smem = 0;
    int side = -1;                          // SMs of the side stream (-1: the context's choice)
    // workspace bytes per operand plane
    size_t bytes_w = 0, bytes_m = 0, bytes_e = 0, bytes_p = 0, bytes_t = 0;
};

// Shapes of the chained kernel for n <= 96 modes (K half kcp): tensor memory holds D2 (2 kcp
// columns) and D3 (Re | Im of all rb3 = n rounded to 16 partner modes); shared memory holds the
// two eigenvector tables and every M chunk of one item (stages >= nk).
bool chain_shapes(TcPlan& P) {
    if (P.kcp > 96 || P.n > 96) return false;
    const int planes = P.prec == P_BF16X3 ? 2 : 1;
    P.c_rb3 = round_up(P.n, 16);
    P.c_ra = round_up(P.n, 8);
    const size_t fixed = (size_t)planes * P.nk * kChunkBytes * (P.c_ra + P.c_rb3);
    const size_t stage = (size_t)planes * P.kcp * kChunkBytes;
    const size_t avail = kSmemLimit - 8192 - 1024;
    if (P.nk > kMaxStages || fixed + (size_t)P.nk * stage > avail) return false;
    // whole items of M chunks (the kernel's ring holds stages / nk items)
    P.c_stages = (int)std::min<size_t>(kMaxStages, (avail - fixed) / stage) / P.nk * P.nk;
    P.c_smem = 1024 + fixed + (size_t)P.c_stages * stage;
    // the stage-2 MMA reads 128 rows from every A block (rows >= ra land in the next block and
    // only feed output rows that are discarded): that read must stay inside the allocation
    const size_t a_read_end = 1024 + (size_t)(planes * P.nk - 1) * P.c_ra * kChunkBytes + 128 * kChunkBytes;
    if (a_read_end > P.c_smem) P.c_smem = a_read_end;
    if (P.c_smem > kSmemLimit - 8192) return false;
    return true;
}

// chain_pref: -1 follows PHX_OPT_CHAIN, 0 never, 1 wherever the chained kernel fits
phx_status tc_plan(phx_ctx* ctx, const phx_fc3* f, int prec, int q_override, TcPlan* pl, int chain_pref = -1) {
    TcPlan P;
    P.prec = prec;
    const int n = f->n, nq = f->nq;
    P.n = n;
    P.nq = nq;
    const int esz = prec == P_BF16X3 ? 2 : 4;
    const int planes = prec == P_BF16X3 ? 2 : 1;
    P.kcp = round_up(n, 32);
    P.kr = 2 * P.kcp;
    const int kelems = kChunkBytes / esz;
    P.nk = P.kr / kelems;
    // Output columns: the eigenvector B table stays resident in shared memory when it fits
    // (one column group); otherwise the modes are split into groups of mg <= 128 whose Re/Im
    // halves share one accumulator and B is streamed with every A chunk.
    P.np = round_up(n, 16);
    P.mg = P.np;
    if (P.np > 128 || !plan_stages(prec, false, P.nk, P.mg, &P.st_e)) {
        P.stream_b = true;
        P.n_groups = (P.np + 127) / 128;
        while (true) {
            P.mg = round_up((P.np + P.n_groups - 1) / P.n_groups, 16);
            if (plan_stages(prec, true, P.nk, P.mg, &P.st_e)) break;
            if (P.mg <= 16) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path: n = %d does not fit", n);
            ++P.n_groups;
        }
        P.np = P.mg * P.n_groups;
    }
    if (P.np > kMaxNp) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path: n = %d > %d", n, kMaxNp);
    P.kcp_d = round_up(f->n_d, 32);
    P.kr_d = 2 * P.kcp_d;
    P.nk_d = P.kr_d / kelems;
    // Working set: modes of q in chunks of n_nu (W of a chunk <= 1 GB; measured on GB300 at 96
    // modes, chunking for L2 residency loses more to launch count than it gains) and q' in
    // tiles of Q (M and X of a tile together <= 2.5 GB: 128 q' at 96 modes, the most the
    // Fourier GEMM's double-buffered accumulator holds (2 x 256 of the 512 tensor-memory
    // columns); each doubling of Q halves the re-reads of W, and 128 ran the whole step 9 %
    // faster than 64 on GB300).  PHX_NU_CHUNK / PHX_Q_TILE or the autotuner override the
    // defaults.
    const int64_t n2 = (int64_t)n * n;
    P.n_nu = (int)std::max<int64_t>(1, std::min<int64_t>(n, ((int64_t)1 << 30) / (n2 * P.kr_d * esz * planes)));
    if (const char* env = getenv("PHX_NU_CHUNK")) {
        const int v = atoi(env);
        if (v > 0) P.n_nu = std::min(v, n);
    }
    const int64_t per_qp = 2 * (int64_t)P.n_nu * n * P.kr * esz * planes;   // M + X of one q'
    int Q = (int)std::max<int64_t>(1, std::min<int64_t>(nq, ((int64_t)2560 << 20) / per_qp));
    Q = std::min(Q, 128);
    if (const char* env = getenv("PHX_Q_TILE")) {
        const int v = atoi(env);
        if (v > 0) Q = std::min(std::min(v, 128), nq);
    }
    if (q_override > 0) Q = std::min(std::min(q_override, 128), nq);
    while (!plan_stages(prec, false, P.nk_d, round_up(Q, 8), &P.st_d)) {   // phase table must fit too
        if (Q <= 8)
            return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path: %d lattice differences exceed shared memory", f->n_d);
        Q = std::max(8, Q / 2);
    }
    P.Q = Q;
    P.qp_np = round_up(Q, 8);
    P.n_tiles_q = (nq + Q - 1) / Q;
    P.rows_w = (int64_t)P.n_nu * n2;
    P.rows_a = (int64_t)P.n_nu * n;
    if (P.rows_w > INT32_MAX / 2) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path: W chunk too large");
    P.bytes_w = (size_t)P.rows_w * P.kr_d * esz;
    P.bytes_m = (size_t)Q * P.rows_a * P.kr * esz;
    if ((int64_t)Q * P.rows_a * P.kr >= ((int64_t)1 << 31))   // the Fourier epilogue indexes M in 32 bits
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path: q' tile of M too large");
    P.bytes_e = (size_t)nq * 2 * P.np * P.kr * esz;
    P.bytes_p = (size_t)P.n_tiles_q * 2 * P.qp_np * P.kr_d * esz;
    // Chained contractions: by default where they beat the three-GEMM chain (64 < n <= 96: the
    // MMA rows are modes, so small n would leave most of the 128 rows idle); PHX_OPT_CHAIN
    // forces them on (any n they fit) or off.
    const int oc = chain_pref == 0 ? 2 : chain_pref == 1 ? 1 : ctx->opt_chain;
    if (oc != 2 && (oc == 1 || (n > 64 && n <= 96))) P.chain = chain_shapes(P);
    if (P.chain) {
        P.bytes_t = (size_t)nq * n * P.kr * esz;
        P.bytes_e = 0;
    }
    *pl = P;
    return PHX_OK;
}

// Per-crystal device tables (kept with the Phi3 handle): the entries grouped by (b, c), then
// d, then a, with their source positions.  Host work; must run before any stream capture.
phx_status tc_prepare_fc3(phx_ctx* ctx, phx_fc3* f) {
    if (f->tc_bc_start) return PHX_OK;
    const int n = f->n;
    const int64_t n2 = (int64_t)n * n, nnz = f->nnz, ns = f->n_seg;
    std::vector<int32_t> keys((size_t)ns * 3), ea((size_t)nnz);
    std::vector<int64_t> ss((size_t)ns + 1, 0);
    if (ns > 0) {
        PHX_CUDA_CHECK(ctx, cudaMemcpy(keys.data(), f->seg_key, keys.size() * 4, cudaMemcpyDeviceToHost));
        PHX_CUDA_CHECK(ctx, cudaMemcpy(ss.data(), f->seg_start, ss.size() * 8, cudaMemcpyDeviceToHost));
        PHX_CUDA_CHECK(ctx, cudaMemcpy(ea.data(), f->ent_a, ea.size() * 4, cudaMemcpyDeviceToHost));
    }
    std::vector<int64_t> start((size_t)n2 + 1, 0);
    for (int64_t sg = 0; sg < ns; ++sg) start[(int64_t)keys[3 * sg + 1] * n + keys[3 * sg + 2] + 1] += ss[sg + 1] - ss[sg];
    for (int64_t b = 0; b < n2; ++b) start[b + 1] += start[b];
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    std::vector<int2> ad((size_t)nnz);
    std::vector<int32_t> src((size_t)nnz);
    // segments are stored in (d, b, c) order and their entries in a order, so each pair's
    // entries come out in (d, a) order
    for (int64_t sg = 0; sg < ns; ++sg) {
        const int64_t bc = (int64_t)keys[3 * sg + 1] * n + keys[3 * sg + 2];
        for (int64_t k = ss[sg]; k < ss[sg + 1]; ++k) {
            const int64_t j = fill[bc]++;
            ad[j] = make_int2(ea[k], keys[3 * sg]);
            src[j] = (int32_t)k;
        }
    }
    int64_t* dstart = nullptr;
    int2* dad = nullptr;
    int32_t* dsrc = nullptr;
    if (cudaMalloc(&dstart, start.size() * 8) != cudaSuccess ||
        cudaMalloc(&dad, std::max<size_t>(ad.size() * sizeof(int2), 16)) != cudaSuccess ||
        cudaMalloc(&dsrc, std::max<size_t>(src.size() * 4, 16)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dstart);
        cudaFree(dad);
        return phx_set_error(ctx, PHX_ERR_NOMEM, "tensor-core tables: allocation failed");
    }
    PHX_CUDA_CHECK(ctx, cudaMemcpy(dstart, start.data(), start.size() * 8, cudaMemcpyHostToDevice));
    if (nnz > 0) {
        PHX_CUDA_CHECK(ctx, cudaMemcpy(dad, ad.data(), ad.size() * sizeof(int2), cudaMemcpyHostToDevice));
        PHX_CUDA_CHECK(ctx, cudaMemcpy(dsrc, src.data(), src.size() * 4, cudaMemcpyHostToDevice));
    }
    f->tc_bc_start = dstart;
    f->tc_ent_ad = dad;
    f->tc_ent_src = dsrc;
    return PHX_OK;
}

struct TcBuffers {
    Operand W, M, M2, X, E, P, T;
    size_t m2_bytes = 0;        // bytes of each plane of M's second buffer (side stream), 0 without
    int32_t* qp = nullptr;      // q' list of the current irreducible q (pair_list_kernel)
    int32_t* qpp = nullptr;     // and their q''
    float2* wph = nullptr;
    float2* eqf = nullptr;
};

// Workspace large enough for the given byte counts (per plane) and element counts.
phx_status tc_alloc(phx_ctx* ctx, int prec, size_t bw, size_t bm, size_t bx, size_t be, size_t bp, size_t bt,
                    int64_t max_nq, int64_t max_nnz, int64_t max_n2, TcBuffers* b, size_t bm2 = 0) {
    const int planes = prec == P_BF16X3 ? 2 : 1;
    auto get = [&](const char* name, size_t bytes, Operand* o) -> bool {
        std::string nh = std::string(name) + ".hi", nl = std::string(name) + ".lo";
        o->hi = phx_ws(ctx, nh.c_str(), bytes);
        o->lo = planes == 2 ? phx_ws(ctx, nl.c_str(), bytes) : nullptr;
        return o->hi && (planes == 1 || o->lo);
    };
    b->m2_bytes = bm2;
    if (!get("tc.W", bw, &b->W) || !get("tc.M", bm, &b->M) || !get("tc.X", bx, &b->X) || !get("tc.E", be, &b->E) ||
        !get("tc.P", bp, &b->P) || !get("tc.T", bt, &b->T) || (bm2 > 0 && !get("tc.M2", bm2, &b->M2)))
        return PHX_ERR_NOMEM;
    b->qp = (int32_t*)phx_ws(ctx, "tc.qp", (size_t)max_nq * 8);      // two lists (by q parity)
    b->qpp = (int32_t*)phx_ws(ctx, "tc.qpp", (size_t)max_nq * 8);
    b->wph = (float2*)phx_ws(ctx, "tc.wph", (size_t)std::max<int64_t>(max_nnz, 1) * sizeof(float2));
    b->eqf = (float2*)phx_ws(ctx, "tc.eqf", (size_t)max_n2 * sizeof(float2));
    if (!b->qp || !b->qpp || !b->wph || !b->eqf) return PHX_ERR_NOMEM;
    return PHX_OK;
}

// Side stream and events of the tensor-core path (created once per context, outside any capture).
phx_status ensure_side(phx_ctx* ctx) {
    if (ctx->side_stream) return PHX_OK;
    PHX_CUDA_CHECK(ctx, cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ctx->side_ev) PHX_CUDA_CHECK(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return PHX_OK;
}

// SMs given to the side stream: the option, else PHX_SIDE_SMS, else 48 of 152 (measured at
// fcc32 8^3: 24 / 32 / 40 / 48 side SMs give 713 / 556 / 464 / 412 ms per step against 441 ms
// on one stream; the fold and Fourier GEMM of a tile then take about as long on 48 SMs as
// the chained kernel on the other 104).
// The scattering-row (Gamma1) and multi-temperature epilogues make the contractions longer
// for the same side-stream work, so their default share is smaller (`mode`: CHAIN_G, CHAIN_GT,
// CHAIN_GS; the environment variable PHX_SIDE_SMS_GT / PHX_SIDE_SMS_GS overrides those).
// Measured at fcc32 8^3: the Gamma1 pass 610 / 524 / 533 / 561 ms per step at 28 / 34 / 40 /
// 48 side SMs; four temperatures in one pass 519 / 530 / 570 ms at 32 / 40 / 48.
int side_sms(const phx_ctx* ctx, int sms, int mode = 0) {
    int v = ctx->opt_side_sms;
    if (v < 0) {
        const int base = mode == 2 ? 34 : mode == 1 ? 32 : 48;
        v = base * sms / 152;
        const char* env = getenv(mode == 2 ? "PHX_SIDE_SMS_GS" : mode == 1 ? "PHX_SIDE_SMS_GT" : "PHX_SIDE_SMS");
        if (!env) env = getenv("PHX_SIDE_SMS");
        if (env) v = atoi(env);
    }
    return std::max(0, std::min(v, sms / 2));
}

// Enqueue the whole linewidth computation of one job on `s` (kernel launches and memsets
// only, so it can be captured into a graph).  gacc/wacc: [n_irr][n] accumulators, zeroed.
// n_t > 0: the multi-temperature epilogue for n_t <= kMaxT occupation tables nb_stride apart,
// accumulating into n_t linewidth arrays t_stride apart (wacc unused).
template <int PREC>
phx_status tc_enqueue(phx_ctx* ctx, const TcPlan& P, const phx_fc3* f, const TcBuffers& B, const double* freq,
                      const double* evec, const double* nB, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                      double* gacc, double* wacc, cudaStream_t s, int n_t = 0, int64_t nb_stride = 0,
                      int64_t t_stride = 0, const G1Target* g1 = nullptr) {
    const int n = P.n, nq = P.nq, kr = P.kr, kcp = P.kcp, kr_d = P.kr_d, kcp_d = P.kcp_d;
    const int np = P.np, mg = P.mg, Q = P.Q, qp_np = P.qp_np, n_nu = P.n_nu;
    const int64_t n2 = (int64_t)n * n;
    const int esz = PREC == P_BF16X3 ? 2 : 4;
    const int planes = PREC == P_BF16X3 ? 2 : 1;
    if (!get_encoder()) return phx_set_error(ctx, PHX_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    // padding columns of M, X and W must read as zero for this job's layout
    for (int pl = 0; pl < planes; ++pl) {
        PHX_CUDA_CHECK(ctx, cudaMemsetAsync(pl ? B.M.lo : B.M.hi, 0, P.bytes_m, s));
        if (!P.chain) PHX_CUDA_CHECK(ctx, cudaMemsetAsync(pl ? B.X.lo : B.X.hi, 0, P.bytes_m, s));
        if (B.m2_bytes >= P.bytes_m) PHX_CUDA_CHECK(ctx, cudaMemsetAsync(pl ? B.M2.lo : B.M2.hi, 0, P.bytes_m, s));
        PHX_CUDA_CHECK(ctx, cudaMemsetAsync(pl ? B.W.lo : B.W.hi, 0, P.bytes_w, s));
    }
    if (P.chain)
        prep_evec_rows<PREC><<<2048, 256, 0, s>>>((const double2*)evec, nq, n, kcp, B.T.hi, B.T.lo);
    else
        prep_evec_tables<PREC><<<2048, 256, 0, s>>>((const double2*)evec, nq, n, np, kcp, B.E.hi, B.E.lo);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 1;
    const bool pair = ctx->opt_pair != 0;

    TcArgs aD{}, aA{}, aB{};
    ChainArgs aC{};
    CUtensorMap m_map2[2];          // M maps of the second buffer (chained kernel / EPI_X operand A)
    const int64_t m_rows = (int64_t)Q * P.rows_a;
    for (int pl = 0; pl < planes; ++pl) {
        const void* w = pl ? B.W.lo : B.W.hi;
        const void* m = pl ? B.M.lo : B.M.hi;
        const void* ph = pl ? B.P.lo : B.P.hi;
        bool ok = make_map(&aD.a_map[pl], w, PREC, P.rows_w, kr_d, kBoxRows) &&
                  make_map(&aD.b_map[pl], ph, PREC, (int64_t)P.n_tiles_q * 2 * qp_np, kr_d, qp_np);
        if (P.chain) {
            const void* t = pl ? B.T.lo : B.T.hi;
            ok = ok && make_map(&aC.ta_map[pl], t, PREC, (int64_t)nq * n, kr, P.c_ra) &&
                 make_map(&aC.tb_map[pl], t, PREC, (int64_t)nq * n, kr, P.c_rb3) &&
                 make_map(&aC.m_map[pl], m, PREC, m_rows, kr, kcp);
            if (B.m2_bytes >= P.bytes_m) ok = ok && make_map(&m_map2[pl], pl ? B.M2.lo : B.M2.hi, PREC, m_rows, kr, kcp);
        } else {
            const void* x = pl ? B.X.lo : B.X.hi;
            const void* e = pl ? B.E.lo : B.E.hi;
            ok = ok && make_map(&aA.a_map[pl], m, PREC, m_rows, kr, kBoxRows) &&
                 make_map(&aA.b_map[pl], e, PREC, (int64_t)nq * 2 * np, kr, mg) &&
                 (B.m2_bytes < P.bytes_m || make_map(&m_map2[pl], pl ? B.M2.lo : B.M2.hi, PREC, m_rows, kr, kBoxRows)) &&
                 make_map(&aB.a_map[pl], x, PREC, m_rows, kr, kBoxRows) &&
                 make_map(&aB.b_map[pl], e, PREC, (int64_t)nq * 2 * np, kr, mg);
        }
        if (!ok) return phx_set_error(ctx, PHX_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
    const unsigned long long wait_ns = ctx->opt_wait_ns;
    const int starve = ctx->opt_starve;
    aD.wait_ns = aA.wait_ns = aB.wait_ns = aC.wait_ns = wait_ns;
    aD.starve = aA.starve = aB.starve = aC.starve = starve;
    if (P.chain) {
        aC.n = n; aC.kcp = kcp; aC.nkc = P.nk; aC.ra = P.c_ra; aC.rb3 = P.c_rb3; aC.stages = P.c_stages;
        aC.freq = freq; aC.nB = nB;
        aC.sigma = (float)gp.sigma; aC.window = (float)gp.window; aC.f_min = (float)gp.f_min; aC.shape = gp.shape;
        aC.status = (int32_t*)ctx->status_word;
        aC.n_t = n_t; aC.nb_stride = nb_stride; aC.t_stride = t_stride;
        if (g1) {
            aC.g1 = (float*)g1->mat; aC.g1_ld = g1->ld; aC.tr_code = g1->tr_code; aC.g1_scale = (float)g1->scale;
            aC.g1_rows = (int64_t)n_irr * n;
            aC.lam = g1->lam; aC.ylam = g1->y;
        }
    }
    const bool g1_apply = g1 && g1->lam;
    const int chain_mode = n_t > 0 ? CHAIN_GT : (g1 ? (g1_apply ? CHAIN_GL : CHAIN_GS) : CHAIN_G);
    aD.np = qp_np; aD.mg = qp_np; aD.n_groups = 1; aD.nk = P.nk_d; aD.stages = P.st_d;
    aD.n_acc = (4 * qp_np <= 512) ? 2 : 1;
    aD.tmem_cols = tmem_cols_for(2 * qp_np, aD.n_acc);
    aD.a_rows_per_problem = 0; aD.b_idx = nullptr;
    aD.status = (int32_t*)ctx->status_word;
    aD.out_hi = B.M.hi; aD.out_lo = B.M.lo; aD.out_kr = kr; aD.out_kcp = kcp;
    aD.n = n;
    aA.np = np; aA.mg = mg; aA.n_groups = P.n_groups; aA.nk = P.nk; aA.stages = P.st_e;
    aA.n_acc = (4 * mg <= 512) ? 2 : 1;
    aA.tmem_cols = tmem_cols_for(2 * mg, aA.n_acc);
    aA.status = aD.status;
    aA.out_hi = B.X.hi; aA.out_lo = B.X.lo; aA.out_kr = kr; aA.out_kcp = kcp;
    aA.n = n;
    aB.np = np; aB.mg = mg; aB.n_groups = P.n_groups; aB.nk = P.nk; aB.stages = P.st_e; aB.n_acc = aA.n_acc;
    aB.tmem_cols = aA.tmem_cols;
    aB.status = aD.status;
    aB.n = n; aB.freq = freq; aB.nB = nB;
    aB.m1 = f->mesh[0]; aB.m2 = f->mesh[1]; aB.m3 = f->mesh[2];
    aB.sigma = (float)gp.sigma; aB.window = (float)gp.window; aB.f_min = (float)gp.f_min; aB.shape = gp.shape;
    aB.n_t = n_t; aB.nb_stride = nb_stride; aB.t_stride = t_stride;
    if (g1) {
        aB.g1 = (float*)g1->mat; aB.g1_ld = g1->ld; aB.tr_code = g1->tr_code; aB.g1_scale = g1->scale;
        aB.g1_rows = (int64_t)n_irr * n;
        aB.lam = g1->lam; aB.ylam = g1->y;
    }

    // With a side stream: the per-q lists, the fold and the Fourier GEMM run on s2 over `side`
    // SMs, the contractions (chained kernel, or the e_q'' and e_q' GEMMs) on s over the others.
    // M alternates between two buffers by tile and the q' lists between two by q; events order
    // every producer before its consumer and every consumer before the producer that
    // overwrites its buffer.
    const int side = (ctx->side_stream && B.m2_bytes >= P.bytes_m)
                         ? (P.side >= 0 ? std::min(P.side, sms / 2)
                                        : side_sms(ctx, sms, n_t > 0 ? CHAIN_GT : (g1 ? CHAIN_GS : CHAIN_G)))
                         : 0;
    cudaStream_t s2 = side > 0 ? ctx->side_stream : s;
    cudaEvent_t* ev = ctx->side_ev;       // [0] fork, [1] join, [2..3] M ready, [4..5] M free, [6..7] lists free
    const int main_ctas = sms - side, side_ctas = side > 0 ? side : sms;
    if (side > 0) {
        PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[0], s));
        PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s2, ev[0], 0));
    }
    int64_t g = 0;                        // tiles enqueued so far
    for (int si = 0; si < n_irr; ++si) {
        const int iq = irr_host[si];
        const int k1 = iq / (f->mesh[1] * f->mesh[2]), k2 = (iq / f->mesh[2]) % f->mesh[1], k3 = iq % f->mesh[2];
        const int qb = side > 0 ? (si & 1) : 0;
        int32_t* qp_l = B.qp + (int64_t)qb * nq;
        int32_t* qpp_l = B.qpp + (int64_t)qb * nq;
        if (side > 0 && si >= 2) PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s2, ev[6 + qb], 0));
        // this q's q' list (exchange pairs) in tiles of at most Q, balanced, and their phase tables
        pair_list_kernel<<<1, 1024, 0, s2>>>(iq, f->mesh[0], f->mesh[1], f->mesh[2], pair ? 1 : 0, qp_l, qpp_l);
        const int count = pair_count(iq, f->mesh, pair);
        const int n_tq = (count + Q - 1) / Q, Qb = (count + n_tq - 1) / n_tq;
        prep_phase_tables<PREC><<<64, 256, 0, s2>>>(f->d_int, f->n_d, f->mesh[0], f->mesh[1], f->mesh[2], qp_l, count,
                                                    Qb, n_tq, qp_np, kcp_d, B.P.hi, B.P.lo);
        PHX_CUDA_CHECK(ctx, cudaGetLastError());
        ctx->launches += 2;
        const int pblocks = (int)std::min<int64_t>((f->nnz + n2 + 255) / 256, 4096);
        fold_phase_kernel<<<pblocks, 256, 0, s2>>>(f->tc_ent_src, f->ent_r2, f->ent_w, f->nnz, (double)k1 / f->mesh[0],
                                                   (double)k2 / f->mesh[1], (double)k3 / f->mesh[2], B.wph,
                                                   (const double2*)evec + (int64_t)iq * n2, (int)n2, B.eqf);
        PHX_CUDA_CHECK(ctx, cudaGetLastError());
        ctx->launches += 2;
        aB.iq = iq;
        aB.gacc = gacc + (int64_t)si * n;
        aB.wacc = wacc ? wacc + (int64_t)si * n : nullptr;
        aC.iq = iq; aC.gacc = aB.gacc; aC.wacc = aB.wacc;
        for (int nu0 = 0; nu0 < n; nu0 += n_nu) {
            const int nnu = std::min(n_nu, n - nu0);
            const int64_t rw = (int64_t)nnu * n2, ra = (int64_t)nnu * n;
            {
                const int pf = phx_prof_begin(ctx, s2);
                const int64_t items = n2 * ((nnu + 31) / 32);
                // e_q in shared memory beside 16 warps' tiles when it fits (one CTA per SM), else
                // 8 warps per CTA and three CTAs per SM
                const bool eq_smem = 16 * kFoldTile + (size_t)n2 * sizeof(float2) <= kFoldSmemMax;
                const int fw = eq_smem ? 16 : 8, per_sm = eq_smem ? 1 : 3;
                const size_t fsmem = fw * kFoldTile + (eq_smem ? (size_t)n2 * sizeof(float2) : 0);
                const int blocks = (int)std::min<int64_t>((items + fw - 1) / fw, (int64_t)side_ctas * per_sm);
                static bool fold_attr = false;
                if (!fold_attr) {
                    PHX_CUDA_CHECK(ctx, cudaFuncSetAttribute(fold_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                             (int)kFoldSmemMax));
                    fold_attr = true;
                }
                fold_tc_kernel<PREC><<<blocks, 32 * fw, fsmem, s2>>>(f->tc_bc_start, f->tc_ent_ad, B.wph, B.eqf, n, nu0,
                                                                    nnu, kcp_d, eq_smem ? 1 : 0, B.W.hi, B.W.lo);
                PHX_CUDA_CHECK(ctx, cudaGetLastError());
                phx_prof_end(ctx, pf, s2, PHX_K_FOLD, 8.0 * (double)f->nnz * nnu, (double)rw * kr_d * esz * planes);
                ctx->launches += 1;
            }
            aD.rows = (int)rw; aD.tiles = (int)((rw + kBoxRows - 1) / kBoxRows);
            aD.out_rows_per_slot = (int)ra;
            aA.rows = (int)ra; aA.tiles = (int)((ra + kBoxRows - 1) / kBoxRows);
            aA.a_rows_per_problem = (int)ra; aA.out_rows_per_slot = (int)ra;
            aB.rows = (int)ra; aB.tiles = aA.tiles; aB.a_rows_per_problem = (int)ra;
            aB.nu0 = nu0;
            aB.g1_row0 = (int64_t)si * n + nu0;
            for (int tq = 0; tq < n_tq; ++tq, ++g) {
                const int t0 = tq * Qb, Qt = std::min(Qb, count - t0);
                const int mb = side > 0 ? (int)(g & 1) : 0;
                aD.b_base = tq;
                aD.nq_slots = Qt;
                aD.out_hi = mb ? B.M2.hi : B.M.hi;
                aD.out_lo = mb ? B.M2.lo : B.M.lo;
                // algorithmic work: complex MACs x 8 flops; bytes: operands read + results written once
                const double fl_d = 8.0 * (double)rw * Qt * f->n_d;
                const double fl_e = 8.0 * (double)Qt * ra * n * n;
                const double op_bytes = (double)planes * esz * 2.0;   // one complex value of an operand
                if (side > 0 && g >= 2) PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s2, ev[4 + mb], 0));
                int pp = phx_prof_begin(ctx, s2);
                PHX_CUDA_CHECK(ctx, (launch_gemm<PREC, EPI_M, false>(ctx, aD, 1, side_ctas, s2)));
                phx_prof_end(ctx, pp, s2, PHX_K_DFT, fl_d, op_bytes * ((double)rw * f->n_d + (double)Qt * ra * n));
                if (side > 0) {
                    PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[2 + mb], s2));
                    PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s, ev[2 + mb], 0));
                }
                if (P.chain) {
                    aC.n_items = Qt * nnu; aC.nnu = nnu; aC.rows_per_slot = (int)ra;
                    aC.qp = qp_l + t0; aC.qpp = qpp_l + t0; aC.pair = pair ? 1 : 0; aC.nu0 = nu0;
                    aC.g1_row0 = (int64_t)si * n + nu0;
                    ChainArgs ac = aC;
                    if (mb) { ac.m_map[0] = m_map2[0]; ac.m_map[1] = m_map2[1]; }
                    pp = phx_prof_begin(ctx, s);
                    PHX_CUDA_CHECK(ctx, launch_chain_mode<PREC>(ac, chain_mode, P.c_smem, main_ctas, s));
                    // two contractions; bytes: the M operand read once
                    phx_prof_end(ctx, pp, s, PHX_K_CHAIN, 2.0 * fl_e, op_bytes * (double)Qt * ra * n);
                    if (side > 0) PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[4 + mb], s));
                    ctx->launches += 2;
                    continue;
                }
                aA.b_idx = qpp_l + t0;
                TcArgs aa = aA;
                if (mb) { aa.a_map[0] = m_map2[0]; aa.a_map[1] = m_map2[1]; }
                pp = phx_prof_begin(ctx, s);
                PHX_CUDA_CHECK(ctx, (launch_gemm_any<PREC, EPI_X>(ctx, aa, P.stream_b, Qt, main_ctas, s)));
                phx_prof_end(ctx, pp, s, PHX_K_GEMM_E2, fl_e, op_bytes * 2.0 * Qt * ra * n);
                if (side > 0) PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[4 + mb], s));   // M[mb] read
                aB.b_idx = qp_l + t0;
                aB.qp1 = qp_l + t0;
                aB.pair = pair ? 1 : 0;
                pp = phx_prof_begin(ctx, s);
                if (n_t > 0)
                    PHX_CUDA_CHECK(ctx, (launch_gemm_any<PREC, EPI_GT>(ctx, aB, P.stream_b, Qt, main_ctas, s)));
                else if (g1_apply)
                    PHX_CUDA_CHECK(ctx, (launch_gemm_any<PREC, EPI_GL>(ctx, aB, P.stream_b, Qt, main_ctas, s)));
                else if (g1)
                    PHX_CUDA_CHECK(ctx, (launch_gemm_any<PREC, EPI_GS>(ctx, aB, P.stream_b, Qt, main_ctas, s)));
                else
                    PHX_CUDA_CHECK(ctx, (launch_gemm_any<PREC, EPI_G>(ctx, aB, P.stream_b, Qt, main_ctas, s)));
                phx_prof_end(ctx, pp, s, PHX_K_GEMM_E1, fl_e, op_bytes * (double)Qt * ra * n);
                ctx->launches += 3;
            }
        }
        if (side > 0) PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[6 + qb], s));
    }
    if (side > 0) {
        PHX_CUDA_CHECK(ctx, cudaEventRecord(ev[1], s2));
        PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(s, ev[1], 0));
    }
    return PHX_OK;
}

template <int PREC>
phx_status run_tc(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec, const double* nB,
                  const int32_t* irr_host, int n_irr, const GammaParams& gp, double* gacc, double* wacc,
                  cudaStream_t s, int n_t = 0, int64_t nb_stride = 0, int64_t t_stride = 0,
                  const G1Target* g1 = nullptr) {
    TcPlan P;
    PHX_TRY(tc_plan(ctx, f, PREC, 0, &P));
    PHX_TRY(tc_prepare_fc3(ctx, const_cast<phx_fc3*>(f)));
    TcBuffers B;
    const bool two_m = side_sms(ctx, ctx->sm_count > 0 ? ctx->sm_count : 148) > 0;
    if (two_m) PHX_TRY(ensure_side(ctx));
    PHX_TRY(tc_alloc(ctx, PREC, P.bytes_w, P.bytes_m, P.chain ? 0 : P.bytes_m, P.bytes_e, P.bytes_p, P.bytes_t, P.nq,
                     f->nnz, (int64_t)P.n * P.n, &B, two_m ? P.bytes_m : 0));
    return tc_enqueue<PREC>(ctx, P, f, B, freq, evec, nB, irr_host, n_irr, gp, gacc, wacc, s, n_t, nb_stride,
                            t_stride, g1);
}

}  // namespace

int phx_side_sms(const phx_ctx* ctx) { return side_sms(ctx, ctx->sm_count > 0 ? ctx->sm_count : 148); }

phx_status phx_gamma_tc(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec, const double* nB,
                        const int32_t* irr_host, int n_irr, const GammaParams& gp, int prec, double* gacc,
                        double* wacc, cudaStream_t s, const G1Target* g1) {
    if (ctx->cc_major != 10)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path needs a Blackwell (sm_10x) device");
    if (g1 && wacc) return phx_set_error(ctx, PHX_ERR_INVALID, "scattering rows and WP2 in one pass");
    if (prec == PHX_BF16X3) return run_tc<P_BF16X3>(ctx, f, freq, evec, nB, irr_host, n_irr, gp, gacc, wacc, s, 0, 0, 0, g1);
    return run_tc<P_TF32>(ctx, f, freq, evec, nB, irr_host, n_irr, gp, gacc, wacc, s, 0, 0, 0, g1);
}

phx_status phx_gamma_tc_multi_t(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                                const double* nB, int n_t, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                                int prec, double* gacc, cudaStream_t s) {
    if (ctx->cc_major != 10)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path needs a Blackwell (sm_10x) device");
    if (n_t < 1 || n_t > kMaxT) return phx_set_error(ctx, PHX_ERR_INVALID, "multi-temperature pass of %d", n_t);
    const int64_t nb_stride = (int64_t)f->nq * f->n, t_stride = (int64_t)n_irr * f->n;
    if (prec == PHX_BF16X3)
        return run_tc<P_BF16X3>(ctx, f, freq, evec, nB, irr_host, n_irr, gp, gacc, nullptr, s, n_t, nb_stride, t_stride);
    return run_tc<P_TF32>(ctx, f, freq, evec, nB, irr_host, n_irr, gp, gacc, nullptr, s, n_t, nb_stride, t_stride);
}

// ---------------------------------------------------------------- batched jobs (one CUDA graph)

namespace {

// Best (q' tile, contraction kernel, side-stream share) of a job class, timed on up to three
// irreducible q-points of the job (the side stream overlaps the next q-point's fold and Fourier
// GEMM with this one's contractions, which a single q-point does not show; best of two runs
// per candidate): every tile 8..128 with the two GEMMs and, where it fits, with the chained
// kernel, at the context's side share; then the side share for the fastest pair (0, 24, 32,
// 40, 48, 56 of 152 SMs, scaled to the device) unless the context fixes it.
template <int PREC>
phx_status autotune_q(phx_ctx* ctx, const phx_job& job, cudaStream_t s, int* best_q, int* best_chain,
                      int* best_side) {
    const phx_fc3* f = job.fc3;
    const int n_time = std::min(job.n_irr, 3);
    const int32_t* iq = job.irr_q;
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
    GammaParams gp{};
    gp.n = f->n; gp.nq = f->nq; gp.T = job.temperature; gp.shape = job.br.shape; gp.sigma = job.br.sigma_thz;
    gp.window = job.br.window; gp.f_min = job.f_min_thz;
    double* nB = (double*)phx_ws(ctx, "b.nB", (size_t)f->nq * f->n * 8);
    double* gacc = (double*)phx_ws(ctx, "b.gacc", (size_t)n_time * f->n * 8);
    if (!nB || !gacc) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, phx_launch_occupations(job.freq_thz, f->nq * f->n, job.temperature, 0, nB, nullptr, s));
    auto time_plan = [&](const TcPlan& P, float* out_ms) -> phx_status {
        const int side = P.side >= 0 ? P.side : side_sms(ctx, sms);
        TcBuffers B;
        if (side > 0) PHX_TRY(ensure_side(ctx));
        PHX_TRY(tc_alloc(ctx, PREC, P.bytes_w, P.bytes_m, P.chain ? 0 : P.bytes_m, P.bytes_e, P.bytes_p, P.bytes_t,
                         P.nq, f->nnz, (int64_t)P.n * P.n, &B, side > 0 ? P.bytes_m : 0));
        float best_rep = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0.f;
            PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_in, s));
            PHX_TRY(tc_enqueue<PREC>(ctx, P, f, B, job.freq_thz, job.evec, nB, iq, n_time, gp, gacc, nullptr, s));
            PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_out, s));
            PHX_CUDA_CHECK(ctx, cudaEventSynchronize(ctx->ev_out));
            PHX_CUDA_CHECK(ctx, cudaEventElapsedTime(&ms, ctx->ev_in, ctx->ev_out));
            best_rep = std::min(best_rep, ms);
        }
        *out_ms = best_rep;
        return PHX_OK;
    };
    float best_ms = 1e30f;
    TcPlan best{};
    *best_q = 0;
    *best_chain = 0;
    *best_side = -1;
    for (int chain = 0; chain < 2; ++chain) {
        int last_q = -1;
        for (int cand : {8, 16, 32, 64, 128}) {
            TcPlan P;
            if (tc_plan(ctx, f, PREC, cand, &P, chain) != PHX_OK) continue;
            if (P.chain != (chain == 1)) break;          // the chained kernel does not fit this class
            if (P.Q == last_q) continue;                 // clamped to the mesh size already tried
            last_q = P.Q;
            float ms = 0.f;
            PHX_TRY(time_plan(P, &ms));
            if (ms < best_ms) { best_ms = ms; best = P; *best_q = P.Q; *best_chain = chain; }
        }
    }
    if (*best_q == 0) return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "autotune: no q' tile fits");
    if (ctx->opt_side_sms < 0) {
        const int dflt = side_sms(ctx, sms);
        int chosen = dflt;
        for (int base : {0, 24, 32, 40, 48, 56}) {
            const int cand = std::min(base * sms / 152, sms / 2);
            if (cand == dflt) continue;                  // timed above
            TcPlan P = best;
            P.side = cand;
            float ms = 0.f;
            PHX_TRY(time_plan(P, &ms));
            if (ms < best_ms) { best_ms = ms; chosen = cand; }
        }
        *best_side = chosen;
    }
    return PHX_OK;
}

template <int PREC>
phx_status run_batched(phx_ctx* ctx, int n_jobs, const phx_job* jobs, phx_tune* tune, cudaStream_t user) {
    if (!ctx->cap_stream) {
        PHX_CUDA_CHECK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        PHX_CUDA_CHECK(ctx, cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDefault));
        PHX_CUDA_CHECK(ctx, cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDefault));
    }
    cudaStream_t cs = ctx->cap_stream;
    // the batch starts after the work already queued on the caller's stream
    PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_in, user));
    PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(cs, ctx->ev_in, 0));

    // plans (q' tile from the caller, the autotune table, or a fresh tuning run)
    std::vector<TcPlan> plans(n_jobs);
    std::vector<int> qtiles(n_jobs, 0), chains(n_jobs, -1), sides(n_jobs, -1);
    for (int j = 0; j < n_jobs; ++j) {
        const phx_job& jb = jobs[j];
        PHX_TRY(tc_prepare_fc3(ctx, const_cast<phx_fc3*>(jb.fc3)));
        const bool given = tune && tune[j].q_tile > 0;
        int q = given ? tune[j].q_tile : 0;
        int ch = given ? tune[j].chain : -1;
        int sd = given ? tune[j].side_sms : -1;
        if (q == 0) {
            const std::vector<int> key = {PREC, jb.fc3->n, jb.fc3->mesh[0], jb.fc3->mesh[1], jb.fc3->mesh[2],
                                          jb.fc3->n_d, ctx->opt_side_sms};
            auto it = ctx->tune_q.find(key);
            if (it == ctx->tune_q.end()) {
                PHX_TRY(autotune_q<PREC>(ctx, jb, cs, &q, &ch, &sd));
                ctx->tune_q[key] = {q, ch, sd};
            } else {
                q = it->second[0];
                ch = it->second[1];
                sd = it->second[2];
            }
            if (tune) { tune[j].q_tile = q; tune[j].chain = ch; tune[j].side_sms = sd; }
        }
        qtiles[j] = q;
        chains[j] = ch;
        sides[j] = sd;
        PHX_TRY(tc_plan(ctx, jb.fc3, PREC, q, &plans[j], ch));
        plans[j].side = sd;
    }
    // workspace for the largest job, allocated before any capture (as are the side stream and its
    // events: chained jobs then keep a second M buffer in the X workspace)
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
    int side = 0;
    for (int j = 0; j < n_jobs; ++j) side = std::max(side, sides[j] >= 0 ? std::min(sides[j], sms / 2) : side_sms(ctx, sms));
    if (side > 0) PHX_TRY(ensure_side(ctx));
    size_t bw = 0, bm = 0, bx = 0, be = 0, bp = 0, bt = 0;
    int64_t mnq = 1, mnnz = 1, mn2 = 1, mnb = 1, mg = 1;
    for (int j = 0; j < n_jobs; ++j) {
        const TcPlan& P = plans[j];
        bw = std::max(bw, P.bytes_w); bm = std::max(bm, P.bytes_m); be = std::max(be, P.bytes_e);
        bp = std::max(bp, P.bytes_p); bt = std::max(bt, P.bytes_t);
        if (!P.chain) bx = std::max(bx, P.bytes_m);
        mnq = std::max<int64_t>(mnq, P.nq); mnnz = std::max<int64_t>(mnnz, jobs[j].fc3->nnz);
        mn2 = std::max<int64_t>(mn2, (int64_t)P.n * P.n);
        mnb = std::max<int64_t>(mnb, (int64_t)P.nq * P.n);
        mg = std::max<int64_t>(mg, (int64_t)jobs[j].n_irr * P.n);
    }
    TcBuffers B;
    PHX_TRY(tc_alloc(ctx, PREC, bw, bm, bx, be, bp, bt, mnq, mnnz, mn2, &B, side > 0 ? bm : 0));
    double* nB = (double*)phx_ws(ctx, "b.nB", (size_t)mnb * 8);
    double* gacc = (double*)phx_ws(ctx, "b.gacc", (size_t)mg * 8);
    double* acc9 = (double*)phx_ws(ctx, "b.acc9", (size_t)n_jobs * 9 * 8);
    if (!nB || !gacc || !acc9) return PHX_ERR_NOMEM;

    // graph key: the job list, the precision, the pair option and the tiles
    std::vector<uint8_t> key(sizeof(phx_job) * n_jobs + sizeof(int) * (3 * n_jobs + 2));
    uint8_t* kp = key.data();
    std::memcpy(kp, jobs, sizeof(phx_job) * n_jobs);
    kp += sizeof(phx_job) * n_jobs;
    std::memcpy(kp, qtiles.data(), sizeof(int) * n_jobs);
    kp += sizeof(int) * n_jobs;
    std::memcpy(kp, chains.data(), sizeof(int) * n_jobs);
    kp += sizeof(int) * n_jobs;
    std::memcpy(kp, sides.data(), sizeof(int) * n_jobs);
    kp += sizeof(int) * n_jobs;
    // the pair and side-stream options change the launches
    const int opts[2] = {PREC + 16 * ctx->opt_pair, side_sms(ctx, sms)};
    std::memcpy(kp, opts, sizeof(opts));
    // host irr lists are part of the key by content
    for (int j = 0; j < n_jobs; ++j) {
        const uint8_t* b = (const uint8_t*)jobs[j].irr_q;
        key.insert(key.end(), b, b + sizeof(int32_t) * jobs[j].n_irr);
    }
    if (!ctx->graph_exec || key != ctx->graph_key) {
        if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
        const bool prof = ctx->prof;
        ctx->prof = false;                     // event records are not captured
        const int64_t l0 = ctx->launches;
        PHX_CUDA_CHECK(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        phx_status st = PHX_OK;
        for (int j = 0; j < n_jobs && st == PHX_OK; ++j) {
            const phx_job& jb = jobs[j];
            const TcPlan& P = plans[j];
            const phx_fc3* f = jb.fc3;
            GammaParams gp{};
            gp.n = f->n; gp.nq = f->nq; gp.T = jb.temperature; gp.shape = jb.br.shape; gp.sigma = jb.br.sigma_thz;
            gp.window = jb.br.window; gp.f_min = jb.f_min_thz;
            if (phx_launch_occupations(jb.freq_thz, f->nq * f->n, jb.temperature, 0, nB, nullptr, cs) != cudaSuccess ||
                cudaMemsetAsync(gacc, 0, (size_t)jb.n_irr * f->n * 8, cs) != cudaSuccess) {
                st = phx_set_error(ctx, PHX_ERR_CUDA, "batched: launch failed during capture");
                break;
            }
            ctx->launches += 1;
            st = tc_enqueue<PREC>(ctx, P, f, B, jb.freq_thz, jb.evec, nB, jb.irr_q, jb.n_irr, gp, gacc, nullptr, cs);
            if (st != PHX_OK) break;
            const double conv = phx::kEvA2AmuToPs2;
            const double pref = phx::kPi * phx::kHbarEvPs * conv * conv * conv / (8.0 * f->nq);
            // the irreducible list also has to be on the device for the finalize kernel
            const int32_t* irr_dev = jb.irr_q_dev;
            if (!irr_dev) { st = phx_set_error(ctx, PHX_ERR_INVALID, "batched: job %d has no irr_q_dev", j); break; }
            if (phx_launch_finalize(jb.n_irr * f->n, f->n, irr_dev, jb.freq_thz, gacc, nullptr, pref, 1.0 / f->nq,
                                    jb.f_min_thz, jb.gamma, nullptr, cs) != cudaSuccess) {
                st = phx_set_error(ctx, PHX_ERR_CUDA, "batched: finalize launch failed");
                break;
            }
            ctx->launches += 1;
            if (jb.vv) {
                double* a9 = acc9 + 9 * j;
                if (phx_launch_unfold(jb.n_irr, f->nq, f->n, jb.freq_thz, irr_dev, jb.gamma, jb.full_to_irr,
                                      jb.gamma_full, cs) != cudaSuccess ||
                    cudaMemsetAsync(a9, 0, 72, cs) != cudaSuccess ||
                    phx_launch_kappa(f->nq, f->n, jb.freq_thz, nullptr, jb.vv, jb.gamma_full, jb.temperature,
                                     jb.f_min_thz, 0, a9, cs) != cudaSuccess ||
                    phx_launch_scale9(a9, phx::kEvPsAKToWmK / ((double)f->nq * jb.volume), jb.kappa, cs) !=
                        cudaSuccess) {
                    st = phx_set_error(ctx, PHX_ERR_CUDA, "batched: conductivity launch failed");
                    break;
                }
                ctx->launches += 3;
            }
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        ctx->prof = prof;
        if (st != PHX_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (ec != cudaSuccess) return phx_set_error(ctx, PHX_ERR_CUDA, "batched: capture failed: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->graph_exec = nullptr;
            return phx_set_error(ctx, PHX_ERR_CUDA, "batched: instantiate failed: %s", cudaGetErrorString(ei));
        }
        ctx->graph_key = key;
        ctx->graph_launches = ctx->launches - l0;
        ctx->launches = l0;
    }
    PHX_CUDA_CHECK(ctx, cudaGraphLaunch(ctx->graph_exec, cs));
    ctx->launches += ctx->graph_launches;
    PHX_CUDA_CHECK(ctx, cudaEventRecord(ctx->ev_out, cs));
    PHX_CUDA_CHECK(ctx, cudaStreamWaitEvent(user, ctx->ev_out, 0));
    return PHX_OK;
}

}  // namespace

extern "C" phx_status phx_gamma_batched(phx_ctx* ctx, int32_t n_jobs, const phx_job* jobs, int32_t prec,
                                        phx_tune* tune, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_batched: bad job list");
    if (n_jobs == 0) return PHX_OK;
    if (prec != PHX_BF16X3 && prec != PHX_TF32)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_gamma_batched: tensor-core precisions only");
    if (ctx->cc_major != 10)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "tensor-core path needs a Blackwell (sm_10x) device");
    for (int j = 0; j < n_jobs; ++j) {
        const phx_job& jb = jobs[j];
        if (!jb.fc3 || jb.fc3->ctx != ctx || !jb.freq_thz || !jb.evec || !jb.gamma || jb.n_irr <= 0 || !jb.irr_q ||
            !jb.irr_q_dev)
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_batched: job %d incomplete", j);
        if (!(jb.temperature > 0.0) || !(jb.br.sigma_thz > 0.0) || !(jb.br.window > 0.0) || !(jb.f_min_thz > 0.0) ||
            (jb.br.shape != PHX_GAUSS && jb.br.shape != PHX_LORENTZ))
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_batched: job %d parameters", j);
        for (int i = 0; i < jb.n_irr; ++i)
            if (jb.irr_q[i] < 0 || jb.irr_q[i] >= jb.fc3->nq)
                return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_batched: job %d irr_q[%d] outside the mesh", j, i);
        if (jb.vv && (!jb.full_to_irr || !jb.gamma_full || !jb.kappa || !(jb.volume > 0.0)))
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_batched: job %d conductivity arguments", j);
    }
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == PHX_BF16X3) return run_batched<P_BF16X3>(ctx, n_jobs, jobs, tune, s);
    return run_batched<P_TF32>(ctx, n_jobs, jobs, tune, s);
}
