// Chained eigenvector contractions of the linewidth path (paper Sec. "Three-Phonon Scattering",
// Eq. (phi3_proj): the projection as "two ... tensor multiplications", Sec. "Computational
// Implementation"), with the weighting of Eqs. (gamma), (broadening) fused behind them.  For
// one q' slot p and one band nu of q the kernel computes, without writing X to memory,
//
//   X^T[nu''][b]  = sum_c e_q''[c][nu''] M[(nu, b)][c]          (stage 2, accumulator D2)
//   V[nu''][nu']  = sum_b X^T[nu''][b] e_q'[b][nu']              (stage 3, accumulator D3)
//   gamma[nu]    += sum |V|^2 w(f, f', f'')                       (epilogue)
//
// Operands (real arithmetic on complex numbers, each complex K vector stored as one row
// [Re(0..kcp) | Im(0..kcp)]):
//   * eigenvector row table T[q][j] = [Re e_q(:, j) | Im e_q(:, j)] (one row per mode j).  Stage
//     2's A is T[q''] (rows nu'', resident in shared memory), stage 3's B is T[q'] (rows nu').
//   * stage 2's B is the block of M rows (nu, b), streamed by TMA in 128-byte K chunks.
//   * stage 3's A is X^T itself: the epilogue warps convert D2 in place in tensor memory to
//     the MMA operand format (bf16 hi/lo pairs or tf32) and the MMA reads A from tensor memory.
// A complex product is four real MMAs over the K halves, Re D = Re.Re - Im.Im (the second
// with the instruction's negate-A bit) and Im D = Re.Im + Im.Re; BF16x3 splits every
// operand into hi + lo and issues hi.hi + hi.lo + lo.hi.
//
// Rows of both stages are modes (nu'' in lane nu''), so an MMA's 128 rows hold n <= 96 of
// them and every MMA covers all partner modes at once (N = n rounded up to 16): an MMA
// instruction costs at least ~40 cycles to issue on GB300, so few wide MMAs beat many narrow
// ones even with one accumulator of each kind.
//
// Warp roles (the tensor-memory lane quarter of warp w is w % 4; quarter 3 holds no mode):
// warps 0-2, 4-6 and 8-10 (three per quarter) convert D2 and run the weighting epilogue on
// D3, warp 3 owns tensor memory and issues the MMAs, warp 7 issues TMA loads (tables per q'
// slot, M chunks per item), warp 11 idles.  Per item: stage 2 issues the Re-output MMAs, commits, then the Im-output MMAs, so
// the epilogue converts the Re half of X^T while the Im half accumulates; stage 3 consumes
// the two halves in K order; the weighting of item i overlaps stage 2 of item i + 1.
// Every wait is bounded.
#pragma once

struct ChainArgs {
    CUtensorMap ta_map[2];      // eigenvector row table planes, box = ra rows (stage 2 A)
    CUtensorMap tb_map[2];      // eigenvector row table planes, box = rb3 rows (stage 3 B)
    CUtensorMap m_map[2];       // M planes, box = kcp rows (stage 2 B)
    int n;                      // modes
    int kcp;                    // K half (multiple of 32); row = [Re (kcp) | Im (kcp)]
    int nkc;                    // 128-byte K chunks per operand row and plane
    int ra;                     // rows of the stage-2 A block in shared memory (n rounded to 8)
    int rb3;                    // rows of the stage-3 B block = partner modes per MMA (n rounded to 16)
    int stages;                 // M chunk ring: stages / nkc item slots of nkc chunks (>= 1)
    int n_items;                // q' slots x bands of this launch (slot-major)
    int nnu;                    // bands nu per slot
    int rows_per_slot;          // rows of M per q' slot
    const int32_t* qp;          // per slot: mesh index of q'
    const int32_t* qpp;         // per slot: mesh index of q''
    int pair;                   // nonzero: each q' stands for its exchange pair (q', q'')
    int nu0;                    // first band of the chunk
    int iq;
    const double* freq;
    const double* nB;
    float sigma, window, f_min;
    int shape;
    double* gacc;               // [n] of this irreducible q
    double* wacc;               // may be null
    int32_t* status;
    unsigned long long wait_ns; // bound of every barrier wait
    int starve;                 // test hook: the producer issues nothing (waits then run out)
    // CHAIN_GT: n_t temperatures (occupation tables nb_stride apart, accumulators t_stride apart)
    int n_t;
    int64_t nb_stride, t_stride;
    // CHAIN_GS: off-diagonal scattering rows of Eq. (gamma1), folded onto time-reversal
    // representatives (row g1_row0 + nu of this chunk; see G1Target)
    float* g1;
    int64_t g1_rows, g1_ld, g1_row0;
    const int32_t* tr_code;
    float g1_scale;
    // CHAIN_GL: the same rows applied to mean free paths, y[a][r] += sum_c Gamma1[r][c] lam[a][c]
    // (planes [3][g1_ld], FP64; rows and columns as CHAIN_GS)
    const double* lam;
    double* ylam;
};

// epilogue variants: linewidths (+ WP2), linewidths at several temperatures, linewidths plus
// the off-diagonal scattering rows, linewidths plus those rows applied to mean free paths
enum { CHAIN_G = 0, CHAIN_GT = 1, CHAIN_GS = 2, CHAIN_GL = 3 };

// 2^x by the special-function unit (approximate, flushes denormals; the weights use it on
// arguments <= 0 only)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kChainThreads = 384;
constexpr int kChainEpiParts = 3;                          // epilogue warps per tensor-memory lane quarter
constexpr int kChainEpiThreads = 32 * 3 * kChainEpiParts;  // warps 0-2, 4-6, 8-10
constexpr int kChainMmaWarp = 3, kChainTmaWarp = 7, kChainIdleWarp = 11;

template <int PREC, int MODE>
__global__ void __launch_bounds__(kChainThreads, 1) chain_kernel(const __grid_constant__ ChainArgs args) {
    constexpr int kPlanes = (PREC == P_BF16X3) ? 2 : 1;
    constexpr uint32_t kFmt = (PREC == P_BF16X3) ? 1u : 2u;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t a2_full, a2_empty, b3_full, b3_empty;
    __shared__ __align__(8) uint64_t d2_full[2], a3_ready[2], s3_done, d3_empty, drain_bar;
    __shared__ uint32_t tmem_base_slot;
    __shared__ volatile int abort_flag;
    __shared__ float4 s_tab[kMaxNp];       // per partner mode nu' at q': (f', n', 1/f' or 0, -)
    __shared__ float s_n1t[MODE == CHAIN_GT ? kMaxT : 1][MODE == CHAIN_GT ? kMaxNp : 1];
    // CHAIN_GS: per item (double-buffered) the Gamma1 column sums over nu'' (partners at q') and
    // the row sums over nu' (partners at q''), and the q'' frequencies of the slot
    __shared__ float s_col[MODE == CHAIN_GS ? 2 : 1][MODE == CHAIN_GS ? kMaxNp : 1];
    __shared__ float s_row[MODE == CHAIN_GS ? 2 : 1][MODE == CHAIN_GS ? kMaxNp : 1];
    __shared__ float s_f2[MODE == CHAIN_GS ? kMaxNp : 1];
    // CHAIN_GL: per partner mode nu' at q' the signed f' lambda(q', nu') of its column
    __shared__ float s_lam[MODE == CHAIN_GL ? 3 : 1][MODE == CHAIN_GL ? kMaxNp : 1];

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int n = args.n, kcp = args.kcp, nkc = args.nkc, ra = args.ra, rb3 = args.rb3;
    const int stages = args.stages, nnu = args.nnu;
    const uint32_t blk_a = (uint32_t)ra * kChunkBytes, blk_b = (uint32_t)rb3 * kChunkBytes;
    const uint32_t blk_m = (uint32_t)kcp * kChunkBytes;
    uint8_t* sA2 = smem;                                       // [plane][chunk][ra rows][128 B]
    uint8_t* sB3 = sA2 + (size_t)kPlanes * nkc * blk_a;        // [plane][chunk][rb3 rows][128 B]
    uint8_t* sB2 = sB3 + (size_t)kPlanes * nkc * blk_b;        // [slot][chunk][plane][kcp rows][128 B]
    const uint32_t stage_bytes = kPlanes * blk_m;
    const uint32_t slot_bytes = (uint32_t)nkc * stage_bytes;
    const int n_slots = stages / nkc;                          // items of M in flight
    const int hs = kcp * (PREC == P_BF16X3 ? 2 : 4) / 32;      // 32-byte K steps per half
    const uint64_t wl = args.wait_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item_begin = (int)((int64_t)args.n_items * blockIdx.x / gridDim.x);
    const int item_end = (int)((int64_t)args.n_items * (blockIdx.x + 1) / gridDim.x);
    const int L = item_end - item_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < n_slots; ++s) { tc::mbar_init(&full_bar[s], 1); tc::mbar_init(&empty_bar[s], 1); }
        tc::mbar_init(&a2_full, 1); tc::mbar_init(&a2_empty, 1);
        tc::mbar_init(&b3_full, 1); tc::mbar_init(&b3_empty, 1);
        for (int h = 0; h < 2; ++h) { tc::mbar_init(&d2_full[h], 1); tc::mbar_init(&a3_ready[h], kChainEpiThreads); }
        tc::mbar_init(&s3_done, 1); tc::mbar_init(&d3_empty, kChainEpiThreads);
        tc::mbar_init(&drain_bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == kChainTmaWarp && lane == 0) {
        for (int pl = 0; pl < kPlanes; ++pl) {
            tc::prefetch_tmap(&args.ta_map[pl]); tc::prefetch_tmap(&args.tb_map[pl]); tc::prefetch_tmap(&args.m_map[pl]);
        }
    }
    if (warp == kChainMmaWarp) tc::tmem_alloc(&tmem_base_slot, 512);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = tmem_base_slot;
    // tensor memory: D2 / stage-3 A at columns [0, 2 kcp), D3 = [Re (rb3) | Im (rb3)] after it
    const uint32_t d3_col0 = 2u * kcp;

    auto fail = [&]() {
        abort_flag = 1;
        atomicExch(args.status, (int)PHX_ERR_TIMEOUT);
    };

    if (warp == kChainTmaWarp) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0 && !args.starve && L > 0) {
            const int kelems = kChunkBytes / (PREC == P_BF16X3 ? 2 : 4);
            int stage = 0;
            uint32_t phase = 0;
            bool pending[kMaxStages];
            uint32_t pend_phase[kMaxStages];
            for (int s = 0; s < kMaxStages; ++s) { pending[s] = false; pend_phase[s] = 0; }
            bool a2_pend = false, b3_pend = false;
            uint32_t a2_pp = 0, b3_pp = 0;
            int n_a2 = 0, n_b3 = 0, cur_p = -1;
            bool ok = true;
            for (int li = 0; ok && li < L; ++li) {
                const int it = item_begin + li;
                const int p = it / nnu, nu = it % nnu;
                const bool new_p = p != cur_p;
                if (new_p) {
                    // stage-2 table of q'' once the previous slot's stage-2 MMAs are done
                    if (n_a2 > 0 && !tc::mbar_wait(&a2_empty, (n_a2 - 1) & 1, &abort_flag, wl)) { fail(); break; }
                    const int row = args.qpp[p] * n;
                    tc::mbar_expect_tx(&a2_full, kPlanes * nkc * blk_a);
                    for (int pl = 0; pl < kPlanes; ++pl)
                        for (int c = 0; c < nkc; ++c)
                            tc::tma_load_2d(sA2 + (size_t)(pl * nkc + c) * blk_a, &args.ta_map[pl], &a2_full, c * kelems, row);
                    a2_pend = true; a2_pp = n_a2 & 1;
                    ++n_a2;
                }
                const int mrow = p * args.rows_per_slot + nu * n;
                // every chunk of the item's M block into one slot (one barrier, one release)
                if (!tc::mbar_wait(&empty_bar[stage], phase ^ 1, &abort_flag, wl)) { fail(); break; }
                uint8_t* sl = sB2 + (size_t)stage * slot_bytes;
                tc::mbar_expect_tx(&full_bar[stage], slot_bytes);
                for (int c = 0; c < nkc; ++c)
                    for (int pl = 0; pl < kPlanes; ++pl)
                        tc::tma_load_2d(sl + (size_t)c * stage_bytes + (size_t)pl * blk_m, &args.m_map[pl], &full_bar[stage],
                                        c * kelems, mrow);
                pending[stage] = true; pend_phase[stage] = phase;
                if (++stage == n_slots) { stage = 0; phase ^= 1; }
                if (new_p) {
                    // stage-3 table of q' once the previous slot's stage-3 MMAs are done
                    if (n_b3 > 0 && !tc::mbar_wait(&b3_empty, (n_b3 - 1) & 1, &abort_flag, wl)) { fail(); break; }
                    const int row = args.qp[p] * n;
                    tc::mbar_expect_tx(&b3_full, kPlanes * nkc * blk_b);
                    for (int pl = 0; pl < kPlanes; ++pl)
                        for (int c = 0; c < nkc; ++c)
                            tc::tma_load_2d(sB3 + (size_t)(pl * nkc + c) * blk_b, &args.tb_map[pl], &b3_full, c * kelems, row);
                    b3_pend = true; b3_pp = n_b3 & 1;
                    ++n_b3;
                    cur_p = p;
                }
            }
            if (abort_flag) {
                // let loads already issued land before the CTA retires (bounded)
                for (int s = 0; s < n_slots; ++s)
                    if (pending[s]) {
                        const uint64_t t0 = tc::global_ns();
                        while (!tc::mbar_try_wait(&full_bar[s], pend_phase[s]) && tc::global_ns() - t0 < wl) {
                        }
                    }
                const uint64_t t0 = tc::global_ns();
                while (a2_pend && !tc::mbar_try_wait(&a2_full, a2_pp) && tc::global_ns() - t0 < wl) {
                }
                while (b3_pend && !tc::mbar_try_wait(&b3_full, b3_pp) && tc::global_ns() - t0 < wl) {
                }
            }
        }
    } else if (warp == kChainMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && L > 0) {
            // descriptors: start address >> 4 sits in the low bits, so an address offset is
            // added to a base descriptor as (offset >> 4) (all offsets stay inside the 256 KB window)
            const uint64_t a2d = tc::sdesc_sw128(tc::smem_u32(sA2)), b3d = tc::sdesc_sw128(tc::smem_u32(sB3));
            const uint64_t b2d = tc::sdesc_sw128(tc::smem_u32(sB2));
            const uint32_t a_lo = (uint32_t)(nkc * blk_a) >> 4, b3_lo = (uint32_t)(nkc * blk_b) >> 4;
            const uint32_t m_lo = blk_m >> 4;
            const uint32_t id2_p = tc::idesc(128, kcp, kFmt, 0), id2_n = tc::idesc(128, kcp, kFmt, 1);
            const uint32_t id3_p = tc::idesc(128, rb3, kFmt, 0), id3_n = tc::idesc(128, rb3, kFmt, 1);
            const uint32_t d2 = tmem_base, d3 = tmem_base + d3_col0;
            auto a2_off = [&](int t) { return (uint32_t)((t >> 2) * blk_a + (t & 3) * 32) >> 4; };
            auto b3_off = [&](int t) { return (uint32_t)((t >> 2) * blk_b + (t & 3) * 32) >> 4; };
            int stage0 = 0, n_a2 = 0, n_b3 = 0;
            uint32_t phase0 = 0;
            bool ok = true;
            auto slot_of = [&](int li) { return (item_begin + li) / nnu; };
            for (int li = 0; ok && li < L; ++li) {
                const bool new_p = li == 0 || slot_of(li) != slot_of(li - 1);
                const bool last_p = li + 1 == L || slot_of(li + 1) != slot_of(li);
                // ---- stage 2: D2 = T[q''] M_nu^T from one slot holding every M chunk of the item
                if (new_p && !tc::mbar_wait(&a2_full, n_a2++ & 1, &abort_flag, wl)) { ok = false; break; }
                if (li > 0 && !tc::mbar_wait(&s3_done, (li - 1) & 1, &abort_flag, wl)) { ok = false; break; }
                if (!tc::mbar_wait(&full_bar[stage0], phase0, &abort_flag, wl)) { ok = false; break; }
                tc::tc_fence_after();
                for (int part = 0; part < 2; ++part) {        // 0: Re outputs, 1: Im outputs
                    const uint32_t dd = d2 + (uint32_t)(part * kcp);
                    for (int c = 0; c < nkc; ++c) {
                        const uint64_t bb = b2d + (((uint32_t)stage0 * slot_bytes + (uint32_t)c * stage_bytes) >> 4);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int t = c * 4 + k;                      // K step of B (the M rows)
                            const int ta = part == 0 ? t : (t < hs ? t + hs : t - hs);   // A step paired with it
                            const uint32_t id = part == 0 && t >= hs ? id2_n : id2_p;
                            const uint32_t acc = t > 0 ? 1u : 0u;
                            const uint64_t ah = a2d + a2_off(ta), bh = bb + (uint32_t)(2 * k);
                            if (PREC == P_BF16X3) {
                                tc::mma_f16(dd, ah, bh, id, acc);
                                tc::mma_f16(dd, ah, bh + m_lo, id, 1u);
                                tc::mma_f16(dd, ah + a_lo, bh, id, 1u);
                            } else {
                                tc::mma_tf32(dd, ah, bh, id, acc);
                            }
                        }
                    }
                    tc::mma_commit(&d2_full[part]);
                }
                tc::mma_commit(&empty_bar[stage0]);
                if (++stage0 == n_slots) { stage0 = 0; phase0 ^= 1; }
                if (last_p) tc::mma_commit(&a2_empty);
                // ---- stage 3: D3 = X^T T[q']^T, A from tensor memory, K halves as they are converted
                if (new_p && !tc::mbar_wait(&b3_full, n_b3++ & 1, &abort_flag, wl)) { ok = false; break; }
                if (!tc::mbar_wait(&d3_empty, (li & 1) ^ 1, &abort_flag, wl)) { ok = false; break; }
                for (int h = 0; h < 2 && ok; ++h) {
                    if (!tc::mbar_wait(&a3_ready[h], li & 1, &abort_flag, wl)) { ok = false; break; }
                    tc::tc_fence_after();
                    for (int t = h * hs; t < (h + 1) * hs; ++t) {
                        const int tb = t < hs ? t + hs : t - hs;
                        const uint32_t acc = t > 0 ? 1u : 0u;
                        const uint32_t idr = t < hs ? id3_p : id3_n;
                        const uint64_t br = b3d + b3_off(t), bi = b3d + b3_off(tb);
                        if (PREC == P_BF16X3) {
                            // A step t = K elements 16t .. 16t+15: hi in columns 32(t/2) + 8(t%2), lo 16 further
                            const uint32_t ah = d2 + (uint32_t)(32 * (t >> 1) + 8 * (t & 1)), al = ah + 16;
                            tc::mma_f16_ts(d3, ah, br, idr, acc);
                            tc::mma_f16_ts(d3, ah, br + b3_lo, idr, 1u);
                            tc::mma_f16_ts(d3, al, br, idr, 1u);
                            tc::mma_f16_ts(d3 + rb3, ah, bi, id3_p, acc);
                            tc::mma_f16_ts(d3 + rb3, ah, bi + b3_lo, id3_p, 1u);
                            tc::mma_f16_ts(d3 + rb3, al, bi, id3_p, 1u);
                        } else {
                            const uint32_t a = d2 + (uint32_t)(8 * t);
                            tc::mma_tf32_ts(d3, a, br, idr, acc);
                            tc::mma_tf32_ts(d3 + rb3, a, bi, id3_p, acc);
                        }
                    }
                }
                if (!ok) break;
                tc::mma_commit(&s3_done);           // D3 complete and the stage-3 A operand free
                if (last_p) tc::mma_commit(&b3_empty);
            }
            if (!ok) fail();
            // every MMA of this thread has completed once drain_bar flips
            tc::mma_commit(&drain_bar);
            const uint64_t t0 = tc::global_ns();
            while (!tc::mbar_try_wait(&drain_bar, 0) && tc::global_ns() - t0 < wl) {
            }
        }
    } else if (warp != kChainIdleWarp && L > 0) {
        // ------------------------------------------------------------ epilogue (warps 0-2, 4-6, 8-10)
        const int et = (warp & 3) * 32 + (warp >> 2) * 96 + lane;   // 0 .. kChainEpiThreads - 1
        const int qd = warp & 3;                          // tensor-memory lane quarter (0..2)
        const int part = warp >> 2;                       // 0 .. kChainEpiParts - 1
        const int nu2 = qd * 32 + lane;                   // row of this thread (band nu'')
        const uint32_t lane_off = (uint32_t)(qd * 32) << 16;
        const bool quarter_live = qd * 32 < n;
        int cur_p = -1;
        float f2 = 0.f, nn2 = 0.f;

        // D2 -> stage-3 A operand in place, one K half (Re or Im outputs of stage 2) at a time;
        // each thread rewrites its own lane only
        auto convert = [&](int li) {
            for (int h = 0; h < 2; ++h) {
                bool ok = tc::mbar_wait(&d2_full[h], li & 1, &abort_flag, wl);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) { fail(); return; }
                tc::tc_fence_after();
                if (quarter_live) {
                    const uint32_t base = tmem_base + lane_off + (uint32_t)(h * kcp);
                    for (int ch = part; ch < kcp / 32; ch += kChainEpiParts) {
                        float v[32];
                        tc::tmem_ld16(base + 32 * ch, v);
                        tc::tmem_ld16(base + 32 * ch + 16, v + 16);
                        if (PREC == P_BF16X3) {
                            uint32_t hi[16], lo[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) tc::split_bf16x2(v[2 * i], v[2 * i + 1], &hi[i], &lo[i]);
                            tc::tmem_st16(base + 32 * ch, hi);
                            tc::tmem_st16(base + 32 * ch + 16, lo);
                        } else {
                            uint32_t r[32];
#pragma unroll
                            for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(tc::round_tf32(v[i]));
                            tc::tmem_st16(base + 32 * ch, r);
                            tc::tmem_st16(base + 32 * ch + 16, r + 16);
                        }
                    }
                    tc::tmem_wait_st();
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&a3_ready[h]);
            }
        };

        const bool gauss = args.shape == PHX_GAUSS;
        const float sg = args.sigma, lim = args.window * sg;
        // Gaussian: exp(-x^2/s^2) = 2^(ga2 x^2) with ga2 = -log2(e)/s^2 (one ex2 instruction)
        const float ga2 = -1.4426950408889634f / (sg * sg), h2 = 0.25f * sg * sg;
        const float norm = gauss ? 0.56418958354775628f / sg : 0.5f * sg / 3.14159265358979f;
        const bool want_w = MODE == CHAIN_G && args.wacc != nullptr;
        float nn2t[kMaxT];
#pragma unroll
        for (int t = 0; t < kMaxT; ++t) nn2t[t] = 0.f;
        int c1 = 0, c2 = 0;                              // CHAIN_GS: time-reversal codes of q', q''
        float lam2[3] = {0.f, 0.f, 0.f};                 // CHAIN_GL: f'' lambda of this lane's column
        // element weight cA (1+n'+n'') g(f-f'-f'') + cB (n'-n'') (g(f+f'-f'') - [pk] g(f+f''-f')):
        // (1, 2, no) for one ordered q' term; with exchange pairs (2, 2, yes) for q' != q'' (both
        // orderings) and (1, 1, yes) for q' = q'' (its (nu', nu'') sum already holds both)
        float cA = 1.f, cB = 2.f;
        bool pk = false;
        // CHAIN_GS: the column sums of item li are complete once every epilogue thread has passed
        // the barrier at the start of item li + 1; they are flushed to Gamma1 there (before the
        // partner tables change) from a buffer the next item does not use
        int prev_nu = -1, prev_c1 = 0, prev_c2 = 0;
        float prev_rs = 0.f;
        // Gamma1 row (q, nu) of the previous item += its column sums x f'/f at the q' block and its
        // row sums x f''/f at the q'' block: 16-byte reductions of four adjacent entries when n is a
        // multiple of 4 (rows are 128-entry aligned), single ones otherwise; the buffer is zeroed
        const bool vec4 = (n & 3) == 0;
        auto flush_sums = [&](int buf) {
            const bool row_ok = prev_nu >= 0 && args.g1_row0 + prev_nu < args.g1_rows;
            float* grow = args.g1 + (args.g1_row0 + prev_nu) * args.g1_ld;
            const int per = vec4 ? 4 : 1, nb = (rb3 + per - 1) / per;
            for (int t = et; t < 2 * nb; t += kChainEpiThreads) {
                const bool rows = t >= nb;                   // 0: columns at q', 1: rows at q''
                const int j0 = (rows ? t - nb : t) * per;
                const int code = rows ? prev_c2 : prev_c1;
                float* src = rows ? &s_row[buf][j0] : &s_col[buf][j0];
                float v[4] = {0.f, 0.f, 0.f, 0.f}, fp[4] = {0.f, 0.f, 0.f, 0.f};
                bool any = false;
                for (int k = 0; k < per; ++k) {
                    v[k] = src[k];
                    src[k] = 0.f;
                    fp[k] = rows ? s_f2[j0 + k] : s_tab[j0 + k].x;
                    any |= v[k] != 0.f && j0 + k < n;
                }
                if (!any || code == 0 || !row_ok) continue;
                const float r = code > 0 ? prev_rs : -prev_rs;
                const int64_t gc = (int64_t)(abs(code) - 1) * n + j0;
                if (gc + per - 1 >= args.g1_ld) { atomicExch(args.status, (int)PHX_ERR_INVALID); continue; }   // bounds self-check
                if (vec4)
                    atomicAdd(reinterpret_cast<float4*>(grow + gc),
                              make_float4(r * fp[0] * v[0], r * fp[1] * v[1], r * fp[2] * v[2], r * fp[3] * v[3]));
                else
                    atomicAdd(grow + gc, r * fp[0] * v[0]);
            }
        };
        if (MODE == CHAIN_GS)
            for (int j = et; j < 2 * kMaxNp; j += kChainEpiThreads) { (&s_col[0][0])[j] = 0.f; (&s_row[0][0])[j] = 0.f; }
        convert(0);
        for (int li = 0; li < L; ++li) {
            const int it = item_begin + li;
            const int p = it / nnu, nu = it % nnu;
            if (epi_barrier_any(kChainEpiThreads, abort_flag != 0)) break;   // one decision for all
            if (MODE == CHAIN_GS && li > 0) flush_sums((li - 1) & 1);
            if (p != cur_p) {
                // partner tables of this slot's q' (every thread has finished the previous item:
                // barrier above) and this thread's row constants at q''
                if (MODE == CHAIN_GS) epi_barrier(kChainEpiThreads);    // flush read the old tables
                const int q1 = args.qp[p], q2 = args.qpp[p];
                pk = args.pair != 0;
                cA = pk && q1 != q2 ? 2.f : 1.f;
                cB = pk && q1 == q2 ? 1.f : 2.f;
                for (int j = et; j < rb3; j += kChainEpiThreads) {
                    const bool v = j < n;
                    const float f1 = v ? (float)args.freq[(int64_t)q1 * n + j] : 0.0f;
                    // 1/f' = 0 masks padding and soft partners
                    s_tab[j] = make_float4(f1, v ? (float)args.nB[(int64_t)q1 * n + j] : 0.0f,
                                           (v && f1 >= args.f_min) ? 1.0f / f1 : 0.0f, 0.0f);
                    if (MODE == CHAIN_GS) s_f2[j] = v ? (float)args.freq[(int64_t)q2 * n + j] : 0.0f;
                    if (MODE == CHAIN_GL) {
                        const int cq = args.tr_code[q1];
                        const int64_t col = (int64_t)(abs(cq) - 1) * n + j;
                        const bool use = v && cq != 0 && col < args.g1_ld;
                        const double fs = cq > 0 ? (double)f1 : -(double)f1;
                        for (int a = 0; a < 3; ++a) s_lam[a][j] = use ? (float)(fs * args.lam[a * args.g1_ld + col]) : 0.0f;
                    }
                    if (MODE == CHAIN_GT)
                        for (int t = 0; t < kMaxT; ++t)
                            s_n1t[t][j] = (v && t < args.n_t) ? (float)args.nB[t * args.nb_stride + (int64_t)q1 * n + j]
                                                              : 0.0f;
                }
                f2 = nu2 < n ? (float)args.freq[(int64_t)q2 * n + nu2] : 0.f;
                nn2 = nu2 < n ? (float)args.nB[(int64_t)q2 * n + nu2] : 0.f;
                if (MODE == CHAIN_GT)
#pragma unroll
                    for (int t = 0; t < kMaxT; ++t)
                        nn2t[t] = (nu2 < n && t < args.n_t) ? (float)args.nB[t * args.nb_stride + (int64_t)q2 * n + nu2]
                                                            : 0.f;
                if (MODE == CHAIN_GS) { c1 = args.tr_code[q1]; c2 = args.tr_code[q2]; }
                if (MODE == CHAIN_GL) {
                    // this lane's column (q'', nu''): signed f'' lambda(q'', nu'')
                    const int cq = args.tr_code[q2];
                    const int64_t col = (int64_t)(abs(cq) - 1) * n + nu2;
                    const bool use = nu2 < n && cq != 0 && col < args.g1_ld;
                    const double fs = cq > 0 ? (double)f2 : -(double)f2;
                    for (int a = 0; a < 3; ++a) lam2[a] = use ? (float)(fs * args.lam[a * args.g1_ld + col]) : 0.f;
                }
                epi_barrier(kChainEpiThreads);
                cur_p = p;
            }
            const float f0 = (float)args.freq[(int64_t)args.iq * n + args.nu0 + nu];
            const bool live = nu2 < n && f0 >= args.f_min && f2 >= args.f_min;
            // w = [...] / (2 pi)^4 / (f0 f1 f2): delta(w) = g(f)/(2 pi) and 1/(w0 w1 w2)
            const float inv_f02 = live ? 1.0f / (1558.5454565440389f * f0 * f2) : 0.0f;
            const float rowfac = norm * inv_f02;
            const float d02 = f0 - f2, s02 = f0 + f2, one_n2 = 1.f + nn2;
            float gs = 0.f, ws = 0.f;
            float yl[3] = {0.f, 0.f, 0.f};               // CHAIN_GL: sum of e f' lambda' over columns
            float gst[kMaxT];
#pragma unroll
            for (int t = 0; t < kMaxT; ++t) gst[t] = 0.f;
            bool ok = tc::mbar_wait(&s3_done, li & 1, &abort_flag, wl);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                tc::tc_fence_after();
                if (quarter_live) {
                    const uint32_t d3 = tmem_base + lane_off + d3_col0;
                    for (int c0 = part * 16; c0 < rb3; c0 += 16 * kChainEpiParts) {
                        float v[16], vi[16], e[16];
                        tc::tmem_ld16(d3 + c0, v);
                        tc::tmem_ld16(d3 + rb3 + c0, vi);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int jj = c0 + i;
                            const float4 tb = s_tab[jj];
                            const float f1 = tb.x, n1 = tb.y, if1 = tb.z;
                            const float x = d02 - f1, y = d02 + f1, z = s02 - f1;
                            const float gd = fabsf(x) < lim ? (gauss ? ex2_approx(ga2 * x * x) : __frcp_rn(x * x + h2)) : 0.f;
                            const float ga = fabsf(y) < lim ? (gauss ? ex2_approx(ga2 * y * y) : __frcp_rn(y * y + h2)) : 0.f;
                            const float gb = pk && fabsf(z) < lim ? (gauss ? ex2_approx(ga2 * z * z) : __frcp_rn(z * z + h2)) : 0.f;
                            const float v2 = fmaf(v[i], v[i], vi[i] * vi[i]);
                            if (MODE == CHAIN_GT) {
                                const float gdd = cA * gd, gad = cB * (ga - gb);
#pragma unroll
                                for (int t = 0; t < kMaxT; ++t) {
                                    const float n1t = s_n1t[t][jj];
                                    gst[t] = fmaf(v2 * if1, (1.f + nn2t[t] + n1t) * gdd + (n1t - nn2t[t]) * gad, gst[t]);
                                }
                            } else {
                                const float w = (cA * (one_n2 + n1) * gd + cB * (n1 - nn2) * (ga - gb)) * if1;
                                if (MODE == CHAIN_GS) {
                                    // full element weight; rows without a live mode add nothing (select,
                                    // not product: such lanes of D3 may hold anything)
                                    e[i] = live ? v2 * w * rowfac : 0.f;
                                    gs += e[i];
                                } else if (MODE == CHAIN_GL) {
                                    const float el = live ? v2 * w * rowfac : 0.f;
                                    gs += el;
                                    yl[0] = fmaf(el, s_lam[0][jj], yl[0]);
                                    yl[1] = fmaf(el, s_lam[1][jj], yl[1]);
                                    yl[2] = fmaf(el, s_lam[2][jj], yl[2]);
                                } else {
                                    gs = fmaf(v2, w, gs);
                                    if (want_w) ws += w;
                                }
                            }
                        }
                        if (MODE == CHAIN_GS) {
                            // halving exchange: lanes 2c, 2c+1 end with the warp's sum of column c0 + c
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
                            if (!(lane & 1) && a1 != 0.f) atomicAdd(&s_col[li & 1][c0 + (lane >> 1)], a1);
                        }
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&d3_empty);
            } else {
                fail();
            }
            if (li + 1 < L) convert(li + 1);
            // all rows of the item belong to band nu: one warp sum, one atomic per warp
            if (MODE == CHAIN_GT) {
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) {
                    if (t >= args.n_t) break;
                    double dg = live ? (double)(gst[t] * rowfac) : 0.0;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) dg += __shfl_xor_sync(0xffffffffu, dg, off);
                    if (lane == 0 && ok && !abort_flag && dg != 0.0) atomicAdd(&args.gacc[t * args.t_stride + args.nu0 + nu], dg);
                }
            } else if (MODE == CHAIN_GL) {
                // linewidth, and y of row (q, nu) += (scale / f) sum e (f' lambda' + f'' lambda'')
                double dg = (double)gs;
                double dy[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) dy[a] = (double)fmaf(gs, lam2[a], yl[a]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    dg += __shfl_xor_sync(0xffffffffu, dg, off);
#pragma unroll
                    for (int a = 0; a < 3; ++a) dy[a] += __shfl_xor_sync(0xffffffffu, dy[a], off);
                }
                const int64_t row = args.g1_row0 + nu;
                if (lane == 0 && ok && !abort_flag) {
                    if (dg != 0.0) atomicAdd(&args.gacc[args.nu0 + nu], dg);
                    if (row < args.g1_rows) {
                        const double rs = (double)args.g1_scale / (double)f0;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            if (dy[a] != 0.0) atomicAdd(&args.ylam[a * args.g1_ld + row], rs * dy[a]);
                    }
                }
            } else {
                double dg = MODE == CHAIN_GS ? (double)gs : (live ? (double)(gs * rowfac) : 0.0);
                double dw = live ? (double)(ws * rowfac) : 0.0;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    dg += __shfl_xor_sync(0xffffffffu, dg, off);
                    if (MODE == CHAIN_G) dw += __shfl_xor_sync(0xffffffffu, dw, off);
                }
                if (lane == 0 && ok && !abort_flag) {
                    if (dg != 0.0) atomicAdd(&args.gacc[args.nu0 + nu], dg);
                    if (MODE == CHAIN_G && args.wacc && dw != 0.0) atomicAdd(&args.wacc[args.nu0 + nu], dw);
                }
            }
            if (MODE == CHAIN_GS) {
                // column (q'', nu''): this lane's row sum over this warp's partner columns
                if (ok && live && gs != 0.f) atomicAdd(&s_row[li & 1][nu2], gs);
                prev_nu = nu;
                prev_c1 = c1;
                prev_c2 = c2;
                prev_rs = args.g1_scale / f0;
            }
        }
        if (MODE == CHAIN_GS) {
            epi_barrier(kChainEpiThreads);
            if (!abort_flag && prev_nu >= 0) flush_sums((L - 1) & 1);
        }
    }
    __syncthreads();
    if (warp == kChainMmaWarp) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, 512);
    }
}
