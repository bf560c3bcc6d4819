// Internal declarations shared by the translation units of libphx (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/phx.h"

// Physical constants (CODATA 2018) and unit conversions used by the library.
namespace phx {
constexpr double kHbarEvPs = 6.582119569e-4;    // eV ps
constexpr double kKbEvK = 8.617333262e-5;       // eV / K
constexpr double kEvJ = 1.602176634e-19;        // J / eV
constexpr double kAmuKg = 1.66053906660e-27;    // kg / amu
// eV/(A^2 amu) -> ps^-2 and eV/(ps A K) -> W/(m K)
constexpr double kEvA2AmuToPs2 = kEvJ / (1e-20 * kAmuKg) * 1e-24;
constexpr double kEvPsAKToWmK = kEvJ / 1e-12 / 1e-10;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.1415926535897932384626433832795;
constexpr double kDegenerateRelTol = 1e-5;
}  // namespace phx

// Device-memory workspace owned by a context: grow-only named buffers.
struct phx_ctx {
    int device = 0;
    std::string err;
    std::map<std::string, std::pair<void*, size_t>> ws;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    void* status_word = nullptr;     // device int32 written by kernels with bounded waits
    // profiling: event pairs around launches of instrumented kernel classes
    bool prof = false;
    struct Rec { int kernel; cudaEvent_t a, b; double flops, bytes; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[PHX_K_COUNT] = {0};
    int64_t prof_n[PHX_K_COUNT] = {0};
    double prof_flops[PHX_K_COUNT] = {0}, prof_bytes[PHX_K_COUNT] = {0};
    int64_t launches = 0;            // kernels launched since the last profile enable
    // batched path: capture stream, cached graph of the last job list, q'-tile autotune table
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // tensor-core linewidth path: side stream of the fold and Fourier GEMM, with its fork, join and
    // buffer events (created outside any capture)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_ev[8] = {};
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint8_t> graph_key;
    int64_t graph_launches = 0;
    std::map<std::vector<int>, std::array<int, 3>> tune_q;   // job class -> (q' tile, chained kernel, side SMs)
    // options (phx_set_option)
    int opt_chain = 0;                            // 0 auto, 1 force the chained kernel, 2 never
    int opt_pair = 1;                             // evaluate each exchange pair {q', q''} once
    int opt_side_sms = -1;                        // SMs of the side stream (-1: default, 0: one stream)
    int opt_vel_fp32 = 0;                         // velocity products of phx_harmonic in FP32
    int opt_harm_tr = 1;                          // phx_harmonic solves one q of each {q, -q} pair
    int opt_sc_mfree = 0;                         // phx_kappa_sc: 0 dense Gamma1 when it fits, 1 matrix-free, 2 dense
    unsigned long long opt_wait_ns = 2000000000ull;   // bound of every device barrier wait
    int opt_starve = 0;                           // test hook: tensor-core producers issue nothing
};

// SMs the tensor-core linewidth path gives to its side stream (gamma_tc.cu)
int phx_side_sms(const phx_ctx* ctx);

// Profiling helpers: begin returns a record slot (or -1 when profiling is off).
int phx_prof_begin(phx_ctx* ctx, cudaStream_t s);
void phx_prof_end(phx_ctx* ctx, int slot, cudaStream_t s, int kernel, double flops, double bytes);

struct phx_fc3 {
    phx_ctx* ctx = nullptr;
    int n = 0;                  // modes per q (3 * n_atoms)
    int mesh[3] = {1, 1, 1};
    int nq = 1;
    int n_d = 0;                // distinct folded lattice differences
    int64_t nnz = 0;
    int64_t n_seg = 0;          // distinct (d, b, c) keys
    // device arrays
    int32_t* d_int = nullptr;       // [n_d][3] folded d in mesh units (0..n_i-1)
    int32_t* seg_key = nullptr;     // [n_seg][3] (d index, b, c)
    int64_t* seg_start = nullptr;   // [n_seg + 1]
    int32_t* ent_a = nullptr;       // [nnz] component index a of each entry (sorted)
    int32_t* ent_r2 = nullptr;      // [nnz][3] R'' of each entry
    double* ent_w = nullptr;        // [nnz] Phi3 / sqrt(m_a m_b m_c)
    // tensor-core path tables, built on first use (before any capture)
    // the entries again, grouped by (b, c), then by d, then a: entry j of pair bc = b*n + c is
    // j in [tc_bc_start[bc], tc_bc_start[bc + 1]), with (a, d) = tc_ent_ad[j] and its position in
    // the arrays above tc_ent_src[j]
    int64_t* tc_bc_start = nullptr; // [n*n + 1]
    int2* tc_ent_ad = nullptr;      // [nnz]
    int32_t* tc_ent_src = nullptr;  // [nnz]
    // Gamma-only large-cell path (mesh 1x1x1): permutation-symmetrised F = Phi3/sqrt(mmm) with
    // images summed, grouped by (row atom J, neighbour slot of atom K, gamma, beta) for
    // W_a[3J+beta][3K+gamma] = sum_i F[i][3J+beta][3K+gamma] e_a[i]
    bool g0_ready = false;
    int g0_slots = 0;               // (J, K) atom pairs
    int g0_max_slots = 0;           // largest neighbour count of one atom
    int64_t g0_nnz = 0;
    int32_t* g0_nbr_start = nullptr;   // [n_atoms + 1]
    int32_t* g0_nbr_atom = nullptr;    // [g0_slots]
    int64_t* g0_seg_start = nullptr;   // [9 g0_slots + 1]
    int32_t* g0_ent_i = nullptr;       // [g0_nnz]
    double* g0_ent_w = nullptr;        // [g0_nnz]
};
// gamma_cell.cu: builds the g0_* tables of a 1x1x1-mesh handle (host sort, upload)
phx_status phx_fc3_prepare_cell(phx_ctx* ctx, const phx_cell* cell, const phx_ifc3* fc3, phx_fc3* h);

// ---------------------------------------------------------------- host helpers

phx_status phx_set_error(phx_ctx* ctx, phx_status st, const char* fmt, ...);
void* phx_ws(phx_ctx* ctx, const char* name, size_t bytes);   // nullptr on failure (error set)

#define PHX_CUDA_CHECK(ctx, expr)                                                        \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return phx_set_error((ctx), PHX_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,    \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

#define PHX_TRY(expr)                 \
    do {                              \
        phx_status s_ = (expr);       \
        if (s_ != PHX_OK) return s_;  \
    } while (0)

// Input staging: returns a device pointer holding `count` elements of `host_or_dev`.
// For PHX_MEM_HOST the data are copied into workspace buffer `name` on `stream`.
template <typename T>
static inline phx_status phx_stage_in(phx_ctx* ctx, const char* name, const T* p, size_t count,
                                      int mem, cudaStream_t stream, const T** out) {
    if (mem == PHX_MEM_DEVICE || count == 0) {
        *out = p;
        return PHX_OK;
    }
    T* d = (T*)phx_ws(ctx, name, count * sizeof(T));
    if (!d) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, stream));
    *out = d;
    return PHX_OK;
}

template <typename T>
static inline phx_status phx_stage_out_buf(phx_ctx* ctx, const char* name, T* p, size_t count,
                                           int mem, T** out) {
    if (mem == PHX_MEM_DEVICE || count == 0) {
        *out = p;
        return PHX_OK;
    }
    T* d = (T*)phx_ws(ctx, name, count * sizeof(T));
    if (!d) return PHX_ERR_NOMEM;
    *out = d;
    return PHX_OK;
}

// ---------------------------------------------------------------- kernels (launchers)
// Each launcher enqueues on `stream` and returns the launch error.

// harmonic.cu
// skip (optional, per q of the launch): nonzero = the q is filled later from its time-reversal
// partner by phx_launch_tr_fill, so the kernel leaves it alone
cudaError_t phx_launch_dynmat(const double* q_frac, int nq, int n_atoms, const int32_t* blk_idx,
                              const double* blk_val, const int32_t* pair_start, const double* masses,
                              const double* lattice, double* D, double* dD, cudaStream_t s,
                              const int32_t* skip = nullptr);
// scratch: 4 n doubles per matrix (Householder path for n <= 96; nullptr selects Jacobi)
cudaError_t phx_launch_jacobi(double* A, double* V, int n, int nq, double* freq, double* evec,
                              int32_t* status, cudaStream_t s, double* scratch = nullptr,
                              const int32_t* skip = nullptr);
cudaError_t phx_launch_velocity(const double* evec, const double* Y, const double* freq, int n,
                                int nq, double* vel, double* vv, cudaStream_t s, const int32_t* skip = nullptr);
// Time-reversal classes of a q list: q_i and q_j are in one class when q_j = q_i or q_j = -q_i
// (mod G, components within 1e-9).  code[i] = 2 r + c with r the smallest index of the class and
// c = 1 when q_r = -q_i (and not q_r = q_i); skip[i] = (r != i).
cudaError_t phx_launch_tr_classes(const double* q_frac, int nq, int32_t* code, int32_t* skip, cudaStream_t s);
// Fill every q with r != i from its class representative: D(-q) = conj D(q) (the dynamical
// matrix is G-periodic and Hermitian), so f(-q) = f(q), e(-q) = conj e(q), v(-q) = -v(q) and
// v (x) v unchanged; a copy where q_r = q_i.  vel, vv may be null.
cudaError_t phx_launch_tr_fill(const int32_t* code, int nq, int n, double* freq, double* evec, double* vel,
                               double* vv, cudaStream_t s);
// eigh_large.cu: Gamma point of a cell with more than 64 atoms (device pair CSR in, device out)
constexpr int kPhxMaxLargeModes = 8192;
phx_status phx_eigh_gamma_large(phx_ctx* ctx, int na, const double* blk_val, const int32_t* pair_start,
                                const double* masses, double* freq, double* evec, cudaStream_t s);

// zgemm.cu: batched complex FP64 GEMM, row-major; see the kernel for the batch addressing.
struct ZgemmBatch {
    // C_b[M x N] = opA(A_b)[M x K] * B_b[K x N]
    const double* A;    // complex
    const double* B;
    double* C;
    int64_t strideA, strideB, strideC;   // complex elements per batch step (when no index map)
    const int32_t* idxA;                 // optional: A_b = A + idxA[b / divA] * strideA
    const int32_t* idxB;                 // optional: B_b = B + idxB[b / divB] * strideB
    int divA, divB;                      // batch divisors for the index maps (>= 1)
    int64_t strideB_inner;               // added per (b % divB) when idxB given
    int lda, ldb, ldc;
    int transA;                          // 1: A stored [K][M] (plain transpose, no conjugate)
    int fp32;                            // 1: products and sums in FP32 (FP64 inputs and output)
    const int32_t* skip;                 // optional: batch b is not computed when skip[b / skip_div] != 0
    int skip_div;
};
cudaError_t phx_launch_zgemm(int M, int N, int K, int batch, const ZgemmBatch& p, cudaStream_t s);

// transport.cu
cudaError_t phx_launch_occupations(const double* freq, int count, double T, int is_classic,
                                   double* nB, double* cV, cudaStream_t s);
cudaError_t phx_launch_unfold(int n_irr, int nq, int n, const double* freq_full, const int32_t* irr_q,
                              const double* gamma_irr, const int32_t* full_to_irr,
                              double* gamma_full, cudaStream_t s);
cudaError_t phx_launch_kappa(int nq, int n, const double* freq, const double* vel,
                             const double* vv, const double* gamma_full, double T, double f_min,
                             int is_classic, double* acc9, cudaStream_t s);

cudaError_t phx_launch_third_index(int iq, const int* mesh, int32_t* qpp, cudaStream_t s);
cudaError_t phx_launch_finalize(int count, int n, const int32_t* irr, const double* freq, const double* gacc,
                                const double* wacc, double pref, double inv_nq, double f_min, double* gamma,
                                double* wp2, cudaStream_t s);
cudaError_t phx_launch_scale9(const double* acc, double scale, double* out, cudaStream_t s);

// Off-diagonal scattering rows (Eq. gamma1) accumulated by a linewidth contraction, folded
// onto time-reversal representatives: row (position s of the representative, band nu) is
// s * n + nu; mesh point p with band nu' is column (|tr_code[p]| - 1) * n + nu', added with
// the sign of tr_code[p]; tr_code[p] = 0 (p = -p mod G) drops the column.
struct G1Target {
    void* mat;                  // float [rows][ld] (tensor-core paths) or double (FP64 path)
    int64_t ld;                 // row stride (elements)
    const int32_t* tr_code;     // device, [nq]
    double scale;               // the linewidth prefactor pi hbar conv^3 / (8 N_q)
    // matrix-free form (tensor-core paths): with lam set, mat is unused and the pass adds
    // y[a][r] += sum_c Gamma1[r][c] lam[a][c] (planes [3][ld], FP64) for every row r it covers
    const double* lam = nullptr;
    double* y = nullptr;
};

// gamma path shared parameters
struct GammaParams {
    int n;                 // modes
    int mesh[3];
    int nq;
    double T;
    int shape;
    double sigma;
    double window;
    double f_min;
};

// Linewidth contractions (gacc/wacc: [n_irr][n] device accumulators, zeroed by the caller);
// g1 (optional): also accumulate the off-diagonal scattering rows of the irreducible points.
phx_status phx_gamma_fp64(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                          const double* nB, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                          double* gacc, double* wacc, cudaStream_t s, const G1Target* g1 = nullptr);
phx_status phx_gamma_tc(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                        const double* nB, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                        int prec, double* gacc, double* wacc, cudaStream_t s, const G1Target* g1 = nullptr);
