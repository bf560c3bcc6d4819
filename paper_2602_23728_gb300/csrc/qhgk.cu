// Quasi-harmonic Green-Kubo conductivity of a Gamma-only cell (paper Sec. "Quasi-Harmonic
// Green-Kubo (QHGK)", Eq. (qhgk)):
//     kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} Re(v^a_{mu mu'} v^b_{mu' mu}) tau_{mu mu'}
// with c_{mu mu'} = (hbar w w'/T)(n - n')/(w' - w) (c_mu for pairs closer than 1e-5 f_max),
// v^a_{mu mu'} = -i V^a_{mu mu'} / (2 sqrt(w w')), V^a = E^T G^a E, G^a_{ij} = sum_R (x_j + R
// - x_i)_a Phi2(0i, Rj)/sqrt(m_i m_j) (the atom-position-gauge dD/dq at Gamma is -i G^a), and
// tau_{mu mu'} = g/(2((w - w')^2 + g^2)), g = (gamma_mu + gamma_mu')/4.
// For real eigenvectors V^a is antisymmetric, so the summand is
// c tau V^a V^b / (4 w w'), symmetric in (mu, mu'), and only mu < mu' is summed (twice).
//
//   ymat_kernel   Y^a = G^a E   (sparse: atom-pair blocks, all three a at once; FP64)
//   vtile_kernel  V^a = E^T Y^a on 128 x 128 tiles with b-tile <= c-tile (FP64 CUDA cores)
//   pairs_kernel  the weighted pair sum into the 3 x 3 tensor (FP64 atomics per CTA)
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.h"

namespace {

constexpr int kTile = 128;

__global__ void real_part_kernel(const double2* __restrict__ evec, int64_t count, double* __restrict__ e,
                                 int32_t* __restrict__ status) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const double2 z = evec[t];
        e[t] = z.x;
        if (z.y != 0.0) atomicExch(status, (int)PHX_ERR_INVALID);
    }
}

// Y[a][3J+beta][c] = sum over blocks b of row atom J: r_a(b) sum_gamma P_b[beta][gamma] E[3K+gamma][c]
// (P_b = Phi2 block / sqrt(m m), r the bond vector).  Grid: (column chunks of 256, atoms J).
__global__ void __launch_bounds__(256)
ymat_kernel(const double* __restrict__ E, int n, const int32_t* __restrict__ row_start,
            const int32_t* __restrict__ blk_col, const double* __restrict__ blk_val, const double* __restrict__ blk_r,
            double* __restrict__ Y) {
    const int c = blockIdx.x * 256 + threadIdx.x;
    const int J = blockIdx.y;
    if (c >= n) return;
    double acc[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[a][0] = acc[a][1] = acc[a][2] = 0.0;
    for (int b = row_start[J]; b < row_start[J + 1]; ++b) {
        const int K = blk_col[b];
        const double e0 = E[(int64_t)(3 * K) * n + c], e1 = E[(int64_t)(3 * K + 1) * n + c],
                     e2 = E[(int64_t)(3 * K + 2) * n + c];
        const double* P = blk_val + 9 * (int64_t)b;
        const double r0 = blk_r[3 * (int64_t)b], r1 = blk_r[3 * (int64_t)b + 1], r2 = blk_r[3 * (int64_t)b + 2];
#pragma unroll
        for (int be = 0; be < 3; ++be) {
            const double t = P[3 * be] * e0 + P[3 * be + 1] * e1 + P[3 * be + 2] * e2;
            acc[0][be] += r0 * t;
            acc[1][be] += r1 * t;
            acc[2][be] += r2 * t;
        }
    }
    const int64_t nn = (int64_t)n * n;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int be = 0; be < 3; ++be) Y[a * nn + (int64_t)(3 * J + be) * n + c] = acc[a][be];
}

// V[a][mu][mu'] = sum_k E[k][mu] Y[a][k][mu'] for the tiles (a, bt, ct) listed (bt <= ct);
// 256 threads x (8 x 8) outputs, K in steps of 16.
__global__ void __launch_bounds__(256)
vtile_kernel(const double* __restrict__ E, const double* __restrict__ Y, int n, const int4* __restrict__ tiles,
             double* __restrict__ V) {
    __shared__ double As[16][kTile + 1], Bs[16][kTile + 1];
    const int4 w = tiles[blockIdx.x];
    const int a = w.x, r0 = w.y * kTile, c0 = w.z * kTile;
    const int64_t nn = (int64_t)n * n;
    const double* Ya = Y + a * nn;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int t = threadIdx.x; t < kTile * 16; t += 256) {
            const int k = t >> 7, r = t & (kTile - 1);
            const bool kin = k0 + k < n;
            As[k][r] = (kin && r0 + r < n) ? E[(int64_t)(k0 + k) * n + r0 + r] : 0.0;
            Bs[k][r] = (kin && c0 + r < n) ? Ya[(int64_t)(k0 + k) * n + c0 + r] : 0.0;
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
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < n) V[a * nn + (int64_t)r * n + c] = acc[i][j];
        }
    }
}

// sum over mu < mu' of 2 c tau V^a V^b / (4 w w'), reduced per CTA into acc[9]
__global__ void __launch_bounds__(256)
pairs_kernel(const double* __restrict__ V, const double* __restrict__ freq, const double* __restrict__ nocc,
             const double* __restrict__ cmode, const double* __restrict__ gamma, int n, double T, double f_min,
             double deg_tol, double* __restrict__ acc) {
    __shared__ double red[9][8];
    const int64_t nn = (int64_t)n * n;
    double s[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) s[t] = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(p / n), mp = (int)(p % n);
        if (mp <= m) continue;
        const double f = freq[m], fp = freq[mp];
        if (f < f_min || fp < f_min) continue;
        const double g = 0.25 * (gamma[m] + gamma[mp]);
        if (!(gamma[m] > 0.0) || !(gamma[mp] > 0.0)) continue;
        const double w = phx::kTwoPi * f, wp = phx::kTwoPi * fp;
        double c;
        if (fabs(fp - f) < deg_tol) c = 0.5 * (cmode[m] + cmode[mp]);
        else c = phx::kHbarEvPs * w * wp * (nocc[m] - nocc[mp]) / (T * (wp - w));
        const double dw = w - wp;
        const double tau = g / (2.0 * (dw * dw + g * g));
        const double wt = 2.0 * c * tau / (4.0 * w * wp);
        const double vx = V[(int64_t)m * n + mp], vy = V[nn + (int64_t)m * n + mp], vz = V[2 * nn + (int64_t)m * n + mp];
        const double v[3] = {vx, vy, vz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) s[3 * a + b] += wt * v[a] * v[b];
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        double x = s[t];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double x = 0.0;
        for (int wv = 0; wv < 8; ++wv) x += red[threadIdx.x][wv];
        if (x != 0.0) atomicAdd(&acc[threadIdx.x], x);
    }
}

__global__ void mode_tables_kernel(const double* __restrict__ freq, int n, double T, double f_min,
                                   double* __restrict__ nocc, double* __restrict__ cmode) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double f = freq[m];
    if (!(f > 0.0) || f < f_min) { nocc[m] = 0.0; cmode[m] = 0.0; return; }
    const double x = phx::kHbarEvPs * phx::kTwoPi * f / (phx::kKbEvK * T);
    const double em = expm1(x);
    nocc[m] = 1.0 / em;
    cmode[m] = phx::kKbEvK * x * x * exp(x) / (em * em);
}

}  // namespace

extern "C" phx_status phx_kappa_qhgk(phx_ctx* ctx, const phx_cell* cell, const phx_ifc2* fc2, const double* freq_thz,
                                     const double* evec, const double* gamma, double temperature, double f_min_thz,
                                     double kappa_wmk[9], int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!cell || !fc2 || !cell->masses || !cell->positions || !freq_thz || !evec || !gamma || !kappa_wmk)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: null argument");
    if (!(temperature > 0.0) || !(f_min_thz > 0.0) || !std::isfinite(temperature))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: T and f_min must be finite and > 0");
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: bad mem flag %d", mem);
    const int na = cell->n_atoms, n = 3 * na;
    if (na <= 0 || n > kPhxMaxLargeModes)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_kappa_qhgk: n_atoms=%d (need 1..%d)", na,
                             kPhxMaxLargeModes / 3);
    const int nb = fc2->n_blocks;
    if (nb < 0 || (nb > 0 && (!fc2->idx || !fc2->val))) return phx_set_error(ctx, PHX_ERR_INVALID, "bad fc2");
    const double* L = cell->lattice;
    const double vol = std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                                 L[2] * (L[3] * L[7] - L[4] * L[6]));
    if (!(vol > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: degenerate lattice");
    // blocks by row atom: bond vector and mass-scaled values
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    for (int b = 0; b < nb; ++b) {
        const int i = fc2->idx[5 * b], j = fc2->idx[5 * b + 1];
        if (i < 0 || i >= na || j < 0 || j >= na)
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: block %d atom index out of range", b);
        if (!(cell->masses[i] > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "mass %d not positive", i);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return fc2->idx[5 * x] < fc2->idx[5 * y]; });
    std::vector<int32_t> row_start(na + 1, 0), blk_col(nb);
    std::vector<double> blk_val((size_t)nb * 9), blk_r((size_t)nb * 3);
    for (int k = 0; k < nb; ++k) {
        const int b = order[k];
        const int32_t* e = fc2->idx + 5 * b;
        const int i = e[0], j = e[1];
        row_start[i + 1] += 1;
        blk_col[k] = j;
        const double sc = 1.0 / std::sqrt(cell->masses[i] * cell->masses[j]);
        for (int t = 0; t < 9; ++t) blk_val[9 * k + t] = fc2->val[9 * b + t] * sc;
        for (int a = 0; a < 3; ++a)
            blk_r[3 * k + a] = cell->positions[3 * j + a] + e[2] * L[a] + e[3] * L[3 + a] + e[4] * L[6 + a] -
                               cell->positions[3 * i + a];
    }
    for (int i = 0; i < na; ++i) row_start[i + 1] += row_start[i];
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nn = (int64_t)n * n;
    const double *d_f = nullptr, *d_e = nullptr, *d_g = nullptr;
    PHX_TRY(phx_stage_in(ctx, "qh.f", freq_thz, (size_t)n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "qh.e", evec, (size_t)nn * 2, mem, s, &d_e));
    PHX_TRY(phx_stage_in(ctx, "qh.g", gamma, (size_t)n, mem, s, &d_g));
    int32_t* d_rs = (int32_t*)phx_ws(ctx, "qh.rs", (size_t)(na + 1) * 4);
    int32_t* d_col = (int32_t*)phx_ws(ctx, "qh.col", (size_t)std::max(nb, 1) * 4);
    double* d_val = (double*)phx_ws(ctx, "qh.val", (size_t)std::max(nb, 1) * 72);
    double* d_r = (double*)phx_ws(ctx, "qh.r", (size_t)std::max(nb, 1) * 24);
    double* E = (double*)phx_ws(ctx, "qh.E", nn * 8);
    double* Y = (double*)phx_ws(ctx, "qh.Y", 3 * nn * 8);
    double* V = (double*)phx_ws(ctx, "qh.V", 3 * nn * 8);
    double* tabs = (double*)phx_ws(ctx, "qh.tab", (size_t)2 * n * 8 + 9 * 8);
    const int nt = (n + kTile - 1) / kTile;
    std::vector<int4> tiles;
    for (int a = 0; a < 3; ++a)
        for (int bt = 0; bt < nt; ++bt)
            for (int ct = bt; ct < nt; ++ct) tiles.push_back(make_int4(a, bt, ct, 0));
    int4* d_tiles = (int4*)phx_ws(ctx, "qh.tiles", tiles.size() * 16);
    if (!d_rs || !d_col || !d_val || !d_r || !E || !Y || !V || !tabs || !d_tiles) return PHX_ERR_NOMEM;
    double *nocc = tabs, *cmode = tabs + n, *acc = tabs + 2 * n;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_rs, row_start.data(), row_start.size() * 4, cudaMemcpyHostToDevice, s));
    if (nb > 0) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_col, blk_col.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_val, blk_val.data(), (size_t)nb * 72, cudaMemcpyHostToDevice, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_r, blk_r.data(), (size_t)nb * 24, cudaMemcpyHostToDevice, s));
    }
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * 16, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(acc, 0, 9 * 8, s));
    real_part_kernel<<<4 * ctx->sm_count, 256, 0, s>>>((const double2*)d_e, nn, E, (int32_t*)ctx->status_word);
    mode_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(d_f, n, temperature, f_min_thz, nocc, cmode);
    dim3 yg((n + 255) / 256, na);
    ymat_kernel<<<yg, 256, 0, s>>>(E, n, d_rs, d_col, d_val, d_r, Y);
    vtile_kernel<<<(unsigned)tiles.size(), 256, 0, s>>>(E, Y, n, d_tiles, V);
    // frequencies decide the degenerate tolerance: 1e-5 of the largest |f| (read on the host)
    std::vector<double> fh(n);
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(fh.data(), d_f, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    double fmax = 0.0;
    for (double f : fh) fmax = std::max(fmax, std::fabs(f));
    pairs_kernel<<<8 * ctx->sm_count, 256, 0, s>>>(V, d_f, nocc, cmode, d_g, n, temperature, f_min_thz,
                                                  phx::kDegenerateRelTol * fmax, acc);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 6;
    double h[9];
    int32_t st = 0;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(h, acc, 9 * 8, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    if (st != 0) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_qhgk: eigenvectors must be real (Gamma point)");
    // V in eV/(A amu) -> A/ps^2 twice (conv^2); kappa in eV/(ps A K) -> W/(m K)
    const double conv = phx::kEvA2AmuToPs2;
    for (int t = 0; t < 9; ++t) kappa_wmk[t] = h[t] * conv * conv / vol * phx::kEvPsAKToWmK;
    return PHX_OK;
}
