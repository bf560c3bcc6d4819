// Harmonic phonons on the GPU in FP64 (paper Sec. "Interatomic Force Constants", Eqs.
// (dynmat), (dynmat_reciprocal), (eigenvalue_crystal); Sec. "Group Velocities", Eq. (groupvel)).
//
//  dynmat_kernel    D(q) = sum_R Phi2(0i, Rj) exp(-2 pi i q.R) / sqrt(m_i m_j) and the analytic
//                   dD/dq_a = sum_R (-i R_a) (...) for a batch of q (one CTA per q)
//  jacobi_kernel    batched complex-Hermitian cyclic Jacobi eigensolver, one CTA per matrix,
//                   round-robin ordering (n/2 disjoint rotations per step applied as one
//                   left and one right multiplication); matrix in shared memory when it fits
//  velocity_kernel  v_a = Re<e|dD/dq_a|e>/(2w) and the basis-invariant v(x)v per degenerate set
#include <cstdlib>

#include "common.h"

namespace {

constexpr int kJacobiThreads = 256;
constexpr int kMaxModes = 192;
constexpr int kMaxPairs = kMaxModes / 2;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One CTA per q.  pair_start is a CSR over (i, j) atom pairs (n_atoms^2 + 1 entries) into
// blocks sorted by (i, j).
__global__ void dynmat_kernel(const double* __restrict__ q_frac, int n_atoms,
                              const int32_t* __restrict__ blk_idx, const double* __restrict__ blk_val,
                              const int32_t* __restrict__ pair_start, const double* __restrict__ masses,
                              const double* __restrict__ lattice, double2* __restrict__ D,
                              double2* __restrict__ dD, const int32_t* __restrict__ skip) {
    const int q = blockIdx.x;
    if (skip && skip[q]) return;
    const int n = 3 * n_atoms;
    const int64_t nn = (int64_t)n * n;
    const double q0 = q_frac[3 * q], q1 = q_frac[3 * q + 1], q2 = q_frac[3 * q + 2];
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int row = (int)(e / n), col = (int)(e % n);
        const int i = row / 3, al = row % 3, j = col / 3, be = col % 3;
        const int p = i * n_atoms + j;
        double2 acc = make_double2(0.0, 0.0);
        double2 dacc[3] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
        for (int b = pair_start[p]; b < pair_start[p + 1]; ++b) {
            const int r1 = blk_idx[5 * b + 2], r2 = blk_idx[5 * b + 3], r3 = blk_idx[5 * b + 4];
            const double x = 2.0 * (q0 * r1 + q1 * r2 + q2 * r3);
            double s, c;
            sincospi(x, &s, &c);                 // exp(-i pi x) = c - i s
            const double v = blk_val[9 * b + 3 * al + be];
            acc.x += v * c;
            acc.y -= v * s;
            if (dD) {
                for (int a = 0; a < 3; ++a) {
                    const double Ra = r1 * lattice[a] + r2 * lattice[3 + a] + r3 * lattice[6 + a];
                    // (-i Ra) (c - i s) v = v Ra (-s - i c)
                    dacc[a].x += -v * Ra * s;
                    dacc[a].y += -v * Ra * c;
                }
            }
        }
        const double sc = 1.0 / sqrt(masses[i] * masses[j]);
        D[(int64_t)q * nn + e] = make_double2(acc.x * sc, acc.y * sc);
        if (dD) {
            for (int a = 0; a < 3; ++a)
                dD[((int64_t)q * 3 + a) * nn + e] = make_double2(dacc[a].x * sc, dacc[a].y * sc);
        }
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// Position of player x in round r of a round-robin tournament over m (even) players:
// player 0 stays, the others rotate.
__device__ __forceinline__ int rr_player(int x, int r, int m) {
    return x == 0 ? 0 : 1 + ((x - 1 + r) % (m - 1));
}

template <bool kSmem>
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_kernel(double2* __restrict__ Ag, double2* __restrict__ Vg, int n, double* __restrict__ freq,
              double2* __restrict__ evec, int32_t* __restrict__ status, const int32_t* __restrict__ skip) {
    if (skip && skip[blockIdx.x]) return;
    extern __shared__ double2 shA[];
    __shared__ double rc[kMaxPairs], rs[kMaxPairs], rpc[kMaxPairs], rps[kMaxPairs];
    __shared__ int rp[kMaxPairs], rq[kMaxPairs], ract[kMaxPairs];
    __shared__ double red[32];
    __shared__ double lam[kMaxModes];
    __shared__ int rank_of[kMaxModes];

    const int qi = blockIdx.x;
    const int64_t nn = (int64_t)n * n;
    double2* A = kSmem ? shA : Ag + (int64_t)qi * nn;
    double2* V = Vg + (int64_t)qi * nn;
    const int tid = threadIdx.x, nt = blockDim.x;

    // Hermitian part (D + D^H)/2: the two triangles of D(q) are summed from different blocks
    // and differ at the rounding level, which would otherwise keep the off-norm from vanishing
    // (at Gamma D is pure rounding noise).
    {
        const double2* Dq = Ag + (int64_t)qi * nn;
        for (int64_t e = tid; e < nn; e += nt) {
            const int i = (int)(e / n), j = (int)(e % n);
            if (i > j) continue;
            const double2 a = Dq[(int64_t)i * n + j], b = Dq[(int64_t)j * n + i];
            const double2 h = make_double2(0.5 * (a.x + b.x), i == j ? 0.0 : 0.5 * (a.y - b.y));
            A[(int64_t)i * n + j] = h;
            A[(int64_t)j * n + i] = make_double2(h.x, -h.y);
        }
    }
    for (int64_t e = tid; e < nn; e += nt) V[e] = make_double2((e / n == e % n) ? 1.0 : 0.0, 0.0);
    __syncthreads();

    const int m = n + (n & 1);
    const int np = m / 2;
    int converged = 0, extra = 0;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int64_t e = tid; e < nn; e += nt) {
            const double2 a = A[e];
            const double v = a.x * a.x + a.y * a.y;
            tot += v;
            if (e / n != e % n) off += v;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (off <= 1e-26 * tot || tot == 0.0) {
            if (extra) { converged = 1; break; }
            extra = 1;  // one more sweep past the threshold
        }
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < np; k += nt) {
                int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
                if (p > q) { int t = p; p = q; q = t; }
                int act = 0;
                double c = 1.0, s = 0.0, pc = 1.0, ps = 0.0;
                if (q < n) {
                    const double2 apq = A[(int64_t)p * n + q];
                    const double h = hypot(apq.x, apq.y);
                    if (h > 1e-300) {
                        const double app = A[(int64_t)p * n + p].x, aqq = A[(int64_t)q * n + q].x;
                        const double th = (aqq - app) / (2.0 * h);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                        pc = apq.x / h;   // exp(i phi)
                        ps = apq.y / h;
                        act = 1;
                    }
                }
                rc[k] = c; rs[k] = s; rpc[k] = pc; rps[k] = ps; rp[k] = p; rq[k] = q; ract[k] = act;
            }
            __syncthreads();
            // rows: A <- U^H A ; row p: c a_p - s e^{i phi} a_q ; row q: s a_p + c e^{i phi} a_q
            for (int64_t t = tid; t < (int64_t)np * n; t += nt) {
                const int k = (int)(t / n), j = (int)(t % n);
                if (!ract[k]) continue;
                const int p = rp[k], q = rq[k];
                const double c = rc[k], s = rs[k];
                const double2 ph = make_double2(rpc[k], rps[k]);
                const double2 ap = A[(int64_t)p * n + j], aq = A[(int64_t)q * n + j];
                const double2 eaq = cmul(ph, aq);
                A[(int64_t)p * n + j] = make_double2(c * ap.x - s * eaq.x, c * ap.y - s * eaq.y);
                A[(int64_t)q * n + j] = make_double2(s * ap.x + c * eaq.x, s * ap.y + c * eaq.y);
            }
            __syncthreads();
            // columns: A <- A U, V <- V U ; col p: c a_p - s e^{-i phi} a_q ; col q: s a_p + c e^{-i phi} a_q
            for (int64_t t = tid; t < (int64_t)np * n; t += nt) {
                const int i = (int)(t / np), k = (int)(t % np);
                if (!ract[k]) continue;
                const int p = rp[k], q = rq[k];
                const double c = rc[k], s = rs[k];
                const double2 phc = make_double2(rpc[k], -rps[k]);
                {
                    const double2 ap = A[(int64_t)i * n + p], aq = A[(int64_t)i * n + q];
                    const double2 eaq = cmul(phc, aq);
                    A[(int64_t)i * n + p] = make_double2(c * ap.x - s * eaq.x, c * ap.y - s * eaq.y);
                    A[(int64_t)i * n + q] = make_double2(s * ap.x + c * eaq.x, s * ap.y + c * eaq.y);
                }
                {
                    const double2 vp = V[(int64_t)i * n + p], vq = V[(int64_t)i * n + q];
                    const double2 evq = cmul(phc, vq);
                    V[(int64_t)i * n + p] = make_double2(c * vp.x - s * evq.x, c * vp.y - s * evq.y);
                    V[(int64_t)i * n + q] = make_double2(s * vp.x + c * evq.x, s * vp.y + c * evq.y);
                }
            }
            __syncthreads();
        }
    }
    if (!converged && tid == 0) atomicExch(status, (int)PHX_ERR_NUMERIC);

    for (int i = tid; i < n; i += nt) lam[i] = A[(int64_t)i * n + i].x;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        int r = 0;
        const double li = lam[i];
        for (int j = 0; j < n; ++j) r += (lam[j] < li) || (lam[j] == li && j < i);
        rank_of[i] = r;
        const double w2 = li * phx::kEvA2AmuToPs2;
        freq[(int64_t)qi * n + r] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / phx::kTwoPi;
    }
    __syncthreads();
    // gauge: largest-modulus component real positive (first index on ties); one warp per column
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int col = warp; col < n; col += nw) {
        double best = -1.0;
        int bi = 0;
        for (int i = lane; i < n; i += 32) {
            const double2 v = V[(int64_t)i * n + col];
            const double a = v.x * v.x + v.y * v.y;
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const double2 vm = V[(int64_t)bi * n + col];
        const double h = hypot(vm.x, vm.y);
        const double2 g = h > 0.0 ? make_double2(vm.x / h, -vm.y / h) : make_double2(1.0, 0.0);
        const int dst = rank_of[col];
        for (int i = lane; i < n; i += 32)
            evec[(int64_t)qi * nn + (int64_t)i * n + dst] = cmul(V[(int64_t)i * n + col], g);
    }
}

// Batched complex-Hermitian eigensolver for n <= kHhqlMaxModes in two kernels:
//  hh_reduce_kernel  (one CTA per matrix, the matrix in shared memory) Householder reduction
//     to tridiagonal form, H_k = I - beta v v^H with v = x + e^{i phi}|x| e1 (x = column k below
//     the diagonal, phi = arg x_0), rank-2 update A22 -= v w^H + w v^H with
//     w = p - (beta v^H p / 2) v, p = beta A22 v.  Writes the reflectors (row k of R holds v_k),
//     beta, the diagonal and the complex subdiagonal.
//  ql_back_kernel    (one small CTA per matrix, many per SM so their serial parts overlap) the
//     subdiagonal made real by the phases delta_{k+1} = delta_k e_k/|e_k|, implicit symmetric QR
//     steps with Wilkinson shifts (thread 0 forms a round's rotations, every thread applies them
//     to its rows of Z), eigenvalue ranks, back-transformation E = H_0 ... H_{n-3} diag(delta) Z written
//     straight into the sorted output column, then the gauge (largest-modulus component real
//     and positive, as the Jacobi solver).
// About 15 n^3 real flops per matrix against ~200 n^3 for the cyclic Jacobi sweeps.
constexpr int kHhqlMaxModes = 96;
constexpr int kQlMaxIter = 60;
constexpr int kQlThreads = 128;

// per-matrix scratch (doubles): d[n], e re/im [2n], beta[n]
__global__ void __launch_bounds__(256)
hh_reduce_kernel(const double2* __restrict__ Dg, double2* __restrict__ Rg, double* __restrict__ scratch, int n,
                 const int32_t* __restrict__ skip) {
    if (skip && skip[blockIdx.x]) return;
    extern __shared__ double2 A[];                           // n x n, row-major
    __shared__ double red[32];
    const int qi = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int64_t nn = (int64_t)n * n;
    const double2* Dq = Dg + (int64_t)qi * nn;
    double2* R = Rg + (int64_t)qi * nn;
    double* sc = scratch + (int64_t)qi * 4 * n;
    double *sd = sc, *se = sc + n, *sb = sc + 3 * n;
    for (int64_t t = tid; t < nn; t += nt) {
        const int i = (int)(t / n), j = (int)(t % n);
        const double2 a = Dq[(int64_t)i * n + j], b = Dq[(int64_t)j * n + i];
        A[t] = make_double2(0.5 * (a.x + b.x), i == j ? 0.0 : 0.5 * (a.y - b.y));
    }
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double s2 = 0.0;
        for (int i = 1 + tid; i < m; i += nt) { const double2 x = A[(k + 1 + i) * n + k]; s2 += x.x * x.x + x.y * x.y; }
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) red[warp] = s2;
        __syncthreads();
        double tail = 0.0;
        for (int w = 0; w < nw; ++w) tail += red[w];
        const double2 x0 = A[(k + 1) * n + k];
        const double a0 = hypot(x0.x, x0.y);
        double beta = 0.0;
        double2 alpha = x0, v0 = make_double2(0.0, 0.0);
        if (tail > 0.0) {
            const double nrm = sqrt(a0 * a0 + tail);
            const double2 u = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
            alpha = make_double2(-u.x * nrm, -u.y * nrm);
            v0 = make_double2(x0.x + u.x * nrm, x0.y + u.y * nrm);
            beta = 2.0 / (v0.x * v0.x + v0.y * v0.y + tail);
        }
        __syncthreads();                                     // all read x0 before it is replaced
        if (tid == 0) {
            se[2 * k] = alpha.x;
            se[2 * k + 1] = alpha.y;
            sb[k] = beta;
            A[(k + 1) * n + k] = v0;                         // v_0; v_i (i >= 1) = x_i in place
        }
        __syncthreads();
        for (int i = tid; i < m; i += nt) R[(int64_t)k * n + i] = A[(k + 1 + i) * n + k];
        if (beta != 0.0) {
            // p = beta A22 v (one warp per row), kept in row k (columns k+1..) as scratch
            for (int r = warp; r < m; r += nw) {
                double2 acc = make_double2(0.0, 0.0);
                for (int c = lane; c < m; c += 32) {
                    const double2 a = A[(k + 1 + r) * n + k + 1 + c], v = A[(k + 1 + c) * n + k];
                    acc.x += a.x * v.x - a.y * v.y;
                    acc.y += a.x * v.y + a.y * v.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                }
                if (lane == 0) A[k * n + k + 1 + r] = make_double2(beta * acc.x, beta * acc.y);
            }
            __syncthreads();
            double kr = 0.0;                                 // K = beta/2 v^H p (real)
            for (int c = tid; c < m; c += nt) {
                const double2 v = A[(k + 1 + c) * n + k], p = A[k * n + k + 1 + c];
                kr += v.x * p.x + v.y * p.y;
            }
            for (int o = 16; o > 0; o >>= 1) kr += __shfl_xor_sync(0xffffffffu, kr, o);
            if (lane == 0) red[warp] = kr;
            __syncthreads();
            double K = 0.0;
            for (int w = 0; w < nw; ++w) K += red[w];
            K *= 0.5 * beta;
            __syncthreads();
            for (int c = tid; c < m; c += nt) {              // w = p - K v
                const double2 v = A[(k + 1 + c) * n + k], p = A[k * n + k + 1 + c];
                A[k * n + k + 1 + c] = make_double2(p.x - K * v.x, p.y - K * v.y);
            }
            __syncthreads();
            for (int t = tid; t < m * m; t += nt) {          // A22 -= v w^H + w v^H
                const int r = t / m, c = t % m;
                const double2 vr = A[(k + 1 + r) * n + k], vc = A[(k + 1 + c) * n + k];
                const double2 wr = A[k * n + k + 1 + r], wc = A[k * n + k + 1 + c];
                const double re = vr.x * wc.x + vr.y * wc.y + wr.x * vc.x + wr.y * vc.y;
                const double im = vr.y * wc.x - vr.x * wc.y + wr.y * vc.x - wr.x * vc.y;
                double2& a = A[(k + 1 + r) * n + k + 1 + c];
                a.x -= re;
                a.y -= im;
            }
            __syncthreads();
        }
    }
    for (int k = tid; k < n; k += nt) sd[k] = A[k * n + k].x;
    if (tid == 0 && n >= 2) {                                // last subdiagonal (no reflector)
        const double2 a = A[(n - 1) * n + n - 2];
        se[2 * (n - 2)] = a.x;
        se[2 * (n - 2) + 1] = a.y;
        sb[n - 2] = 0.0;
    }
}

__global__ void __launch_bounds__(kQlThreads)
ql_back_kernel(const double2* __restrict__ Rg, const double* __restrict__ scratch, int n,
               double* __restrict__ freq, double2* __restrict__ evec, int32_t* __restrict__ status,
               const int32_t* __restrict__ skip) {
    if (skip && skip[blockIdx.x]) return;
    extern __shared__ double Z[];                            // real n x n, column-major
    __shared__ double d[kHhqlMaxModes], e[kHhqlMaxModes];
    __shared__ double rcb[2][kHhqlMaxModes], rsb[2][kHhqlMaxModes];   // rotations of two rounds
    __shared__ double2 ph[kHhqlMaxModes];
    __shared__ int rank_of[kHhqlMaxModes];
    __shared__ int sw_lo[2], sw_hi[2], sweep_fail;
    const int qi = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int64_t nn = (int64_t)n * n;
    const double2* R = Rg + (int64_t)qi * nn;
    const double* sc = scratch + (int64_t)qi * 4 * n;
    double2* Eo = evec + (int64_t)qi * nn;
    if (tid == 0) {
        double2 dl = make_double2(1.0, 0.0);
        for (int k = 0; k < n; ++k) d[k] = sc[k];
        for (int k = 0; k + 1 < n; ++k) {
            const double2 a = make_double2(sc[n + 2 * k], sc[n + 2 * k + 1]);
            const double m = hypot(a.x, a.y);
            e[k] = m;
            const double2 u = m > 0.0 ? make_double2(a.x / m, a.y / m) : make_double2(1.0, 0.0);
            ph[k] = dl;                                      // delta_k
            dl = make_double2(dl.x * u.x - dl.y * u.y, dl.x * u.y + dl.y * u.x);
        }
        ph[n - 1] = dl;
        e[n - 1] = 0.0;
        sweep_fail = 0;
    }
    for (int64_t t = tid; t < nn; t += nt) Z[t] = (t / n == t % n) ? 1.0 : 0.0;
    __syncthreads();
    // Symmetric tridiagonal QR iteration (Golub & Van Loan, "Matrix Computations", the implicit
    // symmetric QR step with Wilkinson shift inside the symmetric QR algorithm): every round
    // zeroes the negligible off-diagonals, takes the lowest unreduced block [lo, hi], and chases
    // one bulge from its top to its bottom with Givens rotations Q_k on rows/columns (k, k+1),
    // T <- Q_k T Q_k^T, Z <- Z Q_k^T.  The rounds are pipelined: warp 0 finds and chases round
    // r + 1 (it needs only d and e) while warps 1-3 apply the rotations of round r to the rows
    // of Z, one row per thread, from a second buffer.
    const int max_rounds = kQlMaxIter * (n > 0 ? n : 1);
    auto chase = [&](int b, int round) {
        // deflation test of every off-diagonal, lanes in parallel
        for (int k = lane; k + 1 < n; k += 32)
            if (fabs(e[k]) <= 2.2204460492503131e-16 * (fabs(d[k]) + fabs(d[k + 1]))) e[k] = 0.0;
        __syncwarp();
        int hk = -1;                                         // the last nonzero off-diagonal
        for (int k = lane; k + 1 < n; k += 32)
            if (e[k] != 0.0) hk = k;
        for (int o = 16; o > 0; o >>= 1) hk = max(hk, __shfl_xor_sync(0xffffffffu, hk, o));
        const int hi = hk + 1;
        int zk = -1;                                         // the last zero one below it
        for (int k = lane; k < hi - 1; k += 32)
            if (e[k] == 0.0) zk = k;
        for (int o = 16; o > 0; o >>= 1) zk = max(zk, __shfl_xor_sync(0xffffffffu, zk, o));
        const int lo = zk + 1;
        if (lane == 0) {
            if (hk < 0 || round >= max_rounds) {
                sw_lo[b] = sw_hi[b] = 0;                     // done (or given up)
                if (hk >= 0) sweep_fail = 1;
            } else {
                // Wilkinson shift: the eigenvalue of the block's trailing 2x2 nearer d[hi]
                const double dl = 0.5 * (d[hi - 1] - d[hi]), bq = e[hi - 1];
                const double den = dl + copysign(hypot(dl, bq), dl);
                const double mu = d[hi] - (den != 0.0 ? bq * (bq / den) : bq);
                double x = d[lo] - mu, z = e[lo];
                // d[k] and e[k] of the rotation in flight are carried in registers (each rotation
                // rewrites them for the next), so the serial chain touches shared memory only
                // for the incoming d[k+1], e[k+1] and the outgoing values
                double a = d[lo], bb = e[lo];
                for (int k = lo; k < hi; ++k) {
                    // Givens rotation from one reciprocal square root (the entries are far from
                    // the FP64 overflow and underflow limits, so |(x, z)|^2 is formed directly;
                    // GB300's FP64 pipe is narrow and this chain is the kernel's serial path)
                    const double r2 = fma(x, x, z * z);
                    const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;
                    const double r = r2 * ir;
                    const double c = r2 > 0.0 ? x * ir : 1.0, sn = r2 > 0.0 ? z * ir : 0.0;
                    if (k > lo) e[k - 1] = r;                    // the bulge at (k+1, k-1) folds into e[k-1]
                    const double dd = d[k + 1], en = k + 1 < hi ? e[k + 1] : 0.0;
                    d[k] = c * c * a + 2.0 * c * sn * bb + sn * sn * dd;
                    const double dk1 = sn * sn * a - 2.0 * c * sn * bb + c * c * dd;
                    const double ek = c * sn * (dd - a) + (c * c - sn * sn) * bb;
                    d[k + 1] = dk1;
                    e[k] = ek;
                    if (k + 1 < hi) {                            // new bulge at (k+2, k)
                        x = ek;
                        z = sn * en;
                        e[k + 1] = en * c;
                        a = dk1;
                        bb = en * c;
                    }
                    rcb[b][k] = c;
                    rsb[b][k] = sn;
                }
                sw_lo[b] = lo;
                sw_hi[b] = hi;
            }
        }
        __syncwarp();
    };
    if (warp == 0) chase(0, 0);
    __syncthreads();
    for (int round = 0;; ++round) {
        const int b = round & 1;
        const int lo = sw_lo[b], hi = sw_hi[b];
        if (hi <= lo) break;                                 // same decision in every thread
        if (warp == 0) {
            chase(b ^ 1, round + 1);
        } else {
            // Z <- Z Q_lo^T ... Q_{hi-1}^T on columns (k, k+1) of this thread's row: column k is
            // final after rotation k, column k+1 is carried to the next rotation in a register
            const int row = tid - 32;
            if (row < n) {
                double carry = Z[(int64_t)lo * n + row];
                for (int k = lo; k < hi; ++k) {
                    const double c = rcb[b][k], sn = rsb[b][k];
                    const double z1 = Z[(int64_t)(k + 1) * n + row];
                    Z[(int64_t)k * n + row] = c * carry + sn * z1;
                    carry = c * z1 - sn * carry;
                }
                Z[(int64_t)hi * n + row] = carry;
            }
        }
        __syncthreads();
    }
    if (tid == 0 && sweep_fail) atomicExch(status, (int)PHX_ERR_NUMERIC);
    for (int i = tid; i < n; i += nt) {
        int r = 0;
        const double li = d[i];
        for (int j = 0; j < n; ++j) r += (d[j] < li) || (d[j] == li && j < i);
        rank_of[i] = r;
        const double w2 = li * phx::kEvA2AmuToPs2;
        freq[(int64_t)qi * n + r] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / phx::kTwoPi;
    }
    __syncthreads();
    // E = H_0 ... H_{n-3} diag(delta) Z, column j written into the sorted output column
    for (int j = tid; j < n; j += nt) {
        const int dst = rank_of[j];
        for (int i = 0; i < n; ++i) {
            const double z = Z[(int64_t)j * n + i];
            Eo[(int64_t)i * n + dst] = make_double2(ph[i].x * z, ph[i].y * z);
        }
        for (int k = n - 3; k >= 0; --k) {
            const double beta = sc[3 * n + k];
            if (beta == 0.0) continue;
            const int m = n - k - 1;
            const double2* v = R + (int64_t)k * n;
            double2 s = make_double2(0.0, 0.0);
            for (int i = 0; i < m; ++i) {
                const double2 vi = v[i], x = Eo[(int64_t)(k + 1 + i) * n + dst];
                s.x += vi.x * x.x + vi.y * x.y;                  // conj(v) x
                s.y += vi.x * x.y - vi.y * x.x;
            }
            s.x *= beta;
            s.y *= beta;
            for (int i = 0; i < m; ++i) {
                const double2 vi = v[i];
                double2& x = Eo[(int64_t)(k + 1 + i) * n + dst];
                x.x -= vi.x * s.x - vi.y * s.y;
                x.y -= vi.x * s.y + vi.y * s.x;
            }
        }
    }
    __syncthreads();
    // gauge: largest-modulus component real positive (first index on ties); one warp per column
    for (int col = warp; col < n; col += nw) {
        double best = -1.0;
        int bi = 0;
        for (int i = lane; i < n; i += 32) {
            const double2 v = Eo[(int64_t)i * n + col];
            const double a = v.x * v.x + v.y * v.y;
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const double2 vm = Eo[(int64_t)bi * n + col];
        const double h = hypot(vm.x, vm.y);
        const double2 g = h > 0.0 ? make_double2(vm.x / h, -vm.y / h) : make_double2(1.0, 0.0);
        __syncwarp();
        for (int i = lane; i < n; i += 32) Eo[(int64_t)i * n + col] = cmul(Eo[(int64_t)i * n + col], g);
    }
}

// One CTA per q.  Y[q][a] = dD_a(q) E(q) (complex), E sorted by frequency.
__global__ void velocity_kernel(const double2* __restrict__ E, const double2* __restrict__ Y,
                                const double* __restrict__ freq, int n, double* __restrict__ vel,
                                double* __restrict__ vv, const int32_t* __restrict__ skip) {
    __shared__ int grp_lo[kMaxModes], grp_hi[kMaxModes];
    const int q = blockIdx.x;
    if (skip && skip[q]) return;
    const int64_t nn = (int64_t)n * n;
    const double* f = freq + (int64_t)q * n;
    if (threadIdx.x == 0) {
        double fm = 0.0;
        for (int i = 0; i < n; ++i) fm = fmax(fm, fabs(f[i]));
        const double tol = phx::kDegenerateRelTol * fmax(fm, 1e-30);
        int i = 0;
        while (i < n) {          // frequencies ascend: groups anchored at their first member
            int j = i + 1;
            while (j < n && f[j] - f[i] < tol) ++j;
            for (int k = i; k < j; ++k) { grp_lo[k] = i; grp_hi[k] = j; }
            i = j;
        }
    }
    __syncthreads();
    const double2* Eq = E + (int64_t)q * nn;
    for (int mu = threadIdx.x; mu < n; mu += blockDim.x) {
        const double w = f[mu] * phx::kTwoPi;
        double v[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) {
            const double2* Ya = Y + ((int64_t)q * 3 + a) * nn;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const double2 e = Eq[(int64_t)i * n + mu], y = Ya[(int64_t)i * n + mu];
                acc += e.x * y.x + e.y * y.y;        // Re(conj(e) y)
            }
            v[a] = w > 0.0 ? acc * phx::kEvA2AmuToPs2 / (2.0 * w) : 0.0;
        }
        if (vel)
            for (int a = 0; a < 3; ++a) vel[((int64_t)q * n + mu) * 3 + a] = v[a];
        if (vv) {
            double t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            const int lo = grp_lo[mu], hi = grp_hi[mu];
            const double w0 = f[lo] * phx::kTwoPi;
            if (w0 > 0.0) {
                for (int m1 = lo; m1 < hi; ++m1)
                    for (int m2 = lo; m2 < hi; ++m2) {
                        double2 G12[3], G21[3];     // G^a_{m1 m2}, G^a_{m2 m1}
                        for (int a = 0; a < 3; ++a) {
                            const double2* Ya = Y + ((int64_t)q * 3 + a) * nn;
                            double2 g12 = make_double2(0, 0), g21 = make_double2(0, 0);
                            for (int i = 0; i < n; ++i) {
                                const double2 e1 = Eq[(int64_t)i * n + m1], e2 = Eq[(int64_t)i * n + m2];
                                const double2 y1 = Ya[(int64_t)i * n + m1], y2 = Ya[(int64_t)i * n + m2];
                                g12.x += e1.x * y2.x + e1.y * y2.y; g12.y += e1.x * y2.y - e1.y * y2.x;
                                g21.x += e2.x * y1.x + e2.y * y1.y; g21.y += e2.x * y1.y - e2.y * y1.x;
                            }
                            G12[a] = g12; G21[a] = g21;
                        }
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b)
                                t[3 * a + b] += G12[a].x * G21[b].x - G12[a].y * G21[b].y;
                    }
                const double sc = phx::kEvA2AmuToPs2 * phx::kEvA2AmuToPs2 / (4.0 * w0 * w0 * (hi - lo));
                for (int k = 0; k < 9; ++k) t[k] *= sc;
            }
            for (int k = 0; k < 9; ++k) vv[((int64_t)q * n + mu) * 9 + k] = t[k];
        }
    }
}

// |x - nearest integer| below the tolerance of q-point identity (reduced coordinates)
__device__ __forceinline__ bool near_integer(double x) { return fabs(x - rint(x)) < 1e-9; }

// One warp per q_i: the first j (ascending, j < i) with q_j = q_i or q_j = -q_i mod G, found
// 32 candidates at a time with a ballot.  The classes are unions of two G-translate sets, so
// the first index met is the class minimum and every member finds the same one.
__global__ void __launch_bounds__(256)
tr_classes_kernel(const double* __restrict__ q_frac, int nq, int32_t* __restrict__ code, int32_t* __restrict__ skip) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nq) return;                                   // whole warp
    const double a0 = q_frac[3 * i], a1 = q_frac[3 * i + 1], a2 = q_frac[3 * i + 2];
    int rep = i, cj = 0;
    for (int j0 = 0; j0 < i; j0 += 32) {
        const int j = j0 + lane;
        bool same = false, neg = false;
        if (j < i) {
            const double b0 = q_frac[3 * j], b1 = q_frac[3 * j + 1], b2 = q_frac[3 * j + 2];
            same = near_integer(b0 - a0) && near_integer(b1 - a1) && near_integer(b2 - a2);
            neg = near_integer(b0 + a0) && near_integer(b1 + a1) && near_integer(b2 + a2);
        }
        const unsigned m = __ballot_sync(0xffffffffu, same || neg);
        if (m) {
            const int k = __ffs(m) - 1;
            rep = j0 + k;
            cj = __shfl_sync(0xffffffffu, (same ? 0 : 1), k);
            break;
        }
    }
    if (lane == 0) {
        code[i] = 2 * rep + cj;
        skip[i] = rep != i;
    }
}

// One CTA per q: copy (or conjugate) the representative's outputs into q's rows.
__global__ void __launch_bounds__(256)
tr_fill_kernel(const int32_t* __restrict__ code, int n, double* __restrict__ freq, double2* __restrict__ evec,
               double* __restrict__ vel, double* __restrict__ vv) {
    const int i = blockIdx.x;
    const int c = code[i], r = c >> 1;
    if (r == i) return;
    const bool cj = (c & 1) != 0;
    const int64_t nn = (int64_t)n * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) freq[(int64_t)i * n + k] = freq[(int64_t)r * n + k];
    for (int64_t k = threadIdx.x; k < nn; k += blockDim.x) {
        double2 e = evec[(int64_t)r * nn + k];
        if (cj) e.y = -e.y;
        evec[(int64_t)i * nn + k] = e;
    }
    if (vel)
        for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) {
            const double v = vel[(int64_t)r * 3 * n + k];
            vel[(int64_t)i * 3 * n + k] = cj ? -v : v;
        }
    if (vv)
        for (int k = threadIdx.x; k < 9 * n; k += blockDim.x) vv[(int64_t)i * 9 * n + k] = vv[(int64_t)r * 9 * n + k];
}

}  // namespace

cudaError_t phx_launch_tr_classes(const double* q_frac, int nq, int32_t* code, int32_t* skip, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    tr_classes_kernel<<<(int)(((int64_t)nq * 32 + 255) / 256), 256, 0, s>>>(q_frac, nq, code, skip);
    return cudaGetLastError();
}

cudaError_t phx_launch_tr_fill(const int32_t* code, int nq, int n, double* freq, double* evec, double* vel,
                               double* vv, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    tr_fill_kernel<<<nq, 256, 0, s>>>(code, n, freq, (double2*)evec, vel, vv);
    return cudaGetLastError();
}

cudaError_t phx_launch_dynmat(const double* q_frac, int nq, int n_atoms, const int32_t* blk_idx,
                              const double* blk_val, const int32_t* pair_start, const double* masses,
                              const double* lattice, double* D, double* dD, cudaStream_t s, const int32_t* skip) {
    if (nq <= 0) return cudaSuccess;
    dynmat_kernel<<<nq, 256, 0, s>>>(q_frac, n_atoms, blk_idx, blk_val, pair_start, masses, lattice,
                                     (double2*)D, (double2*)dD, skip);
    return cudaGetLastError();
}

cudaError_t phx_launch_jacobi(double* A, double* V, int n, int nq, double* freq, double* evec,
                              int32_t* status, cudaStream_t s, double* scratch, const int32_t* skip) {
    if (nq <= 0) return cudaSuccess;
    if (n > kMaxModes) return cudaErrorInvalidValue;
    const size_t smem = (size_t)n * n * sizeof(double2);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (n <= kHhqlMaxModes && scratch && !std::getenv("PHX_EIG_JACOBI")) {
        // Householder reduction (reflectors into V's buffer), then QL + back-transformation
        // with Z (real) in A's buffer
        cudaError_t e = cudaFuncSetAttribute(hh_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        hh_reduce_kernel<<<nq, 256, smem, s>>>((const double2*)A, (double2*)V, scratch, n, skip);
        // Z (real n x n) in shared memory
        const size_t zbytes = (size_t)n * n * sizeof(double);
        e = cudaFuncSetAttribute(ql_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes);
        if (e != cudaSuccess) return e;
        ql_back_kernel<<<nq, kQlThreads, zbytes, s>>>((const double2*)V, scratch, n, freq, (double2*)evec, status,
                                                      skip);
        return cudaGetLastError();
    }
    const size_t static_bytes = 8 * 1024;     // rotation tables etc. (upper bound)
    if (smem + static_bytes <= (size_t)optin) {
        cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_kernel<true><<<nq, kJacobiThreads, smem, s>>>((double2*)A, (double2*)V, n, freq,
                                                             (double2*)evec, status, skip);
    } else {
        jacobi_kernel<false><<<nq, kJacobiThreads, 0, s>>>((double2*)A, (double2*)V, n, freq,
                                                           (double2*)evec, status, skip);
    }
    return cudaGetLastError();
}

cudaError_t phx_launch_velocity(const double* evec, const double* Y, const double* freq, int n,
                                int nq, double* vel, double* vv, cudaStream_t s, const int32_t* skip) {
    if (nq <= 0) return cudaSuccess;
    velocity_kernel<<<nq, 128, 0, s>>>((const double2*)evec, (const double2*)Y, freq, n, vel, vv, skip);
    return cudaGetLastError();
}
