// C-ABI entry points of libphx: argument validation, host-side preparation, staging of
// host buffers, and dispatch to the kernels.  See include/phx.h for the contract.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <numeric>
#include <set>
#include <tuple>

#include "common.h"

phx_status phx_gamma_tc_multi_t(phx_ctx* ctx, const phx_fc3* f, const double* freq, const double* evec,
                                const double* nB, int n_t, const int32_t* irr_host, int n_irr, const GammaParams& gp,
                                int prec, double* gacc, cudaStream_t s);
constexpr int kTPerPass = 4;     // temperatures per tensor-core pass (the epilogue's occupation tables)

phx_status phx_set_error(phx_ctx* ctx, phx_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

void* phx_ws(phx_ctx* ctx, const char* name, size_t bytes) {
    auto it = ctx->ws.find(name);
    if (it != ctx->ws.end() && it->second.second >= bytes) return it->second.first;
    if (it != ctx->ws.end()) {
        cudaDeviceSynchronize();            // the old buffer may still be in use by queued work
        cudaFree(it->second.first);
        ctx->ws.erase(it);
        if (ctx->graph_exec) {              // a cached batch graph points at the old buffer
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
            ctx->graph_key.clear();
        }
    }
    void* p = nullptr;
    size_t sz = std::max<size_t>(bytes, 256);
    if (cudaMalloc(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        phx_set_error(ctx, PHX_ERR_NOMEM, "cudaMalloc of %zu bytes for workspace '%s' failed", sz, name);
        return nullptr;
    }
    ctx->ws[name] = {p, sz};
    return p;
}

static cudaEvent_t pool_get(phx_ctx* ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

int phx_prof_begin(phx_ctx* ctx, cudaStream_t s) {
    if (!ctx->prof) return -1;
    phx_ctx::Rec r{0, pool_get(ctx), pool_get(ctx), 0.0, 0.0};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    ctx->recs.push_back(r);
    return (int)ctx->recs.size() - 1;
}

void phx_prof_end(phx_ctx* ctx, int slot, cudaStream_t s, int kernel, double flops, double bytes) {
    if (slot < 0) return;
    auto& r = ctx->recs[slot];
    r.kernel = kernel;
    r.flops = flops;
    r.bytes = bytes;
    cudaEventRecord(r.b, s);
}

namespace {

__global__ void finalize_gamma_kernel(int count, int n, const int32_t* irr, const double* freq,
                                      const double* gacc, const double* wacc, double pref, double inv_nq,
                                      double f_min, double* gamma, double* wp2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int s = i / n, nu = i % n;
        const double f = freq[(int64_t)irr[s] * n + nu];
        const bool ok = f >= f_min;
        gamma[i] = ok ? pref * gacc[i] : 0.0;
        if (wp2) wp2[i] = ok ? inv_nq * wacc[i] : 0.0;
    }
}

}  // namespace

cudaError_t phx_launch_finalize(int count, int n, const int32_t* irr, const double* freq, const double* gacc,
                                const double* wacc, double pref, double inv_nq, double f_min, double* gamma,
                                double* wp2, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    finalize_gamma_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, n, irr, freq, gacc, wacc, pref, inv_nq, f_min,
                                                            gamma, wp2);
    return cudaGetLastError();
}

namespace {

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" {

const char* phx_version(void) { return "phx 1.0 sm_103a"; }

phx_status phx_create(phx_ctx** out, int device) {
    if (!out) return PHX_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return PHX_ERR_CUDA;
    }
    if (device < 0 || device >= count) return PHX_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return PHX_ERR_CUDA;
    phx_ctx* c = new phx_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    if (cudaMalloc(&c->status_word, 64) != cudaSuccess) {
        delete c;
        return PHX_ERR_NOMEM;
    }
    cudaMemset(c->status_word, 0, 64);
    *out = c;
    return PHX_OK;
}

void phx_destroy(phx_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->ws) cudaFree(kv.second.first);
    cudaFree(ctx->status_word);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    for (cudaEvent_t e : ctx->side_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    delete ctx;
}

const char* phx_last_error(const phx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static void prof_collect(phx_ctx* ctx) {
    for (auto& r : ctx->recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.kernel] += ms;
            ctx->prof_n[r.kernel] += 1;
            ctx->prof_flops[r.kernel] += r.flops;
            ctx->prof_bytes[r.kernel] += r.bytes;
        }
        cudaGetLastError();
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
}

phx_status phx_set_option(phx_ctx* ctx, int32_t option, int64_t value) {
    if (!ctx) return PHX_ERR_INVALID;
    switch (option) {
        case PHX_OPT_CHAIN:
            if (value < 0 || value > 2) return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_CHAIN %lld", (long long)value);
            ctx->opt_chain = (int)value;
            return PHX_OK;
        case PHX_OPT_WAIT_LIMIT_NS:
            if (value < 1000 || value > 60000000000ll)
                return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_WAIT_LIMIT_NS %lld outside [1e3, 6e10]", (long long)value);
            ctx->opt_wait_ns = (unsigned long long)value;
            return PHX_OK;
        case PHX_OPT_STARVE:
            ctx->opt_starve = value != 0;
            return PHX_OK;
        case PHX_OPT_SIDE_SMS:
            if (value < -1 || value > 76) return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_SIDE_SMS %lld", (long long)value);
            ctx->opt_side_sms = (int)value;
            return PHX_OK;
        case PHX_OPT_VEL_FP32:
            if (value < 0 || value > 1) return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_VEL_FP32 %lld", (long long)value);
            ctx->opt_vel_fp32 = (int)value;
            return PHX_OK;
        case PHX_OPT_PAIR:
            if (value < 0 || value > 1) return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_PAIR %lld", (long long)value);
            ctx->opt_pair = (int)value;
            return PHX_OK;
        case PHX_OPT_HARMONIC_TR:
            if (value < 0 || value > 1)
                return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_HARMONIC_TR %lld", (long long)value);
            ctx->opt_harm_tr = (int)value;
            return PHX_OK;
        case PHX_OPT_SC_MATRIX_FREE:
            if (value < 0 || value > 2)
                return phx_set_error(ctx, PHX_ERR_INVALID, "PHX_OPT_SC_MATRIX_FREE %lld", (long long)value);
            ctx->opt_sc_mfree = (int)value;
            return PHX_OK;
        default:
            return phx_set_error(ctx, PHX_ERR_INVALID, "unknown option %d", option);
    }
}

phx_status phx_get_option(phx_ctx* ctx, int32_t option, int64_t* value) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!value) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_get_option: null value");
    switch (option) {
        case PHX_OPT_CHAIN: *value = ctx->opt_chain; return PHX_OK;
        case PHX_OPT_WAIT_LIMIT_NS: *value = (int64_t)ctx->opt_wait_ns; return PHX_OK;
        case PHX_OPT_STARVE: *value = ctx->opt_starve; return PHX_OK;
        case PHX_OPT_PAIR: *value = ctx->opt_pair; return PHX_OK;
        case PHX_OPT_SIDE_SMS: *value = phx_side_sms(ctx); return PHX_OK;
        case PHX_OPT_VEL_FP32: *value = ctx->opt_vel_fp32; return PHX_OK;
        case PHX_OPT_HARMONIC_TR: *value = ctx->opt_harm_tr; return PHX_OK;
        case PHX_OPT_SC_MATRIX_FREE: *value = ctx->opt_sc_mfree; return PHX_OK;
        default: return phx_set_error(ctx, PHX_ERR_INVALID, "unknown option %d", option);
    }
}

phx_status phx_profile_enable(phx_ctx* ctx, int32_t on) {
    if (!ctx) return PHX_ERR_INVALID;
    cudaSetDevice(ctx->device);
    prof_collect(ctx);
    for (int k = 0; k < PHX_K_COUNT; ++k) {
        ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; ctx->prof_flops[k] = 0.0; ctx->prof_bytes[k] = 0.0;
    }
    ctx->launches = 0;
    ctx->prof = on != 0;
    return PHX_OK;
}

phx_status phx_profile_read(phx_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches, double* flops,
                            double* bytes) {
    if (!ctx || kernel < -1 || kernel >= PHX_K_COUNT) return PHX_ERR_INVALID;
    cudaSetDevice(ctx->device);
    prof_collect(ctx);
    if (kernel == -1) {
        if (launches) *launches = ctx->launches;
        if (total_ms) *total_ms = 0.0;
        if (flops) *flops = 0.0;
        if (bytes) *bytes = 0.0;
        return PHX_OK;
    }
    if (total_ms) *total_ms = ctx->prof_ms[kernel];
    if (launches) *launches = ctx->prof_n[kernel];
    if (flops) *flops = ctx->prof_flops[kernel];
    if (bytes) *bytes = ctx->prof_bytes[kernel];
    return PHX_OK;
}

// ---------------------------------------------------------------- grid

phx_status phx_irreducible(const int32_t mesh[3], int32_t n_rot, const int32_t* rot, int32_t* irr,
                           int32_t* n_irr, int32_t* full_to_irr, int32_t* weight) {
    if (!mesh || !irr || !n_irr || !full_to_irr || !weight || n_rot < 0 || (n_rot > 0 && !rot))
        return PHX_ERR_INVALID;
    const int m1 = mesh[0], m2 = mesh[1], m3 = mesh[2];
    if (m1 <= 0 || m2 <= 0 || m3 <= 0) return PHX_ERR_INVALID;
    const int nq = m1 * m2 * m3;
    // group: the rotations and their negatives (time reversal); identity always included
    std::vector<std::array<int, 9>> ops;
    ops.push_back({1, 0, 0, 0, 1, 0, 0, 0, 1});
    ops.push_back({-1, 0, 0, 0, -1, 0, 0, 0, -1});
    for (int r = 0; r < n_rot; ++r) {
        std::array<int, 9> a, b;
        for (int k = 0; k < 9; ++k) { a[k] = rot[9 * r + k]; b[k] = -rot[9 * r + k]; }
        ops.push_back(a);
        ops.push_back(b);
    }
    auto apply = [&](const std::array<int, 9>& R, int k1, int k2, int k3, int* o1, int* o2, int* o3) {
        // q_red = k / m; R q_red must again lie on the mesh: (R k)_i * m_j / m_i integral
        long x[3];
        const int kk[3] = {k1, k2, k3}, mm[3] = {m1, m2, m3};
        for (int i = 0; i < 3; ++i) {
            // (R q)_i = sum_j R_ij k_j / m_j ; mesh coordinate = m_i * that
            long num = 0;
            long den = 1;
            for (int j = 0; j < 3; ++j) den = std::lcm(den, (long)mm[j]);
            for (int j = 0; j < 3; ++j) num += (long)R[3 * i + j] * kk[j] * (den / mm[j]);
            const long t = num * mm[i];
            if (t % den != 0) return false;
            x[i] = ((t / den) % mm[i] + mm[i]) % mm[i];
        }
        *o1 = (int)x[0]; *o2 = (int)x[1]; *o3 = (int)x[2];
        return true;
    };
    std::vector<int> rep(nq, -1);
    for (int i = 0; i < nq; ++i) {
        if (rep[i] >= 0) continue;
        const int k1 = i / (m2 * m3), k2 = (i / m3) % m2, k3 = i % m3;
        std::vector<int> orbit;
        for (const auto& R : ops) {
            int o1, o2, o3;
            if (!apply(R, k1, k2, k3, &o1, &o2, &o3)) return PHX_ERR_INVALID;
            orbit.push_back((o1 * m2 + o2) * m3 + o3);
        }
        const int mn = *std::min_element(orbit.begin(), orbit.end());
        // smallest index of the orbit: every member of an orbit is reached from every other
        for (int j : orbit) rep[j] = mn;
    }
    // orbits computed from each representative only: make every point point to the
    // smallest index of its whole orbit (union through representatives)
    for (int pass = 0; pass < 4; ++pass)
        for (int i = 0; i < nq; ++i) rep[i] = std::min(rep[i], rep[rep[i]]);
    std::vector<int> reps;
    for (int i = 0; i < nq; ++i)
        if (rep[i] == i) reps.push_back(i);
    std::vector<int> pos(nq, -1);
    for (size_t p = 0; p < reps.size(); ++p) pos[reps[p]] = (int)p;
    for (size_t p = 0; p < reps.size(); ++p) { irr[p] = reps[p]; weight[p] = 0; }
    for (int i = 0; i < nq; ++i) {
        const int p = pos[rep[i]];
        if (p < 0) return PHX_ERR_INVALID;
        full_to_irr[i] = p;
        weight[p] += 1;
    }
    *n_irr = (int32_t)reps.size();
    return PHX_OK;
}

// ---------------------------------------------------------------- harmonic

phx_status phx_harmonic(phx_ctx* ctx, const phx_cell* cell, const phx_ifc2* fc2, const double* q_frac,
                        int32_t nq, double* freq_thz, double* evec, double* vel, double* vv, int32_t mem,
                        void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!cell || !fc2 || !cell->masses || (nq > 0 && (!q_frac || !freq_thz || !evec)))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_harmonic: null argument");
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_harmonic: bad mem flag %d", mem);
    const int na = cell->n_atoms, n = 3 * na;
    if (na <= 0 || n > kPhxMaxLargeModes)
        return phx_set_error(ctx, PHX_ERR_UNSUPPORTED, "phx_harmonic: n_atoms=%d (need 1..%d)", na,
                             kPhxMaxLargeModes / 3);
    if (nq < 0) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_harmonic: nq < 0");
    if (nq == 0) return PHX_OK;
    // cells above 64 atoms: the large real-symmetric solver, Gamma point only, no velocities
    const bool large = n > 192;
    if (large) {
        if (vel || vv)
            return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                                 "phx_harmonic: velocities need n_atoms <= 64 (larger cells are solved at Gamma)");
        std::vector<double> hq((size_t)nq * 3);
        if (mem == PHX_MEM_DEVICE) {
            cudaSetDevice(ctx->device);
            PHX_CUDA_CHECK(ctx, cudaMemcpy(hq.data(), q_frac, hq.size() * 8, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(hq.data(), q_frac, hq.size() * 8);
        }
        for (double v : hq)
            if (!(std::fabs(v - std::nearbyint(v)) < 1e-12))
                return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                                     "phx_harmonic: cells above 64 atoms are solved at Gamma only (q = %g)", v);
    }
    for (int i = 0; i < na; ++i)
        if (!(cell->masses[i] > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "mass %d not positive", i);
    const int nb = fc2->n_blocks;
    if (nb < 0 || (nb > 0 && (!fc2->idx || !fc2->val))) return phx_set_error(ctx, PHX_ERR_INVALID, "bad fc2");
    if (!finite_all(fc2->val, (size_t)nb * 9)) return phx_set_error(ctx, PHX_ERR_INVALID, "fc2 not finite");
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);

    // sort blocks by atom pair, CSR over pairs
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    for (int b = 0; b < nb; ++b) {
        const int i = fc2->idx[5 * b], j = fc2->idx[5 * b + 1];
        if (i < 0 || i >= na || j < 0 || j >= na)
            return phx_set_error(ctx, PHX_ERR_INVALID, "fc2 block %d atom index out of range", b);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return std::make_pair(fc2->idx[5 * x], fc2->idx[5 * x + 1]) < std::make_pair(fc2->idx[5 * y], fc2->idx[5 * y + 1]);
    });
    std::vector<int32_t> sidx((size_t)nb * 5), pstart((size_t)na * na + 1, 0);
    std::vector<double> sval((size_t)nb * 9);
    for (int k = 0; k < nb; ++k) {
        const int b = order[k];
        std::memcpy(&sidx[5 * k], &fc2->idx[5 * b], 5 * sizeof(int32_t));
        std::memcpy(&sval[9 * k], &fc2->val[9 * b], 9 * sizeof(double));
        pstart[(size_t)fc2->idx[5 * b] * na + fc2->idx[5 * b + 1] + 1] += 1;
    }
    for (size_t p = 0; p < (size_t)na * na; ++p) pstart[p + 1] += pstart[p];

    int32_t* d_idx = (int32_t*)phx_ws(ctx, "h.idx", sidx.size() * 4);
    double* d_val = (double*)phx_ws(ctx, "h.val", sval.size() * 8);
    int32_t* d_ps = (int32_t*)phx_ws(ctx, "h.ps", pstart.size() * 4);
    double* d_m = (double*)phx_ws(ctx, "h.m", (size_t)na * 8);
    double* d_lat = (double*)phx_ws(ctx, "h.lat", 9 * 8);
    if (!d_idx || !d_val || !d_ps || !d_m || !d_lat) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_idx, sidx.data(), sidx.size() * 4, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_val, sval.data(), sval.size() * 8, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_ps, pstart.data(), pstart.size() * 4, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_m, cell->masses, (size_t)na * 8, cudaMemcpyHostToDevice, s));
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(d_lat, cell->lattice, 9 * 8, cudaMemcpyHostToDevice, s));

    const double* dq = nullptr;
    PHX_TRY(phx_stage_in(ctx, "h.q", q_frac, (size_t)nq * 3, mem, s, &dq));
    double *o_f = nullptr, *o_e = nullptr, *o_v = nullptr, *o_vv = nullptr;
    const int64_t n2 = (int64_t)n * n;
    PHX_TRY(phx_stage_out_buf(ctx, "h.of", freq_thz, (size_t)nq * n, mem, &o_f));
    PHX_TRY(phx_stage_out_buf(ctx, "h.oe", evec, (size_t)nq * n2 * 2, mem, &o_e));
    if (vel) PHX_TRY(phx_stage_out_buf(ctx, "h.ov", vel, (size_t)nq * n * 3, mem, &o_v));
    if (vv) PHX_TRY(phx_stage_out_buf(ctx, "h.ovv", vv, (size_t)nq * n * 9, mem, &o_vv));
    const bool want_v = vel || vv;

    if (large) {
        PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));
        for (int q = 0; q < nq; ++q)
            PHX_TRY(phx_eigh_gamma_large(ctx, na, d_val, d_ps, d_m, o_f + (int64_t)q * n, o_e + (int64_t)q * n2 * 2, s));
    }
    // q chunks bounded to ~1 GB of work buffers
    const int64_t per_q = n2 * 16 * (want_v ? 8 : 2);
    const int chunk = large ? 0 : (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)nq, ((int64_t)1 << 30) / per_q, (int64_t)16384}));
    double* D = large ? nullptr : (double*)phx_ws(ctx, "h.D", (size_t)chunk * n2 * 16);
    double* hsc = large ? nullptr : (double*)phx_ws(ctx, "h.hsc", (size_t)chunk * n * 4 * 8);
    double* Vw = large ? nullptr : (double*)phx_ws(ctx, "h.V", (size_t)chunk * n2 * 16);
    double* dD = want_v ? (double*)phx_ws(ctx, "h.dD", (size_t)chunk * 3 * n2 * 16) : nullptr;
    double* Y = want_v ? (double*)phx_ws(ctx, "h.Y", (size_t)chunk * 3 * n2 * 16) : nullptr;
    if (!large && (!D || !Vw || !hsc || (want_v && (!dD || !Y)))) return PHX_ERR_NOMEM;
    if (!large) PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));
    // time reversal (Eq. (dynmat_reciprocal): D(-q) = conj D(q)): one q of every {q, -q} pair of
    // the list is solved, the other filled from it after the loop
    int32_t *tr_code = nullptr, *tr_skip = nullptr;
    if (!large && ctx->opt_harm_tr && nq > 1) {
        tr_code = (int32_t*)phx_ws(ctx, "h.trc", (size_t)nq * 4);
        tr_skip = (int32_t*)phx_ws(ctx, "h.trs", (size_t)nq * 4);
        if (!tr_code || !tr_skip) return PHX_ERR_NOMEM;
        PHX_CUDA_CHECK(ctx, phx_launch_tr_classes(dq, nq, tr_code, tr_skip, s));
        ctx->launches += 1;
    }
    for (int q0 = 0; !large && q0 < nq; q0 += chunk) {
        const int c = std::min(chunk, nq - q0);
        const int32_t* skip = tr_skip ? tr_skip + q0 : nullptr;
        PHX_CUDA_CHECK(ctx, phx_launch_dynmat(dq + 3 * q0, c, na, d_idx, d_val, d_ps, d_m, d_lat, D, dD, s, skip));
        const int ps = phx_prof_begin(ctx, s);
        PHX_CUDA_CHECK(ctx, phx_launch_jacobi(D, Vw, n, c, o_f + (int64_t)q0 * n, o_e + (int64_t)q0 * n2 * 2,
                                              (int32_t*)ctx->status_word, s, hsc, skip));
        phx_prof_end(ctx, ps, s, PHX_K_EIGEN, 0.0, 0.0);
        ctx->launches += 2;
        if (want_v) {
            ZgemmBatch p{};
            p.A = dD; p.strideA = n2; p.divA = 1;
            p.B = o_e + (int64_t)q0 * n2 * 2; p.strideB = n2; p.divB = 3;
            p.C = Y; p.strideC = n2;
            p.lda = n; p.ldb = n; p.ldc = n;
            p.fp32 = ctx->opt_vel_fp32;
            p.skip = skip; p.skip_div = 3;
            PHX_CUDA_CHECK(ctx, phx_launch_zgemm(n, n, n, 3 * c, p, s));
            PHX_CUDA_CHECK(ctx, phx_launch_velocity(o_e + (int64_t)q0 * n2 * 2, Y, o_f + (int64_t)q0 * n, n, c,
                                                    o_v ? o_v + (int64_t)q0 * n * 3 : nullptr,
                                                    o_vv ? o_vv + (int64_t)q0 * n * 9 : nullptr, s, skip));
            ctx->launches += 2;
        }
    }
    if (tr_code) {
        PHX_CUDA_CHECK(ctx, phx_launch_tr_fill(tr_code, nq, n, o_f, o_e, o_v, o_vv, s));
        ctx->launches += 1;
    }
    int32_t st = 0;
    if (mem == PHX_MEM_HOST) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(freq_thz, o_f, (size_t)nq * n * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(evec, o_e, (size_t)nq * n2 * 16, cudaMemcpyDeviceToHost, s));
        if (vel) PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(vel, o_v, (size_t)nq * n * 3 * 8, cudaMemcpyDeviceToHost, s));
        if (vv) PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(vv, o_vv, (size_t)nq * n * 9 * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_harmonic: eigensolver did not converge");
    }
    return PHX_OK;
}

// ---------------------------------------------------------------- third-order IFCs

phx_status phx_fc3_create(phx_ctx* ctx, const phx_cell* cell, const phx_ifc3* fc3, const int32_t mesh[3],
                          phx_fc3** out) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!cell || !fc3 || !mesh || !out || !cell->masses)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_fc3_create: null argument");
    *out = nullptr;
    const int na = cell->n_atoms, n = 3 * na;
    if (na <= 0) return phx_set_error(ctx, PHX_ERR_INVALID, "n_atoms <= 0");
    if (mesh[0] <= 0 || mesh[1] <= 0 || mesh[2] <= 0) return phx_set_error(ctx, PHX_ERR_INVALID, "bad mesh");
    const int64_t nnz = fc3->nnz;
    if (nnz < 0 || (nnz > 0 && (!fc3->idx || !fc3->val))) return phx_set_error(ctx, PHX_ERR_INVALID, "bad fc3");
    if (!finite_all(fc3->val, (size_t)nnz)) return phx_set_error(ctx, PHX_ERR_INVALID, "fc3 not finite");
    for (int i = 0; i < na; ++i)
        if (!(cell->masses[i] > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "mass %d not positive", i);
    cudaSetDevice(ctx->device);
    const int m1 = mesh[0], m2 = mesh[1], m3 = mesh[2];
    auto md = [](int v, int m) { return ((v % m) + m) % m; };
    // distinct folded d = R' - R''
    std::vector<int> dkey(nnz);
    std::set<int> dset;
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t* e = fc3->idx + 9 * k;
        for (int c = 0; c < 3; ++c)
            if (e[c] < 0 || e[c] >= n) return phx_set_error(ctx, PHX_ERR_INVALID, "fc3 entry %lld index out of range", (long long)k);
        const int d1 = md(e[3] - e[6], m1), d2 = md(e[4] - e[7], m2), d3 = md(e[5] - e[8], m3);
        dkey[k] = (d1 * m2 + d2) * m3 + d3;
        dset.insert(dkey[k]);
    }
    std::vector<int> dlist(dset.begin(), dset.end());
    std::vector<int> dpos(m1 * m2 * m3, -1);
    for (size_t i = 0; i < dlist.size(); ++i) dpos[dlist[i]] = (int)i;
    std::vector<int64_t> order(nnz);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const int32_t* a = fc3->idx + 9 * x;
        const int32_t* b = fc3->idx + 9 * y;
        return std::make_tuple(dpos[dkey[x]], a[1], a[2], a[0]) < std::make_tuple(dpos[dkey[y]], b[1], b[2], b[0]);
    });
    std::vector<int32_t> seg_key, ent_a(nnz), ent_r2((size_t)nnz * 3);
    std::vector<int64_t> seg_start;
    std::vector<double> ent_w(nnz);
    std::tuple<int, int, int> last{-1, -1, -1};
    for (int64_t k = 0; k < nnz; ++k) {
        const int64_t o = order[k];
        const int32_t* e = fc3->idx + 9 * o;
        const auto key = std::make_tuple(dpos[dkey[o]], (int)e[1], (int)e[2]);
        if (key != last) {
            seg_key.push_back(std::get<0>(key));
            seg_key.push_back(std::get<1>(key));
            seg_key.push_back(std::get<2>(key));
            seg_start.push_back(k);
            last = key;
        }
        ent_a[k] = e[0];
        ent_r2[3 * k] = e[6]; ent_r2[3 * k + 1] = e[7]; ent_r2[3 * k + 2] = e[8];
        const double ma = cell->masses[e[0] / 3], mb = cell->masses[e[1] / 3], mc = cell->masses[e[2] / 3];
        ent_w[k] = fc3->val[o] / std::sqrt(ma * mb * mc);
    }
    seg_start.push_back(nnz);
    std::vector<int32_t> d_int(dlist.size() * 3);
    for (size_t i = 0; i < dlist.size(); ++i) {
        d_int[3 * i] = dlist[i] / (m2 * m3);
        d_int[3 * i + 1] = (dlist[i] / m3) % m2;
        d_int[3 * i + 2] = dlist[i] % m3;
    }
    phx_fc3* h = new phx_fc3();
    h->ctx = ctx;
    h->n = n;
    h->mesh[0] = m1; h->mesh[1] = m2; h->mesh[2] = m3;
    h->nq = m1 * m2 * m3;
    h->n_d = (int)dlist.size();
    h->nnz = nnz;
    h->n_seg = (int64_t)seg_start.size() - 1;
    auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
        if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        return bytes == 0 || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up((void**)&h->d_int, d_int.data(), d_int.size() * 4) &&
              up((void**)&h->seg_key, seg_key.data(), seg_key.size() * 4) &&
              up((void**)&h->seg_start, seg_start.data(), seg_start.size() * 8) &&
              up((void**)&h->ent_a, ent_a.data(), ent_a.size() * 4) &&
              up((void**)&h->ent_r2, ent_r2.data(), ent_r2.size() * 4) &&
              up((void**)&h->ent_w, ent_w.data(), ent_w.size() * 8);
    if (!ok) {
        cudaGetLastError();
        phx_fc3_destroy(h);
        return phx_set_error(ctx, PHX_ERR_NOMEM, "phx_fc3_create: device upload failed");
    }
    if (m1 == 1 && m2 == 1 && m3 == 1) {
        const phx_status st = phx_fc3_prepare_cell(ctx, cell, fc3, h);
        if (st != PHX_OK) {
            phx_fc3_destroy(h);
            return st;
        }
    }
    *out = h;
    return PHX_OK;
}

void phx_fc3_destroy(phx_fc3* h) {
    if (!h) return;
    cudaFree(h->d_int); cudaFree(h->seg_key); cudaFree(h->seg_start);
    cudaFree(h->ent_a); cudaFree(h->ent_r2); cudaFree(h->ent_w);
    cudaFree(h->tc_bc_start); cudaFree(h->tc_ent_ad); cudaFree(h->tc_ent_src);
    cudaFree(h->g0_nbr_start); cudaFree(h->g0_nbr_atom); cudaFree(h->g0_seg_start);
    cudaFree(h->g0_ent_i); cudaFree(h->g0_ent_w);
    delete h;
}

int32_t phx_fc3_num_d(const phx_fc3* h) { return h ? h->n_d : -1; }

// ---------------------------------------------------------------- scattering

phx_status phx_gamma(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz, const double* evec,
                     const int32_t* irr_q, int32_t n_irr, double temperature, phx_broadening br,
                     double f_min_thz, int32_t prec, double* gamma, double* wp2, int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!fc3 || fc3->ctx != ctx) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: fc3 handle from another context");
    if (n_irr < 0) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: n_irr < 0");
    if (n_irr == 0) return PHX_OK;
    if (!freq_thz || !evec || !irr_q || !gamma) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: null argument");
    if (!(temperature > 0.0) || !(br.sigma_thz > 0.0) || !(br.window > 0.0) || !(f_min_thz > 0.0) ||
        !std::isfinite(f_min_thz) || !std::isfinite(temperature))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: T, sigma, window and f_min must be finite and > 0");
    if (br.shape != PHX_GAUSS && br.shape != PHX_LORENTZ)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: unknown broadening shape %d", br.shape);
    if (prec != PHX_FP64 && prec != PHX_TF32 && prec != PHX_BF16X3)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: unknown precision %d", prec);
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: bad mem flag %d", mem);
    if (fc3->nq == 1 && fc3->n > 192) {
        // cells above 64 atoms at Gamma: the large-cell path (one irreducible point, no WP2)
        if (n_irr != 1 || wp2)
            return phx_set_error(ctx, PHX_ERR_UNSUPPORTED,
                                 "phx_gamma: a Gamma-only cell above 64 atoms takes n_irr = 1 and no wp2");
        int32_t q0 = 0;
        if (mem == PHX_MEM_HOST) {
            q0 = irr_q[0];
        } else {
            cudaSetDevice(ctx->device);
            PHX_CUDA_CHECK(ctx, cudaMemcpy(&q0, irr_q, 4, cudaMemcpyDeviceToHost));
        }
        if (q0 != 0) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: irr_q[0]=%d outside the mesh", q0);
        return phx_gamma_cell(ctx, fc3, freq_thz, evec, temperature, br, f_min_thz, prec, gamma, mem, stream);
    }
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    const int n = fc3->n, nq = fc3->nq;
    const int64_t n2 = (int64_t)n * n;

    std::vector<int32_t> irr_h(n_irr);
    if (mem == PHX_MEM_HOST) {
        std::memcpy(irr_h.data(), irr_q, n_irr * 4);
    } else {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(irr_h.data(), irr_q, n_irr * 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    for (int i = 0; i < n_irr; ++i)
        if (irr_h[i] < 0 || irr_h[i] >= nq)
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma: irr_q[%d]=%d outside the mesh", i, irr_h[i]);

    const double *d_f = nullptr, *d_e = nullptr;
    const int32_t* d_irr = nullptr;
    PHX_TRY(phx_stage_in(ctx, "g.f", freq_thz, (size_t)nq * n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "g.e", evec, (size_t)nq * n2 * 2, mem, s, &d_e));
    PHX_TRY(phx_stage_in(ctx, "g.irr", irr_q, (size_t)n_irr, mem, s, &d_irr));
    double *o_g = nullptr, *o_w = nullptr;
    PHX_TRY(phx_stage_out_buf(ctx, "g.og", gamma, (size_t)n_irr * n, mem, &o_g));
    if (wp2) PHX_TRY(phx_stage_out_buf(ctx, "g.ow", wp2, (size_t)n_irr * n, mem, &o_w));

    double* nB = (double*)phx_ws(ctx, "g.nB", (size_t)nq * n * 8);
    double* gacc = (double*)phx_ws(ctx, "g.gacc", (size_t)n_irr * n * 8);
    double* wacc = (double*)phx_ws(ctx, "g.wacc", (size_t)n_irr * n * 8);
    if (!nB || !gacc || !wacc) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, phx_launch_occupations(d_f, nq * n, temperature, 0, nB, nullptr, s));
    ctx->launches += 1;
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(gacc, 0, (size_t)n_irr * n * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(wacc, 0, (size_t)n_irr * n * 8, s));
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));

    GammaParams gp{};
    gp.n = n;
    gp.mesh[0] = fc3->mesh[0]; gp.mesh[1] = fc3->mesh[1]; gp.mesh[2] = fc3->mesh[2];
    gp.nq = nq;
    gp.T = temperature;
    gp.shape = br.shape;
    gp.sigma = br.sigma_thz;
    gp.window = br.window;
    gp.f_min = f_min_thz;
    if (prec == PHX_FP64) {
        PHX_TRY(phx_gamma_fp64(ctx, fc3, d_f, d_e, nB, irr_h.data(), n_irr, gp, gacc, wp2 ? wacc : nullptr, s));
    } else {
        PHX_TRY(phx_gamma_tc(ctx, fc3, d_f, d_e, nB, irr_h.data(), n_irr, gp, prec, gacc, wp2 ? wacc : nullptr, s));
    }
    const double conv = phx::kEvA2AmuToPs2;
    const double pref = phx::kPi * phx::kHbarEvPs * conv * conv * conv / (8.0 * nq);
    const int count = n_irr * n;
    finalize_gamma_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, n, d_irr, d_f, gacc, wacc, pref, 1.0 / nq,
                                                            f_min_thz, o_g, o_w);
    PHX_CUDA_CHECK(ctx, cudaGetLastError());
    ctx->launches += 1;
    if (mem == PHX_MEM_HOST) {
        int32_t st = 0;
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma, o_g, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
        if (wp2) PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(wp2, o_w, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_gamma: a device wait gave up (status %d)", st);
    }
    return PHX_OK;
}

phx_status phx_gamma_multi_t(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz, const double* evec,
                             const int32_t* irr_q, int32_t n_irr, const double* temperatures, int32_t n_t,
                             phx_broadening br, double f_min_thz, int32_t prec, double* gamma, int32_t mem,
                             void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (n_t < 0 || (n_t > 0 && !temperatures))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: bad temperature list");
    if (n_t == 0 || n_irr == 0) return PHX_OK;
    for (int t = 0; t < n_t; ++t)
        if (!(temperatures[t] > 0.0) || !std::isfinite(temperatures[t]))
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: temperature %d not finite and > 0", t);
    if (!fc3 || fc3->ctx != ctx) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: bad fc3 handle");
    const int64_t per_t = (int64_t)n_irr * fc3->n;
    const bool one_pass = prec != PHX_FP64 && !(fc3->nq == 1 && fc3->n > 192);
    if (!one_pass) {
        // FP64 reference and the Gamma-only cell: one full evaluation per temperature
        for (int t = 0; t < n_t; ++t)
            PHX_TRY(phx_gamma(ctx, fc3, freq_thz, evec, irr_q, n_irr, temperatures[t], br, f_min_thz, prec,
                              gamma + t * per_t, nullptr, mem, stream));
        return PHX_OK;
    }
    // argument checks of phx_gamma (first temperature), then the shared-contraction passes
    if (n_irr < 0 || !freq_thz || !evec || !irr_q || !gamma)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: null argument");
    if (!(br.sigma_thz > 0.0) || !(br.window > 0.0) || !(f_min_thz > 0.0) || !std::isfinite(f_min_thz))
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: sigma, window and f_min must be > 0");
    if (br.shape != PHX_GAUSS && br.shape != PHX_LORENTZ)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: unknown broadening shape %d", br.shape);
    if (prec != PHX_TF32 && prec != PHX_BF16X3)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: unknown precision %d", prec);
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: bad mem flag %d", mem);
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    const int n = fc3->n, nq = fc3->nq;
    const int64_t n2 = (int64_t)n * n;
    std::vector<int32_t> irr_h(n_irr);
    if (mem == PHX_MEM_HOST) {
        std::memcpy(irr_h.data(), irr_q, n_irr * 4);
    } else {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(irr_h.data(), irr_q, n_irr * 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    for (int i = 0; i < n_irr; ++i)
        if (irr_h[i] < 0 || irr_h[i] >= nq)
            return phx_set_error(ctx, PHX_ERR_INVALID, "phx_gamma_multi_t: irr_q[%d]=%d outside the mesh", i, irr_h[i]);
    const double *d_f = nullptr, *d_e = nullptr;
    const int32_t* d_irr = nullptr;
    PHX_TRY(phx_stage_in(ctx, "g.f", freq_thz, (size_t)nq * n, mem, s, &d_f));
    PHX_TRY(phx_stage_in(ctx, "g.e", evec, (size_t)nq * n2 * 2, mem, s, &d_e));
    PHX_TRY(phx_stage_in(ctx, "g.irr", irr_q, (size_t)n_irr, mem, s, &d_irr));
    double* o_g = nullptr;
    PHX_TRY(phx_stage_out_buf(ctx, "g.og", gamma, (size_t)n_t * per_t, mem, &o_g));
    double* nB = (double*)phx_ws(ctx, "g.nBt", (size_t)kTPerPass * nq * n * 8);
    double* gacc = (double*)phx_ws(ctx, "g.gacct", (size_t)kTPerPass * per_t * 8);
    if (!nB || !gacc) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(ctx->status_word, 0, 4, s));
    GammaParams gp{};
    gp.n = n;
    gp.mesh[0] = fc3->mesh[0]; gp.mesh[1] = fc3->mesh[1]; gp.mesh[2] = fc3->mesh[2];
    gp.nq = nq;
    gp.shape = br.shape;
    gp.sigma = br.sigma_thz;
    gp.window = br.window;
    gp.f_min = f_min_thz;
    const double conv = phx::kEvA2AmuToPs2;
    const double pref = phx::kPi * phx::kHbarEvPs * conv * conv * conv / (8.0 * nq);
    for (int t0 = 0; t0 < n_t; t0 += kTPerPass) {
        const int nt = std::min(kTPerPass, n_t - t0);
        for (int t = 0; t < nt; ++t)
            PHX_CUDA_CHECK(ctx, phx_launch_occupations(d_f, nq * n, temperatures[t0 + t], 0, nB + (int64_t)t * nq * n,
                                                       nullptr, s));
        PHX_CUDA_CHECK(ctx, cudaMemsetAsync(gacc, 0, (size_t)nt * per_t * 8, s));
        gp.T = temperatures[t0];
        PHX_TRY(phx_gamma_tc_multi_t(ctx, fc3, d_f, d_e, nB, nt, irr_h.data(), n_irr, gp, prec, gacc, s));
        for (int t = 0; t < nt; ++t)
            PHX_CUDA_CHECK(ctx, phx_launch_finalize((int)per_t, n, d_irr, d_f, gacc + t * per_t, nullptr, pref,
                                                    1.0 / nq, f_min_thz, o_g + (t0 + t) * per_t, nullptr, s));
        ctx->launches += 2 * nt;
    }
    if (mem == PHX_MEM_HOST) {
        int32_t st = 0;
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma, o_g, (size_t)n_t * per_t * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(&st, ctx->status_word, 4, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
        if (st != 0) return phx_set_error(ctx, (phx_status)st, "phx_gamma_multi_t: a device wait gave up (status %d)", st);
    }
    return PHX_OK;
}

// ---------------------------------------------------------------- transport

phx_status phx_unfold(phx_ctx* ctx, int32_t n_irr, int32_t nq, int32_t n, const double* freq_full,
                      const int32_t* irr_q, const double* gamma_irr, const int32_t* full_to_irr, double* gamma_full,
                      int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (n_irr <= 0 || nq <= 0 || n <= 0 || !freq_full || !irr_q || !gamma_irr || !full_to_irr || !gamma_full)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_unfold: bad argument");
    if (mem != PHX_MEM_HOST && mem != PHX_MEM_DEVICE)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_unfold: bad mem flag %d", mem);
    if (mem == PHX_MEM_HOST) {
        for (int i = 0; i < nq; ++i)
            if (full_to_irr[i] < 0 || full_to_irr[i] >= n_irr)
                return phx_set_error(ctx, PHX_ERR_INVALID, "phx_unfold: full_to_irr[%d] out of range", i);
        for (int i = 0; i < n_irr; ++i)
            if (irr_q[i] < 0 || irr_q[i] >= nq)
                return phx_set_error(ctx, PHX_ERR_INVALID, "phx_unfold: irr_q[%d] out of range", i);
    }
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    const double *f = nullptr, *g = nullptr;
    const int32_t *m = nullptr, *ir = nullptr;
    PHX_TRY(phx_stage_in(ctx, "u.f", freq_full, (size_t)nq * n, mem, s, &f));
    PHX_TRY(phx_stage_in(ctx, "u.i", irr_q, (size_t)n_irr, mem, s, &ir));
    PHX_TRY(phx_stage_in(ctx, "u.g", gamma_irr, (size_t)n_irr * n, mem, s, &g));
    PHX_TRY(phx_stage_in(ctx, "u.m", full_to_irr, (size_t)nq, mem, s, &m));
    double* o = nullptr;
    PHX_TRY(phx_stage_out_buf(ctx, "u.o", gamma_full, (size_t)nq * n, mem, &o));
    PHX_CUDA_CHECK(ctx, phx_launch_unfold(n_irr, nq, n, f, ir, g, m, o, s));
    ctx->launches += 1;
    if (mem == PHX_MEM_HOST) {
        PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(gamma_full, o, (size_t)nq * n * 8, cudaMemcpyDeviceToHost, s));
        PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    }
    return PHX_OK;
}

phx_status phx_kappa_rta(phx_ctx* ctx, const phx_cell* cell, int32_t nq, int32_t n, const double* freq_thz,
                         const double* vel, const double* vv, const double* gamma_full, double temperature,
                         double f_min_thz, int32_t is_classic, double* kappa_wmk, int32_t mem, void* stream) {
    if (!ctx) return PHX_ERR_INVALID;
    if (!cell || nq <= 0 || n <= 0 || !freq_thz || (!vel && !vv) || !gamma_full || !kappa_wmk)
        return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_rta: bad argument");
    if (!(temperature > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_rta: T must be > 0");
    const double* L = cell->lattice;
    const double vol = std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                                 L[2] * (L[3] * L[7] - L[4] * L[6]));
    if (!(vol > 0.0)) return phx_set_error(ctx, PHX_ERR_INVALID, "phx_kappa_rta: zero cell volume");
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    const double *f = nullptr, *v = nullptr, *w = nullptr, *g = nullptr;
    PHX_TRY(phx_stage_in(ctx, "k.f", freq_thz, (size_t)nq * n, mem, s, &f));
    if (vv) PHX_TRY(phx_stage_in(ctx, "k.vv", vv, (size_t)nq * n * 9, mem, s, &w));
    else PHX_TRY(phx_stage_in(ctx, "k.v", vel, (size_t)nq * n * 3, mem, s, &v));
    PHX_TRY(phx_stage_in(ctx, "k.g", gamma_full, (size_t)nq * n, mem, s, &g));
    double* acc = (double*)phx_ws(ctx, "k.acc", 9 * 8);
    if (!acc) return PHX_ERR_NOMEM;
    PHX_CUDA_CHECK(ctx, cudaMemsetAsync(acc, 0, 72, s));
    PHX_CUDA_CHECK(ctx, phx_launch_kappa(nq, n, f, v, w, g, temperature, f_min_thz, is_classic, acc, s));
    ctx->launches += 1;
    double h[9];
    PHX_CUDA_CHECK(ctx, cudaMemcpyAsync(h, acc, 72, cudaMemcpyDeviceToHost, s));
    PHX_CUDA_CHECK(ctx, cudaStreamSynchronize(s));
    const double sc = phx::kEvPsAKToWmK / ((double)nq * vol);
    for (int k = 0; k < 9; ++k) kappa_wmk[k] = h[k] * sc;
    return PHX_OK;
}

}  // extern "C"
