// C ABI of the IBIM library: context lifetime, geometry builds, operator
// dispatch, diagnostics.  Every entry point returns an ibim_status and keeps
// the failure message in a thread-local string (ibim_last_error).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

ibim_status cuda_fail(cudaError_t e, const char* what, const char* file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what,
             file, line);
    g_err = buf;
    return IBIM_ERR_CUDA;
}

static ibim_status fail(ibim_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

ibim_status ensure(ibim_ctx* c, void** buf, size_t* have, size_t need)
{
    if (*have >= need && *buf != nullptr) return IBIM_OK;
    if (*buf != nullptr) {
        IBIM_CUDA(cudaStreamSynchronize(c->stream));
        IBIM_CUDA(cudaFree(*buf));
        *buf = nullptr;
        *have = 0;
    }
    IBIM_CUDA(cudaMalloc(buf, need));
    *have = need;
    ++c->ws_generation;
    return IBIM_OK;
}

ibim_status check_phys(const ibim_phys* p)
{
    if (p == nullptr) return fail(IBIM_ERR_ARG, "phys is NULL");
    if (!(p->eps_in > 0.0) || !(p->eps_out > 0.0) || !isfinite(p->eps_in) || !isfinite(p->eps_out))
        return fail(IBIM_ERR_ARG, "eps_in and eps_out must be finite and > 0");
    if (!(p->kappa >= 0.0) || !isfinite(p->kappa)) return fail(IBIM_ERR_ARG, "kappa must be finite and >= 0");
    if (!(p->tau > 0.0) || !isfinite(p->tau)) return fail(IBIM_ERR_ARG, "tau must be finite and > 0");
    if (p->tube_rule != 0 && p->tube_rule != 1) return fail(IBIM_ERR_ARG, "tube_rule must be 0 or 1");
    return IBIM_OK;
}

// Sec. 2.2 / Sec. 3.3: Lambda = diag((1+eps_E/eps_I)/2, (1+eps_I/eps_E)/2);
// Sec. 2.2.1: tube value of K12 = (exp(-kappa tau) - 1 + kappa tau)/(2 pi kappa tau^2),
// stored times 4 pi (the kernels run without the common 1/(4 pi)).
PairConsts make_consts(const ibim_phys& p)
{
    PairConsts k;
    k.th1 = p.eps_out / p.eps_in;
    k.th2 = p.eps_in / p.eps_out;
    k.lambda1 = 0.5 * (1.0 + k.th1);
    k.lambda2 = 0.5 * (1.0 + k.th2);
    k.kappa = p.kappa;
    k.tau2 = p.tau * p.tau;
    k.four_tau2 = (p.tube_rule == 0) ? 4.0 * p.tau * p.tau : HUGE_VAL;
    const double kt = p.kappa * p.tau;
    double tube = 0.0;
    if (kt > 1e-4)
        tube = (exp(-kt) - 1.0 + kt) / (2.0 * kPi * p.kappa * p.tau * p.tau);
    else if (kt > 0.0)  // series of (e^{-x} - 1 + x)/x^2 = 1/2 - x/6 + x^2/24 - ...
        tube = p.kappa * (0.5 - kt / 6.0 + kt * kt / 24.0) / (2.0 * kPi);
    k.k12_tube = 4.0 * kPi * tube;
    return k;
}

PairSchedule make_schedule(int64_t n_targets, int ttile, int64_t n_sources, int stile, int grid_cap,
                           int64_t)
{
    PairSchedule s;
    s.n_ttiles = (n_targets + ttile - 1) / ttile;
    s.n_stiles = (n_sources + stile - 1) / stile;
    s.total = s.n_ttiles * s.n_stiles;
    int64_t g = std::min<int64_t>(grid_cap, s.total);
    if (g < 1) g = 1;
    s.per_cta = (s.total + g - 1) / g;
    s.grid = (int)((s.total + s.per_cta - 1) / s.per_cta);
    s.max_segs = (int)((s.per_cta + s.n_stiles - 1) / s.n_stiles + 1);
    // Rows visit their source tiles with a stride near n_stiles / golden ratio
    // (coprime to n_stiles, so a permutation): the few expensive near-field
    // tiles, which sit together around the diagonal, are then spread evenly
    // over the CTAs that share a row instead of landing on one of them.
    s.sperm = 1;
    if (s.n_stiles > 2) {
        int64_t m = (int64_t)llround(0.6180339887498949 * (double)s.n_stiles);
        if (m < 1) m = 1;
        auto gcd = [](int64_t a, int64_t b) {
            while (b != 0) {
                const int64_t r = a % b;
                a = b;
                b = r;
            }
            return a;
        };
        while (gcd(m, s.n_stiles) != 1) ++m;
        s.sperm = m % s.n_stiles;
    }
    return s;
}

// ---------------------------------------------------------------- timing
ibim_status timing_begin(ibim_ctx* c)
{
    Timing& T = c->timing;
    if (!T.enabled) return IBIM_OK;
    if (T.used + 2 > T.pool.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            IBIM_CUDA(cudaEventCreate(&e));
            T.pool.push_back(e);
        }
    }
    IBIM_CUDA(cudaEventRecord(T.pool[T.used], c->stream));
    return IBIM_OK;
}

ibim_status timing_end(ibim_ctx* c, int64_t interactions)
{
    Timing& T = c->timing;
    if (!T.enabled) return IBIM_OK;
    IBIM_CUDA(cudaEventRecord(T.pool[T.used + 1], c->stream));
    T.used += 2;
    T.pair_launches += 1;
    T.pair_interactions += interactions;
    if (T.used >= 4096) return timing_collect(c);
    return IBIM_OK;
}

ibim_status timing_collect(ibim_ctx* c)
{
    Timing& T = c->timing;
    for (size_t q = 0; q + 1 < T.used; q += 2) {
        IBIM_CUDA(cudaEventSynchronize(T.pool[q + 1]));
        float ms = 0.0f;
        IBIM_CUDA(cudaEventElapsedTime(&ms, T.pool[q], T.pool[q + 1]));
        T.pair_ms += ms;
    }
    T.used = 0;
    return IBIM_OK;
}

// Source payload and partial-sum buffers large enough for both precisions
// and every FP32 variant, so operator applications never reallocate them.
ibim_status ensure_operator_workspaces(ibim_ctx* c)
{
    if (c->ws_sized) return IBIM_OK;
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, &c->d_src, &c->src_bytes,
                    std::max(std::max((size_t)N * 8 * sizeof(double), (size_t)padded_nodes(N) * 2 * sizeof(float4)),
                             ff_src_bytes(N))));
    IBIM_TRY(ff_prepare_context(c));
    const PairSchedule s64 = make_schedule(N, kF64TTile, N, kF64STile, f64_grid_cap(c));
    size_t need = (size_t)s64.grid * s64.max_segs * 2 * kF64TTile * sizeof(double);
    need = std::max(need, ff_part_doubles(c) * sizeof(double));
    const int keep = c->f32_variant, keep_bps = c->f32_bps;
    c->f32_bps = 0;
    for (int v = 0; v < f32_variant_count(); ++v) {
        c->f32_variant = v;
        need = std::max(need, f32_part_doubles(c) * sizeof(double));
    }
    c->f32_variant = keep;
    c->f32_bps = keep_bps;
    IBIM_TRY(ensure(c, (void**)&c->d_yrev, &c->yrev_bytes, sym_yrev_bytes(N)));
    IBIM_TRY(ensure(c, (void**)&c->d_part, &c->part_bytes, need));
    c->ws_sized = true;
    return IBIM_OK;
}

// --------------------------------------------------------------- operator
ibim_status apply_operator(ibim_ctx* c, const PairConsts& k, int precision, VecRef in, OutRef out,
                           const int* d_skip)
{
    const int64_t N = c->N;
    IBIM_TRY(ensure_operator_workspaces(c));
    if (precision == IBIM_F32C) {
        const PairSchedule s = f32_schedule(c);
        IBIM_TRY(f32_pack(c, in, d_skip));
        IBIM_TRY(timing_begin(c));
        IBIM_TRY(f32_pairs(c, k, s, d_skip));
        IBIM_TRY(timing_end(c, N * N));
        return f32_fixup(c, k, s, in, out, d_skip);
    }
    if (precision == IBIM_F32T) return tc_apply(c, k, in, out, d_skip);
    if (precision == IBIM_F64) {
        const PairSchedule s = make_schedule(N, kF64TTile, N, kF64STile, f64_grid_cap(c));
        IBIM_TRY(f64_pack(c, in, d_skip));
        IBIM_TRY(timing_begin(c));
        IBIM_TRY(f64_pairs(c, k, s, d_skip));
        IBIM_TRY(timing_end(c, N * N));
        return f64_fixup(c, k, s, in, out, d_skip);
    }
    if (precision == IBIM_FF) {
        const PairSchedule s = ff_schedule(c);
        IBIM_TRY(ff_pack(c, in, d_skip));
        IBIM_TRY(timing_begin(c));
        IBIM_TRY(ff_pairs(c, k, s, d_skip));
        IBIM_TRY(timing_end(c, N * N));
        return ff_fixup(c, k, s, in, out, d_skip);
    }
    return fail(IBIM_ERR_ARG, "precision must be IBIM_F64 (64), IBIM_FF (65), IBIM_F32C (32) or IBIM_F32T (33)");
}

static bool valid_precision(int p) { return p == IBIM_F64 || p == IBIM_FF || p == IBIM_F32C || p == IBIM_F32T; }

// Reads the device error word after a synchronisation point.
static ibim_status check_device_error(ibim_ctx* c)
{
    unsigned e = 0;
    IBIM_CUDA(cudaMemcpyAsync(&e, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    if (e != 0) {
        IBIM_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
        if (e & kDevErrTimeout) return fail(IBIM_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up");
        return fail(IBIM_ERR_CUDA, "device error word set");
    }
    return IBIM_OK;
}

static ibim_status ctx_new(void* stream, ibim_ctx** out)
{
    if (out == nullptr) return fail(IBIM_ERR_ARG, "out is NULL");
    *out = nullptr;
    ibim_ctx* c = new ibim_ctx();
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) {
        ibim_destroy(c);
        return cuda_fail(e, "context creation", __FILE__, __LINE__);
    }
    *out = c;
    return IBIM_OK;
}

}  // namespace ibim

using namespace ibim;

extern "C" {

const char* ibim_last_error(void) { return g_err.c_str(); }

ibim_status ibim_set_ff_kernel(ibim_ctx* c, int symmetric)
{
    if (c == nullptr || (symmetric != 0 && symmetric != 1)) return fail(IBIM_ERR_ARG, "need a context and 0 or 1");
    c->ff_symmetric = symmetric;
    return IBIM_OK;
}

// One thread sets bits of the device error word, as a kernel whose bounded
// wait gave up does (the failure-path test hook below).
__global__ void raise_device_error_kernel(unsigned* __restrict__ err, unsigned bits) { atomicOr(err, bits); }

ibim_status ibim_debug_raise_device_error(ibim_ctx* c, int status)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    if (status != IBIM_ERR_DEVICE_TIMEOUT) return fail(IBIM_ERR_ARG, "only IBIM_ERR_DEVICE_TIMEOUT can be raised");
    raise_device_error_kernel<<<1, 1, 0, c->stream>>>(c->d_err, kDevErrTimeout);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

void ibim_destroy(ibim_ctx* c)
{
    if (c == nullptr) return;
    cudaStreamSynchronize(c->stream);
    gmres_free(c);
    for (cudaEvent_t e : c->timing.pool) cudaEventDestroy(e);
    cudaFree(c->d_geo64);
    cudaFree(c->d_dist);
    cudaFree(c->d_curv);
    cudaFree(c->d_sig2);
    cudaFree(c->d_w1);
    cudaFree(c->d_ijk);
    cudaFree(c->d_pos32);
    cudaFree(c->d_nrm32);
    cudaFree(c->d_frames);
    cudaFree(c->d_z);
    cudaFree(c->d_q);
    cudaFree(c->d_src);
    cudaFree(c->d_part);
    cudaFree(c->d_red);
    cudaFree(c->d_err);
    cudaFree(c->d_io);
    cudaFree(c->d_aux);
    cudaFree(c->d_yrev);
    cudaFree(c->d_fftab);
    ibim::tc_destroy(c->tc);
    cudaFree(c->d_phi);
    delete c;
}

ibim_status ibim_build_sphere(double R, const double* centre, const double* origin, double h,
                              double band_eps, void* stream, ibim_ctx** out)
{
    if (centre == nullptr) return fail(IBIM_ERR_ARG, "centre is NULL");
    if (!(R > 0.0) || !(h > 0.0) || !(band_eps > 0.0) || !isfinite(R) || !isfinite(h) || !isfinite(band_eps))
        return fail(IBIM_ERR_ARG, "R, h and band_eps must be finite and > 0");
    const double o0[3] = {0.0, 0.0, 0.0};
    const double* o = origin ? origin : o0;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(centre[a]) || !isfinite(o[a])) return fail(IBIM_ERR_NONFINITE, "centre/origin not finite");
    const double span = (2.0 * (R + band_eps)) / h;
    if (span > 2000.0) return fail(IBIM_ERR_ARG, "sphere spans more than 2000 grid cells per axis");
    ibim_ctx* c = nullptr;
    IBIM_TRY(ctx_new(stream, &c));
    c->h = h;
    c->band_eps = band_eps;
    for (int a = 0; a < 3; ++a) c->centroid[a] = centre[a];
    ibim_status s = build_sphere_nodes(c, R, centre, o, h, band_eps);
    if (s == IBIM_OK) s = finish_geometry(c, true);
    if (s != IBIM_OK) {
        std::string msg = g_err;
        ibim_destroy(c);
        g_err = msg;
        return s;
    }
    *out = c;
    return IBIM_OK;
}

ibim_status ibim_build(const double* xyz, const double* radii, const double* charges, int64_t Na, double probe,
                       double h, double band_eps, void* stream, ibim_ctx** out)
{
    if (xyz == nullptr || radii == nullptr || Na < 1) return fail(IBIM_ERR_ARG, "need Na >= 1 atoms with centres and radii");
    if (!(h > 0.0) || !(band_eps > 0.0) || !(probe >= 0.0) || !isfinite(h) || !isfinite(band_eps) || !isfinite(probe))
        return fail(IBIM_ERR_ARG, "need h > 0, band_eps > 0, probe >= 0 (finite)");
    double cen[3] = {0, 0, 0};
    for (int64_t k = 0; k < Na; ++k) {
        if (!isfinite(radii[k]) || !(radii[k] > 0.0)) return fail(IBIM_ERR_ARG, "atom radii must be finite and > 0");
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(xyz[3 * k + a])) return fail(IBIM_ERR_NONFINITE, "non-finite atom centre");
            cen[a] += xyz[3 * k + a];
        }
        if (charges != nullptr && !isfinite(charges[k])) return fail(IBIM_ERR_NONFINITE, "non-finite charge");
    }
    ibim_ctx* c = nullptr;
    IBIM_TRY(ctx_new(stream, &c));
    c->h = h;
    c->band_eps = band_eps;
    for (int a = 0; a < 3; ++a) c->centroid[a] = cen[a] / (double)Na;
    ibim_status s = build_levelset(c, Na, xyz, radii, probe, h, band_eps);
    if (s == IBIM_OK) s = finish_geometry(c, true);
    if (s == IBIM_OK && charges != nullptr) s = ibim_set_charges(c, Na, xyz, charges);
    if (s != IBIM_OK) {
        std::string msg = g_err;
        ibim_destroy(c);
        g_err = msg;
        return s;
    }
    *out = c;
    return IBIM_OK;
}

ibim_status ibim_get_levelset(const ibim_ctx* cc, int64_t* lo, int64_t* n, double* phi)
{
    if (cc == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    ibim_ctx* c = const_cast<ibim_ctx*>(cc);
    if (c->d_phi == nullptr) return fail(IBIM_ERR_STATE, "context was not built from atoms");
    for (int a = 0; a < 3; ++a) {
        if (lo) lo[a] = c->ls_lo[a];
        if (n) n[a] = c->ls_n[a];
    }
    if (phi != nullptr) {
        const int64_t M = c->ls_n[0] * c->ls_n[1] * c->ls_n[2];
        IBIM_CUDA(cudaMemcpyAsync(phi, c->d_phi, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream));
        IBIM_CUDA(cudaStreamSynchronize(c->stream));
    }
    return IBIM_OK;
}

ibim_status ibim_build_from_nodes(int64_t N, const double* xstar, const double* normal, const double* w,
                                  double h, void* stream, ibim_ctx** out)
{
    if (N <= 0) return fail(IBIM_ERR_ARG, "N must be > 0");
    if (N > (int64_t)1 << 31) return fail(IBIM_ERR_ARG, "N too large");
    if (!xstar || !normal || !w) return fail(IBIM_ERR_ARG, "node arrays must not be NULL");
    if (!(h > 0.0)) return fail(IBIM_ERR_ARG, "h must be > 0");
    std::vector<double> geo((size_t)N * 7);
    double cen[3] = {0, 0, 0};
    for (int64_t j = 0; j < N; ++j) {
        for (int a = 0; a < 3; ++a) {
            const double x = xstar[3 * j + a], n = normal[3 * j + a];
            if (!isfinite(x) || !isfinite(n)) return fail(IBIM_ERR_NONFINITE, "non-finite node data");
            geo[(size_t)a * N + j] = x;
            geo[(size_t)(3 + a) * N + j] = n;
            cen[a] += x;
        }
        if (!isfinite(w[j])) return fail(IBIM_ERR_NONFINITE, "non-finite weight");
        geo[(size_t)6 * N + j] = w[j];
    }
    ibim_ctx* c = nullptr;
    IBIM_TRY(ctx_new(stream, &c));
    c->N = N;
    c->h = h;
    for (int a = 0; a < 3; ++a) c->centroid[a] = cen[a] / (double)N;
    std::vector<int32_t> ijk((size_t)N * 3, -1);
    cudaError_t e = cudaMalloc((void**)&c->d_geo64, sizeof(double) * 7 * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_dist, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ijk, sizeof(int32_t) * 3 * N);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_geo64, geo.data(), sizeof(double) * 7 * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_dist, 0, sizeof(double) * N, c->stream);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_curv, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_curv, 0, sizeof(double) * N, c->stream);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_sig2, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_sig2, 0, sizeof(double) * N, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_ijk, ijk.data(), sizeof(int32_t) * 3 * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        ibim_status s = cuda_fail(e, "build_from_nodes upload", __FILE__, __LINE__);
        std::string msg = g_err;
        ibim_destroy(c);
        g_err = msg;
        return s;
    }
    ibim_status s = finish_geometry(c, false);
    if (s != IBIM_OK) {
        std::string msg = g_err;
        ibim_destroy(c);
        g_err = msg;
        return s;
    }
    *out = c;
    return IBIM_OK;
}

ibim_status ibim_set_charges(ibim_ctx* c, int64_t Nc, const double* z, const double* q)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    if (Nc <= 0 || !z || !q) return fail(IBIM_ERR_ARG, "need Nc >= 1 and non-NULL z, q");
    for (int64_t k = 0; k < Nc; ++k) {
        if (!isfinite(q[k]) || !isfinite(z[3 * k]) || !isfinite(z[3 * k + 1]) || !isfinite(z[3 * k + 2]))
            return fail(IBIM_ERR_NONFINITE, "non-finite charge data");
    }
    if (Nc != c->Nc) {
        cudaFree(c->d_z);
        cudaFree(c->d_q);
        c->d_z = c->d_q = nullptr;
        c->Nc = 0;
        IBIM_CUDA(cudaMalloc((void**)&c->d_z, sizeof(double) * 3 * Nc));
        IBIM_CUDA(cudaMalloc((void**)&c->d_q, sizeof(double) * Nc));
    }
    IBIM_CUDA(cudaMemcpyAsync(c->d_z, z, sizeof(double) * 3 * Nc, cudaMemcpyHostToDevice, c->stream));
    IBIM_CUDA(cudaMemcpyAsync(c->d_q, q, sizeof(double) * Nc, cudaMemcpyHostToDevice, c->stream));
    c->Nc = Nc;
    return IBIM_OK;
}

ibim_status ibim_get_curvature(const ibim_ctx* cc, double* curv)
{
    if (cc == nullptr || curv == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    ibim_ctx* c = const_cast<ibim_ctx*>(cc);
    IBIM_CUDA(cudaMemcpyAsync(curv, c->d_curv, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

// J = 1 - d lap + d^2 sig2, clamped at 0 (Sec. 2.2 Jacobian; the last term
// read as the sum of the Hessian's 2x2 principal minors).
__device__ __forceinline__ double full_jacobian(double d, double lap, double sig2)
{
    const double J = 1.0 - d * lap + d * d * sig2;
    return J > 0.0 ? J : 0.0;
}

__global__ void jacobian_kernel(const double* __restrict__ dist, const double* __restrict__ lap,
                                const double* __restrict__ sig2, int64_t N, double* __restrict__ J)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) J[i] = full_jacobian(dist[i], lap[i], sig2[i]);
}

__global__ void jacobian_weights_kernel(const double* __restrict__ w1, const double* __restrict__ dist,
                                        const double* __restrict__ lap, const double* __restrict__ sig2, int64_t N,
                                        int mode, double* __restrict__ w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) w[i] = mode ? w1[i] * full_jacobian(dist[i], lap[i], sig2[i]) : w1[i];
}

ibim_status ibim_get_jacobian(const ibim_ctx* cc, double* J)
{
    if (cc == nullptr || J == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    ibim_ctx* c = const_cast<ibim_ctx*>(cc);
    if (c->d_w1 == nullptr) return fail(IBIM_ERR_STATE, "caller-given nodes carry no distance function");
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, (void**)&c->d_io, &c->io_bytes, sizeof(double) * N));
    jacobian_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->d_dist, c->d_curv, c->d_sig2, N, c->d_io);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemcpyAsync(J, c->d_io, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

ibim_status ibim_set_jacobian(ibim_ctx* c, int mode)
{
    if (c == nullptr || (mode != 0 && mode != 1)) return fail(IBIM_ERR_ARG, "need a context and mode 0 or 1");
    if (c->d_w1 == nullptr) {
        if (mode == 0) return IBIM_OK;
        return fail(IBIM_ERR_STATE, "caller-given nodes carry no distance function: their weights stay as given");
    }
    const int64_t N = c->N;
    jacobian_weights_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->d_w1, c->d_dist, c->d_curv,
                                                                               c->d_sig2, N, mode,
                                                                               c->d_geo64 + 6 * N);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    c->jacobian = mode;
    return IBIM_OK;
}

ibim_status ibim_num_nodes(const ibim_ctx* c, int64_t* N)
{
    if (c == nullptr || N == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    *N = c->N;
    return IBIM_OK;
}

ibim_status ibim_get_nodes(const ibim_ctx* cc, double* xstar, double* normal, double* w, double* d,
                           int32_t* ijk)
{
    if (cc == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    ibim_ctx* c = const_cast<ibim_ctx*>(cc);
    const int64_t N = c->N;
    std::vector<double> geo((size_t)N * 7);
    IBIM_CUDA(cudaMemcpyAsync(geo.data(), c->d_geo64, sizeof(double) * 7 * N, cudaMemcpyDeviceToHost, c->stream));
    if (d) IBIM_CUDA(cudaMemcpyAsync(d, c->d_dist, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    if (ijk) IBIM_CUDA(cudaMemcpyAsync(ijk, c->d_ijk, sizeof(int32_t) * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) {
            if (xstar) xstar[3 * j + a] = geo[(size_t)a * N + j];
            if (normal) normal[3 * j + a] = geo[(size_t)(3 + a) * N + j];
        }
    if (w)
        for (int64_t j = 0; j < N; ++j) w[j] = geo[(size_t)6 * N + j];
    return IBIM_OK;
}

ibim_status ibim_matvec(ibim_ctx* c, const ibim_phys* phys, int precision, const double* d_in, double* d_out)
{
    if (c == nullptr || d_in == nullptr || d_out == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    IBIM_TRY(check_phys(phys));
    if (d_in == d_out) return fail(IBIM_ERR_ARG, "d_in and d_out must not overlap");
    const PairConsts k = make_consts(*phys);
    return apply_operator(c, k, precision, VecRef{d_in, nullptr, 0, 0}, OutRef{d_out, nullptr, 0, 0}, nullptr);
}

ibim_status ibim_matvec_host(ibim_ctx* c, const ibim_phys* phys, int precision, const double* h_in,
                             double* h_out)
{
    if (c == nullptr || h_in == nullptr || h_out == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    IBIM_TRY(check_phys(phys));
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, (void**)&c->d_io, &c->io_bytes, sizeof(double) * 4 * N));
    double* io = c->d_io;
    IBIM_CUDA(cudaMemcpyAsync(io, h_in, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
    IBIM_TRY(ibim_matvec(c, phys, precision, io, io + 2 * N));
    IBIM_CUDA(cudaMemcpyAsync(h_out, io + 2 * N, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

ibim_status ibim_rhs(ibim_ctx* c, double eps_in, double* d_g)
{
    if (c == nullptr || d_g == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    if (!(eps_in > 0.0)) return fail(IBIM_ERR_ARG, "eps_in must be > 0");
    if (c->Nc <= 0) return fail(IBIM_ERR_STATE, "no charges set");
    return rhs_launch(c, eps_in, d_g);
}

ibim_status ibim_energy(ibim_ctx* c, const ibim_phys* phys, int precision, const double* d_p,
                        double* d_psi_rxn, double* gpol)
{
    if (c == nullptr || d_p == nullptr || gpol == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    IBIM_TRY(check_phys(phys));
    if (!valid_precision(precision)) return fail(IBIM_ERR_ARG, "bad precision");
    if (c->Nc <= 0) return fail(IBIM_ERR_STATE, "no charges set");
    IBIM_TRY(energy_launch(c, *phys, d_p, d_psi_rxn, gpol));
    return check_device_error(c);
}

ibim_status ibim_area(ibim_ctx* c, double* area)
{
    if (c == nullptr || area == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    return area_launch(c, area);
}

ibim_status ibim_solve(ibim_ctx* c, const ibim_phys* phys, const ibim_solve_opts* o, double* d_p,
                       ibim_solve_info* info)
{
    if (c == nullptr || o == nullptr || d_p == nullptr || info == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    IBIM_TRY(check_phys(phys));
    if (!valid_precision(o->precision)) return fail(IBIM_ERR_ARG, "bad precision");
    if (o->certify < 0 || o->certify > 2) return fail(IBIM_ERR_ARG, "certify must be 0, 1 or 2");
    if (!(o->tol > 0.0) || o->maxit < 1 || o->restart < 1 || o->restart > 128)
        return fail(IBIM_ERR_ARG, "need tol > 0, maxit >= 1, 1 <= restart <= 128");
    if (o->start != 0 && o->start != 1 && o->start != 3) return fail(IBIM_ERR_ARG, "start must be 0, 1 or 3");
    if (c->Nc <= 0) return fail(IBIM_ERR_STATE, "no charges set");
    memset(info, 0, sizeof(*info));
    ibim_status s = gmres_solve(c, *phys, *o, d_p, info);
    if (s != IBIM_OK && s != IBIM_ERR_NOT_CONVERGED) return s;
    ibim_status s2 = check_device_error(c);
    if (s2 != IBIM_OK) return s2;
    if (s == IBIM_ERR_NOT_CONVERGED) return fail(IBIM_ERR_NOT_CONVERGED, "GMRES reached maxit above tol");
    return IBIM_OK;
}

// p = 2 p_half - p_tau (Richardson step of the tube extrapolation).
__global__ void extrapolate_kernel(double* __restrict__ p_half, const double* __restrict__ p_tau, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p_half[i] = 2.0 * p_half[i] - p_tau[i];
}

ibim_status ibim_solve_extrapolated(ibim_ctx* c, const ibim_phys* phys, const ibim_solve_opts* o, double* d_p,
                                    ibim_solve_info* info)
{
    if (c == nullptr || o == nullptr || d_p == nullptr || info == nullptr) return fail(IBIM_ERR_ARG, "NULL argument");
    IBIM_TRY(check_phys(phys));
    if (!valid_precision(o->precision)) return fail(IBIM_ERR_ARG, "bad precision");
    if (o->certify < 0 || o->certify > 2) return fail(IBIM_ERR_ARG, "certify must be 0, 1 or 2");
    if (!(o->tol > 0.0) || o->maxit < 1 || o->restart < 1 || o->restart > 128)
        return fail(IBIM_ERR_ARG, "need tol > 0, maxit >= 1, 1 <= restart <= 128");
    if (o->start != 0 && o->start != 1 && o->start != 3) return fail(IBIM_ERR_ARG, "start must be 0, 1 or 3");
    if (c->Nc <= 0) return fail(IBIM_ERR_STATE, "no charges set");
    memset(info, 0, sizeof(*info));
    const int64_t len = 2 * c->N;
    IBIM_TRY(ensure(c, (void**)&c->d_aux, &c->aux_bytes, sizeof(double) * len));
    // 1. the system with tau (the caller's start)
    if (o->start == 3)
        IBIM_CUDA(cudaMemcpyAsync(c->d_aux, d_p, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    ibim_solve_info i1;
    memset(&i1, 0, sizeof(i1));
    ibim_status s1 = gmres_solve(c, *phys, *o, c->d_aux, &i1);
    if (s1 != IBIM_OK && s1 != IBIM_ERR_NOT_CONVERGED) return s1;
    // 2. the system with tau/2, started from the tau solution
    ibim_phys half = *phys;
    half.tau = 0.5 * phys->tau;
    ibim_solve_opts o2 = *o;
    o2.start = 3;
    IBIM_CUDA(cudaMemcpyAsync(d_p, c->d_aux, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    ibim_solve_info i2;
    memset(&i2, 0, sizeof(i2));
    ibim_status s2 = gmres_solve(c, half, o2, d_p, &i2);
    if (s2 != IBIM_OK && s2 != IBIM_ERR_NOT_CONVERGED) return s2;
    // 3. p* = 2 p(tau/2) - p(tau); G_pol is linear in p
    extrapolate_kernel<<<(unsigned)((len + 255) / 256), 256, 0, c->stream>>>(d_p, c->d_aux, len);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    double gpol = 0.0, area = 0.0;
    IBIM_TRY(energy_launch(c, *phys, d_p, nullptr, &gpol));
    IBIM_TRY(area_launch(c, &area));
    info->iters = i1.iters + i2.iters;
    info->cycles = i1.cycles + i2.cycles;
    info->converged = (i1.converged && i2.converged) ? 1 : 0;
    info->relres = std::max(i1.relres, i2.relres);
    info->gpol = gpol;
    info->gpol_kcal = gpol * kKcalPerE2A;
    info->area = area;
    info->matvecs_f32 = i1.matvecs_f32 + i2.matvecs_f32;
    info->matvecs_f64 = i1.matvecs_f64 + i2.matvecs_f64;
    IBIM_TRY(check_device_error(c));
    if (!info->converged) return fail(IBIM_ERR_NOT_CONVERGED, "GMRES reached maxit above tol");
    return IBIM_OK;
}

ibim_status ibim_solve_batch(int nmol, ibim_ctx* const* ctxs, const ibim_phys* phys, const ibim_solve_opts* o,
                             double* const* d_p, ibim_solve_info* infos)
{
    if (nmol < 1 || nmol > 1024 || ctxs == nullptr || phys == nullptr || o == nullptr || d_p == nullptr ||
        infos == nullptr)
        return fail(IBIM_ERR_ARG, "need 1 <= nmol <= 1024 and non-NULL arrays");
    if (o->precision != IBIM_F32C || (o->start != 0 && o->start != 3) || o->certify != 0)
        return fail(IBIM_ERR_ARG,
                    "the batched solve runs the FP32 operator without certification, from a zero start (0) or "
                    "from the vectors in d_p (3)");
    if (!(o->tol > 0.0) || o->maxit < 1 || o->restart < 1 || o->restart > 128)
        return fail(IBIM_ERR_ARG, "need tol > 0, maxit >= 1, 1 <= restart <= 128");
    for (int i = 0; i < nmol; ++i) {
        if (ctxs[i] == nullptr || d_p[i] == nullptr) return fail(IBIM_ERR_ARG, "NULL context or output");
        IBIM_TRY(check_phys(&phys[i]));
        if (ctxs[i]->Nc <= 0) return fail(IBIM_ERR_STATE, "a context has no charges");
        if (ctxs[i]->device != ctxs[0]->device) return fail(IBIM_ERR_ARG, "contexts on different devices");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(IBIM_ERR_ARG, "a context appears twice in the batch");
        memset(&infos[i], 0, sizeof(infos[i]));
    }
    ibim_status s = batch_solve(nmol, ctxs, phys, *o, d_p, infos);
    if (s != IBIM_OK) return s;
    for (int i = 0; i < nmol; ++i) IBIM_TRY(check_device_error(ctxs[i]));
    for (int i = 0; i < nmol; ++i)
        if (!infos[i].converged) return fail(IBIM_ERR_NOT_CONVERGED, "a molecule reached maxit above tol");
    return IBIM_OK;
}

ibim_status ibim_solve_host(ibim_ctx* c, const ibim_phys* phys, const ibim_solve_opts* o, int64_t Nc,
                            const double* z, const double* q, double* h_p, ibim_solve_info* info)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    IBIM_TRY(ibim_set_charges(c, Nc, z, q));
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, (void**)&c->d_io, &c->io_bytes, sizeof(double) * 4 * N));
    double* dp = c->d_io;
    if (o != nullptr && o->start == 3) {
        if (h_p == nullptr) return fail(IBIM_ERR_ARG, "start = 3 needs h_p");
        IBIM_CUDA(cudaMemcpyAsync(dp, h_p, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
    }
    const ibim_status s = ibim_solve(c, phys, o, dp, info);
    if ((s == IBIM_OK || s == IBIM_ERR_NOT_CONVERGED) && h_p != nullptr) {
        IBIM_CUDA(cudaMemcpyAsync(h_p, dp, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->stream));
        IBIM_CUDA(cudaStreamSynchronize(c->stream));
    }
    return s;
}

ibim_status ibim_timing_enable(ibim_ctx* c, int enable)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    if (!enable && c->timing.used) IBIM_TRY(timing_collect(c));
    c->timing.enabled = enable != 0;
    return IBIM_OK;
}

ibim_status ibim_timing_reset(ibim_ctx* c)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    c->timing.used = 0;
    c->timing.pair_ms = 0.0;
    c->timing.pair_launches = 0;
    c->timing.pair_interactions = 0;
    c->timing.total_launches = 0;
    return IBIM_OK;
}

ibim_status ibim_timing_get(ibim_ctx* c, double* pair_ms, int64_t* pair_launches, int64_t* pair_interactions,
                            int64_t* total_launches)
{
    if (c == nullptr) return fail(IBIM_ERR_ARG, "ctx is NULL");
    IBIM_TRY(timing_collect(c));
    if (pair_ms) *pair_ms = c->timing.pair_ms;
    if (pair_launches) *pair_launches = c->timing.pair_launches;
    if (pair_interactions) *pair_interactions = c->timing.pair_interactions;
    if (total_launches) *total_launches = c->timing.total_launches;
    return IBIM_OK;
}

}  // extern "C"
