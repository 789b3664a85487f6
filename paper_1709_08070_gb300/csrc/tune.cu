// Autotuner of the FP32 pair-sum kernel: measures each variant (targets per
// thread x CTAs per SM) on a context's own geometry with CUDA events and keeps
// the fastest, cached per problem-size bucket (floor(log2 N)) for contexts
// built later in the process.
#include <map>
#include <mutex>
#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

namespace {
std::mutex g_tune_mu;
std::map<int, std::pair<int, int>> g_tune_cache;  // bucket -> (tpt, bps)

int size_bucket(int64_t N)
{
    int b = 0;
    while ((int64_t)1 << (b + 1) <= N) ++b;
    return b;
}

__global__ void fill_kernel(double* __restrict__ p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 1.0 + 1e-3 * (double)(i % 97);
}
}  // namespace

void apply_cached_tuning(ibim_ctx* c)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(size_bucket(c->N));
    if (it != g_tune_cache.end()) {
        c->f32_tpt = it->second.first;
        c->f32_bps = it->second.second;
        c->tuned = 1;
    }
}

}  // namespace ibim

using namespace ibim;

extern "C" ibim_status ibim_autotune(ibim_ctx* c, const ibim_phys* phys, int* tpt_out, int* bps_out,
                                     double* best_ms)
{
    if (c == nullptr) {
        set_error("ctx is NULL");
        return IBIM_ERR_ARG;
    }
    IBIM_TRY(check_phys(phys));
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, (void**)&c->d_io, &c->io_bytes, sizeof(double) * 4 * N));
    double* in = c->d_io;
    double* out = c->d_io + 2 * N;
    fill_kernel<<<(unsigned)((2 * N + 255) / 256), 256, 0, c->stream>>>(in, 2 * N);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    const PairConsts k = make_consts(*phys);

    std::vector<std::pair<int, int>> cand;
    for (int tpt : {2, 4}) {
        const int occ = f32_max_bps(tpt);
        cand.push_back({tpt, occ});
        if (occ > 1) cand.push_back({tpt, occ / 2 > 0 ? occ / 2 : 1});
    }
    // Each repetition costs about N^2 / 5e11 s; keep the whole search short.
    const double est_ms = (double)N * (double)N / 5e8;
    const int reps = est_ms > 200.0 ? 1 : 2;
    cudaEvent_t e0, e1;
    IBIM_CUDA(cudaEventCreate(&e0));
    IBIM_CUDA(cudaEventCreate(&e1));
    const bool timing_was = c->timing.enabled;
    c->timing.enabled = false;
    double best = 1e300;
    std::pair<int, int> pick{c->f32_tpt, c->f32_bps};
    ibim_status st = IBIM_OK;
    for (const auto& v : cand) {
        c->f32_tpt = v.first;
        c->f32_bps = v.second;
        st = apply_operator(c, k, IBIM_F32C, VecRef{in, nullptr, 0, 0}, OutRef{out, nullptr, 0, 0}, nullptr);
        if (st != IBIM_OK) break;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && st == IBIM_OK; ++r)
            st = apply_operator(c, k, IBIM_F32C, VecRef{in, nullptr, 0, 0}, OutRef{out, nullptr, 0, 0}, nullptr);
        cudaEventRecord(e1, c->stream);
        if (st != IBIM_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best) {
            best = ms / reps;
            pick = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing.enabled = timing_was;
    c->f32_tpt = pick.first;
    c->f32_bps = pick.second;
    if (st != IBIM_OK) return st;
    c->tuned = 1;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[size_bucket(N)] = pick;
    }
    if (tpt_out) *tpt_out = pick.first;
    if (bps_out) *bps_out = pick.second;
    if (best_ms) *best_ms = best;
    return IBIM_OK;
}

extern "C" ibim_status ibim_set_f32_variant(ibim_ctx* c, int tpt, int bps)
{
    if (c == nullptr || (tpt != 2 && tpt != 4) || bps < 0) {
        set_error("need a context, targets_per_thread 2 or 4 and ctas_per_sm >= 0");
        return IBIM_ERR_ARG;
    }
    c->f32_tpt = tpt;
    c->f32_bps = bps;
    return IBIM_OK;
}
