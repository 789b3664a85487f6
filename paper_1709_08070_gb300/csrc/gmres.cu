// Restarted GMRES for (Lambda + K W) p = g (Sec. 3.3), all vector work in FP64
// on the device.
//
// One Arnoldi step is a fixed sequence of launches that reads the step index
// k from a device-resident state, so the same sequence can be captured once
// into a CUDA graph and replayed for every step:
//   pack/pairs/fixup        w = A v_k                       (operator of the chosen precision)
//   dots, reduce, update    classical Gram-Schmidt, twice   (CGS2)
//   norm reduce, scale      v_{k+1} = w / ||w||
//   givens                  rotate column k of H, update the residual estimate,
//                           set `done` on convergence / end of cycle
// Every launch first reads `done` and returns at once when it is set, so the
// host can replay a few steps ahead and poll the flag only occasionally.
//
// Outer loop: r = g - A_out x, one GMRES cycle on A_in d = r from d = 0,
// x += d.  Without certification A_out = A_in (plain restarted GMRES).  With
// certification A_out is an FP64-accurate operator: restarted GMRES with A_in
// runs to half the tolerance, then the residual is recomputed with A_out; if
// it misses the tolerance, the correction equation A e = r_out is solved the
// same way with A_in from e = 0 (its restart residuals r_out - A_in e) and
// x += e (iterative refinement).  The reported residual is the FP64-accurate
// one.
#include <math.h>
#include <string.h>

#include <vector>

#include "gmres_internal.cuh"

namespace ibim {

// ------------------------------------------------------------ vector kernels

// part[b * (k+1) + j] = sum over this block's elements of V_j . V_{k+1}, j <= k
__global__ void __launch_bounds__(kVecThreads)
    gs_dots_kernel(const double* __restrict__ V, int64_t len, const GmState* __restrict__ st,
                   double* __restrict__ part)
{
    if (st->done) return;
    __shared__ double red[kVecThreads / 32][kMaxRestart + 1];
    const int k = st->k;
    const double* w = V + (int64_t)(k + 1) * len;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j <= k; ++j) {
        const double* v = V + (int64_t)j * len;
        double s = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < len; i += (int64_t)gridDim.x * kVecThreads)
            s += v[i] * w[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][j] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= k; j += kVecThreads) {
        double s = 0.0;
        for (int q = 0; q < kVecThreads / 32; ++q) s += red[q][j];
        part[(int64_t)blockIdx.x * (kMaxRestart + 1) + j] = s;
    }
}

// coef[j] = sum_b part[b][j]; hcol[j] (+)= coef[j]  (pass 0 sets, pass 1 adds).
// One warp per coefficient: lane l sums blocks l, l + 32, ..., then a fixed
// butterfly (the same order every time, so the step is deterministic).
__global__ void __launch_bounds__(256)
    gs_reduce_kernel(const double* __restrict__ part, int nblk, GmState* __restrict__ st, int pass)
{
    if (st->done) return;
    const int k = st->k;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x >> 5; j <= k; j += nw) {
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * (kMaxRestart + 1) + j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            st->coef[j] = s;
            st->hcol[j] = (pass == 0) ? s : st->hcol[j] + s;
        }
    }
}

// V_{k+1} -= sum_j coef[j] V_j; optional per-block partial of ||V_{k+1}||^2 into part[b * (m+1) + 0]
__global__ void __launch_bounds__(kVecThreads)
    gs_update_kernel(double* __restrict__ V, int64_t len, const GmState* __restrict__ st,
                     double* __restrict__ part, int with_norm)
{
    if (st->done) return;
    __shared__ double coef[kMaxRestart + 1];
    __shared__ double red[kVecThreads / 32];
    const int k = st->k;
    for (int j = threadIdx.x; j <= k; j += kVecThreads) coef[j] = st->coef[j];
    __syncthreads();
    double* w = V + (int64_t)(k + 1) * len;
    double nn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < len; i += (int64_t)gridDim.x * kVecThreads) {
        double s = w[i];
        for (int j = 0; j <= k; ++j) s -= coef[j] * V[(int64_t)j * len + i];
        w[i] = s;
        nn += s * s;
    }
    if (!with_norm) return;
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kVecThreads / 32; ++q) s += red[q];
        part[(int64_t)blockIdx.x * (kMaxRestart + 1)] = s;
    }
}

__global__ void norm_reduce_kernel(const double* __restrict__ part, int nblk, GmState* __restrict__ st)
{
    if (st->done) return;
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)b * (kMaxRestart + 1)];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) st->hn = sqrt(red[0]);
}

__global__ void scale_kernel(double* __restrict__ V, int64_t len, const GmState* __restrict__ st)
{
    if (st->done) return;
    const double hn = st->hn;
    if (!(hn > 0.0)) return;
    const double inv = 1.0 / hn;
    double* w = V + (int64_t)(st->k + 1) * len;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        w[i] *= inv;
}

// Column k of H: earlier rotations, new rotation, residual estimate |e_{k+1}|.
__global__ void givens_kernel(GmState* __restrict__ st)
{
    if (st->done) return;
    const int k = st->k, m = st->m;
    double* H = st->H;
    for (int j = 0; j <= k; ++j) H[j * m + k] = st->hcol[j];
    const double hn = st->hn;
    H[(k + 1) * m + k] = hn;
    for (int j = 0; j < k; ++j) {
        const double a = H[j * m + k], b = H[(j + 1) * m + k];
        H[j * m + k] = st->cs[j] * a + st->sn[j] * b;
        H[(j + 1) * m + k] = -st->sn[j] * a + st->cs[j] * b;
    }
    const double a = H[k * m + k], b = H[(k + 1) * m + k];
    const double rr = hypot(a, b);
    const double c = (rr > 0.0) ? a / rr : 1.0;
    const double s = (rr > 0.0) ? b / rr : 0.0;
    st->cs[k] = c;
    st->sn[k] = s;
    H[k * m + k] = rr;
    H[(k + 1) * m + k] = 0.0;
    st->e[k + 1] = -s * st->e[k];
    st->e[k] = c * st->e[k];
    st->resid = fabs(st->e[k + 1]);
    st->k = k + 1;
    if (st->resid <= st->target) st->conv = 1;
    if (st->conv || st->k >= st->kmax || !(hn > 0.0)) st->done = 1;
}

// Back substitution H y = e (k x k upper triangular), then nothing else.
__global__ void trisolve_kernel(GmState* __restrict__ st)
{
    const int k = st->k, m = st->m;
    for (int i = k - 1; i >= 0; --i) {
        double s = st->e[i];
        for (int j = i + 1; j < k; ++j) s -= st->H[i * m + j] * st->y[j];
        st->y[i] = s / st->H[i * m + i];
    }
}

// x += sum_{j<k} y_j V_j
__global__ void xupdate_kernel(double* __restrict__ x, const double* __restrict__ V, int64_t len,
                               const GmState* __restrict__ st)
{
    __shared__ double y[kMaxRestart];
    const int k = st->k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) y[j] = st->y[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int j = 0; j < k; ++j) s += y[j] * V[(int64_t)j * len + i];
        x[i] = s;
    }
}

// r = g - t and per-block partial of ||r||^2 (part[b * (m+1)])
__global__ void __launch_bounds__(kVecThreads)
    residual_kernel(const double* __restrict__ g, const double* __restrict__ t, double* __restrict__ r, int64_t len,
                    double* __restrict__ part)
{
    __shared__ double red[kVecThreads / 32];
    double nn = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < len; i += (int64_t)gridDim.x * kVecThreads) {
        const double v = g[i] - (t ? t[i] : 0.0);
        r[i] = v;
        nn += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kVecThreads / 32; ++q) s += red[q];
        part[(int64_t)blockIdx.x * (kMaxRestart + 1)] = s;
    }
}

// New cycle: beta = sqrt(sum part), V_0 = r / beta, state reset with e = (beta, 0, ...).
__global__ void cycle_begin_reduce_kernel(const double* __restrict__ part, int nblk, GmState* __restrict__ st,
                                          double target, int kmax)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(int64_t)b * (kMaxRestart + 1)];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double beta = sqrt(red[0]);
        st->hn = beta;  // carries beta to the scaling kernel
        st->k = 0;
        st->conv = (beta <= target) ? 1 : 0;
        st->done = st->conv;
        st->kmax = kmax;
        st->target = target;
        st->resid = beta;
        for (int j = 0; j <= st->m; ++j) st->e[j] = 0.0;
        st->e[0] = beta;
    }
}

__global__ void cycle_begin_scale_kernel(const double* __restrict__ r, double* __restrict__ V0, int64_t len,
                                         const GmState* __restrict__ st)
{
    const double beta = st->hn;
    const double inv = (beta > 0.0) ? 1.0 / beta : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        V0[i] = r[i] * inv;
}

// x += y
__global__ void add_kernel(double* __restrict__ x, const double* __restrict__ y, int64_t len)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += y[i];
}

// x0 = Lambda^{-1} g (Sec. 3.3 initial guess with D = 0)
__global__ void lambda_inv_kernel(const double* __restrict__ g, double* __restrict__ x, int64_t N, double l1,
                                  double l2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    x[i] = g[i] / l1;
    x[N + i] = g[N + i] / l2;
}

// ------------------------------------------------------------------ host side

void gmres_free(ibim_ctx* c)
{
    GmresWork* w = c->gm;
    if (w == nullptr) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->gs) cudaStreamDestroy(w->gs);
    cudaFree(w->V);
    cudaFree(w->x);
    cudaFree(w->r);
    cudaFree(w->t);
    cudaFree(w->g);
    cudaFree(w->xb);
    cudaFree(w->gin);
    cudaFree(w->part);
    cudaFree(w->st);
    cudaFreeHost(w->h_st);
    delete w;
    c->gm = nullptr;
}

ibim_status gm_alloc(ibim_ctx* c, int m)
{
    const int64_t len = 2 * c->N;
    if (c->gm && c->gm->m >= m && c->gm->len == len) return IBIM_OK;
    gmres_free(c);
    GmresWork* w = new GmresWork();
    c->gm = w;
    w->m = m;
    w->len = len;
    w->nblk = (int)std::min<int64_t>(2 * c->num_sms, (len + kVecThreads - 1) / kVecThreads);
    if (w->nblk < 1) w->nblk = 1;
    IBIM_CUDA(cudaMalloc((void**)&w->V, sizeof(double) * (size_t)(m + 1) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->x, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->r, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->t, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->g, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->xb, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->gin, sizeof(double) * len));
    IBIM_CUDA(cudaMalloc((void**)&w->part, sizeof(double) * (size_t)w->nblk * (kMaxRestart + 1)));
    IBIM_CUDA(cudaMalloc((void**)&w->st, sizeof(GmState)));
    IBIM_CUDA(cudaMallocHost((void**)&w->h_st, sizeof(GmState)));
    IBIM_CUDA(cudaStreamCreateWithFlags(&w->gs, cudaStreamNonBlocking));
    IBIM_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
    return IBIM_OK;
}

ibim_status gm_ortho(ibim_ctx* c)
{
    GmresWork* w = c->gm;
    const int64_t len = w->len;
    for (int pass = 0; pass < 2; ++pass) {
        gs_dots_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->V, len, w->st, w->part);
        gs_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st, pass);
        gs_update_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->V, len, w->st, w->part, pass == 1);
    }
    norm_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st);
    scale_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->V, len, w->st);
    givens_kernel<<<1, 1, 0, c->stream>>>(w->st);
    count_launch(c, 9);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

// One Arnoldi step (see the file comment), all launches on c->stream.
static ibim_status arnoldi_step(ibim_ctx* c, const PairConsts& k, int precision)
{
    GmresWork* w = c->gm;
    const int64_t len = w->len;
    const int* skip = &w->st->done;
    VecRef in{w->V, &w->st->k, len, 0};
    OutRef out{w->V, &w->st->k, len, 1};
    IBIM_TRY(apply_operator(c, k, precision, in, out, skip));
    return gm_ortho(c);
}

ibim_status gm_cycle_begin(ibim_ctx* c, bool x_zero, double target, int kmax)
{
    GmresWork* w = c->gm;
    const int64_t len = w->len;
    residual_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->g, x_zero ? nullptr : w->t, w->r, len, w->part);
    cycle_begin_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st, target, kmax);
    cycle_begin_scale_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->r, w->V, len, w->st);
    count_launch(c, 3);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status gm_cycle_end(ibim_ctx* c)
{
    GmresWork* w = c->gm;
    trisolve_kernel<<<1, 1, 0, c->stream>>>(w->st);
    xupdate_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->x, w->V, w->len, w->st);
    count_launch(c, 2);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status gm_fetch_state(ibim_ctx* c)
{
    IBIM_CUDA(cudaMemcpyAsync(c->gm->h_st, c->gm->st, 64, cudaMemcpyDeviceToHost, c->stream));
    return IBIM_OK;
}

ibim_status gm_init(ibim_ctx* c, const ibim_phys& p, int m, double* gnorm)
{
    GmresWork* w = c->gm;
    GmState init;
    memset(&init, 0, sizeof(init));
    init.m = m;
    IBIM_CUDA(cudaMemcpyAsync(w->st, &init, sizeof(GmState), cudaMemcpyHostToDevice, c->stream));
    IBIM_TRY(rhs_launch(c, p.eps_in, w->g));
    residual_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->g, nullptr, w->r, w->len, w->part);
    cycle_begin_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st, 0.0, 0);
    count_launch(c, 2);
    IBIM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * w->len, c->stream));
    IBIM_CUDA(cudaMemcpyAsync(w->h_st, w->st, 64, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    *gnorm = w->h_st->resid;
    return IBIM_OK;
}

// r = rhs - A x with the operator of precision `prec` (or r = rhs when x is
// known to be zero); starts a cycle on r.
static ibim_status begin_cycle(ibim_ctx* c, const PairConsts& k, int prec, const double* rhs, bool x_zero,
                               double target, int kmax, double* beta_host)
{
    GmresWork* w = c->gm;
    const int64_t len = w->len;
    if (!x_zero)
        IBIM_TRY(apply_operator(c, k, prec, VecRef{w->x, nullptr, 0, 0}, OutRef{w->t, nullptr, 0, 0}, nullptr));
    residual_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(rhs, x_zero ? nullptr : w->t, w->r, len, w->part);
    cycle_begin_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st, target, kmax);
    cycle_begin_scale_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->r, w->V, len, w->st);
    count_launch(c, 3);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemcpyAsync(w->h_st, w->st, 64, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    *beta_host = w->h_st->resid;
    return IBIM_OK;
}

static ibim_status capture_step(ibim_ctx* c, const PairConsts& k, int precision)
{
    GmresWork* w = c->gm;
    // Every workspace the step (or a later operator application of either
    // precision) touches is sized for both precisions before capture, so that
    // no later call reallocates a buffer the graph holds a pointer to.
    IBIM_TRY(ensure_operator_workspaces(c));
    if (w->graph_valid && w->graph_prec == precision && memcmp(&w->graph_k, &k, sizeof(k)) == 0 &&
        w->graph_generation == c->ws_generation && w->graph_variant == c->f32_variant && w->graph_bps == c->f32_bps)
        return IBIM_OK;
    if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
    }
    w->graph_valid = false;
    cudaGraph_t graph = nullptr;
    IBIM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t launches_before = c->timing.total_launches;
    ibim_status s = arnoldi_step(c, k, precision);
    c->timing.total_launches = launches_before;  // capture does not launch
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (s != IBIM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "capture of the Arnoldi step", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&w->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate", __FILE__, __LINE__);
    w->graph_valid = true;
    w->graph_prec = precision;
    w->graph_k = k;
    w->graph_generation = c->ws_generation;
    w->graph_variant = c->f32_variant;
    w->graph_bps = c->f32_bps;
    return IBIM_OK;
}

// Runs steps until the device sets `done`; returns the steps taken.
static ibim_status run_cycle(ibim_ctx* c, const PairConsts& k, int precision, bool use_graph, int* steps,
                             int* conv)
{
    GmresWork* w = c->gm;
    const int per_poll = 2;
    int launched = 0;
    for (;;) {
        for (int q = 0; q < per_poll; ++q) {
            if (use_graph) {
                if (!w->graph_valid || w->graph_generation != c->ws_generation) {
                    set_error("captured GMRES step is stale (workspace reallocated)");
                    return IBIM_ERR_STATE;
                }
                IBIM_CUDA(cudaGraphLaunch(w->exec, c->stream));
                count_launch(c, 12);  // kernels in one captured step
            } else {
                IBIM_TRY(arnoldi_step(c, k, precision));
            }
            ++launched;
        }
        IBIM_CUDA(cudaMemcpyAsync(w->h_st, w->st, 64, cudaMemcpyDeviceToHost, c->stream));
        IBIM_CUDA(cudaStreamSynchronize(c->stream));
        if (w->h_st->done) break;
        if (launched > kMaxRestart + 4) {
            set_error("GMRES cycle did not terminate");
            return IBIM_ERR_CUDA;
        }
    }
    *steps = w->h_st->k;
    *conv = w->h_st->conv;
    return IBIM_OK;
}

ibim_status gmres_solve(ibim_ctx* c, const ibim_phys& p, const ibim_solve_opts& o, double* d_p,
                        ibim_solve_info* info)
{
    const int m = std::min(o.restart, kMaxRestart);
    IBIM_TRY(gm_alloc(c, m));
    GmresWork* w = c->gm;
    const int64_t len = w->len, N = c->N;
    const PairConsts k = make_consts(p);
    const int prec_in = o.precision;
    // The symmetric FP32 kernels add their reverse sums in a varying order, so
    // two applications to the same vector differ by about 1e-8 of |A p|; a
    // restart residual then cannot settle below that.  Uncertified solves asked
    // for a tighter tolerance run the one-directional kernel instead (restored
    // on exit).  Certified solves keep the symmetric kernel: once the first
    // check fails, the inner solves work on the correction equation, whose
    // right-hand side is the current residual, so the noise scales with it.
    struct KeepVariant {
        ibim_ctx* c;
        int v, b;
        ~KeepVariant()
        {
            c->f32_variant = v;
            c->f32_bps = b;
        }
    } keep_variant{c, c->f32_variant, c->f32_bps};
    if (prec_in == IBIM_F32C && o.certify == 0 && o.tol < kSymTolFloor && f32_variant_symmetric(c->f32_variant)) {
        c->f32_variant = f32_deterministic_variant();
        c->f32_bps = 0;
    }
    // certification operator: 1 = float-float pair sums (FP64-accurate on the
    // FP32 pipe), 2 = plain FP64 pair sums
    const int prec_out = o.certify == 2 ? IBIM_F64 : (o.certify ? IBIM_FF : o.precision);

    // Work on the solver's own stream (graph capture needs a non-legacy
    // stream), ordered after everything already queued on the caller's.
    cudaStream_t user = c->stream;
    IBIM_CUDA(cudaEventRecord(w->ev, user));
    IBIM_CUDA(cudaStreamWaitEvent(w->gs, w->ev, 0));
    c->stream = w->gs;
    struct Restore {
        ibim_ctx* c;
        cudaStream_t user;
        ~Restore()
        {
            cudaEventRecord(c->gm->ev, c->stream);
            cudaStreamWaitEvent(user, c->gm->ev, 0);
            c->stream = user;
        }
    } restore{c, user};

    GmState init;
    memset(&init, 0, sizeof(init));
    init.m = m;
    IBIM_CUDA(cudaMemcpyAsync(w->st, &init, sizeof(GmState), cudaMemcpyHostToDevice, c->stream));

    IBIM_TRY(rhs_launch(c, p.eps_in, w->g));
    // ||g||
    residual_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->g, nullptr, w->r, len, w->part);
    cycle_begin_reduce_kernel<<<1, 256, 0, c->stream>>>(w->part, w->nblk, w->st, 0.0, 0);
    count_launch(c, 2);
    IBIM_CUDA(cudaMemcpyAsync(w->h_st, w->st, 64, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    const double gnorm = w->h_st->resid;

    bool x_zero = false;
    if (o.start == 0) {
        IBIM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * len, c->stream));
        x_zero = true;
    } else if (o.start == 1) {
        lambda_inv_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(w->g, w->x, N, k.lambda1, k.lambda2);
        count_launch(c);
    } else {
        IBIM_CUDA(cudaMemcpyAsync(w->x, d_p, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
    }

    const bool use_graph = !c->timing.enabled;
    const double target_abs = o.tol * gnorm;
    const double inner_target = o.certify ? 0.5 * target_abs : target_abs;
    int iters = 0, cycles = 0;
    double beta = 0.0;
    bool converged = false;
    if (gnorm == 0.0) {
        IBIM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * len, c->stream));
        converged = true;
    }
    // Restart residuals use the iteration's operator; with certification the
    // residual is recomputed with the FP64-accurate operator once the iteration's
    // residual meets the inner target (or the iteration budget is spent).  A
    // failed check starts a solve of the correction equation on that residual:
    // xb keeps the iterate, x the correction from zero, gin the residual, and
    // restarts compute gin - A_in x until the next check adds xb back.  (Restart
    // residuals g - A_in x of the whole system would pull the iterate back to
    // A_in's own solution, which misses the tolerance whenever A_in differs
    // from A_out by more than the inner target, e.g. a treecode operator.)
    // A cycle that meets the inner target by its own estimate is followed by
    // the check at once: a restart residual with A_in could only confirm the
    // estimate (then the check follows) or show A_in's accuracy floor (the
    // FP32 operator is linear only to about 1e-8 of |A x|; further cycles
    // could not go lower, so the check follows as well).
    bool check = false, refining = false;
    while (!converged) {
        const int kmax = std::min(m, o.maxit - iters);
        const int prec_r = (check || kmax <= 0) ? prec_out : prec_in;
        if (prec_r == prec_out && refining) {
            add_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->x, w->xb, len);
            count_launch(c);
            refining = false;
        }
        if (!x_zero) {
            if (prec_r == IBIM_F32C || prec_r == IBIM_F32T) info->matvecs_f32 += 1;
            else info->matvecs_f64 += 1;
        }
        IBIM_TRY(begin_cycle(c, k, prec_r, refining ? w->gin : w->g, x_zero, inner_target, std::max(kmax, 0),
                             &beta));
        x_zero = false;
        if (prec_r == prec_out && beta <= target_abs) {
            converged = true;
            break;
        }
        if (prec_r != prec_out && beta <= inner_target) {
            check = true;
            continue;
        }
        check = false;
        if (kmax <= 0) break;
        if (prec_r != prec_in) {  // failed check: the cycle below starts on r = g - A_out x
            IBIM_CUDA(cudaMemcpyAsync(w->xb, w->x, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
            IBIM_CUDA(cudaMemcpyAsync(w->gin, w->r, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
            IBIM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * len, c->stream));
            refining = true;
        }
        if (use_graph) IBIM_TRY(capture_step(c, k, prec_in));
        int steps = 0, conv = 0;
        IBIM_TRY(run_cycle(c, k, prec_in, use_graph, &steps, &conv));
        iters += steps;
        ++cycles;
        check = prec_out != prec_in && conv != 0;
        info->matvecs_f32 += (prec_in == IBIM_F32C || prec_in == IBIM_F32T) ? steps : 0;
        info->matvecs_f64 += (prec_in == IBIM_F64 || prec_in == IBIM_FF) ? steps : 0;
        if (steps > 0) {
            trisolve_kernel<<<1, 1, 0, c->stream>>>(w->st);
            xupdate_kernel<<<w->nblk, kVecThreads, 0, c->stream>>>(w->x, w->V, len, w->st);
            count_launch(c, 2);
            IBIM_CUDA(cudaGetLastError());
        }
    }
    info->iters = iters;
    info->cycles = cycles;
    info->converged = converged ? 1 : 0;
    info->relres = (gnorm > 0.0) ? beta / gnorm : 0.0;
    IBIM_CUDA(cudaMemcpyAsync(d_p, w->x, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));

    double gpol = 0.0, area = 0.0;
    IBIM_TRY(energy_launch(c, p, w->x, nullptr, &gpol));
    IBIM_TRY(area_launch(c, &area));
    info->gpol = gpol;
    info->gpol_kcal = gpol * kKcalPerE2A;
    info->area = area;
    return converged ? IBIM_OK : IBIM_ERR_NOT_CONVERGED;
}

}  // namespace ibim
