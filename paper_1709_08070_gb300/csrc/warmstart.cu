// Learned warm start for GMRES (not part of the paper's method): a small
// per-node network maps local, size-free features of the right-hand side,
// the geometry and the physical constants to an initial [psi; psin].  GMRES
// from the zero start remains the reference; the network only shortens it.
//
// Features of node i (all O(1) and independent of the molecule's size):
//   S1 = sqrt(sum w g1^2 / sum w), S2 = same for g2 (w = quadrature weights),
//   L = S1/S2 (a length), f0 = g1/S1, f1 = g2/S2, f2 = d/eps (offset in the
//   band), f3 = clamp(H L, -10, 10)/10 (H = Laplacian of the distance),
//   f4 = kappa L/(1 + kappa L), f5 = ln(eps_E/eps_I)/5,
//   f6 = (eps_I/eps_E)/(1 + kappa L), f7 = r1/S1, f8 = r2/S2 with
//   r = g - A Lambda^-1 g = -K Lambda^-1 g, the residual of the Lambda^-1 g
//   start (one application of the FP32 operator): the only non-local input,
//   it carries the reaction field of the first Neumann step to every node.
// Network: 9 -> 64 -> 64 -> 2, tanh hidden layers; BF16 weights, FP32
// arithmetic and accumulation; FP32 master weights and Adam moments.
// Outputs: psi_i = S1 o0 / lambda1, psin_i = S2 o1 / lambda2 (Lambda the
// diagonal of the system, Sec. 3.3).
// Training loss: sum over sampled nodes of (w_i / mean w) |o - t|^2 / batch,
// t = (lambda1 psi/S1, lambda2 psin/S2) of solutions the method computed.
// Scaling the targets by Lambda weights the two blocks by their share of
// the initial residual g - A p0 (A = Lambda + K), which is what GMRES sees:
// unscaled, the psi block (lambda1 = (1 + eps_E/eps_I)/2, 40.5 for
// water/protein) would be under-weighted by lambda1^2.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

constexpr int kWsIn = 9, kWsH = 64, kWsOut = 2;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kWsH * kWsIn;
constexpr int kOffW2 = kOffB1 + kWsH;
constexpr int kOffB2 = kOffW2 + kWsH * kWsH;
constexpr int kOffW3 = kOffB2 + kWsH;
constexpr int kOffB3 = kOffW3 + kWsOut * kWsH;
constexpr int kWsParams = kOffB3 + kWsOut;  // 4930
constexpr int kWsThreads = 128;             // nodes per training block
constexpr int kHPad = kWsH + 1;             // padded smem row (bank conflicts)

static_assert(kWsParams == IBIM_WS_NPARAMS, "parameter count");

}  // namespace ibim

struct ibim_wsnet {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* d_w = nullptr;           // FP32 master parameters
    __nv_bfloat16* d_wb = nullptr;  // BF16 parameters used by the kernels
    float* d_m = nullptr;           // Adam first moment
    float* d_v = nullptr;           // Adam second moment
    float* d_g = nullptr;           // gradient accumulator
    double* d_loss = nullptr;
    double* d_scal = nullptr;       // S1, S2 scratch
    float* d_feat = nullptr;        // training features (n_ex x 8)
    float* d_tgt = nullptr;         // training targets (n_ex x 2)
    float* d_wt = nullptr;          // training node weights (n_ex)
    int64_t n_ex = 0, cap_ex = 0;
    int64_t step = 0;
    uint64_t seed = 0;
};

namespace ibim {

// ---------------------------------------------------------------- features

// S1, S2 (one CTA, fixed summation order).
__global__ void ws_scales_kernel(const double* __restrict__ g, const double* __restrict__ w, int64_t N,
                                 double* __restrict__ scal)
{
    __shared__ double r[3][256];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        a += w[i] * g[i] * g[i];
        b += w[i] * g[N + i] * g[N + i];
        c += w[i];
    }
    r[0][threadIdx.x] = a;
    r[1][threadIdx.x] = b;
    r[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sw = r[2][0] > 0.0 ? r[2][0] : 1.0;
        const double s1 = sqrt(r[0][0] / sw), s2 = sqrt(r[1][0] / sw);
        scal[0] = s1 > 0.0 ? s1 : 1.0;
        scal[1] = s2 > 0.0 ? s2 : 1.0;
        scal[2] = sw / (double)(N > 0 ? N : 1);  // mean weight
    }
}

struct WsPhys {
    double kappa, eps_ratio_log, inv_ratio, band_eps;
};

__global__ void ws_features_kernel(const double* __restrict__ g, const double* __restrict__ Ax0,
                                   const double* __restrict__ dist, const double* __restrict__ curv, int64_t N,
                                   const double* __restrict__ scal, WsPhys ph, float* __restrict__ feat)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double S1 = scal[0], S2 = scal[1];
    const double L = S1 / S2;
    const double kL = ph.kappa * L;
    double hl = curv[i] * L;
    hl = hl > 10.0 ? 10.0 : (hl < -10.0 ? -10.0 : hl);
    float* f = feat + i * kWsIn;
    f[0] = (float)(g[i] / S1);
    f[1] = (float)(g[N + i] / S2);
    f[2] = (float)(ph.band_eps > 0.0 ? dist[i] / ph.band_eps : 0.0);
    f[3] = (float)(hl / 10.0);
    f[4] = (float)(kL / (1.0 + kL));
    f[5] = (float)(ph.eps_ratio_log / 5.0);
    f[6] = (float)(ph.inv_ratio / (1.0 + kL));
    f[7] = (float)((g[i] - Ax0[i]) / S1);
    f[8] = (float)((g[N + i] - Ax0[N + i]) / S2);
}

// x0 = Lambda^-1 g (the start of Sec. 3.3).
__global__ void ws_start_kernel(const double* __restrict__ g, int64_t N, double lambda1, double lambda2,
                                double* __restrict__ x0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    x0[i] = g[i] / lambda1;
    x0[N + i] = g[N + i] / lambda2;
}

__global__ void ws_targets_kernel(const double* __restrict__ p, const double* __restrict__ w, int64_t N,
                                  const double* __restrict__ scal, double lambda1, double lambda2,
                                  float* __restrict__ tgt, float* __restrict__ wt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    tgt[2 * i] = (float)(lambda1 * p[i] / scal[0]);
    tgt[2 * i + 1] = (float)(lambda2 * p[N + i] / scal[1]);
    wt[i] = (float)(w[i] / scal[2]);
}

// ----------------------------------------------------------------- network

__device__ __forceinline__ void load_params(const __nv_bfloat16* __restrict__ wb, float* sp)
{
    for (int q = threadIdx.x; q < kWsParams; q += blockDim.x) sp[q] = __bfloat162float(wb[q]);
}

// Forward pass of one node from its features (params in shared memory).
__device__ __forceinline__ void ws_forward(const float* sp, const float* x, float* h1, float* h2, float* o)
{
    for (int a = 0; a < kWsH; ++a) {
        float s = sp[kOffB1 + a];
#pragma unroll
        for (int b = 0; b < kWsIn; ++b) s = fmaf(sp[kOffW1 + a * kWsIn + b], x[b], s);
        h1[a] = tanhf(s);
    }
    for (int a = 0; a < kWsH; ++a) {
        float s = sp[kOffB2 + a];
        for (int b = 0; b < kWsH; ++b) s = fmaf(sp[kOffW2 + a * kWsH + b], h1[b], s);
        h2[a] = tanhf(s);
    }
    for (int c = 0; c < kWsOut; ++c) {
        float s = sp[kOffB3 + c];
        for (int a = 0; a < kWsH; ++a) s = fmaf(sp[kOffW3 + c * kWsH + a], h2[a], s);
        o[c] = s;
    }
}

__global__ void __launch_bounds__(kWsThreads)
    ws_predict_kernel(const float* __restrict__ feat, int64_t N, const __nv_bfloat16* __restrict__ wb,
                      const double* __restrict__ scal, double lambda1, double lambda2, double* __restrict__ p0)
{
    extern __shared__ float smem[];
    float* sp = smem;
    float* rows = smem + kWsParams;  // per thread: h1, h2 (2 x kHPad)
    load_params(wb, sp);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[kWsIn];
#pragma unroll
    for (int b = 0; b < kWsIn; ++b) x[b] = feat[i * kWsIn + b];
    float* h1 = rows + threadIdx.x * 2 * kHPad;
    float* h2 = h1 + kHPad;
    float o[kWsOut];
    ws_forward(sp, x, h1, h2, o);
    p0[i] = scal[0] * (double)o[0] / lambda1;
    p0[N + i] = scal[1] * (double)o[1] / lambda2;
}

// splitmix64 (Steele, Lea, Flood 2014) for minibatch sampling.
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Loss and gradient over a batch: node of slot (block, thread) is either
// consecutive (first + slot, full-batch mode) or drawn at random.
__global__ void __launch_bounds__(kWsThreads)
    ws_grad_kernel(const float* __restrict__ feat, const float* __restrict__ tgt, const float* __restrict__ wt,
                   int64_t n_ex, int64_t first, int64_t count, int random, uint64_t seed, double inv_batch,
                   const __nv_bfloat16* __restrict__ wb, float* __restrict__ grad, double* __restrict__ loss)
{
    extern __shared__ float smem[];
    float* sp = smem;                               // params
    float* X = sp + kWsParams;                      // [128][kWsIn]
    float* H1 = X + kWsThreads * kWsIn;             // [128][kHPad]
    float* H2 = H1 + kWsThreads * kHPad;
    float* D1 = H2 + kWsThreads * kHPad;
    float* D2 = D1 + kWsThreads * kHPad;
    float* DO = D2 + kWsThreads * kHPad;            // [128][2]
    __shared__ double lred[kWsThreads];
    load_params(wb, sp);
    __syncthreads();
    const int t = threadIdx.x;
    const int64_t slot = (int64_t)blockIdx.x * kWsThreads + t;
    const bool live = slot < count;
    float* x = X + t * kWsIn;
    float* h1 = H1 + t * kHPad;
    float* h2 = H2 + t * kHPad;
    float* d1 = D1 + t * kHPad;
    float* d2 = D2 + t * kHPad;
    float* dO = DO + t * kWsOut;
    double l = 0.0;
    if (live) {
        const int64_t i = random ? (int64_t)(mix64(seed ^ (uint64_t)slot) % (uint64_t)n_ex) : first + slot;
        for (int b = 0; b < kWsIn; ++b) x[b] = feat[i * kWsIn + b];
        float o[kWsOut];
        ws_forward(sp, x, h1, h2, o);
        const float w = wt[i];
        const float e0 = o[0] - tgt[2 * i], e1 = o[1] - tgt[2 * i + 1];
        l = (double)w * ((double)e0 * e0 + (double)e1 * e1) * inv_batch;
        dO[0] = (float)(2.0 * inv_batch) * w * e0;
        dO[1] = (float)(2.0 * inv_batch) * w * e1;
        for (int a = 0; a < kWsH; ++a) {
            float s = 0.0f;
            for (int c = 0; c < kWsOut; ++c) s = fmaf(sp[kOffW3 + c * kWsH + a], dO[c], s);
            d2[a] = s * (1.0f - h2[a] * h2[a]);
        }
        for (int b = 0; b < kWsH; ++b) {
            float s = 0.0f;
            for (int a = 0; a < kWsH; ++a) s = fmaf(sp[kOffW2 + a * kWsH + b], d2[a], s);
            d1[b] = s * (1.0f - h1[b] * h1[b]);
        }
    } else {
        for (int b = 0; b < kWsIn; ++b) x[b] = 0.0f;
        for (int a = 0; a < kWsH; ++a) h1[a] = h2[a] = d1[a] = d2[a] = 0.0f;
        dO[0] = dO[1] = 0.0f;
    }
    lred[t] = l;
    __syncthreads();
    // weight gradients: contractions over the block's nodes
    for (int e = t; e < kWsH * kWsH; e += kWsThreads) {  // dW2[a][b] = sum_n d2[n][a] h1[n][b]
        const int a = e / kWsH, b = e % kWsH;
        float s = 0.0f;
        for (int n = 0; n < kWsThreads; ++n) s = fmaf(D2[n * kHPad + a], H1[n * kHPad + b], s);
        atomicAdd(grad + kOffW2 + e, s);
    }
    for (int e = t; e < kWsH * kWsIn; e += kWsThreads) {  // dW1[a][b] = sum_n d1[n][a] x[n][b]
        const int a = e / kWsIn, b = e % kWsIn;
        float s = 0.0f;
        for (int n = 0; n < kWsThreads; ++n) s = fmaf(D1[n * kHPad + a], X[n * kWsIn + b], s);
        atomicAdd(grad + kOffW1 + e, s);
    }
    for (int e = t; e < kWsOut * kWsH; e += kWsThreads) {  // dW3[c][a] = sum_n dO[n][c] h2[n][a]
        const int c = e / kWsH, a = e % kWsH;
        float s = 0.0f;
        for (int n = 0; n < kWsThreads; ++n) s = fmaf(DO[n * kWsOut + c], H2[n * kHPad + a], s);
        atomicAdd(grad + kOffW3 + e, s);
    }
    if (t < kWsH) {
        float s1 = 0.0f, s2 = 0.0f;
        for (int n = 0; n < kWsThreads; ++n) {
            s1 += D1[n * kHPad + t];
            s2 += D2[n * kHPad + t];
        }
        atomicAdd(grad + kOffB1 + t, s1);
        atomicAdd(grad + kOffB2 + t, s2);
    }
    if (t < kWsOut) {
        float s = 0.0f;
        for (int n = 0; n < kWsThreads; ++n) s += DO[n * kWsOut + t];
        atomicAdd(grad + kOffB3 + t, s);
    }
    for (int o = kWsThreads / 2; o > 0; o >>= 1) {
        __syncthreads();
        if (t < o) lred[t] += lred[t + o];
    }
    if (t == 0) atomicAdd(loss, lred[0]);
}

// Adam (Kingma and Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void ws_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                               const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, float lr, float b1,
                               float b2, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kWsParams) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
    w[q] = wq;
    wb[q] = __float2bfloat16_rn(wq);
}

__global__ void ws_to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kWsParams) wb[q] = __float2bfloat16_rn(w[q]);
}

static size_t grad_smem() { return sizeof(float) * (kWsParams + kWsThreads * (kWsIn + 4 * kHPad + kWsOut)); }
static size_t predict_smem() { return sizeof(float) * (kWsParams + kWsThreads * 2 * kHPad); }

// Features (into c->d_io as floats after the RHS) and scales of one context.
static ibim_status ws_prepare(ibim_wsnet* net, ibim_ctx* c, const ibim_phys& p, float** feat_out)
{
    const int64_t N = c->N;
    // d_io: 2N doubles RHS g, 2N doubles x0 = Lambda^-1 g, 2N doubles A x0,
    // then N x kWsIn floats features
    IBIM_TRY(ensure(c, (void**)&c->d_io, &c->io_bytes, sizeof(double) * 6 * N + sizeof(float) * kWsIn * N + 64));
    double* g = c->d_io;
    double* x0 = c->d_io + 2 * N;
    double* ax0 = c->d_io + 4 * N;
    float* feat = (float*)(c->d_io + 6 * N);
    IBIM_TRY(rhs_launch(c, p.eps_in, g));
    const PairConsts k = make_consts(p);
    ws_start_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(g, N, k.lambda1, k.lambda2, x0);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_TRY(apply_operator(c, k, IBIM_F32C, VecRef{x0, nullptr, 0, 0}, OutRef{ax0, nullptr, 0, 0}, nullptr));
    ws_scales_kernel<<<1, 256, 0, c->stream>>>(g, c->d_geo64 + 6 * N, N, net->d_scal);
    WsPhys ph;
    ph.kappa = p.kappa;
    ph.eps_ratio_log = log(p.eps_out / p.eps_in);
    ph.inv_ratio = p.eps_in / p.eps_out;
    ph.band_eps = c->band_eps;
    ws_features_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(g, ax0, c->d_dist, c->d_curv, N,
                                                                          net->d_scal, ph, feat);
    count_launch(c, 2);
    IBIM_CUDA(cudaGetLastError());
    *feat_out = feat;
    return IBIM_OK;
}

// Splitmix-driven uniform initialisation, Glorot bounds per layer.
static void init_params(uint64_t seed, std::vector<float>& w)
{
    w.assign(kWsParams, 0.0f);
    uint64_t s = seed;
    auto next = [&]() {
        s += 0x9e3779b97f4a7c15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int fan_in, int fan_out) {
        const double a = sqrt(6.0 / (fan_in + fan_out));
        for (int q = 0; q < fan_in * fan_out; ++q) w[off + q] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(kOffW1, kWsIn, kWsH);
    fill(kOffW2, kWsH, kWsH);
    fill(kOffW3, kWsH, kWsOut);
}

}  // namespace ibim

using namespace ibim;

extern "C" {

void ibim_wsnet_destroy(ibim_wsnet* n)
{
    if (n == nullptr) return;
    cudaStreamSynchronize(n->stream);
    cudaFree(n->d_w);
    cudaFree(n->d_wb);
    cudaFree(n->d_m);
    cudaFree(n->d_v);
    cudaFree(n->d_g);
    cudaFree(n->d_loss);
    cudaFree(n->d_scal);
    cudaFree(n->d_feat);
    cudaFree(n->d_tgt);
    cudaFree(n->d_wt);
    delete n;
}

ibim_status ibim_wsnet_create(uint64_t seed, void* stream, ibim_wsnet** out)
{
    if (out == nullptr) {
        set_error("out is NULL");
        return IBIM_ERR_ARG;
    }
    *out = nullptr;
    ibim_wsnet* n = new ibim_wsnet();
    n->stream = (cudaStream_t)stream;
    n->seed = seed;
    std::vector<float> w;
    init_params(seed, w);
    cudaError_t e = cudaGetDevice(&n->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_w, sizeof(float) * kWsParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_wb, sizeof(__nv_bfloat16) * kWsParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_m, sizeof(float) * kWsParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_v, sizeof(float) * kWsParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_g, sizeof(float) * kWsParams);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_scal, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->d_w, w.data(), sizeof(float) * kWsParams, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_m, 0, sizeof(float) * kWsParams, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_v, 0, sizeof(float) * kWsParams, n->stream);
    if (e == cudaSuccess) {
        ws_to_bf16_kernel<<<(kWsParams + 255) / 256, 256, 0, n->stream>>>(n->d_w, n->d_wb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)predict_smem());
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        ibim_wsnet_destroy(n);
        return cuda_fail(e, "wsnet create", __FILE__, __LINE__);
    }
    *out = n;
    return IBIM_OK;
}

ibim_status ibim_wsnet_get_params(const ibim_wsnet* n, float* h_params)
{
    if (n == nullptr || h_params == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    IBIM_CUDA(cudaMemcpyAsync(h_params, n->d_w, sizeof(float) * kWsParams, cudaMemcpyDeviceToHost, n->stream));
    IBIM_CUDA(cudaStreamSynchronize(n->stream));
    return IBIM_OK;
}

ibim_status ibim_wsnet_set_params(ibim_wsnet* n, const float* h_params)
{
    if (n == nullptr || h_params == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    for (int q = 0; q < kWsParams; ++q)
        if (!isfinite(h_params[q])) {
            set_error("non-finite parameter");
            return IBIM_ERR_NONFINITE;
        }
    IBIM_CUDA(cudaMemcpyAsync(n->d_w, h_params, sizeof(float) * kWsParams, cudaMemcpyHostToDevice, n->stream));
    ws_to_bf16_kernel<<<(kWsParams + 255) / 256, 256, 0, n->stream>>>(n->d_w, n->d_wb);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemsetAsync(n->d_m, 0, sizeof(float) * kWsParams, n->stream));
    IBIM_CUDA(cudaMemsetAsync(n->d_v, 0, sizeof(float) * kWsParams, n->stream));
    IBIM_CUDA(cudaStreamSynchronize(n->stream));
    n->step = 0;
    return IBIM_OK;
}

ibim_status ibim_wsnet_features(ibim_wsnet* n, ibim_ctx* c, const ibim_phys* p, float* h_feat, double* h_scales)
{
    if (n == nullptr || c == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    IBIM_TRY(check_phys(p));
    if (c->Nc <= 0) {
        set_error("no charges set");
        return IBIM_ERR_STATE;
    }
    float* feat = nullptr;
    IBIM_TRY(ws_prepare(n, c, *p, &feat));
    if (h_feat) IBIM_CUDA(cudaMemcpyAsync(h_feat, feat, sizeof(float) * kWsIn * c->N, cudaMemcpyDeviceToHost, c->stream));
    if (h_scales) IBIM_CUDA(cudaMemcpyAsync(h_scales, n->d_scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

ibim_status ibim_wsnet_add_example(ibim_wsnet* n, ibim_ctx* c, const ibim_phys* p, const double* d_p)
{
    if (n == nullptr || c == nullptr || d_p == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    IBIM_TRY(check_phys(p));
    if (c->Nc <= 0) {
        set_error("no charges set");
        return IBIM_ERR_STATE;
    }
    const int64_t N = c->N;
    if (n->n_ex + N > n->cap_ex) {
        int64_t cap = std::max<int64_t>(2 * n->cap_ex, n->n_ex + N);
        float *f = nullptr, *t = nullptr, *w = nullptr;
        IBIM_CUDA(cudaStreamSynchronize(n->stream));
        IBIM_CUDA(cudaMalloc((void**)&f, sizeof(float) * kWsIn * cap));
        IBIM_CUDA(cudaMalloc((void**)&t, sizeof(float) * kWsOut * cap));
        IBIM_CUDA(cudaMalloc((void**)&w, sizeof(float) * cap));
        if (n->n_ex > 0) {
            IBIM_CUDA(cudaMemcpy(f, n->d_feat, sizeof(float) * kWsIn * n->n_ex, cudaMemcpyDeviceToDevice));
            IBIM_CUDA(cudaMemcpy(t, n->d_tgt, sizeof(float) * kWsOut * n->n_ex, cudaMemcpyDeviceToDevice));
            IBIM_CUDA(cudaMemcpy(w, n->d_wt, sizeof(float) * n->n_ex, cudaMemcpyDeviceToDevice));
        }
        cudaFree(n->d_feat);
        cudaFree(n->d_tgt);
        cudaFree(n->d_wt);
        n->d_feat = f;
        n->d_tgt = t;
        n->d_wt = w;
        n->cap_ex = cap;
    }
    float* feat = nullptr;
    IBIM_TRY(ws_prepare(n, c, *p, &feat));
    IBIM_CUDA(cudaMemcpyAsync(n->d_feat + kWsIn * n->n_ex, feat, sizeof(float) * kWsIn * N, cudaMemcpyDeviceToDevice,
                              c->stream));
    const PairConsts k = make_consts(*p);
    ws_targets_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(
        d_p, c->d_geo64 + 6 * N, N, n->d_scal, k.lambda1, k.lambda2, n->d_tgt + kWsOut * n->n_ex, n->d_wt + n->n_ex);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    n->n_ex += N;
    return IBIM_OK;
}

ibim_status ibim_wsnet_num_examples(const ibim_wsnet* n, int64_t* count)
{
    if (n == nullptr || count == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    *count = n->n_ex;
    return IBIM_OK;
}

ibim_status ibim_wsnet_gradient(ibim_wsnet* n, int64_t first, int64_t count, double* loss, float* h_grad)
{
    if (n == nullptr || loss == nullptr || h_grad == nullptr || first < 0 || count < 1 || first + count > n->n_ex) {
        set_error("need a net and 0 <= first, first + count <= number of examples, count >= 1");
        return IBIM_ERR_ARG;
    }
    IBIM_CUDA(cudaMemsetAsync(n->d_g, 0, sizeof(float) * kWsParams, n->stream));
    IBIM_CUDA(cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
    const unsigned blocks = (unsigned)((count + kWsThreads - 1) / kWsThreads);
    ws_grad_kernel<<<blocks, kWsThreads, grad_smem(), n->stream>>>(n->d_feat, n->d_tgt, n->d_wt, n->n_ex, first, count,
                                                                   0, 0, 1.0 / (double)count, n->d_wb, n->d_g,
                                                                   n->d_loss);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemcpyAsync(h_grad, n->d_g, sizeof(float) * kWsParams, cudaMemcpyDeviceToHost, n->stream));
    IBIM_CUDA(cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    IBIM_CUDA(cudaStreamSynchronize(n->stream));
    return IBIM_OK;
}

ibim_status ibim_wsnet_train(ibim_wsnet* n, int steps, int batch_nodes, double lr, double* last_loss)
{
    if (n == nullptr || steps < 1 || batch_nodes < 1 || !(lr > 0.0)) {
        set_error("need a net, steps >= 1, batch_nodes >= 1, lr > 0");
        return IBIM_ERR_ARG;
    }
    if (n->n_ex < 1) {
        set_error("no training examples");
        return IBIM_ERR_STATE;
    }
    const unsigned blocks = (unsigned)((batch_nodes + kWsThreads - 1) / kWsThreads);
    const double b1 = 0.9, b2 = 0.999;
    for (int s = 0; s < steps; ++s) {
        ++n->step;
        IBIM_CUDA(cudaMemsetAsync(n->d_g, 0, sizeof(float) * kWsParams, n->stream));
        IBIM_CUDA(cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
        const uint64_t sd = n->seed * 0x9e3779b97f4a7c15ull + (uint64_t)n->step * 0xd1b54a32d192ed03ull;
        ws_grad_kernel<<<blocks, kWsThreads, grad_smem(), n->stream>>>(n->d_feat, n->d_tgt, n->d_wt, n->n_ex, 0,
                                                                       batch_nodes, 1, sd, 1.0 / (double)batch_nodes,
                                                                       n->d_wb, n->d_g, n->d_loss);
        const float c1 = (float)(1.0 - pow(b1, (double)n->step)), c2 = (float)(1.0 - pow(b2, (double)n->step));
        ws_adam_kernel<<<(kWsParams + 255) / 256, 256, 0, n->stream>>>(n->d_w, n->d_m, n->d_v, n->d_g, n->d_wb,
                                                                       (float)lr, (float)b1, (float)b2, c1, c2);
        IBIM_CUDA(cudaGetLastError());
    }
    if (last_loss) {
        IBIM_CUDA(cudaMemcpyAsync(last_loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        IBIM_CUDA(cudaStreamSynchronize(n->stream));
    }
    return IBIM_OK;
}

ibim_status ibim_wsnet_predict(ibim_wsnet* n, ibim_ctx* c, const ibim_phys* p, double* d_p0)
{
    if (n == nullptr || c == nullptr || d_p0 == nullptr) {
        set_error("NULL argument");
        return IBIM_ERR_ARG;
    }
    IBIM_TRY(check_phys(p));
    if (c->Nc <= 0) {
        set_error("no charges set");
        return IBIM_ERR_STATE;
    }
    // order the net's own work (training) before the context's stream
    cudaEvent_t ev;
    IBIM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    IBIM_CUDA(cudaEventRecord(ev, n->stream));
    IBIM_CUDA(cudaStreamWaitEvent(c->stream, ev, 0));
    IBIM_CUDA(cudaEventDestroy(ev));
    float* feat = nullptr;
    IBIM_TRY(ws_prepare(n, c, *p, &feat));
    const unsigned blocks = (unsigned)((c->N + kWsThreads - 1) / kWsThreads);
    const PairConsts k = make_consts(*p);
    ws_predict_kernel<<<blocks, kWsThreads, predict_smem(), c->stream>>>(feat, c->N, n->d_wb, n->d_scal, k.lambda1,
                                                                         k.lambda2, d_p0);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

}  // extern "C"
