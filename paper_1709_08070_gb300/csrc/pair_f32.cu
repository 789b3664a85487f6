// FP32 compensated pair sums of the IBIM operator (Sec. 2.2 discrete system,
// Sec. 2.2.1 regularisation), sm_103a.
//
// One launch evaluates all N x N (target, source) interactions of
//   y1_i = sum_j [K11 a_j - K12 b_j],  y2_i = sum_j [K21 a_j - K22 b_j],
// a_j = w_j psi_j, b_j = w_j psin_j, with the kernels written (times 4 pi) as
//   K11 = s_y (1 - th1 A) / rho^3        K12 = (1 - E) / rho
//   K21 = [(1 - A) c - (3 - B) s_x s_y / rho^2] / rho^3
//   K22 = -s_x (1 - th2 A) / rho^3
// where E = exp(-kappa rho), A = E (1 + kappa rho), B = E (3 + 3 kappa rho + kappa^2 rho^2).
// With x = kappa rho the differences are formed as g = 1 - A = (1 - E) - E x,
// 3 - B = 3 g - E x^2 and 1 - E = g + E x.
//
// Schedule: persistent CTAs walk a stream-K range of (target tile, source
// tile) steps.  Source tiles (kF32STile nodes, 32 B each) are brought into
// shared memory by bulk async copies with an mbarrier per stage (double
// buffered).  Each thread owns TPT targets.
//
// Near/far split: every step compares the bounding spheres of its target tile
// and source tile.  When they are at least `far_dist` apart (>= 2 tau and
// >= 1.5 A), no pair of the step can lie in the regularisation tube
// (tube rule 0) and the cancellation in g is harmless, so the step runs a
// branch-free loop with no tube masks.  Otherwise every pair gets the tube
// test and, when any lane of the warp has x < 0.5, g from its Taylor series
// (from the exponential series).  The choice is uniform over the CTA.
//
// Accumulation: per target the two sums run in FP32 over chunks of
// kChunk sources (fused into the FMAs), each chunk sum is Kahan-added into a
// compensated FP32 pair (s, c), and at the end of each source tile the
// compensated value s - c is added to FP64 accumulators.  Every CTA writes one
// FP64 partial per target tile it touched; the fixup kernel adds the
// partials, scales by 1/(4 pi) and adds the diagonal Lambda p.
#include "ibim_internal.cuh"
#include "ptx.cuh"

namespace ibim {

struct F32Consts {
    float th1, th2, omth1, omth2;
    float kappa, kl2e;        // kappa and -kappa log2(e)
    float tau2, four_tau2, k12t;
    float far_dist;           // minimum bounding-sphere gap of a far step (A)
    int rule0;                // tube rule 0 (far steps allowed)
};

static F32Consts f32_consts(const PairConsts& k)
{
    F32Consts c;
    c.th1 = (float)k.th1;
    c.th2 = (float)k.th2;
    c.omth1 = (float)(1.0 - k.th1);
    c.omth2 = (float)(1.0 - k.th2);
    c.kappa = (float)k.kappa;
    c.kl2e = (float)(-k.kappa * 1.4426950408889634);
    c.tau2 = (float)k.tau2;
    c.rule0 = (k.four_tau2 < 3.0e38) ? 1 : 0;
    c.four_tau2 = c.rule0 ? (float)k.four_tau2 : __builtin_huge_valf();
    c.k12t = (float)k.k12_tube;
    const double two_tau = 2.0 * sqrt(k.tau2);
    c.far_dist = (float)((two_tau > 1.5 ? two_tau : 1.5) * 1.001 + 1e-3);
    return c;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// g(x) = 1 - e^{-x}(1 + x) = sum_{n>=2} (-1)^n (n-1) x^n / n!, to n = 9
// (relative truncation error < 3e-8 for x < 0.5).
__device__ __forceinline__ float g_series(float x)
{
    float p = -1.0f / 45360.0f;
    p = fmaf(p, x, 1.0f / 5760.0f);
    p = fmaf(p, x, -1.0f / 840.0f);
    p = fmaf(p, x, 1.0f / 144.0f);
    p = fmaf(p, x, -1.0f / 30.0f);
    p = fmaf(p, x, 1.0f / 8.0f);
    p = fmaf(p, x, -1.0f / 3.0f);
    p = fmaf(p, x, 0.5f);
    return p * x * x;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kChunk = 16;

// Far pair: no tube, exp-form g.  Accumulates into t1, t2.
__device__ __forceinline__ void pair_far(const float3& xi, const float3& ni, const float4& y, const float4& m,
                                         const F32Consts& k, float& t1, float& t2)
{
    const float rx = xi.x - y.x, ry = xi.y - y.y, rz = xi.z - y.z;
    const float rr = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float sx = fmaf(rx, ni.x, fmaf(ry, ni.y, rz * ni.z));
    const float sy = fmaf(rx, m.x, fmaf(ry, m.y, rz * m.z));
    const float cc = fmaf(ni.x, m.x, fmaf(ni.y, m.y, ni.z * m.z));
    const float inv = ptx::rsqrt_approx(rr);
    const float rho = rr * inv;
    const float x = k.kappa * rho;
    const float E = ptx::ex2_approx(rho * k.kl2e);
    const float Ex = E * x;
    const float f = 1.0f - E;
    const float g = f - Ex;
    const float hh = fmaf(3.0f, g, -Ex * x);
    const float inv2 = inv * inv;
    const float inv3 = inv2 * inv;
    const float u1 = fmaf(k.th1, g, k.omth1);
    const float u2 = fmaf(k.th2, g, k.omth2);
    const float A1 = inv3 * y.w;
    t1 = fmaf(sy * u1, A1, t1);
    t1 = fmaf(-f, inv * m.w, t1);
    const float w21 = fmaf(g, cc, -(hh * sx) * (sy * inv2));
    t2 = fmaf(w21, A1, t2);
    t2 = fmaf(sx * u2, inv3 * m.w, t2);
}

template <int TPT>
__global__ void __launch_bounds__(kF32Threads)
    pair_f32_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm,
                    const float4* __restrict__ src, int64_t N, PairSchedule s, F32Consts k,
                    double* __restrict__ part, unsigned* __restrict__ err, const int* __restrict__ skip,
                    const float4* __restrict__ tbound, const float4* __restrict__ sbound)
{
    constexpr int TTILE = kF32Threads * TPT;
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) float4 sbuf[kF32Stages][2 * kF32STile];
    __shared__ __align__(8) uint64_t bars[kF32Stages];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * s.per_cta;
    const int64_t s1 = (s0 + s.per_cta < s.total) ? s0 + s.per_cta : s.total;
    if (s0 >= s1) return;

    if (tid == 0) {
        for (int q = 0; q < kF32Stages; ++q) ptx::mbar_init(&bars[q], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int64_t u) {
        const int64_t st = u % s.n_stiles;
        const int64_t j0 = st * kF32STile;
        const int64_t cnt = (N - j0 < kF32STile) ? N - j0 : kF32STile;
        const int stage = (int)((u - s0) % kF32Stages);
        const uint32_t bytes = (uint32_t)(cnt * 2 * sizeof(float4));
        ptx::mbar_arrive_expect_tx(&bars[stage], bytes);
        ptx::bulk_g2s(&sbuf[stage][0], src + 2 * j0, bytes, &bars[stage]);
    };
    if (tid == 0)
        for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);

    const int64_t t_first = s0 / s.n_stiles;
    int64_t t = t_first;
    float3 xi[TPT], ni[TPT];
    double D1[TPT], D2[TPT];
    float4 tb = make_float4(0.0f, 0.0f, 0.0f, __builtin_huge_valf());

    auto load_targets = [&](int64_t tile) {
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = tile * TTILE + q * kF32Threads + tid;
            if (i < N) {
                const float4 a = tpos[i];
                const float4 b = tnrm[i];
                xi[q] = make_float3(a.x, a.y, a.z);
                ni[q] = make_float3(b.x, b.y, b.z);
            } else {  // padding target far from every node; its sums are discarded
                xi[q] = make_float3(1.0e6f, 1.0e6f, 1.0e6f);
                ni[q] = make_float3(0.0f, 0.0f, 1.0f);
            }
            D1[q] = 0.0;
            D2[q] = 0.0;
        }
        if (tbound != nullptr) tb = tbound[tile];
    };
    load_targets(t);

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kF32Stages);
        const uint32_t parity = (uint32_t)(((u - s0) / kF32Stages) & 1);
        if (!ptx::mbar_wait_bounded(&bars[stage], parity, kWaitLimitNs)) {
            abort_flag = 1;
            atomicOr(err, kDevErrTimeout);
        }
        __syncthreads();
        if (abort_flag) return;

        const int64_t st = u % s.n_stiles;
        const int64_t j0 = st * kF32STile;
        const int cnt = (int)((N - j0 < kF32STile) ? N - j0 : kF32STile);
        const float4* sb = &sbuf[stage][0];

        bool far = false;
        if (tbound != nullptr && k.rule0) {
            const float4 b = sbound[st];
            const float dx = tb.x - b.x, dy = tb.y - b.y, dz = tb.z - b.z;
            const float lim = k.far_dist + tb.w + b.w;
            far = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim;
        }

        float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;

        if (far) {
            for (int c0 = 0; c0 < cnt; c0 += kChunk) {
                const int c1 = (c0 + kChunk < cnt) ? c0 + kChunk : cnt;
                float t1[TPT], t2[TPT];
#pragma unroll
                for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = 0.0f;
#pragma unroll 4
                for (int j = c0; j < c1; ++j) {
                    const float4 y = sb[2 * j];
                    const float4 m = sb[2 * j + 1];
#pragma unroll
                    for (int q = 0; q < TPT; ++q) pair_far(xi[q], ni[q], y, m, k, t1[q], t2[q]);
                }
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    kahan_add(S1[q], C1[q], t1[q]);
                    kahan_add(S2[q], C2[q], t2[q]);
                }
            }
        } else {
            for (int c0 = 0; c0 < cnt; c0 += kChunk) {
                const int c1 = (c0 + kChunk < cnt) ? c0 + kChunk : cnt;
                float t1[TPT], t2[TPT];
#pragma unroll
                for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = 0.0f;
                for (int j = c0; j < c1; ++j) {
                    const float4 y = sb[2 * j];
                    const float4 m = sb[2 * j + 1];
                    float rr[TPT], sx[TPT], sy[TPT], cc[TPT], inv[TPT], x[TPT], E[TPT];
                    bool tube[TPT];
                    bool need = false;
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        const float rx = xi[q].x - y.x, ry = xi[q].y - y.y, rz = xi[q].z - y.z;
                        rr[q] = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                        sx[q] = fmaf(rx, ni[q].x, fmaf(ry, ni[q].y, rz * ni[q].z));
                        sy[q] = fmaf(rx, m.x, fmaf(ry, m.y, rz * m.z));
                        cc[q] = fmaf(ni[q].x, m.x, fmaf(ni[q].y, m.y, ni[q].z * m.z));
                        const float rp2 = fmaf(-sx[q], sx[q], rr[q]);
                        tube[q] = (rp2 < k.tau2) & (rr[q] < k.four_tau2);
                        const float rrs = fmaxf(rr[q], 1.0e-30f);
                        inv[q] = ptx::rsqrt_approx(rrs);
                        const float rho = rrs * inv[q];
                        x[q] = k.kappa * rho;
                        E[q] = ptx::ex2_approx(rho * k.kl2e);
                        need |= (x[q] < 0.5f);
                    }
                    const bool series = __any_sync(0xffffffffu, need);
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        const float Ex = E[q] * x[q];
                        float f = 1.0f - E[q];
                        float g = f - Ex;
                        if (series && x[q] < 0.5f) {
                            g = g_series(x[q]);
                            f = g + Ex;
                        }
                        const float hh = fmaf(3.0f, g, -Ex * x[q]);
                        const float inv2 = inv[q] * inv[q];
                        const float inv3 = inv2 * inv[q];
                        const float u1 = fmaf(k.th1, g, k.omth1);
                        const float u2 = fmaf(k.th2, g, k.omth2);
                        const float i3 = tube[q] ? 0.0f : inv3;
                        const float Q = tube[q] ? k.k12t : f * inv[q];
                        const float A1 = i3 * y.w;
                        t1[q] = fmaf(sy[q] * u1, A1, t1[q]);
                        t1[q] = fmaf(-Q, m.w, t1[q]);
                        const float w21 = fmaf(g, cc[q], -(hh * sx[q]) * (sy[q] * inv2));
                        t2[q] = fmaf(w21, A1, t2[q]);
                        t2[q] = fmaf(sx[q] * u2, i3 * m.w, t2[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    kahan_add(S1[q], C1[q], t1[q]);
                    kahan_add(S2[q], C2[q], t2[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            D1[q] += (double)S1[q] - (double)C1[q];
            D2[q] += (double)S2[q] - (double)C2[q];
        }
        __syncthreads();  // every thread is done with this stage
        if (tid == 0 && u + kF32Stages < s1) {
            ptx::fence_proxy_async_smem();
            issue(u + kF32Stages);
        }

        if (st == s.n_stiles - 1 || u + 1 == s1) {
            const int seg = (int)(t - t_first);
            double* dst = part + ((int64_t)blockIdx.x * s.max_segs + seg) * 2 * TTILE;
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                dst[q * kF32Threads + tid] = D1[q];
                dst[TTILE + q * kF32Threads + tid] = D2[q];
            }
            if (st == s.n_stiles - 1 && u + 1 < s1) {
                ++t;
                load_targets(t);
            }
        }
    }
}

// Bounding sphere (centre, radius) of each tile of `tile` consecutive nodes,
// in the FP32 centroid frame, radius padded by 1e-3 A for rounding.
__global__ void tile_bounds_kernel(const float4* __restrict__ pos, int64_t N, int tile, float4* __restrict__ out)
{
    __shared__ float red[4][256];
    const int64_t j0 = (int64_t)blockIdx.x * tile;
    const int64_t j1 = (j0 + tile < N) ? j0 + tile : N;
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        sx += pos[j].x;
        sy += pos[j].y;
        sz += pos[j].z;
    }
    red[0][threadIdx.x] = sx;
    red[1][threadIdx.x] = sy;
    red[2][threadIdx.x] = sz;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + o];
        __syncthreads();
    }
    const float inv = 1.0f / (float)(j1 - j0);
    const float cx = red[0][0] * inv, cy = red[1][0] * inv, cz = red[2][0] * inv;
    __syncthreads();
    float r2 = 0.0f;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const float dx = pos[j].x - cx, dy = pos[j].y - cy, dz = pos[j].z - cz;
        r2 = fmaxf(r2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
    red[3][threadIdx.x] = r2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[3][threadIdx.x] = fmaxf(red[3][threadIdx.x], red[3][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = make_float4(cx, cy, cz, sqrtf(red[3][0]) * 1.0001f + 1e-3f);
}

// Source payload: node j -> float4 (y* - centroid, w psi), float4 (n, w psin).
__global__ void pack_f32_kernel(const float4* __restrict__ pos, const float4* __restrict__ nrm,
                                const double* __restrict__ w, VecRef in, int64_t N,
                                float4* __restrict__ src, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    const float4 a = pos[j];
    const float4 b = nrm[j];
    const double wj = w[j];
    src[2 * j] = make_float4(a.x, a.y, a.z, (float)(wj * p[j]));
    src[2 * j + 1] = make_float4(b.x, b.y, b.z, (float)(wj * p[N + j]));
}

// y = Lambda p + (1/(4 pi)) sum of the partials of every CTA that touched the tile.
__global__ void fixup_kernel(const double* __restrict__ part, PairSchedule s, int ttile, int64_t N,
                             double lambda1, double lambda2, VecRef in, OutRef out,
                             const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    double* y = out.base + (out.kidx ? (int64_t)(*out.kidx + out.koff) * out.stride : 0);
    const int64_t t = i / ttile;
    const int64_t l = i - t * ttile;
    const int64_t c0 = (t * s.n_stiles) / s.per_cta;
    const int64_t c1 = ((t + 1) * s.n_stiles - 1) / s.per_cta;
    double a1 = 0.0, a2 = 0.0;
    for (int64_t c = c0; c <= c1; ++c) {
        const int64_t seg = t - (c * s.per_cta) / s.n_stiles;
        const double* src = part + (c * s.max_segs + seg) * 2 * ttile;
        a1 += src[l];
        a2 += src[ttile + l];
    }
    y[i] = lambda1 * p[i] + kInv4Pi * a1;
    y[N + i] = lambda2 * p[N + i] + kInv4Pi * a2;
}

static int occupancy_per_sm(int tpt)
{
    int occ = 0;
    if (tpt == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f32_kernel<4>, kF32Threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f32_kernel<2>, kF32Threads, 0);
    return occ < 1 ? 1 : occ;
}

int f32_max_bps(int tpt) { return occupancy_per_sm(tpt); }

int f32_ttile(const ibim_ctx* c) { return kF32Threads * (c->f32_tpt == 4 ? 4 : 2); }

int f32_grid_cap(ibim_ctx* c)
{
    const int occ = occupancy_per_sm(c->f32_tpt);
    const int bps = (c->f32_bps > 0 && c->f32_bps < occ) ? c->f32_bps : occ;
    return bps * c->num_sms;
}

PairSchedule f32_schedule(ibim_ctx* c)
{
    return make_schedule(c->N, f32_ttile(c), c->N, kF32STile, f32_grid_cap(c));
}

ibim_status f32_tile_bounds(ibim_ctx* c)
{
    const int64_t N = c->N;
    const int64_t n2 = (N + 2 * kF32Threads - 1) / (2 * kF32Threads);
    const int64_t n4 = (N + 4 * kF32Threads - 1) / (4 * kF32Threads);
    const int64_t ns = (N + kF32STile - 1) / kF32STile;
    IBIM_CUDA(cudaMalloc((void**)&c->d_tb32_2, sizeof(float4) * n2));
    IBIM_CUDA(cudaMalloc((void**)&c->d_tb32_4, sizeof(float4) * n4));
    IBIM_CUDA(cudaMalloc((void**)&c->d_sb32, sizeof(float4) * ns));
    tile_bounds_kernel<<<(unsigned)n2, 256, 0, c->stream>>>(c->d_pos32, N, 2 * kF32Threads, c->d_tb32_2);
    tile_bounds_kernel<<<(unsigned)n4, 256, 0, c->stream>>>(c->d_pos32, N, 4 * kF32Threads, c->d_tb32_4);
    tile_bounds_kernel<<<(unsigned)ns, 256, 0, c->stream>>>(c->d_pos32, N, kF32STile, c->d_sb32);
    count_launch(c, 3);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f32_pack(ibim_ctx* c, VecRef in, const int* d_skip)
{
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, &c->d_src, &c->src_bytes, (size_t)N * 2 * sizeof(float4)));
    const double* w = c->d_geo64 + 6 * N;
    const int bs = 256;
    pack_f32_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_pos32, c->d_nrm32, w, in, N, (float4*)c->d_src, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f32_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip)
{
    const int ttile = f32_ttile(c);
    const size_t need = (size_t)s.grid * s.max_segs * 2 * ttile * sizeof(double);
    IBIM_TRY(ensure(c, (void**)&c->d_part, &c->part_bytes, need));
    const F32Consts kk = f32_consts(k);
    if (ttile == 4 * kF32Threads)
        pair_f32_kernel<4><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, (const float4*)c->d_src,
                                                                   c->N, s, kk, c->d_part, c->d_err, d_skip,
                                                                   c->d_tb32_4, c->d_sb32);
    else
        pair_f32_kernel<2><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, (const float4*)c->d_src,
                                                                   c->N, s, kk, c->d_part, c->d_err, d_skip,
                                                                   c->d_tb32_2, c->d_sb32);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status fixup_launch(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, int ttile, VecRef in,
                         OutRef out, const int* d_skip)
{
    const int bs = 256;
    fixup_kernel<<<(unsigned)((c->N + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_part, s, ttile, c->N, k.lambda1, k.lambda2, in, out, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f32_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                      const int* d_skip)
{
    return fixup_launch(c, k, s, f32_ttile(c), in, out, d_skip);
}

// Launchers on caller-supplied buffers (used by the allocation-free entry point).
int f32_occupancy_per_sm() { return occupancy_per_sm(kF32Tpt); }

cudaError_t launch_pair_f32_raw(const float4* tpos, const float4* tnrm, const float4* src, int64_t N,
                                const PairSchedule& s, const PairConsts& k, double* part, unsigned* err,
                                cudaStream_t stream)
{
    pair_f32_kernel<kF32Tpt><<<s.grid, kF32Threads, 0, stream>>>(tpos, tnrm, src, N, s, f32_consts(k), part, err,
                                                                  nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_fixup_raw(const double* part, const PairSchedule& s, int64_t N, const PairConsts& k,
                             const double* d_in, double* d_out, cudaStream_t stream)
{
    const int bs = 256;
    fixup_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, stream>>>(part, s, kF32TTile, N, k.lambda1, k.lambda2,
                                                                  VecRef{d_in, nullptr, 0, 0},
                                                                  OutRef{d_out, nullptr, 0, 0}, nullptr);
    return cudaGetLastError();
}

}  // namespace ibim
