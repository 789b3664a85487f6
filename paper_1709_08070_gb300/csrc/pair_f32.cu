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
// The differences 1 - A and 3 - B cancel for small x = kappa rho; they are
// formed as g = 1 - A and 3 - B = 3 g - E x^2, with g taken from its Taylor
// series in x (from the exponential series) when any lane of the warp has
// x < 0.5, and 1 - E = g + E x.
//
// Schedule: persistent CTAs walk a stream-K range of (target tile, source
// tile) steps.  Source tiles (kF32STile nodes, 32 B each) are brought into
// shared memory by bulk async copies with an mbarrier per stage (double
// buffered).  Each thread owns kF32Tpt targets; per target the two sums are
// Kahan-compensated in FP32 within a source tile and the tile result is added
// to FP64 accumulators.  Every CTA writes one FP64 partial per target tile it
// touched; the fixup kernel adds the partials, scales by 1/(4 pi) and adds
// the diagonal Lambda p.
#include "ibim_internal.cuh"
#include "ptx.cuh"

namespace ibim {

struct F32Consts {
    float th1, th2, omth1, omth2;
    float kappa, tau2, four_tau2, k12t;
};

static F32Consts f32_consts(const PairConsts& k)
{
    F32Consts c;
    c.th1 = (float)k.th1;
    c.th2 = (float)k.th2;
    c.omth1 = (float)(1.0 - k.th1);
    c.omth2 = (float)(1.0 - k.th2);
    c.kappa = (float)k.kappa;
    c.tau2 = (float)k.tau2;
    c.four_tau2 = (k.four_tau2 > 3.0e38) ? __builtin_huge_valf() : (float)k.four_tau2;
    c.k12t = (float)k.k12_tube;
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

constexpr float kLog2e = 1.4426950408889634f;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__global__ void __launch_bounds__(kF32Threads)
    pair_f32_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm,
                    const float4* __restrict__ src, int64_t N, PairSchedule s, F32Consts k,
                    double* __restrict__ part, unsigned* __restrict__ err, const int* __restrict__ skip)
{
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
    float3 xi[kF32Tpt], ni[kF32Tpt];
    double D1[kF32Tpt], D2[kF32Tpt];

    auto load_targets = [&](int64_t tile) {
#pragma unroll
        for (int q = 0; q < kF32Tpt; ++q) {
            const int64_t i = tile * kF32TTile + q * kF32Threads + tid;
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

        float S1[kF32Tpt], C1[kF32Tpt], S2[kF32Tpt], C2[kF32Tpt];
#pragma unroll
        for (int q = 0; q < kF32Tpt; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;

#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            const float4 y = sb[2 * j];
            const float4 m = sb[2 * j + 1];
            float rr[kF32Tpt], sx[kF32Tpt], sy[kF32Tpt], cc[kF32Tpt], inv[kF32Tpt], x[kF32Tpt],
                E[kF32Tpt];
            bool tube[kF32Tpt];
            bool need = false;
#pragma unroll
            for (int q = 0; q < kF32Tpt; ++q) {
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
                E[q] = ptx::ex2_approx(x[q] * -kLog2e);
                need |= (x[q] < 0.5f);
            }
            const bool series = __any_sync(0xffffffffu, need);
#pragma unroll
            for (int q = 0; q < kF32Tpt; ++q) {
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
                const float v1 = fmaf(i3, sy[q] * u1 * y.w, -Q * m.w);
                const float w21 = fmaf(g, cc[q], -hh * sx[q] * sy[q] * inv2);
                const float v2 = i3 * fmaf(w21, y.w, sx[q] * u2 * m.w);
                kahan_add(S1[q], C1[q], v1);
                kahan_add(S2[q], C2[q], v2);
            }
        }
#pragma unroll
        for (int q = 0; q < kF32Tpt; ++q) {
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
            double* dst = part + ((int64_t)blockIdx.x * s.max_segs + seg) * 2 * kF32TTile;
#pragma unroll
            for (int q = 0; q < kF32Tpt; ++q) {
                dst[q * kF32Threads + tid] = D1[q];
                dst[kF32TTile + q * kF32Threads + tid] = D2[q];
            }
            if (st == s.n_stiles - 1 && u + 1 < s1) {
                ++t;
                load_targets(t);
            }
        }
    }
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

int f32_grid_cap(ibim_ctx* c)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f32_kernel, kF32Threads, 0);
    if (occ < 1) occ = 1;
    return occ * c->num_sms;
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
    const size_t need = (size_t)s.grid * s.max_segs * 2 * kF32TTile * sizeof(double);
    IBIM_TRY(ensure(c, (void**)&c->d_part, &c->part_bytes, need));
    pair_f32_kernel<<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32,
                                                            (const float4*)c->d_src, c->N, s,
                                                            f32_consts(k), c->d_part, c->d_err,
                                                            d_skip);
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
    return fixup_launch(c, k, s, kF32TTile, in, out, d_skip);
}

// Launchers on caller-supplied buffers (used by the allocation-free entry point).
int f32_occupancy_per_sm()
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f32_kernel, kF32Threads, 0);
    return occ < 1 ? 1 : occ;
}

cudaError_t launch_pair_f32_raw(const float4* tpos, const float4* tnrm, const float4* src, int64_t N,
                                const PairSchedule& s, const PairConsts& k, double* part, unsigned* err,
                                cudaStream_t stream)
{
    pair_f32_kernel<<<s.grid, kF32Threads, 0, stream>>>(tpos, tnrm, src, N, s, f32_consts(k), part, err, nullptr);
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
