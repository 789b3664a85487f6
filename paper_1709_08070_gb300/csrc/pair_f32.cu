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
// tile) steps.  Source tiles (kF32STile nodes, 32 B each, plus the frames of
// their 32-node chunks) are brought into shared memory by bulk async copies
// with an mbarrier per stage (double buffered).  Each thread owns TPT
// targets; the 32 lanes of a warp hold one aligned 32-node block per target
// slot.
//
// Chunk frames: every aligned block of 32 consecutive (Morton-ordered) nodes
// has a centre C stored as two floats (hi + lo) and a radius; node
// coordinates are stored relative to their own block's centre.  For each
// (warp, source chunk) the centre offset D = C_target_block - C_source_chunk
// is formed from the hi and lo parts and added to the warp's targets once, so
// the per-pair difference r = (x - C_t + D) - (y - C_s) stays accurate to a
// few 1e-7 of |r| however far the molecule extends from the origin.
//
// Near/far split per (warp, chunk): when the two blocks' bounding spheres are
// at least `far_dist` apart (>= 2 tau and >= 1.5 A), no pair can lie in the
// regularisation tube (tube rule 0) and the cancellation in g is harmless, so
// the chunk runs a branch-free loop with no tube masks.  Otherwise every pair
// gets the tube test and, when any lane of the warp has x < 0.5, g from its
// Taylor series (from the exponential series).  The decision is warp-uniform.
//
// Accumulation: per target the two sums run in FP32 over one 32-source chunk
// (fused into the FMAs), each chunk sum is Kahan-added into a compensated FP32
// pair (s, c), and at the end of each source tile the compensated value s - c
// is added to FP64 accumulators.  Every CTA writes one FP64 partial per target
// tile it touched; the fixup kernel adds the partials, scales by 1/(4 pi) and
// adds the diagonal Lambda p.
#include "pair_f32_core.cuh"

namespace ibim {

template <int TPT, int MINB>
__global__ void __launch_bounds__(kF32Threads, MINB)
    pair_f32_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm,
                    const float4* __restrict__ src, const float4* __restrict__ frames, int64_t N, PairSchedule s,
                    F32Consts k, double* __restrict__ part, unsigned* __restrict__ err, const int* __restrict__ skip,
                    Geo64 g64)
{
    constexpr int TTILE = kF32Threads * TPT;
    constexpr int CPT = kF32STile / kChunk;  // chunks per source tile
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) float4 sbuf[kF32Stages][2 * kF32STile];
    __shared__ __align__(128) float4 sfrm[kF32Stages][2 * CPT];
    __shared__ __align__(8) uint64_t bars[kF32Stages];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t s0 = (int64_t)blockIdx.x * s.per_cta;
    const int64_t s1 = (s0 + s.per_cta < s.total) ? s0 + s.per_cta : s.total;
    if (s0 >= s1) return;
    const bool have_frames = frames != nullptr;

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
        const int64_t nch = (cnt + kChunk - 1) / kChunk;
        const uint32_t fbytes = have_frames ? (uint32_t)(nch * 2 * sizeof(float4)) : 0u;
        ptx::mbar_arrive_expect_tx(&bars[stage], bytes + fbytes);
        ptx::bulk_g2s(&sbuf[stage][0], src + 2 * j0, bytes, &bars[stage]);
        if (have_frames) ptx::bulk_g2s(&sfrm[stage][0], frames + 2 * (j0 / kChunk), fbytes, &bars[stage]);
    };
    if (tid == 0)
        for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);

    const int64_t t_first = s0 / s.n_stiles;
    int64_t t = t_first;
    float3 xi[TPT], ni[TPT];
    float4 bh[TPT];  // target block centre (hi) and radius
    float3 bl[TPT];  // target block centre (lo)
    int64_t gi[TPT];  // target node indices
    double D1[TPT], D2[TPT];

    auto load_targets = [&](int64_t tile) {
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t blk0 = tile * TTILE + q * kF32Threads + warp * 32;  // first node of the warp's block
            const int64_t i = blk0 + (tid & 31);
            gi[q] = (i < N) ? i : 0;
            if (i < N) {
                const float4 a = tpos[i];
                const float4 b = tnrm[i];
                xi[q] = make_float3(a.x, a.y, a.z);
                ni[q] = make_float3(b.x, b.y, b.z);
            } else {  // padding target far from every node; its sums are discarded
                xi[q] = make_float3(1.0e6f, 1.0e6f, 1.0e6f);
                ni[q] = make_float3(0.0f, 0.0f, 1.0f);
            }
            if (have_frames && blk0 < N) {
                bh[q] = frames[2 * (blk0 / kChunk)];
                const float4 l = frames[2 * (blk0 / kChunk) + 1];
                bl[q] = make_float3(l.x, l.y, l.z);
            } else {
                bh[q] = make_float4(0.0f, 0.0f, 0.0f, __builtin_huge_valf());
                bl[q] = make_float3(0.0f, 0.0f, 0.0f);
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

        float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;

        tile_sums<TPT>(xi, ni, bh, bl, have_frames, sb, &sfrm[stage][0], cnt, k, S1, C1, S2, C2, g64, gi, j0);
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

// Frames of the aligned 32-node chunks (FP64 centre split into hi + lo
// floats, radius padded for rounding) and node coordinates relative to their
// chunk centre.  One thread per chunk.
__global__ void chunk_frames_kernel(const double* __restrict__ geo, int64_t N, float4* __restrict__ rel,
                                    float4* __restrict__ frames)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j0 = c * kChunk;
    if (j0 >= N) return;
    const int64_t j1 = (j0 + kChunk < N) ? j0 + kChunk : N;
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        cx += geo[j];
        cy += geo[N + j];
        cz += geo[2 * N + j];
    }
    const double inv = 1.0 / (double)(j1 - j0);
    cx *= inv;
    cy *= inv;
    cz *= inv;
    double r2 = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double dx = geo[j] - cx, dy = geo[N + j] - cy, dz = geo[2 * N + j] - cz;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
        rel[j] = make_float4((float)dx, (float)dy, (float)dz, (float)geo[6 * N + j]);
    }
    const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
    frames[2 * c] = make_float4(hx, hy, hz, (float)(sqrt(r2) * 1.0001 + 1e-4));
    frames[2 * c + 1] = make_float4((float)(cx - (double)hx), (float)(cy - (double)hy), (float)(cz - (double)hz), 0.0f);
}

// Source payload: node j -> float4 (position in its chunk frame, w psi), float4 (n, w psin).
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

// Compiled variants: targets per thread x minimum CTAs per SM (register budget).
struct F32Variant {
    int tpt, minb;
    const void* fn;
};
static const F32Variant kVariants[] = {
    {2, 1, (const void*)pair_f32_kernel<2, 1>}, {2, 6, (const void*)pair_f32_kernel<2, 6>},
    {2, 8, (const void*)pair_f32_kernel<2, 8>}, {4, 1, (const void*)pair_f32_kernel<4, 1>},
    {4, 4, (const void*)pair_f32_kernel<4, 4>},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

int f32_variant_count() { return kNumVariants; }
void f32_variant_info(int v, int* tpt, int* minb)
{
    *tpt = kVariants[v].tpt;
    *minb = kVariants[v].minb;
}

static int occupancy_of(int v)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kVariants[v].fn, kF32Threads, 0);
    return occ < 1 ? 1 : occ;
}

int f32_max_bps(int v) { return occupancy_of(v); }

int f32_ttile(const ibim_ctx* c) { return kF32Threads * kVariants[c->f32_variant].tpt; }

int f32_grid_cap(ibim_ctx* c)
{
    const int occ = occupancy_of(c->f32_variant);
    const int bps = (c->f32_bps > 0 && c->f32_bps < occ) ? c->f32_bps : occ;
    return bps * c->num_sms;
}

PairSchedule f32_schedule(ibim_ctx* c)
{
    return make_schedule(c->N, f32_ttile(c), c->N, kF32STile, f32_grid_cap(c));
}

ibim_status f32_chunk_frames(ibim_ctx* c)
{
    const int64_t N = c->N;
    const int64_t nch = (N + kChunk - 1) / kChunk;
    IBIM_CUDA(cudaMalloc((void**)&c->d_frames, sizeof(float4) * 2 * nch));
    chunk_frames_kernel<<<(unsigned)((nch + 127) / 128), 128, 0, c->stream>>>(c->d_geo64, N, c->d_pos32, c->d_frames);
    count_launch(c);
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
    const float4* srcp = (const float4*)c->d_src;
    const Geo64 g64{c->d_geo64, c->d_geo64 + 3 * c->N, 1, c->N};
    switch (c->f32_variant) {
    case 1:
        pair_f32_kernel<2, 6><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, srcp, c->d_frames, c->N,
                                                                      s, kk, c->d_part, c->d_err, d_skip, g64);
        break;
    case 2:
        pair_f32_kernel<2, 8><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, srcp, c->d_frames, c->N,
                                                                      s, kk, c->d_part, c->d_err, d_skip, g64);
        break;
    case 3:
        pair_f32_kernel<4, 1><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, srcp, c->d_frames, c->N,
                                                                      s, kk, c->d_part, c->d_err, d_skip, g64);
        break;
    case 4:
        pair_f32_kernel<4, 4><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, srcp, c->d_frames, c->N,
                                                                      s, kk, c->d_part, c->d_err, d_skip, g64);
        break;
    default:
        pair_f32_kernel<2, 1><<<s.grid, kF32Threads, 0, c->stream>>>(c->d_pos32, c->d_nrm32, srcp, c->d_frames, c->N,
                                                                      s, kk, c->d_part, c->d_err, d_skip, g64);
        break;
    }
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
int f32_occupancy_per_sm() { return occupancy_of(0); }

cudaError_t launch_pair_f32_raw(const float4* tpos, const float4* tnrm, const float4* src, int64_t N,
                                const PairSchedule& s, const PairConsts& k, double* part, unsigned* err,
                                cudaStream_t stream, const double* xs_aos, const double* nrm_aos)
{
    const Geo64 g64{xs_aos, nrm_aos, 3, 1};
    pair_f32_kernel<kF32Tpt, 1><<<s.grid, kF32Threads, 0, stream>>>(tpos, tnrm, src, nullptr, N, s, f32_consts(k),
                                                                     part, err, nullptr, g64);
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
