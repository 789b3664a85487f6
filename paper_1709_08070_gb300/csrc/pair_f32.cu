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
// through kF32Stages stages with a full and an empty mbarrier each; warps
// consume and release stages independently (no CTA-wide barrier in the step
// loop) and thread 0 refills a stage once every warp has released it.  Each
// thread owns TPT targets; the 32 lanes of a warp hold one aligned 32-node
// block per target slot.
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
// the chunk runs a branch-free loop with no tube masks on packed float2
// operands, one lane per source of a payload pair (the FP32 pipe then does
// two interactions per issued instruction).  Otherwise the chunk runs the
// same packed formula with, per lane, the tube test (selects on rho^-3 and the
// 1/rho factor) and, where x < 0.5, g from its Taylor series (pair_near2).
// The decision is warp-uniform.
//
// Accumulation: per target the two sums run in FP32 over one 32-source chunk
// (fused into the FMAs, even and odd sources apart), each chunk sum is
// Kahan-added into a compensated FP32 pair (s, c), and at the end of each
// source tile the compensated value s - c is added to FP64 accumulators.
// Every CTA writes one FP64 partial per target tile it touched; the fixup
// kernel adds the partials, scales by 1/(4 pi) and adds the diagonal Lambda p.
#include "pair_f32_core.cuh"

namespace ibim {

template <int TPT, int MINB, int THREADS>
__global__ void __launch_bounds__(THREADS, MINB)
    pair_f32_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm,
                    const float4* __restrict__ src, const float4* __restrict__ frames, int64_t N, PairSchedule s,
                    F32Consts k, double* __restrict__ part, unsigned* __restrict__ err, const int* __restrict__ skip,
                    Geo64 g64)
{
    constexpr int TTILE = THREADS * TPT;
    constexpr int NW = THREADS / 32;
    static_assert(TTILE <= kF32MaxTTile, "target tile");
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(16) float4 tfrm[NW][2 * TPT];
    __shared__ __align__(8) StagePipe pipe;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t s0 = (int64_t)blockIdx.x * s.per_cta;
    const int64_t s1 = (s0 + s.per_cta < s.total) ? s0 + s.per_cta : s.total;
    if (s0 >= s1) return;
    const bool have_frames = frames != nullptr;

    if (tid == 0) pipe_init(pipe, NW);
    __syncthreads();

    auto issue = [&](int64_t u) {
        const int64_t st = ((u % s.n_stiles) * s.sperm) % s.n_stiles;
        const int stage = (int)((u - s0) % kF32Stages);
        pipe_issue(pipe, stg[stage], stage, src + st * (kF32STile / 2) * kPairF4,
                   have_frames ? frames + st * 2 * kChunksPerTile : nullptr);
    };
    if (tid == 0)
        for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);

    const int64_t t_first = s0 / s.n_stiles;
    int64_t t = t_first;
    Targets<TPT> T;
    int64_t gi0 = 0;  // node index of the thread's slot-0 target (slot q adds q * THREADS)
    bool idle = false;  // every block of the warp lies past N
    double D1[TPT], D2[TPT];

    // Targets and target-block frames of tile `tile` (arrays padded, so every
    // index below is in range; placeholder targets give discarded sums).
    auto load_targets = [&](int64_t tile) {
        gi0 = tile * TTILE + tid;
        idle = tile * TTILE + warp * 32 >= N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;
            const float4 a = tpos[i];
            const float4 b = tnrm[i];
            T.x[q] = make_float3(a.x, a.y, a.z);
            T.nx[q] = f2(b.x);
            T.ny[q] = f2(b.y);
            T.nz[q] = f2(b.z);
            D1[q] = 0.0;
            D2[q] = 0.0;
        }
        __syncwarp();
        if (have_frames && lane < 2 * TPT) {
            const int64_t blk0 = tile * TTILE + (int64_t)(lane >> 1) * THREADS + warp * 32;
            tfrm[warp][lane] = frames[2 * (blk0 / kChunk) + (lane & 1)];
        }
        __syncwarp();
    };
    load_targets(t);

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kF32Stages);
        const uint32_t parity = (uint32_t)(((u - s0) / kF32Stages) & 1);
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
            if (lane == 0) atomicOr(err, kDevErrTimeout);
            return;
        }
        const int64_t sp = u % s.n_stiles;               // position in the row
        const int64_t st = (sp * s.sperm) % s.n_stiles;  // source tile visited there
        float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;
        if (!idle)
            tile_sums<TPT>(T, &tfrm[warp][0], have_frames, stg[stage].buf, stg[stage].frm, k, S1, C1, S2, C2, g64,
                           gi0, THREADS, st * kF32STile, N);
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            D1[q] += (double)S1[q] - (double)C1[q];
            D2[q] += (double)S2[q] - (double)C2[q];
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
        // thread 0 refills the stage of step u - 1 with step u - 1 + kF32Stages
        if (warp == 0) {
            bool ok = true;
            if (lane == 0 && u > s0 && u - 1 + kF32Stages < s1) {
                const int64_t v = u - 1 - s0;
                ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(v % kF32Stages)], (uint32_t)((v / kF32Stages) & 1),
                                            kWaitLimitNs);
                if (ok) {
                    ptx::fence_proxy_async_smem();
                    issue(u - 1 + kF32Stages);
                } else {
                    atomicOr(err, kDevErrTimeout);
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;
        }

        if (sp == s.n_stiles - 1 || u + 1 == s1) {
            const int seg = (int)(t - t_first);
            double* dst = part + ((int64_t)blockIdx.x * s.max_segs + seg) * 2 * TTILE;
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                dst[q * THREADS + tid] = D1[q];
                dst[TTILE + q * THREADS + tid] = D2[q];
            }
            if (sp == s.n_stiles - 1 && u + 1 < s1) {
                ++t;
                load_targets(t);
            }
        }
    }
}

// Frames of the aligned 32-node chunks (FP64 centre split into hi + lo
// floats, radius padded for rounding) and node coordinates relative to their
// chunk centre; chunks and nodes past N (up to the padded count) get a zero
// frame and placeholder target positions.  One thread per chunk.
__global__ void chunk_frames_kernel(const double* __restrict__ geo, int64_t N, int64_t n_chunks,
                                    float4* __restrict__ rel, float4* __restrict__ frames)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const int64_t j0 = c * kChunk;
    const int64_t j1 = (j0 + kChunk < N) ? j0 + kChunk : (N > j0 ? N : j0);
    for (int64_t j = j1; j < j0 + kChunk; ++j) rel[j] = pad_target_pos();
    if (j1 == j0) {
        frames[2 * c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        frames[2 * c + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
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

// Source payload of the padded node range, one thread per node pair:
// positions in their chunk frame, a = w psi, b = w psin (placeholders past N).
__global__ void pack_f32_kernel(const float4* __restrict__ pos, const float4* __restrict__ nrm,
                                const double* __restrict__ w, VecRef in, int64_t N, int64_t n_pairs,
                                float4* __restrict__ src, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= n_pairs) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    float4 y[2], m[2];
    float a[2], b[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int64_t j = 2 * pr + e;
        if (j < N) {
            y[e] = pos[j];
            m[e] = nrm[j];
            const double wj = w[j];
            a[e] = (float)(wj * p[j]);
            b[e] = (float)(wj * p[N + j]);
        } else {
            y[e] = pad_source_pos();
            m[e] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            a[e] = b[e] = 0.0f;
        }
    }
    write_source_pair(src + kPairF4 * pr, y[0], y[1], m[0], m[1], a[0], a[1], b[0], b[1]);
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
struct PairArgs {
    const float4* tpos;
    const float4* tnrm;
    const float4* src;
    const float4* frames;
    int64_t N;
    PairSchedule s;
    F32Consts k;
    double* part;
    unsigned* err;
    const int* skip;
    Geo64 g64;
};

template <int TPT, int MINB, int THREADS>
static void launch_variant(const PairArgs& a, cudaStream_t stream)
{
    pair_f32_kernel<TPT, MINB, THREADS><<<a.s.grid, THREADS, 0, stream>>>(a.tpos, a.tnrm, a.src, a.frames, a.N, a.s,
                                                                          a.k, a.part, a.err, a.skip, a.g64);
}

struct F32Variant {
    int tpt, minb, threads;
    const void* fn;
    void (*launch)(const PairArgs&, cudaStream_t);
};
#define IBIM_F32_VARIANT(T, M, W) {T, M, W, (const void*)pair_f32_kernel<T, M, W>, launch_variant<T, M, W>}
static const F32Variant kVariants[] = {
    IBIM_F32_VARIANT(2, 1, 128), IBIM_F32_VARIANT(2, 3, 128), IBIM_F32_VARIANT(2, 4, 128),
    IBIM_F32_VARIANT(1, 6, 128), IBIM_F32_VARIANT(2, 2, 256), IBIM_F32_VARIANT(2, 1, 512),
    IBIM_F32_VARIANT(1, 1, 512),
};
#undef IBIM_F32_VARIANT
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// Variants kNumVariants.. are the symmetric kernel's (pair_sym.cu).
int f32_variant_count() { return kNumVariants + sym_variant_count(); }
static bool is_sym(int v) { return v >= kNumVariants; }
bool f32_variant_symmetric(int v) { return is_sym(v); }
int f32_deterministic_variant() { return 5; }  // (2 targets/thread, 1 CTA/SM, 512 threads)
static_assert(5 < kNumVariants, "deterministic variant");

void f32_variant_info(int v, int* tpt, int* minb, int* threads, int* symmetric)
{
    if (is_sym(v)) {
        sym_variant_info(v - kNumVariants, tpt, minb, threads, symmetric);
        return;
    }
    *tpt = kVariants[v].tpt;
    *minb = kVariants[v].minb;
    *threads = kVariants[v].threads;
    *symmetric = 0;
}

static int occupancy_of(int v)
{
    if (is_sym(v)) return sym_occupancy(v - kNumVariants);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kVariants[v].fn, kVariants[v].threads, 0);
    return occ < 1 ? 1 : occ;
}

int f32_max_bps(int v) { return occupancy_of(v); }

int f32_ttile(const ibim_ctx* c)
{
    int tpt, minb, threads, sym;
    f32_variant_info(c->f32_variant, &tpt, &minb, &threads, &sym);
    return threads * tpt;
}

int f32_grid_cap(ibim_ctx* c)
{
    const int occ = occupancy_of(c->f32_variant);
    const int bps = (c->f32_bps > 0 && c->f32_bps < occ) ? c->f32_bps : occ;
    return bps * c->num_sms;
}

// Partial-sum doubles the current variant needs.
size_t f32_part_doubles(ibim_ctx* c)
{
    if (is_sym(c->f32_variant)) return sym_part_doubles(c->N, f32_ttile(c), f32_grid_cap(c));
    const PairSchedule s = make_schedule(c->N, f32_ttile(c), c->N, kF32STile, f32_grid_cap(c));
    return (size_t)s.grid * s.max_segs * 2 * f32_ttile(c);
}

PairSchedule f32_schedule(ibim_ctx* c)
{
    return make_schedule(c->N, f32_ttile(c), c->N, kF32STile, f32_grid_cap(c));
}

ibim_status f32_chunk_frames(ibim_ctx* c)
{
    const int64_t nch = padded_nodes(c->N) / kChunk;
    IBIM_CUDA(cudaMalloc((void**)&c->d_frames, sizeof(float4) * 2 * nch));
    chunk_frames_kernel<<<(unsigned)((nch + 127) / 128), 128, 0, c->stream>>>(c->d_geo64, c->N, nch, c->d_pos32,
                                                                               c->d_frames);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f32_pack(ibim_ctx* c, VecRef in, const int* d_skip)
{
    const int64_t N = c->N;
    const int64_t n_pairs = padded_nodes(N) / 2;
    IBIM_TRY(ensure(c, &c->d_src, &c->src_bytes, (size_t)n_pairs * kPairF4 * sizeof(float4)));
    if (is_sym(c->f32_variant)) {
        IBIM_TRY(ensure(c, (void**)&c->d_yrev, &c->yrev_bytes, sym_yrev_bytes(N)));
        return sym_pack(c, in, d_skip);
    }
    const double* w = c->d_geo64 + 6 * N;
    const int bs = 256;
    pack_f32_kernel<<<(unsigned)((n_pairs + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_pos32, c->d_nrm32, w, in, N, n_pairs, (float4*)c->d_src, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f32_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip)
{
    IBIM_TRY(ensure(c, (void**)&c->d_part, &c->part_bytes, f32_part_doubles(c) * sizeof(double)));
    if (is_sym(c->f32_variant)) return sym_pairs(c, c->f32_variant - kNumVariants, f32_grid_cap(c), k, d_skip);
    const PairArgs a{c->d_pos32, c->d_nrm32, (const float4*)c->d_src, c->d_frames, c->N, s, f32_consts(k),
                     c->d_part, c->d_err, d_skip, Geo64{c->d_geo64, c->d_geo64 + 3 * c->N, 1, c->N}};
    kVariants[c->f32_variant].launch(a, c->stream);
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
    if (is_sym(c->f32_variant))
        return sym_fixup(c, c->f32_variant - kNumVariants, f32_grid_cap(c), k, in, out, d_skip);
    return fixup_launch(c, k, s, f32_ttile(c), in, out, d_skip);
}

// FP32 source payload of the context's nodes for input `in`, written to dst
// (padded N / 2 node pairs; the treecode packs into its own tile buffer).
ibim_status f32_pack_to(ibim_ctx* c, VecRef in, float4* dst, const int* d_skip)
{
    const int64_t n_pairs = padded_nodes(c->N) / 2;
    const int bs = 256;
    pack_f32_kernel<<<(unsigned)((n_pairs + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_pos32, c->d_nrm32, c->d_geo64 + 6 * c->N, in, c->N, n_pairs, dst, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

// Launchers on caller-supplied buffers (used by the allocation-free entry
// point): variant (kF32Tpt, 1), chunk frames and positions in them as a
// context's, arrays padded as above.
int f32_occupancy_per_sm()
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f32_kernel<kF32Tpt, 1, kF32Threads>, kF32Threads, 0);
    return occ < 1 ? 1 : occ;
}

cudaError_t launch_pair_f32_raw(const float4* tpos, const float4* tnrm, const float4* src, const float4* frames,
                                int64_t N, const PairSchedule& s, const PairConsts& k, double* part, unsigned* err,
                                cudaStream_t stream, const double* xs_aos, const double* nrm_aos)
{
    const PairArgs a{tpos, tnrm, src, frames, N, s, f32_consts(k), part, err, nullptr, Geo64{xs_aos, nrm_aos, 3, 1}};
    launch_variant<kF32Tpt, 1, kF32Threads>(a, stream);
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
