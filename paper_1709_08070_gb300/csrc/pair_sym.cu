// Symmetric FP32 pair sums of the IBIM operator (Sec. 2.2 discrete system,
// Sec. 2.2.1 regularisation), sm_103a.
//
// The pair geometry (r, |r|, e^{-kappa rho}, g, 3 - B, rho^-3, the theta
// terms) is the same for the ordered pairs (i <- j) and (j <- i), so one
// evaluation of an unordered pair gives both contributions: 48 FP32
// lane-operations per pair instead of 2 x 36 (28 shared and 10 per direction
// in pair_far_sym; 36 shared and 6 per direction in the rotation scheme's
// pair_far_sym_acc, which forms the factors common to both directions
// once).  Each aligned 32-node block pair
// (A, B) is evaluated once: by the warp holding target block A when B > A
// (both directions), B == A gives the forward direction only (it holds the
// self pairs), and B < A is skipped (the warp holding B covered it).
//
// Schedule: stream-K over the upper triangle of (target tile t, source tile
// s) steps, s >= R t with R = target tile / source tile; rows are visited in
// the order t = 0, n-1, 1, n-2, ..., so that every stretch of the step
// sequence holds the same share of diagonal (partly skipped, near-field)
// steps, and each row pair has the same length.  The step sequence is cut
// into contiguous segments: one large segment per CTA (9/10 of an even
// share), taken statically, then about 16 small segments per CTA handed out
// by an atomic counter, so that CTAs whose large segment held cheaper steps take
// more of the rest and all finish within about one small segment.
//
// Accumulation: the forward sums of a thread's targets run as in the
// one-directional kernel (FP32 over a chunk, Kahan across chunks, FP64
// across tiles, FP64 partials per (segment, row) summed in fixed order by
// the fixup, so the forward part does not depend on which CTA ran a segment).  The reverse contribution of a target to a source is summed over
// the warp's targets with shuffles (warp_sum4_add), over the CTA's warps with
// FP32 shared-memory atomics, and added to a global FP64 vector with atomics
// when the stage is released.  The order of both atomic sums varies from run
// to run, so the result varies at the FP32 rounding level of one tile's
// reverse partial (a few 1e-10 of max |y| measured), well inside the FP32
// operator's own error against FP64.
//
// Source payload (by node pairs, 64 bytes a pair, placeholders past N), four
// float4 components per pair:
//   A = (-y0.x, -y1.x, -y0.y, -y1.y)   minus the position in its chunk frame
//   B = (-y0.z, -y1.z,  b0,    b1  )   b = w psin
//   C = (m0.x, m1.x, m0.y, m1.y)       unit normals
//   D = (m0.z, m1.z, a0, a1)            a = w psi
// stored per 32-node chunk component by component (the 16 A's of the chunk,
// then its 16 B's, C's and D's), so that 16 lanes reading 16 different pairs
// of one chunk touch 256 contiguous bytes.
//
// Two schemes for the reverse sums (a variant parameter):
//   * warp reduction: per payload pair, the warp's reverse contributions are
//     summed by a transposed 4-value butterfly (warp_sum4_add) and added to
//     the stage's shared reverse buffer by four lanes;
//   * rotation (far chunks): each half-warp walks the chunk's 16 payload pairs
//     in a staggered order, lane l taking pair (l + k) mod 16 at step k, and
//     the reverse accumulators of a pair move with it from lane to lane (one
//     shuffle per value and step, the adds folded into the pair formula's
//     FMAs); after 16 steps each lane holds one pair's sums over its
//     half-warp, the two halves are added and 16 + 16 lanes add them to the
//     shared buffer.  Near chunks take the same walk with the packed near
//     formula (pair_near_sym_acc: series g, both directions' tube tests as
//     per-lane selects); the warp-reduction scheme evaluates them with the
//     scalar near path.  The rotation loop's unroll depth is a variant
//     parameter too (see tile_sums_sym).
#include <algorithm>

#include "pair_sym_core.cuh"

namespace ibim {


template <int TPT, int MINB, int THREADS, bool ROT, int UNR>
__global__ void __launch_bounds__(THREADS, MINB)
    pair_sym_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm,
                    const float4* __restrict__ src, const float4* __restrict__ frames, int64_t N, int64_t n_pad,
                    SymSchedule s, F32Consts k, double* __restrict__ part, double* __restrict__ yrev,
                    unsigned* __restrict__ err, const int* __restrict__ skip, Geo64 g64)
{
    constexpr int TTILE = THREADS * TPT;
    constexpr int NW = THREADS / 32;
    static_assert(TTILE <= kF32MaxTTile && TTILE % kF32STile == 0, "target tile");
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(16) float4 tfrm[NW][2 * TPT];
    __shared__ __align__(8) StagePipe pipe;
    constexpr int REVOFF = sym_rev_off(ROT);
    __shared__ float racc[kF32Stages][sym_rev_row(ROT)];
    __shared__ int64_t stage_st[kF32Stages];

    __shared__ int64_t seg_next[2];
    __shared__ int abort_sh;  // a bounded wait gave up: every warp leaves after the segment barrier

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    unsigned long long* seg_ctr = reinterpret_cast<unsigned long long*>(yrev + 2 * n_pad);

    for (int q = tid; q < kF32Stages * sym_rev_row(ROT); q += THREADS) (&racc[0][0])[q] = 0.0f;
    if (tid == 0) {
        pipe_init(pipe, NW);
        abort_sh = 0;
    }
    __syncthreads();

    // Ring position: step u of the current segment is this CTA's step number
    // u + off = done + (u - s0), where done counts the CTA's earlier steps
    // (stage = that mod kF32Stages, phase parity from its quotient).
    int64_t s0 = 0, s1 = 0, off = 0, done = 0;
    auto issue = [&](int64_t u) {
        int64_t t, rho, pos;
        sym_locate(s, u, t, rho, pos);
        const int64_t st = s.R * t + pos;
        const int stage = (int)((u + off) % kF32Stages);
        stage_st[stage] = st;
        pipe_issue(pipe, stg[stage], stage, src + st * (kF32STile / 2) * kPairF4, frames + st * 2 * kChunksPerTile);
    };

    int64_t t, rho, pos;
    SymTargets<TPT> T;
    int64_t gi0 = 0;
    int Ablk[TPT];
    bool idle = false;
    double D1[TPT], D2[TPT];

    auto load_targets = [&]() {
        gi0 = t * TTILE + tid;
        idle = t * TTILE + warp * 32 >= N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;  // < n_pad
            const float4 a = tpos[i];
            const float4 b = tnrm[i];
            T.x[q] = make_float3(a.x, a.y, a.z);
            T.nx[q] = f2(b.x);
            T.ny[q] = f2(b.y);
            T.nz[q] = f2(b.z);
            const float4 pb = src[sym_pair_offset(i >> 1, 1)];
            const float4 pa = src[sym_pair_offset(i >> 1, 3)];
            const float ai = (i & 1) ? pa.w : pa.z;
            const float bi = (i & 1) ? pb.w : pb.z;
            T.a[q] = f2(ai);
            T.nb[q] = f2(-bi);
            Ablk[q] = (int)((t * TTILE + (int64_t)q * THREADS + warp * 32) / kChunk);
            D1[q] = 0.0;
            D2[q] = 0.0;
        }
        __syncwarp();
        if (lane < 2 * TPT) {
            const int64_t blk0 = t * TTILE + (int64_t)(lane >> 1) * THREADS + warp * 32;
            tfrm[warp][lane] = frames[2 * (blk0 / kChunk) + (lane & 1)];
        }
        __syncwarp();
    };

    // warp 0: add the reverse sums of step v to the global vector and clear them
    auto flush = [&](int64_t v) {
        const int sv = (int)((v + off) % kF32Stages);
        const int64_t j0 = stage_st[sv] * kF32STile;
        for (int jj = lane; jj < kF32STile; jj += 32) {
            const float v1 = racc[sv][jj], v2 = racc[sv][REVOFF + jj];
            if (v1 != 0.0f) atomicAdd(yrev + j0 + jj, (double)v1);
            if (v2 != 0.0f) atomicAdd(yrev + n_pad + j0 + jj, (double)v2);
            racc[sv][jj] = 0.0f;
            racc[sv][REVOFF + jj] = 0.0f;
        }
        __syncwarp();
    };
    auto give_up = [&]() {
        if (lane == 0) {
            atomicOr(err, kDevErrTimeout);
            *(volatile int*)&abort_sh = 1;
        }
    };
    // warp 0: wait until every warp is past step v (its stage may be reused)
    auto wait_empty = [&](int64_t v) -> bool {
        bool ok = true;
        const int64_t w = v + off;
        if (lane == 0)
            ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(w % kF32Stages)], (uint32_t)((w / kF32Stages) & 1),
                                        kWaitLimitNs);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) give_up();
        return ok;
    };

    // The CTA's large segment first, then small segments from the counter.
    int64_t seg = blockIdx.x;
    int sp = 0;
    while (seg < s.nseg) {
        s0 = sym_seg_start(s, seg);
        s1 = sym_seg_start(s, seg + 1);
        off = done - s0;
        // every stage is free here: warp 0 waited for each earlier step's release
        if (tid == 0) {
            ptx::fence_proxy_async_smem();
            for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);
        }
        sym_locate(s, s0, t, rho, pos);
        load_targets();

        bool bad = false;
        for (int64_t u = s0; u < s1; ++u) {
            const int stage = (int)((u + off) % kF32Stages);
            const uint32_t parity = (uint32_t)(((u + off) / kF32Stages) & 1);
            if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
                give_up();
                bad = true;
                break;
            }
            const int64_t st = s.R * t + pos;
            float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;
            if (!idle)
                tile_sums_sym<TPT, ROT, UNR>(T, &tfrm[warp][0], stg[stage].buf, stg[stage].frm, k, S1, C1, S2, C2, g64, gi0,
                                   THREADS, st * kF32STile, N, Ablk, st * kChunksPerTile, &racc[stage][0]);
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                D1[q] += (double)S1[q] - (double)C1[q];
                D2[q] += (double)S2[q] - (double)C2[q];
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
            // warp 0: once every warp is past step u - 1, flush its reverse sums and refill its stage
            if (warp == 0 && u > s0) {
                if (!wait_empty(u - 1)) {
                    bad = true;
                    break;
                }
                flush(u - 1);
                if (lane == 0 && u - 1 + kF32Stages < s1) {
                    ptx::fence_proxy_async_smem();
                    issue(u - 1 + kF32Stages);
                }
                __syncwarp();
            }

            if (pos == sym_row_len(s, t) - 1 || u + 1 == s1) {
                double* dst = part + (seg + rho) * 2 * TTILE;
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    dst[q * THREADS + tid] = D1[q];
                    dst[TTILE + q * THREADS + tid] = D2[q];
                }
                if (u + 1 < s1) {
                    sym_locate(s, u + 1, t, rho, pos);
                    load_targets();
                }
            } else {
                ++pos;
            }
        }
        if (warp == 0) {  // the segment's last step: reverse sums, then the next segment
            if (!bad && wait_empty(s1 - 1)) {
                flush(s1 - 1);
                if (lane == 0) seg_next[sp] = s.nbig + (int64_t)atomicAdd(seg_ctr, 1ull);
            } else if (lane == 0) {
                seg_next[sp] = s.nseg;
            }
        }
        done += s1 - s0;
        __syncthreads();
        if (*(volatile int*)&abort_sh) return;
        seg = seg_next[sp];
        sp ^= 1;
    }
}

// Symmetric payload of the padded node range and a cleared reverse-sum vector.
__global__ void pack_sym_kernel(const float4* __restrict__ pos, const float4* __restrict__ nrm,
                                const double* __restrict__ w, VecRef in, int64_t N, int64_t n_pairs,
                                float4* __restrict__ src, double* __restrict__ yrev, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= n_pairs) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    const int64_t n_pad = 2 * n_pairs;
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
        yrev[j] = 0.0;
        yrev[n_pad + j] = 0.0;
    }
    if (pr == 0) *reinterpret_cast<unsigned long long*>(yrev + 2 * n_pad) = 0ull;  // small-segment counter
    write_source_pair_sym(src, pr, y[0], y[1], m[0], m[1], a[0], a[1], b[0], b[1]);
}

// y = Lambda p + (1/(4 pi)) (forward partials of the row + reverse sums).
// kFixParts threads per target, each summing a fixed share of the row's slots
// (a row near the end of the step sequence has one slot per small segment),
// then the shares in a fixed order: deterministic.  A block holds kFixTargets
// consecutive targets (a divisor of every target tile, so one row) for each
// share, so that a warp's loads of one slot are contiguous.
constexpr int kFixParts = 4, kFixTargets = 64;
__global__ void __launch_bounds__(kFixParts * kFixTargets)
    fixup_sym_kernel(const double* __restrict__ part, SymSchedule s, int ttile, int64_t N, int64_t n_pad,
                     double lambda1, double lambda2, VecRef in, OutRef out, const double* __restrict__ yrev,
                     const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    __shared__ double sh1[kFixParts][kFixTargets], sh2[kFixParts][kFixTargets];
    const int tl = threadIdx.x % kFixTargets, pr = threadIdx.x / kFixTargets;
    const int64_t i = (int64_t)blockIdx.x * kFixTargets + tl;
    double a1 = 0.0, a2 = 0.0;
    if (i < N) {
        const int64_t t = i / ttile;
        const int64_t l = i - t * ttile;
        int64_t start, rho;
        sym_row_start(s, t, start, rho);
        const int64_t c0 = sym_seg_of(s, start);
        const int64_t n = sym_seg_of(s, start + sym_row_len(s, t) - 1) - c0 + 1;
        const int64_t q0 = c0 + (n * pr) / kFixParts, q1 = c0 + (n * (pr + 1)) / kFixParts;
        // four slots per round with their loads independent (the row's slots are
        // consecutive, 2 ttile doubles apart)
        const int64_t ts = 2 * (int64_t)ttile;
        const double* src = part + (q0 + rho) * ts + l;
        int64_t c = q0;
        for (; c + 4 <= q1; c += 4, src += 4 * ts) {
            const double x0 = src[0], x1 = src[ts], x2 = src[2 * ts], x3 = src[3 * ts];
            const double y0 = src[ttile], y1 = src[ts + ttile], y2 = src[2 * ts + ttile], y3 = src[3 * ts + ttile];
            a1 += (x0 + x1) + (x2 + x3);
            a2 += (y0 + y1) + (y2 + y3);
        }
        for (; c < q1; ++c, src += ts) {
            a1 += src[0];
            a2 += src[ttile];
        }
    }
    sh1[pr][tl] = a1;
    sh2[pr][tl] = a2;
    __syncthreads();
    if (pr != 0 || i >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    double* y = out.base + (out.kidx ? (int64_t)(*out.kidx + out.koff) * out.stride : 0);
    const double f1 = yrev[i] + ((sh1[0][tl] + sh1[1][tl]) + (sh1[2][tl] + sh1[3][tl]));
    const double f2 = yrev[n_pad + i] + ((sh2[0][tl] + sh2[1][tl]) + (sh2[2][tl] + sh2[3][tl]));
    y[i] = lambda1 * p[i] + kInv4Pi * f1;
    y[N + i] = lambda2 * p[N + i] + kInv4Pi * f2;
}

// ------------------------------------------------------------------ host side

struct SymArgs {
    const float4* tpos;
    const float4* tnrm;
    const float4* src;
    const float4* frames;
    int64_t N, n_pad;
    SymSchedule s;
    F32Consts k;
    double* part;
    double* yrev;
    unsigned* err;
    const int* skip;
    Geo64 g64;
};

template <int TPT, int MINB, int THREADS, bool ROT, int UNR>
static void launch_sym(const SymArgs& a, cudaStream_t st)
{
    pair_sym_kernel<TPT, MINB, THREADS, ROT, UNR><<<a.s.grid, THREADS, 0, st>>>(
        a.tpos, a.tnrm, a.src, a.frames, a.N, a.n_pad, a.s, a.k, a.part, a.yrev, a.err, a.skip, a.g64);
}

// scheme: 1 = warp reduction of the reverse sums, 2 = rotation (see the file comment)
struct SymVariant {
    int tpt, minb, threads, scheme;
    const void* fn;
    void (*launch)(const SymArgs&, cudaStream_t);
};
#define IBIM_SYM_VARIANT(T, M, W, R, U) \
    {T, M, W, (R) ? 2 : 1, (const void*)pair_sym_kernel<T, M, W, R, U>, launch_sym<T, M, W, R, U>}
static const SymVariant kSymVariants[] = {
    IBIM_SYM_VARIANT(2, 1, 512, false, 2), IBIM_SYM_VARIANT(1, 1, 512, false, 2),
    IBIM_SYM_VARIANT(2, 1, 512, true, 1), IBIM_SYM_VARIANT(1, 1, 512, true, 4),
};
#undef IBIM_SYM_VARIANT
constexpr int kNumSymVariants = (int)(sizeof(kSymVariants) / sizeof(kSymVariants[0]));

int sym_variant_count() { return kNumSymVariants; }
void sym_variant_info(int v, int* tpt, int* minb, int* threads, int* scheme)
{
    *tpt = kSymVariants[v].tpt;
    *minb = kSymVariants[v].minb;
    *threads = kSymVariants[v].threads;
    *scheme = kSymVariants[v].scheme;
}
int sym_occupancy(int v)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kSymVariants[v].fn, kSymVariants[v].threads, 0);
    return occ < 1 ? 1 : occ;
}

// Large segments hold kSymBigShare (of kSymShareDen) of an even per-CTA share;
// the rest is cut into about kSymSmallPerCta small segments per CTA.
constexpr int64_t kSymBigShare = 9, kSymShareDen = 10, kSymSmallPerCta = 16;

SymSchedule make_sym_schedule(int64_t N, int ttile, int grid_cap)
{
    SymSchedule s;
    s.n_t = (N + ttile - 1) / ttile;
    s.n_s = (N + kF32STile - 1) / kF32STile;
    s.R = ttile / kF32STile;
    s.npairs = s.n_t / 2;
    s.L2 = 2 * s.n_s - s.R * (s.n_t - 1);
    s.total = s.npairs * s.L2 + ((s.n_t & 1) ? sym_row_len(s, s.npairs) : 0);
    int64_t g = std::min<int64_t>(grid_cap, s.total);
    if (g < 1) g = 1;
    s.nbig = g;
    s.Lb = std::max<int64_t>(1, (kSymBigShare * s.total) / (kSymShareDen * g));  // g Lb <= total as g <= total
    const int64_t rest = s.total - g * s.Lb;
    s.Ls = std::max<int64_t>(1, (rest + kSymSmallPerCta * g - 1) / (kSymSmallPerCta * g));
    s.nseg = g + (rest + s.Ls - 1) / s.Ls;
    s.grid = (int)g;
    return s;
}

// Partial slots (segment + row sequence index < nseg + n_t).
size_t sym_part_doubles(int64_t N, int ttile, int grid_cap)
{
    const SymSchedule s = make_sym_schedule(N, ttile, grid_cap);
    return (size_t)(s.nseg + s.n_t) * 2 * ttile;
}

// The reverse-sum vector (2 x padded N doubles) and, behind it, the
// small-segment counter (one 8-byte word).
size_t sym_yrev_bytes(int64_t N) { return sizeof(double) * (2 * (size_t)padded_nodes(N) + 1); }

ibim_status sym_pack(ibim_ctx* c, VecRef in, const int* d_skip)
{
    const int64_t N = c->N;
    const int64_t n_pairs = padded_nodes(N) / 2;
    const int bs = 256;
    pack_sym_kernel<<<(unsigned)((n_pairs + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_pos32, c->d_nrm32, c->d_geo64 + 6 * N, in, N, n_pairs, (float4*)c->d_src, c->d_yrev, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status sym_pairs(ibim_ctx* c, int sv, int grid_cap, const PairConsts& k, const int* d_skip)
{
    const SymVariant& v = kSymVariants[sv];
    const SymSchedule s = make_sym_schedule(c->N, v.tpt * v.threads, grid_cap);
    const int64_t n_pad = padded_nodes(c->N);
    const F32Consts kk = f32_consts(k);
    const Geo64 g64{c->d_geo64, c->d_geo64 + 3 * c->N, 1, c->N};
    const SymArgs a{c->d_pos32, c->d_nrm32, (const float4*)c->d_src, c->d_frames, c->N, n_pad, s, kk, c->d_part,
                    c->d_yrev, c->d_err, d_skip, g64};
    v.launch(a, c->stream);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status sym_fixup(ibim_ctx* c, int sv, int grid_cap, const PairConsts& k, VecRef in, OutRef out,
                      const int* d_skip)
{
    const SymVariant& v = kSymVariants[sv];
    return sym_fixup_tiles(c, v.tpt * v.threads, grid_cap, k, in, out, d_skip);
}

// y = Lambda p + (1/(4 pi)) (forward partials + reverse sums) for a symmetric
// launch of `ttile`-target tiles on a grid of at most grid_cap CTAs.
ibim_status sym_fixup_tiles(ibim_ctx* c, int ttile, int grid_cap, const PairConsts& k, VecRef in, OutRef out,
                            const int* d_skip)
{
    const SymSchedule s = make_sym_schedule(c->N, ttile, grid_cap);
    static_assert(kFixParts == 4 && kF32STile % kFixTargets == 0, "fixup shares");
    fixup_sym_kernel<<<(unsigned)((c->N + kFixTargets - 1) / kFixTargets), kFixParts * kFixTargets, 0, c->stream>>>(
        c->d_part, s, ttile, c->N, padded_nodes(c->N), k.lambda1, k.lambda2, in, out, c->d_yrev, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

}  // namespace ibim
