// Batched IBIM solves: many molecules with uneven narrowband sizes advance
// their GMRES iterations in lock-step, and every round's operator
// applications for all still-active molecules run as ONE persistent launch.
//
// Round (captured once into a CUDA graph and replayed):
//   batch_plan_kernel   active molecules (GMRES not done) and the prefix sums
//                       of their (target tile x source tile) step counts;
//                       steps per CTA for the persistent grid
//   batch_pack_kernel   each active molecule's FP32 source payload from its
//                       current Krylov vector, and y = Lambda p (diagonal)
//   batch_pair_kernel   stream-K over the concatenated step space; each step
//                       looks up its molecule, stages that molecule's source
//                       tile with a bulk async copy and evaluates it with the
//                       same arithmetic as the single-molecule kernel; tile
//                       sums are added to the molecule's output in FP64
//                       (atomic adds: the few CTAs sharing a target tile)
//   per molecule        CGS2 orthogonalisation, normalisation and Givens
//                       (the single-molecule kernels, skipped once done)
// Molecules that converge drop out of the plan, so later rounds only spend
// time on the molecules still iterating.
#include <string.h>

#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gmres_internal.cuh"
#include "pair_sym_core.cuh"

namespace ibim {

constexpr int kMaxBatch = 1024;
// Batched pair-kernel variants (targets per thread x CTA size x minimum CTAs
// per SM, i.e. target tiles of 512, 256 or 128 nodes; one target per thread,
// because the per-molecule state of the batched walk leaves no registers for
// a second slot without spilling).  The first batched solve of a size class
// times each one on its first round and keeps the fastest (see batch_solve).

struct BatchMol {
    const float4* pos;
    const float4* nrm;
    const float4* frames;
    float4* src;
    const double* w;
    double* V;
    double* x;
    double* t;
    GmState* st;
    int64_t N, n_stiles;
    int64_t sperm;  // source-tile visiting stride (see make_schedule)
    F32Consts k;
    double lambda1, lambda2;
    Geo64 g64;
};

struct BatchPlan {
    int nactive;
    int pad;
    int64_t total;
    int64_t per_cta;
    int mol[kMaxBatch];
    int64_t off[kMaxBatch + 1];
};

// mode 0: Arnoldi round (active = GMRES not done; in = V_k, out = V_{k+1});
// mode 1: residual round (active = want[m]; in = x, out = t).
__device__ __forceinline__ const double* batch_in(const BatchMol& M, int mode)
{
    return mode == 0 ? M.V + (int64_t)M.st->k * 2 * M.N : M.x;
}
__device__ __forceinline__ double* batch_out(const BatchMol& M, int mode)
{
    return mode == 0 ? M.V + (int64_t)(M.st->k + 1) * 2 * M.N : M.t;
}

// Steps of one molecule: every (target tile, source tile) pair, or with R > 0
// (symmetric kernel, R = target tile / source tile) the upper triangle: row t
// holds the source tiles R t .. n_s - 1.
__host__ __device__ __forceinline__ int64_t batch_mol_steps(int64_t N, int64_t ttile, int64_t n_s, int64_t R)
{
    const int64_t n_t = (N + ttile - 1) / ttile;
    return R > 0 ? n_t * n_s - R * n_t * (n_t - 1) / 2 : n_t * n_s;
}

__global__ void batch_plan_kernel(const BatchMol* __restrict__ mols, int nmol, int mode, const int* __restrict__ want,
                                  int64_t ttile, int64_t sym_R, int grid, BatchPlan* __restrict__ plan)
{
    if (threadIdx.x != 0) return;
    int a = 0;
    int64_t total = 0;
    for (int m = 0; m < nmol; ++m) {
        const bool active = (mode == 0) ? (mols[m].st->done == 0) : (want[m] != 0);
        if (!active) continue;
        plan->mol[a] = m;
        plan->off[a] = total;
        total += batch_mol_steps(mols[m].N, ttile, mols[m].n_stiles, sym_R);
        ++a;
    }
    plan->off[a] = total;
    plan->nactive = a;
    plan->total = total;
    plan->per_cta = total > 0 ? (total + grid - 1) / grid : 1;
}

__global__ void batch_pack_kernel(const BatchMol* __restrict__ mols, const BatchPlan* __restrict__ plan, int mode)
{
    const int a = blockIdx.y;
    if (a >= plan->nactive) return;
    const BatchMol& M = mols[plan->mol[a]];
    const double* p = batch_in(M, mode);
    double* y = batch_out(M, mode);
    const int64_t N = M.N;
    const int64_t n_pairs = padded_nodes(N) / 2;
    for (int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pr < n_pairs;
         pr += (int64_t)gridDim.x * blockDim.x) {
        float4 q[2], n[2];
        float av[2], bv[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t j = 2 * pr + e;
            if (j < N) {
                q[e] = M.pos[j];
                n[e] = M.nrm[j];
                const double wj = M.w[j];
                const double pj = p[j], pn = p[N + j];
                av[e] = (float)(wj * pj);
                bv[e] = (float)(wj * pn);
                y[j] = M.lambda1 * pj;
                y[N + j] = M.lambda2 * pn;
            } else {
                q[e] = pad_source_pos();
                n[e] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
                av[e] = bv[e] = 0.0f;
            }
        }
        write_source_pair(M.src + kPairF4 * pr, q[0], q[1], n[0], n[1], av[0], av[1], bv[0], bv[1]);
    }
}

// As batch_pack_kernel, with the symmetric kernel's payload layout.
__global__ void batch_sym_pack_kernel(const BatchMol* __restrict__ mols, const BatchPlan* __restrict__ plan, int mode)
{
    const int a = blockIdx.y;
    if (a >= plan->nactive) return;
    const BatchMol& M = mols[plan->mol[a]];
    const double* p = batch_in(M, mode);
    double* y = batch_out(M, mode);
    const int64_t N = M.N;
    const int64_t n_pairs = padded_nodes(N) / 2;
    for (int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pr < n_pairs;
         pr += (int64_t)gridDim.x * blockDim.x) {
        float4 q[2], n[2];
        float av[2], bv[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t j = 2 * pr + e;
            if (j < N) {
                q[e] = M.pos[j];
                n[e] = M.nrm[j];
                const double wj = M.w[j];
                const double pj = p[j], pn = p[N + j];
                av[e] = (float)(wj * pj);
                bv[e] = (float)(wj * pn);
                y[j] = M.lambda1 * pj;
                y[N + j] = M.lambda2 * pn;
            } else {
                q[e] = pad_source_pos();
                n[e] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
                av[e] = bv[e] = 0.0f;
            }
        }
        write_source_pair_sym(M.src, pr, q[0], q[1], n[0], n[1], av[0], av[1], bv[0], bv[1]);
    }
}

// Symmetric batched pair sums (rotation scheme of pair_sym.cu): stream-K over
// the concatenated upper triangles of the active molecules' (target tile,
// source tile) steps.  Forward sums of a row are added to the molecule's
// output with FP64 atomics when the row (or the CTA's range) ends; the
// reverse sums of a staged source tile are collected in shared memory and
// added to the output with FP64 atomics once every warp has released the
// stage (warp 0, before it refills the stage).  UNR: unroll depth of the
// rotation loop (4 with one target per thread: 8.98e11 against 8.74e11
// interactions/s at 2 over 8 rounds of the 64-globule batch).
template <int TPT, int THREADS, int UNR>
__global__ void __launch_bounds__(THREADS, 1)
    batch_sym_kernel(const BatchMol* __restrict__ mols, const BatchPlan* __restrict__ plan, int mode,
                     unsigned* __restrict__ err)
{
    constexpr int TTILE = TPT * THREADS;
    constexpr int NW = THREADS / 32;
    constexpr int64_t R = TTILE / kF32STile;
    constexpr int REVOFF = sym_rev_off(true);
    static_assert(TTILE <= kF32MaxTTile && TTILE % kF32STile == 0, "target tile");
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(16) float4 tfrm[NW][2 * TPT];
    __shared__ __align__(8) StagePipe pipe;
    __shared__ float racc[kF32Stages][sym_rev_row(true)];
    __shared__ int stage_mol[kF32Stages];
    __shared__ int64_t stage_st[kF32Stages];
    // constants of the molecule of each staged tile (written with the stage's
    // copy, read by the warps that consume the stage)
    __shared__ F32Consts stage_k[kF32Stages];
    __shared__ Geo64 stage_g[kF32Stages];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t total = plan->total;
    const int64_t per_cta = plan->per_cta;
    const int64_t s0 = (int64_t)blockIdx.x * per_cta;
    const int64_t s1 = (s0 + per_cta < total) ? s0 + per_cta : total;
    if (s0 >= s1) return;
    const int nact = plan->nactive;
    const int* __restrict__ s_mol = plan->mol;
    const int64_t* __restrict__ s_off = plan->off;
    for (int q = tid; q < kF32Stages * sym_rev_row(true); q += THREADS) (&racc[0][0])[q] = 0.0f;
    if (tid == 0) pipe_init(pipe, NW);
    __syncthreads();

    // step u -> active index a, row t and position in the row
    auto locate = [&](int64_t u, int& a, int64_t& t, int64_t& pos) {
        int lo = 0, hi = nact - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        a = lo;
        const BatchMol& M = mols[s_mol[a]];
        const int64_t v = u - s_off[a];
        const int64_t n_s = M.n_stiles, n_t = (M.N + TTILE - 1) / TTILE;
        // rows before t hold t n_s - R t (t - 1) / 2 steps (increasing in t)
        int64_t tl = 0, th = n_t - 1;
        while (tl < th) {
            const int64_t mid = (tl + th + 1) >> 1;
            if (mid * n_s - R * mid * (mid - 1) / 2 <= v) tl = mid;
            else th = mid - 1;
        }
        t = tl;
        pos = v - (tl * n_s - R * tl * (tl - 1) / 2);
    };
    auto issue = [&](int64_t u) {
        int a;
        int64_t t, pos;
        locate(u, a, t, pos);
        const BatchMol& M = mols[s_mol[a]];
        const int64_t st = R * t + pos;
        const int stage = (int)((u - s0) % kF32Stages);
        stage_mol[stage] = s_mol[a];
        stage_st[stage] = st;
        stage_k[stage] = M.k;
        stage_g[stage] = M.g64;
        pipe_issue(pipe, stg[stage], stage, M.src + st * (kF32STile / 2) * kPairF4, M.frames + st * 2 * kChunksPerTile);
    };
    if (tid == 0)
        for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);

    int a;
    int64_t t, pos;
    locate(s0, a, t, pos);
    const BatchMol* M = &mols[s_mol[a]];
    SymTargets<TPT> T;
    int64_t gi0 = 0;
    int Ablk[TPT];
    bool idle = false;
    double D1[TPT], D2[TPT];

    auto load_targets = [&]() {
        gi0 = t * TTILE + tid;
        idle = t * TTILE + warp * 32 >= M->N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;  // < padded N
            const float4 p4 = M->pos[i];
            const float4 n4 = M->nrm[i];
            T.x[q] = make_float3(p4.x, p4.y, p4.z);
            T.nx[q] = f2(n4.x);
            T.ny[q] = f2(n4.y);
            T.nz[q] = f2(n4.z);
            const float4 pb = M->src[sym_pair_offset(i >> 1, 1)];
            const float4 pa = M->src[sym_pair_offset(i >> 1, 3)];
            T.a[q] = f2((i & 1) ? pa.w : pa.z);
            T.nb[q] = f2(-((i & 1) ? pb.w : pb.z));
            Ablk[q] = (int)((t * TTILE + (int64_t)q * THREADS + warp * 32) / kChunk);
            D1[q] = 0.0;
            D2[q] = 0.0;
        }
        __syncwarp();
        if (lane < 2 * TPT) {
            const int64_t blk0 = t * TTILE + (int64_t)(lane >> 1) * THREADS + warp * 32;
            tfrm[warp][lane] = M->frames[2 * (blk0 / kChunk) + (lane & 1)];
        }
        __syncwarp();
    };
    // forward sums of the current row into the molecule's output
    auto flush_rows = [&]() {
        double* y = batch_out(*M, mode);
        const int64_t N = M->N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;
            if (i < N) {
                atomicAdd(y + i, kInv4Pi * D1[q]);
                atomicAdd(y + N + i, kInv4Pi * D2[q]);
            }
        }
    };
    // warp 0: reverse sums of the tile staged for step v into its molecule's output
    auto flush_rev = [&](int64_t v) {
        const int sv = (int)((v - s0) % kF32Stages);
        const BatchMol& S = mols[stage_mol[sv]];
        double* y = batch_out(S, mode);
        const int64_t N = S.N;
        const int64_t j0 = stage_st[sv] * kF32STile;
        for (int jj = lane; jj < kF32STile; jj += 32) {
            const float v1 = racc[sv][jj], v2 = racc[sv][REVOFF + jj];
            if (j0 + jj < N) {
                if (v1 != 0.0f) atomicAdd(y + j0 + jj, kInv4Pi * (double)v1);
                if (v2 != 0.0f) atomicAdd(y + N + j0 + jj, kInv4Pi * (double)v2);
            }
            racc[sv][jj] = 0.0f;
            racc[sv][REVOFF + jj] = 0.0f;
        }
        __syncwarp();
    };
    // warp 0: wait until every warp is past step v
    auto wait_empty = [&](int64_t v) -> bool {
        bool ok = true;
        const int64_t w = v - s0;
        if (lane == 0)
            ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(w % kF32Stages)], (uint32_t)((w / kF32Stages) & 1),
                                        kWaitLimitNs);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) atomicOr(err, kDevErrTimeout);
        return ok;
    };
    load_targets();

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kF32Stages);
        const uint32_t parity = (uint32_t)(((u - s0) / kF32Stages) & 1);
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
            if (lane == 0) atomicOr(err, kDevErrTimeout);
            return;
        }
        const int64_t st = R * t + pos;
        float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;
        if (!idle)
            tile_sums_sym<TPT, true, UNR>(T, &tfrm[warp][0], stg[stage].buf, stg[stage].frm, stage_k[stage], S1, C1, S2, C2,
                                     stage_g[stage], gi0, THREADS, st * kF32STile, M->N, Ablk, st * kChunksPerTile,
                                     &racc[stage][0]);
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            D1[q] += (double)S1[q] - (double)C1[q];
            D2[q] += (double)S2[q] - (double)C2[q];
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
        if (warp == 0 && u > s0) {
            if (!wait_empty(u - 1)) return;
            flush_rev(u - 1);
            if (lane == 0 && u - 1 + kF32Stages < s1) {
                ptx::fence_proxy_async_smem();
                issue(u - 1 + kF32Stages);
            }
            __syncwarp();
        }
        // advance to step u + 1
        const int64_t row_len = M->n_stiles - R * t;
        const bool row_ends = (pos + 1 == row_len);
        if (row_ends || u + 1 == s1) flush_rows();
        if (u + 1 == s1) break;
        if (!row_ends) {
            ++pos;
        } else {
            pos = 0;
            if (t + 1 < (M->N + TTILE - 1) / TTILE) {
                ++t;
            } else {
                ++a;
                M = &mols[s_mol[a]];
                t = 0;
            }
            load_targets();
        }
    }
    if (warp == 0 && wait_empty(s1 - 1)) flush_rev(s1 - 1);
}

template <int TPT, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    batch_pair_kernel(const BatchMol* __restrict__ mols, const BatchPlan* __restrict__ plan, int mode,
                      unsigned* __restrict__ err)
{
    constexpr int TTILE = TPT * THREADS;
    constexpr int NW = THREADS / 32;
    static_assert(TTILE <= kF32MaxTTile, "target tile");
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(16) float4 tfrm[NW][2 * TPT];
    __shared__ __align__(8) StagePipe pipe;
    __shared__ int s_nact;
    __shared__ int s_mol[kMaxBatch];
    __shared__ int64_t s_off[kMaxBatch + 1];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int64_t total = plan->total;
    const int64_t per_cta = plan->per_cta;
    const int64_t s0 = (int64_t)blockIdx.x * per_cta;
    const int64_t s1 = (s0 + per_cta < total) ? s0 + per_cta : total;
    if (s0 >= s1) return;
    const int nact = plan->nactive;
    for (int q = tid; q < nact; q += blockDim.x) s_mol[q] = plan->mol[q];
    for (int q = tid; q <= nact; q += blockDim.x) s_off[q] = plan->off[q];
    if (tid == 0) {
        s_nact = nact;
        pipe_init(pipe, NW);
    }
    __syncthreads();

    // active index of step u: s_off[a] <= u < s_off[a + 1]
    auto locate = [&](int64_t u) {
        int lo = 0, hi = s_nact - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    auto issue = [&](int64_t u) {
        const int a = locate(u);
        const BatchMol& M = mols[s_mol[a]];
        const int64_t st = (((u - s_off[a]) % M.n_stiles) * M.sperm) % M.n_stiles;
        const int stage = (int)((u - s0) % kF32Stages);
        pipe_issue(pipe, stg[stage], stage, M.src + st * (kF32STile / 2) * kPairF4,
                   M.frames + st * 2 * kChunksPerTile);
    };
    if (tid == 0)
        for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);

    int a = locate(s0);
    const BatchMol* M = &mols[s_mol[a]];
    int64_t v = s0 - s_off[a];
    int64_t t = v / M->n_stiles;
    int64_t st = v % M->n_stiles;
    Targets<TPT> T;
    int64_t gi0 = 0;
    bool idle = false;
    double D1[TPT], D2[TPT];

    auto load_targets = [&]() {
        gi0 = t * TTILE + tid;
        idle = t * TTILE + warp * 32 >= M->N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;
            const float4 p4 = M->pos[i];
            const float4 n4 = M->nrm[i];
            T.x[q] = make_float3(p4.x, p4.y, p4.z);
            T.nx[q] = f2(n4.x);
            T.ny[q] = f2(n4.y);
            T.nz[q] = f2(n4.z);
            D1[q] = 0.0;
            D2[q] = 0.0;
        }
        __syncwarp();
        if (lane < 2 * TPT) {
            const int64_t blk0 = t * TTILE + (int64_t)(lane >> 1) * THREADS + warp * 32;
            tfrm[warp][lane] = M->frames[2 * (blk0 / kChunk) + (lane & 1)];
        }
        __syncwarp();
    };
    auto flush = [&]() {
        double* y = batch_out(*M, mode);
        const int64_t N = M->N;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t i = gi0 + (int64_t)q * THREADS;
            if (i < N) {
                atomicAdd(y + i, kInv4Pi * D1[q]);
                atomicAdd(y + N + i, kInv4Pi * D2[q]);
            }
        }
    };
    load_targets();

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kF32Stages);
        const uint32_t parity = (uint32_t)(((u - s0) / kF32Stages) & 1);
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
            if (lane == 0) atomicOr(err, kDevErrTimeout);
            return;
        }
        float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;
        if (!idle)
            tile_sums<TPT>(T, &tfrm[warp][0], true, stg[stage].buf, stg[stage].frm, M->k, S1, C1, S2, C2, M->g64, gi0,
                           THREADS, ((st * M->sperm) % M->n_stiles) * kF32STile, M->N);
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            D1[q] += (double)S1[q] - (double)C1[q];
            D2[q] += (double)S2[q] - (double)C2[q];
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
        if (warp == 0) {
            bool ok = true;
            if (lane == 0 && u > s0 && u - 1 + kF32Stages < s1) {
                const int64_t w = u - 1 - s0;
                ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(w % kF32Stages)], (uint32_t)((w / kF32Stages) & 1),
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
        // advance to step u + 1
        const bool tile_ends = (st + 1 == M->n_stiles);
        if (tile_ends || u + 1 == s1) flush();
        if (u + 1 == s1) break;
        if (!tile_ends) {
            ++st;
        } else {
            st = 0;
            if (t + 1 < (M->N + TTILE - 1) / TTILE) {
                ++t;
            } else {
                ++a;
                M = &mols[s_mol[a]];
                t = 0;
            }
            load_targets();
        }
    }
}

struct BatchVariant {
    int tpt, threads, minb, sym;
    const void* fn;
    void (*launch)(int grid, cudaStream_t st, const BatchMol* mols, const BatchPlan* plan, int mode, unsigned* err);
};
template <int T, int W, int M>
static void launch_batch_pair(int grid, cudaStream_t st, const BatchMol* mols, const BatchPlan* plan, int mode,
                              unsigned* err)
{
    batch_pair_kernel<T, W, M><<<grid, W, 0, st>>>(mols, plan, mode, err);
}
template <int T, int W, int U>
static void launch_batch_sym(int grid, cudaStream_t st, const BatchMol* mols, const BatchPlan* plan, int mode,
                             unsigned* err)
{
    batch_sym_kernel<T, W, U><<<grid, W, 0, st>>>(mols, plan, mode, err);
}
#define IBIM_BATCH_VARIANT(T, W, M) {T, W, M, 0, (const void*)batch_pair_kernel<T, W, M>, launch_batch_pair<T, W, M>}
#define IBIM_BATCH_SYM_VARIANT(T, W, U) \
    {T, W, 1, 1, (const void*)batch_sym_kernel<T, W, U>, launch_batch_sym<T, W, U>}
static const BatchVariant kBatchVariants[] = {
    IBIM_BATCH_VARIANT(1, 512, 1), IBIM_BATCH_VARIANT(1, 256, 2), IBIM_BATCH_VARIANT(1, 128, 4),
    IBIM_BATCH_SYM_VARIANT(1, 512, 4),
};
#undef IBIM_BATCH_VARIANT
#undef IBIM_BATCH_SYM_VARIANT
constexpr int kNumBatchVariants = (int)(sizeof(kBatchVariants) / sizeof(kBatchVariants[0]));

// ------------------------------------------------------------------ host side

namespace {

struct BatchRun {
    int nmol = 0;
    BatchMol* d_mols = nullptr;
    BatchPlan* d_plan = nullptr;
    int* d_want = nullptr;
    cudaStream_t bs = nullptr;
    cudaGraphExec_t exec = nullptr;
    int variant = 0;
    int grid = 0;
    int pack_blocks = 0;
    int sms = 0;
    void set_variant(int v)
    {
        variant = v;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kBatchVariants[v].fn, kBatchVariants[v].threads, 0);
        grid = (occ < 1 ? 1 : occ) * sms;
    }
    ~BatchRun()
    {
        if (exec) cudaGraphExecDestroy(exec);
        cudaFree(d_mols);
        cudaFree(d_plan);
        cudaFree(d_want);
        if (bs) cudaStreamDestroy(bs);
    }
};

std::mutex g_batch_tune_mu;
// (device, floor(log2 sum N^2), tolerance below kSymTolFloor) -> variant
std::map<std::tuple<int, int, int>, int> g_batch_tune;
int g_batch_forced = -1;                           // ibim_set_batch_variant (-1: measured choice)

}  // namespace

static ibim_status batch_operator(ibim_ctx* c0, BatchRun& R, int mode)
{
    const BatchVariant& v = kBatchVariants[R.variant];
    const int64_t ttile = (int64_t)v.tpt * v.threads;
    batch_plan_kernel<<<1, 32, 0, R.bs>>>(R.d_mols, R.nmol, mode, R.d_want, ttile, v.sym ? ttile / kF32STile : 0,
                                          R.grid, R.d_plan);
    if (v.sym)
        batch_sym_pack_kernel<<<dim3(R.pack_blocks, R.nmol), 256, 0, R.bs>>>(R.d_mols, R.d_plan, mode);
    else
        batch_pack_kernel<<<dim3(R.pack_blocks, R.nmol), 256, 0, R.bs>>>(R.d_mols, R.d_plan, mode);
    v.launch(R.grid, R.bs, R.d_mols, R.d_plan, mode, c0->d_err);
    count_launch(c0, 3);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

static ibim_status tune_batch_variant(ibim_ctx* c0, BatchRun& R, double tol)
{
    cudaEvent_t e0, e1;
    IBIM_CUDA(cudaEventCreate(&e0));
    IBIM_CUDA(cudaEventCreate(&e1));
    float best = 3.0e38f;
    int pick = R.variant;
    ibim_status st = IBIM_OK;
    for (int v = 0; v < kNumBatchVariants && st == IBIM_OK; ++v) {
        if (kBatchVariants[v].sym && tol < kSymTolFloor) continue;  // see kSymTolFloor
        R.set_variant(v);
        cudaEventRecord(e0, R.bs);
        st = batch_operator(c0, R, 0);
        cudaEventRecord(e1, R.bs);
        if (st == IBIM_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    R.set_variant(pick);
    return st;
}

static thread_local int batch_last_variant = -1;

int batch_variant_count() { return kNumBatchVariants; }
void batch_variant_info(int v, int* tpt, int* threads, int* symmetric)
{
    *tpt = kBatchVariants[v].tpt;
    *threads = kBatchVariants[v].threads;
    *symmetric = kBatchVariants[v].sym;
}
void batch_force_variant(int v)
{
    std::lock_guard<std::mutex> lock(g_batch_tune_mu);
    g_batch_forced = v;
}
int batch_last_variant_used() { return batch_last_variant; }

ibim_status batch_solve(int nmol, ibim_ctx* const* ctxs, const ibim_phys* phys, const ibim_solve_opts& o,
                        double* const* d_p, ibim_solve_info* infos)
{
    const int m = std::min(o.restart, kMaxRestart);
    BatchRun R;
    R.nmol = nmol;
    IBIM_CUDA(cudaStreamCreateWithFlags(&R.bs, cudaStreamNonBlocking));
    std::vector<cudaStream_t> user(nmol);
    std::vector<BatchMol> h(nmol);
    std::vector<double> gnorm(nmol, 0.0);
    int64_t maxN = 0;
    int sms = ctxs[0]->num_sms;
    // order every molecule's queued work before the batch stream
    cudaEvent_t ev;
    IBIM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (int i = 0; i < nmol; ++i) {
        IBIM_CUDA(cudaEventRecord(ev, ctxs[i]->stream));
        IBIM_CUDA(cudaStreamWaitEvent(R.bs, ev, 0));
    }
    for (int i = 0; i < nmol; ++i) {
        user[i] = ctxs[i]->stream;
        ctxs[i]->stream = R.bs;
    }
    struct Restore {
        int n;
        ibim_ctx* const* c;
        std::vector<cudaStream_t>* u;
        cudaStream_t bs;
        cudaEvent_t ev;
        ~Restore()
        {
            cudaEventRecord(ev, bs);
            for (int i = 0; i < n; ++i) {
                c[i]->stream = (*u)[i];
                cudaStreamWaitEvent(c[i]->stream, ev, 0);
            }
            cudaEventDestroy(ev);
        }
    } restore{nmol, ctxs, &user, R.bs, ev};
    for (int i = 0; i < nmol; ++i) {
        ibim_ctx* c = ctxs[i];
        IBIM_TRY(gm_alloc(c, m));
        IBIM_TRY(ensure_operator_workspaces(c));
        IBIM_TRY(gm_init(c, phys[i], m, &gnorm[i]));
        const PairConsts pk = make_consts(phys[i]);
        BatchMol& b = h[i];
        b.pos = c->d_pos32;
        b.nrm = c->d_nrm32;
        b.frames = c->d_frames;
        b.src = (float4*)c->d_src;
        b.w = c->d_geo64 + 6 * c->N;
        b.V = c->gm->V;
        b.x = c->gm->x;
        b.t = c->gm->t;
        b.st = c->gm->st;
        b.N = c->N;
        b.n_stiles = (c->N + kF32STile - 1) / kF32STile;
        b.sperm = make_schedule(c->N, kF32STile, c->N, kF32STile, 1).sperm;  // depends on n_stiles only
        b.k = f32_consts(pk);
        b.lambda1 = pk.lambda1;
        b.lambda2 = pk.lambda2;
        b.g64 = Geo64{c->d_geo64, c->d_geo64 + 3 * c->N, 1, c->N};
        maxN = std::max(maxN, c->N);
    }
    IBIM_CUDA(cudaMalloc((void**)&R.d_mols, sizeof(BatchMol) * nmol));
    IBIM_CUDA(cudaMalloc((void**)&R.d_plan, sizeof(BatchPlan)));
    IBIM_CUDA(cudaMalloc((void**)&R.d_want, sizeof(int) * nmol));
    IBIM_CUDA(cudaMemcpyAsync(R.d_mols, h.data(), sizeof(BatchMol) * nmol, cudaMemcpyHostToDevice, R.bs));
    R.sms = sms;
    double sum_n2 = 0.0;
    for (int i = 0; i < nmol; ++i) sum_n2 += (double)ctxs[i]->N * (double)ctxs[i]->N;
    const int bucket = (int)floor(log2(sum_n2 > 1.0 ? sum_n2 : 1.0));
    int cached = -1;
    {
        std::lock_guard<std::mutex> lock(g_batch_tune_mu);
        auto it = g_batch_tune.find({ctxs[0]->device, bucket, o.tol < kSymTolFloor ? 1 : 0});
        if (it != g_batch_tune.end()) cached = it->second;
        if (g_batch_forced >= 0) cached = g_batch_forced;
    }
    R.set_variant(cached >= 0 ? cached : 0);
    R.pack_blocks = (int)std::min<int64_t>(256, (maxN + 255) / 256);

    std::vector<int> iters(nmol, 0), cycles(nmol, 0), conv(nmol, 0), finished(nmol, 0);
    std::vector<double> beta(nmol, 0.0);
    std::vector<char> x_zero(nmol, 1);
    std::vector<int> want(nmol, 0);
    for (int i = 0; i < nmol; ++i)
        if (gnorm[i] == 0.0) finished[i] = conv[i] = 1;
    if (o.start == 3)  // the caller's vectors are the starting iterates (a residual round comes first)
        for (int i = 0; i < nmol; ++i) {
            if (finished[i]) continue;
            IBIM_CUDA(cudaMemcpyAsync(ctxs[i]->gm->x, d_p[i], sizeof(double) * 2 * ctxs[i]->N,
                                      cudaMemcpyDeviceToDevice, R.bs));
            x_zero[i] = 0;
        }

    for (int cycle_guard = 0; cycle_guard < 1000; ++cycle_guard) {
        // residuals of the molecules that have an iterate
        int nres = 0;
        for (int i = 0; i < nmol; ++i) {
            want[i] = (!finished[i] && !x_zero[i]) ? 1 : 0;
            nres += want[i];
        }
        if (nres > 0) {
            for (int i = 0; i < nmol; ++i) infos[i].matvecs_f32 += want[i];
            IBIM_CUDA(cudaMemcpyAsync(R.d_want, want.data(), sizeof(int) * nmol, cudaMemcpyHostToDevice, R.bs));
            IBIM_TRY(batch_operator(ctxs[0], R, 1));
        }
        int nactive = 0;
        for (int i = 0; i < nmol; ++i) {
            if (finished[i]) continue;
            const int kmax = std::max(0, std::min(m, o.maxit - iters[i]));
            IBIM_TRY(gm_cycle_begin(ctxs[i], x_zero[i] != 0, o.tol * gnorm[i], kmax));
            IBIM_TRY(gm_fetch_state(ctxs[i]));
        }
        IBIM_CUDA(cudaStreamSynchronize(R.bs));
        for (int i = 0; i < nmol; ++i) {
            if (finished[i]) continue;
            x_zero[i] = 0;
            beta[i] = ctxs[i]->gm->h_st->resid;
            const int kmax = std::max(0, std::min(m, o.maxit - iters[i]));
            if (beta[i] <= o.tol * gnorm[i]) {
                finished[i] = conv[i] = 1;
            } else if (kmax <= 0) {
                finished[i] = 1;
            } else {
                ++nactive;
            }
        }
        if (nactive == 0) break;
        // First round of a size class not seen before: time every variant on
        // this round (plan + pack + pairs recompute V_{k+1} from scratch, so
        // repeating them is harmless) and keep the fastest.
        if (cached < 0) {
            IBIM_TRY(tune_batch_variant(ctxs[0], R, o.tol));
            cached = R.variant;
            std::lock_guard<std::mutex> lock(g_batch_tune_mu);
            g_batch_tune[{ctxs[0]->device, bucket, o.tol < kSymTolFloor ? 1 : 0}] = cached;
        }
        batch_last_variant = R.variant;
        // one graph per solve: plan + pack + batched pairs + every molecule's orthogonalisation
        if (R.exec == nullptr) {
            cudaGraph_t graph = nullptr;
            const int64_t before = ctxs[0]->timing.total_launches;
            IBIM_CUDA(cudaStreamBeginCapture(R.bs, cudaStreamCaptureModeThreadLocal));
            ibim_status s = batch_operator(ctxs[0], R, 0);
            for (int i = 0; i < nmol && s == IBIM_OK; ++i) s = gm_ortho(ctxs[i]);
            cudaError_t e = cudaStreamEndCapture(R.bs, &graph);
            ctxs[0]->timing.total_launches = before;
            for (int i = 1; i < nmol; ++i) ctxs[i]->timing.total_launches -= 9;
            if (s != IBIM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (e != cudaSuccess) return cuda_fail(e, "capture of the batched round", __FILE__, __LINE__);
            e = cudaGraphInstantiate(&R.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate (batch)", __FILE__, __LINE__);
        }
        for (int round = 0; round <= kMaxRestart + 2; ++round) {
            IBIM_CUDA(cudaGraphLaunch(R.exec, R.bs));
            count_launch(ctxs[0], 3 + 9 * nmol);
            if (round % 2 == 1 || round == kMaxRestart + 2) {
                for (int i = 0; i < nmol; ++i) IBIM_TRY(gm_fetch_state(ctxs[i]));
                IBIM_CUDA(cudaStreamSynchronize(R.bs));
                bool all = true;
                for (int i = 0; i < nmol; ++i) all = all && (ctxs[i]->gm->h_st->done != 0);
                if (all) break;
            }
        }
        for (int i = 0; i < nmol; ++i) IBIM_TRY(gm_fetch_state(ctxs[i]));
        IBIM_CUDA(cudaStreamSynchronize(R.bs));
        for (int i = 0; i < nmol; ++i) {
            if (finished[i]) continue;
            const int steps = ctxs[i]->gm->h_st->k;
            iters[i] += steps;
            cycles[i] += 1;
            infos[i].matvecs_f32 += steps;
            if (steps > 0) IBIM_TRY(gm_cycle_end(ctxs[i]));
        }
    }
    for (int i = 0; i < nmol; ++i) {
        ibim_ctx* c = ctxs[i];
        infos[i].iters = iters[i];
        infos[i].cycles = cycles[i];
        infos[i].converged = conv[i];
        infos[i].relres = gnorm[i] > 0.0 ? beta[i] / gnorm[i] : 0.0;
        IBIM_CUDA(cudaMemcpyAsync(d_p[i], c->gm->x, sizeof(double) * 2 * c->N, cudaMemcpyDeviceToDevice, R.bs));
        double gpol = 0.0, area = 0.0;
        IBIM_TRY(energy_launch(c, phys[i], c->gm->x, nullptr, &gpol));
        IBIM_TRY(area_launch(c, &area));
        infos[i].gpol = gpol;
        infos[i].gpol_kcal = gpol * kKcalPerE2A;
        infos[i].area = area;
    }
    return IBIM_OK;
}

}  // namespace ibim
