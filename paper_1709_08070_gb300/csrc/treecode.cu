// Treecode form of the FP32 operator: far-field acceleration of the pair sums
// (the role the paper gives to its black-box FMM, Sec. 4), sm_103a.
//
// Every kernel of the operator (Sec. 2.2, discrete system) is linear in the
// source's densities d_j = a_j m_j (a vector) and b_j:
//   K11 a_j = r.d_j (1 - th1 A) / (4 pi rho^3),   K12 b_j = (1 - E) b_j / (4 pi rho),
//   K21 a_j = [(1 - A) n.d_j - (3 - B) s_x r.d_j / rho^2] / (4 pi rho^3),
//   K22 b_j = -s_x (1 - th2 A) b_j / (4 pi rho^3),
// so the sum over a cluster of sources seen from far away is approximated by
// moving the densities onto the 216 proxies of the cluster's bounding cube (6
// Chebyshev points of the second kind per axis): D_k = sum_j L_k(y_j) d_j,
// beta_k = sum_j L_k(y_j) b_j, L_k the tensor-product Lagrange basis.
//
// A proxy tile holds one cluster's proxies in the FP32 source payload format
// (-t, beta, D; 40 zero-density pads at the cube centre), so the list kernel
// streams proxy tiles and ordinary 256-node source tiles through the same
// stage ring and chunk code as the direct kernel: ordinary tiles keep the
// tube rule and the near/far split, proxy tiles always take the far branch.
//
// Tree: clusters are node ranges split as the coordinate bisection of the node
// order splits them (left part B max(1, round(n / 2B)), B = 1024 for n >= 2048,
// 256 otherwise) down to 256-node tiles.  Target tiles: 512 nodes.  A
// cluster C is far from a target tile T when r_T + r_C <= theta D and
// D >= far_dist + r_T + r_C + 0.25 A (D the distance of the box centres, r_T
// the tile box half-diagonal, r_C the cube half-diagonal, far_dist =
// max(2 tau_max, 1.5) 1.001 + 1e-3): no target-proxy distance is below
// far_dist, so no proxy enters the regularisation tube (Sec. 2.2.1, tube
// rule 0).  Lists come from a depth-first traversal from the root.
//
// Target-side interpolation (optional): a far cluster that is also far from
// the target tile's own Chebyshev cube (r_Tc + r_C <= theta D, D >= far_dist +
// r_Tc + r_C + 0.25 A, r_Tc the cube half-diagonal) is evaluated at the tile's
// 216 target proxies instead of its 512 targets (tc_m2l_kernel).  y1 is a
// scalar field of the target position and y2 = n_x . V(x) with
//   V = [g d - (3 - B) (r.d / rho^2) r + (1 - th2 A) b r] / (4 pi rho^3),
// so the fixup interpolates the four fields (y1, V) to each target.
//
// Per operator application: pack the node payload into the tile buffer,
// proxies of the leaves from their nodes (P2M), of each inner cluster from its
// two children's proxies (M2M: exact for this interpolation, the parent's
// basis being a polynomial of degree 5 per axis), level by level; then the
// list kernel (stream-K over the flattened lists, FP64 partial per (CTA,
// target tile)) and the fixup.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pair_f32_core.cuh"

namespace ibim {

// Chebyshev order NC (points per axis, 4, 5 or 6): NC^3 proxies fill the
// first kChunks chunks of a 256-node proxy tile (the rest is padding).
template <int NC>
struct Cheb {
    static constexpr int kProxies = NC * NC * NC;
    static constexpr int kChunks = (kProxies + kChunk - 1) / kChunk;
    static constexpr int kM2lThreads = (kProxies + 31) / 32 * 32;  // one thread per target proxy
};
constexpr int kMaxProxies = Cheb<6>::kProxies;  // stride of the per-tile field buffer
// 512-node target tiles (two targets per thread, 256-thread CTAs, two CTAs
// per SM): measured against 1024-node tiles, the smaller tiles' near regions
// cut the list work by a fifth to a third at the same pair rate.
constexpr int kTcTpt = 2, kTcThreads = 256, kTcMinCtas = 2;
constexpr int kTcTTile = kTcTpt * kTcThreads;  // 512 targets
constexpr double kTcMinHalf = 1e-3;            // smallest proxy-cube half side (A)
constexpr double kTcFarMargin = 0.25;          // extra gap of a far cluster (A)
static_assert(kMaxProxies <= kF32STile, "proxies of a cluster fit one source tile");

struct TcCube {  // proxy cube of a cluster: centre and half side
    double x, y, z, w;
};

struct TcItem {  // m2l work item: entries [e0, e1) of target tile t's interpolated list
    int64_t t, e0, e1;
};

struct TcClusters {  // device arrays, one entry per cluster
    const int64_t* j0;
    const int64_t* j1;
    const int2* child;      // (-1, -1) for a leaf
    const TcCube* cube;    // centre and half side
};

struct TreeCode {
    double theta = 0.0, tau_max = 0.0;
    int order = 6;             // Chebyshev points per axis (4, 5 or 6)
    int64_t n_real_tiles = 0;  // padded N / 256
    int n_clusters = 0;
    int64_t n_t = 0;           // target tiles
    int64_t near_steps = 0, far_steps = 0, total = 0;
    int64_t Lb = 0, Ls = 0, nseg = 0;  // large segments (one per CTA) of Lb steps, then small ones of Ls
    int grid = 0;
    std::vector<int> level_off;  // clusters by height: ids[level_off[h] .. level_off[h + 1])
    int64_t* d_j0 = nullptr;
    int64_t* d_j1 = nullptr;
    int2* d_child = nullptr;
    TcCube* d_cube = nullptr;
    int* d_ids = nullptr;
    float4* d_src = nullptr;       // payload of the real tiles, then one proxy tile per cluster
    float4* d_frm = nullptr;       // chunk frames of all those tiles
    int64_t* d_row_ptr = nullptr;  // n_t + 1
    int32_t* d_step_src = nullptr; // total: source tile of each step
    double* d_part = nullptr;      // (nseg + n_t) x 2 x kTcTTile
    unsigned long long* d_ctr = nullptr;  // [0] list-kernel segments, [1] m2l tiles (reset by the leaf upward launch)
    // target-side interpolation
    int interp = 0;
    int64_t interp_steps = 0, n_items = 0;
    int m2l_grid = 0;
    int64_t* d_irow = nullptr;     // n_t + 1: interpolated far clusters of tile t = isrc[irow[t] .. irow[t + 1])
    int32_t* d_isrc = nullptr;     // their proxy tiles
    TcItem* d_items = nullptr;     // m2l work items
    TcCube* d_tcube = nullptr;     // target proxy cube of each tile
    double* d_fields = nullptr;    // n_t x 216 x (y1, Vx, Vy, Vz) at the target proxies
};

void tc_destroy(TreeCode* t)
{
    if (t == nullptr) return;
    cudaFree(t->d_j0);
    cudaFree(t->d_j1);
    cudaFree(t->d_child);
    cudaFree(t->d_cube);
    cudaFree(t->d_ids);
    cudaFree(t->d_src);
    cudaFree(t->d_frm);
    cudaFree(t->d_row_ptr);
    cudaFree(t->d_step_src);
    cudaFree(t->d_part);
    cudaFree(t->d_ctr);
    cudaFree(t->d_irow);
    cudaFree(t->d_isrc);
    cudaFree(t->d_items);
    cudaFree(t->d_tcube);
    cudaFree(t->d_fields);
    delete t;
}

// ------------------------------------------------------------------ device

// The NC Chebyshev points of the second kind cos(k pi / (NC - 1)) on [-1, 1].
template <int NC>
__device__ __forceinline__ double cheb_point(int k)
{
    static_assert(NC >= 4 && NC <= 6, "Chebyshev order 4, 5 or 6");
    if (NC == 6) {
        const double c1 = 0.8090169943749475, c2 = 0.30901699437494745;  // cos(pi/5), cos(2 pi/5)
        return k == 0 ? 1.0 : k == 1 ? c1 : k == 2 ? c2 : k == 3 ? -c2 : k == 4 ? -c1 : -1.0;
    }
    if (NC == 5) {
        const double c1 = 0.7071067811865476;  // cos(pi/4)
        return k == 0 ? 1.0 : k == 1 ? c1 : k == 2 ? 0.0 : k == 3 ? -c1 : -1.0;
    }
    return k == 0 ? 1.0 : k == 1 ? 0.5 : k == 2 ? -0.5 : -1.0;  // cos(k pi / 3)
}

// Lagrange basis of those points at u in FP32 (barycentric form, weights
// (-1)^k halved at the ends; u on a point gives the unit vector).
template <int NC>
__device__ __forceinline__ void cheb_basis(float u, float (&l)[NC])
{
    float q[NC], s = 0.0f;
    int hit = -1;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float wk = ((k & 1) ? -1.0f : 1.0f) * ((k == 0 || k == NC - 1) ? 0.5f : 1.0f);
        const float d = u - (float)cheb_point<NC>(k);
        if (d == 0.0f) hit = k;
        q[k] = wk / d;
        s += q[k];
    }
    const float rs = 1.0f / s;
#pragma unroll
    for (int k = 0; k < NC; ++k) l[k] = (hit >= 0) ? (k == hit ? 1.0f : 0.0f) : q[k] * rs;
}

// Proxies of the clusters ids[0 .. gridDim.x) (one CTA of kF32STile threads
// each): from the cluster's nodes for a leaf, from its children's proxies
// otherwise; written as the cluster's proxy tile in the source payload format.
template <int NC>
__global__ void __launch_bounds__(kF32STile)
    tc_upward_kernel(TcClusters cl, const int* __restrict__ ids, const double* __restrict__ geo, int64_t N,
                     int64_t n_real_tiles, float4* __restrict__ src, unsigned long long* __restrict__ ctr,
                     const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    if (ctr != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {  // the list and m2l kernels' counters
        ctr[0] = 0ull;
        ctr[1] = 0ull;
    }
    __shared__ float lw[kF32STile][3 * NC];
    __shared__ float4 dens[kF32STile];   // (d.x, d.y, d.z, b) of each source of the pass
    __shared__ float4 outp[kF32STile];   // (rel.x, rel.y, rel.z, b) of each proxy
    __shared__ float4 outd[kF32STile];   // (D.x, D.y, D.z, 0)
    const int tid = threadIdx.x;
    const int ci = ids[blockIdx.x];
    const TcCube cube = cl.cube[ci];
    const double inv = 1.0 / cube.w;
    const int2 ch = cl.child[ci];
    const int kx = tid / (NC * NC), ky = (tid / NC) % NC, kz = tid % NC;
    float ax = 0.0f, ay = 0.0f, az = 0.0f, ab = 0.0f;

    auto accumulate = [&](int count) {
        __syncthreads();
        if (tid < Cheb<NC>::kProxies)
            for (int s = 0; s < count; ++s) {
                const float wgt = lw[s][kx] * lw[s][NC + ky] * lw[s][2 * NC + kz];
                const float4 d = dens[s];
                ax = fmaf(wgt, d.x, ax);
                ay = fmaf(wgt, d.y, ay);
                az = fmaf(wgt, d.z, az);
                ab = fmaf(wgt, d.w, ab);
            }
        __syncthreads();
    };
    auto set_source = [&](double x, double y, double z, float4 d) {
        float l[NC];
        cheb_basis<NC>((float)((x - cube.x) * inv), l);
#pragma unroll
        for (int k = 0; k < NC; ++k) lw[tid][k] = l[k];
        cheb_basis<NC>((float)((y - cube.y) * inv), l);
#pragma unroll
        for (int k = 0; k < NC; ++k) lw[tid][NC + k] = l[k];
        cheb_basis<NC>((float)((z - cube.z) * inv), l);
#pragma unroll
        for (int k = 0; k < NC; ++k) lw[tid][2 * NC + k] = l[k];
        dens[tid] = d;
    };

    if (ch.x < 0) {  // leaf: its nodes (payload densities of this application)
        const int64_t j0 = cl.j0[ci], j1 = cl.j1[ci];
        for (int64_t base = j0; base < j1; base += kF32STile) {
            const int64_t j = base + tid;
            if (j < j1) {
                const float4* pr = src + kPairF4 * (j >> 1);
                const float4 B = pr[1], C = pr[2], D = pr[3];
                const bool odd = j & 1;
                const float4 d = odd ? make_float4(C.y, C.w, D.y, B.w) : make_float4(C.x, C.z, D.x, B.z);
                set_source(geo[j], geo[N + j], geo[2 * N + j], d);
            } else {
                set_source(cube.x, cube.y, cube.z, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            }
            const int64_t left = j1 - base;
            accumulate(left < kF32STile ? (int)left : kF32STile);
        }
    } else {  // inner cluster: the proxies of its two children
        for (int side = 0; side < 2; ++side) {
            const int cc = side ? ch.y : ch.x;
            const TcCube cb = cl.cube[cc];
            if (tid < Cheb<NC>::kProxies) {
                const int qx = tid / (NC * NC), qy = (tid / NC) % NC, qz = tid % NC;
                const float4* pr = src + (n_real_tiles + cc) * (kF32STile / 2) * kPairF4 + kPairF4 * (tid >> 1);
                const float4 B = pr[1], C = pr[2], D = pr[3];
                const bool odd = tid & 1;
                const float4 d = odd ? make_float4(C.y, C.w, D.y, B.w) : make_float4(C.x, C.z, D.x, B.z);
                set_source(cb.x + cb.w * cheb_point<NC>(qx), cb.y + cb.w * cheb_point<NC>(qy), cb.z + cb.w * cheb_point<NC>(qz), d);
            }
            accumulate(Cheb<NC>::kProxies);
        }
    }

    // proxy tile: positions relative to the cube centre (the tile's chunk frame)
    if (tid < Cheb<NC>::kProxies) {
        outp[tid] = make_float4((float)(cube.w * cheb_point<NC>(kx)), (float)(cube.w * cheb_point<NC>(ky)),
                                (float)(cube.w * cheb_point<NC>(kz)), ab);
        outd[tid] = make_float4(ax, ay, az, 0.0f);
    } else {
        outp[tid] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        outd[tid] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    if (tid < kF32STile / 2) {
        const float4 p0 = outp[2 * tid], p1 = outp[2 * tid + 1];
        const float4 d0 = outd[2 * tid], d1 = outd[2 * tid + 1];
        float4* dst = src + (n_real_tiles + ci) * (kF32STile / 2) * kPairF4 + kPairF4 * tid;
        dst[0] = make_float4(-p0.x, -p1.x, -p0.y, -p1.y);
        dst[1] = make_float4(-p0.z, -p1.z, p0.w, p1.w);
        dst[2] = make_float4(d0.x, d1.x, d0.y, d1.y);
        dst[3] = make_float4(d0.z, d1.z, 0.0f, 0.0f);
    }
}

struct TcSchedule {
    const int64_t* row_ptr;   // n_t + 1, row t = steps [row_ptr[t], row_ptr[t + 1])
    const int32_t* step_src;  // source tile of each step (>= n_real_tiles: a proxy tile)
    int64_t n_t, total, n_real_tiles;
    int64_t Lb, nbig, Ls, nseg;  // segments: nbig of Lb steps, then small ones of Ls steps
    int proxy_chunks;            // chunks of a proxy tile that hold proxies
};

// First step of segment q (total for q = nseg) and the segment of step u.
__host__ __device__ __forceinline__ int64_t tc_seg_start(const TcSchedule& s, int64_t q)
{
    const int64_t v = q < s.nbig ? q * s.Lb : s.nbig * s.Lb + (q - s.nbig) * s.Ls;
    return v < s.total ? v : s.total;
}
__host__ __device__ __forceinline__ int64_t tc_seg_of(const TcSchedule& s, int64_t u)
{
    const int64_t big = s.nbig * s.Lb;
    return u < big ? u / s.Lb : s.nbig + (u - big) / s.Ls;
}

// The FP32 pair sums over the interaction lists: as pair_f32_kernel, with the
// (target tile, source tile) of each step read from the lists.  The step
// sequence is cut into one large segment per CTA (9/10 of an even share)
// and small segments handed out by a counter, so that CTAs whose steps were
// cheaper (far steps skip the tube tests) take more of the rest.  Partials:
// one per (segment, target tile), slot = segment + tile.
template <int TPT, int MINB, int THREADS>
__global__ void __launch_bounds__(THREADS, MINB)
    tc_pair_kernel(const float4* __restrict__ tpos, const float4* __restrict__ tnrm, const float4* __restrict__ src,
                   const float4* __restrict__ frames, int64_t N, TcSchedule s, F32Consts k,
                   double* __restrict__ part, unsigned long long* __restrict__ ctr, unsigned* __restrict__ err,
                   const int* __restrict__ skip, Geo64 g64)
{
    constexpr int TTILE = THREADS * TPT;
    constexpr int NW = THREADS / 32;
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(16) float4 tfrm[NW][2 * TPT];
    __shared__ __align__(8) StagePipe pipe;
    __shared__ int64_t seg_next[2];
    __shared__ int abort_sh;  // a bounded wait gave up: every warp leaves after the segment barrier

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    if (tid == 0) {
        pipe_init(pipe, NW);
        abort_sh = 0;
    }
    __syncthreads();

    // ring position of step u of the current segment: done + (u - s0) = u + off
    int64_t s0 = 0, s1 = 0, off = 0, done = 0;
    auto issue = [&](int64_t u) {
        const int64_t st = s.step_src[u];
        const int stage = (int)((u + off) % kF32Stages);
        pipe_issue(pipe, stg[stage], stage, src + st * (kF32STile / 2) * kPairF4, frames + st * 2 * kChunksPerTile);
    };
    auto give_up = [&]() {
        if (lane == 0) {
            atomicOr(err, kDevErrTimeout);
            *(volatile int*)&abort_sh = 1;
        }
    };

    int64_t t = 0, row_end = 0;
    Targets<TPT> T;
    int64_t gi0 = 0;
    bool idle = false;
    double D1[TPT], D2[TPT];

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
        if (lane < 2 * TPT) {
            const int64_t blk0 = tile * TTILE + (int64_t)(lane >> 1) * THREADS + warp * 32;
            tfrm[warp][lane] = frames[2 * (blk0 / kChunk) + (lane & 1)];
        }
        __syncwarp();
    };

    int64_t seg = blockIdx.x;
    int sp = 0;
    while (seg < s.nseg) {
        s0 = tc_seg_start(s, seg);
        s1 = tc_seg_start(s, seg + 1);
        off = done - s0;
        // every stage is free here: thread 0 waited for each earlier step's release
        if (tid == 0) {
            ptx::fence_proxy_async_smem();
            for (int q = 0; q < kF32Stages && s0 + q < s1; ++q) issue(s0 + q);
        }
        // the row holding step s0: the last t with row_ptr[t] <= s0
        int64_t lo = 0, hi = s.n_t;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (s.row_ptr[mid] <= s0) lo = mid;
            else hi = mid;
        }
        t = lo;
        row_end = s.row_ptr[t + 1];
        load_targets(t);

        bool bad = false;
        for (int64_t u = s0; u < s1; ++u) {
            const int stage = (int)((u + off) % kF32Stages);
            const uint32_t parity = (uint32_t)(((u + off) / kF32Stages) & 1);
            if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
                give_up();
                bad = true;
                break;
            }
            const int64_t st = s.step_src[u];
            float S1[TPT], C1[TPT], S2[TPT], C2[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) S1[q] = C1[q] = S2[q] = C2[q] = 0.0f;
            if (!idle)
                tile_sums<TPT, true>(T, &tfrm[warp][0], true, stg[stage].buf, stg[stage].frm, k, S1, C1, S2, C2,
                                     g64, gi0, THREADS, st * kF32STile, N, st >= s.n_real_tiles,
                                     st >= s.n_real_tiles ? s.proxy_chunks : kChunksPerTile);
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                D1[q] += (double)S1[q] - (double)C1[q];
                D2[q] += (double)S2[q] - (double)C2[q];
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
            if (warp == 0) {  // thread 0 refills the stage of step u - 1
                bool ok = true;
                if (lane == 0 && u > s0 && u - 1 + kF32Stages < s1) {
                    const int64_t v = u - 1 + off;
                    ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(v % kF32Stages)], (uint32_t)((v / kF32Stages) & 1),
                                                kWaitLimitNs);
                    if (ok) {
                        ptx::fence_proxy_async_smem();
                        issue(u - 1 + kF32Stages);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    give_up();
                    bad = true;
                    break;
                }
            }

            if (u + 1 == row_end || u + 1 == s1) {
                double* dst = part + (seg + t) * 2 * TTILE;
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    dst[q * THREADS + tid] = D1[q];
                    dst[TTILE + q * THREADS + tid] = D2[q];
                }
                if (u + 1 < s1) {  // rows are never empty: the next step starts row t + 1
                    ++t;
                    row_end = s.row_ptr[t + 1];
                    load_targets(t);
                }
            }
        }
        // before the next segment reuses the stages: every step of this one released
        if (warp == 0) {
            bool ok = !bad;
            if (ok && lane == 0) {
                const int64_t first = (s1 - s0 > kF32Stages) ? s1 - kF32Stages : s0;
                for (int64_t v = first; v < s1 && ok; ++v) {
                    const int64_t w = v + off;
                    ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(w % kF32Stages)], (uint32_t)((w / kF32Stages) & 1),
                                                kWaitLimitNs);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok && !bad) give_up();
            if (lane == 0) seg_next[sp] = ok ? s.nbig + (int64_t)atomicAdd(ctr, 1ull) : s.nseg;
        }
        done += s1 - s0;
        __syncthreads();
        if (*(volatile int*)&abort_sh) return;
        seg = seg_next[sp];
        sp ^= 1;
    }
}

// The fields at target proxies of one packed pair of source proxies (the two
// lanes of each float2): y1 as in pair_far2, and V with y2 = n_x . V.
__device__ __forceinline__ void pair_field2(float2 Xx, float2 Xy, float2 Xz, const float4& A, const float4& B,
                                            const float4& C, const float4& D, const FarConsts& c, float2& f1,
                                            float2& vx, float2& vy, float2& vz)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 b = make_float2(B.z, B.w);
    const float2 dx = make_float2(C.x, C.y), dy = make_float2(C.z, C.w), dz = make_float2(D.x, D.y);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sd = __fmul2_rn(rx, dx);
    sd = __ffma2_rn(ry, dy, sd);
    sd = __ffma2_rn(rz, dz, sd);
    const float2 inv = make_float2(ptx::rsqrt_approx(rr.x), ptx::rsqrt_approx(rr.y));
    const float2 rho = __fmul2_rn(rr, inv);
    const float2 ea = __fmul2_rn(rho, c.kl2e);
    const float2 xn = __fmul2_rn(rho, c.nkappa);
    const float2 E = make_float2(ptx::ex2_approx(ea.x), ptx::ex2_approx(ea.y));
    const float2 En = __fmul2_rn(E, xn);
    const float2 fn = __fadd2_rn(E, c.neg1);               // -(1 - E)
    const float2 g = __ffma2_rn(fn, c.neg1, En);           // 1 - A
    const float2 hn = __ffma2_rn(g, c.neg3, __fmul2_rn(En, xn));  // -(3 - B)
    const float2 inv2 = __fmul2_rn(inv, inv);
    const float2 P = __fmul2_rn(inv2, inv);
    const float2 u1 = __ffma2_rn(c.th1, g, c.omth1);
    const float2 u2 = __ffma2_rn(c.th2, g, c.omth2);
    f1 = __ffma2_rn(P, __fmul2_rn(u1, sd), f1);
    f1 = __ffma2_rn(__fmul2_rn(fn, inv), b, f1);
    const float2 v = __ffma2_rn(__fmul2_rn(hn, inv2), sd, __fmul2_rn(u2, b));
    const float2 Pg = __fmul2_rn(P, g), Pv = __fmul2_rn(P, v);
    vx = __ffma2_rn(Pg, dx, __ffma2_rn(Pv, rx, vx));
    vy = __ffma2_rn(Pg, dy, __ffma2_rn(Pv, ry, vy));
    vz = __ffma2_rn(Pg, dz, __ffma2_rn(Pv, rz, vz));
}

struct TcM2l {
    const int64_t* irow;      // n_t + 1
    const int32_t* isrc;      // proxy tile of each entry
    const TcItem* items;      // work items
    const TcCube* tcube;      // target proxy cube per tile
    int64_t n_items;
};

// Fields at the target proxies of each target tile from the proxy tiles of
// its interpolated far clusters.  Work items are runs of at least 8 entries of
// one tile's list: CTA b takes item b and then items from the counter; the
// source proxy tiles stream through the stage ring as in the list kernel
// (ring position continued across items), and each item adds its fields to
// the tile's (zeroed before the launch) with FP64 atomics.
template <int NC>
__global__ void __launch_bounds__(Cheb<NC>::kM2lThreads)
    tc_m2l_kernel(const float4* __restrict__ src, const float4* __restrict__ frames, TcM2l m, F32Consts k,
                  double* __restrict__ fields, unsigned long long* __restrict__ ctr, unsigned* __restrict__ err,
                  const int* __restrict__ skip)
{
    constexpr int NW = Cheb<NC>::kM2lThreads / 32;
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) SourceStage stg[kF32Stages];
    __shared__ __align__(8) StagePipe pipe;
    __shared__ int64_t tile_next[2];
    __shared__ int abort_sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const bool active = tid < Cheb<NC>::kProxies;
    const int lx = tid / (NC * NC), ly = (tid / NC) % NC, lz = tid % NC;
    if (tid == 0) {
        pipe_init(pipe, NW);
        abort_sh = 0;
    }
    __syncthreads();
    const FarConsts fc = far_consts(k);
    int64_t done = 0, off = 0, e1 = 0;
    auto issue = [&](int64_t u) {
        const int64_t st = m.isrc[u];
        const int stage = (int)((u + off) % kF32Stages);
        pipe_issue(pipe, stg[stage], stage, src + st * (kF32STile / 2) * kPairF4, frames + st * 2 * kChunksPerTile);
    };
    auto give_up = [&]() {
        if (lane == 0) {
            atomicOr(err, kDevErrTimeout);
            *(volatile int*)&abort_sh = 1;
        }
    };

    int64_t q = blockIdx.x;
    int sp = 0;
    while (q < m.n_items) {
        const TcItem item = m.items[q];
        const int64_t t = item.t;
        const int64_t e0 = item.e0;
        e1 = item.e1;
        off = done - e0;
        if (tid == 0) {
            ptx::fence_proxy_async_smem();
            for (int r = 0; r < kF32Stages && e0 + r < e1; ++r) issue(e0 + r);
        }
        const TcCube cube = m.tcube[t];
        // target proxy relative to the cube centre; the centre as hi + lo floats
        const float3 X0 = make_float3((float)(cube.w * cheb_point<NC>(lx)), (float)(cube.w * cheb_point<NC>(ly)),
                                      (float)(cube.w * cheb_point<NC>(lz)));
        const float hx = (float)cube.x, hy = (float)cube.y, hz = (float)cube.z;
        const float3 lo = make_float3((float)(cube.x - (double)hx), (float)(cube.y - (double)hy),
                                      (float)(cube.z - (double)hz));
        double F1 = 0.0, FX = 0.0, FY = 0.0, FZ = 0.0;
        bool bad = false;
        for (int64_t u = e0; u < e1; ++u) {
            const int stage = (int)((u + off) % kF32Stages);
            const uint32_t parity = (uint32_t)(((u + off) / kF32Stages) & 1);
            if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&pipe.full[stage], parity, kWaitLimitNs))) {
                give_up();
                bad = true;
                break;
            }
            if (active) {
                const float4 mh = stg[stage].frm[0], ml = stg[stage].frm[1];  // one frame for the whole proxy tile
                const float2 Xx = f2(X0.x + ((hx - mh.x) + (lo.x - ml.x)));
                const float2 Xy = f2(X0.y + ((hy - mh.y) + (lo.y - ml.y)));
                const float2 Xz = f2(X0.z + ((hz - mh.z) + (lo.z - ml.z)));
                float2 f1 = make_float2(0.0f, 0.0f), vx = f1, vy = f1, vz = f1;
                const float4* cb = stg[stage].buf;
#pragma unroll 4
                for (int pr = 0; pr < Cheb<NC>::kChunks * kPairsPerChunk; ++pr) {
                    const float4 A = cb[kPairF4 * pr], B = cb[kPairF4 * pr + 1];
                    const float4 C = cb[kPairF4 * pr + 2], D = cb[kPairF4 * pr + 3];
                    pair_field2(Xx, Xy, Xz, A, B, C, D, fc, f1, vx, vy, vz);
                }
                F1 += (double)f1.x + (double)f1.y;
                FX += (double)vx.x + (double)vx.y;
                FY += (double)vy.x + (double)vy.y;
                FZ += (double)vz.x + (double)vz.y;
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&pipe.empty[stage]);
            if (warp == 0) {  // thread 0 refills the stage of step u - 1
                bool ok = true;
                if (lane == 0 && u > e0 && u - 1 + kF32Stages < e1) {
                    const int64_t v = u - 1 + off;
                    ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(v % kF32Stages)], (uint32_t)((v / kF32Stages) & 1),
                                                kWaitLimitNs);
                    if (ok) {
                        ptx::fence_proxy_async_smem();
                        issue(u - 1 + kF32Stages);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    give_up();
                    bad = true;
                    break;
                }
            }
        }
        if (active && !bad) {
            double* f = fields + (t * kMaxProxies + tid) * 4;
            atomicAdd(f, F1);
            atomicAdd(f + 1, FX);
            atomicAdd(f + 2, FY);
            atomicAdd(f + 3, FZ);
        }
        if (warp == 0) {  // every step of this tile released before the stages are reused
            bool ok = !bad;
            if (ok && lane == 0) {
                const int64_t first = (e1 - e0 > kF32Stages) ? e1 - kF32Stages : e0;
                for (int64_t v = first; v < e1 && ok; ++v) {
                    const int64_t w = v + off;
                    ok = ptx::mbar_wait_bounded(&pipe.empty[(int)(w % kF32Stages)], (uint32_t)((w / kF32Stages) & 1),
                                                kWaitLimitNs);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok && !bad) give_up();
            if (lane == 0) tile_next[sp] = ok ? (int64_t)gridDim.x + (int64_t)atomicAdd(ctr, 1ull) : m.n_items;
        }
        done += e1 - e0;
        __syncthreads();
        if (*(volatile int*)&abort_sh) return;
        q = tile_next[sp];
        sp ^= 1;
    }
}

// y = Lambda p + (1/(4 pi)) (partials of the segments that covered the row
// + the interpolated far fields of the row's target proxies, when it has any).
// One 256-thread block lies inside one target tile.
template <int NC>
__global__ void __launch_bounds__(256)
    tc_fixup_kernel(const double* __restrict__ part, TcSchedule s, int64_t N, double lambda1, double lambda2,
                    VecRef in, OutRef out, TcM2l m, const double* __restrict__ fields,
                    const double* __restrict__ geo, int interp, const int* __restrict__ skip)
{
    static_assert(kTcTTile % 256 == 0, "a fixup block lies in one target tile");
    if (skip != nullptr && *skip) return;
    constexpr int NP = Cheb<NC>::kProxies;
    __shared__ float fl[NP][4];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x) / kTcTTile;
    const bool has = interp && m.irow[t + 1] > m.irow[t];
    if (has)
        for (int q = threadIdx.x; q < NP * 4; q += blockDim.x) (&fl[0][0])[q] = (float)fields[t * kMaxProxies * 4 + q];
    __syncthreads();
    if (i >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    double* y = out.base + (out.kidx ? (int64_t)(*out.kidx + out.koff) * out.stride : 0);
    const int64_t l = i - t * kTcTTile;
    const int64_t c0 = tc_seg_of(s, s.row_ptr[t]);
    const int64_t c1 = tc_seg_of(s, s.row_ptr[t + 1] - 1);
    double a1 = 0.0, a2 = 0.0;
    for (int64_t c = c0; c <= c1; ++c) {
        const double* q = part + (c + t) * 2 * kTcTTile;
        a1 += q[l];
        a2 += q[kTcTTile + l];
    }
    if (has) {  // L2P: the tile's fields at this target
        const TcCube cube = m.tcube[t];
        const double inv = 1.0 / cube.w;
        float wx[NC], wy[NC], wz[NC];
        cheb_basis<NC>((float)((geo[i] - cube.x) * inv), wx);
        cheb_basis<NC>((float)((geo[N + i] - cube.y) * inv), wy);
        cheb_basis<NC>((float)((geo[2 * N + i] - cube.z) * inv), wz);
        float F1 = 0.0f, FX = 0.0f, FY = 0.0f, FZ = 0.0f;
        for (int ax = 0; ax < NC; ++ax)
            for (int ay = 0; ay < NC; ++ay) {
                const float wxy = wx[ax] * wy[ay];
#pragma unroll
                for (int az = 0; az < NC; ++az) {
                    const float wgt = wxy * wz[az];
                    const float* f = fl[(ax * NC + ay) * NC + az];
                    F1 = fmaf(wgt, f[0], F1);
                    FX = fmaf(wgt, f[1], FX);
                    FY = fmaf(wgt, f[2], FY);
                    FZ = fmaf(wgt, f[3], FZ);
                }
            }
        a1 += (double)F1;
        a2 += geo[3 * N + i] * (double)FX + geo[4 * N + i] * (double)FY + geo[5 * N + i] * (double)FZ;
    }
    y[i] = lambda1 * p[i] + kInv4Pi * a1;
    y[N + i] = lambda2 * p[N + i] + kInv4Pi * a2;
}

// ------------------------------------------------------------------ host

static ibim_status tc_fail(ibim_status s, const char* msg)
{
    set_error(msg);
    return s;
}

namespace {

struct HostCluster {
    int64_t j0, j1;
    int c0 = -1, c1 = -1;
    int height = 0;
    double cx, cy, cz, half, radius;
};

int64_t tc_split_point(int64_t n)
{
    const int64_t B = n >= 2048 ? 1024 : 256;
    const int64_t half = std::max<int64_t>(1, (int64_t)std::floor((double)n / (2.0 * (double)B) + 0.5));
    return B * half;
}

void box_of(const std::vector<double>& xs, int64_t N, int64_t j0, int64_t j1, double mn[3], double mx[3])
{
    for (int a = 0; a < 3; ++a) {
        mn[a] = HUGE_VAL;
        mx[a] = -HUGE_VAL;
    }
    for (int64_t j = j0; j < j1; ++j)
        for (int a = 0; a < 3; ++a) {
            const double v = xs[a * N + j];
            mn[a] = std::min(mn[a], v);
            mx[a] = std::max(mx[a], v);
        }
}

// Cluster of nodes [j0, j1) and its subtree (pre-order indices).  Its proxy
// cube bounds its nodes and its children's cubes, so M2M never evaluates a
// parent's basis outside its cube.
int make_cluster(std::vector<HostCluster>& cl, const std::vector<double>& xs, int64_t N, int64_t j0, int64_t j1)
{
    const int idx = (int)cl.size();
    cl.emplace_back();
    HostCluster c;
    c.j0 = j0;
    c.j1 = j1;
    if (j1 - j0 > kF32STile) {
        const int64_t k = tc_split_point(j1 - j0);
        c.c0 = make_cluster(cl, xs, N, j0, j0 + k);
        c.c1 = make_cluster(cl, xs, N, j0 + k, j1);
        c.height = 1 + std::max(cl[c.c0].height, cl[c.c1].height);
    }
    double mn[3], mx[3];
    box_of(xs, N, j0, j1, mn, mx);
    for (int side = 0; side < 2 && c.c0 >= 0; ++side) {
        const HostCluster& q = cl[side ? c.c1 : c.c0];
        const double qc[3] = {q.cx, q.cy, q.cz};
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], qc[a] - q.half);
            mx[a] = std::max(mx[a], qc[a] + q.half);
        }
    }
    c.cx = 0.5 * (mn[0] + mx[0]);
    c.cy = 0.5 * (mn[1] + mx[1]);
    c.cz = 0.5 * (mn[2] + mx[2]);
    const double e0 = 0.5 * (mx[0] - mn[0]), e1 = 0.5 * (mx[1] - mn[1]), e2 = 0.5 * (mx[2] - mn[2]);
    c.half = std::max(std::max(std::max(e0, e1), e2), kTcMinHalf);
    c.radius = std::sqrt(3.0 * c.half * c.half);
    cl[idx] = c;
    return idx;
}

template <class T>
ibim_status upload(T** dst, const std::vector<T>& v)
{
    IBIM_CUDA(cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) IBIM_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return IBIM_OK;
}

}  // namespace

template <int NC>
static int m2l_occupancy()
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_m2l_kernel<NC>, Cheb<NC>::kM2lThreads, 0);
    return occ < 1 ? 1 : occ;
}

// Tree, target tiles and interaction lists of N nodes (coordinates SoA:
// x[0..N), y[N..2N), z[2N..3N)); host only.
struct TcPlan {
    std::vector<HostCluster> cl;
    int64_t n_t = 0, n_real = 0;
    std::vector<double> tcx, tcy, tcz, thalf;
    std::vector<int64_t> row_ptr, irow;
    std::vector<int32_t> steps, isrc;
    int64_t near_steps = 0, far_steps = 0;
};

TcPlan tc_plan(const std::vector<double>& xs, int64_t N, double theta, double tau_max, int interp)
{
    TcPlan P;
    std::vector<HostCluster>& cl = P.cl;
    cl.reserve((size_t)(2 * (N / kF32STile) + 4));
    make_cluster(cl, xs, N, 0, N);

    // target tiles
    const int64_t n_t = (N + kTcTTile - 1) / kTcTTile;
    P.n_t = n_t;
    P.tcx.resize(n_t);
    P.tcy.resize(n_t);
    P.tcz.resize(n_t);
    P.thalf.resize(n_t);
    std::vector<double> trad(n_t), tcrad(n_t);
    for (int64_t t = 0; t < n_t; ++t) {
        double mn[3], mx[3];
        box_of(xs, N, t * kTcTTile, std::min<int64_t>((t + 1) * kTcTTile, N), mn, mx);
        P.tcx[t] = 0.5 * (mn[0] + mx[0]);
        P.tcy[t] = 0.5 * (mn[1] + mx[1]);
        P.tcz[t] = 0.5 * (mn[2] + mx[2]);
        const double e0 = 0.5 * (mx[0] - mn[0]), e1 = 0.5 * (mx[1] - mn[1]), e2 = 0.5 * (mx[2] - mn[2]);
        trad[t] = std::sqrt((e0 * e0 + e1 * e1) + e2 * e2);
        P.thalf[t] = std::max(std::max(std::max(e0, e1), e2), kTcMinHalf);  // target proxy cube
        tcrad[t] = std::sqrt(3.0 * P.thalf[t] * P.thalf[t]);
    }

    // lists, depth-first from the root
    const int64_t n_real = padded_nodes(N) / kF32STile;
    P.n_real = n_real;
    const double fd = std::max(2.0 * tau_max, 1.5) * 1.001 + 1e-3;
    P.row_ptr.assign(n_t + 1, 0);
    P.irow.assign(n_t + 1, 0);
    std::vector<int> stack;
    for (int64_t t = 0; t < n_t; ++t) {
        stack.assign(1, 0);
        while (!stack.empty()) {
            const int ci = stack.back();
            stack.pop_back();
            const HostCluster& q = cl[ci];
            const double dx = P.tcx[t] - q.cx, dy = P.tcy[t] - q.cy, dz = P.tcz[t] - q.cz;
            const double D = std::sqrt((dx * dx + dy * dy) + dz * dz);
            const double rT = trad[t];
            const bool far = (rT + q.radius <= theta * D) && (D >= fd + rT + q.radius + kTcFarMargin);
            const double rTc = tcrad[t];
            const bool fint =
                far && interp && (rTc + q.radius <= theta * D) && (D >= fd + rTc + q.radius + kTcFarMargin);
            if (fint) {
                P.isrc.push_back((int32_t)(n_real + ci));
            } else if (far) {
                P.steps.push_back((int32_t)(n_real + ci));
                ++P.far_steps;
            } else if (q.c0 < 0) {
                P.steps.push_back((int32_t)(q.j0 / kF32STile));
                ++P.near_steps;
            } else {
                stack.push_back(q.c1);
                stack.push_back(q.c0);
            }
        }
        P.row_ptr[t + 1] = (int64_t)P.steps.size();
        P.irow[t + 1] = (int64_t)P.isrc.size();
    }
    return P;
}

ibim_status tc_setup(ibim_ctx* c, double theta, double tau_max, int order, int interp)
{
    const int64_t N = c->N;
    std::vector<double> xs(3 * (size_t)N);
    IBIM_CUDA(cudaMemcpyAsync(xs.data(), c->d_geo64, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    TcPlan P = tc_plan(xs, N, theta, tau_max, interp);
    const std::vector<HostCluster>& cl = P.cl;
    const int nc = (int)cl.size();
    const int64_t n_t = P.n_t, n_real = P.n_real;
    const std::vector<double>&tcx = P.tcx, &tcy = P.tcy, &tcz = P.tcz, &thalf = P.thalf;
    const std::vector<int64_t>&row_ptr = P.row_ptr, &irow = P.irow;
    const std::vector<int32_t>&steps = P.steps, &isrc = P.isrc;
    const int64_t near_steps = P.near_steps, far_steps = P.far_steps;
    if (n_real + nc > INT32_MAX) return tc_fail(IBIM_ERR_ARG, "treecode: too many tiles");

    // clusters by height (leaves first) for the upward pass
    int hmax = 0;
    for (const HostCluster& q : cl) hmax = std::max(hmax, q.height);
    std::vector<int> ids;
    std::vector<int> level_off(1, 0);
    for (int h = 0; h <= hmax; ++h) {
        for (int i = 0; i < nc; ++i)
            if (cl[i].height == h) ids.push_back(i);
        level_off.push_back((int)ids.size());
    }

    // proxy frames: every chunk of a proxy tile has the cube centre (hi + lo) and radius
    std::vector<float4> pfrm((size_t)nc * 2 * kChunksPerTile);
    for (int i = 0; i < nc; ++i) {
        const float hx = (float)cl[i].cx, hy = (float)cl[i].cy, hz = (float)cl[i].cz;
        const float4 f0 = make_float4(hx, hy, hz, (float)(cl[i].radius * 1.0001 + 1e-4));
        const float4 f1 = make_float4((float)(cl[i].cx - (double)hx), (float)(cl[i].cy - (double)hy),
                                      (float)(cl[i].cz - (double)hz), 0.0f);
        for (int ch = 0; ch < kChunksPerTile; ++ch) {
            pfrm[(size_t)i * 2 * kChunksPerTile + 2 * ch] = f0;
            pfrm[(size_t)i * 2 * kChunksPerTile + 2 * ch + 1] = f1;
        }
    }
    std::vector<TcCube> tcube(n_t);
    for (int64_t t = 0; t < n_t; ++t) tcube[t] = TcCube{tcx[t], tcy[t], tcz[t], thalf[t]};
    std::vector<int64_t> hj0(nc), hj1(nc);
    std::vector<int2> hch(nc);
    std::vector<TcCube> hcube(nc);
    for (int i = 0; i < nc; ++i) {
        hj0[i] = cl[i].j0;
        hj1[i] = cl[i].j1;
        hch[i] = make_int2(cl[i].c0, cl[i].c1);
        hcube[i] = TcCube{cl[i].cx, cl[i].cy, cl[i].cz, cl[i].half};
    }

    TreeCode* T = new TreeCode();
    T->theta = theta;
    T->tau_max = tau_max;
    T->order = order;
    T->n_real_tiles = n_real;
    T->n_clusters = nc;
    T->n_t = n_t;
    T->near_steps = near_steps;
    T->far_steps = far_steps;
    T->total = (int64_t)steps.size();
    T->level_off = level_off;
    T->interp = interp ? 1 : 0;
    T->interp_steps = (int64_t)isrc.size();
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_pair_kernel<kTcTpt, kTcMinCtas, kTcThreads>, kTcThreads, 0);
    const int64_t cap = (int64_t)std::max(1, occ) * c->num_sms;
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>(cap, T->total));
    T->Lb = std::max<int64_t>(1, (9 * T->total) / (10 * g));  // g Lb <= total as g <= total
    const int64_t rest = T->total - g * T->Lb;
    T->Ls = std::max<int64_t>(1, (rest + 16 * g - 1) / (16 * g));
    T->nseg = g + (rest + T->Ls - 1) / T->Ls;
    T->grid = (int)g;
    // m2l work items: runs of at least 8 entries of one tile's list, about
    // four per resident CTA
    const int occm = order == 4 ? m2l_occupancy<4>() : order == 5 ? m2l_occupancy<5>() : m2l_occupancy<6>();
    const int64_t slots = (int64_t)occm * c->num_sms;
    const int64_t run = std::max<int64_t>(8, (T->interp_steps + 4 * slots - 1) / (4 * slots));
    std::vector<TcItem> items;
    for (int64_t t = 0; t < n_t; ++t)
        for (int64_t e = irow[t]; e < irow[t + 1]; e += run)
            items.push_back(TcItem{t, e, std::min(e + run, irow[t + 1])});
    T->n_items = (int64_t)items.size();
    T->m2l_grid = (int)std::max<int64_t>(1, std::min<int64_t>(slots, T->n_items));

    ibim_status st = IBIM_OK;
    auto chk = [&](ibim_status s) {
        if (st == IBIM_OK) st = s;
    };
    chk(upload(&T->d_j0, hj0));
    chk(upload(&T->d_j1, hj1));
    chk(upload(&T->d_child, hch));
    chk(upload(&T->d_cube, hcube));
    chk(upload(&T->d_ids, ids));
    chk(upload(&T->d_row_ptr, row_ptr));
    chk(upload(&T->d_step_src, steps));
    if (T->interp) {
        chk(upload(&T->d_irow, irow));
        chk(upload(&T->d_isrc, isrc));
        chk(upload(&T->d_items, items));
        chk(upload(&T->d_tcube, tcube));
    }
    const size_t frm_real = (size_t)n_real * 2 * kChunksPerTile;
    if (st == IBIM_OK) {
        cudaError_t e = cudaMalloc((void**)&T->d_src, sizeof(float4) * (size_t)(n_real + nc) * (kF32STile / 2) * kPairF4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&T->d_frm, sizeof(float4) * (frm_real + pfrm.size()));
        if (e == cudaSuccess)
            e = cudaMalloc((void**)&T->d_part, sizeof(double) * (size_t)(T->nseg + n_t) * 2 * kTcTTile);
        if (e == cudaSuccess) e = cudaMalloc((void**)&T->d_ctr, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess && T->interp)
            e = cudaMalloc((void**)&T->d_fields, sizeof(double) * (size_t)n_t * kMaxProxies * 4);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T->d_frm, c->d_frames, sizeof(float4) * frm_real, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T->d_frm + frm_real, pfrm.data(), sizeof(float4) * pfrm.size(), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = tc_fail(IBIM_ERR_CUDA, cudaGetErrorString(e));
    }
    if (st != IBIM_OK) {
        tc_destroy(T);
        return st;
    }
    tc_destroy(c->tc);
    c->tc = T;
    c->ws_generation += 1;  // graphs captured with another tree must be re-captured
    return IBIM_OK;
}

template <int NC>
static ibim_status tc_apply_order(ibim_ctx* c, TreeCode* T, const PairConsts& k, VecRef in, OutRef out,
                                  const int* d_skip)
{
    const int64_t N = c->N;
    IBIM_TRY(f32_pack_to(c, in, T->d_src, d_skip));
    const TcClusters cl{T->d_j0, T->d_j1, T->d_child, T->d_cube};
    for (size_t h = 0; h + 1 < T->level_off.size(); ++h) {
        const int n = T->level_off[h + 1] - T->level_off[h];
        if (n == 0) continue;
        tc_upward_kernel<NC><<<n, kF32STile, 0, c->stream>>>(cl, T->d_ids + T->level_off[h], c->d_geo64, N,
                                                             T->n_real_tiles, T->d_src, h == 0 ? T->d_ctr : nullptr,
                                                             d_skip);
        count_launch(c);
        IBIM_CUDA(cudaGetLastError());
    }
    const TcSchedule s{T->d_row_ptr, T->d_step_src, T->n_t, T->total, T->n_real_tiles,
                       T->Lb, (int64_t)T->grid, T->Ls, T->nseg, Cheb<NC>::kChunks};
    const Geo64 g64{c->d_geo64, c->d_geo64 + 3 * N, 1, N};
    IBIM_TRY(timing_begin(c));
    tc_pair_kernel<kTcTpt, kTcMinCtas, kTcThreads><<<T->grid, kTcThreads, 0, c->stream>>>(
        c->d_pos32, c->d_nrm32, T->d_src, T->d_frm, N, s, f32_consts(k), T->d_part, T->d_ctr, c->d_err, d_skip, g64);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_TRY(timing_end(c, (T->near_steps * kF32STile + T->far_steps * Cheb<NC>::kChunks * kChunk) * (int64_t)kTcTTile));
    const TcM2l m{T->d_irow, T->d_isrc, T->d_items, T->d_tcube, T->n_items};
    if (T->interp && T->n_items > 0) {
        IBIM_CUDA(cudaMemsetAsync(T->d_fields, 0, sizeof(double) * (size_t)T->n_t * kMaxProxies * 4, c->stream));
        tc_m2l_kernel<NC><<<T->m2l_grid, Cheb<NC>::kM2lThreads, 0, c->stream>>>(
            T->d_src, T->d_frm, m, f32_consts(k), T->d_fields, T->d_ctr + 1, c->d_err, d_skip);
        count_launch(c);
        IBIM_CUDA(cudaGetLastError());
    }
    const int bs = 256;
    tc_fixup_kernel<NC><<<(unsigned)((N + bs - 1) / bs), bs, 0, c->stream>>>(
        T->d_part, s, N, k.lambda1, k.lambda2, in, out, m, T->d_fields, c->d_geo64, T->interp, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status tc_apply(ibim_ctx* c, const PairConsts& k, VecRef in, OutRef out, const int* d_skip)
{
    TreeCode* T = c->tc;
    if (T == nullptr) return tc_fail(IBIM_ERR_STATE, "the treecode operator needs ibim_treecode_setup first");
    if (!(k.four_tau2 < 3.0e38)) return tc_fail(IBIM_ERR_ARG, "the treecode operator needs tube rule 0");
    if (std::sqrt(k.tau2) > T->tau_max * (1.0 + 1e-12))
        return tc_fail(IBIM_ERR_ARG, "tau exceeds the tau_max the treecode lists were built for");
    if (T->order == 4) return tc_apply_order<4>(c, T, k, in, out, d_skip);
    if (T->order == 5) return tc_apply_order<5>(c, T, k, in, out, d_skip);
    return tc_apply_order<6>(c, T, k, in, out, d_skip);
}

}  // namespace ibim

extern "C" ibim_status ibim_treecode_setup(ibim_ctx* c, double theta, double tau_max, int order, int target_interp)
{
    using namespace ibim;
    if (c == nullptr || !(theta > 0.0 && theta < 1.0) || !(tau_max > 0.0) || !std::isfinite(tau_max))
        return tc_fail(IBIM_ERR_ARG, "need a context, 0 < theta < 1 and a finite tau_max > 0");
    if (c->N <= 0 || c->d_frames == nullptr) return tc_fail(IBIM_ERR_STATE, "the context has no nodes");
    if (target_interp != 0 && target_interp != 1) return tc_fail(IBIM_ERR_ARG, "target_interp must be 0 or 1");
    if (order < 4 || order > 6) return tc_fail(IBIM_ERR_ARG, "the Chebyshev order must be 4, 5 or 6");
    return tc_setup(c, theta, tau_max, order, target_interp);
}

extern "C" ibim_status ibim_treecode_plan(const double* xyz, int64_t N, double theta, double tau_max,
                                          int target_interp, int64_t* sizes, int64_t* row_ptr, int32_t* steps,
                                          int64_t* irow, int32_t* isrc)
{
    using namespace ibim;
    if (xyz == nullptr || N <= 0 || sizes == nullptr || !(theta > 0.0 && theta < 1.0) || !(tau_max > 0.0) ||
        !std::isfinite(tau_max) || (target_interp != 0 && target_interp != 1))
        return tc_fail(IBIM_ERR_ARG, "need N > 0 coordinates, sizes, 0 < theta < 1, a finite tau_max > 0 and "
                                     "target_interp 0 or 1");
    std::vector<double> xs(3 * (size_t)N);
    for (int64_t j = 0; j < N; ++j) {
        for (int a = 0; a < 3; ++a) {
            const double v = xyz[3 * j + a];
            if (!std::isfinite(v)) return tc_fail(IBIM_ERR_NONFINITE, "non-finite coordinate");
            xs[a * N + j] = v;
        }
    }
    const TcPlan P = tc_plan(xs, N, theta, tau_max, target_interp);
    sizes[0] = P.n_t;
    sizes[1] = (int64_t)P.cl.size();
    sizes[2] = (int64_t)P.steps.size();
    sizes[3] = (int64_t)P.isrc.size();
    sizes[4] = P.n_real;
    if (row_ptr) std::copy(P.row_ptr.begin(), P.row_ptr.end(), row_ptr);
    if (steps) std::copy(P.steps.begin(), P.steps.end(), steps);
    if (irow) std::copy(P.irow.begin(), P.irow.end(), irow);
    if (isrc) std::copy(P.isrc.begin(), P.isrc.end(), isrc);
    return IBIM_OK;
}

extern "C" ibim_status ibim_treecode_info(ibim_ctx* c, int64_t* near_steps, int64_t* far_steps,
                                          int64_t* interp_steps, int64_t* clusters, int64_t* target_tiles)
{
    using namespace ibim;
    if (c == nullptr) return tc_fail(IBIM_ERR_ARG, "need a context");
    if (c->tc == nullptr) return tc_fail(IBIM_ERR_STATE, "no treecode: call ibim_treecode_setup");
    if (near_steps) *near_steps = c->tc->near_steps;
    if (far_steps) *far_steps = c->tc->far_steps;
    if (interp_steps) *interp_steps = c->tc->interp_steps;
    if (clusters) *clusters = c->tc->n_clusters;
    if (target_tiles) *target_tiles = c->tc->n_t;
    return IBIM_OK;
}
