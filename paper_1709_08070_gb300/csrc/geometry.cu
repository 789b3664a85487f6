// Narrowband geometry on the GPU (Sec. 2.2, Sec. 3.2): band extraction
// {|d| < eps} over the Cartesian grid, closest-point projection
// x* = x - d grad d, unit normals and weights w = J delta_eps(d) h^3 (J = 1,
// cosine weight).  Grid nodes are enumerated in Morton (Z-curve) order of
// their box-local coordinates; the compaction keeps that order (block counts,
// one scan, ordered writes), and finish_geometry then reorders the nodes of
// built geometries into compact 32-node blocks by coordinate bisection.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

__host__ __device__ __forceinline__ uint32_t compact1by2(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

struct SphereBox {
    int64_t lo[3];
    int64_t n[3];
    double c[3], o[3];
    double R, h, eps;
};

// Band test for one Morton code; returns true and fills the node when kept.
__device__ __forceinline__ bool sphere_node(const SphereBox& B, uint64_t code, double* x, double* nrm,
                                            double* d, int32_t* ijk)
{
    const uint32_t a = compact1by2(code), b = compact1by2(code >> 1), cc = compact1by2(code >> 2);
    if (a >= B.n[0] || b >= B.n[1] || cc >= B.n[2]) return false;
    const int64_t gi = B.lo[0] + a, gj = B.lo[1] + b, gk = B.lo[2] + cc;
    const double p0 = B.o[0] + B.h * (double)gi, p1 = B.o[1] + B.h * (double)gj, p2 = B.o[2] + B.h * (double)gk;
    const double v0 = p0 - B.c[0], v1 = p1 - B.c[1], v2 = p2 - B.c[2];
    const double len = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    const double dd = len - B.R;  // signed distance, negative inside
    if (!(fabs(dd) < B.eps) || len == 0.0) return false;
    nrm[0] = v0 / len;
    nrm[1] = v1 / len;
    nrm[2] = v2 / len;
    x[0] = p0 - dd * nrm[0];
    x[1] = p1 - dd * nrm[1];
    x[2] = p2 - dd * nrm[2];
    *d = dd;
    ijk[0] = (int32_t)gi;
    ijk[1] = (int32_t)gj;
    ijk[2] = (int32_t)gk;
    return true;
}

constexpr int kCompactBlock = 1024;

__global__ void __launch_bounds__(kCompactBlock) sphere_count_kernel(SphereBox B, uint64_t ncodes, int* __restrict__ counts)
{
    const uint64_t code = (uint64_t)blockIdx.x * kCompactBlock + threadIdx.x;
    double x[3], n[3], d;
    int32_t ijk[3];
    const bool keep = code < ncodes && sphere_node(B, code, x, n, &d, ijk);
    const int c = __syncthreads_count(keep);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of the block counts in one CTA (sequential per thread chunk).
__global__ void scan_counts_kernel(int* __restrict__ counts, int64_t nblocks, int64_t* __restrict__ total)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (nblocks + 1023) / 1024;
    const int64_t b0 = t * per, b1 = (b0 + per < nblocks) ? b0 + per : nblocks;
    int64_t s = 0;
    for (int64_t b = b0; b < b1; ++b) s += counts[b];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int q = 0; q < 1024; ++q) {
            const int64_t v = part[q];
            part[q] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t b = b0; b < b1; ++b) {
        const int v = counts[b];
        counts[b] = (int)run;
        run += v;
    }
}

__global__ void __launch_bounds__(kCompactBlock) sphere_write_kernel(SphereBox B, uint64_t ncodes, const int* __restrict__ offsets, int64_t N,
                                    double* __restrict__ geo, double* __restrict__ dist,
                                    int32_t* __restrict__ ijk_out, double* __restrict__ lap,
                                    double* __restrict__ sig2)
{
    __shared__ int warp_tot[kCompactBlock / 32];
    const uint64_t code = (uint64_t)blockIdx.x * kCompactBlock + threadIdx.x;
    double x[3], n[3], d = 0.0;
    int32_t ijk[3];
    const bool keep = code < ncodes && sphere_node(B, code, x, n, &d, ijk);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < warp; ++q) before += warp_tot[q];
    if (!keep) return;
    const int64_t j = (int64_t)offsets[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    const double w = (1.0 + cos(kPi * d / B.eps)) / (2.0 * B.eps) * B.h * B.h * B.h;
    geo[j] = x[0];
    geo[N + j] = x[1];
    geo[2 * N + j] = x[2];
    geo[3 * N + j] = n[0];
    geo[4 * N + j] = n[1];
    geo[5 * N + j] = n[2];
    geo[6 * N + j] = w;
    dist[j] = d;
    // Laplacian of d = |x - c| - R at the grid node and the sum of the 2x2
    // principal minors of its Hessian (eigenvalues 1/|x-c| twice and 0)
    const double len = B.R + d;
    lap[j] = 2.0 / len;
    sig2[j] = 1.0 / (len * len);
    ijk_out[3 * j] = ijk[0];
    ijk_out[3 * j + 1] = ijk[1];
    ijk_out[3 * j + 2] = ijk[2];
}

ibim_status build_sphere_nodes(ibim_ctx* c, double R, const double* centre, const double* origin, double h,
                               double eps)
{
    SphereBox B;
    int64_t P = 1;
    for (int a = 0; a < 3; ++a) {
        B.c[a] = centre[a];
        B.o[a] = origin[a];
        B.lo[a] = (int64_t)floor((centre[a] - R - eps - origin[a]) / h) - 1;
        const int64_t hi = (int64_t)ceil((centre[a] + R + eps - origin[a]) / h) + 1;
        B.n[a] = hi - B.lo[a] + 1;
        while (P < B.n[a]) P <<= 1;
    }
    B.R = R;
    B.h = h;
    B.eps = eps;
    const uint64_t ncodes = (uint64_t)P * P * P;
    const int64_t nblocks = (int64_t)((ncodes + kCompactBlock - 1) / kCompactBlock);
    int* d_counts = nullptr;
    int64_t* d_total = nullptr;
    IBIM_CUDA(cudaMalloc((void**)&d_counts, sizeof(int) * nblocks));
    IBIM_CUDA(cudaMalloc((void**)&d_total, sizeof(int64_t)));
    sphere_count_kernel<<<(unsigned)nblocks, kCompactBlock, 0, c->stream>>>(B, ncodes, d_counts);
    scan_counts_kernel<<<1, 1024, 0, c->stream>>>(d_counts, nblocks, d_total);
    count_launch(c, 2);
    int64_t N = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&N, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess || N == 0) {
        cudaFree(d_counts);
        cudaFree(d_total);
        if (e != cudaSuccess) return cuda_fail(e, "sphere band count", __FILE__, __LINE__);
        set_error("the narrowband holds no grid node");
        return IBIM_ERR_EMPTY_BAND;
    }
    c->N = N;
    e = cudaMalloc((void**)&c->d_geo64, sizeof(double) * 7 * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_dist, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ijk, sizeof(int32_t) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_curv, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_sig2, sizeof(double) * N);
    if (e == cudaSuccess) {
        sphere_write_kernel<<<(unsigned)nblocks, kCompactBlock, 0, c->stream>>>(B, ncodes, d_counts, N, c->d_geo64,
                                                                                c->d_dist, c->d_ijk, c->d_curv,
                                                                                c->d_sig2);
        count_launch(c);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_counts);
    cudaFree(d_total);
    if (e != cudaSuccess) return cuda_fail(e, "sphere band write", __FILE__, __LINE__);
    return IBIM_OK;
}

// FP32 copies of the geometry over the padded node range (positions relative
// to the centroid; the chunk-frame pass replaces them), placeholder normals
// past N.
__global__ void pack_geometry_f32_kernel(const double* __restrict__ geo, int64_t N, int64_t n_pad, double c0,
                                         double c1, double c2, float4* __restrict__ pos, float4* __restrict__ nrm)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    if (j >= N) {
        pos[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        nrm[j] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
        return;
    }
    pos[j] = make_float4((float)(geo[j] - c0), (float)(geo[N + j] - c1), (float)(geo[2 * N + j] - c2),
                         (float)geo[6 * N + j]);
    nrm[j] = make_float4((float)geo[3 * N + j], (float)geo[4 * N + j], (float)geo[5 * N + j], 0.0f);
}

// out[i] = in[perm[i]] for `fields` interleaved-by-field arrays of N values
// (field f of node j at in[f * N + j]).
template <typename T>
__global__ void gather_fields_kernel(const T* __restrict__ in, const int64_t* __restrict__ perm, int64_t N,
                                     int fields, T* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t j = perm[i];
    for (int f = 0; f < fields; ++f) out[f * N + i] = in[f * N + j];
}

// out[3 i + a] = in[3 perm[i] + a] (node-major triples).
__global__ void gather_triples_kernel(const int32_t* __restrict__ in, const int64_t* __restrict__ perm, int64_t N,
                                      int32_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t j = perm[i];
    for (int a = 0; a < 3; ++a) out[3 * i + a] = in[3 * j + a];
}

namespace {

// Recursive coordinate bisection of x* into aligned blocks of kRcbLeaf nodes:
// each range of n nodes is split across the longest side of its bounding box,
// the left part holding B max(1, round(n / 2B)) nodes with B = 1024 for
// n >= 2048, 256 for n >= 512 and kRcbLeaf below (ties broken by node index,
// so the order is a deterministic function of the coordinates).  Aligned runs
// of 32, 256 and 1024 nodes are then bisection ranges (all but those holding
// the last node), so the pair kernels' chunks, source tiles and target tiles
// and the treecode's clusters are compact.
constexpr int64_t kRcbLeaf = 32;

void rcb_split(const std::vector<double>& xs, int64_t N, std::vector<int64_t>& perm, int64_t lo, int64_t hi)
{
    const int64_t n = hi - lo;
    if (n <= kRcbLeaf) return;
    double mn[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, mx[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int64_t q = lo; q < hi; ++q)
        for (int a = 0; a < 3; ++a) {
            const double v = xs[a * N + perm[q]];
            mn[a] = std::min(mn[a], v);
            mx[a] = std::max(mx[a], v);
        }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
    const int64_t B = n >= 2048 ? 1024 : (n >= 512 ? 256 : kRcbLeaf);
    const int64_t half = std::max<int64_t>(1, (int64_t)llround((double)n / (2.0 * (double)B)));
    const int64_t k = lo + B * half;
    const double* key = xs.data() + ax * N;
    std::nth_element(perm.begin() + lo, perm.begin() + k, perm.begin() + hi, [key](int64_t a, int64_t b) {
        return key[a] < key[b] || (key[a] == key[b] && a < b);
    });
    rcb_split(xs, N, perm, lo, k);
    rcb_split(xs, N, perm, k, hi);
}

}  // namespace

// Reorders the nodes of a built geometry (every per-node array) into compact
// aligned 32-node blocks: the blocks are the pair kernels' chunks, whose
// bounding spheres decide the near/far split, so a block that straddles two
// distant pieces of the band would send whole rows down the near path.
static ibim_status compact_order(ibim_ctx* c)
{
    const int64_t N = c->N;
    if (N <= kRcbLeaf) return IBIM_OK;
    std::vector<double> xs(3 * (size_t)N);
    IBIM_CUDA(cudaMemcpyAsync(xs.data(), c->d_geo64, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int64_t> perm(N);
    for (int64_t i = 0; i < N; ++i) perm[i] = i;
    rcb_split(xs, N, perm, 0, N);

    int64_t* d_perm = nullptr;
    double* geo = nullptr;
    double* dist = nullptr;
    double* curv = nullptr;
    double* sig2 = nullptr;
    int32_t* ijk = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_perm, sizeof(int64_t) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&geo, sizeof(double) * 7 * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dist, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&curv, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sig2, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ijk, sizeof(int32_t) * 3 * N);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_perm, perm.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        const unsigned nb = (unsigned)((N + 255) / 256);
        gather_fields_kernel<double><<<nb, 256, 0, c->stream>>>(c->d_geo64, d_perm, N, 7, geo);
        gather_fields_kernel<double><<<nb, 256, 0, c->stream>>>(c->d_dist, d_perm, N, 1, dist);
        gather_fields_kernel<double><<<nb, 256, 0, c->stream>>>(c->d_curv, d_perm, N, 1, curv);
        gather_fields_kernel<double><<<nb, 256, 0, c->stream>>>(c->d_sig2, d_perm, N, 1, sig2);
        gather_triples_kernel<<<nb, 256, 0, c->stream>>>(c->d_ijk, d_perm, N, ijk);
        count_launch(c, 5);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_perm);
    if (e != cudaSuccess) {
        cudaFree(geo);
        cudaFree(dist);
        cudaFree(curv);
        cudaFree(sig2);
        cudaFree(ijk);
        return cuda_fail(e, "compact node order", __FILE__, __LINE__);
    }
    std::swap(c->d_geo64, geo);
    std::swap(c->d_dist, dist);
    std::swap(c->d_curv, curv);
    std::swap(c->d_sig2, sig2);
    std::swap(c->d_ijk, ijk);
    cudaFree(geo);
    cudaFree(dist);
    cudaFree(curv);
    cudaFree(sig2);
    cudaFree(ijk);
    return IBIM_OK;
}

ibim_status finish_geometry(ibim_ctx* c, bool reorder)
{
    if (reorder) IBIM_TRY(compact_order(c));
    const int64_t N = c->N;
    if (reorder) {  // built geometries: keep the J = 1 weights for ibim_set_jacobian
        IBIM_CUDA(cudaMalloc((void**)&c->d_w1, sizeof(double) * N));
        IBIM_CUDA(cudaMemcpyAsync(c->d_w1, c->d_geo64 + 6 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                  c->stream));
    }
    const int64_t n_pad = padded_nodes(N);
    IBIM_CUDA(cudaMalloc((void**)&c->d_pos32, sizeof(float4) * n_pad));
    IBIM_CUDA(cudaMalloc((void**)&c->d_nrm32, sizeof(float4) * n_pad));
    const int bs = 256;
    pack_geometry_f32_kernel<<<(unsigned)((n_pad + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_geo64, N, n_pad, c->centroid[0], c->centroid[1], c->centroid[2], c->d_pos32, c->d_nrm32);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_TRY(f32_chunk_frames(c));  // overwrites d_pos32 with chunk-frame positions
    apply_cached_tuning(c);
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

}  // namespace ibim
