// Level-set construction of the solvent excluded surface (Sec. 3.1) and its
// narrowband nodes (Sec. 3.2) on the GPU, FP64.
//
//   F(x) = min_k (|x - z_k| - r_k)           vdW level set, clamped at L
//   phi = F - rho0                            solvent accessible surface
//   d phi/dt = |grad phi|, t in (0, rho0]     inward eikonal flow (TVD-RK3,
//                                             Godunov, WENO5, zero Neumann)
//   cavity removal                            flood fill of {phi > 0} from the
//                                             box boundary; other phi > 0 nodes
//                                             and their eps-neighbourhood := -eps
//   phi_t + sgn_h(phi0)(|grad phi| - 1) = 0   reinitialisation, ceil((k1+4)/k0)
//                                             steps of dt = k0 h, k0 = 1/2
//   band {|phi| < eps}                        n = grad phi/|grad phi| with
//                                             grad = (p_- + p_+)/2 (WENO5),
//                                             x* = x - phi n, w = delta_eps(phi) h^3
// The grid is origin-free: node (i, j, k) sits at h (lo + (i, j, k)).  The
// file is compiled without FMA contraction so that the stencil arithmetic
// rounds like plain C.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

struct LsGrid {
    int64_t lo[3];
    int64_t n[3];
    double h;
};

__device__ __forceinline__ int64_t ls_idx(const LsGrid& g, int64_t i, int64_t j, int64_t k)
{
    return (k * g.n[1] + j) * g.n[0] + i;
}

__device__ __forceinline__ int64_t clamp_i(int64_t v, int64_t n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// ------------------------------------------------------------- vdW level set
struct __align__(32) Atom {
    double x, y, z, r;
};

struct CellList {
    double co[3];  // origin of cell (0,0,0)
    double cs;     // cell size (>= cutoff)
    int nc[3];
};

__global__ void vdw_kernel(LsGrid g, CellList cl, const Atom* __restrict__ atoms, const int* __restrict__ start,
                           double L, double probe, double* __restrict__ phi)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    const double x0 = g.h * (double)(g.lo[0] + i), x1 = g.h * (double)(g.lo[1] + j), x2 = g.h * (double)(g.lo[2] + k);
    const int c0 = (int)floor((x0 - cl.co[0]) / cl.cs), c1 = (int)floor((x1 - cl.co[1]) / cl.cs),
              c2 = (int)floor((x2 - cl.co[2]) / cl.cs);
    double f = L;
    for (int dz = -1; dz <= 1; ++dz) {
        const int cz = c2 + dz;
        if (cz < 0 || cz >= cl.nc[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int cy = c1 + dy;
            if (cy < 0 || cy >= cl.nc[1]) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int cx = c0 + dx;
                if (cx < 0 || cx >= cl.nc[0]) continue;
                const int cell = (cz * cl.nc[1] + cy) * cl.nc[0] + cx;
                for (int a = start[cell]; a < start[cell + 1]; ++a) {
                    const Atom z = atoms[a];
                    const double d0 = x0 - z.x, d1 = x1 - z.y, d2 = x2 - z.z;
                    const double v = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - z.r;
                    f = fmin(f, v);
                }
            }
        }
    }
    phi[id] = f - probe;
}

// ---------------------------------------------------------------- WENO5
// Fifth-order WENO one-sided derivative (Jiang-Peng weights) from five first
// differences ordered along the upwind direction.
__device__ __forceinline__ double weno5(double v1, double v2, double v3, double v4, double v5)
{
    const double q1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
    const double q2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
    const double q3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
    const double d1 = v1 - 2.0 * v2 + v3, e1 = v1 - 4.0 * v2 + 3.0 * v3;
    const double d2 = v2 - 2.0 * v3 + v4, e2 = v2 - v4;
    const double d3 = v3 - 2.0 * v4 + v5, e3 = 3.0 * v3 - 4.0 * v4 + v5;
    const double s1 = 13.0 / 12.0 * d1 * d1 + 0.25 * e1 * e1;
    const double s2 = 13.0 / 12.0 * d2 * d2 + 0.25 * e2 * e2;
    const double s3 = 13.0 / 12.0 * d3 * d3 + 0.25 * e3 * e3;
    const double m = fmax(fmax(fmax(v1 * v1, v2 * v2), fmax(v3 * v3, v4 * v4)), v5 * v5);
    const double e = 1e-6 * m + 1e-99;
    const double a1 = 0.1 / ((s1 + e) * (s1 + e));
    const double a2 = 0.6 / ((s2 + e) * (s2 + e));
    const double a3 = 0.3 / ((s3 + e) * (s3 + e));
    return (a1 * q1 + a2 * q2 + a3 * q3) / (a1 + a2 + a3);
}

// p_- (backward) and p_+ (forward) along axis `ax` at node (i, j, k).
__device__ __forceinline__ void weno_pair(const LsGrid& g, const double* __restrict__ phi, int64_t i, int64_t j,
                                          int64_t k, int ax, double& pm, double& pp)
{
    double f[7];
#pragma unroll
    for (int s = -3; s <= 3; ++s) {
        int64_t ii = i, jj = j, kk = k;
        if (ax == 0) ii = clamp_i(i + s, g.n[0]);
        else if (ax == 1) jj = clamp_i(j + s, g.n[1]);
        else kk = clamp_i(k + s, g.n[2]);
        f[s + 3] = phi[ls_idx(g, ii, jj, kk)];
    }
    double D[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) D[m] = (f[m + 1] - f[m]) / g.h;
    pm = weno5(D[0], D[1], D[2], D[3], D[4]);
    pp = weno5(D[5], D[4], D[3], D[2], D[1]);
}

// One TVD-RK3 stage: out = a base + b (in + dt L(in)).
//   mode 0: L = |grad phi| with the Godunov form for speed -1 (inward flow);
//   mode 1: L = -sgn_h(phi0) (|grad phi| - 1) (reinitialisation).
__global__ void ls_stage_kernel(LsGrid g, const double* __restrict__ in, const double* __restrict__ base,
                                const double* __restrict__ phi0, double* __restrict__ out, double a, double b,
                                double dt, int mode)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    double s = 0.0;
    double p0 = 0.0;
    if (mode == 1) p0 = phi0[id];
    for (int ax = 0; ax < 3; ++ax) {
        double pm, pp;
        weno_pair(g, in, i, j, k, ax, pm, pp);
        if (mode == 0 || p0 <= 0.0) {  // upwind from the larger phi
            const double u = pm < 0.0 ? pm : 0.0, v = pp > 0.0 ? pp : 0.0;
            s += fmax(u * u, v * v);
        } else {
            const double u = pm > 0.0 ? pm : 0.0, v = pp < 0.0 ? pp : 0.0;
            s += fmax(u * u, v * v);
        }
    }
    double L;
    if (mode == 0) {
        L = sqrt(s);
    } else {
        const double sg = p0 / sqrt(p0 * p0 + g.h * g.h);
        L = -sg * (sqrt(s) - 1.0);
    }
    out[id] = a * base[id] + b * (in[id] + dt * L);
}

// --------------------------------------------------------------- cavities
__global__ void cav_init_kernel(LsGrid g, const double* __restrict__ phi, uint8_t* __restrict__ lab)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    const bool edge = i == 0 || j == 0 || k == 0 || i == g.n[0] - 1 || j == g.n[1] - 1 || k == g.n[2] - 1;
    lab[id] = (edge && phi[id] > 0.0) ? 1 : 0;
}

// One flood pass: an unlabelled phi > 0 node next to an exterior node joins the exterior.
__global__ void cav_flood_kernel(LsGrid g, const double* __restrict__ phi, uint8_t* __restrict__ lab,
                                 int* __restrict__ changed)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    if (lab[id] != 0 || !(phi[id] > 0.0)) return;
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    const int64_t sx = 1, sy = g.n[0], sz = g.n[0] * g.n[1];
    bool hit = (i > 0 && lab[id - sx] == 1) || (i + 1 < g.n[0] && lab[id + sx] == 1) ||
               (j > 0 && lab[id - sy] == 1) || (j + 1 < g.n[1] && lab[id + sy] == 1) ||
               (k > 0 && lab[id - sz] == 1) || (k + 1 < g.n[2] && lab[id + sz] == 1);
    if (hit) {
        lab[id] = 1;
        *changed = 1;
    }
}

__global__ void cav_mark_kernel(LsGrid g, const double* __restrict__ phi, uint8_t* __restrict__ lab,
                                unsigned long long* __restrict__ ncav)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    if (lab[id] == 0 && phi[id] > 0.0) {
        lab[id] = 2;
        atomicAdd(ncav, 1ull);
    }
}

// Nodes (not exterior, not cavity) within Euclidean distance eps of a cavity node -> label 3.
__global__ void cav_dilate_kernel(LsGrid g, uint8_t* __restrict__ lab, int R, double e2)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    if (lab[id] != 0) return;
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    for (int c = -R; c <= R; ++c)
        for (int b = -R; b <= R; ++b)
            for (int a = -R; a <= R; ++a) {
                if ((double)(a * a + b * b + c * c) > e2) continue;
                const int64_t ii = i + a, jj = j + b, kk = k + c;
                if (ii < 0 || jj < 0 || kk < 0 || ii >= g.n[0] || jj >= g.n[1] || kk >= g.n[2]) continue;
                if (lab[ls_idx(g, ii, jj, kk)] == 2) {
                    lab[id] = 3;
                    return;
                }
            }
}

__global__ void cav_apply_kernel(LsGrid g, const uint8_t* __restrict__ lab, double eps, double* __restrict__ phi)
{
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M) return;
    if (lab[id] == 2 || lab[id] == 3) phi[id] = -eps;
}

// ------------------------------------------------------------------- band
__host__ __device__ __forceinline__ uint32_t ls_compact1by2(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

constexpr int kBandBlock = 256;  // band_write_kernel needs ~94 registers per thread

__device__ __forceinline__ bool band_node(const LsGrid& g, const double* __restrict__ phi, double eps, uint64_t code,
                                          int64_t* idout)
{
    const uint32_t a = ls_compact1by2(code), b = ls_compact1by2(code >> 1), c = ls_compact1by2(code >> 2);
    if (a >= g.n[0] || b >= g.n[1] || c >= g.n[2]) return false;
    const int64_t id = ls_idx(g, a, b, c);
    *idout = id;
    return fabs(phi[id]) < eps;
}

__global__ void __launch_bounds__(kBandBlock) band_count_kernel(LsGrid g, const double* __restrict__ phi, double eps, uint64_t ncodes,
                                  int* __restrict__ counts)
{
    const uint64_t code = (uint64_t)blockIdx.x * kBandBlock + threadIdx.x;
    int64_t id = 0;
    const bool keep = code < ncodes && band_node(g, phi, eps, code, &id);
    const int c = __syncthreads_count(keep);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void band_scan_kernel(int* __restrict__ counts, int64_t nblocks, int64_t* __restrict__ total)
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

__global__ void __launch_bounds__(kBandBlock) band_write_kernel(LsGrid g, const double* __restrict__ phi, double eps, uint64_t ncodes,
                                  const int* __restrict__ offsets, int64_t N, double* __restrict__ geo,
                                  double* __restrict__ dist, int32_t* __restrict__ ijk, double* __restrict__ curv,
                                  double* __restrict__ sig2)
{
    __shared__ int warp_tot[kBandBlock / 32];
    const uint64_t code = (uint64_t)blockIdx.x * kBandBlock + threadIdx.x;
    int64_t id = 0;
    const bool keep = code < ncodes && band_node(g, phi, eps, code, &id);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < warp; ++q) before += warp_tot[q];
    if (!keep) return;
    const int64_t jn = (int64_t)offsets[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    const int64_t i = id % g.n[0], j = (id / g.n[0]) % g.n[1], k = id / (g.n[0] * g.n[1]);
    double gr[3];
    for (int ax = 0; ax < 3; ++ax) {
        double pm, pp;
        weno_pair(g, phi, i, j, k, ax, pm, pp);
        gr[ax] = 0.5 * (pm + pp);
    }
    const double len = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    const double p = phi[id];
    const int64_t gi[3] = {g.lo[0] + i, g.lo[1] + j, g.lo[2] + k};
    for (int a = 0; a < 3; ++a) {
        const double nv = (len > 0.0) ? gr[a] / len : 0.0;
        geo[(3 + a) * N + jn] = nv;
        geo[a * N + jn] = g.h * (double)gi[a] - p * nv;
        ijk[3 * jn + a] = (int32_t)gi[a];
    }
    geo[6 * N + jn] = (1.0 + cos(kPi * p / eps)) / (2.0 * eps) * g.h * g.h * g.h;
    dist[jn] = p;
    // Hessian of phi by central differences (indices clamped at the box):
    // its trace (the Laplacian, twice the mean curvature) and the sum of its
    // 2x2 principal minors, the inputs of the full Jacobian (Sec. 2.2)
    double H[3][3];
    const int64_t c0[3] = {i, j, k};
    double lap = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        int64_t im[3] = {i, j, k}, ip[3] = {i, j, k};
        im[ax] = clamp_i(im[ax] - 1, g.n[ax]);
        ip[ax] = clamp_i(ip[ax] + 1, g.n[ax]);
        H[ax][ax] = (phi[ls_idx(g, ip[0], ip[1], ip[2])] - 2.0 * p + phi[ls_idx(g, im[0], im[1], im[2])]) / (g.h * g.h);
        lap += H[ax][ax];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) {
            double v[4];
            for (int t = 0; t < 4; ++t) {
                int64_t e[3] = {c0[0], c0[1], c0[2]};
                e[a] = clamp_i(e[a] + ((t < 2) ? 1 : -1), g.n[a]);
                e[b] = clamp_i(e[b] + ((t & 1) ? -1 : 1), g.n[b]);
                v[t] = phi[ls_idx(g, e[0], e[1], e[2])];
            }
            H[a][b] = H[b][a] = (v[0] - v[1] - v[2] + v[3]) / (4.0 * g.h * g.h);
        }
    curv[jn] = lap;
    sig2[jn] = H[0][0] * H[1][1] - H[0][1] * H[0][1] + H[0][0] * H[2][2] - H[0][2] * H[0][2] + H[1][1] * H[2][2] -
               H[1][2] * H[1][2];
}

// ------------------------------------------------------------------ driver

static LsGrid make_grid(int64_t Na, const double* z, const double* r, double probe, double h, double eps)
{
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = 0; k < Na; ++k)
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], z[3 * k + a] - r[k]);
            mx[a] = std::max(mx[a], z[3 * k + a] + r[k]);
        }
    LsGrid g;
    const double pad = probe + eps + 8.0 * h;  // SAS plus the band and the WENO stencil reach
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = (int64_t)floor((mn[a] - pad) / h);
        g.n[a] = (int64_t)ceil((mx[a] + pad) / h) - g.lo[a] + 1;
    }
    g.h = h;
    return g;
}

ibim_status build_levelset(ibim_ctx* c, int64_t Na, const double* z, const double* r, double probe, double h,
                           double eps)
{
    const LsGrid g = make_grid(Na, z, r, probe, h, eps);
    const int64_t M = g.n[0] * g.n[1] * g.n[2];
    if (M > (int64_t)1 << 31) {
        set_error("level-set grid larger than 2^31 nodes");
        return IBIM_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        c->ls_lo[a] = g.lo[a];
        c->ls_n[a] = g.n[a];
    }
    // Cell list of the atoms on the host (cell size >= the clamp cutoff L + r_max).
    const double L = 2.0 * probe + eps + 6.0 * h;
    double rmax = 0.0, mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = 0; k < Na; ++k) {
        rmax = std::max(rmax, r[k]);
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], z[3 * k + a]);
            mx[a] = std::max(mx[a], z[3 * k + a]);
        }
    }
    CellList cl;
    cl.cs = L + rmax + 1e-9;
    for (int a = 0; a < 3; ++a) {
        cl.co[a] = mn[a] - cl.cs;
        cl.nc[a] = (int)floor((mx[a] - cl.co[a]) / cl.cs) + 2;
    }
    const int ncell = cl.nc[0] * cl.nc[1] * cl.nc[2];
    std::vector<int> start(ncell + 1, 0), cellof(Na);
    for (int64_t k = 0; k < Na; ++k) {
        int cc[3];
        for (int a = 0; a < 3; ++a) cc[a] = (int)floor((z[3 * k + a] - cl.co[a]) / cl.cs);
        cellof[k] = (cc[2] * cl.nc[1] + cc[1]) * cl.nc[0] + cc[0];
        start[cellof[k] + 1]++;
    }
    for (int q = 0; q < ncell; ++q) start[q + 1] += start[q];
    std::vector<int> fill(start.begin(), start.end() - 1);
    std::vector<Atom> atoms(Na);
    for (int64_t k = 0; k < Na; ++k) atoms[fill[cellof[k]]++] = Atom{z[3 * k], z[3 * k + 1], z[3 * k + 2], r[k]};

    Atom* d_atoms = nullptr;
    int* d_start = nullptr;
    double *d_phi = nullptr, *d_t1 = nullptr, *d_t2 = nullptr, *d_phi0 = nullptr;
    uint8_t* d_lab = nullptr;
    int* d_flag = nullptr;
    unsigned long long* d_ncav = nullptr;
    ibim_status st = IBIM_OK;
    auto cleanup = [&]() {
        cudaFree(d_atoms);
        cudaFree(d_start);
        cudaFree(d_t1);
        cudaFree(d_t2);
        cudaFree(d_phi0);
        cudaFree(d_lab);
        cudaFree(d_flag);
        cudaFree(d_ncav);
    };
#define LS_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) {                                          \
            st = cuda_fail(_e, #call, __FILE__, __LINE__);                \
            cleanup();                                                    \
            return st;                                                    \
        }                                                                 \
    } while (0)
    LS_CUDA(cudaMalloc((void**)&d_atoms, sizeof(Atom) * Na));
    LS_CUDA(cudaMalloc((void**)&d_start, sizeof(int) * (ncell + 1)));
    LS_CUDA(cudaMalloc((void**)&d_phi, sizeof(double) * M));
    c->d_phi = d_phi;
    LS_CUDA(cudaMalloc((void**)&d_t1, sizeof(double) * M));
    LS_CUDA(cudaMalloc((void**)&d_t2, sizeof(double) * M));
    LS_CUDA(cudaMalloc((void**)&d_phi0, sizeof(double) * M));
    LS_CUDA(cudaMalloc((void**)&d_lab, M));
    LS_CUDA(cudaMalloc((void**)&d_flag, sizeof(int)));
    LS_CUDA(cudaMalloc((void**)&d_ncav, sizeof(unsigned long long)));
    LS_CUDA(cudaMemcpyAsync(d_atoms, atoms.data(), sizeof(Atom) * Na, cudaMemcpyHostToDevice, c->stream));
    LS_CUDA(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * (ncell + 1), cudaMemcpyHostToDevice, c->stream));

    const int bs = 256;
    const unsigned nb = (unsigned)((M + bs - 1) / bs);
    vdw_kernel<<<nb, bs, 0, c->stream>>>(g, cl, d_atoms, d_start, L, probe, d_phi);
    count_launch(c);
    LS_CUDA(cudaGetLastError());

    // inward eikonal flow for t in (0, probe]
    if (probe > 0.0) {
        const int steps = (int)ceil(probe / (0.5 * h));
        const double dt = probe / steps;
        for (int s = 0; s < steps; ++s) {
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_phi, d_phi, nullptr, d_t1, 0.0, 1.0, dt, 0);
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_t1, d_phi, nullptr, d_t2, 0.75, 0.25, dt, 0);
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_t2, d_phi, nullptr, d_phi, 1.0 / 3.0, 2.0 / 3.0, dt, 0);
            count_launch(c, 3);
        }
        LS_CUDA(cudaGetLastError());
    }
    // cavity removal
    {
        cav_init_kernel<<<nb, bs, 0, c->stream>>>(g, d_phi, d_lab);
        count_launch(c);
        int h_flag = 1;
        const int64_t max_pass = M + 1;
        int64_t pass = 0;
        while (h_flag && pass < max_pass) {
            LS_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), c->stream));
            for (int q = 0; q < 16; ++q) {
                cav_flood_kernel<<<nb, bs, 0, c->stream>>>(g, d_phi, d_lab, d_flag);
                count_launch(c);
            }
            pass += 16;
            LS_CUDA(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            LS_CUDA(cudaStreamSynchronize(c->stream));
        }
        LS_CUDA(cudaMemsetAsync(d_ncav, 0, sizeof(unsigned long long), c->stream));
        cav_mark_kernel<<<nb, bs, 0, c->stream>>>(g, d_phi, d_lab, d_ncav);
        count_launch(c);
        unsigned long long ncav = 0;
        LS_CUDA(cudaMemcpyAsync(&ncav, d_ncav, sizeof(ncav), cudaMemcpyDeviceToHost, c->stream));
        LS_CUDA(cudaStreamSynchronize(c->stream));
        c->ls_cavity_nodes = (int64_t)ncav;
        if (ncav > 0) {
            const int R = (int)ceil(eps / h);
            cav_dilate_kernel<<<nb, bs, 0, c->stream>>>(g, d_lab, R, eps * eps / (h * h));
            cav_apply_kernel<<<nb, bs, 0, c->stream>>>(g, d_lab, eps, d_phi);
            count_launch(c, 2);
        }
        LS_CUDA(cudaGetLastError());
    }
    // reinitialisation
    {
        const double k0 = 0.5, k1 = eps / h;
        const int steps = (int)ceil((k1 + 4.0) / k0 - 1e-9);
        const double dt = k0 * h;
        LS_CUDA(cudaMemcpyAsync(d_phi0, d_phi, sizeof(double) * M, cudaMemcpyDeviceToDevice, c->stream));
        for (int s = 0; s < steps; ++s) {
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_phi, d_phi, d_phi0, d_t1, 0.0, 1.0, dt, 1);
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_t1, d_phi, d_phi0, d_t2, 0.75, 0.25, dt, 1);
            ls_stage_kernel<<<nb, bs, 0, c->stream>>>(g, d_t2, d_phi, d_phi0, d_phi, 1.0 / 3.0, 2.0 / 3.0, dt, 1);
            count_launch(c, 3);
        }
        LS_CUDA(cudaGetLastError());
    }
    // band extraction in Morton order
    {
        int64_t P = 1;
        while (P < g.n[0] || P < g.n[1] || P < g.n[2]) P <<= 1;
        const uint64_t ncodes = (uint64_t)P * P * P;
        const int64_t nblocks = (int64_t)((ncodes + kBandBlock - 1) / kBandBlock);
        int* d_counts = nullptr;
        int64_t* d_total = nullptr;
        LS_CUDA(cudaMalloc((void**)&d_counts, sizeof(int) * nblocks));
        cudaError_t e = cudaMalloc((void**)&d_total, sizeof(int64_t));
        int64_t N = 0;
        if (e == cudaSuccess) {
            band_count_kernel<<<(unsigned)nblocks, kBandBlock, 0, c->stream>>>(g, d_phi, eps, ncodes, d_counts);
            band_scan_kernel<<<1, 1024, 0, c->stream>>>(d_counts, nblocks, d_total);
            count_launch(c, 2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&N, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess && N > 0) {
            c->N = N;
            e = cudaMalloc((void**)&c->d_geo64, sizeof(double) * 7 * N);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_dist, sizeof(double) * N);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ijk, sizeof(int32_t) * 3 * N);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_curv, sizeof(double) * N);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_sig2, sizeof(double) * N);
            if (e == cudaSuccess) {
                band_write_kernel<<<(unsigned)nblocks, kBandBlock, 0, c->stream>>>(g, d_phi, eps, ncodes, d_counts, N,
                                                                                   c->d_geo64, c->d_dist, c->d_ijk,
                                                                                   c->d_curv, c->d_sig2);
                count_launch(c);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        }
        cudaFree(d_counts);
        cudaFree(d_total);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "band extraction", __FILE__, __LINE__);
            cleanup();
            return st;
        }
        if (N == 0) {
            cleanup();
            set_error("the narrowband holds no grid node");
            return IBIM_ERR_EMPTY_BAND;
        }
    }
#undef LS_CUDA
    cleanup();
    return IBIM_OK;
}

}  // namespace ibim
