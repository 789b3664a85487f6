// Right-hand side (Sec. 2.2), reaction potential and polarization energy
// (Sec. 3.5) and surface area (Sec. 3.4), FP64.  These are N x Nc pair sums
// evaluated once per solve; all reductions are deterministic (per-block
// partials summed in a fixed order).
#include <vector>

#include "ibim_internal.cuh"

namespace ibim {

constexpr int kRhsThreads = 256;
constexpr int kRhsAtomTile = 256;

// g1_i = sum_k q_k/eps_I G0(x*_i, z_k);  g2_i = sum_k q_k/eps_I dG0(x*_i, z_k)/dn(x*_i),
// dG0(x, z)/dn(x) = -(x - z).n / (4 pi |x - z|^3).
__global__ void __launch_bounds__(kRhsThreads)
    rhs_kernel(const double* __restrict__ geo, int64_t N, const double* __restrict__ z,
               const double* __restrict__ q, int64_t Nc, double inv_eps_in, double* __restrict__ g)
{
    __shared__ double sz[kRhsAtomTile][4];
    const int64_t i = (int64_t)blockIdx.x * kRhsThreads + threadIdx.x;
    double x0 = 0, x1 = 0, x2 = 0, n0 = 0, n1 = 0, n2 = 0;
    if (i < N) {
        x0 = geo[i];
        x1 = geo[N + i];
        x2 = geo[2 * N + i];
        n0 = geo[3 * N + i];
        n1 = geo[4 * N + i];
        n2 = geo[5 * N + i];
    }
    double g1 = 0.0, g2 = 0.0;
    for (int64_t k0 = 0; k0 < Nc; k0 += kRhsAtomTile) {
        const int cnt = (int)((Nc - k0 < kRhsAtomTile) ? Nc - k0 : kRhsAtomTile);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += kRhsThreads) {
            sz[t][0] = z[3 * (k0 + t)];
            sz[t][1] = z[3 * (k0 + t) + 1];
            sz[t][2] = z[3 * (k0 + t) + 2];
            sz[t][3] = q[k0 + t];
        }
        __syncthreads();
        if (i < N) {
            for (int t = 0; t < cnt; ++t) {
                const double r0 = x0 - sz[t][0], r1 = x1 - sz[t][1], r2 = x2 - sz[t][2];
                const double rr = r0 * r0 + r1 * r1 + r2 * r2;
                const double inv = rsqrt(rr);
                const double sn = r0 * n0 + r1 * n1 + r2 * n2;
                g1 += sz[t][3] * inv;
                g2 -= sz[t][3] * sn * inv * inv * inv;
            }
        }
    }
    if (i < N) {
        g[i] = kInv4Pi * inv_eps_in * g1;
        g[N + i] = kInv4Pi * inv_eps_in * g2;
    }
}

ibim_status rhs_launch(ibim_ctx* c, double eps_in, double* d_g)
{
    const int64_t N = c->N;
    rhs_kernel<<<(unsigned)((N + kRhsThreads - 1) / kRhsThreads), kRhsThreads, 0, c->stream>>>(
        c->d_geo64, N, c->d_z, c->d_q, c->Nc, 1.0 / eps_in, d_g);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

// psi_rxn(z_k) = sum_j w_j [ (th1 A - 1) s_y / (4 pi rho^3) psi_j + (1 - E)/(4 pi rho) psin_j ],
// r = z_k - y*_j, s_y = r.n(y*_j), E = exp(-kappa rho), A = E (1 + kappa rho).
// Grid: (atom groups of kEnAtoms) x (node splits); each CTA writes one partial per atom.
constexpr int kEnThreads = 256;
constexpr int kEnAtoms = 4;

__global__ void __launch_bounds__(kEnThreads)
    energy_partial_kernel(const double* __restrict__ geo, int64_t N, const double* __restrict__ z, int64_t Nc,
                          const double* __restrict__ p, double th1, double kappa, int64_t chunk,
                          double* __restrict__ part)
{
    __shared__ double red[kEnThreads / 32][kEnAtoms];
    const int64_t a0 = (int64_t)blockIdx.x * kEnAtoms;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = (j0 + chunk < N) ? j0 + chunk : N;
    double zx[kEnAtoms], zy[kEnAtoms], zz[kEnAtoms], acc[kEnAtoms];
#pragma unroll
    for (int a = 0; a < kEnAtoms; ++a) {
        const int64_t k = (a0 + a < Nc) ? a0 + a : Nc - 1;
        zx[a] = z[3 * k];
        zy[a] = z[3 * k + 1];
        zz[a] = z[3 * k + 2];
        acc[a] = 0.0;
    }
    for (int64_t j = j0 + threadIdx.x; j < j1; j += kEnThreads) {
        const double y0 = geo[j], y1 = geo[N + j], y2 = geo[2 * N + j];
        const double m0 = geo[3 * N + j], m1 = geo[4 * N + j], m2 = geo[5 * N + j];
        const double w = geo[6 * N + j];
        const double a = w * p[j], b = w * p[N + j];
#pragma unroll
        for (int q = 0; q < kEnAtoms; ++q) {
            const double r0 = zx[q] - y0, r1 = zy[q] - y1, r2 = zz[q] - y2;
            const double rr = r0 * r0 + r1 * r1 + r2 * r2;
            const double inv = rsqrt(rr);
            const double rho = rr * inv;
            const double E = exp(-kappa * rho);
            const double A = E * (1.0 + kappa * rho);
            const double sy = r0 * m0 + r1 * m1 + r2 * m2;
            acc[q] += (th1 * A - 1.0) * sy * inv * inv * inv * a + (1.0 - E) * inv * b;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kEnAtoms; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kEnAtoms) {
        double v = 0.0;
        for (int w = 0; w < kEnThreads / 32; ++w) v += red[w][threadIdx.x];
        const int64_t k = a0 + threadIdx.x;
        if (k < Nc) part[(int64_t)blockIdx.y * Nc + k] = v;
    }
}

// psi_rxn[k] = (1/(4 pi)) sum_splits part; out[0] = G_pol = 1/2 sum q_k psi_rxn[k].
__global__ void energy_final_kernel(const double* __restrict__ part, int64_t nsplit, int64_t Nc,
                                    const double* __restrict__ q, double* __restrict__ psi, double* __restrict__ out)
{
    __shared__ double red[1024];
    double g = 0.0;
    for (int64_t k = threadIdx.x; k < Nc; k += blockDim.x) {
        double v = 0.0;
        for (int64_t s = 0; s < nsplit; ++s) v += part[s * Nc + k];
        v *= kInv4Pi;
        if (psi != nullptr) psi[k] = v;
        g += q[k] * v;
    }
    red[threadIdx.x] = g;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * red[0];
}

ibim_status energy_launch(ibim_ctx* c, const ibim_phys& p, const double* d_p, double* d_psi, double* gpol_host)
{
    const int64_t N = c->N, Nc = c->Nc;
    const int64_t groups = (Nc + kEnAtoms - 1) / kEnAtoms;
    int64_t nsplit = (4LL * c->num_sms + groups - 1) / groups;
    const int64_t maxsplit = (N + kEnThreads - 1) / kEnThreads;
    if (nsplit > maxsplit) nsplit = maxsplit;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 65535) nsplit = 65535;
    const int64_t chunk = (N + nsplit - 1) / nsplit;
    IBIM_TRY(ensure(c, (void**)&c->d_red, &c->red_bytes, sizeof(double) * (nsplit * Nc + 8)));
    double* part = c->d_red + 8;
    dim3 grid((unsigned)groups, (unsigned)nsplit);
    energy_partial_kernel<<<grid, kEnThreads, 0, c->stream>>>(c->d_geo64, N, c->d_z, Nc, d_p,
                                                             p.eps_out / p.eps_in, p.kappa, chunk, part);
    energy_final_kernel<<<1, 1024, 0, c->stream>>>(part, nsplit, Nc, c->d_q, d_psi, c->d_red);
    count_launch(c, 2);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemcpyAsync(gpol_host, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

// Surface area: sum_j w_j (Sec. 3.4), deterministic two-level sum.
__global__ void area_kernel(const double* __restrict__ w, int64_t N, double* __restrict__ out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) s += w[j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

ibim_status area_launch(ibim_ctx* c, double* area_host)
{
    IBIM_TRY(ensure(c, (void**)&c->d_red, &c->red_bytes, sizeof(double) * 8));
    area_kernel<<<1, 1024, 0, c->stream>>>(c->d_geo64 + 6 * c->N, c->N, c->d_red + 1);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(cudaMemcpyAsync(area_host, c->d_red + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    return IBIM_OK;
}

}  // namespace ibim
