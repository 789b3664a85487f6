// Plain FP64 pair sums of the IBIM operator (Sec. 2.2 discrete system,
// Sec. 2.2.1 regularisation), sm_103a.  Same stream-K schedule and partial
// layout as the FP32 path; one target per thread, kF64STile source nodes
// (64 B each: y*, w psi, n(y*), w psin) per shared-memory stage.  The kernels
// are evaluated directly from their definitions (times 4 pi):
//   K11 = s_y (1 - th1 A)/rho^3, K12 = (1 - E)/rho,
//   K21 = [(1 - A) c - (3 - B) s_x s_y/rho^2]/rho^3, K22 = -s_x (1 - th2 A)/rho^3.
#include "ibim_internal.cuh"
#include "ptx.cuh"

namespace ibim {

struct F64Consts {
    double th1, th2, kappa, tau2, four_tau2, k12t;
};

constexpr uint64_t kWaitLimitNs64 = 2000000000ull;  // 2 s
constexpr int kF64Stages = 2;

__global__ void __launch_bounds__(kF64Threads)
    pair_f64_kernel(const double* __restrict__ geo, const double* __restrict__ src, int64_t N,
                    PairSchedule s, F64Consts k, double* __restrict__ part,
                    unsigned* __restrict__ err, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) double sbuf[kF64Stages][8 * kF64STile];
    __shared__ __align__(8) uint64_t bars[kF64Stages];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * s.per_cta;
    const int64_t s1 = (s0 + s.per_cta < s.total) ? s0 + s.per_cta : s.total;
    if (s0 >= s1) return;
    if (tid == 0) {
        for (int q = 0; q < kF64Stages; ++q) ptx::mbar_init(&bars[q], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int64_t u) {
        const int64_t st = u % s.n_stiles;
        const int64_t j0 = st * kF64STile;
        const int64_t cnt = (N - j0 < kF64STile) ? N - j0 : kF64STile;
        const int stage = (int)((u - s0) % kF64Stages);
        const uint32_t bytes = (uint32_t)(cnt * 8 * sizeof(double));
        ptx::mbar_arrive_expect_tx(&bars[stage], bytes);
        ptx::bulk_g2s(&sbuf[stage][0], src + 8 * j0, bytes, &bars[stage]);
    };
    if (tid == 0)
        for (int q = 0; q < kF64Stages && s0 + q < s1; ++q) issue(s0 + q);

    const int64_t t_first = s0 / s.n_stiles;
    int64_t t = t_first;
    double x0, x1, x2, n0, n1, n2, D1 = 0.0, D2 = 0.0;
    auto load_target = [&](int64_t tile) {
        const int64_t i = tile * kF64TTile + tid;
        if (i < N) {
            x0 = geo[i];
            x1 = geo[N + i];
            x2 = geo[2 * N + i];
            n0 = geo[3 * N + i];
            n1 = geo[4 * N + i];
            n2 = geo[5 * N + i];
        } else {
            x0 = x1 = x2 = 1.0e6;
            n0 = n1 = 0.0;
            n2 = 1.0;
        }
        D1 = D2 = 0.0;
    };
    load_target(t);

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kF64Stages);
        const uint32_t parity = (uint32_t)(((u - s0) / kF64Stages) & 1);
        if (!ptx::mbar_wait_bounded(&bars[stage], parity, kWaitLimitNs64)) {
            abort_flag = 1;
            atomicOr(err, kDevErrTimeout);
        }
        __syncthreads();
        if (abort_flag) return;
        const int64_t st = u % s.n_stiles;
        const int64_t j0 = st * kF64STile;
        const int cnt = (int)((N - j0 < kF64STile) ? N - j0 : kF64STile);
        const double* sb = &sbuf[stage][0];
        for (int j = 0; j < cnt; ++j) {
            const double* e = sb + 8 * j;
            const double r0 = x0 - e[0], r1 = x1 - e[1], r2 = x2 - e[2];
            const double a = e[3], b = e[7];
            const double rr = r0 * r0 + r1 * r1 + r2 * r2;
            const double sx = r0 * n0 + r1 * n1 + r2 * n2;
            const double rp2 = rr - sx * sx;
            if (rp2 < k.tau2 && rr < k.four_tau2) {
                D1 -= k.k12t * b;
                continue;
            }
            const double sy = r0 * e[4] + r1 * e[5] + r2 * e[6];
            const double cc = n0 * e[4] + n1 * e[5] + n2 * e[6];
            const double inv = rsqrt(rr);
            const double rho = rr * inv;
            const double xk = k.kappa * rho;
            const double E = exp(-xk);
            const double A = E * (1.0 + xk);
            const double B = E * (3.0 + 3.0 * xk + xk * xk);
            const double inv3 = inv * inv * inv;
            const double K11 = sy * (1.0 - k.th1 * A) * inv3;
            const double K12 = (1.0 - E) * inv;
            const double K21 = ((1.0 - A) * cc - (3.0 - B) * sx * sy * inv * inv) * inv3;
            const double K22 = -sx * (1.0 - k.th2 * A) * inv3;
            D1 += K11 * a - K12 * b;
            D2 += K21 * a - K22 * b;
        }
        __syncthreads();
        if (tid == 0 && u + kF64Stages < s1) {
            ptx::fence_proxy_async_smem();
            issue(u + kF64Stages);
        }
        if (st == s.n_stiles - 1 || u + 1 == s1) {
            const int seg = (int)(t - t_first);
            double* dst = part + ((int64_t)blockIdx.x * s.max_segs + seg) * 2 * kF64TTile;
            dst[tid] = D1;
            dst[kF64TTile + tid] = D2;
            if (st == s.n_stiles - 1 && u + 1 < s1) {
                ++t;
                load_target(t);
            }
        }
    }
}

// Source payload: node j -> (x*, y*, z*, w psi, nx, ny, nz, w psin), FP64.
__global__ void pack_f64_kernel(const double* __restrict__ geo, VecRef in, int64_t N,
                                double* __restrict__ src, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    const double w = geo[6 * N + j];
    double* d = src + 8 * j;
    d[0] = geo[j];
    d[1] = geo[N + j];
    d[2] = geo[2 * N + j];
    d[3] = w * p[j];
    d[4] = geo[3 * N + j];
    d[5] = geo[4 * N + j];
    d[6] = geo[5 * N + j];
    d[7] = w * p[N + j];
}

int f64_grid_cap(ibim_ctx* c)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_f64_kernel, kF64Threads, 0);
    if (occ < 1) occ = 1;
    return occ * c->num_sms;
}

ibim_status f64_pack(ibim_ctx* c, VecRef in, const int* d_skip)
{
    const int64_t N = c->N;
    IBIM_TRY(ensure(c, &c->d_src, &c->src_bytes, (size_t)N * 8 * sizeof(double)));
    const int bs = 256;
    pack_f64_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, c->stream>>>(c->d_geo64, in, N,
                                                                          (double*)c->d_src, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status f64_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip)
{
    const size_t need = (size_t)s.grid * s.max_segs * 2 * kF64TTile * sizeof(double);
    IBIM_TRY(ensure(c, (void**)&c->d_part, &c->part_bytes, need));
    F64Consts kk;
    kk.th1 = k.th1;
    kk.th2 = k.th2;
    kk.kappa = k.kappa;
    kk.tau2 = k.tau2;
    kk.four_tau2 = k.four_tau2;
    kk.k12t = k.k12_tube;
    pair_f64_kernel<<<s.grid, kF64Threads, 0, c->stream>>>(c->d_geo64, (const double*)c->d_src, c->N,
                                                            s, kk, c->d_part, c->d_err, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status fixup_launch(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, int ttile, VecRef in,
                         OutRef out, const int* d_skip);

ibim_status f64_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                      const int* d_skip)
{
    return fixup_launch(c, k, s, kF64TTile, in, out, d_skip);
}

}  // namespace ibim
