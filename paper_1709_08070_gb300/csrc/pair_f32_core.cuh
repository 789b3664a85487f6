// Pair arithmetic of the FP32 compensated operator, shared by the
// single-molecule and batched pair-sum kernels.  See pair_f32.cu for the
// formulas, the chunk frames, the near/far split and the accumulation.
#pragma once
#include "ibim_internal.cuh"
#include "ptx.cuh"

namespace ibim {

struct F32Consts {
    float th1, th2, omth1, omth2;
    float kappa, kl2e;        // kappa and -kappa log2(e)
    float tau2, four_tau2, k12t;
    float far_dist;           // minimum bounding-sphere gap of a far step (A)
    int rule0;                // tube rule 0 (far steps allowed)
    double tau2_d, four_tau2_d;  // the tube thresholds in FP64 (near-tie decisions)
};

// FP64 node coordinates for re-deciding near-ties of the tube test:
// component a of node i is x[i * si + a * sa] (same for the normals n).
struct Geo64 {
    const double* x;
    const double* n;
    int64_t si, sa;
};

inline F32Consts f32_consts(const PairConsts& k)
{
    F32Consts c;
    c.th1 = (float)k.th1;
    c.th2 = (float)k.th2;
    c.omth1 = (float)(1.0 - k.th1);
    c.omth2 = (float)(1.0 - k.th2);
    c.kappa = (float)k.kappa;
    c.kl2e = (float)(-k.kappa * 1.4426950408889634);
    c.tau2 = (float)k.tau2;
    c.rule0 = (k.four_tau2 < 3.0e38) ? 1 : 0;
    c.four_tau2 = c.rule0 ? (float)k.four_tau2 : __builtin_huge_valf();
    c.k12t = (float)k.k12_tube;
    c.tau2_d = k.tau2;
    c.four_tau2_d = k.four_tau2;
    const double two_tau = 2.0 * sqrt(k.tau2);
    c.far_dist = (float)((two_tau > 1.5 ? two_tau : 1.5) * 1.001 + 1e-3);
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

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kChunk = 32;  // chunk = frame block = compensation unit

// Far pair: no tube, exp-form g.  Accumulates into t1, t2.
__device__ __forceinline__ void pair_far(const float3& xi, const float3& ni, const float4& y, const float4& m,
                                         const F32Consts& k, float& t1, float& t2)
{
    const float rx = xi.x - y.x, ry = xi.y - y.y, rz = xi.z - y.z;
    const float rr = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float sx = fmaf(rx, ni.x, fmaf(ry, ni.y, rz * ni.z));
    const float sy = fmaf(rx, m.x, fmaf(ry, m.y, rz * m.z));
    const float cc = fmaf(ni.x, m.x, fmaf(ni.y, m.y, ni.z * m.z));
    const float inv = ptx::rsqrt_approx(rr);
    const float rho = rr * inv;
    const float x = k.kappa * rho;
    const float E = ptx::ex2_approx(rho * k.kl2e);
    const float Ex = E * x;
    const float f = 1.0f - E;
    const float g = f - Ex;
    const float hh = fmaf(3.0f, g, -Ex * x);
    const float inv2 = inv * inv;
    const float inv3 = inv2 * inv;
    const float u1 = fmaf(k.th1, g, k.omth1);
    const float u2 = fmaf(k.th2, g, k.omth2);
    const float A1 = inv3 * y.w;
    t1 = fmaf(sy * u1, A1, t1);
    t1 = fmaf(-f, inv * m.w, t1);
    const float w21 = fmaf(g, cc, -(hh * sx) * (sy * inv2));
    t2 = fmaf(w21, A1, t2);
    t2 = fmaf(sx * u2, inv3 * m.w, t2);
}

// All interactions of the warp's targets with one staged source tile (cnt
// nodes at sb, chunk frames at sfrm).  xi/ni: targets in their block frame,
// bh/bl: the target blocks' frames (radius in bh.w).  Adds the tile's sums
// to the compensated pairs (S, C).
// Tube test of one pair in FP64 from the FP64 coordinates of target i and
// source j (the oracle's definition): used when the FP32 test is within
// rounding of a threshold, so that near-ties are decided as in FP64.
static __device__ __noinline__ bool tube_f64(const Geo64& g, int64_t i, int64_t j, double tau2, double four_tau2)
{
    double r[3], nx[3];
    for (int a = 0; a < 3; ++a) {
        r[a] = g.x[i * g.si + a * g.sa] - g.x[j * g.si + a * g.sa];
        nx[a] = g.n[i * g.si + a * g.sa];
    }
    const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double sx = r[0] * nx[0] + r[1] * nx[1] + r[2] * nx[2];
    return (rr - sx * sx < tau2) && (rr < four_tau2);
}

// Relative width of the band around the tube thresholds inside which the
// FP32 tube test defers to tube_f64.
constexpr float kTieBand = 1e-5f;

template <int TPT>
__device__ __forceinline__ void tile_sums(const float3 (&xi)[TPT], const float3 (&ni)[TPT], const float4 (&bh)[TPT],
                                          const float3 (&bl)[TPT], bool have_frames, const float4* sb,
                                          const float4* sfrm, int cnt, const F32Consts& k, float (&S1)[TPT],
                                          float (&C1)[TPT], float (&S2)[TPT], float (&C2)[TPT], const Geo64& g64,
                                          const int64_t (&gi)[TPT], int64_t j0)
{
    for (int c0 = 0; c0 < cnt; c0 += kChunk) {
        const int c1 = (c0 + kChunk < cnt) ? c0 + kChunk : cnt;
        // targets in the source chunk's frame; far test on the two bounding spheres
        float3 X[TPT];
        bool far = have_frames && k.rule0;
        if (have_frames) {
            const float4 mh = sfrm[2 * (c0 / kChunk)];
            const float4 ml = sfrm[2 * (c0 / kChunk) + 1];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                const float dx = (bh[q].x - mh.x) + (bl[q].x - ml.x);
                const float dy = (bh[q].y - mh.y) + (bl[q].y - ml.y);
                const float dz = (bh[q].z - mh.z) + (bl[q].z - ml.z);
                X[q] = make_float3(xi[q].x + dx, xi[q].y + dy, xi[q].z + dz);
                const float lim = k.far_dist + bh[q].w + mh.w;
                far = far && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim);
            }
        } else {
#pragma unroll
            for (int q = 0; q < TPT; ++q) X[q] = xi[q];
        }
        float t1[TPT], t2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = 0.0f;
        if (far) {
#pragma unroll 4
            for (int j = c0; j < c1; ++j) {
                const float4 y = sb[2 * j];
                const float4 m = sb[2 * j + 1];
#pragma unroll
                for (int q = 0; q < TPT; ++q) pair_far(X[q], ni[q], y, m, k, t1[q], t2[q]);
            }
        } else {
            for (int j = c0; j < c1; ++j) {
                const float4 y = sb[2 * j];
                const float4 m = sb[2 * j + 1];
                float rr[TPT], sx[TPT], sy[TPT], cc[TPT], inv[TPT], x[TPT], E[TPT];
                bool tube[TPT];
                bool need = false;
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    const float rx = X[q].x - y.x, ry = X[q].y - y.y, rz = X[q].z - y.z;
                    rr[q] = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    sx[q] = fmaf(rx, ni[q].x, fmaf(ry, ni[q].y, rz * ni[q].z));
                    sy[q] = fmaf(rx, m.x, fmaf(ry, m.y, rz * m.z));
                    cc[q] = fmaf(ni[q].x, m.x, fmaf(ni[q].y, m.y, ni[q].z * m.z));
                    const float rp2 = fmaf(-sx[q], sx[q], rr[q]);
                    tube[q] = (rp2 < k.tau2) & (rr[q] < k.four_tau2);
                    const bool tie = (fabsf(rp2 - k.tau2) < kTieBand * k.tau2) |
                                     (fabsf(rr[q] - k.four_tau2) < kTieBand * k.four_tau2);
                    if (tie && g64.x != nullptr) tube[q] = tube_f64(g64, gi[q], j0 + j, k.tau2_d, k.four_tau2_d);
                    const float rrs = fmaxf(rr[q], 1.0e-30f);
                    inv[q] = ptx::rsqrt_approx(rrs);
                    const float rho = rrs * inv[q];
                    x[q] = k.kappa * rho;
                    E[q] = ptx::ex2_approx(rho * k.kl2e);
                    need |= (x[q] < 0.5f);
                }
                const bool series = __any_sync(0xffffffffu, need);
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
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
                    const float A1 = i3 * y.w;
                    t1[q] = fmaf(sy[q] * u1, A1, t1[q]);
                    t1[q] = fmaf(-Q, m.w, t1[q]);
                    const float w21 = fmaf(g, cc[q], -(hh * sx[q]) * (sy[q] * inv2));
                    t2[q] = fmaf(w21, A1, t2[q]);
                    t2[q] = fmaf(sx[q] * u2, i3 * m.w, t2[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            kahan_add(S1[q], C1[q], t1[q]);
            kahan_add(S2[q], C2[q], t2[q]);
        }
    }
}

}  // namespace ibim
