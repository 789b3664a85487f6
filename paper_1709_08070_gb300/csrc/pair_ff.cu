// Float-float ("double-single") pair sums of the IBIM operator (Sec. 2.2
// discrete system, Sec. 2.2.1 regularisation) on the FP32 pipe, sm_103a.
//
// Purpose: an operator as accurate as the plain FP64 path (it is held to the
// same 1e-10 element bar against the FP64 oracle) that runs on the GB300's
// FP32 pipe instead of its FP64 pipe, which has a small fraction of the FP32
// rate.  The certification of an FP32 solve (one residual g - A p with an
// FP64-accurate operator) uses it.
//
// Every quantity is an unevaluated sum h + l of two floats (about 48
// significant bits), built from error-free transformations: Knuth's two-sum
// (s + e == a + b exactly) and the FMA two-product (p + e == a b exactly);
// products drop the l l' term (relative 2^-48) and sums renormalise with
// Dekker's fast two-sum where the result is accumulated.
//
//   * Positions.  Node coordinates relative to the molecule centroid are
//     split as x = xh + xl with xh on a power-of-two grid 2^-q fine enough
//     that |x| 2^q < 2^23; the difference of two hi parts is then exact, and
//     r = (xh - yh) + (xl - yl) carries about 2^-41 of the box size.
//   * 1/rho: the MUFU estimate y0 of rsqrt(|r|^2) refined by one Newton step
//     in float-float, y0 (1 - d/2 + 3 d^2/8) with 1 + d = |r|^2 y0^2.
//   * E = exp(-kappa rho): Tang's table-driven method (ACM TOMS 15, 1989):
//     z = -kappa rho log2(e) = k/256 + f with |f| <= 1/512, 2^(k/256) from a
//     256-entry float-float table (2^(i/256), i = 0..255, computed with FP64
//     exp2 on the device), e^(f ln 2) from its Taylor series (the terms past
//     the linear one in FP32), and the power 2^floor(k/256) put into the
//     exponent bits.  z is clamped at -120 (E < 1e-36 there).
//   * Kernels (times 4 pi), with g = 1 - A = (1 - E) - E x, 3 - B = 3 g - E x^2:
//       y1 += s_y (1 - th1 A) a / rho^3 - (1 - E) b / rho
//       y2 += [(g c - (3 - B) s_x s_y / rho^2) a + s_x (1 - th2 A) b] / rho^3
//     and inside the tube (near chunks only) y1 -= K12_tube b.
//   * Tube test (Sec. 2.2.1) in float-float; a pair within 1e-9 (relative)
//     of a threshold is decided again in FP64 with the oracle's operation
//     order, so ties fall as they do in FP64.
//   * Sums: float-float per target over a source tile (renormalised per
//     pair), FP64 across tiles, FP64 partials per (CTA, target tile) summed by
//     the FP32 path's fixup kernel in a fixed order.
//
// Schedule: the one-directional stream-K walk of pair_f32.cu (persistent
// CTAs, source tiles in the golden-ratio order of each row), one target per
// thread, 256-source tiles through two shared-memory stages filled by bulk
// async copies; chunk pairs whose bounding spheres are at least the far
// distance apart skip the tube test, as in the FP32 kernel.
#include "pair_sym_core.cuh"

namespace ibim {

constexpr int kFFThreads = 256;  // one target per thread
constexpr int kFFTTile = kFFThreads;
constexpr int kFFSTile = 256;    // sources per stage
constexpr int kFFStages = 2;
constexpr int kFFChunk = 32;
constexpr int kFFChunksPerTile = kFFSTile / kFFChunk;
constexpr int kFFTab = 256;      // table of 2^(i/256)
constexpr uint64_t kFFWaitNs = 2000000000ull;  // 2 s
static_assert(kPadNodes % kFFSTile == 0 && kPadNodes % kFFTTile == 0, "padding");
// payload per node: (xh, ah), (xl, al), (nh, bh), (nl, bl), stored per aligned
// 32-node chunk component by component (the chunk's 32 first float4, then its
// 32 second ones, ...), so that 32 lanes reading 32 different nodes of a chunk
// touch 512 contiguous bytes
constexpr int kFFNodeF4 = 4;
__host__ __device__ __forceinline__ int64_t ff_off(int64_t j, int comp)
{
    return (j >> 5) * (32 * kFFNodeF4) + comp * 32 + (j & 31);
}
constexpr uint32_t kFFStageBytes = kFFSTile * kFFNodeF4 * sizeof(float4);
constexpr uint32_t kFFFrameBytes = 2 * kFFChunksPerTile * sizeof(float4);
constexpr float kFFPad = 1.0e4f;  // placeholder coordinate (sources +, targets -)

// ------------------------------------------------------ float-float arithmetic

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_of(float2 v) { return ff{v.x, v.y}; }

// Knuth's two-sum: s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

// Dekker's fast two-sum (exact when |a| >= |b|, or a == 0).
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a b with the l l' term dropped (result nearly normalised).
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff{p, e};
}

// a b for a plain float b.
__device__ __forceinline__ ff ff_mulf(ff a, float b)
{
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return ff{p, e};
}

// a + b, renormalised (absolute error about 2^-47 max(|a|, |b|)).
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.h, -b.l}); }

// a0 b0 + a1 b1 + a2 b2 for float-float vectors (the l l' terms dropped).
__device__ __forceinline__ ff ff_dot3(float ah0, float al0, float ah1, float al1, float ah2, float al2, float bh0,
                                      float bl0, float bh1, float bl1, float bh2, float bl2)
{
    const ff p0 = ff_mul(ff{ah0, al0}, ff{bh0, bl0});
    const ff p1 = ff_mul(ff{ah1, al1}, ff{bh1, bl1});
    const ff p2 = ff_mul(ff{ah2, al2}, ff{bh2, bl2});
    const ff s = two_sum(p0.h, p1.h);
    const ff t = two_sum(s.h, p2.h);
    const float lo = __fadd_rn(__fadd_rn(s.l, t.l), __fadd_rn(__fadd_rn(p0.l, p1.l), p2.l));
    return fast_two_sum(t.h, lo);
}

// (h + l)^2 summed over three components.
__device__ __forceinline__ ff ff_norm2(float h0, float l0, float h1, float l1, float h2, float l2)
{
    const float p0 = __fmul_rn(h0, h0), p1 = __fmul_rn(h1, h1), p2 = __fmul_rn(h2, h2);
    // (h + l)^2 - h h rounded = fma error of h h + (2 h + l) l
    const float e0 = __fmaf_rn(__fmaf_rn(2.0f, h0, l0), l0, __fmaf_rn(h0, h0, -p0));
    const float e1 = __fmaf_rn(__fmaf_rn(2.0f, h1, l1), l1, __fmaf_rn(h1, h1, -p1));
    const float e2 = __fmaf_rn(__fmaf_rn(2.0f, h2, l2), l2, __fmaf_rn(h2, h2, -p2));
    const ff s = two_sum(p0, p1);
    const ff t = two_sum(s.h, p2);
    const float lo = __fadd_rn(__fadd_rn(s.l, t.l), __fadd_rn(__fadd_rn(e0, e1), e2));
    return fast_two_sum(t.h, lo);
}

// 2^z for z <= 0 (float-float), Tang's table-driven reduction; tab[i] = 2^(i/256).
__device__ __forceinline__ ff ff_exp2(ff z, const float2* __restrict__ tab)
{
    const bool clamp = z.h < -120.0f;
    const float zh = clamp ? -120.0f : z.h;
    const float zl = clamp ? 0.0f : z.l;
    // round(zh 256) sits in the low mantissa bits of zh 256 + 1.5 2^23
    const float t = __fmaf_rn(zh, 256.0f, 12582912.0f);
    const int ki = __float_as_int(t) - 0x4B400000;
    const float kf = __fsub_rn(t, 12582912.0f);
    const float fh = __fmaf_rn(kf, -0.00390625f, zh);  // zh - k/256, exact, |fh| <= 1/512
    // u = (fh + zl) ln 2, |u| <= 0.00136
    const float L2h = 0.693147182464599609375f, L2l = -1.904654323148236e-09f;
    const float uh = __fmul_rn(fh, L2h);
    float ul = __fmaf_rn(fh, L2h, -uh);
    ul = __fmaf_rn(fh, L2l, ul);
    ul = __fmaf_rn(zl, L2h, ul);
    // e^u = 1 + u + u^2 (1/2 + u/6 + u^2/24) + O(u^5)
    float q = __fmaf_rn(uh, 1.0f / 24.0f, 1.0f / 6.0f);
    q = __fmaf_rn(uh, q, 0.5f);
    const float P = __fmul_rn(__fmul_rn(uh, uh), q);
    const float s = __fadd_rn(1.0f, uh);
    const float el = __fsub_rn(uh, __fsub_rn(s, 1.0f));
    const float lo = __fadd_rn(el, __fadd_rn(ul, P));
    const float2 T = tab[ki & (kFFTab - 1)];
    const ff m = ff_mul(ff{T.x, T.y}, ff{s, lo});
    const float sc = __int_as_float(((ki >> 8) + 127) << 23);  // 2^floor(k / 256), k >= -30720
    return ff{__fmul_rn(m.h, sc), __fmul_rn(m.l, sc)};
}

// ---------------------------------------------------------------- constants

struct FFConsts {
    float2 kap, cz;          // kappa and -kappa log2(e)
    float2 th1, th2;         // eps_E/eps_I, eps_I/eps_E
    float2 om1, om2;         // 1 - th1, 1 - th2
    float2 nk12t;            // -(4 pi x tube value of K12)
    float2 tau2, four_tau2;  // tube thresholds
    double tau2_d, four_tau2_d;
    float far_dist;          // minimum bounding-sphere gap of a far chunk pair (A)
    int rule0;
};

static float2 split(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

static FFConsts ff_consts(const PairConsts& k)
{
    FFConsts c;
    c.kap = split(k.kappa);
    c.cz = split(-k.kappa * 1.4426950408889634074);
    c.th1 = split(k.th1);
    c.th2 = split(k.th2);
    c.om1 = split(1.0 - k.th1);
    c.om2 = split(1.0 - k.th2);
    c.nk12t = split(-k.k12_tube);
    c.rule0 = (k.four_tau2 < 3.0e38) ? 1 : 0;
    c.tau2 = split(k.tau2);
    c.four_tau2 = c.rule0 ? split(k.four_tau2) : make_float2(__builtin_huge_valf(), 0.0f);
    c.tau2_d = k.tau2;
    c.four_tau2_d = k.four_tau2;
    const double two_tau = 2.0 * sqrt(k.tau2);
    c.far_dist = (float)((two_tau > 1.5 ? two_tau : 1.5) * 1.001 + 1e-3);
    return c;
}

// Tube test of one pair in FP64 with the oracle's operations in its order
// (no contraction): used for pairs within rounding of a threshold.
static __device__ __noinline__ bool tube_f64_ordered(const double* __restrict__ geo, int64_t N, int64_t i, int64_t j,
                                                     double tau2, double four_tau2)
{
    const double r0 = __dsub_rn(geo[i], geo[j]);
    const double r1 = __dsub_rn(geo[N + i], geo[N + j]);
    const double r2 = __dsub_rn(geo[2 * N + i], geo[2 * N + j]);
    const double rho2 = __dadd_rn(__dadd_rn(__dmul_rn(r0, r0), __dmul_rn(r1, r1)), __dmul_rn(r2, r2));
    const double sx = __dadd_rn(__dadd_rn(__dmul_rn(r0, geo[3 * N + i]), __dmul_rn(r1, geo[4 * N + i])),
                                __dmul_rn(r2, geo[5 * N + i]));
    const double rp2 = __dsub_rn(rho2, __dmul_rn(sx, sx));
    return (rp2 < tau2) && (rho2 < four_tau2);
}

// ---------------------------------------------------------------- pair

struct FFTarget {
    float xh0, xh1, xh2, xl0, xl1, xl2;
    float nh0, nh1, nh2, nl0, nl1, nl2;
};

// One (target <- source) interaction added to (S1, S2).  NEAR: the pair may
// lie in the regularisation tube.
template <bool NEAR>
__device__ __forceinline__ void ff_pair(const FFTarget& T, const float4& F0, const float4& F1, const float4& F2,
                                        const float4& F3, const FFConsts& k, const float2* __restrict__ tab, ff& S1,
                                        ff& S2, const double* __restrict__ geo, int64_t i, int64_t j, int64_t N)
{
    // r = x - y: the hi parts share the grid, so their difference is exact
    const float rh0 = __fsub_rn(T.xh0, F0.x), rh1 = __fsub_rn(T.xh1, F0.y), rh2 = __fsub_rn(T.xh2, F0.z);
    const float rl0 = __fsub_rn(T.xl0, F1.x), rl1 = __fsub_rn(T.xl1, F1.y), rl2 = __fsub_rn(T.xl2, F1.z);
    const ff rr = ff_norm2(rh0, rl0, rh1, rl1, rh2, rl2);
    const ff sx = ff_dot3(rh0, rl0, rh1, rl1, rh2, rl2, T.nh0, T.nl0, T.nh1, T.nl1, T.nh2, T.nl2);
    const ff b = ff{F2.w, F3.w};
    if (NEAR) {
        // rho_P^2 = |r|^2 - s_x^2 < tau^2 and |r|^2 < 4 tau^2 (tube rule 0)
        const ff sx2 = ff_mul(sx, sx);
        const ff rp2 = ff_sub(rr, sx2);
        const float d1 = __fadd_rn(__fsub_rn(rp2.h, k.tau2.x), __fsub_rn(rp2.l, k.tau2.y));
        const float d2 = __fadd_rn(__fsub_rn(rr.h, k.four_tau2.x), __fsub_rn(rr.l, k.four_tau2.y));
        bool tube = (d1 < 0.0f) && (d2 < 0.0f);
        const bool tie = (fabsf(d1) < 1e-9f * k.tau2.x) || (fabsf(d2) < 1e-9f * k.four_tau2.x);
        if (tie && i < N && j < N) tube = tube_f64_ordered(geo, N, i, j, k.tau2_d, k.four_tau2_d);
        if (tube) {
            const ff c = ff_mul(ff_of(k.nk12t), b);
            const ff s = two_sum(S1.h, c.h);
            S1 = fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(S1.l, c.l)));
            return;
        }
    }
    const ff sy = ff_dot3(rh0, rl0, rh1, rl1, rh2, rl2, F2.x, F3.x, F2.y, F3.y, F2.z, F3.z);
    const ff cc = ff_dot3(T.nh0, T.nl0, T.nh1, T.nl1, T.nh2, T.nl2, F2.x, F3.x, F2.y, F3.y, F2.z, F3.z);
    // 1/rho: MUFU estimate, one Newton step in float-float
    const float y0 = ptx::rsqrt_approx(rr.h);
    const ff q = ff_mul(rr, ff{__fmul_rn(y0, y0), __fmaf_rn(y0, y0, -__fmul_rn(y0, y0))});
    const float d = __fadd_rn(__fsub_rn(q.h, 1.0f), q.l);
    const ff inv = ff{y0, __fmul_rn(__fmul_rn(y0, d), __fmaf_rn(0.375f, d, -0.5f))};
    const ff rho = ff_mul(rr, inv);
    const ff x = ff_mul(ff_of(k.kap), rho);
    const ff E = ff_exp2(ff_mul(ff_of(k.cz), rho), tab);
    const ff Ex = ff_mul(E, x);
    // f = 1 - E (0 < E <= 1: fast two-sum of 1 and -E.h)
    const float fh = __fsub_rn(1.0f, E.h);
    const ff f = ff{fh, __fsub_rn(__fsub_rn(__fsub_rn(1.0f, fh), E.h), E.l)};
    const ff g = ff_sub(f, Ex);                               // 1 - A
    const ff u1 = ff_add(ff_of(k.om1), ff_mul(ff_of(k.th1), g));  // 1 - th1 A
    const ff u2 = ff_add(ff_of(k.om2), ff_mul(ff_of(k.th2), g));  // 1 - th2 A
    const ff hb = ff_sub(ff_mulf(g, 3.0f), ff_mul(Ex, x));     // 3 - B
    const ff inv2 = ff_mul(inv, inv);
    const ff inv3 = ff_mul(inv2, inv);
    const ff a = ff{F0.w, F1.w};
    const ff c1 = ff_sub(ff_mul(ff_mul(u1, ff_mul(sy, a)), inv3), ff_mul(ff_mul(f, inv), b));
    const ff br = ff_sub(ff_mul(g, cc), ff_mul(hb, ff_mul(ff_mul(sx, sy), inv2)));
    const ff c2 = ff_mul(ff_add(ff_mul(br, a), ff_mul(ff_mul(u2, sx), b)), inv3);
    const ff s1 = two_sum(S1.h, c1.h);
    S1 = fast_two_sum(s1.h, __fadd_rn(s1.l, __fadd_rn(S1.l, c1.l)));
    const ff s2 = two_sum(S2.h, c2.h);
    S2 = fast_two_sum(s2.h, __fadd_rn(s2.l, __fadd_rn(S2.l, c2.l)));
}

// ---------------------------------------------------------------- kernels

__global__ void __launch_bounds__(kFFThreads, 2)
    pair_ff_kernel(const float4* __restrict__ src, const float4* __restrict__ frames, const float2* __restrict__ tab_g,
                   const double* __restrict__ geo, int64_t N, PairSchedule s, FFConsts k, double* __restrict__ part,
                   unsigned* __restrict__ err, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) float4 sbuf[kFFStages][kFFSTile * kFFNodeF4];
    __shared__ __align__(16) float4 sfrm[kFFStages][2 * kFFChunksPerTile];
    __shared__ float2 tab[kFFTab];
    __shared__ __align__(8) uint64_t bars[kFFStages];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t s0 = (int64_t)blockIdx.x * s.per_cta;
    const int64_t s1 = (s0 + s.per_cta < s.total) ? s0 + s.per_cta : s.total;
    if (s0 >= s1) return;
    for (int q = tid; q < kFFTab; q += kFFThreads) tab[q] = tab_g[q];
    if (tid == 0) {
        for (int q = 0; q < kFFStages; ++q) ptx::mbar_init(&bars[q], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int64_t u) {
        const int64_t st = ((u % s.n_stiles) * s.sperm) % s.n_stiles;
        const int stage = (int)((u - s0) % kFFStages);
        ptx::mbar_arrive_expect_tx(&bars[stage], kFFStageBytes + kFFFrameBytes);
        ptx::bulk_g2s(&sbuf[stage][0], src + st * kFFSTile * kFFNodeF4, kFFStageBytes, &bars[stage]);
        ptx::bulk_g2s(&sfrm[stage][0], frames + st * 2 * kFFChunksPerTile, kFFFrameBytes, &bars[stage]);
    };
    if (tid == 0)
        for (int q = 0; q < kFFStages && s0 + q < s1; ++q) issue(s0 + q);

    const int64_t t_first = s0 / s.n_stiles;
    int64_t t = t_first;
    FFTarget T;
    float4 tfh, tfl;  // frame of the warp's target block
    int64_t gi = 0;
    bool idle = false;
    double D1 = 0.0, D2 = 0.0;
    auto load_target = [&](int64_t tile) {
        gi = tile * kFFTTile + tid;
        idle = tile * kFFTTile + warp * kFFChunk >= N;
        const float4 a = src[ff_off(gi, 0)], b = src[ff_off(gi, 1)];
        const float4 c = src[ff_off(gi, 2)], e = src[ff_off(gi, 3)];
        const bool pad = gi >= N;  // placeholder targets away from placeholder sources
        T.xh0 = pad ? -kFFPad : a.x;
        T.xh1 = pad ? -kFFPad : a.y;
        T.xh2 = pad ? -kFFPad : a.z;
        T.xl0 = pad ? 0.0f : b.x;
        T.xl1 = pad ? 0.0f : b.y;
        T.xl2 = pad ? 0.0f : b.z;
        T.nh0 = c.x;
        T.nh1 = c.y;
        T.nh2 = c.z;
        T.nl0 = e.x;
        T.nl1 = e.y;
        T.nl2 = e.z;
        const int64_t blk = (tile * kFFTTile + warp * kFFChunk) / kFFChunk;
        tfh = frames[2 * blk];
        tfl = frames[2 * blk + 1];
        D1 = D2 = 0.0;
    };
    load_target(t);

    for (int64_t u = s0; u < s1; ++u) {
        const int stage = (int)((u - s0) % kFFStages);
        const uint32_t parity = (uint32_t)(((u - s0) / kFFStages) & 1);
        if (!ptx::mbar_wait_bounded(&bars[stage], parity, kFFWaitNs)) {
            abort_flag = 1;
            atomicOr(err, kDevErrTimeout);
        }
        __syncthreads();
        if (abort_flag) return;
        const int64_t sp = u % s.n_stiles;
        const int64_t st = (sp * s.sperm) % s.n_stiles;
        if (!idle) {
            ff S1{0.0f, 0.0f}, S2{0.0f, 0.0f};
            const float4* sb = &sbuf[stage][0];
#pragma unroll 1
            for (int c = 0; c < kFFChunksPerTile; ++c) {
                // far chunk pair: the two blocks' bounding spheres are apart by more than the tube reaches
                const float4 mh = sfrm[stage][2 * c], ml = sfrm[stage][2 * c + 1];
                const float dx = (tfh.x - mh.x) + (tfl.x - ml.x);
                const float dy = (tfh.y - mh.y) + (tfl.y - ml.y);
                const float dz = (tfh.z - mh.z) + (tfl.z - ml.z);
                const float lim = k.far_dist + tfh.w + mh.w;
                const bool far = k.rule0 && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim);
                const float4* cb = sb + c * kFFChunk * kFFNodeF4;
                const int64_t j0 = st * kFFSTile + c * kFFChunk;
                if (far) {
#pragma unroll 2
                    for (int p = 0; p < kFFChunk; ++p)
                        ff_pair<false>(T, cb[p], cb[32 + p], cb[64 + p], cb[96 + p], k, tab, S1, S2, geo, gi, j0 + p,
                                       N);
                } else {
#pragma unroll 1
                    for (int p = 0; p < kFFChunk; ++p)
                        ff_pair<true>(T, cb[p], cb[32 + p], cb[64 + p], cb[96 + p], k, tab, S1, S2, geo, gi, j0 + p,
                                      N);
                }
            }
            D1 += (double)S1.h + (double)S1.l;
            D2 += (double)S2.h + (double)S2.l;
        }
        __syncthreads();
        if (tid == 0 && u + kFFStages < s1) {
            ptx::fence_proxy_async_smem();
            issue(u + kFFStages);
        }
        if (sp == s.n_stiles - 1 || u + 1 == s1) {
            const int seg = (int)(t - t_first);
            double* dst = part + ((int64_t)blockIdx.x * s.max_segs + seg) * 2 * kFFTTile;
            dst[tid] = D1;
            dst[kFFTTile + tid] = D2;
            if (sp == s.n_stiles - 1 && u + 1 < s1) {
                ++t;
                load_target(t);
            }
        }
    }
}

// ---------------------------------------------------------------- symmetric
//
// The same operator with each unordered node pair evaluated once for both
// directions (as the symmetric FP32 kernel of pair_sym.cu does): the shared
// float-float work (r, |r|^2, s_x, s_y, n . m, 1/rho, E, g, 1 - th A, 3 - B,
// the combination g c - (3 - B) s_x s_y / rho^2 and the powers of 1/rho) is
// done once, and the reverse direction (target j <- source i) is formed from
// it with r' = -r, s_x' = -s_y, s_y' = -s_x, c' = c:
//   forward   y1_i += u1 s_y a_j / rho^3 - (1 - E) b_j / rho
//             y2_i += [br a_j + u2 s_x b_j] / rho^3
//   reverse   y1_j += -u1 s_x a_i / rho^3 - (1 - E) b_i / rho
//             y2_j += [br a_i - u2 s_y b_i] / rho^3
// with br = g c - (3 - B) s_x s_y / rho^2.  Each direction takes its own tube
// test (the reverse one on the source's normal, rho_P'^2 = |r|^2 - s_y^2).
// 432 FP32 operations per unordered pair against 2 x 366.
//
// Per warp and source chunk the 32 lanes hold 32 targets and walk the chunk's
// 32 sources in a staggered order (lane l takes source (l + k) mod 32 at step
// k); the float-float reverse sums of a source ride along with it from lane to
// lane (four shuffles a step), so after 32 steps lane l holds source l's
// reverse sums over the warp's targets and adds them, as doubles, to the
// reverse vector with FP64 atomics.  Forward sums and the schedule (upper
// triangle, large and small segments, partials per (segment, row)) are those
// of the symmetric FP32 kernel, and its fixup adds everything up.

// One unordered pair: forward into (S1, S2), reverse (when rev) into (R1, R2).
template <bool NEAR>
__device__ __forceinline__ void ffs_pair(const FFTarget& T, ff ai, ff bi, const float4& F0, const float4& F1,
                                         const float4& F2, const float4& F3, const FFConsts& k,
                                         const float2* __restrict__ tab, bool rev, ff& S1, ff& S2, ff& R1, ff& R2,
                                         const double* __restrict__ geo, int64_t i, int64_t j, int64_t N)
{
    const float rh0 = __fsub_rn(T.xh0, F0.x), rh1 = __fsub_rn(T.xh1, F0.y), rh2 = __fsub_rn(T.xh2, F0.z);
    const float rl0 = __fsub_rn(T.xl0, F1.x), rl1 = __fsub_rn(T.xl1, F1.y), rl2 = __fsub_rn(T.xl2, F1.z);
    const ff rr = ff_norm2(rh0, rl0, rh1, rl1, rh2, rl2);
    const ff sx = ff_dot3(rh0, rl0, rh1, rl1, rh2, rl2, T.nh0, T.nl0, T.nh1, T.nl1, T.nh2, T.nl2);
    const ff sy = ff_dot3(rh0, rl0, rh1, rl1, rh2, rl2, F2.x, F3.x, F2.y, F3.y, F2.z, F3.z);
    const ff aj = ff{F0.w, F1.w}, bj = ff{F2.w, F3.w};
    bool tube_f = false, tube_r = false;
    if (NEAR) {
        const float d2 = __fadd_rn(__fsub_rn(rr.h, k.four_tau2.x), __fsub_rn(rr.l, k.four_tau2.y));
        const bool tie2 = fabsf(d2) < 1e-9f * k.four_tau2.x;
        const ff pf = ff_sub(rr, ff_mul(sx, sx));
        const float d1f = __fadd_rn(__fsub_rn(pf.h, k.tau2.x), __fsub_rn(pf.l, k.tau2.y));
        tube_f = (d1f < 0.0f) && (d2 < 0.0f);
        if ((tie2 || fabsf(d1f) < 1e-9f * k.tau2.x) && i < N && j < N)
            tube_f = tube_f64_ordered(geo, N, i, j, k.tau2_d, k.four_tau2_d);
        if (rev) {
            const ff pr = ff_sub(rr, ff_mul(sy, sy));
            const float d1r = __fadd_rn(__fsub_rn(pr.h, k.tau2.x), __fsub_rn(pr.l, k.tau2.y));
            tube_r = (d1r < 0.0f) && (d2 < 0.0f);
            if ((tie2 || fabsf(d1r) < 1e-9f * k.tau2.x) && i < N && j < N)
                tube_r = tube_f64_ordered(geo, N, j, i, k.tau2_d, k.four_tau2_d);
        }
        if (tube_f && (tube_r || !rev)) {  // both directions regularised (the self pair among them)
            const ff c = ff_mul(ff_of(k.nk12t), bj);
            const ff s = two_sum(S1.h, c.h);
            S1 = fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(S1.l, c.l)));
            if (rev) {
                const ff cr = ff_mul(ff_of(k.nk12t), bi);
                const ff t = two_sum(R1.h, cr.h);
                R1 = fast_two_sum(t.h, __fadd_rn(t.l, __fadd_rn(R1.l, cr.l)));
            }
            return;
        }
    }
    const ff cc = ff_dot3(T.nh0, T.nl0, T.nh1, T.nl1, T.nh2, T.nl2, F2.x, F3.x, F2.y, F3.y, F2.z, F3.z);
    const float y0 = ptx::rsqrt_approx(rr.h);
    const ff q = ff_mul(rr, ff{__fmul_rn(y0, y0), __fmaf_rn(y0, y0, -__fmul_rn(y0, y0))});
    const float d = __fadd_rn(__fsub_rn(q.h, 1.0f), q.l);
    const ff inv = ff{y0, __fmul_rn(__fmul_rn(y0, d), __fmaf_rn(0.375f, d, -0.5f))};
    const ff rho = ff_mul(rr, inv);
    const ff x = ff_mul(ff_of(k.kap), rho);
    const ff E = ff_exp2(ff_mul(ff_of(k.cz), rho), tab);
    const ff Ex = ff_mul(E, x);
    const float fh = __fsub_rn(1.0f, E.h);
    const ff f = ff{fh, __fsub_rn(__fsub_rn(__fsub_rn(1.0f, fh), E.h), E.l)};
    const ff g = ff_sub(f, Ex);
    const ff u1 = ff_add(ff_of(k.om1), ff_mul(ff_of(k.th1), g));
    const ff u2 = ff_add(ff_of(k.om2), ff_mul(ff_of(k.th2), g));
    const ff hb = ff_sub(ff_mulf(g, 3.0f), ff_mul(Ex, x));
    const ff inv2 = ff_mul(inv, inv);
    const ff inv3 = ff_mul(inv2, inv);
    const ff br = ff_sub(ff_mul(g, cc), ff_mul(hb, ff_mul(ff_mul(sx, sy), inv2)));
    const ff P1 = ff_mul(u1, inv3), Q = ff_mul(f, inv), P2 = ff_mul(u2, inv3), B3 = ff_mul(br, inv3);
    ff c1, c2;
    if (NEAR && tube_f) {
        c1 = ff_mul(ff_of(k.nk12t), bj);
        c2 = ff{0.0f, 0.0f};
    } else {
        c1 = ff_sub(ff_mul(P1, ff_mul(sy, aj)), ff_mul(Q, bj));
        c2 = ff_add(ff_mul(B3, aj), ff_mul(ff_mul(P2, sx), bj));
    }
    const ff s1 = two_sum(S1.h, c1.h);
    S1 = fast_two_sum(s1.h, __fadd_rn(s1.l, __fadd_rn(S1.l, c1.l)));
    const ff s2 = two_sum(S2.h, c2.h);
    S2 = fast_two_sum(s2.h, __fadd_rn(s2.l, __fadd_rn(S2.l, c2.l)));
    if (!rev) return;
    ff e1, e2;
    if (NEAR && tube_r) {
        e1 = ff_mul(ff_of(k.nk12t), bi);
        e2 = ff{0.0f, 0.0f};
    } else {
        const ff m = ff_mul(P1, ff_mul(sx, ai));
        e1 = ff_sub(ff{-m.h, -m.l}, ff_mul(Q, bi));
        e2 = ff_sub(ff_mul(B3, ai), ff_mul(ff_mul(P2, sy), bi));
    }
    const ff r1 = two_sum(R1.h, e1.h);
    R1 = fast_two_sum(r1.h, __fadd_rn(r1.l, __fadd_rn(R1.l, e1.l)));
    const ff r2 = two_sum(R2.h, e2.h);
    R2 = fast_two_sum(r2.h, __fadd_rn(r2.l, __fadd_rn(R2.l, e2.l)));
}

constexpr int kFFSThreads = 256;  // one target per thread; target tile = source tile (R = 1)

__global__ void __launch_bounds__(kFFSThreads, 2)
    pair_ffs_kernel(const float4* __restrict__ src, const float4* __restrict__ frames,
                    const float2* __restrict__ tab_g, const double* __restrict__ geo, int64_t N, int64_t n_pad,
                    SymSchedule s, FFConsts k, double* __restrict__ part, double* __restrict__ yrev,
                    unsigned* __restrict__ err, const int* __restrict__ skip)
{
    constexpr int TTILE = kFFSThreads;
    if (skip != nullptr && *skip) return;
    __shared__ __align__(128) float4 sbuf[kFFStages][kFFSTile * kFFNodeF4];
    __shared__ __align__(16) float4 sfrm[kFFStages][2 * kFFChunksPerTile];
    __shared__ float2 tab[kFFTab];
    __shared__ __align__(8) uint64_t bars[kFFStages];
    __shared__ int abort_flag;
    __shared__ int64_t seg_next;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    unsigned long long* seg_ctr = reinterpret_cast<unsigned long long*>(yrev + 2 * n_pad);
    for (int q = tid; q < kFFTab; q += kFFSThreads) tab[q] = tab_g[q];
    if (tid == 0) {
        for (int q = 0; q < kFFStages; ++q) ptx::mbar_init(&bars[q], 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    // ring position: this CTA's n-th step uses stage n mod kFFStages, phase (n / kFFStages) mod 2
    int64_t n_done = 0;
    auto issue = [&](int64_t u, int64_t n) {
        int64_t t, rho, pos;
        sym_locate(s, u, t, rho, pos);
        const int64_t st = s.R * t + pos;
        const int stage = (int)(n % kFFStages);
        ptx::mbar_arrive_expect_tx(&bars[stage], kFFStageBytes + kFFFrameBytes);
        ptx::bulk_g2s(&sbuf[stage][0], src + st * kFFSTile * kFFNodeF4, kFFStageBytes, &bars[stage]);
        ptx::bulk_g2s(&sfrm[stage][0], frames + st * 2 * kFFChunksPerTile, kFFFrameBytes, &bars[stage]);
    };

    FFTarget T;
    ff ai, bi;
    float4 tfh, tfl;
    int64_t gi = 0;
    int Ablk = 0;
    bool idle = false;
    double D1 = 0.0, D2 = 0.0;
    auto load_target = [&](int64_t tile) {
        gi = tile * TTILE + tid;
        idle = tile * TTILE + warp * kFFChunk >= N;
        const float4 a = src[ff_off(gi, 0)], b = src[ff_off(gi, 1)];
        const float4 c = src[ff_off(gi, 2)], e = src[ff_off(gi, 3)];
        const bool pad = gi >= N;
        T.xh0 = pad ? -kFFPad : a.x;
        T.xh1 = pad ? -kFFPad : a.y;
        T.xh2 = pad ? -kFFPad : a.z;
        T.xl0 = pad ? 0.0f : b.x;
        T.xl1 = pad ? 0.0f : b.y;
        T.xl2 = pad ? 0.0f : b.z;
        T.nh0 = c.x;
        T.nh1 = c.y;
        T.nh2 = c.z;
        T.nl0 = e.x;
        T.nl1 = e.y;
        T.nl2 = e.z;
        ai = ff{a.w, b.w};
        bi = ff{c.w, e.w};
        Ablk = (int)((tile * TTILE + warp * kFFChunk) / kFFChunk);
        const int64_t blk = Ablk;
        tfh = frames[2 * blk];
        tfl = frames[2 * blk + 1];
        D1 = D2 = 0.0;
    };

    int64_t seg = blockIdx.x;
    while (seg < s.nseg) {
        const int64_t s0 = sym_seg_start(s, seg), s1 = sym_seg_start(s, seg + 1);
        if (tid == 0)
            for (int q = 0; q < kFFStages && s0 + q < s1; ++q) issue(s0 + q, n_done + q);
        int64_t t, rho, pos;
        sym_locate(s, s0, t, rho, pos);
        load_target(t);
        for (int64_t u = s0; u < s1; ++u) {
            const int64_t n = n_done + (u - s0);
            const int stage = (int)(n % kFFStages);
            if (!ptx::mbar_wait_bounded(&bars[stage], (uint32_t)((n / kFFStages) & 1), kFFWaitNs)) {
                abort_flag = 1;
                atomicOr(err, kDevErrTimeout);
            }
            __syncthreads();
            if (abort_flag) return;
            const int64_t st = s.R * t + pos;
            if (!idle) {
                ff S1{0.0f, 0.0f}, S2{0.0f, 0.0f};
                const float4* sb = &sbuf[stage][0];
#pragma unroll 1
                for (int c = 0; c < kFFChunksPerTile; ++c) {
                    const int64_t Bc = st * kFFChunksPerTile + c;
                    if (Bc < Ablk) continue;  // the warp holding block Bc covers this block pair
                    const bool rev = Bc > Ablk;
                    const float4 mh = sfrm[stage][2 * c], ml = sfrm[stage][2 * c + 1];
                    const float dx = (tfh.x - mh.x) + (tfl.x - ml.x);
                    const float dy = (tfh.y - mh.y) + (tfl.y - ml.y);
                    const float dz = (tfh.z - mh.z) + (tfl.z - ml.z);
                    const float lim = k.far_dist + tfh.w + mh.w;
                    const bool far = k.rule0 && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim);
                    const float4* cb = sb + c * kFFChunk * kFFNodeF4;
                    const int64_t j0 = Bc * kFFChunk;
                    ff R1{0.0f, 0.0f}, R2{0.0f, 0.0f};
                    if (far) {
#pragma unroll 1
                        for (int step = 0; step < kFFChunk; ++step) {
                            const int p = (lane + step) & (kFFChunk - 1);
                            ffs_pair<false>(T, ai, bi, cb[p], cb[32 + p], cb[64 + p], cb[96 + p], k, tab, rev, S1, S2,
                                            R1, R2, geo, gi, j0 + p, N);
                            R1.h = __shfl_sync(0xffffffffu, R1.h, lane + 1);  // source p goes to lane - 1
                            R1.l = __shfl_sync(0xffffffffu, R1.l, lane + 1);
                            R2.h = __shfl_sync(0xffffffffu, R2.h, lane + 1);
                            R2.l = __shfl_sync(0xffffffffu, R2.l, lane + 1);
                        }
                    } else {
#pragma unroll 1
                        for (int step = 0; step < kFFChunk; ++step) {
                            const int p = (lane + step) & (kFFChunk - 1);
                            ffs_pair<true>(T, ai, bi, cb[p], cb[32 + p], cb[64 + p], cb[96 + p], k, tab, rev, S1, S2,
                                           R1, R2, geo, gi, j0 + p, N);
                            R1.h = __shfl_sync(0xffffffffu, R1.h, lane + 1);
                            R1.l = __shfl_sync(0xffffffffu, R1.l, lane + 1);
                            R2.h = __shfl_sync(0xffffffffu, R2.h, lane + 1);
                            R2.l = __shfl_sync(0xffffffffu, R2.l, lane + 1);
                        }
                    }
                    if (rev) {  // lane l holds source j0 + l's reverse sums over the warp's targets
                        atomicAdd(yrev + j0 + lane, (double)R1.h + (double)R1.l);
                        atomicAdd(yrev + n_pad + j0 + lane, (double)R2.h + (double)R2.l);
                    }
                }
                D1 += (double)S1.h + (double)S1.l;
                D2 += (double)S2.h + (double)S2.l;
            }
            __syncthreads();
            if (tid == 0 && u + kFFStages < s1) {
                ptx::fence_proxy_async_smem();
                issue(u + kFFStages, n + kFFStages);
            }
            if (pos == sym_row_len(s, t) - 1 || u + 1 == s1) {
                double* dst = part + (seg + rho) * 2 * TTILE;
                dst[tid] = D1;
                dst[TTILE + tid] = D2;
                if (u + 1 < s1) {
                    sym_locate(s, u + 1, t, rho, pos);
                    load_target(t);
                }
            } else {
                ++pos;
            }
        }
        n_done += s1 - s0;
        if (tid == 0) seg_next = s.nbig + (int64_t)atomicAdd(seg_ctr, 1ull);
        __syncthreads();
        seg = seg_next;
        __syncthreads();
    }
}

// 2^(i/256) as float-float pairs, i = 0..255 (FP64 exp2 of the CUDA math library).
__global__ void ff_table_kernel(float2* __restrict__ tab)
{
    const int i = threadIdx.x;
    if (i >= kFFTab) return;
    const double v = exp2((double)i / (double)kFFTab);
    const float h = (float)v;
    tab[i] = make_float2(h, (float)(v - (double)h));
}

// Largest |x* - centroid| component (one CTA; fixed order).
__global__ void ff_extent_kernel(const double* __restrict__ geo, int64_t N, double c0, double c1, double c2,
                                 double* __restrict__ out)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x)
        m = fmax(m, fmax(fabs(geo[j] - c0), fmax(fabs(geo[N + j] - c1), fabs(geo[2 * N + j] - c2))));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Float-float payload of the padded node range for input `in` (one thread
// per node): coordinates relative to the centroid split on the 2^-q grid,
// normals, a = w psi and b = w psin split into hi + lo.
__global__ void ff_pack_kernel(const double* __restrict__ geo, int64_t N, int64_t n_pad, double c0, double c1,
                               double c2, double grid_scale, VecRef in, float4* __restrict__ src,
                               double* __restrict__ yrev, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    if (yrev != nullptr) {  // symmetric kernel: clear its reverse sums and its segment counter
        yrev[j] = 0.0;
        yrev[n_pad + j] = 0.0;
        if (j == 0) *reinterpret_cast<unsigned long long*>(yrev + 2 * n_pad) = 0ull;
    }
    if (j >= N) {
        src[ff_off(j, 0)] = make_float4(kFFPad, kFFPad, kFFPad, 0.0f);
        src[ff_off(j, 1)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        src[ff_off(j, 2)] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
        src[ff_off(j, 3)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    const double cen[3] = {c0, c1, c2};
    float xh[3], xl[3], nh[3], nl[3];
    for (int a = 0; a < 3; ++a) {
        const double x = geo[a * N + j] - cen[a];
        const double xg = rint(x * grid_scale) / grid_scale;  // on the grid: exact as a float
        xh[a] = (float)xg;
        xl[a] = (float)(x - xg);
        const double n = geo[(3 + a) * N + j];
        nh[a] = (float)n;
        nl[a] = (float)(n - (double)nh[a]);
    }
    const double w = geo[6 * N + j];
    const double av = w * p[j], bv = w * p[N + j];
    const float ah = (float)av, bh = (float)bv;
    src[ff_off(j, 0)] = make_float4(xh[0], xh[1], xh[2], ah);
    src[ff_off(j, 1)] = make_float4(xl[0], xl[1], xl[2], (float)(av - (double)ah));
    src[ff_off(j, 2)] = make_float4(nh[0], nh[1], nh[2], bh);
    src[ff_off(j, 3)] = make_float4(nl[0], nl[1], nl[2], (float)(bv - (double)bh));
}

// ------------------------------------------------------------------ host side

int ff_grid_cap(ibim_ctx* c)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_ff_kernel, kFFThreads, 0);
    return (occ < 1 ? 1 : occ) * c->num_sms;
}

PairSchedule ff_schedule(ibim_ctx* c) { return make_schedule(c->N, kFFTTile, c->N, kFFSTile, ff_grid_cap(c)); }

size_t ffs_part_doubles(ibim_ctx* c);

size_t ff_part_doubles(ibim_ctx* c)
{
    const PairSchedule s = ff_schedule(c);
    return std::max((size_t)s.grid * s.max_segs * 2 * kFFTTile, ffs_part_doubles(c));
}

size_t ff_src_bytes(int64_t N) { return (size_t)padded_nodes(N) * kFFNodeF4 * sizeof(float4); }

// Table and grid of the context (once): the 2^(i/256) table and the
// power-of-two grid 2^-q of the hi parts, with |x - centroid| 2^q < 2^23.
static ibim_status ff_prepare(ibim_ctx* c)
{
    if (c->d_fftab != nullptr) return IBIM_OK;
    IBIM_TRY(ensure(c, (void**)&c->d_red, &c->red_bytes, std::max(c->red_bytes, (size_t)4096)));
    ff_extent_kernel<<<1, 256, 0, c->stream>>>(c->d_geo64, c->N, c->centroid[0], c->centroid[1], c->centroid[2],
                                              c->d_red);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    double ext = 0.0;
    IBIM_CUDA(cudaMemcpyAsync(&ext, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    IBIM_CUDA(cudaStreamSynchronize(c->stream));
    int e = 0;
    frexp(ext > 1e-3 ? ext : 1e-3, &e);  // ext < 2^e
    c->ff_grid_scale = ldexp(1.0, 23 - e);
    IBIM_CUDA(cudaMalloc((void**)&c->d_fftab, sizeof(float2) * kFFTab));
    ff_table_kernel<<<1, kFFTab, 0, c->stream>>>(c->d_fftab);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status ff_prepare_context(ibim_ctx* c) { return ff_prepare(c); }

int ffs_grid_cap(ibim_ctx* c)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_ffs_kernel, kFFSThreads, 0);
    return (occ < 1 ? 1 : occ) * c->num_sms;
}

size_t ffs_part_doubles(ibim_ctx* c) { return sym_part_doubles(c->N, kFFSThreads, ffs_grid_cap(c)); }

ibim_status ff_pack(ibim_ctx* c, VecRef in, const int* d_skip)
{
    IBIM_TRY(ff_prepare(c));
    const int64_t N = c->N, n_pad = padded_nodes(N);
    const int bs = 256;
    ff_pack_kernel<<<(unsigned)((n_pad + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_geo64, N, n_pad, c->centroid[0], c->centroid[1], c->centroid[2], c->ff_grid_scale, in,
        (float4*)c->d_src, c->ff_symmetric ? c->d_yrev : nullptr, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status ff_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip)
{
    if (c->ff_symmetric) {
        const SymSchedule ss = make_sym_schedule(c->N, kFFSThreads, ffs_grid_cap(c));
        pair_ffs_kernel<<<ss.grid, kFFSThreads, 0, c->stream>>>(
            (const float4*)c->d_src, c->d_frames, c->d_fftab, c->d_geo64, c->N, padded_nodes(c->N), ss, ff_consts(k),
            c->d_part, c->d_yrev, c->d_err, d_skip);
    } else {
        pair_ff_kernel<<<s.grid, kFFThreads, 0, c->stream>>>((const float4*)c->d_src, c->d_frames, c->d_fftab,
                                                              c->d_geo64, c->N, s, ff_consts(k), c->d_part, c->d_err,
                                                              d_skip);
    }
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

ibim_status ff_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                     const int* d_skip)
{
    if (c->ff_symmetric) return sym_fixup_tiles(c, kFFSThreads, ffs_grid_cap(c), k, in, out, d_skip);
    return fixup_launch(c, k, s, kFFTTile, in, out, d_skip);
}

}  // namespace ibim
