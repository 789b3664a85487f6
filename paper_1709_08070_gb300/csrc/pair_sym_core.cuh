// Pair arithmetic, payload layout and tile loop of the symmetric FP32
// operator (each unordered node pair evaluated once for both directions),
// shared by the single-molecule kernel (pair_sym.cu) and the batched one
// (batch.cu).  See pair_sym.cu for the method.
#pragma once
#include "pair_f32_core.cuh"

namespace ibim {

// Stream-K schedule of a symmetric launch over the upper triangle of
// (target tile, source tile) steps (see pair_sym.cu).
struct SymSchedule {
    int64_t n_t, n_s, R;  // target tiles, source tiles, source tiles per target tile
    int64_t npairs;       // row pairs (n_t / 2); an odd row count leaves a middle row at the end
    int64_t L2;           // steps of a row pair: 2 n_s - R (n_t - 1)
    int64_t total;        // steps
    int64_t Lb, nbig;     // large segments: nbig (= grid) of Lb steps, first
    int64_t Ls, nseg;     // then small segments of Ls steps (the last may be shorter); nseg in all
    int grid;
};

// First step of segment q (q <= nseg; total for q = nseg).
__host__ __device__ __forceinline__ int64_t sym_seg_start(const SymSchedule& s, int64_t q)
{
    const int64_t v = q < s.nbig ? q * s.Lb : s.nbig * s.Lb + (q - s.nbig) * s.Ls;
    return v < s.total ? v : s.total;
}

// Segment holding step u (u < total).
__host__ __device__ __forceinline__ int64_t sym_seg_of(const SymSchedule& s, int64_t u)
{
    const int64_t big = s.nbig * s.Lb;
    return u < big ? u / s.Lb : s.nbig + (u - big) / s.Ls;
}

__host__ __device__ __forceinline__ int64_t sym_row_len(const SymSchedule& s, int64_t t) { return s.n_s - s.R * t; }

// Step u of the sequence -> row t, its sequence index rho and the position in the row.
__host__ __device__ __forceinline__ void sym_locate(const SymSchedule& s, int64_t u, int64_t& t, int64_t& rho,
                                                    int64_t& pos)
{
    const int64_t p = u / s.L2;
    if (p < s.npairs) {
        const int64_t r = u - p * s.L2;
        const int64_t l0 = sym_row_len(s, p);
        if (r < l0) {
            t = p;
            rho = 2 * p;
            pos = r;
        } else {
            t = s.n_t - 1 - p;
            rho = 2 * p + 1;
            pos = r - l0;
        }
    } else {
        t = s.npairs;
        rho = 2 * s.npairs;
        pos = u - s.npairs * s.L2;
    }
}

// First step of row t in the sequence and its sequence index.
__host__ __device__ __forceinline__ void sym_row_start(const SymSchedule& s, int64_t t, int64_t& start,
                                                       int64_t& rho)
{
    if (t < s.npairs) {
        start = t * s.L2;
        rho = 2 * t;
    } else if (t >= s.n_t - s.npairs) {
        const int64_t p = s.n_t - 1 - t;
        start = p * s.L2 + sym_row_len(s, p);
        rho = 2 * p + 1;
    } else {
        start = s.npairs * s.L2;
        rho = 2 * s.npairs;
    }
}

SymSchedule make_sym_schedule(int64_t N, int ttile, int grid_cap);

// Float4 offset of component `comp` (0..3 = A..D) of payload pair `pr`.
__host__ __device__ __forceinline__ int64_t sym_pair_offset(int64_t pr, int comp)
{
    return (pr / kPairsPerChunk) * (kPairsPerChunk * kPairF4) + comp * kPairsPerChunk + (pr % kPairsPerChunk);
}

__device__ __forceinline__ void write_source_pair_sym(float4* __restrict__ src, int64_t pr, float4 y0, float4 y1,
                                                      float4 m0, float4 m1, float a0, float a1, float b0, float b1)
{
    src[sym_pair_offset(pr, 0)] = make_float4(-y0.x, -y1.x, -y0.y, -y1.y);
    src[sym_pair_offset(pr, 1)] = make_float4(-y0.z, -y1.z, b0, b1);
    src[sym_pair_offset(pr, 2)] = make_float4(m0.x, m1.x, m0.y, m1.y);
    src[sym_pair_offset(pr, 3)] = make_float4(m0.z, m1.z, a0, a1);
}

// Per-thread targets with their own weights (the reverse direction's sources).
template <int TPT>
struct SymTargets {
    float3 x[TPT];
    float2 nx[TPT], ny[TPT], nz[TPT];
    float2 a[TPT], nb[TPT];  // a = w psi and -b = -w psin of the target
};

// Far pair, both directions, packed over the two sources of a payload pair.
// Forward (target i <- source j) into t1, t2; reverse (source j <- target i)
// returned as nr1 = -(first reverse sum) and r2.  See pair_far2 for the
// forward form; the reverse form swaps the roles: r' = -r, s_x' = -s_y,
// s_y' = -s_x, c' = c.
__device__ __forceinline__ void pair_far_sym(float2 Xx, float2 Xy, float2 Xz, float2 nx, float2 ny, float2 nz,
                                             float2 ai, float2 nbi, const float4& A,
                                             const float4& B, const float4& C, const float4& D, const FarConsts& c,
                                             float2& t1, float2& t2, float2& nr1, float2& r2)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 bj = make_float2(B.z, B.w);
    const float2 mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w), mz = make_float2(D.x, D.y);
    const float2 aj = make_float2(D.z, D.w);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sx = __fmul2_rn(rx, nx);
    sx = __ffma2_rn(ry, ny, sx);
    sx = __ffma2_rn(rz, nz, sx);
    float2 sy = __fmul2_rn(rx, mx);
    sy = __ffma2_rn(ry, my, sy);
    sy = __ffma2_rn(rz, mz, sy);
    float2 cc = __fmul2_rn(nx, mx);
    cc = __ffma2_rn(ny, my, cc);
    cc = __ffma2_rn(nz, mz, cc);
    const float2 inv = make_float2(ptx::rsqrt_approx(rr.x), ptx::rsqrt_approx(rr.y));
    const float2 rho = __fmul2_rn(rr, inv);
    const float2 ea = __fmul2_rn(rho, c.kl2e);
    const float2 xn = __fmul2_rn(rho, c.nkappa);
    const float2 E = make_float2(ptx::ex2_approx(ea.x), ptx::ex2_approx(ea.y));
    const float2 En = __fmul2_rn(E, xn);
    const float2 fn = __fadd2_rn(E, c.neg1);
    const float2 g = __ffma2_rn(fn, c.neg1, En);
    const float2 hn = __ffma2_rn(g, c.neg3, __fmul2_rn(En, xn));
    const float2 inv2 = make_float2(ptx::rcp_approx(rr.x), ptx::rcp_approx(rr.y));
    const float2 P = __fmul2_rn(inv2, inv);
    const float2 u1 = __ffma2_rn(c.th1, g, c.omth1);
    const float2 u2 = __ffma2_rn(c.th2, g, c.omth2);
    const float2 hi = __fmul2_rn(hn, inv2);
    const float2 qf = __fmul2_rn(fn, inv);
    // forward
    const float2 sa = __fmul2_rn(aj, sy);
    const float2 ca = __fmul2_rn(aj, cc);
    t1 = __ffma2_rn(P, __fmul2_rn(u1, sa), t1);
    t1 = __ffma2_rn(qf, bj, t1);
    const float2 v = __ffma2_rn(hi, sa, __fmul2_rn(u2, bj));
    t2 = __ffma2_rn(P, __ffma2_rn(sx, v, __fmul2_rn(g, ca)), t2);
    // reverse (a_i s_x' ... with s_y' = -s_x: psa = a_i s_x = -a_i s_y')
    const float2 psa = __fmul2_rn(ai, sx);
    nr1 = __ffma2_rn(P, __fmul2_rn(u1, psa), __fmul2_rn(qf, nbi));
    const float2 nv = __ffma2_rn(hi, psa, __fmul2_rn(u2, nbi));
    r2 = __fmul2_rn(P, __ffma2_rn(sy, nv, __fmul2_rn(g, __fmul2_rn(ai, cc))));
}

// pair_far_sym with the reverse sums accumulated into (nR1, R2) (rotation
// scheme): nR1 -= first reverse sum, R2 += second.  The factors common to both
// directions are formed once, P u1, P u2, P g c and P hn rho^-2, and rho^-2 is
// the square of the MUFU rsqrt (two MUFU operations per source, 48 packed
// operations per source pair as in pair_far_sym: 36 shared, 6 per direction):
//   t1 += (P u1) s_a + qf b,   t2 += s_x [(P hn rho^-2) s_a + (P u2) b] + (P g c) a
// and the reverse sums likewise with (s_a, b, s_x, a) -> (a_i s_x, -b_i, s_y, a_i).
// (Measured against pair_far_sym's order of operations inside the rotation
// loop: 5.66 against 5.74 ms per application on the 80k-node sphere.)
__device__ __forceinline__ void pair_far_sym_acc(float2 Xx, float2 Xy, float2 Xz, float2 nx, float2 ny, float2 nz,
                                                 float2 ai, float2 nbi, const float4& A, const float4& B,
                                                 const float4& C, const float4& D, const FarConsts& c, float2& t1,
                                                 float2& t2, float2& nR1, float2& R2)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 bj = make_float2(B.z, B.w);
    const float2 mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w), mz = make_float2(D.x, D.y);
    const float2 aj = make_float2(D.z, D.w);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sx = __fmul2_rn(rx, nx);
    sx = __ffma2_rn(ry, ny, sx);
    sx = __ffma2_rn(rz, nz, sx);
    float2 sy = __fmul2_rn(rx, mx);
    sy = __ffma2_rn(ry, my, sy);
    sy = __ffma2_rn(rz, mz, sy);
    float2 cc = __fmul2_rn(nx, mx);
    cc = __ffma2_rn(ny, my, cc);
    cc = __ffma2_rn(nz, mz, cc);
    const float2 inv = make_float2(ptx::rsqrt_approx(rr.x), ptx::rsqrt_approx(rr.y));
    const float2 rho = __fmul2_rn(rr, inv);
    const float2 ea = __fmul2_rn(rho, c.kl2e);
    const float2 xn = __fmul2_rn(rho, c.nkappa);
    const float2 E = make_float2(ptx::ex2_approx(ea.x), ptx::ex2_approx(ea.y));
    const float2 En = __fmul2_rn(E, xn);
    const float2 fn = __fadd2_rn(E, c.neg1);
    const float2 g = __ffma2_rn(fn, c.neg1, En);
    const float2 hn = __ffma2_rn(g, c.neg3, __fmul2_rn(En, xn));
    const float2 inv2 = __fmul2_rn(inv, inv);
    const float2 P = __fmul2_rn(inv2, inv);
    const float2 Pu1 = __fmul2_rn(P, __ffma2_rn(c.th1, g, c.omth1));
    const float2 Pu2 = __fmul2_rn(P, __ffma2_rn(c.th2, g, c.omth2));
    const float2 Pgc = __fmul2_rn(__fmul2_rn(P, g), cc);
    const float2 Phi = __fmul2_rn(hn, __fmul2_rn(inv2, P));
    const float2 qf = __fmul2_rn(fn, inv);
    // forward
    const float2 sa = __fmul2_rn(aj, sy);
    t1 = __ffma2_rn(Pu1, sa, t1);
    t1 = __ffma2_rn(qf, bj, t1);
    t2 = __ffma2_rn(sx, __ffma2_rn(Phi, sa, __fmul2_rn(Pu2, bj)), t2);
    t2 = __ffma2_rn(Pgc, aj, t2);
    // reverse, accumulated
    const float2 psa = __fmul2_rn(ai, sx);
    nR1 = __ffma2_rn(Pu1, psa, nR1);
    nR1 = __ffma2_rn(qf, nbi, nR1);
    R2 = __ffma2_rn(sy, __ffma2_rn(Phi, psa, __fmul2_rn(Pu2, nbi)), R2);
    R2 = __ffma2_rn(Pgc, ai, R2);
}

// Near pairs in the rotation scheme, both directions, packed over the two
// sources of a payload pair: pair_far_sym_acc's formula with, per lane, g
// from its series where kappa rho < 0.5 (f = 1 - E = g + E x there), as in
// near_one, and each direction's tube test (Sec. 2.2.1: rho_P^2 on the
// target's tangent plane forward, on the source's in reverse).  A
// regularised direction keeps only K12's tube value: selects zero its a
// weight and the b weight of its second sum and put the tube value in place
// of its 1/rho factor, so the products with the powers of 1/rho stay shared.
// rho^2 is kept >= 1e-12, so that coincident nodes (the self pair among
// them, always in the tube) leave every product finite.  When any of the
// four tests lies within kTieBand of a threshold, all four are decided again
// in FP64 (tube_f64), which the FP32 tests agree with outside the band.
// i: the target's node index, j: the first source's.
__device__ __forceinline__ void pair_near_sym_acc(float2 Xx, float2 Xy, float2 Xz, float2 nx, float2 ny, float2 nz,
                                                  float2 ai, float2 nbi, const float4& A, const float4& B,
                                                  const float4& C, const float4& D, const FarConsts& c,
                                                  const F32Consts& k, float2& t1, float2& t2, float2& nR1,
                                                  float2& R2, const Geo64& g64, int64_t i, int64_t j, int64_t N)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 bj = make_float2(B.z, B.w);
    const float2 mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w), mz = make_float2(D.x, D.y);
    const float2 aj = make_float2(D.z, D.w);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sx = __fmul2_rn(rx, nx);
    sx = __ffma2_rn(ry, ny, sx);
    sx = __ffma2_rn(rz, nz, sx);
    float2 sy = __fmul2_rn(rx, mx);
    sy = __ffma2_rn(ry, my, sy);
    sy = __ffma2_rn(rz, mz, sy);
    float2 cc = __fmul2_rn(nx, mx);
    cc = __ffma2_rn(ny, my, cc);
    cc = __ffma2_rn(nz, mz, cc);
    // tube tests: forward (f) on rho^2 - s_x^2, reverse (r) on rho^2 - s_y^2
    const float2 rpf = __ffma2_rn(__fmul2_rn(sx, c.neg1), sx, rr);
    const float2 rpr = __ffma2_rn(__fmul2_rn(sy, c.neg1), sy, rr);
    const bool in0 = rr.x < k.four_tau2, in1 = rr.y < k.four_tau2;
    bool tf0 = (rpf.x < k.tau2) & in0, tf1 = (rpf.y < k.tau2) & in1;
    bool tr0 = (rpr.x < k.tau2) & in0, tr1 = (rpr.y < k.tau2) & in1;
    const float bt = kTieBand * k.tau2, b4 = kTieBand * k.four_tau2;
    const bool tie = (fabsf(rpf.x - k.tau2) < bt) | (fabsf(rpf.y - k.tau2) < bt) | (fabsf(rpr.x - k.tau2) < bt) |
                     (fabsf(rpr.y - k.tau2) < bt) | (fabsf(rr.x - k.four_tau2) < b4) |
                     (fabsf(rr.y - k.four_tau2) < b4);
    if (tie && g64.x != nullptr && i < N) {
        if (j < N) {
            tf0 = tube_f64(g64, i, j, k.tau2_d, k.four_tau2_d);
            tr0 = tube_f64(g64, j, i, k.tau2_d, k.four_tau2_d);
        }
        if (j + 1 < N) {
            tf1 = tube_f64(g64, i, j + 1, k.tau2_d, k.four_tau2_d);
            tr1 = tube_f64(g64, j + 1, i, k.tau2_d, k.four_tau2_d);
        }
    }
    const float2 rrs = make_float2(fmaxf(rr.x, 1.0e-12f), fmaxf(rr.y, 1.0e-12f));
    const float2 inv = make_float2(ptx::rsqrt_approx(rrs.x), ptx::rsqrt_approx(rrs.y));
    const float2 rho = __fmul2_rn(rrs, inv);
    const float2 ea = __fmul2_rn(rho, c.kl2e);
    const float2 xn = __fmul2_rn(rho, c.nkappa);
    const float2 E = make_float2(ptx::ex2_approx(ea.x), ptx::ex2_approx(ea.y));
    const float2 En = __fmul2_rn(E, xn);
    float2 fn = __fadd2_rn(E, c.neg1);
    float2 g = __ffma2_rn(fn, c.neg1, En);
    if (-xn.x < 0.5f) {  // kappa rho < 0.5: series of g, fn = -(g + E x)
        g.x = g_series(-xn.x);
        fn.x = En.x - g.x;
    }
    if (-xn.y < 0.5f) {
        g.y = g_series(-xn.y);
        fn.y = En.y - g.y;
    }
    const float2 hn = __ffma2_rn(g, c.neg3, __fmul2_rn(En, xn));
    const float2 inv2 = __fmul2_rn(inv, inv);
    const float2 P = __fmul2_rn(inv2, inv);
    const float2 Pu1 = __fmul2_rn(P, __ffma2_rn(c.th1, g, c.omth1));
    const float2 Pu2 = __fmul2_rn(P, __ffma2_rn(c.th2, g, c.omth2));
    const float2 Pgc = __fmul2_rn(__fmul2_rn(P, g), cc);
    const float2 Phi = __fmul2_rn(hn, __fmul2_rn(inv2, P));
    const float2 qf = __fmul2_rn(fn, inv);
    // forward; a regularised pair adds -K12_tube b only
    const float2 ajf = make_float2(tf0 ? 0.0f : aj.x, tf1 ? 0.0f : aj.y);
    const float2 bjt = make_float2(tf0 ? 0.0f : bj.x, tf1 ? 0.0f : bj.y);
    const float2 qff = make_float2(tf0 ? -k.k12t : qf.x, tf1 ? -k.k12t : qf.y);
    const float2 sa = __fmul2_rn(ajf, sy);
    t1 = __ffma2_rn(Pu1, sa, t1);
    t1 = __ffma2_rn(qff, bj, t1);
    t2 = __ffma2_rn(sx, __ffma2_rn(Phi, sa, __fmul2_rn(Pu2, bjt)), t2);
    t2 = __ffma2_rn(Pgc, ajf, t2);
    // reverse, accumulated (nbi = -b_i)
    const float2 air = make_float2(tr0 ? 0.0f : ai.x, tr1 ? 0.0f : ai.y);
    const float2 nbt = make_float2(tr0 ? 0.0f : nbi.x, tr1 ? 0.0f : nbi.y);
    const float2 qfr = make_float2(tr0 ? -k.k12t : qf.x, tr1 ? -k.k12t : qf.y);
    const float2 psa = __fmul2_rn(air, sx);
    nR1 = __ffma2_rn(Pu1, psa, nR1);
    nR1 = __ffma2_rn(qfr, nbi, nR1);
    R2 = __ffma2_rn(sy, __ffma2_rn(Phi, psa, __fmul2_rn(Pu2, nbt)), R2);
    R2 = __ffma2_rn(Pgc, air, R2);
}

// One ordered near pair (target <- source), scalar: tube test on the target's
// normal (FP64 re-decision of near-ties), series g when `series`.
// r = target - source; s_x = r . n_target, s_y = r . m_source, c = n . m.
__device__ __forceinline__ void near_one(float rr, float sx, float sy, float cc, float inv, float xk, float E,
                                         bool tube, bool series, float a_s, float b_s, const F32Consts& k,
                                         float& d1, float& d2)
{
    const float Ex = E * xk;
    float f = 1.0f - E;
    float g = f - Ex;
    if (series && xk < 0.5f) {
        g = g_series(xk);
        f = g + Ex;
    }
    const float hh = fmaf(3.0f, g, -Ex * xk);
    const float inv2 = inv * inv;
    const float i3 = tube ? 0.0f : inv2 * inv;
    const float Q = tube ? k.k12t : f * inv;
    const float u1 = fmaf(k.th1, g, k.omth1);
    const float u2 = fmaf(k.th2, g, k.omth2);
    const float sa = a_s * sy, ca = a_s * cc;
    d1 = fmaf(i3 * u1, sa, -Q * b_s);
    const float v = fmaf(u2, b_s, -(hh * inv2) * sa);
    d2 = i3 * fmaf(g, ca, sx * v);
}

__device__ __forceinline__ bool tube_test(float rr, float s, const F32Consts& k, const Geo64& g64, int64_t it,
                                          int64_t js, int64_t N)
{
    const float rp2 = fmaf(-s, s, rr);
    bool tube = (rp2 < k.tau2) & (rr < k.four_tau2);
    const bool tie = (fabsf(rp2 - k.tau2) < kTieBand * k.tau2) | (fabsf(rr - k.four_tau2) < kTieBand * k.four_tau2);
    if (tie && g64.x != nullptr && it < N && js < N) tube = tube_f64(g64, it, js, k.tau2_d, k.four_tau2_d);
    return tube;
}

// Near pairs of one payload pair, scalar, forward and (when rev) reverse.
template <int TPT>
__device__ __forceinline__ void near_pair_sym(const float3 (&X)[TPT], const SymTargets<TPT>& T, const bool (&rev)[TPT],
                                              const bool (&act)[TPT], const float4& A, const float4& B,
                                              const float4& C, const float4& D, const F32Consts& k,
                                              float2 (&t1)[TPT], float2 (&t2)[TPT], float2 (&r1)[TPT],
                                              float2 (&r2)[TPT], const Geo64& g64, int64_t gi0, int qstride,
                                              int64_t j, int64_t N)
{
    const float yx[2] = {A.x, A.y}, yy[2] = {A.z, A.w}, yz[2] = {B.x, B.y}, bb[2] = {B.z, B.w};
    const float mx[2] = {C.x, C.y}, my[2] = {C.z, C.w}, mz[2] = {D.x, D.y}, aa[2] = {D.z, D.w};
    float rr[TPT][2], sx[TPT][2], sy[TPT][2], cc[TPT][2], inv[TPT][2], xk[TPT][2], E[TPT][2];
    bool need = false;
#pragma unroll
    for (int q = 0; q < TPT; ++q)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float rx = X[q].x + yx[e], ry = X[q].y + yy[e], rz = X[q].z + yz[e];
            const float r2_ = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
            rr[q][e] = r2_;
            sx[q][e] = fmaf(rx, T.nx[q].x, fmaf(ry, T.ny[q].x, rz * T.nz[q].x));
            sy[q][e] = fmaf(rx, mx[e], fmaf(ry, my[e], rz * mz[e]));
            cc[q][e] = fmaf(T.nx[q].x, mx[e], fmaf(T.ny[q].x, my[e], T.nz[q].x * mz[e]));
            const float rrs = fmaxf(r2_, 1.0e-30f);
            inv[q][e] = ptx::rsqrt_approx(rrs);
            const float rho = rrs * inv[q][e];
            xk[q][e] = k.kappa * rho;
            E[q][e] = ptx::ex2_approx(rho * k.kl2e);
            need |= act[q] && (xk[q][e] < 0.5f);
        }
    const bool series = __any_sync(0xffffffffu, need);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        if (!act[q]) continue;
        const int64_t i = gi0 + (int64_t)q * qstride;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float d1, d2;
            const bool tf = tube_test(rr[q][e], sx[q][e], k, g64, i, j + e, N);
            near_one(rr[q][e], sx[q][e], sy[q][e], cc[q][e], inv[q][e], xk[q][e], E[q][e], tf, series, aa[e], bb[e],
                     k, d1, d2);
            float e1 = 0.0f, e2 = 0.0f;
            if (rev[q]) {  // target j <- source i: r' = -r, s_x' = -s_y, s_y' = -s_x
                const bool tr = tube_test(rr[q][e], sy[q][e], k, g64, j + e, i, N);
                near_one(rr[q][e], -sy[q][e], -sx[q][e], cc[q][e], inv[q][e], xk[q][e], E[q][e], tr, series,
                         T.a[q].x, -T.nb[q].x, k, e1, e2);
                e1 = -e1;  // carried negated, as in the far path
            }
            if (e == 0) {
                t1[q].x += d1;
                t2[q].x += d2;
                r1[q].x += e1;
                r2[q].x += e2;
            } else {
                t1[q].y += d1;
                t2[q].y += d2;
                r1[q].y += e1;
                r2[q].y += e2;
            }
        }
    }
}

// Shared reverse-sum layout of one stage: the first-block sums at [0, STILE),
// the second-block sums from rev_off: two words past a 128-byte multiple in
// the warp-reduction scheme, so that the four addresses of one warp_sum4_add
// (2p, 2p + 1 of each block) fall in four different banks; one word past it
// in the rotation scheme, so that the 16 + 16 lanes adding the first and the
// second sums of 16 pairs use the even and the odd banks.
__host__ __device__ constexpr int sym_rev_off(bool rot) { return kF32STile + (rot ? 1 : 2); }
__host__ __device__ constexpr int sym_rev_row(bool rot) { return sym_rev_off(rot) + kF32STile; }

// Sums of four per-lane values over the warp's 32 lanes, added to four
// shared-memory addresses: the values are exchanged half by half (lane^16,
// then lane^8) so that each lane carries one of them, then a 3-step
// butterfly completes the sums; lanes 0, 8, 16 and 24 hold the four totals.
// 6 shuffles and 6 adds instead of 4 x 5 of each for four butterflies.
// v0 and v1 arrive negated (the first reverse sums) and are added negated.
__device__ __forceinline__ void warp_sum4_add(float v0, float v1, float v2, float v3, int lane, float* a0,
                                              float* a1, float* a2, float* a3)
{
    const bool b4 = lane & 16, b3 = lane & 8;
    float ka = b4 ? v2 : v0, kb = b4 ? v3 : v1;
    ka += __shfl_xor_sync(0xffffffffu, b4 ? v0 : v2, 16);
    kb += __shfl_xor_sync(0xffffffffu, b4 ? v1 : v3, 16);
    float k = b3 ? kb : ka;
    k += __shfl_xor_sync(0xffffffffu, b3 ? ka : kb, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    if ((lane & 7) == 0) atomicAdd(b4 ? (b3 ? a3 : a2) : (b3 ? a1 : a0), b4 ? k : -k);
}

// All interactions of one thread's targets with one staged source tile.
// Ablk[q]: chunk index of target slot q's block; B0: chunk index of the
// tile's first chunk.  Forward sums go to the compensated pairs (S, C);
// reverse sums of every source of the tile go to racc[.] (first block) and
// racc[sym_rev_off(ROT) + .] (second block) by shared-memory atomics.  ROT:
// the rotation scheme, far chunks by pair_far_sym_acc and near chunks by
// pair_near_sym_acc, decided per target slot (each slot's 32 targets are one
// block of the warp, so the choice is warp-uniform; inactive slots are
// skipped there); otherwise the warp reduction, near chunks by the scalar
// near_pair_sym.  UNR: unroll depth of the rotation loop over far chunks.
// Measured on the 80k-node sphere (before the packed near path):
// two targets per thread run fastest at 1 (5.65 ms; 5.72 at 2, spills at 4),
// one target per thread at 4 (5.86 ms; 6.11 at 2, 6.22 at 1).
template <int TPT, bool ROT, int UNR = 2>
__device__ __forceinline__ void tile_sums_sym(const SymTargets<TPT>& T, const float4* tfrm, const float4* sb,
                                              const float4* sfrm, const F32Consts& k, float (&S1)[TPT],
                                              float (&C1)[TPT], float (&S2)[TPT], float (&C2)[TPT],
                                              const Geo64& g64, int64_t gi0, int qstride, int64_t j0, int64_t N,
                                              const int (&Ablk)[TPT], int64_t B0, float* racc)
{
    constexpr int P = kPairsPerChunk;
    const FarConsts fc = far_consts(k);
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int c = 0; c < kChunksPerTile; ++c) {
        const int64_t Bc = B0 + c;
        bool act[TPT], rev[TPT];
        bool any = false, anyrev = false;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            act[q] = Bc >= Ablk[q];
            rev[q] = Bc > Ablk[q];
            any |= act[q];
            anyrev |= rev[q];
        }
        if (!any) continue;
        float3 X[TPT];
        bool far = k.rule0 != 0, allact = true;
        bool farq[TPT];  // per slot (one target block per warp and slot: warp-uniform)
        {
            const float4 mh = sfrm[2 * c];
            const float4 ml = sfrm[2 * c + 1];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                const float4 th = tfrm[2 * q];
                const float4 tl = tfrm[2 * q + 1];
                const float dx = (th.x - mh.x) + (tl.x - ml.x);
                const float dy = (th.y - mh.y) + (tl.y - ml.y);
                const float dz = (th.z - mh.z) + (tl.z - ml.z);
                X[q] = make_float3(T.x[q].x + dx, T.x[q].y + dy, T.x[q].z + dz);
                const float lim = k.far_dist + th.w + mh.w;
                farq[q] = (k.rule0 != 0) && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim);
                far = far && farq[q];
                allact = allact && act[q];
            }
        }
        float2 t1[TPT], t2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = make_float2(0.0f, 0.0f);
        const float4* cb = sb + c * P * kPairF4;
        float* ra = racc + c * kChunk;
        float* rb = racc + sym_rev_off(ROT) + c * kChunk;
        if (far || ROT) {  // the rotation scheme takes near chunks too (pair_near_sym_acc)
            float2 Xx[TPT], Xy[TPT], Xz[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                Xx[q] = f2(X[q].x);
                Xy[q] = f2(X[q].y);
                Xz[q] = f2(X[q].z);
            }
            if (ROT) {
                // slots whose reverse direction does not count here add zeros
                float2 aq[TPT], nbq[TPT];
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    aq[q] = rev[q] ? T.a[q] : f2(0.0f);
                    nbq[q] = rev[q] ? T.nb[q] : f2(0.0f);
                }
                const int hl = lane & (P - 1);
                const int nxt = (hl + 1) & (P - 1);
                float2 nR1 = make_float2(0.0f, 0.0f), R2 = make_float2(0.0f, 0.0f);
                if (far && allact) {
#pragma unroll UNR
                    for (int step = 0; step < P; ++step) {
                        const int p = (hl + step) & (P - 1);
                        const float4 A = cb[p], B = cb[P + p], C = cb[2 * P + p], D = cb[3 * P + p];
#pragma unroll
                        for (int q = 0; q < TPT; ++q)
                            pair_far_sym_acc(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], aq[q], nbq[q], A, B, C,
                                             D, fc, t1[q], t2[q], nR1, R2);
                        // pair p goes to lane hl - 1 at the next step: its sums follow it
                        nR1.x = __shfl_sync(0xffffffffu, nR1.x, nxt, P);
                        nR1.y = __shfl_sync(0xffffffffu, nR1.y, nxt, P);
                        R2.x = __shfl_sync(0xffffffffu, R2.x, nxt, P);
                        R2.y = __shfl_sync(0xffffffffu, R2.y, nxt, P);
                    }
                } else {  // a near slot or an inactive one: per slot (uniform branches)
                    const int64_t jc = j0 + (int64_t)c * kChunk;
#pragma unroll 2
                    for (int step = 0; step < P; ++step) {
                        const int p = (hl + step) & (P - 1);
                        const float4 A = cb[p], B = cb[P + p], C = cb[2 * P + p], D = cb[3 * P + p];
#pragma unroll
                        for (int q = 0; q < TPT; ++q) {
                            if (!act[q]) continue;
                            if (TPT > 1 && farq[q])  // (one slot: this loop runs near chunks only)
                                pair_far_sym_acc(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], aq[q], nbq[q], A, B,
                                                 C, D, fc, t1[q], t2[q], nR1, R2);
                            else
                                pair_near_sym_acc(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], aq[q], nbq[q], A,
                                                  B, C, D, fc, k, t1[q], t2[q], nR1, R2, g64,
                                                  gi0 + (int64_t)q * qstride, jc + 2 * p, N);
                        }
                        nR1.x = __shfl_sync(0xffffffffu, nR1.x, nxt, P);
                        nR1.y = __shfl_sync(0xffffffffu, nR1.y, nxt, P);
                        R2.x = __shfl_sync(0xffffffffu, R2.x, nxt, P);
                        R2.y = __shfl_sync(0xffffffffu, R2.y, nxt, P);
                    }
                }
                // lane hl holds pair hl's sums over its half-warp; add the other half's
                nR1.x += __shfl_xor_sync(0xffffffffu, nR1.x, P);
                nR1.y += __shfl_xor_sync(0xffffffffu, nR1.y, P);
                R2.x += __shfl_xor_sync(0xffffffffu, R2.x, P);
                R2.y += __shfl_xor_sync(0xffffffffu, R2.y, P);
                if (anyrev) {
                    if (lane < P) {
                        atomicAdd(ra + 2 * hl, -nR1.x);
                        atomicAdd(ra + 2 * hl + 1, -nR1.y);
                    } else {
                        atomicAdd(rb + 2 * hl, R2.x);
                        atomicAdd(rb + 2 * hl + 1, R2.y);
                    }
                }
            } else {
#pragma unroll 8
                for (int p = 0; p < P; ++p) {
                    const float4 A = cb[p], B = cb[P + p];
                    const float4 C = cb[2 * P + p], D = cb[3 * P + p];
                    float2 s1 = make_float2(0.0f, 0.0f), s2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        float2 r1, r2;
                        pair_far_sym(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], T.a[q], T.nb[q], A, B, C, D,
                                     fc, t1[q], t2[q], r1, r2);
                        if (rev[q]) {
                            s1 = __fadd2_rn(s1, r1);
                            s2 = __fadd2_rn(s2, r2);
                        }
                    }
                    if (anyrev)
                        warp_sum4_add(s1.x, s1.y, s2.x, s2.y, lane, ra + 2 * p, ra + 2 * p + 1, rb + 2 * p,
                                      rb + 2 * p + 1);
                }
            }
        } else {
            for (int p = 0; p < P; ++p) {
                const float4 A = cb[p], B = cb[P + p];
                const float4 C = cb[2 * P + p], D = cb[3 * P + p];
                float2 r1[TPT], r2[TPT];
#pragma unroll
                for (int q = 0; q < TPT; ++q) r1[q] = r2[q] = make_float2(0.0f, 0.0f);
                near_pair_sym<TPT>(X, T, rev, act, A, B, C, D, k, t1, t2, r1, r2, g64, gi0, qstride,
                                   j0 + (int64_t)c * kChunk + 2 * p, N);
                if (anyrev) {
                    float2 s1 = make_float2(0.0f, 0.0f), s2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int q = 0; q < TPT; ++q)
                        if (rev[q]) {
                            s1 = __fadd2_rn(s1, r1[q]);
                            s2 = __fadd2_rn(s2, r2[q]);
                        }
                    warp_sum4_add(s1.x, s1.y, s2.x, s2.y, lane, ra + 2 * p, ra + 2 * p + 1, rb + 2 * p,
                                  rb + 2 * p + 1);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q)
            if (act[q]) {
                kahan_add(S1[q], C1[q], t1[q].x + t1[q].y);
                kahan_add(S2[q], C2[q], t2[q].x + t2[q].y);
            }
    }
}

}  // namespace ibim
