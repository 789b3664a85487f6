// Symmetric FP32 pair sums of the IBIM operator (Sec. 2.2 discrete system,
// Sec. 2.2.1 regularisation), sm_103a.
//
// The pair geometry (r, |r|, e^{-kappa rho}, g, 3 - B, rho^-3, the theta
// terms) is the same for the ordered pairs (i <- j) and (j <- i), so one
// evaluation of an unordered pair gives both contributions: 48 FP32
// lane-operations per pair (28 shared, 10 per direction) instead of 2 x 36.  Each aligned 32-node block pair
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
//     shared buffer.  Near chunks use the warp reduction in both schemes.
#include <algorithm>

#include "pair_f32_core.cuh"

namespace ibim {

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

// pair_far_sym with the reverse sums accumulated into (nR1, R2) inside its
// final FMAs (rotation scheme): nR1 -= first reverse sum, R2 += second.
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
    // reverse, accumulated
    const float2 psa = __fmul2_rn(ai, sx);
    nR1 = __ffma2_rn(P, __fmul2_rn(u1, psa), __ffma2_rn(qf, nbi, nR1));
    const float2 nv = __ffma2_rn(hi, psa, __fmul2_rn(u2, nbi));
    R2 = __ffma2_rn(P, __ffma2_rn(sy, nv, __fmul2_rn(g, __fmul2_rn(ai, cc))), R2);
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
// racc[sym_rev_off(ROT) + .] (second block) by shared-memory atomics.
template <int TPT, bool ROT>
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
        bool far = k.rule0 != 0;
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
                far = far && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim);
            }
        }
        float2 t1[TPT], t2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = make_float2(0.0f, 0.0f);
        const float4* cb = sb + c * P * kPairF4;
        float* ra = racc + c * kChunk;
        float* rb = racc + sym_rev_off(ROT) + c * kChunk;
        if (far) {
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
#pragma unroll 2
                for (int step = 0; step < P; ++step) {
                    const int p = (hl + step) & (P - 1);
                    const float4 A = cb[p], B = cb[P + p], C = cb[2 * P + p], D = cb[3 * P + p];
#pragma unroll
                    for (int q = 0; q < TPT; ++q)
                        pair_far_sym_acc(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], aq[q], nbq[q], A, B, C, D,
                                         fc, t1[q], t2[q], nR1, R2);
                    // pair p goes to lane hl - 1 at the next step: its sums follow it
                    nR1.x = __shfl_sync(0xffffffffu, nR1.x, nxt, P);
                    nR1.y = __shfl_sync(0xffffffffu, nR1.y, nxt, P);
                    R2.x = __shfl_sync(0xffffffffu, R2.x, nxt, P);
                    R2.y = __shfl_sync(0xffffffffu, R2.y, nxt, P);
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

template <int TPT, int MINB, int THREADS, bool ROT>
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
                tile_sums_sym<TPT, ROT>(T, &tfrm[warp][0], stg[stage].buf, stg[stage].frm, k, S1, C1, S2, C2, g64, gi0,
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
__global__ void fixup_sym_kernel(const double* __restrict__ part, SymSchedule s, int ttile, int64_t N, int64_t n_pad,
                                 double lambda1, double lambda2, VecRef in, OutRef out,
                                 const double* __restrict__ yrev, const int* __restrict__ skip)
{
    if (skip != nullptr && *skip) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* p = in.base + (in.kidx ? (int64_t)(*in.kidx + in.koff) * in.stride : 0);
    double* y = out.base + (out.kidx ? (int64_t)(*out.kidx + out.koff) * out.stride : 0);
    const int64_t t = i / ttile;
    const int64_t l = i - t * ttile;
    int64_t start, rho;
    sym_row_start(s, t, start, rho);
    const int64_t c0 = sym_seg_of(s, start);
    const int64_t c1 = sym_seg_of(s, start + sym_row_len(s, t) - 1);
    double a1 = yrev[i], a2 = yrev[n_pad + i];
    // four slots per round with their loads independent (the row's slots are
    // consecutive, 2 ttile doubles apart); a fixed order, so deterministic
    const double* src = part + (c0 + rho) * 2 * ttile + l;
    const int64_t ts = 2 * (int64_t)ttile;
    int64_t c = c0;
    for (; c + 3 <= c1; c += 4, src += 4 * ts) {
        const double x0 = src[0], x1 = src[ts], x2 = src[2 * ts], x3 = src[3 * ts];
        const double y0 = src[ttile], y1 = src[ts + ttile], y2 = src[2 * ts + ttile], y3 = src[3 * ts + ttile];
        a1 += (x0 + x1) + (x2 + x3);
        a2 += (y0 + y1) + (y2 + y3);
    }
    for (; c <= c1; ++c, src += ts) {
        a1 += src[0];
        a2 += src[ttile];
    }
    y[i] = lambda1 * p[i] + kInv4Pi * a1;
    y[N + i] = lambda2 * p[N + i] + kInv4Pi * a2;
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

template <int TPT, int MINB, int THREADS, bool ROT>
static void launch_sym(const SymArgs& a, cudaStream_t st)
{
    pair_sym_kernel<TPT, MINB, THREADS, ROT><<<a.s.grid, THREADS, 0, st>>>(
        a.tpos, a.tnrm, a.src, a.frames, a.N, a.n_pad, a.s, a.k, a.part, a.yrev, a.err, a.skip, a.g64);
}

// scheme: 1 = warp reduction of the reverse sums, 2 = rotation (see the file comment)
struct SymVariant {
    int tpt, minb, threads, scheme;
    const void* fn;
    void (*launch)(const SymArgs&, cudaStream_t);
};
#define IBIM_SYM_VARIANT(T, M, W, R) \
    {T, M, W, (R) ? 2 : 1, (const void*)pair_sym_kernel<T, M, W, R>, launch_sym<T, M, W, R>}
static const SymVariant kSymVariants[] = {
    IBIM_SYM_VARIANT(2, 1, 512, false), IBIM_SYM_VARIANT(1, 1, 512, false),
    IBIM_SYM_VARIANT(2, 1, 512, true), IBIM_SYM_VARIANT(1, 1, 512, true),
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
    const int ttile = v.tpt * v.threads;
    const SymSchedule s = make_sym_schedule(c->N, ttile, grid_cap);
    const int bs = 256;
    fixup_sym_kernel<<<(unsigned)((c->N + bs - 1) / bs), bs, 0, c->stream>>>(
        c->d_part, s, ttile, c->N, padded_nodes(c->N), k.lambda1, k.lambda2, in, out, c->d_yrev, d_skip);
    count_launch(c);
    IBIM_CUDA(cudaGetLastError());
    return IBIM_OK;
}

}  // namespace ibim
