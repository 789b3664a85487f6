// Pair arithmetic, source payload and stage pipeline of the FP32 compensated
// operator, shared by the single-molecule and batched pair-sum kernels.  See
// pair_f32.cu for the formulas, the chunk frames, the near/far split and the
// accumulation.
#pragma once
#include "ibim_internal.cuh"
#include "ptx.cuh"

namespace ibim {

struct F32Consts {
    float th1, th2, omth1, omth2;
    float kappa, kl2e;        // kappa and -kappa log2(e)
    float tau2, four_tau2, k12t;
    float far_dist;           // minimum bounding-sphere gap of a far chunk (A)
    int rule0;                // tube rule 0 (far chunks allowed)
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

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kChunk = 32;                        // chunk = frame block = compensation unit
constexpr int kChunksPerTile = kF32STile / kChunk;
constexpr int kPairsPerChunk = kChunk / 2;

// ------------------------------------------------------------ source payload
//
// Sources are stored by pairs of consecutive nodes (2p, 2p + 1), 64 bytes a
// pair, so that the far-field arithmetic runs on packed float2 operands (one
// lane of the pair per source):
//   [0] = (-y0.x, -y1.x, -y0.y, -y1.y)   minus the position in its chunk frame
//   [1] = (-y0.z, -y1.z,  b0,    b1  )   b = w psin
//   [2] = (a0 m0.x, a1 m1.x, a0 m0.y, a1 m1.y)   a = w psi, m the unit normal
//   [3] = (a0 m0.z, a1 m1.z, 0, 0)
// Node arrays are padded to a multiple of kPadNodes with placeholder nodes
// (a = b = 0, far from every frame) so that every source tile is full.
constexpr int kPairF4 = 4;
constexpr float kPadCoord = 1.0e4f;  // placeholder source coordinate (targets use -kPadCoord)

__device__ __forceinline__ void write_source_pair(float4* __restrict__ dst, float4 y0, float4 y1, float4 m0,
                                                  float4 m1, float a0, float a1, float b0, float b1)
{
    dst[0] = make_float4(-y0.x, -y1.x, -y0.y, -y1.y);
    dst[1] = make_float4(-y0.z, -y1.z, b0, b1);
    dst[2] = make_float4(a0 * m0.x, a1 * m1.x, a0 * m0.y, a1 * m1.y);
    dst[3] = make_float4(a0 * m0.z, a1 * m1.z, 0.0f, 0.0f);
}

__device__ __forceinline__ float4 pad_source_pos() { return make_float4(kPadCoord, kPadCoord, kPadCoord, 0.0f); }
__device__ __forceinline__ float4 pad_target_pos() { return make_float4(-kPadCoord, -kPadCoord, -kPadCoord, 0.0f); }

// ------------------------------------------------------------ arithmetic

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

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Packed constants of the far-field formula.
struct FarConsts {
    float2 kl2e, nkappa, neg1, neg3, th1, omth1, th2, omth2;
};

__device__ __forceinline__ FarConsts far_consts(const F32Consts& k)
{
    FarConsts c;
    c.kl2e = f2(k.kl2e);
    c.nkappa = f2(-k.kappa);
    c.neg1 = f2(-1.0f);
    c.neg3 = f2(-3.0f);
    c.th1 = f2(k.th1);
    c.omth1 = f2(k.omth1);
    c.th2 = f2(k.th2);
    c.omth2 = f2(k.omth2);
    return c;
}

// Far pairs: one target against the two sources of a payload pair, no tube,
// exp-form g: 36 packed FP32 operations and three MUFU operations per source
// (rsqrt, rcp and ex2 on the XU pipe, which has spare throughput here).
// With xn = -kappa rho, En = E xn, fn = E - 1 = -(1 - E), g = -fn + En and
// hn = E x^2 - 3 g = -(3 - B):
//   t1 += rho^-3 u1 (r . a m) + fn rho^-1 b
//   t2 += rho^-3 [g (n . a m) + s_x (u2 b + hn rho^-2 (r . a m))]
// (u1 = 1 - th1 A = omth1 + th1 g, u2 likewise).
__device__ __forceinline__ void pair_far2(float2 Xx, float2 Xy, float2 Xz, float2 nx, float2 ny, float2 nz,
                                          const float4& A, const float4& B, const float4& C, const float4& D,
                                          const FarConsts& c, float2& t1, float2& t2)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 b = make_float2(B.z, B.w);
    const float2 mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w), mz = make_float2(D.x, D.y);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sx = __fmul2_rn(rx, nx);
    sx = __ffma2_rn(ry, ny, sx);
    sx = __ffma2_rn(rz, nz, sx);
    float2 sa = __fmul2_rn(rx, mx);
    sa = __ffma2_rn(ry, my, sa);
    sa = __ffma2_rn(rz, mz, sa);
    float2 ca = __fmul2_rn(nx, mx);
    ca = __ffma2_rn(ny, my, ca);
    ca = __ffma2_rn(nz, mz, ca);
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
    t1 = __ffma2_rn(P, __fmul2_rn(u1, sa), t1);
    t1 = __ffma2_rn(__fmul2_rn(fn, inv), b, t1);
    const float2 v = __ffma2_rn(__fmul2_rn(hn, inv2), sa, __fmul2_rn(u2, b));
    const float2 w = __ffma2_rn(sx, v, __fmul2_rn(g, ca));
    t2 = __ffma2_rn(P, w, t2);
}

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

// Near pairs, packed over the two sources of a payload pair (one target):
// pair_far2's formula with, per lane, g from its series where kappa rho <
// 0.5 (f = 1 - E = g + E x there) and the tube test (Sec. 2.2.1): a
// regularised pair keeps only K12's tube value, by selects on rho^-3 and on
// the 1/rho factor of the first sum.  rho^2 is kept >= 1e-12, so that
// coincident nodes (the self pair among them, always in the tube) leave
// every product finite.  When a test lies within kTieBand of a threshold,
// both sources are decided again in FP64 (tube_f64), which the FP32 test
// agrees with outside the band.  i: the target's node index, j: the first
// source's.
__device__ __forceinline__ void pair_near2(float2 Xx, float2 Xy, float2 Xz, float2 nx, float2 ny, float2 nz,
                                           const float4& A, const float4& B, const float4& C, const float4& D,
                                           const FarConsts& c, const F32Consts& k, float2& t1, float2& t2,
                                           const Geo64& g64, int64_t i, int64_t j, int64_t N)
{
    const float2 rx = __fadd2_rn(Xx, make_float2(A.x, A.y));
    const float2 ry = __fadd2_rn(Xy, make_float2(A.z, A.w));
    const float2 rz = __fadd2_rn(Xz, make_float2(B.x, B.y));
    const float2 b = make_float2(B.z, B.w);
    const float2 mx = make_float2(C.x, C.y), my = make_float2(C.z, C.w), mz = make_float2(D.x, D.y);
    float2 rr = __fmul2_rn(rx, rx);
    rr = __ffma2_rn(ry, ry, rr);
    rr = __ffma2_rn(rz, rz, rr);
    float2 sx = __fmul2_rn(rx, nx);
    sx = __ffma2_rn(ry, ny, sx);
    sx = __ffma2_rn(rz, nz, sx);
    float2 sa = __fmul2_rn(rx, mx);
    sa = __ffma2_rn(ry, my, sa);
    sa = __ffma2_rn(rz, mz, sa);
    float2 ca = __fmul2_rn(nx, mx);
    ca = __ffma2_rn(ny, my, ca);
    ca = __ffma2_rn(nz, mz, ca);
    const float2 rp = __ffma2_rn(__fmul2_rn(sx, c.neg1), sx, rr);
    bool t0 = (rp.x < k.tau2) & (rr.x < k.four_tau2), t1b = (rp.y < k.tau2) & (rr.y < k.four_tau2);
    const float bt = kTieBand * k.tau2, b4 = kTieBand * k.four_tau2;
    const bool tie = (fabsf(rp.x - k.tau2) < bt) | (fabsf(rp.y - k.tau2) < bt) | (fabsf(rr.x - k.four_tau2) < b4) |
                     (fabsf(rr.y - k.four_tau2) < b4);
    if (tie && g64.x != nullptr && i < N) {
        if (j < N) t0 = tube_f64(g64, i, j, k.tau2_d, k.four_tau2_d);
        if (j + 1 < N) t1b = tube_f64(g64, i, j + 1, k.tau2_d, k.four_tau2_d);
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
    const float2 P3 = __fmul2_rn(inv2, inv);
    const float2 P = make_float2(t0 ? 0.0f : P3.x, t1b ? 0.0f : P3.y);
    const float2 qf0 = __fmul2_rn(fn, inv);
    const float2 qf = make_float2(t0 ? -k.k12t : qf0.x, t1b ? -k.k12t : qf0.y);
    const float2 u1 = __ffma2_rn(c.th1, g, c.omth1);
    const float2 u2 = __ffma2_rn(c.th2, g, c.omth2);
    t1 = __ffma2_rn(P, __fmul2_rn(u1, sa), t1);
    t1 = __ffma2_rn(qf, b, t1);
    const float2 v = __ffma2_rn(__fmul2_rn(hn, inv2), sa, __fmul2_rn(u2, b));
    const float2 w = __ffma2_rn(sx, v, __fmul2_rn(g, ca));
    t2 = __ffma2_rn(P, w, t2);
}

// Per-thread target slots: position in the target block's frame and the
// normal, duplicated into both lanes of a float2 for the packed formula.
template <int TPT>
struct Targets {
    float3 x[TPT];
    float2 nx[TPT], ny[TPT], nz[TPT];
};

// All interactions of one thread's targets with one staged source tile
// (kF32STile nodes as kF32STile / 2 payload pairs at sb, chunk frames at
// sfrm).  tfrm: the frames of the warp's target blocks (2 float4 per slot).
// Adds the tile's sums to the compensated pairs (S, C).  gi0: node index of
// the thread's slot-0 target, slot q adding q * qstride.  LIST kernels may
// pass force_far for a tile whose every source is known to lie at least
// far_dist from every target (treecode proxies): it then takes the far-field
// branch without the per-chunk distance test; n_chunks < kChunksPerTile
// skips the tile's trailing chunks (all padding).
template <int TPT, bool LIST = false>
__device__ __forceinline__ void tile_sums(const Targets<TPT>& T, const float4* tfrm, bool have_frames,
                                          const float4* sb, const float4* sfrm, const F32Consts& k,
                                          float (&S1)[TPT], float (&C1)[TPT], float (&S2)[TPT], float (&C2)[TPT],
                                          const Geo64& g64, int64_t gi0, int qstride, int64_t j0, int64_t N,
                                          bool force_far = false, int n_chunks = kChunksPerTile)
{
    const FarConsts fc = far_consts(k);
#pragma unroll 1
    for (int c = 0; c < (LIST ? n_chunks : kChunksPerTile); ++c) {
        // targets in the source chunk's frame; far test on the two bounding spheres
        float3 X[TPT];
        const bool forced = LIST && force_far;
        bool far = (have_frames && k.rule0) || forced;
        bool farq[TPT];  // per slot (one target block per warp and slot: warp-uniform)
#pragma unroll
        for (int q = 0; q < TPT; ++q) farq[q] = far;
        if (have_frames) {
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
                farq[q] = farq[q] && (forced || (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= lim * lim));
                far = far && farq[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < TPT; ++q) X[q] = T.x[q];
        }
        float2 t1[TPT], t2[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) t1[q] = t2[q] = make_float2(0.0f, 0.0f);
        const float4* cb = sb + c * kPairsPerChunk * kPairF4;
        if (far) {
            float2 Xx[TPT], Xy[TPT], Xz[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                Xx[q] = f2(X[q].x);
                Xy[q] = f2(X[q].y);
                Xz[q] = f2(X[q].z);
            }
#pragma unroll 8
            for (int p = 0; p < kPairsPerChunk; ++p) {
                const float4 A = cb[kPairF4 * p], B = cb[kPairF4 * p + 1];
                const float4 C = cb[kPairF4 * p + 2], D = cb[kPairF4 * p + 3];
#pragma unroll
                for (int q = 0; q < TPT; ++q)
                    pair_far2(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], A, B, C, D, fc, t1[q], t2[q]);
            }
        } else {  // near chunk: the packed near formula (tube test per lane) for the near slots
            float2 Xx[TPT], Xy[TPT], Xz[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                Xx[q] = f2(X[q].x);
                Xy[q] = f2(X[q].y);
                Xz[q] = f2(X[q].z);
            }
            const int64_t jc = j0 + (int64_t)c * kChunk;
#pragma unroll 1
            for (int p = 0; p < kPairsPerChunk; ++p) {
                const float4 A = cb[kPairF4 * p], B = cb[kPairF4 * p + 1];
                const float4 C = cb[kPairF4 * p + 2], D = cb[kPairF4 * p + 3];
#pragma unroll
                for (int q = 0; q < TPT; ++q) {
                    if (TPT > 1 && farq[q])  // (one slot: this loop runs near chunks only)
                        pair_far2(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], A, B, C, D, fc, t1[q], t2[q]);
                    else
                        pair_near2(Xx[q], Xy[q], Xz[q], T.nx[q], T.ny[q], T.nz[q], A, B, C, D, fc, k, t1[q], t2[q],
                                   g64, gi0 + (int64_t)q * qstride, jc + 2 * p, N);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            kahan_add(S1[q], C1[q], t1[q].x + t1[q].y);
            kahan_add(S2[q], C2[q], t2[q].x + t2[q].y);
        }
    }
}

// ------------------------------------------------------------ stage pipeline
//
// kF32Stages shared-memory stages, each with a `full` barrier (one producer
// arrival + the bulk-copy bytes) and an `empty` barrier (one arrival per
// warp once it is done with the stage).  Warps consume stages independently;
// thread 0 refills the stage of step u - 1 while at step u, so warps never
// meet at a CTA-wide barrier inside the step loop.
struct SourceStage {
    float4 buf[kF32STile / 2 * kPairF4];
    float4 frm[2 * kChunksPerTile];
};
constexpr uint32_t kStagePayloadBytes = kF32STile / 2 * kPairF4 * sizeof(float4);
constexpr uint32_t kStageFrameBytes = 2 * kChunksPerTile * sizeof(float4);

struct StagePipe {
    uint64_t full[kF32Stages];
    uint64_t empty[kF32Stages];
};

__device__ __forceinline__ void pipe_init(StagePipe& P, int nwarps)
{
    for (int q = 0; q < kF32Stages; ++q) {
        ptx::mbar_init(&P.full[q], 1);
        ptx::mbar_init(&P.empty[q], (uint32_t)nwarps);
    }
    ptx::fence_mbar_init();
}

// Stage a source tile (payload at src, frames at frm or none).
__device__ __forceinline__ void pipe_issue(StagePipe& P, SourceStage& S, int stage, const float4* src,
                                           const float4* frm)
{
    const uint32_t fbytes = frm != nullptr ? kStageFrameBytes : 0u;
    ptx::mbar_arrive_expect_tx(&P.full[stage], kStagePayloadBytes + fbytes);
    ptx::bulk_g2s(&S.buf[0], src, kStagePayloadBytes, &P.full[stage]);
    if (frm != nullptr) ptx::bulk_g2s(&S.frm[0], frm, fbytes, &P.full[stage]);
}

}  // namespace ibim
