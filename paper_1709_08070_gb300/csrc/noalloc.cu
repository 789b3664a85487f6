// Allocation-free FP32 compensated operator application.
//
// Some callers cannot allocate device memory: code running where cudaMalloc
// is off limits (inside a host callback, under a memory pool owned by another
// runtime, in a process whose allocator is frozen after start-up) or that must
// not add allocations a memory budget does not account for.  This entry point
// computes the same product as ibim_matvec with IBIM_F32C from caller-owned
// geometry and vectors, and takes its working memory (FP32 node copies in
// their 32-node chunk frames, the frames, the packed source payload, the
// per-CTA partial sums, an error word) from one file-scope device array of
// fixed size.  The array exists on every GPU that loads the library, from
// load until process exit.
#include <mutex>

#include "pair_f32_core.cuh"

namespace ibim {

PairSchedule make_schedule(int64_t n_targets, int ttile, int64_t n_sources, int stile, int grid_cap, int64_t);
int f32_occupancy_per_sm();
cudaError_t launch_pair_f32_raw(const float4* tpos, const float4* tnrm, const float4* src, const float4* frames,
                                int64_t N, const PairSchedule& s, const PairConsts& k, double* part, unsigned* err,
                                cudaStream_t stream, const double* xs_aos, const double* nrm_aos);
cudaError_t launch_fixup_raw(const double* part, const PairSchedule& s, int64_t N, const PairConsts& k,
                             const double* d_in, double* d_out, cudaStream_t stream);

namespace {

constexpr int64_t kMaxNodes = IBIM_NOALLOC_MAX_NODES;
constexpr int kMaxCtas = 1024;  // persistent CTAs per launch at most
constexpr int kMaxSegs = 2;     // partial slots per CTA (enough once the grid has >= one CTA per target tile)
constexpr size_t kHeadBytes = 256;  // error word
constexpr size_t kPosBytes = sizeof(float4) * (size_t)kMaxNodes;
constexpr size_t kFrameBytes = 2 * sizeof(float4) * (size_t)(kMaxNodes / kChunk);
constexpr size_t kSrcBytes = 2 * sizeof(float4) * (size_t)kMaxNodes;
static_assert(kMaxNodes % kPadNodes == 0, "the padded node range must fit the static arrays");
constexpr size_t kPartDoubles = (size_t)kMaxCtas * kMaxSegs * 2 * kF32TTile;
constexpr size_t kScratchBytes =
    kHeadBytes + 2 * kPosBytes + kFrameBytes + kSrcBytes + kPartDoubles * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[128] = {};  // device address of g_noalloc_scratch per device ordinal

// Device address of the scratch array on the current device (looked up once
// per device; the lookup must not happen inside a stream capture).
ibim_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 128) {
        set_error("device ordinal out of range");
        return IBIM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)", __FILE__, __LINE__);
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return IBIM_OK;
}

// Frames of the aligned 32-node chunks of the caller's nodes (x* as N x 3
// row-major FP64): the chunk centre split into hi + lo floats with the chunk
// radius, and every node's position relative to its chunk centre with its
// weight in .w.  Chunks past N get a zero frame and placeholder targets.  The
// same frames as a context's geometry, so the pair kernel forms the offsets
// of close pairs from small numbers however far the nodes lie from the origin.
// One thread per chunk.
__global__ void noalloc_frames_kernel(const double* __restrict__ xs, const double* __restrict__ w, int64_t N,
                                      int64_t n_chunks, float4* __restrict__ rel, float4* __restrict__ frames)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const int64_t j0 = c * kChunk;
    const int64_t j1 = (j0 + kChunk < N) ? j0 + kChunk : (N > j0 ? N : j0);
    for (int64_t j = j1; j < j0 + kChunk; ++j) rel[j] = pad_target_pos();
    if (j1 == j0) {
        frames[2 * c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        frames[2 * c + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        cx += xs[3 * j];
        cy += xs[3 * j + 1];
        cz += xs[3 * j + 2];
    }
    const double inv = 1.0 / (double)(j1 - j0);
    cx *= inv;
    cy *= inv;
    cz *= inv;
    double r2 = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double dx = xs[3 * j] - cx, dy = xs[3 * j + 1] - cy, dz = xs[3 * j + 2] - cz;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
        rel[j] = make_float4((float)dx, (float)dy, (float)dz, (float)w[j]);
    }
    const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
    frames[2 * c] = make_float4(hx, hy, hz, (float)(sqrt(r2) * 1.0001 + 1e-4));
    frames[2 * c + 1] = make_float4((float)(cx - (double)hx), (float)(cy - (double)hy), (float)(cz - (double)hz), 0.0f);
}

// FP32 normals and the source payload of the padded node range (one thread
// per node pair; placeholders past N), source positions in their chunk frames.
__global__ void noalloc_pack_kernel(const float4* __restrict__ tpos, const double* __restrict__ nrm,
                                    const double* __restrict__ w, const double* __restrict__ p, int64_t N,
                                    int64_t n_pairs, float4* __restrict__ tnrm, float4* __restrict__ src)
{
    const int64_t pr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= n_pairs) return;
    float4 y[2], m[2];
    float a[2], b[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int64_t j = 2 * pr + e;
        if (j < N) {
            y[e] = tpos[j];
            m[e] = make_float4((float)nrm[3 * j], (float)nrm[3 * j + 1], (float)nrm[3 * j + 2], 0.0f);
            const double wj = w[j];
            a[e] = (float)(wj * p[j]);
            b[e] = (float)(wj * p[N + j]);
        } else {
            y[e] = pad_source_pos();
            m[e] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            a[e] = b[e] = 0.0f;
        }
        tnrm[j] = m[e];
    }
    write_source_pair(src + kPairF4 * pr, y[0], y[1], m[0], m[1], a[0], a[1], b[0], b[1]);
}

}  // namespace
}  // namespace ibim

using namespace ibim;

extern "C" ibim_status ibim_matvec_noalloc(int64_t N, const double* d_xstar, const double* d_normal,
                                           const double* d_w, const ibim_phys* phys, const double* d_in,
                                           double* d_out, void* stream)
{
    if (N < 1 || N > kMaxNodes) {
        set_error("ibim_matvec_noalloc: N must be in [1, IBIM_NOALLOC_MAX_NODES = 131072]");
        return IBIM_ERR_ARG;
    }
    if (!d_xstar || !d_normal || !d_w || !d_in || !d_out) {
        set_error("ibim_matvec_noalloc: NULL pointer");
        return IBIM_ERR_ARG;
    }
    {
        // the fixup reads d_in while other threads write d_out: reject any
        // overlap of the two 2N-double ranges
        const uintptr_t a0 = (uintptr_t)d_in, b0 = (uintptr_t)d_out;
        const uintptr_t len = (uintptr_t)(2 * N) * sizeof(double);
        if (a0 < b0 + len && b0 < a0 + len) {
            set_error("ibim_matvec_noalloc: the ranges d_in[0, 2N) and d_out[0, 2N) must not overlap");
            return IBIM_ERR_ARG;
        }
    }
    IBIM_TRY(check_phys(phys));
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    IBIM_CUDA(cudaGetDevice(&dev));
    IBIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned char* base = nullptr;
    IBIM_TRY(scratch_address(dev, &base));
    unsigned* err = reinterpret_cast<unsigned*>(base);
    float4* tpos = reinterpret_cast<float4*>(base + kHeadBytes);
    float4* tnrm = reinterpret_cast<float4*>(base + kHeadBytes + kPosBytes);
    float4* frames = reinterpret_cast<float4*>(base + kHeadBytes + 2 * kPosBytes);
    float4* src = reinterpret_cast<float4*>(base + kHeadBytes + 2 * kPosBytes + kFrameBytes);
    double* part = reinterpret_cast<double*>(base + kHeadBytes + 2 * kPosBytes + kFrameBytes + kSrcBytes);

    const PairConsts k = make_consts(*phys);
    // At least one CTA per target tile keeps every CTA within two target tiles.
    const int n_ttiles = (int)((N + kF32TTile - 1) / kF32TTile);
    int cap = f32_occupancy_per_sm() * sms;
    if (cap < n_ttiles) cap = n_ttiles;
    if (cap > kMaxCtas) cap = kMaxCtas;
    const PairSchedule s = make_schedule(N, kF32TTile, N, kF32STile, cap, 0);
    if ((size_t)s.grid * s.max_segs * 2 * kF32TTile > kPartDoubles) {
        set_error("ibim_matvec_noalloc: schedule needs more partial slots than the static region holds");
        return IBIM_ERR_ARG;
    }
    IBIM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    const int64_t n_pad = padded_nodes(N);
    const int64_t n_chunks = n_pad / kChunk;
    noalloc_frames_kernel<<<(unsigned)((n_chunks + 127) / 128), 128, 0, st>>>(d_xstar, d_w, N, n_chunks, tpos,
                                                                             frames);
    IBIM_CUDA(cudaGetLastError());
    const int bs = 256;
    const int64_t n_pairs = n_pad / 2;
    noalloc_pack_kernel<<<(unsigned)((n_pairs + bs - 1) / bs), bs, 0, st>>>(tpos, d_normal, d_w, d_in, N, n_pairs,
                                                                           tnrm, src);
    IBIM_CUDA(cudaGetLastError());
    IBIM_CUDA(launch_pair_f32_raw(tpos, tnrm, src, frames, N, s, k, part, err, st, d_xstar, d_normal));
    IBIM_CUDA(launch_fixup_raw(part, s, N, k, d_in, d_out, st));
    unsigned h_err = 0;
    IBIM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    IBIM_CUDA(cudaStreamSynchronize(st));
    if (h_err & kDevErrTimeout) {
        set_error("ibim_matvec_noalloc: a bounded device wait gave up");
        return IBIM_ERR_DEVICE_TIMEOUT;
    }
    return IBIM_OK;
}
