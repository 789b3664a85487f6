// Internal declarations of the sm_103a IBIM library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <algorithm>
#include <vector>

#include "../../include/ibim.h"

namespace ibim {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * kPi);
constexpr double kKcalPerE2A = 4.0 * kPi * 332.0637;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
ibim_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define IBIM_CUDA(call)                                                    \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define IBIM_TRY(call)                  \
    do {                                \
        ibim_status _s = (call);        \
        if (_s != IBIM_OK) return _s;   \
    } while (0)

// Device-side error word bits (written by bounded waits instead of trapping).
enum : unsigned { kDevErrTimeout = 1u, kDevErrBounds = 2u };

// Pair-kernel tiling of the FP32 path: a CTA of THREADS threads (a variant
// parameter; kF32Threads on the batched and allocation-free paths), each
// thread owning TPT targets, streams sources through kF32Stages shared-memory
// stages in tiles of kF32STile nodes (32 bytes per node).
constexpr int kF32Threads = 128;
constexpr int kF32Tpt = 2;
constexpr int kF32TTile = kF32Threads * kF32Tpt;
constexpr int kF32STile = 256;
constexpr int kF32Stages = 4;
constexpr int kF32MaxTTile = 1024;  // largest target tile of any variant
// FP32 node arrays (targets, payload, chunk frames) are padded to a multiple
// of kPadNodes placeholder-filled nodes: every source tile and every target
// tile then lies inside the arrays.
constexpr int kPadNodes = 1024;
static_assert(kPadNodes % kF32STile == 0 && kPadNodes % kF32MaxTTile == 0, "padding");
__host__ __device__ inline int64_t padded_nodes(int64_t N) { return (N + kPadNodes - 1) / kPadNodes * kPadNodes; }
// FP64 path: one target per thread, 128 threads, 128 sources per tile.
constexpr int kF64Threads = 128;
constexpr int kF64TTile = kF64Threads;
constexpr int kF64STile = 128;

// Stream-K schedule of a pair-sum launch over (target tile, source tile) steps.
struct PairSchedule {
    int64_t n_ttiles;   // target tiles
    int64_t n_stiles;   // source tiles per target tile
    int64_t total;      // n_ttiles * n_stiles
    int64_t per_cta;    // steps per CTA (last CTA may get fewer)
    int grid;           // CTAs launched (persistent, a multiple of the SM count when possible)
    int max_segs;       // partial slots per CTA
    int64_t sperm;      // source-tile stride: position p of a row visits tile (p * sperm) mod n_stiles
};

// Physical constants of one operator application, in the form the kernels use.
struct PairConsts {
    double lambda1, lambda2;  // diagonal of Lambda
    double th1, th2;          // eps_E/eps_I, eps_I/eps_E
    double kappa;
    double tau2;              // tau^2
    double four_tau2;         // (2 tau)^2 (tube_rule 0) or +inf (tube_rule 1)
    double k12_tube;          // 4 pi x tube value of K12 (1/(4 pi) applied at the end)
};

PairConsts make_consts(const ibim_phys& p);
ibim_status check_phys(const ibim_phys* p);

// --------------------------------------------------------------- context
struct GmresWork;
struct TreeCode;

// Pair-kernel timing: event pairs recorded around each pair-sum launch on the
// launching stream while enabled; summed (and recycled) when read.
struct Timing {
    bool enabled = false;
    double pair_ms = 0.0;
    int64_t pair_launches = 0;
    int64_t pair_interactions = 0;
    int64_t total_launches = 0;
    std::vector<cudaEvent_t> pool;  // 2 events per recorded launch
    size_t used = 0;                // events in use
};

}  // namespace ibim

struct ibim_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int64_t N = 0;
    double h = 0.0;
    double band_eps = 0.0;  // band half-width eps (0 for caller-given nodes)
    double centroid[3] = {0, 0, 0};
    // FP64 geometry, SoA: x*, y*, z*, nx, ny, nz, w (7 arrays of N)
    double* d_geo64 = nullptr;
    double* d_dist = nullptr;     // signed distance per node (0 for caller nodes)
    double* d_curv = nullptr;     // Laplacian of the distance at each node (twice the mean curvature)
    double* d_sig2 = nullptr;     // sum of the 2x2 principal minors of the Hessian of the distance
    double* d_w1 = nullptr;       // the J = 1 weights delta_eps(d) h^3 of a built geometry (else NULL)
    int jacobian = 0;             // 0: weights with J = 1; 1: with the full Jacobian
    int32_t* d_ijk = nullptr;     // grid coordinates (N x 3) or -1
    // FP32 geometry: float4 (x* relative to its 32-node chunk centre, w),
    // float4 (n, 0), and per chunk two float4 (centre hi + radius, centre lo)
    float4* d_pos32 = nullptr;
    float4* d_nrm32 = nullptr;
    float4* d_frames = nullptr;
    // level-set grid of contexts built from atoms (kept for inspection)
    double* d_phi = nullptr;
    int64_t ls_lo[3] = {0, 0, 0};
    int64_t ls_n[3] = {0, 0, 0};
    int64_t ls_cavity_nodes = 0;
    // FP32 pair-kernel variant (index into the compiled table) and CTAs per SM
    // (0 = occupancy limit)
    int f32_variant = 0;
    int f32_bps = 0;
    int tuned = 0;
    // charges
    int64_t Nc = 0;
    double* d_z = nullptr;  // Nc x 3
    double* d_q = nullptr;  // Nc
    // per-application workspaces (grown on demand)
    void* d_src = nullptr;  // packed source payload (largest of FP32 / FP64 layouts)
    size_t src_bytes = 0;
    double* d_part = nullptr;  // stream-K partial sums
    size_t part_bytes = 0;
    double* d_red = nullptr;   // small reduction scratch (energy, area, norms)
    size_t red_bytes = 0;
    unsigned* d_err = nullptr; // device error word (kDevErr* bits), zeroed at build
    double* d_io = nullptr;    // staging for the host-buffer entry points
    size_t io_bytes = 0;
    double* d_aux = nullptr;   // the tau solution of an extrapolated solve
    size_t aux_bytes = 0;
    double* d_yrev = nullptr;  // reverse sums of the symmetric FP32 kernel (2 x padded N) + segment counter
    size_t yrev_bytes = 0;
    float2* d_fftab = nullptr;   // float-float table of 2^(i/256) (IBIM_FF), made on first use
    double ff_grid_scale = 0.0;  // 2^q: grid of the hi parts of float-float coordinates
    int ff_symmetric = 1;        // IBIM_FF kernel: 1 symmetric (each unordered pair once), 0 one-directional
    ibim::GmresWork* gm = nullptr;
    ibim::TreeCode* tc = nullptr;  // treecode tree, lists and proxy buffers (ibim_treecode_setup)
    ibim::Timing timing;
    // incremented whenever a workspace is reallocated: CUDA graphs captured
    // with the old pointers must be re-captured
    uint64_t ws_generation = 0;
    bool ws_sized = false;  // operator workspaces already at their final size
};

namespace ibim {

ibim_status ensure(ibim_ctx* c, void** buf, size_t* have, size_t need);
ibim_status ensure_operator_workspaces(ibim_ctx* c);
// Bracket one pair-sum launch with timing events (no-ops when timing is off).
ibim_status timing_begin(ibim_ctx* c);
ibim_status timing_end(ibim_ctx* c, int64_t interactions);
ibim_status timing_collect(ibim_ctx* c);

// Launch counting (every kernel the library launches goes through this).
inline void count_launch(ibim_ctx* c, int n = 1) { c->timing.total_launches += n; }

// Operator application with the payload already derived from `d_in`.
// `d_in` may be read through an indirection (`d_in_base + (*d_kidx) * stride`)
// so that a captured graph can apply the operator to the current Krylov vector.
struct VecRef {
    const double* base;
    const int* kidx;   // nullptr: base is the vector itself
    int64_t stride;    // elements between consecutive vectors
    int koff;          // offset added to *kidx
};
struct OutRef {
    double* base;
    const int* kidx;
    int64_t stride;
    int koff;
};

ibim_status apply_operator(ibim_ctx* c, const PairConsts& k, int precision, VecRef in, OutRef out,
                           const int* d_skip);
PairSchedule make_schedule(int64_t n_targets, int ttile, int64_t n_sources, int stile, int grid_cap,
                           int64_t max_steps_per_cta_hint = 0);

// FP32 path pieces (pair_f32.cu)
ibim_status f32_pack(ibim_ctx* c, VecRef in, const int* d_skip);
ibim_status f32_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip);
ibim_status f32_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                      const int* d_skip);
int f32_grid_cap(ibim_ctx* c);
int f32_ttile(const ibim_ctx* c);
int f32_max_bps(int variant);
int f32_variant_count();
void f32_variant_info(int v, int* tpt, int* minb, int* threads, int* symmetric);
bool f32_variant_symmetric(int v);
int f32_deterministic_variant();  // the one-directional variant used below kSymTolFloor
// Smallest GMRES tolerance solved with a symmetric FP32 kernel (see gmres_solve).
constexpr double kSymTolFloor = 1e-7;
size_t f32_part_doubles(ibim_ctx* c);  // partial-sum doubles of the current variant and grid
// symmetric FP32 pair kernel (pair_sym.cu)
int sym_variant_count();
void sym_variant_info(int v, int* tpt, int* minb, int* threads, int* scheme);
int sym_occupancy(int v);
size_t sym_part_doubles(int64_t N, int ttile, int grid_cap);
size_t sym_yrev_bytes(int64_t N);
ibim_status sym_pack(ibim_ctx* c, VecRef in, const int* d_skip);
ibim_status sym_pairs(ibim_ctx* c, int sv, int grid_cap, const PairConsts& k, const int* d_skip);
ibim_status sym_fixup(ibim_ctx* c, int sv, int grid_cap, const PairConsts& k, VecRef in, OutRef out,
                      const int* d_skip);
ibim_status sym_fixup_tiles(ibim_ctx* c, int ttile, int grid_cap, const PairConsts& k, VecRef in, OutRef out,
                            const int* d_skip);
PairSchedule f32_schedule(ibim_ctx* c);
ibim_status f32_chunk_frames(ibim_ctx* c);
ibim_status f32_pack_to(ibim_ctx* c, VecRef in, float4* dst, const int* d_skip);
// treecode form of the FP32 operator (treecode.cu)
ibim_status tc_setup(ibim_ctx* c, double theta, double tau_max, int order, int interp);
ibim_status tc_apply(ibim_ctx* c, const PairConsts& k, VecRef in, OutRef out, const int* d_skip);
void tc_destroy(TreeCode* t);
ibim_status fixup_launch(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, int ttile, VecRef in,
                         OutRef out, const int* d_skip);
// float-float path (pair_ff.cu)
PairSchedule ff_schedule(ibim_ctx* c);
size_t ff_part_doubles(ibim_ctx* c);
size_t ff_src_bytes(int64_t N);
ibim_status ff_pack(ibim_ctx* c, VecRef in, const int* d_skip);
ibim_status ff_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip);
ibim_status ff_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                     const int* d_skip);
ibim_status ff_prepare_context(ibim_ctx* c);
// FP64 path pieces (pair_f64.cu)
ibim_status f64_pack(ibim_ctx* c, VecRef in, const int* d_skip);
ibim_status f64_pairs(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, const int* d_skip);
ibim_status f64_fixup(ibim_ctx* c, const PairConsts& k, const PairSchedule& s, VecRef in, OutRef out,
                      const int* d_skip);
int f64_grid_cap(ibim_ctx* c);

// RHS / energy / area (rhs_energy.cu)
ibim_status rhs_launch(ibim_ctx* c, double eps_in, double* d_g);
ibim_status energy_launch(ibim_ctx* c, const ibim_phys& p, const double* d_p, double* d_psi,
                          double* gpol_host);
ibim_status area_launch(ibim_ctx* c, double* area_host);

// Geometry (geometry.cu)
ibim_status build_sphere_nodes(ibim_ctx* c, double R, const double* centre, const double* origin,
                               double h, double eps);
// FP32 packing relative to c->centroid and chunk frames; `reorder` first puts
// the nodes into compact aligned 32-node blocks (built geometries only).
ibim_status finish_geometry(ibim_ctx* c, bool reorder);
// Level-set SES (levelset.cu)
ibim_status build_levelset(ibim_ctx* c, int64_t Na, const double* z, const double* r, double probe, double h,
                           double eps);
void apply_cached_tuning(ibim_ctx* c);      // tune.cu

// GMRES (gmres.cu)
ibim_status gmres_solve(ibim_ctx* c, const ibim_phys& p, const ibim_solve_opts& o, double* d_p,
                        ibim_solve_info* info);
void gmres_free(ibim_ctx* c);
ibim_status batch_solve(int nmol, ibim_ctx* const* ctxs, const ibim_phys* phys, const ibim_solve_opts& o,
                        double* const* d_p, ibim_solve_info* infos);
int batch_variant_count();
void batch_variant_info(int v, int* tpt, int* threads, int* symmetric);
void batch_force_variant(int v);
int batch_last_variant_used();

}  // namespace ibim
