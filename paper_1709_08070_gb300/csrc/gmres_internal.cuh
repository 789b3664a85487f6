// Internal GMRES pieces shared by the single-molecule and batched solvers.
#pragma once
#include "ibim_internal.cuh"

namespace ibim {

constexpr int kMaxRestart = 128;
constexpr int kVecThreads = 256;

struct GmState {
    int k;       // current Arnoldi step within the cycle
    int done;    // stop expanding (converged, cycle full or breakdown)
    int conv;    // residual estimate below target
    int kmax;    // steps allowed in this cycle
    int m;       // restart length (row stride of H)
    int pad;
    double target;     // absolute residual target of the cycle
    double resid;      // |e_{k}| after the last rotation
    double hn;         // ||w|| of the current step
    double coef[kMaxRestart + 1];  // Gram-Schmidt coefficients of the current pass
    double hcol[kMaxRestart + 1];  // accumulated column k of H
    double cs[kMaxRestart], sn[kMaxRestart];
    double e[kMaxRestart + 1];
    double y[kMaxRestart];
    double H[(kMaxRestart + 1) * kMaxRestart];  // row-major, row stride m
};

struct GmresWork {
    int m = 0;
    int64_t len = 0;
    double* V = nullptr;       // (m + 1) x len
    double* x = nullptr;       // len: current iterate (solution accumulator)
    double* r = nullptr;       // len: residual / scratch
    double* t = nullptr;       // len: operator output scratch
    double* g = nullptr;       // len: right-hand side
    double* xb = nullptr;      // len: refinement base iterate (x holds the correction to it)
    double* gin = nullptr;     // len: refinement right-hand side (residual at xb)
    double* part = nullptr;    // per-block partial sums ((m + 1) x nblk)
    int nblk = 0;
    GmState* st = nullptr;     // device state
    GmState* h_st = nullptr;   // pinned host mirror (small fields only are read)
    cudaStream_t gs = nullptr; // capture-capable stream owned by the solver
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_prec = 0;
    PairConsts graph_k;
    uint64_t graph_generation = 0;  // workspace generation the graph was captured with
    int graph_variant = -1;         // FP32 pair-kernel variant and CTAs per SM captured in the graph
    int graph_bps = -1;
    bool graph_valid = false;
};


// Building blocks (gmres.cu); every launch goes on c->stream.
ibim_status gm_alloc(ibim_ctx* c, int m);
ibim_status gm_init(ibim_ctx* c, const ibim_phys& p, int m, double* gnorm);  // state, g, ||g||, x = 0; syncs
ibim_status gm_ortho(ibim_ctx* c);  // CGS2 + norm + scale + Givens of one Arnoldi step (after w = A v_k)
ibim_status gm_cycle_begin(ibim_ctx* c, bool x_zero, double target, int kmax);  // r = g - t (t = A x), V0, e
ibim_status gm_cycle_end(ibim_ctx* c);  // y = H^-1 e, x += V y
ibim_status gm_fetch_state(ibim_ctx* c);  // async copy of the small state fields to the pinned mirror

}  // namespace ibim
