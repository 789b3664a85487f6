/*
 * ibim.h -- C ABI of the GB300 (sm_103a) implementation of the implicit
 * boundary integral method (IBIM) for the linearized Poisson-Boltzmann
 * equation (Zhong, Ren, Tsai, arXiv 1709.08070).
 *
 * Conventions shared by every entry point
 *   - Lengths in Angstrom, charges in units of e.  Potentials follow the
 *     paper's psi = q / (4 pi eps r) convention (Sec. 4.2); energies are
 *     returned in e^2/Angstrom and, where stated, in kcal/mol
 *     (x 4 pi 332.0637).
 *   - The unknown of the discrete system (Sec. 2.2, Sec. 3.3) is the 2N vector
 *     p = [psi_bar(0..N-1); psin_bar(0..N-1)] of FP64 values, where psin is
 *     the interior-side normal derivative (Sec. 2.1).  Node j carries its
 *     projection x*_j, unit normal n(x*_j) and weight w_j = J delta_eps(d_j) h^3.
 *   - Pointers named d_* are device pointers on the context's device;
 *     pointers named h_* (or plain host arrays) are host memory.  Caller
 *     arrays are borrowed for the duration of the call only; the context owns
 *     every buffer it allocates and frees them in ibim_destroy.
 *   - All GPU work of a context is issued on the CUDA stream given at build
 *     time (a cudaStream_t passed as void*; NULL is the legacy default
 *     stream).  Calls returning host values synchronise that stream.
 *   - No entry point throws, exits or traps.  Each returns an ibim_status;
 *     ibim_last_error() gives a message for the last failure on the calling
 *     thread.  A context is not thread-safe: serialise calls on one context.
 */
#ifndef IBIM_H
#define IBIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibim_ctx ibim_ctx;

typedef enum {
    IBIM_OK = 0,
    IBIM_ERR_ARG = 1,            /* invalid argument (NULL, size, parameter range) */
    IBIM_ERR_EMPTY_BAND = 2,     /* the narrowband holds no grid node */
    IBIM_ERR_NONFINITE = 3,      /* NaN/Inf in an input */
    IBIM_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has details) */
    IBIM_ERR_NOT_CONVERGED = 5,  /* GMRES spent maxit iterations above tolerance */
    IBIM_ERR_DEVICE_TIMEOUT = 6, /* a bounded device-side wait gave up */
    IBIM_ERR_STATE = 7           /* call not valid in the context's state (e.g. no charges) */
} ibim_status;

/* Arithmetic of the pair sums (the N x N kernel evaluations). */
typedef enum {
    IBIM_F64 = 64,  /* plain FP64 pair sums */
    IBIM_FF = 65,   /* float-float ("double-single") pair sums on the FP32 pipe: every
                       quantity an unevaluated sum of two floats (about 48 bits), exp by a
                       table-driven reduction, 1/rho by a Newton step, tube ties decided in
                       FP64; the same operator as IBIM_F64 to within 1e-10 of max |y| per
                       element, several times faster on a GPU whose FP64 rate is a small
                       fraction of its FP32 rate */
    IBIM_F32C = 32, /* FP32 pair sums, Kahan-compensated per source tile, tile sums in FP64 */
    IBIM_F32T = 33  /* as IBIM_F32C near each target tile, far clusters through Chebyshev
                       proxies (ibim_treecode_setup first; tube rule 0 only) */
} ibim_precision;

/*
 * Physical and regularisation parameters.
 *   eps_in, eps_out : dielectric constants eps_I, eps_E (> 0), Sec. 1.
 *   kappa           : screening constant kappa >= 0 (1/Angstrom), used directly
 *                     in G_kappa = exp(-kappa r)/(4 pi r), Sec. 2.1.
 *   tau             : regularisation radius (> 0, Angstrom), Sec. 2.2.1.
 *   tube_rule       : 0 = a pair is regularised iff its tangent-plane distance
 *                     ||x*-y*||_P < tau and |x*-y*| < 2 tau; 1 = the tangent-plane
 *                     test alone, as printed in Sec. 2.2.1.
 * Inside the tube K11 = K21 = K22 = 0 and
 * K12 = (exp(-kappa tau) - 1 + kappa tau)/(2 pi kappa tau^2) (0 at kappa = 0).
 */
typedef struct {
    double eps_in;
    double eps_out;
    double kappa;
    double tau;
    int tube_rule;
} ibim_phys;

/* ------------------------------------------------------------------ build */

/*
 * Solvent excluded surface of a molecule and its narrowband (paper Stages 1-2,
 * Sec. 3.1-3.2), all on the GPU in FP64: vdW level set F = min_k(|x-z_k|-r_k)
 * (clamped at 2 probe + band_eps + 6h), phi_SAS = F - probe, inward eikonal
 * flow for t in (0, probe] (TVD-RK3, Godunov, WENO5, zero Neumann), cavity
 * removal (flood fill of phi > 0 from the box boundary; other phi > 0 nodes and
 * every node within band_eps of them set to -band_eps), reinitialisation
 * (ceil((k1+4)/k0) steps, dt = k0 h, k0 = 1/2, k1 = band_eps/h), band
 * {|phi| < band_eps} with WENO5 normals, projections x* = x - phi n and
 * weights delta_eps(phi) h^3.  Grid: nodes h * (integer coordinates) covering
 * the atoms' extent plus probe + band_eps + 8h.  Node order: compact aligned
 * blocks of 32 nodes by recursive coordinate bisection of x* (ties by index).
 *   xyz: Na x 3 host centres (A); radii: Na host (> 0); charges: Na host or
 *   NULL (when given they become the context's charges at the centres);
 *   probe >= 0 (rho0), h > 0, band_eps > 0 (eps).
 * Errors: IBIM_ERR_ARG, IBIM_ERR_NONFINITE, IBIM_ERR_EMPTY_BAND, IBIM_ERR_CUDA.
 */
ibim_status ibim_build(const double* xyz, const double* radii, const double* charges, int64_t Na, double probe,
                       double h, double band_eps, void* stream, ibim_ctx** out);

/* Level-set grid of a context built by ibim_build: integer coordinate of node
 * (0,0,0) in lo[3], node counts in n[3], and (when phi is not NULL) the final
 * phi on the grid, n[0] n[1] n[2] doubles with x fastest.  Synchronises. */
ibim_status ibim_get_levelset(const ibim_ctx* ctx, int64_t* lo, int64_t* n, double* phi);

/*
 * Narrowband of an analytic sphere (signed distance d(x) = |x - c| - R),
 * Sec. 2.2 and Sec. 3.2 with J = 1.  Grid U_h = origin + h Z^3; nodes with
 * |d| < band_eps are kept, x* = c + R (x - c)/|x - c|, n = (x - c)/|x - c|,
 * w = delta_eps(d) h^3 (cosine weight).  Node order: compact aligned blocks of
 * 32 nodes by recursive coordinate bisection of x* (use ibim_get_nodes for the
 * grid coordinates of each node).
 *   R > 0, h > 0, band_eps > 0; centre/origin: host double[3] (origin may be NULL = 0).
 * Errors: IBIM_ERR_ARG, IBIM_ERR_EMPTY_BAND, IBIM_ERR_CUDA.
 */
ibim_status ibim_build_sphere(double R, const double* centre, const double* origin, double h,
                              double band_eps, void* stream, ibim_ctx** out);

/*
 * Context from caller-given nodes (host arrays, copied): x* (N x 3, row-major),
 * unit normals (N x 3), weights w (N).  h is informational (> 0).  Nodes keep
 * the caller's order; the FP32 operator is fastest when every aligned block of
 * 32 consecutive nodes is spatially compact (its far-field path is taken per
 * pair of blocks whose bounding spheres are apart).
 * Errors: IBIM_ERR_ARG (N <= 0, NULL), IBIM_ERR_NONFINITE.
 */
ibim_status ibim_build_from_nodes(int64_t N, const double* xstar, const double* normal,
                                  const double* w, double h, void* stream, ibim_ctx** out);

/* Point charges z_k (Nc x 3 host, row-major) and q_k (Nc host) used by the
 * right-hand side and the energy; replaces earlier charges.  Nc >= 1. */
ibim_status ibim_set_charges(ibim_ctx* ctx, int64_t Nc, const double* z, const double* q);

ibim_status ibim_num_nodes(const ibim_ctx* ctx, int64_t* N);

/* Host copies of the node data in the context's order; any pointer may be NULL.
 * xstar, normal: N x 3; w, d: N; ijk: N x 3 grid coordinates (int32; all -1 for
 * caller-given nodes); d is the signed distance (0 for caller-given nodes). */
ibim_status ibim_get_nodes(const ibim_ctx* ctx, double* xstar, double* normal, double* w,
                           double* d, int32_t* ijk);

/* Per-node Laplacian of the signed distance at the grid node (twice the mean
 * curvature of the level surface through it): 2/|x - c| on analytic spheres,
 * second central differences of phi for ibim_build, 0 for caller-given nodes.
 * curv: host, N doubles. */
ibim_status ibim_get_curvature(const ibim_ctx* ctx, double* curv);

/*
 * Full Jacobian of the change of variables between Gamma and the level
 * surface of the distance through each node (Sec. 2.2): J = 1 - d lap(d) +
 * d^2 sigma2(Hess d), the printed last term read as the sum of the 2x2
 * principal minors of the Hessian (so J = (1 - d k1)(1 - d k2) in the level
 * surface's principal curvatures; (R/|x - c|)^2 on a sphere), clamped at 0
 * where the band is wider than a local radius of curvature.  Spheres use the
 * exact derivatives, level sets central differences of phi.
 * ibim_set_jacobian: mode 0 (default, every run of the paper) weights
 * w = delta_eps(d) h^3; mode 1 weights w = J delta_eps(d) h^3, which removes
 * the O(eps^2) bias of the J = 1 weights (a sphere's area becomes 4 pi R^2
 * instead of 4 pi (R^2 + c eps^2)).  Applies to the following operator
 * applications, solves, energies and areas; synchronises.
 * ibim_get_jacobian: host copy of J per node (N doubles).
 * Both return IBIM_ERR_STATE for caller-given nodes (ibim_build_from_nodes:
 * no distance function; mode 0 is accepted and changes nothing).
 */
ibim_status ibim_set_jacobian(ibim_ctx* ctx, int mode);
ibim_status ibim_get_jacobian(const ibim_ctx* ctx, double* J);

/* ----------------------------------------------------------- operator etc. */

/*
 * d_out = (Lambda + K W) d_in, the discrete system of Sec. 2.2 / final linear
 * system of Sec. 3.3, with Lambda = diag((1+eps_E/eps_I)/2 I, (1+eps_I/eps_E)/2 I)
 * and the regularised kernels of Sec. 2.2.1:
 *   y1_i = lambda1 psi_i  + sum_j [K11(i,j) w_j psi_j - K12(i,j) w_j psin_j]
 *   y2_i = lambda2 psin_i + sum_j [K21(i,j) w_j psi_j - K22(i,j) w_j psin_j]
 * d_in, d_out: device, 2N doubles each, must not overlap.  Asynchronous on
 * the context stream.  precision: IBIM_F64, IBIM_FF, IBIM_F32C or IBIM_F32T.
 */
ibim_status ibim_matvec(ibim_ctx* ctx, const ibim_phys* phys, int precision, const double* d_in,
                        double* d_out);

/* Same product with host buffers (copies in, computes, copies out, synchronises). */
ibim_status ibim_matvec_host(ibim_ctx* ctx, const ibim_phys* phys, int precision,
                             const double* h_in, double* h_out);

/* Right-hand side g = [g1; g2] (Sec. 2.2): g1_i = sum_k q_k/eps_I G0(x*_i, z_k),
 * g2_i = sum_k q_k/eps_I dG0(x*_i, z_k)/dn(x*_i).  d_g: device, 2N doubles.
 * Needs charges (IBIM_ERR_STATE otherwise). */
ibim_status ibim_rhs(ibim_ctx* ctx, double eps_in, double* d_g);

/*
 * Reaction potential psi_rxn(z_k) (Sec. 3.5, IBIM sum over the band nodes) and
 * G_pol = 1/2 sum_k q_k psi_rxn(z_k).  d_p: device 2N solution; d_psi_rxn:
 * device Nc doubles or NULL; gpol: host, e^2/Angstrom.  Synchronises.
 */
ibim_status ibim_energy(ibim_ctx* ctx, const ibim_phys* phys, int precision, const double* d_p,
                        double* d_psi_rxn, double* gpol);

/* Surface area sum_j w_j (Sec. 3.4, f = 1).  Synchronises. */
ibim_status ibim_area(ibim_ctx* ctx, double* area);

/* ------------------------------------------------------------------ solve */

typedef struct {
    int precision;  /* IBIM_F64, IBIM_FF, IBIM_F32C or IBIM_F32T: operator used inside GMRES */
    double tol;     /* relative residual ||g - A p||_2 / ||g||_2 target (e.g. 1e-6)      */
    int maxit;      /* maximum Arnoldi steps in total                                    */
    int restart;    /* GMRES restart length m (1..128)                                   */
    int start;      /* 0: p0 = 0; 1: p0 = Lambda^-1 g (Sec. 3.3); 3: caller's d_p on entry */
    int certify;    /* 1: after convergence recompute the residual with an FP64-accurate
                       operator (IBIM_FF) and restart from the current p while it is
                       above tol (iterative refinement); 2: the same with the plain FP64
                       operator (IBIM_F64); 0: residuals use the chosen operator        */
} ibim_solve_opts;

typedef struct {
    int iters;           /* Arnoldi steps taken (the paper's GMRES iteration count)     */
    int cycles;          /* GMRES cycles (restarts + refinement passes)                 */
    int converged;       /* 1 when the reported residual is below tol                   */
    double relres;       /* final ||g - A p|| / ||g|| (FP64-accurate operator when certify > 0) */
    double gpol;         /* G_pol, e^2/Angstrom                                          */
    double gpol_kcal;    /* G_pol, kcal/mol                                              */
    double area;         /* surface area (Angstrom^2)                                    */
    int64_t matvecs_f32; /* operator applications by precision: FP32 (IBIM_F32C/F32T)    */
    int64_t matvecs_f64; /* and FP64-accurate (IBIM_F64 and IBIM_FF)                     */
} ibim_solve_info;

/*
 * Solve (Lambda + K W) p = g by restarted GMRES (Sec. 3.3) with FP64 Arnoldi
 * (classical Gram-Schmidt with one re-orthogonalisation), FP64 Givens
 * least squares on the device and the operator of opts->precision, then
 * evaluate G_pol (Sec. 3.5) and the area (Sec. 3.4).  Each Arnoldi step runs
 * as one CUDA graph replay with no host synchronisation inside the step.
 * The symmetric FP32 kernels vary from one application to the next by about
 * 1e-8 of |A p| (their reverse sums are added in a varying order), which is
 * the floor of a restart residual computed with them; an uncertified
 * IBIM_F32C solve with tol below 1e-7 therefore runs the one-directional FP32
 * kernel (the context's variant is restored afterwards).  Certified solves
 * (opts->certify > 0) keep the context's variant at any tol: after the first
 * FP64-accurate residual misses tol, the iteration solves the correction
 * equation A e = r from e = 0 (restart residuals r - A e, noise relative to
 * |r|) and adds e before the next check (iterative refinement).  A cycle that
 * converges by its own estimate leads to the FP64-accurate check at once (no
 * FP32 restart residual first: it could only confirm the estimate or show the
 * FP32 operator's accuracy, about 1e-8 of |A p|).
 * d_p: device 2N doubles; start vector on entry when opts->start == 3,
 * solution [psi; psin] on exit.  Needs charges.  Returns IBIM_ERR_NOT_CONVERGED
 * (info filled) when maxit is reached above tol.
 */
ibim_status ibim_solve(ibim_ctx* ctx, const ibim_phys* phys, const ibim_solve_opts* opts,
                       double* d_p, ibim_solve_info* info);

/* ibim_solve with host buffers: charges (Nc x 3, Nc) are uploaded first, the
 * solution is copied back into h_p (2N doubles) when h_p is not NULL. */
ibim_status ibim_solve_host(ibim_ctx* ctx, const ibim_phys* phys, const ibim_solve_opts* opts,
                            int64_t Nc, const double* z, const double* q, double* h_p,
                            ibim_solve_info* info);

/* ---------------------------------------------------- learned warm start */

/*
 * A small per-node network that predicts the initial GMRES vector (not part
 * of the paper's method, whose reference start is zero or Lambda^-1 g of
 * Sec. 3.3).  Features of node i: with S1, S2 the weighted RMS of g1, g2 and
 * L = S1/S2, (g1/S1, g2/S2, d/eps, clamp(H L,-10,10)/10, kappa L/(1+kappa L),
 * ln(eps_E/eps_I)/5, (eps_I/eps_E)/(1+kappa L), r1/S1, r2/S2), H from
 * ibim_get_curvature, r = g - A Lambda^-1 g the residual of the Lambda^-1 g
 * start (one application of the FP32 operator, so features and prediction
 * cost one operator application each).  Network 9 -> 64 -> 64 -> 2 (tanh),
 * BF16 weights with
 * FP32 arithmetic; output psi = S1 o0 / lambda1, psin = S2 o1 / lambda2
 * (Lambda = diag(lambda1, lambda2) of Sec. 3.3).  Trained on solutions the
 * method computed (ibim_wsnet_add_example) by Adam on sampled nodes with loss
 * sum (w_i/mean w) |o - t|^2 / batch, t = (lambda1 psi/S1, lambda2 psin/S2),
 * which weights each block by its share of the initial residual.
 * Parameters (IBIM_WS_NPARAMS floats, FP32 master copy): W1[64][9], b1[64],
 * W2[64][64], b2[64], W3[2][64], b3[2].  Use: ibim_wsnet_predict into a
 * device vector, then ibim_solve with start = 3.
 */
#define IBIM_WS_NPARAMS 4930
typedef struct ibim_wsnet ibim_wsnet;
ibim_status ibim_wsnet_create(uint64_t seed, void* stream, ibim_wsnet** out);
ibim_status ibim_wsnet_get_params(const ibim_wsnet* net, float* h_params);
ibim_status ibim_wsnet_set_params(ibim_wsnet* net, const float* h_params);  /* resets Adam */
/* features (host N x 9 floats, may be NULL) and scales (host S1, S2, mean w; may be NULL) */
ibim_status ibim_wsnet_features(ibim_wsnet* net, ibim_ctx* ctx, const ibim_phys* phys, float* h_feat,
                                double* h_scales);
/* appends every node of ctx with the solution d_p (device 2N) as training examples */
ibim_status ibim_wsnet_add_example(ibim_wsnet* net, ibim_ctx* ctx, const ibim_phys* phys, const double* d_p);
ibim_status ibim_wsnet_num_examples(const ibim_wsnet* net, int64_t* count);
/* loss and gradient (host IBIM_WS_NPARAMS floats) over examples [first, first + count) */
ibim_status ibim_wsnet_gradient(ibim_wsnet* net, int64_t first, int64_t count, double* loss, float* h_grad);
ibim_status ibim_wsnet_train(ibim_wsnet* net, int steps, int batch_nodes, double lr, double* last_loss);
ibim_status ibim_wsnet_predict(ibim_wsnet* net, ibim_ctx* ctx, const ibim_phys* phys, double* d_p0);
void ibim_wsnet_destroy(ibim_wsnet* net);

/* ---------------------------------------------------------------- tuning */

/*
 * Treecode form of the operator (far-field acceleration; the paper's own
 * accelerator is a black-box FMM built on Chebyshev interpolation, Sec. 4).
 * Every kernel of the discrete system (Sec. 2.2) is linear in the source's
 * densities d_j = a_j m_j and b_j (a_j = w_j psi_j, b_j = w_j psin_j), so a
 * cluster of sources far from a target tile is replaced by the order^3 proxies
 * (Chebyshev points of the second kind, `order` per axis) of its bounding cube,
 * carrying D_k = sum_j L_k(y_j) d_j and beta_k = sum_j L_k(y_j) b_j (L_k the
 * tensor-product Lagrange basis).  Near sources are summed as in IBIM_F32C,
 * tube rule included.
 *
 * ibim_treecode_setup builds the tree and the interaction lists of the
 * context's current nodes:
 *   - clusters are node ranges split as the coordinate bisection of built
 *     geometries splits them (left part B max(1, round(n / 2B)), B = 1024 for
 *     n >= 2048, 256 otherwise), down to 256-node tiles; target tiles have
 *     512 nodes;
 *   - a cluster is far from a target tile when r_T + r_C <= theta D and
 *     D >= max(2 tau_max, 1.5) 1.001 + 1e-3 + r_T + r_C + 0.25 (Angstrom;
 *     D the distance of the box centres, r_T the tile's box half-diagonal,
 *     r_C the proxy cube's half-diagonal), so no proxy lies in the
 *     regularisation tube (Sec. 2.2.1) of any target.
 * theta in (0, 1) (smaller: more accurate and slower; 0.5-0.8 give relative
 * operator errors of about 1e-9 to 1e-7); tau_max > 0 is the largest tau the
 * operator will be applied with.  order: Chebyshev points per axis, 4, 5 or 6
 * (64, 125 or 216 proxies per cluster; at the same theta 4 is less accurate
 * and makes far steps 3.5x cheaper than 6).  target_interp (0 or 1): with 1, a far
 * cluster that is also far from the target tile's own Chebyshev cube
 * (r_Tc + r_C <= theta D and D >= the same far distance + r_Tc + r_C + 0.25,
 * r_Tc the cube's half-diagonal) is evaluated at the tile's order^3 target proxies,
 * and the fields y1 and V (y2 = n . V) are interpolated to the targets.  Allocates device memory on the context
 * (released by ibim_destroy or a new setup); synchronises the context stream.
 * Caller nodes should be ordered so that runs of consecutive indices are
 * compact (built geometries are).  Applying IBIM_F32T with tau > tau_max or
 * tube_rule 1 returns IBIM_ERR_ARG; before any setup, IBIM_ERR_STATE.
 * Errors: IBIM_ERR_ARG (NULL context, theta or tau_max out of range, order
 * not 4, 5 or 6, target_interp not 0 or 1),
 * IBIM_ERR_STATE (no nodes), IBIM_ERR_CUDA.
 *
 * ibim_treecode_info: list sizes of the current setup (outputs may be NULL):
 * near source-tile steps, far cluster steps (each step is 512 targets x 256
 * sources or proxies), interpolated far cluster steps (order^3 target proxies x order^3
 * proxies each), clusters, target tiles.  IBIM_ERR_STATE before setup.
 */
ibim_status ibim_treecode_setup(ibim_ctx* ctx, double theta, double tau_max, int order, int target_interp);
ibim_status ibim_treecode_info(ibim_ctx* ctx, int64_t* near_steps, int64_t* far_steps, int64_t* interp_steps,
                               int64_t* clusters, int64_t* target_tiles);

/*
 * ibim_treecode_plan: the tree and interaction lists that ibim_treecode_setup
 * builds, computed on the host only (no context, no device; for inspection
 * and tests), for N nodes in the given order.
 *   xyz        host, N x 3 doubles (row-major), the nodes' positions x*.
 *   theta, tau_max, target_interp: as for ibim_treecode_setup.
 *   sizes      host, 5 int64 (required): target tiles n_t, clusters,
 *              list-kernel steps S, interpolated steps I, node tiles n_real.
 *   row_ptr    host, n_t + 1 int64 or NULL: steps of target tile t are
 *              steps[row_ptr[t] .. row_ptr[t + 1]).
 *   steps      host, S int32 or NULL: a value v < n_real is the near source
 *              tile v (nodes 256 v .. 256 v + 255); v >= n_real is far
 *              cluster v - n_real (clusters numbered in pre-order from the
 *              root, node range [0, N)).
 *   irow, isrc host, n_t + 1 int64 and I int32 or NULL: the interpolated far
 *              clusters of each tile, numbered as in steps.
 * Lists are in depth-first order (left child first).  Call once with NULL
 * arrays to read the sizes, then with arrays of those sizes.  Errors:
 * IBIM_ERR_ARG (NULL xyz or sizes, N <= 0, parameters out of range),
 * IBIM_ERR_NONFINITE.
 */
ibim_status ibim_treecode_plan(const double* xyz, int64_t N, double theta, double tau_max, int target_interp,
                               int64_t* sizes, int64_t* row_ptr, int32_t* steps, int64_t* irow, int32_t* isrc);

/*
 * FP32 pair-kernel variants (a GPU tuning device, not part of the paper's
 * method).  The library compiles a small table of variants, each with a fixed
 * number of targets per thread, a register budget (minimum CTAs per SM) and
 * a CTA size, and whether it is the symmetric kernel (each unordered node
 * pair evaluated once for both ordered pairs; its reverse sums are added with
 * FP32 shared-memory and FP64 global atomics in a varying order, so its
 * result varies from run to run at the FP32 rounding level of one tile's
 * partial sum, a few 1e-10 of max |y|).  symmetric: 0 = one-directional,
 * 1 = symmetric with the reverse sums of each source pair reduced across the
 * warp, 2 = symmetric with the reverse sums carried from lane to lane as the
 * source pairs rotate through each half-warp;
 * ibim_f32_variant_info describes entry v of [0, ibim_f32_variant_count())
 * (outputs may be NULL).
 */
int ibim_f32_variant_count(void);
ibim_status ibim_f32_variant_info(int v, int* targets_per_thread, int* min_ctas_per_sm, int* threads_per_cta,
                                  int* symmetric);

/*
 * Autotuner: times every variant on this context's geometry with CUDA events,
 * keeps the fastest for this context and caches it for contexts built later
 * in the process of the same geometry kind (analytic sphere, level-set
 * surface or caller-given nodes) with N in the same power-of-two bucket.  Returns the chosen
 * variant, its resident CTAs per SM and its time per application (outputs
 * may be NULL).  Synchronises; call it outside any stream capture.
 */
ibim_status ibim_autotune(ibim_ctx* ctx, const ibim_phys* phys, int* variant, int* ctas_per_sm, double* best_ms);

/* Manual choice of the FP32 variant and of the CTAs per SM of its persistent
 * grid (0 = the occupancy limit; larger values are clamped to it). */
ibim_status ibim_set_f32_variant(ibim_ctx* ctx, int variant, int ctas_per_sm);

/* Kernel of the float-float operator IBIM_FF on this context: 1 (default) the
 * symmetric kernel, each unordered node pair evaluated once for both
 * directions, reverse sums added in FP64 with atomics (so its last bits vary
 * from run to run, far below its 1e-10 accuracy); 0 the one-directional
 * kernel (repeatable bit for bit).  Both give the FP64 oracle's operator to
 * within 1e-10 of max |y| per element. */
ibim_status ibim_set_ff_kernel(ibim_ctx* ctx, int symmetric);

/* ------------------------------------------------- allocation-free variant */

/*
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory -- code that runs where cudaMalloc is not
 * allowed or not wanted (a host callback, a process whose device allocator is
 * owned by another runtime or frozen after start-up, a service with a fixed
 * device-memory budget).  It computes the same product as ibim_matvec with
 * IBIM_F32C, without a context, from caller-owned device arrays:
 *   d_xstar, d_normal : N x 3 row-major FP64 projections x* and unit normals,
 *   d_w               : N FP64 weights w_j = J delta_eps(d_j) h^3,
 *   d_in, d_out       : 2N FP64 vectors [psi; psin]; the byte ranges of the two
 *                       2N-vectors must not overlap (IBIM_ERR_ARG otherwise),
 *   stream            : cudaStream_t (NULL = legacy default stream).
 * The nodes keep the caller's order; as for ibim_build_from_nodes the product
 * is fastest when every aligned block of 32 consecutive nodes is compact.
 * Working memory (FP32 node copies in the frames of their aligned 32-node
 * blocks, the frames, packed sources, partial sums, an error word) comes from
 * one fixed-size static device array, about 16.9 MB, that every GPU loading
 * this library holds until the process exits.  The call allocates and frees
 * nothing.  Limits: 1 <= N <= IBIM_NOALLOC_MAX_NODES; larger N returns
 * IBIM_ERR_ARG.
 * The first call on each device looks up that device's address of the array
 * (with the device current).  Every call reads the device error word back
 * and synchronises `stream` before returning, so no call may be made inside
 * a stream capture.  All calls share the one array and it keeps the last
 * call's contents: calls that overlap on the GPU (on different streams, or
 * from different host threads) race on it and must be serialised by the
 * caller.  Returns IBIM_ERR_DEVICE_TIMEOUT when a bounded device wait gave up.
 */
#define IBIM_NOALLOC_MAX_NODES 131072
ibim_status ibim_matvec_noalloc(int64_t N, const double* d_xstar, const double* d_normal, const double* d_w,
                                const ibim_phys* phys, const double* d_in, double* d_out, void* stream);

/*
 * Extrapolated tube treatment (the higher-order use of the regularisation of
 * Sec. 2.2.1): the error the tube introduces is, to leading order, linear in
 * tau, so the system is solved with phys->tau and with tau/2 (the second solve
 * starts from the first solution) and d_p = 2 p(tau/2) - p(tau); info->gpol is
 * G_pol of that vector (G_pol is linear in p), iters/cycles/matvecs are the
 * sums over both solves and relres the larger residual.  On the Born sphere
 * (h = 0.25, full Jacobian) this turns a 2.5 % energy error into 0.06 %, and
 * the error falls as h^2.  Arguments and errors as ibim_solve.
 */
ibim_status ibim_solve_extrapolated(ibim_ctx* ctx, const ibim_phys* phys, const ibim_solve_opts* opts, double* d_p,
                                    ibim_solve_info* info);

/*
 * Batched solve of several molecules (contexts with their own geometry and
 * charges, one device): every molecule runs its own restarted GMRES (FP64
 * CGS2 Arnoldi, device Givens) and all molecules still iterating advance one
 * Arnoldi step per round; the operator applications of a round run as ONE
 * persistent FP32 pair-sum launch over a device-built list of the active
 * molecules' (target tile, source tile) steps, and a round is one CUDA graph
 * replay.  Molecules drop out of the list as they converge.  The first
 * batched solve of a size class (device, floor(log2 sum N_m^2)) in the process
 * times each compiled variant of the batched pair kernel (one-directional with
 * target tiles of 512, 256 and 128 nodes, and symmetric; the symmetric one only
 * for tol >= 1e-7, see ibim_solve) on its first round and keeps the fastest.
 *   nmol in [1, 1024]; phys: nmol entries (kappa etc. per molecule); opts must
 *   ask for IBIM_F32C and certify 0, with start 0 (zero start) or 3 (each
 *   d_p[m] holds the starting vector, e.g. an ibim_wsnet_predict result);
 *   d_p: nmol device pointers, 2 N_m doubles each (solutions out); infos:
 *   nmol entries.
 * The call synchronises the contexts' streams.  Returns IBIM_ERR_NOT_CONVERGED
 * (infos filled) when any molecule stopped at maxit above tol.
 */
ibim_status ibim_solve_batch(int nmol, ibim_ctx* const* ctxs, const ibim_phys* phys, const ibim_solve_opts* opts,
                             double* const* d_p, ibim_solve_info* infos);

/*
 * Batched pair-kernel variants (tuning, not part of the paper's method):
 * one-directional kernels with one target per thread in CTAs of 512, 256 or
 * 128 threads, and a symmetric kernel (each unordered node pair of a molecule
 * evaluated once for both directions, reverse sums carried by rotating
 * accumulators as in the single-molecule symmetric kernel).  By default the
 * first batched solve of a size class times every variant on its first round
 * and keeps the fastest; ibim_set_batch_variant(v) forces variant v for later
 * batched solves in the process (-1 restores the measured choice).
 * ibim_batch_variant_info describes variant v (outputs may be NULL) and
 * returns in last_used the variant the calling thread's last batched solve
 * ran (-1 before any).
 */
int ibim_batch_variant_count(void);
ibim_status ibim_batch_variant_info(int v, int* targets_per_thread, int* threads_per_cta, int* symmetric,
                                    int* last_used);
ibim_status ibim_set_batch_variant(int v);

/* ----------------------------------------------------------- diagnostics */

/*
 * Kernel timing: when enabled, the pair-sum kernel launches of this context
 * are bracketed by CUDA events on the context stream.  ibim_timing_get returns
 * the summed event time (ms), the number of pair-kernel launches, the pair
 * interactions they were launched for (N^2 each) and the total number of
 * kernels this context launched since the last reset.  Reading synchronises.
 * GMRES launches its Arnoldi steps in pairs between host polls: when a cycle
 * converges on the first step of a pair, the second launch finds the solver
 * done and returns at once, yet counts here as a launch of N^2 interactions.
 * ibim_solve_info's matvec counts are the applications that ran; divide the
 * event time by those for the time of one application.
 */
ibim_status ibim_timing_enable(ibim_ctx* ctx, int enable);
ibim_status ibim_timing_reset(ibim_ctx* ctx);
ibim_status ibim_timing_get(ibim_ctx* ctx, double* pair_ms, int64_t* pair_launches,
                            int64_t* pair_interactions, int64_t* total_launches);

/*
 * Test hook of the failure path (not part of the paper's method).  A kernel
 * whose bounded device wait gives up records IBIM_ERR_DEVICE_TIMEOUT in the
 * context's device error word and returns; the host reads the word at the
 * next synchronising call (ibim_matvec_host, ibim_energy, ibim_solve,
 * ibim_solve_host, ibim_solve_extrapolated, ibim_solve_batch), which then
 * returns IBIM_ERR_DEVICE_TIMEOUT and clears the word, so the context stays
 * usable.  This call sets the same bit from one device thread on the context
 * stream, after the work already queued there, so that this path can be
 * exercised without making any wait give up.
 *   status: IBIM_ERR_DEVICE_TIMEOUT (anything else is IBIM_ERR_ARG).
 * Asynchronous.
 */
ibim_status ibim_debug_raise_device_error(ibim_ctx* ctx, int status);

const char* ibim_last_error(void);
void ibim_destroy(ibim_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* IBIM_H */
