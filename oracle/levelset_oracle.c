/*
 * levelset_oracle.c -- plain FP64 CPU oracle of the paper's level-set
 * construction of the solvent excluded surface (Sec. 3.1) and of the band
 * nodes, projections, normals and weights (Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY (see ibim_oracle.c): used by the tests, the smoke
 * check and the benchmark's CPU leg, never by the product path, and sharing
 * no code with the CUDA library.
 *
 * Grid: nodes x = h (lo + (i, j, k)), i in [0, n0), ..., linear index
 * (k n1 + j) n0 + i (x fastest).  Readings of the paper used here:
 *   - F (the vdW level set, Sec. 3.1) is evaluated exactly where it is below
 *     a clamp value L and set to L elsewhere (L = 2 rho0 + eps + 6h): the
 *     inward flow for time rho0 only looks rho0 (plus the stencil reach)
 *     beyond the solvent accessible surface.
 *   - Zero Neumann boundary conditions: indices outside the box are clamped
 *     to the nearest boundary node (constant extension).
 *   - The inward eikonal flow d phi/dt = |grad phi| for t in (0, rho0] uses
 *     TVD-RK3 in time with dt = rho0 / ceil(rho0 / (h/2)), the Godunov
 *     Hamiltonian for speed -1 and fifth-order WENO one-sided derivatives.
 *   - Cavity removal (Sec. 3.1.2): the exterior is the 6-connected set of
 *     nodes with phi > 0 reached from the box boundary; cavity nodes are the
 *     other phi > 0 nodes; C_eps is every node within Euclidean distance eps
 *     of a cavity node and not in the exterior; phi := -eps on C_eps.
 *   - Reinitialization (Sec. 3.1.3) with sgn_h(phi0) = phi0/sqrt(phi0^2+h^2),
 *     dt = k0 h with k0 = 1/2 and ceil((k1 + 4)/k0) steps, eps = k1 h.
 *   - Band {|phi| < eps}; grad phi = (p_- + p_+)/2 from WENO5 per axis;
 *     normal n = grad phi / |grad phi|, projection x* = x - phi n,
 *     weight w = delta_eps(phi) h^3 (J = 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int64_t lo[3]; /* integer grid coordinate of node (0,0,0) */
    int64_t n[3];  /* nodes per axis */
    double h;
} orc_grid;

/* Box holding the solvent accessible surface plus a margin of eps + 8h. */
void orc_ls_grid(int64_t Na, const double *z, const double *r, double probe, double h, double eps,
                 orc_grid *g)
{
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = 0; k < Na; ++k)
        for (int a = 0; a < 3; ++a) {
            if (z[3 * k + a] - r[k] < mn[a]) mn[a] = z[3 * k + a] - r[k];
            if (z[3 * k + a] + r[k] > mx[a]) mx[a] = z[3 * k + a] + r[k];
        }
    const double pad = probe + eps + 8.0 * h;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = (int64_t)floor((mn[a] - pad) / h);
        const int64_t hi = (int64_t)ceil((mx[a] + pad) / h);
        g->n[a] = hi - g->lo[a] + 1;
    }
    g->h = h;
}

static inline int64_t idx(const orc_grid *g, int64_t i, int64_t j, int64_t k)
{
    return (k * g->n[1] + j) * g->n[0] + i;
}

static inline int64_t clampi(int64_t v, int64_t n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

/* F(x) = min_k (|x - z_k| - r_k), clamped at L (Sec. 3.1, vdW level set). */
void orc_ls_vdw(const orc_grid *g, int64_t Na, const double *z, const double *r, double L, double *F)
{
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < g->n[2]; ++k)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t i = 0; i < g->n[0]; ++i) {
                const double x0 = h * (double)(g->lo[0] + i), x1 = h * (double)(g->lo[1] + j),
                             x2 = h * (double)(g->lo[2] + k);
                double f = L;
                for (int64_t a = 0; a < Na; ++a) {
                    const double d0 = x0 - z[3 * a], d1 = x1 - z[3 * a + 1], d2 = x2 - z[3 * a + 2];
                    const double v = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - r[a];
                    if (v < f) f = v;
                }
                F[idx(g, i, j, k)] = f;
            }
}

/*
 * Fifth-order WENO approximation (Jiang-Peng) of a one-sided derivative from
 * the five first differences v1..v5, ordered along the upwind direction.
 */
static double weno5(double v1, double v2, double v3, double v4, double v5)
{
    const double p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
    const double p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
    const double p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
    const double s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3) +
                      0.25 * (v1 - 4.0 * v2 + 3.0 * v3) * (v1 - 4.0 * v2 + 3.0 * v3);
    const double s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4) + 0.25 * (v2 - v4) * (v2 - v4);
    const double s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) * (v3 - 2.0 * v4 + v5) +
                      0.25 * (3.0 * v3 - 4.0 * v4 + v5) * (3.0 * v3 - 4.0 * v4 + v5);
    double m = v1 * v1;
    if (v2 * v2 > m) m = v2 * v2;
    if (v3 * v3 > m) m = v3 * v3;
    if (v4 * v4 > m) m = v4 * v4;
    if (v5 * v5 > m) m = v5 * v5;
    const double e = 1e-6 * m + 1e-99;
    const double a1 = 0.1 / ((s1 + e) * (s1 + e));
    const double a2 = 0.6 / ((s2 + e) * (s2 + e));
    const double a3 = 0.3 / ((s3 + e) * (s3 + e));
    return (a1 * p1 + a2 * p2 + a3 * p3) / (a1 + a2 + a3);
}

/* p_- and p_+ (backward/forward WENO5 derivatives) along axis `ax` at node (i,j,k). */
static void weno_pm(const orc_grid *g, const double *phi, int64_t i, int64_t j, int64_t k, int ax, double *pm,
                    double *pp)
{
    double f[7];
    for (int s = -3; s <= 3; ++s) {
        int64_t ii = i, jj = j, kk = k;
        if (ax == 0) ii = clampi(i + s, g->n[0]);
        if (ax == 1) jj = clampi(j + s, g->n[1]);
        if (ax == 2) kk = clampi(k + s, g->n[2]);
        f[s + 3] = phi[idx(g, ii, jj, kk)];
    }
    const double h = g->h;
    double D[6]; /* D[m] = (f[m+1] - f[m]) / h, the difference between offsets m-3 and m-2 */
    for (int m = 0; m < 6; ++m) D[m] = (f[m + 1] - f[m]) / h;
    /* backward: differences D^-phi at offsets -2..+2 -> D[0..4] */
    *pm = weno5(D[0], D[1], D[2], D[3], D[4]);
    /* forward: differences D^+phi at offsets +2..-2 -> D[5..1] */
    *pp = weno5(D[5], D[4], D[3], D[2], D[1]);
}

/* L(phi) = |grad phi| of the inward flow d phi/dt = |grad phi| (speed -1, Godunov). */
static void eikonal_rhs(const orc_grid *g, const double *phi, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < g->n[2]; ++k)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t i = 0; i < g->n[0]; ++i) {
                double s = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    double a, b;
                    weno_pm(g, phi, i, j, k, ax, &a, &b);
                    /* speed -1: phi_x^2 ~ max(min(p_-, 0)^2, max(p_+, 0)^2) */
                    const double am = a < 0.0 ? a : 0.0;
                    const double bp = b > 0.0 ? b : 0.0;
                    s += (am * am > bp * bp) ? am * am : bp * bp;
                }
                out[idx(g, i, j, k)] = sqrt(s);
            }
}

/* L(phi) = -sgn_h(phi0) (|grad phi| - 1) of the reinitialization equation (Godunov). */
static void reinit_rhs(const orc_grid *g, const double *phi, const double *phi0, double *out)
{
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < g->n[2]; ++k)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t i = 0; i < g->n[0]; ++i) {
                const int64_t id = idx(g, i, j, k);
                const double p0 = phi0[id];
                const double sg = p0 / sqrt(p0 * p0 + h * h);
                double s = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    double a, b;
                    weno_pm(g, phi, i, j, k, ax, &a, &b);
                    if (p0 > 0.0) {
                        const double u = a > 0.0 ? a : 0.0, v = b < 0.0 ? b : 0.0;
                        s += (u * u > v * v) ? u * u : v * v;
                    } else {
                        const double u = a < 0.0 ? a : 0.0, v = b > 0.0 ? b : 0.0;
                        s += (u * u > v * v) ? u * u : v * v;
                    }
                }
                out[id] = -sg * (sqrt(s) - 1.0);
            }
}

/* One TVD-RK3 step phi <- phi + dt L(phi) (Shu-Osher form). */
static void rk3_step(const orc_grid *g, double *phi, const double *phi0, double dt, int reinit, double *t1,
                     double *t2, double *L)
{
    const int64_t M = g->n[0] * g->n[1] * g->n[2];
    if (reinit) reinit_rhs(g, phi, phi0, L); else eikonal_rhs(g, phi, L);
    for (int64_t q = 0; q < M; ++q) t1[q] = phi[q] + dt * L[q];
    if (reinit) reinit_rhs(g, t1, phi0, L); else eikonal_rhs(g, t1, L);
    for (int64_t q = 0; q < M; ++q) t2[q] = 0.75 * phi[q] + 0.25 * (t1[q] + dt * L[q]);
    if (reinit) reinit_rhs(g, t2, phi0, L); else eikonal_rhs(g, t2, L);
    for (int64_t q = 0; q < M; ++q) phi[q] = phi[q] / 3.0 + 2.0 / 3.0 * (t2[q] + dt * L[q]);
}

/* Inward eikonal flow for t in (0, probe] (Sec. 3.1.1).  Returns the step count. */
int orc_ls_eikonal(const orc_grid *g, double *phi, double probe)
{
    const int64_t M = g->n[0] * g->n[1] * g->n[2];
    const int steps = (int)ceil(probe / (0.5 * g->h));
    const double dt = probe / steps;
    double *t1 = malloc(sizeof(double) * M), *t2 = malloc(sizeof(double) * M), *L = malloc(sizeof(double) * M);
    for (int s = 0; s < steps; ++s) rk3_step(g, phi, NULL, dt, 0, t1, t2, L);
    free(t1); free(t2); free(L);
    return steps;
}

/* Reinitialization (Sec. 3.1.3) for ceil((k1+4)/k0) steps of dt = k0 h. */
int orc_ls_reinit(const orc_grid *g, double *phi, double eps)
{
    const int64_t M = g->n[0] * g->n[1] * g->n[2];
    const double k0 = 0.5, k1 = eps / g->h;
    const int steps = (int)ceil((k1 + 4.0) / k0 - 1e-9);
    const double dt = k0 * g->h;
    double *phi0 = malloc(sizeof(double) * M);
    memcpy(phi0, phi, sizeof(double) * M);
    double *t1 = malloc(sizeof(double) * M), *t2 = malloc(sizeof(double) * M), *L = malloc(sizeof(double) * M);
    for (int s = 0; s < steps; ++s) rk3_step(g, phi, phi0, dt, 1, t1, t2, L);
    free(t1); free(t2); free(L); free(phi0);
    return steps;
}

/* Cavity removal (Sec. 3.1.2).  Returns the number of nodes set to -eps;
 * `label` (optional, M bytes) receives 1 = exterior, 2 = cavity, 3 = C_eps. */
int64_t orc_ls_cavity(const orc_grid *g, double *phi, double eps, uint8_t *label)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2], M = n0 * n1 * n2;
    uint8_t *lab = label ? label : malloc(M);
    memset(lab, 0, M);
    int64_t *queue = malloc(sizeof(int64_t) * M);
    int64_t head = 0, tail = 0;
    for (int64_t k = 0; k < n2; ++k)
        for (int64_t j = 0; j < n1; ++j)
            for (int64_t i = 0; i < n0; ++i) {
                const int on_boundary = i == 0 || j == 0 || k == 0 || i == n0 - 1 || j == n1 - 1 || k == n2 - 1;
                const int64_t id = idx(g, i, j, k);
                if (on_boundary && phi[id] > 0.0) {
                    lab[id] = 1;
                    queue[tail++] = id;
                }
            }
    while (head < tail) { /* breadth-first search over 6-neighbours with phi > 0 */
        const int64_t id = queue[head++];
        const int64_t i = id % n0, j = (id / n0) % n1, k = id / (n0 * n1);
        const int64_t nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
        for (int q = 0; q < 6; ++q) {
            const int64_t a = nb[q][0], b = nb[q][1], c = nb[q][2];
            if (a < 0 || b < 0 || c < 0 || a >= n0 || b >= n1 || c >= n2) continue;
            const int64_t nid = idx(g, a, b, c);
            if (lab[nid] == 0 && phi[nid] > 0.0) {
                lab[nid] = 1;
                queue[tail++] = nid;
            }
        }
    }
    int64_t ncav = 0;
    for (int64_t q = 0; q < M; ++q)
        if (lab[q] == 0 && phi[q] > 0.0) {
            lab[q] = 2;
            ++ncav;
        }
    int64_t changed = 0;
    if (ncav > 0) {
        const int64_t R = (int64_t)ceil(eps / g->h);
        const double e2 = eps * eps / (g->h * g->h);
        for (int64_t k = 0; k < n2; ++k)
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i) {
                    const int64_t id = idx(g, i, j, k);
                    if (lab[id] != 2) continue;
                    for (int64_t c = -R; c <= R; ++c)
                        for (int64_t b = -R; b <= R; ++b)
                            for (int64_t a = -R; a <= R; ++a) {
                                if ((double)(a * a + b * b + c * c) > e2) continue;
                                const int64_t ii = i + a, jj = j + b, kk = k + c;
                                if (ii < 0 || jj < 0 || kk < 0 || ii >= n0 || jj >= n1 || kk >= n2) continue;
                                const int64_t nid = idx(g, ii, jj, kk);
                                if (lab[nid] == 0) lab[nid] = 3;
                            }
                }
        for (int64_t q = 0; q < M; ++q)
            if (lab[q] == 2 || lab[q] == 3) {
                phi[q] = -eps;
                ++changed;
            }
    }
    free(queue);
    if (!label) free(lab);
    return changed;
}

/* Band nodes {|phi| < eps} (Sec. 3.2) in grid order with WENO5 central
 * gradients, unit normals, projections and cosine weights, the Laplacian of
 * phi (curv) and, when sig2 is not NULL, the sum of the 2x2 principal minors
 * of its Hessian (second central differences, mixed terms by the four-point
 * stencil), the inputs of the full Jacobian J = 1 - phi lap + phi^2 sig2
 * (Sec. 2.2).  Returns the count; arrays are written when cap >= count. */
int64_t orc_ls_band(const orc_grid *g, const double *phi, double eps, int64_t cap, double *xs, double *nrm,
                    double *w, double *dist, int32_t *ijk, double *curv, double *sig2)
{
    const double h = g->h;
    int64_t n = 0;
    for (int64_t k = 0; k < g->n[2]; ++k)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t i = 0; i < g->n[0]; ++i) {
                const double p = phi[idx(g, i, j, k)];
                if (!(fabs(p) < eps)) continue;
                if (n < cap) {
                    double gr[3];
                    for (int ax = 0; ax < 3; ++ax) {
                        double a, b;
                        weno_pm(g, phi, i, j, k, ax, &a, &b);
                        gr[ax] = 0.5 * (a + b);
                    }
                    const double len = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                    const int64_t gi = g->lo[0] + i, gj = g->lo[1] + j, gk = g->lo[2] + k;
                    const double x[3] = {h * (double)gi, h * (double)gj, h * (double)gk};
                    for (int a = 0; a < 3; ++a) {
                        const double nv = (len > 0.0) ? gr[a] / len : 0.0;
                        nrm[3 * n + a] = nv;
                        xs[3 * n + a] = x[a] - p * nv;
                    }
                    w[n] = (1.0 + cos(M_PI * p / eps)) / (2.0 * eps) * h * h * h;
                    dist[n] = p;
                    /* twice the mean curvature: Laplacian of phi by central differences */
                    double lap = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        int64_t lo_[3] = {i, j, k}, hi_[3] = {i, j, k};
                        lo_[ax] = clampi(lo_[ax] - 1, g->n[ax]);
                        hi_[ax] = clampi(hi_[ax] + 1, g->n[ax]);
                        lap += (phi[idx(g, hi_[0], hi_[1], hi_[2])] - 2.0 * p + phi[idx(g, lo_[0], lo_[1], lo_[2])]) /
                               (h * h);
                    }
                    curv[n] = lap;
                    if (sig2) {
                        /* Hessian H_ab by central differences (indices clamped at the box) */
                        double H[3][3];
                        int64_t c0[3] = {i, j, k};
                        for (int a = 0; a < 3; ++a) {
                            int64_t m[3] = {i, j, k}, q[3] = {i, j, k};
                            m[a] = clampi(m[a] - 1, g->n[a]);
                            q[a] = clampi(q[a] + 1, g->n[a]);
                            H[a][a] = (phi[idx(g, q[0], q[1], q[2])] - 2.0 * p + phi[idx(g, m[0], m[1], m[2])]) / (h * h);
                        }
                        for (int a = 0; a < 3; ++a)
                            for (int b = a + 1; b < 3; ++b) {
                                double v[4];
                                const int sa[4] = {1, 1, -1, -1}, sb[4] = {1, -1, 1, -1};
                                for (int t = 0; t < 4; ++t) {
                                    int64_t e[3] = {c0[0], c0[1], c0[2]};
                                    e[a] = clampi(e[a] + sa[t], g->n[a]);
                                    e[b] = clampi(e[b] + sb[t], g->n[b]);
                                    v[t] = phi[idx(g, e[0], e[1], e[2])];
                                }
                                H[a][b] = H[b][a] = (v[0] - v[1] - v[2] + v[3]) / (4.0 * h * h);
                            }
                        sig2[n] = H[0][0] * H[1][1] - H[0][1] * H[0][1] + H[0][0] * H[2][2] - H[0][2] * H[0][2] +
                                  H[1][1] * H[2][2] - H[1][2] * H[1][2];
                    }
                    ijk[3 * n] = (int32_t)gi;
                    ijk[3 * n + 1] = (int32_t)gj;
                    ijk[3 * n + 2] = (int32_t)gk;
                }
                ++n;
            }
    return n;
}

/*
 * Whole Stage 1 of the paper on the grid: F, phi_SAS = F - rho0, inward
 * eikonal flow, cavity removal, reinitialization.  phi must hold
 * n0 n1 n2 doubles.  Returns the number of nodes changed by cavity removal.
 */
int64_t orc_ls_ses(const orc_grid *g, int64_t Na, const double *z, const double *r, double probe, double eps,
                   double *phi)
{
    const int64_t M = g->n[0] * g->n[1] * g->n[2];
    const double L = 2.0 * probe + eps + 6.0 * g->h;
    orc_ls_vdw(g, Na, z, r, L, phi);
    for (int64_t q = 0; q < M; ++q) phi[q] -= probe; /* phi_SAS = F - rho0 */
    orc_ls_eikonal(g, phi, probe);
    const int64_t changed = orc_ls_cavity(g, phi, eps, NULL);
    orc_ls_reinit(g, phi, eps);
    return changed;
}
