/*
 * ibim_oracle.c -- plain, slow, FP64 CPU oracle for the implicit boundary
 * integral method (IBIM) for the linearized Poisson-Boltzmann equation
 * (Zhong, Ren, Tsai, arXiv 1709.08070).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library; it is written directly from the paper's
 * definitions, in the paper's notation, with no blocking, fusion or
 * reordering beyond what the definitions state.  OpenMP parallelises the
 * independent target rows and nothing else.
 *
 * Readings of the paper used here (identical in the CUDA library, which
 * implements them independently):
 *   - Diagonal of the discrete system is lambda1 = (1+eps_E/eps_I)/2 and
 *     lambda2 = (1+eps_I/eps_E)/2 (the continuous equations of Sec. 2.1 and
 *     the matrix Lambda of Sec. 3.3); the extra 1/2 printed in front of
 *     lambda in the discrete system of Sec. 2.2 halves twice and is dropped.
 *   - K22 differentiates along n(x*) (its defining combination in Sec. 2.2
 *     and the continuous equation of Sec. 2.1).
 *   - Tube rule: a pair is regularised iff its tangent-plane distance
 *     ||x*-y*||_P < tau AND |x*-y*| < 2 tau (tube_rule 0); tube_rule 1 is the
 *     literal tangent-plane test alone (Sec. 2.2.1).
 *   - Tube values (Sec. 2.2.1): K11 = K21 = K22 = 0 and
 *     K12 = (exp(-kappa tau) - 1 + kappa tau) / (2 pi kappa tau^2), whose
 *     kappa -> 0 limit is 0.  The self pair i = j lies in the tube.
 *   - delta_eps is 0 for |eta| >= eps (the printed "|eta| >= 0" is a typo);
 *     J = 1 (Sec. 3.2, as in every run of the paper).
 *   - psi_n is the interior-side normal derivative (Sec. 2.1, first system).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double eps_in;   /* epsilon_I, interior dielectric constant            */
    double eps_out;  /* epsilon_E, exterior dielectric constant            */
    double kappa;    /* screening constant kappa (1/Angstrom), Sec. 2.1     */
    double tau;      /* regularisation radius tau (Angstrom), Sec. 2.2.1   */
    int tube_rule;   /* 0: tangent distance < tau and |r| < 2 tau; 1: literal */
} orc_phys;

/* Cosine weight delta_eps(eta), Sec. 3.2 (cosine-kernel equation). */
double orc_delta_eps(double eta, double eps)
{
    if (fabs(eta) >= eps) return 0.0;
    return (1.0 + cos(M_PI * eta / eps)) / (2.0 * eps);
}

/* Fundamental solutions of Sec. 2.1: G0 = 1/(4 pi rho), Gk = exp(-k rho)/(4 pi rho). */
double orc_G0(double rho) { return 1.0 / (4.0 * M_PI * rho); }
double orc_Gk(double rho, double kappa) { return exp(-kappa * rho) / (4.0 * M_PI * rho); }

/*
 * The four regularised kernels K11, K12, K21, K22 of the discrete system
 * (Sec. 2.2, the kernel list after the weights; regularisation Sec. 2.2.1)
 * for one target (x*, n(x*)) and one source (y*, n(y*)).
 *
 * With r = x* - y*, rho = |r|, s_x = r.n(x*), s_y = r.n(y*), c = n(x*).n(y*),
 * E = exp(-kappa rho), A = E (1 + kappa rho), B = E (3 + 3 kappa rho + kappa^2 rho^2):
 *   dG0/dn(y)        =  s_y / (4 pi rho^3)
 *   dGk/dn(y)        =  A s_y / (4 pi rho^3)
 *   dG0/dn(x)        = -s_x / (4 pi rho^3)
 *   dGk/dn(x)        = -A s_x / (4 pi rho^3)
 *   d2G0/dn(x)dn(y)  =  c / (4 pi rho^3) - 3 s_x s_y / (4 pi rho^5)
 *   d2Gk/dn(x)dn(y)  =  A c / (4 pi rho^3) - B s_x s_y / (4 pi rho^5)
 * and the kernels are the combinations the paper lists:
 *   K11 = dG0/dn(y) - (eps_E/eps_I) dGk/dn(y)
 *   K12 = G0 - Gk
 *   K21 = d2G0/dn(x)dn(y) - d2Gk/dn(x)dn(y)
 *   K22 = dG0/dn(x) - (eps_I/eps_E) dGk/dn(x)
 * Returns 1 when the pair is inside the regularisation tube.
 */
int orc_pair_kernels(const double *x, const double *nx, const double *y, const double *ny,
                     const orc_phys *P, double K[4])
{
    const double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
    const double rho2 = r0 * r0 + r1 * r1 + r2 * r2;
    const double s_x = r0 * nx[0] + r1 * nx[1] + r2 * nx[2];
    const double s_y = r0 * ny[0] + r1 * ny[1] + r2 * ny[2];
    const double c = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    const double tau = P->tau, kappa = P->kappa;
    /* ||x* - y*||_P: distance of the projections on the tangent plane at x*. */
    const double rhoP2 = rho2 - s_x * s_x;
    int tube = rhoP2 < tau * tau;
    if (P->tube_rule == 0) tube = tube && (rho2 < 4.0 * tau * tau);
    if (tube) {
        K[0] = 0.0;
        K[1] = (kappa > 0.0) ? (exp(-kappa * tau) - 1.0 + kappa * tau) / (2.0 * M_PI * kappa * tau * tau)
                             : 0.0;
        K[2] = 0.0;
        K[3] = 0.0;
        return 1;
    }
    const double rho = sqrt(rho2);
    const double E = exp(-kappa * rho);
    const double A = E * (1.0 + kappa * rho);
    const double B = E * (3.0 + 3.0 * kappa * rho + kappa * kappa * rho * rho);
    const double fp = 4.0 * M_PI;
    const double rho3 = rho2 * rho;
    const double rho5 = rho3 * rho2;
    const double th1 = P->eps_out / P->eps_in;
    const double th2 = P->eps_in / P->eps_out;

    const double dG0_dny = s_y / (fp * rho3);
    const double dGk_dny = A * s_y / (fp * rho3);
    const double dG0_dnx = -s_x / (fp * rho3);
    const double dGk_dnx = -A * s_x / (fp * rho3);
    const double d2G0 = c / (fp * rho3) - 3.0 * s_x * s_y / (fp * rho5);
    const double d2Gk = A * c / (fp * rho3) - B * s_x * s_y / (fp * rho5);

    K[0] = dG0_dny - th1 * dGk_dny;
    K[1] = orc_G0(rho) - orc_Gk(rho, kappa);
    K[2] = d2G0 - d2Gk;
    K[3] = dG0_dnx - th2 * dGk_dnx;
    return 0;
}

/*
 * One row i of the discrete system Lambda p + K W p (Sec. 2.2, discrete
 * system; Sec. 3.3, final linear system), p = (psi_bar, psin_bar):
 *   y1_i = lambda1 psi_i  + sum_j [K11 w_j psi_j - K12 w_j psin_j]
 *   y2_i = lambda2 psin_i + sum_j [K21 w_j psi_j - K22 w_j psin_j]
 * with w_j = omega_j h^3 (omega_j = J delta_eps(d_j), weights equation).
 */
static void orc_row(int64_t N, const double *xs, const double *nrm, const double *w,
                    const orc_phys *P, const double *p, int64_t i, double *y1, double *y2)
{
    const double lambda1 = 0.5 * (1.0 + P->eps_out / P->eps_in);
    const double lambda2 = 0.5 * (1.0 + P->eps_in / P->eps_out);
    const double *psi = p, *psin = p + N;
    double s1 = 0.0, s2 = 0.0, K[4];
    for (int64_t j = 0; j < N; ++j) {
        orc_pair_kernels(xs + 3 * i, nrm + 3 * i, xs + 3 * j, nrm + 3 * j, P, K);
        s1 += K[0] * w[j] * psi[j] - K[1] * w[j] * psin[j];
        s2 += K[2] * w[j] * psi[j] - K[3] * w[j] * psin[j];
    }
    *y1 = lambda1 * psi[i] + s1;
    *y2 = lambda2 * psin[i] + s2;
}

/* y = (Lambda + K W) p over all 2N rows (y laid out as [y1; y2]). */
void orc_matvec(int64_t N, const double *xs, const double *nrm, const double *w,
                const orc_phys *P, const double *p, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) orc_row(N, xs, nrm, w, P, p, i, y + i, y + N + i);
}

/* Selected rows of the same product: out[2k], out[2k+1] = (y1, y2) of row rows[k]. */
void orc_matvec_rows(int64_t N, const double *xs, const double *nrm, const double *w,
                     const orc_phys *P, const double *p, int64_t nrows, const int64_t *rows,
                     double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nrows; ++k)
        orc_row(N, xs, nrm, w, P, p, rows[k], out + 2 * k, out + 2 * k + 1);
}

/*
 * Dense 2N x 2N matrix of the same system (row-major), for brute-force
 * solves on tiny inputs: column j is Lambda e_j + K W e_j.
 */
void orc_dense(int64_t N, const double *xs, const double *nrm, const double *w,
               const orc_phys *P, double *A)
{
    const double lambda1 = 0.5 * (1.0 + P->eps_out / P->eps_in);
    const double lambda2 = 0.5 * (1.0 + P->eps_in / P->eps_out);
    const int64_t M = 2 * N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double K[4];
        for (int64_t j = 0; j < N; ++j) {
            orc_pair_kernels(xs + 3 * i, nrm + 3 * i, xs + 3 * j, nrm + 3 * j, P, K);
            A[i * M + j] = K[0] * w[j];
            A[i * M + N + j] = -K[1] * w[j];
            A[(N + i) * M + j] = K[2] * w[j];
            A[(N + i) * M + N + j] = -K[3] * w[j];
        }
        A[i * M + i] += lambda1;
        A[(N + i) * M + N + i] += lambda2;
    }
}

/*
 * Right-hand side (Sec. 2.2, definitions of g1 and g2):
 *   g1_i = sum_k (q_k/eps_I) G0(x_i*, z_k)
 *   g2_i = sum_k (q_k/eps_I) dG0(x_i*, z_k)/dn(x_i*),
 * with dG0(x, z)/dn(x) = -(x - z).n(x) / (4 pi |x - z|^3).
 */
void orc_rhs(int64_t N, const double *xs, const double *nrm, int64_t Nc, const double *z,
             const double *q, double eps_in, double *g)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double g1 = 0.0, g2 = 0.0;
        for (int64_t k = 0; k < Nc; ++k) {
            const double r0 = xs[3 * i] - z[3 * k], r1 = xs[3 * i + 1] - z[3 * k + 1],
                         r2 = xs[3 * i + 2] - z[3 * k + 2];
            const double rho = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            const double sn = r0 * nrm[3 * i] + r1 * nrm[3 * i + 1] + r2 * nrm[3 * i + 2];
            g1 += q[k] / eps_in * orc_G0(rho);
            g2 += q[k] / eps_in * (-sn / (4.0 * M_PI * rho * rho * rho));
        }
        g[i] = g1;
        g[N + i] = g2;
    }
}

/*
 * Reaction potential at the charge centres (Sec. 3.5): the IBIM sum of
 *   f(z, y) = ((eps_E/eps_I) dGk(z, y*)/dn(y) - dG0(z, y*)/dn(y)) psi(y)
 *             + (G0(z, y*) - Gk(z, y*)) psin(y)
 * over the band nodes with weights w_j.  Here r = z - y*, s_y = r.n(y*),
 * dG0/dn(y) = s_y/(4 pi rho^3), dGk/dn(y) = A s_y/(4 pi rho^3).
 */
void orc_psi_rxn(int64_t N, const double *xs, const double *nrm, const double *w, int64_t Nc,
                 const double *z, const orc_phys *P, const double *p, double *psi_rxn)
{
    const double th1 = P->eps_out / P->eps_in, kappa = P->kappa;
    const double *psi = p, *psin = p + N;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < Nc; ++k) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            const double r0 = z[3 * k] - xs[3 * j], r1 = z[3 * k + 1] - xs[3 * j + 1],
                         r2 = z[3 * k + 2] - xs[3 * j + 2];
            const double rho = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            const double s_y = r0 * nrm[3 * j] + r1 * nrm[3 * j + 1] + r2 * nrm[3 * j + 2];
            const double E = exp(-kappa * rho);
            const double A = E * (1.0 + kappa * rho);
            const double dG0 = s_y / (4.0 * M_PI * rho * rho * rho);
            const double dGk = A * s_y / (4.0 * M_PI * rho * rho * rho);
            const double f = (th1 * dGk - dG0) * psi[j] + (orc_G0(rho) - orc_Gk(rho, kappa)) * psin[j];
            s += f * w[j];
        }
        psi_rxn[k] = s;
    }
}

/* Polarization energy G_pol = 1/2 sum_k q_k psi_rxn(z_k) (Sec. 3.5), in e^2/Angstrom. */
double orc_gpol(int64_t Nc, const double *q, const double *psi_rxn)
{
    double s = 0.0;
    for (int64_t k = 0; k < Nc; ++k) s += q[k] * psi_rxn[k];
    return 0.5 * s;
}

/* Surface area: the IBIM sum with f = 1 (Sec. 3.4). */
double orc_area(int64_t N, const double *w)
{
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) s += w[j];
    return s;
}

/*
 * Band nodes of a sphere of radius R centred at c, with the analytic signed
 * distance d(x) = |x - c| - R (negative inside, Sec. 2.2).  Grid U_h =
 * origin + h Z^3; nodes with |d| < eps are kept (Sec. 3.2), in lexicographic
 * order (x fastest).  Per node: projection x* = x - d grad d = c + R (x-c)/|x-c|
 * (Sec. 2.2, closest-point projection), unit normal grad d = (x-c)/|x-c|,
 * weight w = J delta_eps(d) h^3 with J = 1 (weights equation, Sec. 3.2), the
 * signed distance and the integer grid coordinates; when lap and sig2 are not
 * NULL also the Laplacian of d at the grid node, 2/|x-c|, and the sum of the
 * 2x2 principal minors of its Hessian, 1/|x-c|^2 (the inputs of the full
 * Jacobian J = 1 - d lap + d^2 sig2, Sec. 2.2).  Returns the node count;
 * arrays are written only when cap >= count.
 */
int64_t orc_sphere_nodes(double R, const double *c, const double *origin, double h, double eps,
                         int64_t cap, double *xs, double *nrm, double *w, double *dist, int32_t *ijk,
                         double *lap, double *sig2)
{
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int64_t)floor((c[a] - R - eps - origin[a]) / h) - 1;
        hi[a] = (int64_t)ceil((c[a] + R + eps - origin[a]) / h) + 1;
    }
    int64_t n = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1 && cap < n) return n;
        n = 0;
        for (int64_t k = lo[2]; k <= hi[2]; ++k)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                    const double x0 = origin[0] + h * (double)i, x1 = origin[1] + h * (double)j,
                                 x2 = origin[2] + h * (double)k;
                    const double v0 = x0 - c[0], v1 = x1 - c[1], v2 = x2 - c[2];
                    const double len = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
                    const double d = len - R;
                    if (!(fabs(d) < eps) || len == 0.0) continue;
                    if (pass == 1) {
                        const double n0 = v0 / len, n1 = v1 / len, n2 = v2 / len;
                        xs[3 * n] = x0 - d * n0;
                        xs[3 * n + 1] = x1 - d * n1;
                        xs[3 * n + 2] = x2 - d * n2;
                        nrm[3 * n] = n0;
                        nrm[3 * n + 1] = n1;
                        nrm[3 * n + 2] = n2;
                        w[n] = orc_delta_eps(d, eps) * h * h * h;
                        dist[n] = d;
                        ijk[3 * n] = (int32_t)i;
                        ijk[3 * n + 1] = (int32_t)j;
                        ijk[3 * n + 2] = (int32_t)k;
                        if (lap) lap[n] = 2.0 / len;
                        if (sig2) sig2[n] = 1.0 / (len * len);
                    }
                    ++n;
                }
    }
    return n;
}

/*
 * Restarted GMRES(m) for (Lambda + K W) p = g (Sec. 3.3: "standard GMRES"),
 * modified Gram-Schmidt Arnoldi and Givens rotations, all in FP64.  The
 * stopping test is the relative residual ||g - A p||_2 / ||g||_2 < tol over
 * the whole 2N vector (reading: the paper does not state the norm).  x holds
 * the start on entry and the solution on exit.  *iters counts Arnoldi steps
 * (one operator application each), the paper's GMRES iteration count; the
 * residual evaluations at restarts are not counted.  Returns 0 on
 * convergence, 1 when maxit Arnoldi steps were spent first.
 */
int orc_gmres(int64_t N, const double *xs, const double *nrm, const double *w, const orc_phys *P,
              const double *g, double *x, double tol, int restart, int maxit, int *iters,
              double *relres_true)
{
    const int64_t M = 2 * N;
    const int m = restart;
    double *V = (double *)malloc(sizeof(double) * (size_t)M * (size_t)(m + 1));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *e = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *yv = (double *)malloc(sizeof(double) * (size_t)m);
    double *t = (double *)malloc(sizeof(double) * (size_t)M);
    double gnorm = 0.0;
    for (int64_t i = 0; i < M; ++i) gnorm += g[i] * g[i];
    gnorm = sqrt(gnorm);
    int total = 0, converged = 0;
    if (gnorm == 0.0) {
        for (int64_t i = 0; i < M; ++i) x[i] = 0.0;
        converged = 1;
    }
    while (!converged && total < maxit) {
        /* r0 = g - A x (not counted as an iteration) */
        orc_matvec(N, xs, nrm, w, P, x, t);
        double beta = 0.0;
        for (int64_t i = 0; i < M; ++i) {
            V[i] = g[i] - t[i];
            beta += V[i] * V[i];
        }
        beta = sqrt(beta);
        if (beta / gnorm < tol) {
            converged = 1;
            break;
        }
        for (int64_t i = 0; i < M; ++i) V[i] /= beta;
        memset(e, 0, sizeof(double) * (size_t)(m + 1));
        e[0] = beta;
        int k = 0;
        for (; k < m && total < maxit; ++k) {
            double *vk1 = V + (size_t)(k + 1) * (size_t)M;
            orc_matvec(N, xs, nrm, w, P, V + (size_t)k * (size_t)M, vk1);
            ++total;
            for (int jj = 0; jj <= k; ++jj) { /* modified Gram-Schmidt */
                const double *vj = V + (size_t)jj * (size_t)M;
                double hij = 0.0;
                for (int64_t i = 0; i < M; ++i) hij += vj[i] * vk1[i];
                for (int64_t i = 0; i < M; ++i) vk1[i] -= hij * vj[i];
                H[jj * m + k] = hij;
            }
            double hn = 0.0;
            for (int64_t i = 0; i < M; ++i) hn += vk1[i] * vk1[i];
            hn = sqrt(hn);
            H[(k + 1) * m + k] = hn;
            if (hn > 0.0)
                for (int64_t i = 0; i < M; ++i) vk1[i] /= hn;
            for (int jj = 0; jj < k; ++jj) { /* apply earlier rotations */
                const double a = H[jj * m + k], b = H[(jj + 1) * m + k];
                H[jj * m + k] = cs[jj] * a + sn[jj] * b;
                H[(jj + 1) * m + k] = -sn[jj] * a + cs[jj] * b;
            }
            const double a = H[k * m + k], b = H[(k + 1) * m + k];
            const double rr = sqrt(a * a + b * b);
            cs[k] = (rr == 0.0) ? 1.0 : a / rr;
            sn[k] = (rr == 0.0) ? 0.0 : b / rr;
            H[k * m + k] = rr;
            H[(k + 1) * m + k] = 0.0;
            e[k + 1] = -sn[k] * e[k];
            e[k] = cs[k] * e[k];
            if (fabs(e[k + 1]) / gnorm < tol) {
                ++k;
                break;
            }
        }
        /* back substitution H y = e, then x += V y */
        for (int ii = k - 1; ii >= 0; --ii) {
            double s = e[ii];
            for (int jj = ii + 1; jj < k; ++jj) s -= H[ii * m + jj] * yv[jj];
            yv[ii] = s / H[ii * m + ii];
        }
        for (int jj = 0; jj < k; ++jj) {
            const double *vj = V + (size_t)jj * (size_t)M;
            for (int64_t i = 0; i < M; ++i) x[i] += yv[jj] * vj[i];
        }
    }
    /* true residual */
    orc_matvec(N, xs, nrm, w, P, x, t);
    double rn = 0.0;
    for (int64_t i = 0; i < M; ++i) rn += (g[i] - t[i]) * (g[i] - t[i]);
    *relres_true = (gnorm > 0.0) ? sqrt(rn) / gnorm : 0.0;
    if (*relres_true < tol) converged = 1;
    *iters = total;
    free(V); free(H); free(cs); free(sn); free(e); free(yv); free(t);
    return converged ? 0 : 1;
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of later oracle calls (n >= 1; no effect
 * when built without OpenMP).  Used to time the oracle on one host core. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
