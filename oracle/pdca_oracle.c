/*
 * Plain FP64 CPU oracle for the preconditioned DCA (pDCA) on the graph
 * Ginzburg-Landau model.  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the CUDA library
 * never links, includes or calls anything from this directory.
 *
 * Every loop is the textbook definition, one node at a time, in the order the
 * paper states the algorithm.  No blocking, fusion or reordering.  Weights are
 * read as float32 and promoted exactly to double; all arithmetic is double.
 *
 * Notation (paper Sec. 2-3):
 *   W = (w_ij) symmetric, w_ij >= 0, no self loops; d_i = sum_j w_ij > 0;
 *   L = D - W;  L_s = I - D^{-1/2} W D^{-1/2};
 *   T = eps*L + eta*Lambda + c*I                       (eq. dca:linear:system:ori)
 *   b^t = eta*Lambda*y + c*u^t - grad W(u^t),
 *   grad W(u) = (u^3 - u)/eps                           (W(u) = (u^2-1)^2/4)
 *   u <- u + G^{-1} (b - T u)                          (eq. general:diag:pre)
 * With a finite step size k > 0 (Lemma preconditioned_DCA:stepsize) the linear
 * system of an outer step is T_k u = b_k^t with T_k = I + k T and
 * b_k^t = u^t + k b^t (eq. btk:utk), preconditioned by the G_k of eqs.
 * pre:unnorm:jacob:richard:k and pre:norm:jacob:richard:k.
 * u is an n x K row-major array; K = 1 is the paper's binary +-1 model, K >= 2
 * runs the same scalar update on every column (one +-1 coding per class) and
 * projects each row onto the simplex after every outer step.
 *
 * The OpenMP build of this same file (-fopenmp) parallelises only loops whose
 * iterations are independent rows, so both builds produce identical bits.
 */
#include "pdca_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Degree matrix D, d_ii = sum_j w_ij (Sec. 2.2, definition of L and L_s).
 * Returns the index of the first node with d_i <= 0, or -1. */
int64_t orc_degrees(int64_t n, const int64_t *row_ptr, const int32_t *col,
                    const float *w, double *d) {
    (void)col;
    int64_t bad = -1;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += (double)w[e];
        d[i] = s;
        if (!(s > 0.0) && bad < 0) bad = i;
    }
    return bad;
}

/* y = L_s x = x - D^{-1/2} W D^{-1/2} x   (Sec. 2.2), K columns. */
void orc_apply_Ls(int64_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                  const float *w, const double *d, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int64_t j = col[e];
                acc += (double)w[e] / sqrt(d[i] * d[j]) * x[j * K + k];
            }
            y[i * K + k] = x[i * K + k] - acc;
        }
    }
}

/* y = L x = D x - W x   (Sec. 2.2), K columns. */
void orc_apply_L(int64_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                 const float *w, const double *d, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                acc += (double)w[e] * x[(int64_t)col[e] * K + k];
            y[i * K + k] = d[i] * x[i * K + k] - acc;
        }
    }
}

static void apply_lap(const orc_problem *p, const double *x, double *y) {
    if (p->laplacian == ORC_LAP_NORMALIZED)
        orc_apply_Ls(p->n, p->K, p->row_ptr, p->col, p->w, p->d, x, y);
    else
        orc_apply_L(p->n, p->K, p->row_ptr, p->col, p->w, p->d, x, y);
}

/* y = T x, T = eps*L + eta*Lambda + c*I   (eq. dca:linear:system:ori). */
void orc_apply_T(const orc_problem *p, const double *x, double *y) {
    const int64_t nk = p->n * (int64_t)p->K;
    apply_lap(p, x, y);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nk; ++q) {
        int64_t i = q / p->K;
        double lam = p->mask[i] ? 1.0 : 0.0;
        y[q] = p->eps * y[q] + p->eta * lam * x[q] + p->c * x[q];
    }
}

/* y = S x for the matrix S of the linear system of one outer step:
 * S = T (infinite step size) or S = T_k = I + k T (step size k > 0). */
void orc_apply_system(const orc_problem *p, const double *x, double *y) {
    orc_apply_T(p, x, y);
    if (p->step_k > 0.0) {
        const int64_t nk = p->n * (int64_t)p->K;
        const double k = p->step_k;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < nk; ++q) y[q] = x[q] + k * y[q];
    }
}

/* Prior y in the +-1 coding.  K = 1: y_i = +1 for class 1, -1 for class 0.
 * K >= 2: y_ik = +1 if k is the node's class, -1 otherwise.  Rows with
 * Lambda_i = 0 get 0 (they never enter the equations). */
void orc_prior(int64_t n, int32_t K, const uint8_t *mask, const int32_t *labels, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = 0; k < K; ++k) {
            double v = 0.0;
            if (mask[i]) {
                if (K == 1) v = labels[i] == 1 ? 1.0 : -1.0;
                else v = labels[i] == k ? 1.0 : -1.0;
            }
            y[i * K + k] = v;
        }
    }
}

/* Initial iterate (the paper does not state one for the supervised case):
 * labelled rows start at their prior, unlabelled rows at the centre of the
 * label set (0 for K = 1; v = 1/K, u = 2v - 1 for K >= 2). */
void orc_init_u(int64_t n, int32_t K, const uint8_t *mask, const int32_t *labels, double *u) {
    orc_prior(n, K, mask, labels, u);
    for (int64_t i = 0; i < n; ++i)
        if (!mask[i])
            for (int32_t k = 0; k < K; ++k) u[i * K + k] = (K == 1) ? 0.0 : 2.0 / K - 1.0;
}

/* Diagonal preconditioner g_i for the infinite step size (Sec. 3.1):
 *   normalized L_s:   Jd: (eps + c + eta*Lambda_i)/omega
 *                     Jp: 2 eps + c + delta0 + eta*Lambda_i
 *                     R : eps*lambda_max + c + delta0 + eta*Lambda_i
 *   unnormalized L:   Jd: (eps*d_i + c + eta*Lambda_i)/omega
 *                     Jp: 2 eps d_i + c + delta0 + eta*Lambda_i
 *                     R : eps*lambda_max + c + delta0 + eta*Lambda_i
 * omega = 1/2 is the paper's G = 2 diag(T).
 * Finite step size k (Sec. 3.1, G_{.,k} and G_{.,ks}), a_i = 1 (L_s) or d_i (L):
 *                     Jd: (1 + k (eps*a_i + c + eta*Lambda_i))/omega   (= diag(T_k)/omega)
 *                     Jp: 1 + k (2 eps a_i + c + eta*Lambda_i) + delta0
 *                     R : 1 + k (eps*lambda_max + c + eta*Lambda_i) + delta0 */
void orc_precond_diag(const orc_problem *p, double *g) {
    for (int64_t i = 0; i < p->n; ++i) {
        double lam = p->mask[i] ? 1.0 : 0.0;
        double dii = (p->laplacian == ORC_LAP_NORMALIZED) ? 1.0 : p->d[i];
        double gi;
        if (p->step_k > 0.0) {
            const double k = p->step_k;
            switch (p->precond) {
            case ORC_JACOBI_DAMPED:
                gi = (1.0 + k * (p->eps * dii + p->c + p->eta * lam)) / p->damping;
                break;
            case ORC_JACOBI_PERTURBED:
                gi = 1.0 + k * (2.0 * p->eps * dii + p->c + p->eta * lam) + p->delta0;
                break;
            default: /* ORC_RICHARDSON */
                gi = 1.0 + k * (p->eps * p->lambda_max + p->c + p->eta * lam) + p->delta0;
                break;
            }
            g[i] = gi;
            continue;
        }
        switch (p->precond) {
        case ORC_JACOBI_DAMPED:
            gi = (p->eps * dii + p->c + p->eta * lam) / p->damping;
            break;
        case ORC_JACOBI_PERTURBED:
            gi = 2.0 * p->eps * dii + p->c + p->delta0 + p->eta * lam;
            break;
        default: /* ORC_RICHARDSON */
            gi = p->eps * p->lambda_max + p->c + p->delta0 + p->eta * lam;
            break;
        }
        g[i] = gi;
    }
}

/* Right-hand side of one outer step's system:
 *   b^t = eta*Lambda*y + c*u^t - (u^t^3 - u^t)/eps     (eq. bt:ut), infinite step;
 *   b_k^t = u^t + k b^t                                 (eq. btk:utk), step size k. */
void orc_rhs(const orc_problem *p, const double *u, double *b) {
    const int64_t nk = p->n * (int64_t)p->K;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nk; ++q) {
        int64_t i = q / p->K;
        double lam = p->mask[i] ? 1.0 : 0.0;
        double grad_w = (u[q] * u[q] * u[q] - u[q]) / p->eps;
        b[q] = p->eta * lam * p->y[q] + p->c * u[q] - grad_w;
        if (p->step_k > 0.0) b[q] = u[q] + p->step_k * b[q];
    }
}

/* One diagonal preconditioned sweep v_new = v + G^{-1}(b - S v)
 * (eq. dampedJacobi:richardson), S = T or T_k: every row reads the old v.
 * tv is scratch. */
void orc_sweep(const orc_problem *p, const double *g, const double *b,
               const double *v, double *tv, double *v_new) {
    const int64_t nk = p->n * (int64_t)p->K;
    orc_apply_system(p, v, tv);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nk; ++q) {
        int64_t i = q / p->K;
        v_new[q] = v[q] + (b[q] - tv[q]) / g[i];
    }
}

/* Euclidean projection of one row onto the simplex, in the coding
 * v = (u + 1)/2:  argmin ||v' - v|| s.t. v' >= 0, sum v' = 1, by the
 * sort-and-threshold method (Held, Wolfe and Crowder 1974).  Sums in double.
 * Writes back u = 2 v' - 1. */
void orc_project_row(int32_t K, double *u) {
    double v[64], mu[64];
    for (int32_t k = 0; k < K; ++k) v[k] = 0.5 * (u[k] + 1.0);
    for (int32_t k = 0; k < K; ++k) mu[k] = v[k];
    /* sort mu descending (insertion sort) */
    for (int32_t a = 1; a < K; ++a) {
        double x = mu[a];
        int32_t b = a - 1;
        while (b >= 0 && mu[b] < x) { mu[b + 1] = mu[b]; --b; }
        mu[b + 1] = x;
    }
    double run = 0.0, theta = 0.0;
    for (int32_t j = 0; j < K; ++j) {
        run += mu[j];
        double t = (run - 1.0) / (double)(j + 1);
        if (mu[j] - t > 0.0) theta = t;   /* last j with a positive gap is rho */
    }
    for (int32_t k = 0; k < K; ++k) {
        double vk = v[k] - theta;
        if (vk < 0.0) vk = 0.0;
        u[k] = 2.0 * vk - 1.0;
    }
}

/* Graph GL energy with fidelity (eqs. gl:functional:graph, functional:GL):
 *   F(u) = (eps/2) <u, L u> + (1/(4 eps)) sum_i (u_i^2 - 1)^2
 *          + (eta/2) sum_i Lambda_i (u_i - y_i)^2,
 * summed over the K columns; L is L_s for the normalized model. */
double orc_energy(const orc_problem *p, const double *u, double *scratch_nk) {
    const int64_t nk = p->n * (int64_t)p->K;
    apply_lap(p, u, scratch_nk);
    double quad = 0.0, well = 0.0, fid = 0.0;
    for (int64_t q = 0; q < nk; ++q) {
        int64_t i = q / p->K;
        quad += u[q] * scratch_nk[q];
        double s = u[q] * u[q] - 1.0;
        well += s * s;
        if (p->mask[i]) {
            double e = u[q] - p->y[q];
            fid += e * e;
        }
    }
    return 0.5 * p->eps * quad + well / (4.0 * p->eps) + 0.5 * p->eta * fid;
}

/* Relative residual ||b - S u|| / ||b|| of the DCA linear system (S = T or T_k). */
double orc_residual(const orc_problem *p, const double *b, const double *u, double *scratch_nk) {
    const int64_t nk = p->n * (int64_t)p->K;
    orc_apply_system(p, u, scratch_nk);
    double rr = 0.0, bb = 0.0;
    for (int64_t q = 0; q < nk; ++q) {
        double r = b[q] - scratch_nk[q];
        rr += r * r;
        bb += b[q] * b[q];
    }
    return bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
}

/* Labels: K = 1: sign(u_i) (u_i >= 0 -> class 1); K >= 2: argmax_k u_ik,
 * the lowest k among equal maxima. */
void orc_labels(int64_t n, int32_t K, const double *u, int32_t *lab) {
    for (int64_t i = 0; i < n; ++i) {
        if (K == 1) {
            lab[i] = u[i] >= 0.0 ? 1 : 0;
        } else {
            int32_t best = 0;
            for (int32_t k = 1; k < K; ++k)
                if (u[i * K + k] > u[i * K + best]) best = k;
            lab[i] = best;
        }
    }
}

/* Power method for the largest eigenvalue of L_s (or L) (Sec. 3.1, used by
 * the generalized Richardson preconditioner): x_0(i) = 1 + 0.5 sin(i+1),
 * x <- A x / ||A x||_2 for `iters` iterations, then the Rayleigh quotient
 * x^T A x / x^T x. */
double orc_power_max_eig(const orc_problem *p, int32_t iters) {
    const int64_t n = p->n;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    orc_problem q = *p;
    q.K = 1;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) { x[i] = 1.0 + 0.5 * sin((double)(i + 1)); nrm += x[i] * x[i]; }
    nrm = sqrt(nrm);
    for (int64_t i = 0; i < n; ++i) x[i] /= nrm;
    for (int32_t it = 0; it < iters; ++it) {
        apply_lap(&q, x, y);
        nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) nrm += y[i] * y[i];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) break;
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    apply_lap(&q, x, y);
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) { num += x[i] * y[i]; den += x[i] * x[i]; }
    free(x);
    free(y);
    return num / den;
}

/* pDCA with the infinite step size (Prop. nopre), or with step size k
 * (Lemma preconditioned_DCA:stepsize, b_k^t, T_k, G_k in place of b^t, T, G):
 * for t = 0..outer-1,
 *   b^t = eta Lambda y + c u^t - grad W(u^t);
 *   v^0 = u^t;  v^{s+1} = v^s + G^{-1}(b^t - T v^s), s < inner;
 *   K >= 2: project each row of v^inner onto the simplex;
 *   u^{t+1} = v^inner;  energy[t] = F(u^{t+1}), residual[t] = ||b^t - T u^{t+1}||/||b^t||.
 * u (n x K) is updated in place.  energy / residual may be NULL.
 * Returns 0, or -1 if a non-finite value appears. */
int orc_pdca_solve(const orc_problem *p, int32_t outer, int32_t inner, double *u,
                   double *energy, double *residual) {
    const int64_t n = p->n;
    const int64_t nk = n * (int64_t)p->K;
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    double *b = (double *)malloc(sizeof(double) * (size_t)nk);
    double *v = (double *)malloc(sizeof(double) * (size_t)nk);
    double *vn = (double *)malloc(sizeof(double) * (size_t)nk);
    double *tv = (double *)malloc(sizeof(double) * (size_t)nk);
    int rc = 0;
    orc_precond_diag(p, g);
    for (int32_t t = 0; t < outer; ++t) {
        orc_rhs(p, u, b);
        memcpy(v, u, sizeof(double) * (size_t)nk);
        for (int32_t s = 0; s < inner; ++s) {
            orc_sweep(p, g, b, v, tv, vn);
            double *sw = v; v = vn; vn = sw;
        }
        if (p->K >= 2)
            for (int64_t i = 0; i < n; ++i) orc_project_row(p->K, v + i * p->K);
        memcpy(u, v, sizeof(double) * (size_t)nk);
        if (residual) residual[t] = orc_residual(p, b, u, tv);
        if (energy) energy[t] = orc_energy(p, u, tv);
        for (int64_t q = 0; q < nk; ++q)
            if (!isfinite(u[q])) { rc = -1; break; }
        if (rc) break;
    }
    free(g); free(b); free(v); free(vn); free(tv);
    return rc;
}
