/*
 * FP64 CPU oracle for pDCA on the graph Ginzburg-Landau model.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the bench).
 * Independent of the CUDA library: no shared headers, helpers or tables.
 */
#ifndef PDCA_ORACLE_H
#define PDCA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LAP_NORMALIZED = 0, ORC_LAP_UNNORMALIZED = 1 };
enum { ORC_JACOBI_DAMPED = 0, ORC_JACOBI_PERTURBED = 1, ORC_RICHARDSON = 2 };

/* One problem: the graph (CSR, symmetric, no self loops), its degrees, the
 * model parameters and the fidelity data.  All arrays are borrowed. */
typedef struct {
    int64_t n;
    int32_t K;
    int32_t laplacian;      /* ORC_LAP_* */
    int32_t precond;        /* ORC_JACOBI_* / ORC_RICHARDSON */
    int32_t pad_;
    const int64_t *row_ptr; /* n+1 */
    const int32_t *col;     /* nnz */
    const float *w;         /* nnz */
    const double *d;        /* n, degrees from orc_degrees */
    const uint8_t *mask;    /* n, Lambda_i in {0,1} */
    const double *y;        /* n*K, prior in +-1 coding (orc_prior) */
    double eps, eta, c;
    double damping;         /* omega for ORC_JACOBI_DAMPED */
    double delta0;
    double lambda_max;      /* for ORC_RICHARDSON */
    double step_k;          /* step size k of the DCA with step size; 0 = infinite */
} orc_problem;

int orc_num_threads(void);
int64_t orc_degrees(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w, double *d);
void orc_apply_Ls(int64_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                  const float *w, const double *d, const double *x, double *y);
void orc_apply_L(int64_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                 const float *w, const double *d, const double *x, double *y);
void orc_apply_T(const orc_problem *p, const double *x, double *y);
void orc_apply_system(const orc_problem *p, const double *x, double *y);
void orc_prior(int64_t n, int32_t K, const uint8_t *mask, const int32_t *labels, double *y);
void orc_init_u(int64_t n, int32_t K, const uint8_t *mask, const int32_t *labels, double *u);
void orc_precond_diag(const orc_problem *p, double *g);
void orc_rhs(const orc_problem *p, const double *u, double *b);
void orc_sweep(const orc_problem *p, const double *g, const double *b,
               const double *v, double *tv, double *v_new);
void orc_project_row(int32_t K, double *u);
double orc_energy(const orc_problem *p, const double *u, double *scratch_nk);
double orc_residual(const orc_problem *p, const double *b, const double *u, double *scratch_nk);
void orc_labels(int64_t n, int32_t K, const double *u, int32_t *lab);
double orc_power_max_eig(const orc_problem *p, int32_t iters);
int orc_pdca_solve(const orc_problem *p, int32_t outer, int32_t inner, double *u,
                   double *energy, double *residual);

#ifdef __cplusplus
}
#endif
#endif
