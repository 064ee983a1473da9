/*
 * pdca.h -- C interface of the GB300 (sm_103a) preconditioned DCA solver for
 * the graph Ginzburg-Landau model (Shen, Sun, Tai, "Preconditioned Algorithm
 * for Difference of Convex Functions with applications to Graph
 * Ginzburg-Landau Model").
 *
 * Problem (Sec. 2, eq. functional:GL): minimise over u (n x K, row-major)
 *   F(u) = (eps/2) <u, L u> + (1/(4 eps)) sum_i (u_i^2 - 1)^2
 *          + (eta/2) sum_i Lambda_i (u_i - y_i)^2
 * with L the graph Laplacian of a symmetric weight matrix W, normalized
 * (L_s = I - D^{-1/2} W D^{-1/2}) by default.  Each outer DCA step (eq.
 * dca:linear:system:ori, Prop. nopre) linearises the double well at u^t,
 *   b^t = eta Lambda y + c u^t - (u^t^3 - u^t)/eps,
 * and replaces the solve of T u = b^t, T = eps L + eta Lambda + c I, by a
 * few diagonal preconditioned sweeps v <- v + G^{-1}(b^t - T v)
 * (eq. general:diag:pre) with the feasible damped-Jacobi, perturbed-Jacobi
 * or generalized-Richardson preconditioner of eq. pre:norm:jacob:richard.
 *
 * K = 1 is the paper's binary model (labels +-1).  K >= 2 runs the same
 * scalar update on every column of a +-1 class coding and projects each row
 * onto the probability simplex (in v = (u+1)/2) after every outer step; the
 * paper has no multi-class form, this extension follows the same equations
 * column by column.
 *
 * Conventions for every call:
 *  - Every function returns a pdca_status; no C++ exception crosses it.
 *  - Pointers documented "host or device" may be either: the library asks
 *    the CUDA runtime which kind it is and copies accordingly.
 *  - The library allocates no device memory (one exception: the device form
 *    of the inspection call pdca_locality_order).  All device state lives
 *    in the caller's workspace (size from pdca_workspace_size), which the
 *    handle borrows until pdca_destroy; the caller frees it afterwards.
 *  - All device work of a handle runs on the stream given to pdca_create,
 *    except that pdca_create may run its renumbering on a stream of its own:
 *    ordered after the work the given stream holds when the call starts, and
 *    finished, with the stream released, before the call returns.  Calls
 *    that return host values synchronise that stream.  Errors of
 *    asynchronous kernels surface at the next synchronising call.
 *  - One handle must not be used from two host threads at once; separate
 *    handles on separate streams are independent.
 */
#ifndef PDCA_H
#define PDCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest number of label columns K supported by the kernels. */
#define PDCA_MAX_K 16

/* Largest graph, in nodes, that pdca_energy_static accepts: its fixed device
 * scratch holds one float per node (4 MiB) plus 64 KiB of partial sums. */
#define PDCA_STATIC_MAX_N (1 << 20)

typedef enum {
    PDCA_OK = 0,
    PDCA_ERR_INVALID_ARG = 1,    /* bad size, pointer, parameter or call order        */
    PDCA_ERR_NOT_SYMMETRIC = 2,  /* w_ij != w_ji or (i,j) stored without (j,i)         */
    PDCA_ERR_ISOLATED_NODE = 3,  /* d_i = sum_j w_ij is not > 0 (Sec. 2.2 needs d > 0) */
    PDCA_ERR_INFEASIBLE = 4,     /* preconditioner not feasible (G > T fails)          */
    PDCA_ERR_NONFINITE = 5,      /* NaN/Inf in the iterate                             */
    PDCA_ERR_OOM = 6,            /* workspace smaller than pdca_workspace_size         */
    PDCA_ERR_CUDA = 7,           /* a CUDA runtime call failed                         */
    PDCA_ERR_TIMEOUT = 8,        /* reserved: no call waits on the device (no spin)   */
    PDCA_ERR_BAD_GRAPH = 9,      /* column out of range, self loop, columns not
                                    strictly increasing, weight < 0 or not finite,
                                    mask not 0/1, or prior label out of range           */
    PDCA_ERR_TOO_LARGE = 10,     /* n above PDCA_STATIC_MAX_N in pdca_energy_static    */
    PDCA_ERR_NOT_CONVERGED = 11  /* pdca_spectral_init reached max_iters before tol    */
} pdca_status;

/* Laplacian (Sec. 2.2): L_s = I - D^{-1/2} W D^{-1/2} (normalized) or
 * L = D - W (unnormalized), d_i = sum_j w_ij. */
enum { PDCA_LAP_NORMALIZED = 0, PDCA_LAP_UNNORMALIZED = 1 };

/* Diagonal preconditioner G (Sec. 3.1), infinite step size, with a_i = 1 for
 * L_s (eq. pre:norm:jacob:richard) and a_i = d_i for L (eqs.
 * pre:unnorm:jacob, pre:unnorm:richard):
 *   PDCA_JACOBI_DAMPED    g_i = (eps a_i + c + eta Lambda_i) / omega
 *                         (the paper's G_Jd = 2 diag(T) is omega = 1/2);
 *   PDCA_JACOBI_PERTURBED g_i = 2 eps a_i + c + delta0 + eta Lambda_i    (G_Jp);
 *   PDCA_RICHARDSON       g_i = eps lambda_max + c + delta0 + eta Lambda_i (G_R),
 *                         lambda_max of L_s or L.
 * With a finite step size k (Lemma preconditioned_DCA:stepsize) the system of
 * an outer step is (I + kT) u = u^t + k b^t with the G_k of eqs.
 * pre:unnorm:jacob:richard:k / pre:norm:jacob:richard:k; divided by k this is
 * the system above with c + 1/k in place of c and delta0/k in place of
 * delta0, which is how the library runs it. */
enum { PDCA_JACOBI_DAMPED = 0, PDCA_JACOBI_PERTURBED = 1, PDCA_RICHARDSON = 2 };

/* Node renumbering at create time (a layout choice; results are returned in
 * the caller's node order either way):
 *   PDCA_REORDER_BFS  (default) nodes are grouped into blocks of 1024 by
 *                     breadth-first search so a block is a compact region of
 *                     the graph, then sorted by degree inside each block;
 *   PDCA_REORDER_NONE rows keep the caller's order except for the degree sort
 *                     inside windows of `sort_window` rows. */
enum { PDCA_REORDER_NONE = 0, PDCA_REORDER_BFS = 1 };

/* Sweep kernels:
 *   PDCA_TILING_AUTO (default) and PDCA_TILING_OFF: neighbour rows are read
 *                    from global memory through L1/L2 (the faster form on
 *                    every workload measured on GB300);
 *   PDCA_TILING_ON   (needs PDCA_REORDER_BFS) tiles of 512 rows first stage
 *                    the distinct neighbour rows they reference in shared
 *                    memory (up to 96 KiB; tiles with larger halos read
 *                    through their halo list) and gather from there with
 *                    16-bit local columns. */
enum { PDCA_TILING_AUTO = 0, PDCA_TILING_OFF = 1, PDCA_TILING_ON = 2 };

/* Order of the entries inside each row of the sliced-ELL operator (a layout
 * choice; the sum over a row's neighbours is the same up to FP32 rounding):
 *   PDCA_ENTRIES_SPREAD (default) the entries of each quarter of a slice
 *                       (8 rows: the rows one L1 wavefront serves when a
 *                       neighbour row of the iterate takes 16 bytes) are
 *                       ordered so that, at each position, their columns
 *                       differ modulo 8 or fall in the same group of 8 rows
 *                       (fewer bank conflicts in the gathers).  The order
 *                       depends on the graph only, not on K or the precision,
 *                       so problems sharing an operator see the same order;
 *   PDCA_ENTRIES_CSR    the order of the caller's CSR columns. */
enum { PDCA_ENTRIES_SPREAD = 0, PDCA_ENTRIES_CSR = 1 };

/* Column indices of the sliced-ELL operator (plain kernels; a layout choice
 * with no effect on the arithmetic):
 *   PDCA_COLUMNS_AUTO (default) a slice whose rows reach only nodes of their
 *                     own 65536-node chunk (new numbering) and of the two
 *                     neighbouring chunks stores 16-bit columns (the low 16
 *                     bits; the chunk of each entry follows from its band,
 *                     see below), other slices store int32 columns.  Inside
 *                     such a slice each row keeps its entries in three
 *                     bands: previous chunk, next chunk, own chunk, with at
 *                     most 63 entries in each of the first two and at most
 *                     4095 entries in all;
 *   PDCA_COLUMNS_32   int32 columns in every slice. */
enum { PDCA_COLUMNS_AUTO = 0, PDCA_COLUMNS_32 = 1 };

/* Arithmetic of the sweeps.
 *   PDCA_FP32               FP32 pre-scaled weights and iterates, FP32
 *                           accumulation; the reductions add per-row terms
 *                           in compensated (two-float) arithmetic and FP64;
 *   PDCA_MIXED_BF16W_FP16U  per outer step one FP32 pass (FP32 weights, FP32
 *                           iterate) forms the residual r = b^t - T u^t and
 *                           stores it in FP32; the inner sweeps then iterate
 *                           the correction e <- e + G^{-1}(r - T e) with BF16
 *                           weights and e stored in FP16 (FP32 arithmetic),
 *                           and u^{t+1} = u^t + e in FP32 -- the same
 *                           iteration as the FP32 sweeps, rearranged;
 *   PDCA_MIXED_BF16W_BF16U  the same with e stored in BF16.
 * The mixed forms use the plain (non-tiled) kernels. */
enum { PDCA_FP32 = 0, PDCA_MIXED_BF16W_FP16U = 1, PDCA_MIXED_BF16W_BF16U = 2 };

typedef struct {
    double eps;          /* diffuse interface parameter epsilon > 0                    */
    double c;            /* convex-split constant c > 0 (eq. dc:functional)           */
    double eta;          /* fidelity weight eta >= 0 (eq. functional:GL)              */
    int32_t laplacian;   /* PDCA_LAP_NORMALIZED (default) / PDCA_LAP_UNNORMALIZED     */
    int32_t precond;     /* PDCA_JACOBI_DAMPED / PDCA_JACOBI_PERTURBED / PDCA_RICHARDSON */
    double damping;      /* omega in (0,1) for PDCA_JACOBI_DAMPED.  Checked at create
                            with c' = c + 1/k (c' = c for the infinite step):
                            L_s: feasible for every graph iff
                            c' > eps (2 omega - 1)/(1 - omega);
                            L:   required c' > eps max_i d_i (2 omega - 1)/(1 - omega),
                            sufficient on every graph, attained on regular
                            bipartite ones                                           */
    double delta0;       /* the small constant delta_0 > 0 of G_Jp and G_R (1e-6)     */
    double lambda_max;   /* lambda_max of L_s (or L) for PDCA_RICHARDSON; 0 = estimate
                            it with the power method at create time, then use
                            min(B, 1.001 * estimate) with the bound B = 2 for L_s
                            and B = 2 max_i d_i for L (Prop. diagonal:pre)           */
    int32_t power_iters; /* power-method iterations (150 in the paper's experiments)   */
    int32_t precision;   /* PDCA_FP32 / PDCA_MIXED_BF16W_FP16U / PDCA_MIXED_BF16W_BF16U */
    int32_t sort_window; /* rows are sorted by degree inside windows of this many rows
                            (a power of two in [32, 8192]).  PDCA_REORDER_NONE: 0 = the
                            smallest window with at most 10% slice padding;
                            PDCA_REORDER_BFS: windows of min(sort_window, 1024) rows
                            inside each 1024-node block, 0 = 1024                    */
    int32_t reorder;     /* PDCA_REORDER_BFS (default) / PDCA_REORDER_NONE             */
    int32_t tiling;      /* PDCA_TILING_AUTO (default) / _OFF / _ON; _ON needs the
                            normalized Laplacian                                     */
    int32_t entry_order; /* PDCA_ENTRIES_SPREAD (default) / PDCA_ENTRIES_CSR              */
    double step_k;       /* step size k > 0 of the DCA with step size, or 0 for the
                            infinite step size (Prop. nopre, the default)            */
    int32_t columns;     /* PDCA_COLUMNS_AUTO (default) / PDCA_COLUMNS_32             */
    int32_t row_split;   /* split length T (plain kernels): a row longer than T keeps
                            its first T entries in the sliced ELL and the rest in an
                            overflow CSR that a pre-pass reduces one warp per row, so
                            a hub row does not hold up its sweep.  0 = automatic
                            (split only if some row is longer than max(256, t), at
                            t = max(64, nnz / 200000)); otherwise T rounded up to a
                            multiple of 4, at most 2044.  Rows longer than 2044 are
                            always split.  Arithmetic: the row's overflow sum is
                            added after its sliced entries                          */
    int32_t block_slices;/* slices one block of the plain sweep, energy and mixed
                            kernels takes from its queue: 8, 16 or 32 (a launch
                            shape; sums are formed the same way), 0 = automatic
                            (32 on large graphs, fewer when the graph is too
                            small to keep every SM busy for several waves)    */
} pdca_params;

typedef struct pdca_problem pdca_problem;

/* Fill *p with the defaults: eps = 1, c = 3, eta = 1, normalized Laplacian,
 * perturbed Jacobi, omega = 0.5, delta0 = 1e-6, lambda_max = 0 (estimate),
 * 150 power iterations, FP32, automatic sort window, BFS renumbering,
 * automatic tiling, infinite step size (step_k = 0). */
void pdca_default_params(pdca_params *p);

/* Device workspace, in bytes, that pdca_create needs for this graph.
 * row_ptr: n+1 CSR row offsets (host or device), row_ptr[0] = 0, non-decreasing.
 * k: label columns (1..PDCA_MAX_K).  p: parameters (NULL = defaults).
 * With PDCA_REORDER_BFS the padded operator depends on the renumbering, so
 * the size is an upper bound computed from the row lengths alone (at most
 * nnz + 32 x the sum of the largest n/1024 degrees entries, plus one int32
 * per nonzero for the halo lists).
 * Errors: PDCA_ERR_INVALID_ARG for n < 1, k out of range, a bad row_ptr or
 * a sort window that is not a power of two in [32, 8192]. */
pdca_status pdca_workspace_size(const int64_t *row_ptr, int32_t n, int32_t k,
                                const pdca_params *p, size_t *bytes);

/* Build a problem (Sec. 2.2 and 3.1): validate the graph, compute the degrees
 * d_i and the pre-scaled weights w_ij / sqrt(d_i d_j), renumber the nodes
 * (on the host: BFS blocks and, for tiling, the halo lists; this reads
 * row_ptr and col, copying them from the device if they live there), pack
 * the sliced-ELL operator, set u^0 and, for Richardson with lambda_max = 0,
 * run the power method.
 *   row_ptr  n+1 int64 CSR offsets            (host or device; read during the call)
 *   col      nnz int32 columns, strictly increasing within each row, no i == j
 *   w        nnz float32 weights, finite and >= 0, symmetric: w_ij == w_ji exactly
 *   fid_mask n uint8 Lambda_i in {0,1}
 *   labels   n int32 prior class per node, read only where fid_mask = 1:
 *            K = 1: class 0 -> y = -1, class 1 -> y = +1;  K >= 2: class in [0, K)
 *   p        parameters (NULL = defaults)
 *   workspace, ws_bytes  caller-owned device memory, 256-byte aligned
 *   stream   cudaStream_t as void* (NULL = legacy default stream)
 *   out      receives the handle (NULL on error)
 * u^0: labelled rows start at their prior y_i; unlabelled rows at 0 (K = 1)
 * or at the simplex centre 2/K - 1 (K >= 2).
 * Errors: INVALID_ARG, OOM (workspace too small), BAD_GRAPH, NOT_SYMMETRIC,
 * ISOLATED_NODE, INFEASIBLE, CUDA. */
pdca_status pdca_create(const int64_t *row_ptr, const int32_t *col, const float *w,
                        int32_t n, int32_t k, const uint8_t *fid_mask, const int32_t *labels,
                        const pdca_params *p, void *workspace, size_t ws_bytes,
                        void *stream, pdca_problem **out);

/* A new problem on the graph of `base`: it borrows base's operator (the
 * renumbering, the sliced-ELL pre-scaled weights and, for Richardson with
 * lambda_max = 0, base's power-method estimate) read-only and owns only its
 * per-problem state (row tags, iterates, reductions) in `workspace`.  K,
 * fidelity data and the model parameters may differ from base's; the
 * precision must be of base's family (FP32, or one of the mixed forms, which
 * share the BF16 weights).  Arguments as for pdca_create; the new problem
 * runs on base's stream.  `base` must outlive the new problem.  This is how a
 * server keeps one prepared operator per graph resident while requests with
 * different labels come and go (the paper solves one problem per graph). */
pdca_status pdca_workspace_size_like(const pdca_problem *base, int32_t k, const pdca_params *p, size_t *bytes);
pdca_status pdca_create_like(const pdca_problem *base, int32_t k, const uint8_t *fid_mask, const int32_t *labels,
                             const pdca_params *p, void *workspace, size_t ws_bytes, pdca_problem **out);

/* pdca_create_like without waiting for the stream, for serving loops that
 * admit requests while earlier problems run.  The fidelity arrays are copied
 * and checked on the stream: they must stay unchanged until the stream has
 * passed the copies (device memory, or page-locked host memory; pageable host
 * memory is accepted but may make the copy wait).  The check's outcome (a
 * mask value above 1 or a label out of range, BAD_GRAPH in
 * pdca_create_like) is not returned here: the bad rows start and stay
 * unlabelled, and pdca_labels returns BAD_GRAPH, pdca_labels_async writes a
 * nonzero status word.  When base holds no lambda estimate and the problem
 * uses Richardson with lambda_max = 0, the power method runs and the call
 * waits for it.  Serving infrastructure; the paper has no counterpart.
 * Errors: as pdca_create_like, less BAD_GRAPH. */
pdca_status pdca_create_like_async(const pdca_problem *base, int32_t k, const uint8_t *fid_mask,
                                   const int32_t *labels, const pdca_params *p, void *workspace, size_t ws_bytes,
                                   pdca_problem **out);

/* Replace the iterate: u (n x K row-major float32, host or device), or NULL
 * to restore u^0.  Clears the record of the last outer step. */
pdca_status pdca_set_u(pdca_problem *h, const float *u);

/* One outer pDCA step (Prop. nopre) with `inner_sweeps` >= 1 preconditioned
 * sweeps; for K >= 2 the last sweep also projects each row onto the simplex.
 * Asynchronous. */
pdca_status pdca_step(pdca_problem *h, int32_t inner_sweeps);

/* `outer_iters` >= 0 outer steps of `inner_sweeps` sweeps each.
 * damping > 0 replaces omega for PDCA_JACOBI_DAMPED (re-checked for
 * feasibility; INFEASIBLE otherwise); pass 0 to keep the current value.
 * energy_trace / residual_trace: NULL, or host or device arrays of
 * outer_iters doubles receiving F(u^{t+1}) and ||b^t - T u^{t+1}|| / ||b^t||
 * after every step (this adds one reduction pass per step and synchronises
 * at the end).  Without traces the call is asynchronous. */
pdca_status pdca_solve(pdca_problem *h, int32_t outer_iters, int32_t inner_sweeps,
                       double damping, double *energy_trace, double *residual_trace);

/* F(u) of the current iterate (FP64 accumulation) and, if rel_residual is
 * not NULL, the relative residual ||b^t - T u^{t+1}||_2 / ||b^t||_2 of the
 * last outer step (NaN if no step was taken since create / set_u).
 * Returns NONFINITE if u holds NaN/Inf.  Synchronises. */
pdca_status pdca_energy(pdca_problem *h, double *F, double *rel_residual);

/* The BFS-block renumbering of PDCA_REORDER_BFS: a permutation of the nodes
 * (structure only, none of the method's arithmetic).  order[p] = the node
 * placed at position p.  Inside chunks of 65536 consecutive nodes (edges
 * leaving a chunk are ignored) nodes are grouped into blocks of 1024 by
 * breadth-first search: a search starts at the lowest node not yet placed
 * and places nodes in FIFO visiting order until the block is full (nodes it
 * queued but did not place become free again); a search that runs dry is
 * followed by the next one in the same block.  Then nodes are sorted by
 * degree (descending, ties in place order) inside windows of sort_window
 * positions (a power of two from 32 to 1024; 0 = 1024).
 *   device = 1: the CUDA kernels pdca_create runs (row_ptr, col, order in
 *     device memory); work on `stream` (NULL: the legacy default stream),
 *     which the call synchronises; 16 bytes per node of scratch are
 *     allocated and freed inside the call.
 *   device = 0: the host implementation (host pointers), which pdca_create
 *     runs for PDCA_TILING_ON.
 * Both give the same order.  row_ptr (n + 1 entries) must start at 0 and not
 * decrease (else PDCA_ERR_INVALID_ARG); columns outside [0, n) are skipped,
 * nothing else of the graph is checked.  PDCA_ERR_OOM: no memory for the
 * scratch; PDCA_ERR_CUDA: a CUDA error. */
pdca_status pdca_locality_order(const int64_t *row_ptr, const int32_t *col, int32_t n, int32_t sort_window,
                                int32_t device, int32_t *order, void *stream);

/* Copy the iterate to u_out (n x K float32, original node order, host or device). */
pdca_status pdca_get_u(pdca_problem *h, float *u_out);

/* Labels of the current iterate into labels_out (n int32, host or device):
 * K = 1: 1 if u_i >= 0 else 0;  K >= 2: argmax_k u_ik, lowest k on ties.
 * Synchronises.  Errors: INVALID_ARG, CUDA, BAD_GRAPH (a problem made by
 * pdca_create_like_async whose fidelity arrays failed the check; the labels
 * are written all the same). */
pdca_status pdca_labels(pdca_problem *h, int32_t *labels_out);

/* pdca_labels enqueued on the handle's stream without waiting: labels_out
 * (n int32, device or page-locked host memory) holds the labels once the
 * stream has passed the call; pageable host memory makes the call wait.
 * fid_status_out: NULL, or one uint32 (device or host) receiving 0 when the
 * fidelity arrays were valid and nonzero when pdca_create_like_async found a
 * bad mask value or label (written on the stream for a problem made by
 * pdca_create_like_async, at once otherwise).  The labels are staged in the
 * handle's spare iterate buffer, so a later step on the same stream is
 * ordered after the copy.  The labels are those of pdca_labels; the
 * asynchronous form has no counterpart in the paper.  Errors: INVALID_ARG,
 * CUDA. */
pdca_status pdca_labels_async(pdca_problem *h, int32_t *labels_out, uint32_t *fid_status_out);

/* The lambda_max in use by the Richardson preconditioner (the power-method
 * estimate raised by 0.1% and capped at 2, or the value given), and the raw
 * estimate (0 if none was computed). */
pdca_status pdca_lambda_max(pdca_problem *h, double *lambda_used, double *lambda_estimate);

/* Layout facts of a created problem: padded sliced-ELL entries, number of
 * 32-row slices, degree-sort window, whether the tiled kernels run, the total
 * and the largest number of halo rows over tiles (0 if not tiled), the
 * number of slices stored with 16-bit columns (PDCA_COLUMNS_AUTO), the split
 * length in use (0 if tiled) and the number of rows longer than it.  Any
 * pointer may be NULL. */
pdca_status pdca_layout(pdca_problem *h, int64_t *sell_entries, int64_t *n_slices,
                        int32_t *sort_window, int32_t *tiled, int64_t *halo_rows, int32_t *max_halo,
                        int64_t *slices16, int32_t *split_len, int64_t *split_rows);

/* CUDA graph replay of pdca_solve: with on = 1, a call without traces (and
 * with profiling off, a plain non-tiled handle and a non-default stream) is
 * captured once into a CUDA graph per (outer, inner, starting buffers,
 * coefficients) and replayed on later calls with the same key (at most 6 kept
 * per handle, oldest dropped first).  The replay launches exactly the kernels
 * and arguments of the direct path, so results are identical; it removes the
 * per-launch host cost, which dominates for small graphs.  The graphs are
 * CUDA driver objects (host and device resources the driver manages); on = 0
 * or pdca_destroy releases them.  Default off.  When the caller's stream is
 * itself being captured, pdca_solve launches directly into that capture. */
pdca_status pdca_graph_enable(pdca_problem *h, int32_t on);

/* Kernel timing for measurement: enable (1) / disable (0) CUDA-event timing
 * of every sweep launch of this handle; read returns the summed sweep time
 * in milliseconds and the number of timed launches since the last read, and
 * resets both (synchronises). */
pdca_status pdca_profile_enable(pdca_problem *h, int32_t on);
pdca_status pdca_profile_read(pdca_problem *h, double *sweep_ms, int64_t *sweep_launches);

/* Spectral initial iterate for the unsupervised model (no labelled nodes,
 * K = 1): the paper initialises its unsupervised clustering runs with the
 * eigenvector of the second-smallest eigenvalue of the normalized graph
 * Laplacian (Sec. 5.3, Table of the clustering data sets).  This computes that
 * eigenpair (lambda_2, v_2) of the handle's Laplacian (L_s, or L for
 * PDCA_LAP_UNNORMALIZED): the smallest eigenpair on the orthogonal complement
 * of the null vector D^1/2 1 (or 1), which is the second-smallest one on a
 * connected graph and stays unique on a graph with several components.  It
 * runs a block LOBPCG on the handle's operator and sets
 * u^0 = v_2 / max_i |v_2,i|, signed so that its largest-magnitude entry
 * (lowest node index among equal ones) is +1.  Where the handle stores BF16
 * weights (mixed precision) the eigenpair is that of the BF16 operator.
 *   workspace: DEVICE scratch of at least pdca_spectral_workspace_size bytes,
 *     256-byte aligned, owned by the caller (free to reuse after the call);
 *   max_iters >= 0: LOBPCG iterations; tol > 0: stop when the residual norm
 *     ||L x - theta x|| of the unit Ritz vector is <= tol B, with B = 2 for
 *     L_s and 2 max_i d_i for L (the bound of the spectrum); FP32 arithmetic
 *     makes values below about 1e-6 unreachable;
 *   lambda2 (nullable, host): the Ritz value of the second-smallest eigenpair;
 *   u0_out (nullable, host or device, n floats): the u^0 that was set;
 *   iters_done (nullable, host): iterations run.
 * Synchronises the handle's stream.  Errors: INVALID_ARG (K != 1, a handle
 * with PDCA_TILING_ON, bad arguments), OOM (workspace too small), NONFINITE,
 * CUDA; NOT_CONVERGED when max_iters ran out first (u^0 is still set, from
 * the last Ritz vector). */
pdca_status pdca_spectral_workspace_size(const pdca_problem *h, size_t *bytes);
pdca_status pdca_spectral_init(pdca_problem *h, void *workspace, size_t ws_bytes, int32_t max_iters, double tol,
                               double *lambda2, float *u0_out, int32_t *iters_done);

/* Nonlocal image graph (Sec. 2.3): w_ij = K(i,j) N(i,j) with the Gaussian
 * kernel of patch distances K (eq. kij, alpha_n = 1) and the window
 * indicator N_s, restricted to each pixel's k window neighbours of smallest
 * patch distance and symmetrised by union (an edge where either end keeps
 * the other).  Pixel i = y W + x.
 *   patch distance d2(i,j) = sum over the (2p+1)^2 patch offsets (raster
 *     order) and the C channels of (a - b)^2, FP32 with every square and sum
 *     rounded separately, patches replicate-padded at the border;
 *   candidates: j != i with max(|y_i - y_j|, |x_i - x_j|) <= r inside the
 *     image; the k smallest (d2, j) are kept (equal distances go to the lower
 *     index);  w_ij = float(exp(-d2 / sigma^2)) (double exp), symmetric bit
 *     for bit.
 *   image: DEVICE, H x W x C float32, row-major (pixel-major, channels last);
 *   1 <= C <= 16, 0 <= patch_radius p <= 4, window_radius r >= 1,
 *   1 <= k <= 32 and (min(H, 2r+1) min(W, 2r+1) - 1) >= k; sigma > 0.
 *   workspace: DEVICE scratch of pdca_image_graph_workspace_size bytes,
 *     256-byte aligned.  row_ptr (H W + 1 int64), col (col_capacity int32)
 *     and w (col_capacity float32): DEVICE outputs; 2 k H W always suffices.
 *   *nnz (host): the number of entries; rows come out with strictly
 *     increasing columns, ready for pdca_create.
 * Synchronises the stream.  Errors: INVALID_ARG (sizes, a host pointer among
 * image/workspace/outputs), OOM (workspace or col_capacity too small; *nnz
 * then holds the size needed), CUDA. */
pdca_status pdca_image_graph_workspace_size(int32_t H, int32_t W, int32_t k, size_t *bytes);
pdca_status pdca_image_graph(const float *image, int32_t H, int32_t W, int32_t C, int32_t patch_radius,
                             int32_t window_radius, int32_t k, double sigma, void *workspace, size_t ws_bytes,
                             int64_t *row_ptr, int32_t *col, float *w, int64_t col_capacity, int64_t *nnz,
                             void *stream);

/* k-NN graph of a point cloud (Sec. 2.3 for clustering): the k nearest
 * neighbours by Euclidean distance (N_c) with the Gaussian kernel of the
 * local-scaling bandwidth of Zelnik-Manor and Perona,
 *   w_ij = exp(-|x_i - x_j|^2 / (sigma_i sigma_j)),
 * sigma_i = distance of i to its scale_nn-th nearest neighbour (self
 * excluded), symmetrised by union (an edge where either end keeps the other).
 * Distances are screened on the mean-centred points (|x|^2 + |y|^2 - 2 x.y,
 * the products on the tensor cores with each FP32 coordinate split into two
 * BF16 parts, FP32 accumulation) to 3k + 8 candidates per point, then
 * recomputed exactly in FP64 as sums of squared coordinate differences; the k
 * smallest (d2, j) are kept (equal distances go to the lower index).  The
 * weights are symmetric bit for bit.
 *   X: DEVICE, n x dim float32, row-major; 2 <= n < 2^31, 1 <= k <= 32,
 *   k <= n - 1, 1 <= scale_nn <= k.
 *   workspace: DEVICE scratch of pdca_point_graph_workspace_size bytes,
 *     256-byte aligned (it holds a tile of min(8192, 2^28 / n) x n FP32
 *     distances, and a centred copy of X).  row_ptr (n + 1 int64), col and w
 *     (col_capacity entries):
 *     DEVICE outputs; 2 k n always suffices.  *nnz (host): the entries.
 * Synchronises the stream.  Errors: INVALID_ARG, OOM (workspace or
 * col_capacity; *nnz then holds the size needed), BAD_GRAPH (some sigma_i = 0:
 * i has scale_nn coincident points), CUDA. */
pdca_status pdca_point_graph_workspace_size(int64_t n, int32_t dim, int32_t k, size_t *bytes);
pdca_status pdca_point_graph(const float *X, int64_t n, int32_t dim, int32_t k, int32_t scale_nn, void *workspace,
                             size_t ws_bytes, int64_t *row_ptr, int32_t *col, float *w, int64_t col_capacity,
                             int64_t *nnz, void *stream);

/* Number of kernels this library has launched in the process so far. */
uint64_t pdca_kernel_launches(void);

/* GL energy F(u) of an iterate, computed directly from a device CSR graph,
 * for callers that cannot allocate device memory and so cannot hand the
 * library a workspace: a host framework that owns every device byte through
 * its own fixed pool and allows no other allocator (or a plug-in loaded into
 * such a process), or a loop that must not pay cudaMalloc's implicit
 * device-wide synchronisation.  The paper has no counterpart of this call; it
 * evaluates the same F as pdca_energy for the normalized Laplacian L_s only
 * (a problem created with PDCA_LAP_UNNORMALIZED has a different F).
 *   row_ptr (n+1 int64), col (nnz int32), w (nnz float32), u (n x k float32,
 *   row-major), fid_mask (n uint8), labels (n int32): DEVICE pointers, same
 *   conventions as pdca_create; eps > 0, eta >= 0; stream: cudaStream_t as
 *   void*; F_out: host or device pointer receiving F (written on success
 *   only; a device F_out is written by a kernel on `stream`).
 * Checks: row_ptr inside [0, nnz], columns in [0, n), no self loop, weights
 * finite and >= 0, mask values 0/1, prior labels in [0, max(k, 2)) on
 * labelled rows.  Symmetry and the column order are NOT checked.
 * Allocates nothing: the scratch is a fixed device array inside the library
 * (about 4.1 MiB, held on every GPU that loads the library until the process
 * exits), limiting n to PDCA_STATIC_MAX_N.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  All calls share
 * the array and overwrite it (the status word is cleared at the start of
 * every call); calls whose kernels overlap on the GPU (two streams, two host
 * threads) race on it and must be serialised by the caller.  The call reads
 * its status back and synchronises `stream` before returning.
 * Errors: INVALID_ARG (bad sizes or a host pointer among the inputs),
 * TOO_LARGE (n > PDCA_STATIC_MAX_N), BAD_GRAPH (a failed check above),
 * ISOLATED_NODE, NONFINITE, CUDA. */
pdca_status pdca_energy_static(const int64_t *row_ptr, const int32_t *col, const float *w,
                               int32_t n, int64_t nnz, int32_t k, const float *u,
                               const uint8_t *fid_mask, const int32_t *labels, double eps,
                               double eta, void *stream, double *F_out);

/* ---- batches: many problems advanced together (continuous batching) ------
 * A batch holds problems that were created on the batch's stream (plain
 * kernels: not PDCA_TILING_ON).  pdca_batch_step advances every member by up
 * to `passes` passes (one pass = one sweep of the FP32 form, or one pass of
 * the mixed form), with one kernel launch per K class per pass: all members
 * of a class share the launch, whatever their sizes, precisions and
 * positions inside their outer steps.  A member leaves the batch after its
 * `outer_iters` outer steps of `inner_sweeps` sweeps; pdca_batch_poll hands
 * finished problems back.  Members may join between steps (continuous
 * batching).  A member's iterates are bit-identical to those of pdca_solve
 * with the same arguments: the batched kernel runs the same per-row code.
 * The paper solves one problem at a time; batching is a serving extension.
 * A batch allocates host memory only.  While a problem is a member, use it
 * only through the batch (its u is mid-step between passes). */
typedef struct pdca_batch pdca_batch;
pdca_status pdca_batch_create(int32_t max_problems, void *stream, pdca_batch **out);
/* INVALID_ARG for a problem on another stream, a tiled problem, a problem
 * already in the batch, a full batch, or outer_iters / inner_sweeps < 1. */
pdca_status pdca_batch_add(pdca_batch *b, pdca_problem *h, int32_t outer_iters, int32_t inner_sweeps);
/* Asynchronous; active_after (nullable) receives the members still running. */
pdca_status pdca_batch_step(pdca_batch *b, int32_t passes, int32_t *active_after);
/* Up to `capacity` finished problems into done[] (count written); removes them. */
pdca_status pdca_batch_poll(pdca_batch *b, pdca_problem **done, int32_t capacity, int32_t *count);
/* Remove a problem (running or finished) without finishing it. */
pdca_status pdca_batch_remove(pdca_batch *b, pdca_problem *h);
/* Synchronises the stream; the member problems stay the caller's. */
void pdca_batch_destroy(pdca_batch *b);

/* Release the handle's host-side state (the workspace stays the caller's).
 * Synchronises the handle's stream first.  NULL is ignored. */
void pdca_destroy(pdca_problem *h);

/* pdca_destroy without waiting for the stream (it still waits when the
 * handle holds captured solve graphs).  Work already enqueued for the
 * handle keeps running and reads the workspace, so the caller reuses the
 * workspace only in the stream's order: on the same stream (a stream-ordered
 * allocator such as PyTorch's caching allocator on that stream), or after an
 * event recorded on the stream has completed.  No counterpart in the
 * paper.  NULL is ignored. */
void pdca_release(pdca_problem *h);

/* Static description of a status code. */
const char *pdca_status_string(pdca_status s);

#ifdef __cplusplus
}
#endif
#endif /* PDCA_H */
