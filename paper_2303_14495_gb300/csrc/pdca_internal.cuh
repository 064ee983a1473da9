// Internal declarations shared by the library's translation units.
//
// Data layout in device memory (all inside the caller's workspace):
//   * nodes are renumbered: inside every window of `sigma` consecutive rows,
//     rows are sorted by degree (descending, ties by original index); the
//     renumbering is applied to rows and columns alike, so u, the tags and
//     the operator all live in the new order;
//   * the operator D^{-1/2} W D^{-1/2} (Sec. 2.2) is stored as sliced ELL
//     with slices of 32 rows (one warp, one lane per row).  Entries go in
//     groups of kVec: entry j of lane l of slice s sits at
//     slice_off[s] + 32 kVec (j / kVec) + kVec l + (j % kVec), so every lane
//     reads kVec consecutive entries with one 128-bit load of columns and
//     one of weights, and a warp reads 512 contiguous bytes per load;
//     slice width = longest row of the slice rounded up to kVec; padding
//     entries point at a valid row with weight 0;
//   * columns: int32 (new numbering), or, in slices that allow it, 16-bit
//     (the low 16 bits; the column's 65536-node chunk is the row's own, the
//     previous or the next one, told apart by the entry's band: each row of
//     such a slice keeps first its entries in the previous chunk, then those
//     in the next chunk, then those in its own chunk and the padding);
//   * rows longer than a split length T (plain kernels only) keep their
//     first T entries in the sliced ELL; the rest go to an overflow CSR (one
//     row per such row, in row order) whose sums a pre-pass forms, one warp
//     per row, before the kernel that needs them;
//   * rowinfo[r] = tag | len << 8 | overflow << 19 (plain kernels: len <= T
//     <= 2044, 11 bits), and in a slice with 16-bit columns also
//     n_prev << 20 (6 bits) | n_next << 26 (6 bits); tiled kernels:
//     tag | len << 8 (24 bits);
//   * u is n_pad x K float32 row-major (n_pad = 32 * number of slices).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "pdca.h"

namespace pdca {

constexpr int kSliceRows = 32;
constexpr int kVec = 4;                        // entries per lane per load
constexpr uint32_t kTagUnlabelled = 0xFFu;
constexpr int kBlockThreads = 256;             // 8 warps = 8 slices per block
constexpr int kWarpsPerBlock = kBlockThreads / 32;
constexpr int kRedSlots = 8;                   // doubles per block partial

// Validation status bits (OR-ed by the validation kernel).
constexpr uint32_t kBadGraph = 1u;
constexpr uint32_t kNotSymmetric = 2u;
constexpr uint32_t kIsolated = 4u;
constexpr uint32_t kLayoutMismatch = 8u;   // internal: packed row longer than its slice

// The Laplacian as (L x)_i = a_i x_i - sum_j w'_ij x_j:  L_s has a_i = 1 and
// w' = w_ij / sqrt(d_i d_j);  L = D - W has a_i = d_i and w' = w_ij.
constexpr int kChunkShift = 16;              // 16-bit columns: 65536-node chunks
constexpr uint8_t kFmt32 = 0, kFmt16 = 1;   // column format of a slice
constexpr uint32_t kBandMax = 63;           // largest n_prev / n_next of a 16-bit row
constexpr uint32_t kLenMask = 0x7FFu;       // rowinfo length field (plain kernels)
constexpr uint32_t kOvFlag = 1u << 19;      // the row continues in the overflow CSR
constexpr int32_t kSplitMax = 2044;         // largest split length (fits kLenMask, multiple of kVec)
constexpr int kFmtGroupSlices = 32;         // slices sharing one column format
struct SellView {
    const int32_t *col;        // padded sliced-ELL column indices (new numbering)
    const uint16_t *col16;     // low 16 bits of the columns (slices with slice_fmt = kFmt16)
    const uint8_t *slice_fmt;  // kFmt32 / kFmt16 per slice; nullptr: every slice kFmt32
    const float *w;            // w'_ij, FP32 (both precisions)
    const __nv_bfloat16 *wb;   // the same in BF16 (mixed-precision path; nullptr otherwise)
    const int64_t *slice_off;  // n_slices + 1 entry offsets
    const uint32_t *rowinfo;   // (len << 8) | tag, n_pad
    const float *self;         // a_i = d_i per row (n_pad) for L; nullptr for L_s
    const int32_t *ov_index;   // overflow row of each row with kOvFlag (n_pad), else unused
    const float *ov_acc;       // the pre-pass sums, K floats per overflow row
    int32_t n_slices;
    int32_t n;                 // real rows; rows >= n are padding
    int32_t stream_rows;       // 1: the iterates exceed L2, store rows with st.global.cs
    int32_t block_iters;       // slice groups of 8 per block range (1, 2, 4); 0 = sweep_iters(n_slices)
};

// The overflow CSR of the rows longer than the split length (entries past
// the first T, in the pack's order), in new row order.
struct OverflowView {
    const int64_t *rp;         // n_rows + 1 offsets
    const int32_t *col;        // columns (new numbering)
    const float *w;            // FP32 weights
    const __nv_bfloat16 *wb;   // BF16 weights (mixed precision; else nullptr)
    int32_t n_rows;
};
enum OvWeights : int32_t { kOvW32 = 0, kOvW16 = 1 };
enum OvRows : int32_t { kOvX32 = 0, kOvXHalf = 1, kOvXBf16 = 2 };

// Resident blocks per SM the plain sweep is compiled for (registers per
// thread <= 65536 / (256 x blocks)).
#ifndef PDCA_SWEEP_MIN_BLOCKS
#define PDCA_SWEEP_MIN_BLOCKS 4
#endif
// A block of the plain sweep handles up to this many consecutive groups of 8
// slices in turn (neighbouring slices of the renumbering share most neighbour
// rows, so later groups find many of them in the same SM's L1); fewer when
// the graph is too small to keep every SM busy for several waves.
#ifndef PDCA_SWEEP_MAX_ITERS
#define PDCA_SWEEP_MAX_ITERS 4
#endif
constexpr int kSmCount = 152;   // GB300
// slice groups per block for a graph of n_slices slices (at least 4 waves):
// 1, 2 or 4, so a block's range of 8 x iters slices never crosses a group of
// kFmtGroupSlices slices (one column format per group)
inline int sweep_iters(int32_t n_slices) {
    const int groups = (n_slices + 7) / 8;
    const int it = groups / (4 * kSmCount * PDCA_SWEEP_MIN_BLOCKS);
    return it >= 4 && PDCA_SWEEP_MAX_ITERS >= 4 ? 4 : (it >= 2 && PDCA_SWEEP_MAX_ITERS >= 2 ? 2 : 1);
}
static_assert(PDCA_SWEEP_MAX_ITERS * 8 <= kFmtGroupSlices, "a queue range must fit in one format group");
// the block range of a problem's queue kernels (a layout choice, pdca_params.block_slices)
inline int view_iters(const SellView &A) { return A.block_iters > 0 ? A.block_iters : sweep_iters(A.n_slices); }

// Tiled form of the operator: tiles of kTileSlices slices; each tile lists
// the distinct rows its entries reference (its halo, sorted), and every entry
// stores the position of its column in that list (16 bits).  The tiled
// kernels stage the halo rows of u in shared memory once per tile.
constexpr int kBfsBlock = 1024;                        // nodes per BFS block (renumbering)
constexpr int kTileSlices = 16;
constexpr int kTileRows = kTileSlices * kSliceRows;    // 512
constexpr int kTileThreads = kTileSlices * 32;         // one warp per slice
// Resident tiled blocks per SM the kernels are compiled for, and the shared
// memory one block may use for its halo (blocks x budget <= 227 KiB).
#ifndef PDCA_TILE_MIN_BLOCKS
#define PDCA_TILE_MIN_BLOCKS 2
#endif
#ifndef PDCA_TILE_SMEM_KB
#define PDCA_TILE_SMEM_KB 96
#endif
constexpr size_t kTileSmemBudget = (size_t)PDCA_TILE_SMEM_KB * 1024;
struct TileView {
    const int64_t *halo_off;   // n_tiles + 1
    const int32_t *halo_idx;   // halo rows (new numbering), sorted inside a tile
    const uint16_t *lcol;      // local column of every sliced-ELL entry
    int32_t n_tiles;
    int32_t max_halo;          // rows of the largest halo
    int32_t smem_rows;         // halo rows staged in shared memory; larger halos are read
                               // through halo_idx from global memory instead
};

// Scalars of one sweep (Sec. 3): T = eps L + eta Lambda + c I (c already
// holds c + 1/k for a finite step size k) and the preconditioner
// g_i = alpha a_i + beta_{Lambda_i}; for L_s (a_i = 1) the two values of
// 1/g_i (unlabelled, labelled rows) are precomputed.
struct Coeffs {
    float eps, inv_eps, c, eta, inv_g0, inv_g1;
    float alpha, beta0, beta1;
};

// Reduction results written by finalize kernels.
struct RedOut {
    double F;           // energy
    double rel_res;     // ||b - T u|| / ||b|| (NaN if no previous iterate)
    double quad, well, fid, rr, bb;
    double nonfinite;
};

// --- sweep / reductions (sweep_kernels.cu) ---------------------------------
// T == nullptr selects the plain kernels (neighbour rows gathered from global
// memory through L1/L2); otherwise the tiled kernels (halo in shared memory).
// A.self != nullptr (unnormalized L) needs T == nullptr.
cudaError_t launch_sweep(int K, bool project, const SellView &A, const TileView *T, const Coeffs &cf,
                         const float *v_src, const float *u_t, float *v_dst, cudaStream_t st);
cudaError_t launch_energy(int K, const SellView &A, const TileView *T, const Coeffs &cf, const float *u,
                          const float *u_prev, double *partials, cudaStream_t st);
// number of block partials the energy / power kernels write
int reduce_parts(const SellView &A, const TileView *T);
// shared memory for `rows` halo rows of K columns (bytes, 16-byte multiple)
__host__ __device__ inline size_t tile_smem_bytes(int K, int32_t rows) {
    return ((size_t)rows * (size_t)K * sizeof(float) + 15) / 16 * 16;
}
cudaError_t launch_energy_finalize(const double *partials, int n_parts, double eps, double eta,
                                   int has_prev, RedOut *out, double *trace_F,
                                   double *trace_r, cudaStream_t st);
cudaError_t launch_power_init(const SellView &A, const int32_t *perm, float *x,
                              double *partials, cudaStream_t st);
// y = L_s (s x); the block that finishes last (ticket counter, reset to 0 by
// it) sums the block partials in a fixed order and writes scale = 1/||y|| and
// lambda = Rayleigh quotient of s x (no separate finalize launch).
cudaError_t launch_power_spmv(const SellView &A, const TileView *T, const float *x, double *scale,
                              float *y, double *partials, unsigned *ticket, double *lambda, cudaStream_t st);
cudaError_t launch_power_finalize(const double *partials, int n_parts, double *scale,
                                  double *lambda, cudaStream_t st);
cudaError_t launch_labels(int K, int32_t n, const float *u, const int32_t *perm,
                          int32_t *out, cudaStream_t st);

// --- overflow pre-pass (overflow.cu) -----------------------------------------
// acc[q K + k] = sum over the overflow entries e of row q of w_e x[col_e][k]
// (x: n_pad x K rows of FP32, FP16 or BF16; weights FP32 or BF16).
cudaError_t launch_overflow(int K, int wkind, int xkind, const OverflowView &O, const void *x, float *acc,
                            cudaStream_t st);

// --- mixed precision (mixed_kernels.cu) --------------------------------------
// r is an n_pad x K FP32 array; e an n_pad x K array of FP16 (bf16u = false)
// or BF16 (bf16u = true).
cudaError_t launch_mixed_residual(int K, bool bf16u, bool last, bool project, const SellView &A,
                                  const Coeffs &cf, const float *u, void *r, void *e, float *u_out,
                                  cudaStream_t st);
cudaError_t launch_mixed_sweep(int K, bool bf16u, bool last, bool project, const SellView &A, const Coeffs &cf,
                               const void *e_src, const void *r, void *e_dst, const float *u, float *u_out,
                               cudaStream_t st);
// the instance sets (mixed_kernels*.cu): L_s or L = D - W, FP16 or BF16 e
#define PDCA_MIXED_DECL(NAME)                                                                                    \
    cudaError_t NAME##_residual(int K, bool last, bool project, const SellView &A, const Coeffs &cf,             \
                                const float *u, void *r, void *e, float *u_out, cudaStream_t st);               \
    cudaError_t NAME##_sweep(int K, bool last, bool project, const SellView &A, const Coeffs &cf,                \
                             const void *e_src, const void *r, void *e_dst, const float *u, float *u_out,        \
                             cudaStream_t st);
PDCA_MIXED_DECL(mixed_ls_f16)
PDCA_MIXED_DECL(mixed_ls_b16)
PDCA_MIXED_DECL(mixed_un_f16)
PDCA_MIXED_DECL(mixed_un_b16)
#undef PDCA_MIXED_DECL
cudaError_t launch_permute_out(int K, int32_t n, const float *u, const int32_t *perm,
                               float *out, cudaStream_t st);
cudaError_t launch_permute_in(int K, int32_t n, int32_t n_pad, const float *in,
                              const int32_t *perm, float *u, cudaStream_t st);
int energy_blocks(int32_t n_slices);
// blocks of the kernels whose block takes view_iters() groups of 8 slices
// from a queue (<= energy_blocks)
int queue_blocks(const SellView &A);

// --- batched passes (batch_kernels.cu) -------------------------------------
// One problem's pass inside a batched launch.  A launch advances every
// problem of its table by one pass; warps find their problem by binary search
// over slice_begin.  The per-row arithmetic is the single-problem kernels'.
enum BatchPassKind : int32_t { kPassFp32 = 0, kPassMixedResidual = 1, kPassMixedSweep = 2 };
struct BatchDesc {
    SellView A;
    Coeffs cf;
    int32_t slice_begin;     // first slice of this problem in the launch's slice range (a multiple of 8)
    int32_t kind;            // BatchPassKind
    int32_t last;            // last pass of the outer step
    int32_t project;         // project rows onto the simplex (last pass, K >= 2)
    int32_t bf16u;           // mixed: e stored as BF16 (else FP16); r is FP32
    int32_t pad_;
    const void *src;         // fp32: v^s;  mixed residual: u^t;  mixed sweep: e^s
    const void *aux;         // fp32: u^t;  mixed sweep: r
    void *dst;               // fp32: v^{s+1};  mixed residual: r;  mixed sweep: e^{s+1}
    void *dst2;              // mixed residual: e^1
    const float *u;          // mixed sweep: u^t
    float *u_out;            // mixed, last pass: u^{t+1}
};
constexpr int kBatchMax = 144;   // descriptors per launch (kernel parameter space)
struct BatchTable {
    int32_t n;
    int32_t total_slices;
    BatchDesc d[kBatchMax];
};
// The overflow pre-pass of a batched pass: every member with overflow rows,
// its rows numbered from q_begin in the launch's overflow-row range.
struct BatchOvDesc {
    OverflowView O;
    const void *x;
    float *acc;
    int32_t q_begin;
    int32_t wkind, xkind;
    int32_t pad_;
};
struct BatchOvTable {
    int32_t n;
    int32_t total_rows;
    BatchOvDesc d[kBatchMax];
};
cudaError_t launch_batch_overflow(int K, const BatchOvTable &t, cudaStream_t st);
// un: the table holds problems on the unnormalized Laplacian (A.self set).
cudaError_t launch_batch_pass(int K, bool un, const BatchTable &t, cudaStream_t st);
// the instance sets (batch_kernels*.cu): L_s or L, K <= 8 or K > 8
cudaError_t batch_pass_ls_lo(int K, const BatchTable &t, cudaStream_t st);
cudaError_t batch_pass_ls_hi(int K, const BatchTable &t, cudaStream_t st);
cudaError_t batch_pass_un_lo(int K, const BatchTable &t, cudaStream_t st);
cudaError_t batch_pass_un_hi(int K, const BatchTable &t, cudaStream_t st);

// --- preparation (prep_kernels.cu) -----------------------------------------
// status[0]: kBadGraph | kNotSymmetric | kIsolated bits; status[2..3]: the
// largest degree as the bits of a double (status must start zeroed).
cudaError_t launch_validate(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                            const float *w, const uint8_t *mask, const int32_t *labels,
                            double *deg, double *isd, uint32_t *status, cudaStream_t st);
cudaError_t launch_window_sort(int32_t n, int32_t n_pad, int32_t sigma, const int64_t *row_ptr,
                               int32_t *perm, int32_t *iperm, cudaStream_t st);
// From a node order already in perm[0, n) (position -> node): perm's padding
// rows set to -1, iperm, and slice_off (n_slices + 1) from the slice widths
// (longest row capped at split, rounded up to kVec).  count: n_slices int32
// scratch; scan_tmp: order_layout_scan_words(n_slices) int64 scratch.
cudaError_t launch_order_layout(int32_t n, int32_t n_pad, int32_t split, const int64_t *row_ptr, int32_t *perm,
                                int32_t *iperm, int32_t *count, int64_t *scan_tmp, int64_t *slice_off,
                                cudaStream_t st);
int64_t order_layout_scan_words(int32_t n_slices);
// BFS-block order of the nodes (order[p] = node at position p), chunks of
// `chunk` nodes (<= 65536) renumbered by one block each.  queue: n int32,
// key: n uint64 scratch; err: set nonzero if the order could not be formed
// (never expected).  Then the degree sort inside windows of sigma (a power
// of two <= 1024) positions, from order into out.
cudaError_t launch_bfs_blocks(int32_t n, int32_t block, int32_t chunk, const int64_t *row_ptr, const int32_t *col,
                              int32_t *queue, unsigned long long *key, int32_t *order, uint32_t *err,
                              cudaStream_t st);
cudaError_t launch_order_sort(int32_t n, int32_t sigma, const int64_t *row_ptr, const int32_t *order, int32_t *out,
                              cudaStream_t st);
// self == nullptr: L_s weights w_ij / sqrt(d_i d_j); else L weights w_ij and
// self[r] = d_i (0 on padding rows).  dsq (nullable): sqrt(d_i) per row.
// rowcls (nullable): entries are written in bands (previous, next, own
// chunk) and rowcls[r] records n_prev | n_next << 8 | 16-bit-capable << 16
// for the row's first split_len entries.  Entries past split_len go to the
// overflow CSR row ov_index[r] (ov_index: -1 for rows that fit).
cudaError_t launch_pack(int32_t n, int32_t n_pad, int32_t K, const int64_t *row_ptr,
                        const int32_t *col, const float *w, const double *deg, const double *isd,
                        const uint8_t *mask, const int32_t *labels, const int32_t *perm,
                        const int32_t *iperm, const int64_t *slice_off, int32_t *sell_col,
                        float *sell_w, __nv_bfloat16 *sell_wb, float *self, float *dsq, uint32_t *rowinfo,
                        uint32_t *rowcls, int32_t split_len, const int32_t *ov_index, const int64_t *ov_rp,
                        int32_t *ov_col, float *ov_w, __nv_bfloat16 *ov_wb, uint32_t *status, cudaStream_t st);
// tiled form: local 16-bit columns (position in the tile's halo) instead of int32
cudaError_t launch_pack_tiled(int32_t n_pad, const int64_t *row_ptr, const int32_t *col, const float *w,
                              const double *deg, const double *isd, const uint8_t *mask, const int32_t *labels,
                              const int32_t *perm, const int32_t *iperm, const int64_t *slice_off,
                              const int64_t *halo_off, const int32_t *halo_idx, uint16_t *lcol,
                              float *sell_w, uint32_t *rowinfo, uint32_t *status, cudaStream_t st);

// Entry order for the gathers (PDCA_ENTRIES_SPREAD), in place after the pack.
// Exactly one of sell_col (plain form) and lcol (tiled form, with its halo
// lists) is given, and exactly one of sell_w (FP32) and sell_wb (BF16).
// rowcls (nullable; from the pack): per row n_prev | n_next << 8 | 16-bit-capable
// << 16; the entries of a row are reordered only inside their band.
// len_mask: the rowinfo length field (kLenMask for the plain layout, 2^24 - 1
// for the tiled one).
cudaError_t launch_spread(int32_t n_pad, const int64_t *slice_off, const uint32_t *rowinfo, uint32_t len_mask,
                          const uint32_t *rowcls, int32_t *sell_col, uint16_t *lcol, const int64_t *halo_off,
                          const int32_t *halo_idx, float *sell_w, __nv_bfloat16 *sell_wb, cudaStream_t st);
// 16-bit columns for every slice whose rows all allow them (rowcls), the
// rowinfo of those rows in the 16-bit form, and slice_fmt per slice.
cudaError_t launch_compress(int32_t n_slices, const int64_t *slice_off, const uint32_t *rowcls,
                            const int32_t *sell_col, uint16_t *col16, uint32_t *rowinfo, uint8_t *slice_fmt,
                            cudaStream_t st);

// f(0) .. f(count - 1) on the host's threads (index order per thread is
// fixed, so results written per index do not depend on the thread count).
void host_parallel_for(int64_t count, const std::function<void(int64_t)> &f);

// --- host symbolic analysis (reorder.cpp) ------------------------------------
// order[new] = old: BFS blocks of `block` nodes inside fixed chunks of `chunk`
// nodes, then a stable degree sort (descending) inside every window of
// `sort_window` positions (a divisor of `block`).
void locality_order(int32_t n, const int64_t *rp, const int32_t *col, int32_t block, int32_t chunk,
                    int32_t sort_window, int32_t *order);
// per tile of tile_rows renumbered rows: sorted distinct neighbour rows.
void tile_halos(int32_t n, int32_t tile_rows, const int64_t *rp, const int32_t *col, const int32_t *perm,
                const int32_t *iperm, std::vector<int64_t> &halo_off, std::vector<int32_t> &halo_idx,
                int32_t *max_halo);
cudaError_t launch_init_u(int32_t n_pad, int32_t K, const uint32_t *rowinfo, float *u,
                          cudaStream_t st);
cudaError_t launch_retag(int32_t n_pad, int32_t K, const uint32_t *base_rowinfo, const int32_t *perm,
                         const uint8_t *mask, const int32_t *labels, uint32_t *rowinfo, uint32_t *status,
                         cudaStream_t st);

// --- spectral initial iterate (spectral.cu) -----------------------------------
size_t spectral_workspace_bytes(int32_t n_pad);
// Smallest eigenpair of the operator A (L_s, or L when un) on the orthogonal
// complement of its null vector q (q = sqrt(d_i) per renumbered row for L_s;
// the constant vector for L, q == nullptr); writes u0 = v2 / max|v2| (sign:
// largest-magnitude entry positive) in the caller's node order to
// out_caller_order (device, n floats).  PDCA_ERR_NOT_CONVERGED when
// max_iters ran out (the output is still written).
pdca_status spectral_eigvec(const SellView &A, const OverflowView &O, bool un, const float *q, const int32_t *perm, int32_t n,
                            int32_t n_pad, cudaStream_t st, void *workspace, int32_t max_iters, double tol,
                            double *lambda2, float *out_caller_order, int32_t *iters_done);

// Kernel launch counter (every launch_* above adds its launches).
void count_launches(uint64_t k);

}  // namespace pdca
