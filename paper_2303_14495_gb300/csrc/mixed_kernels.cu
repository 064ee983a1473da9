// Mixed-precision form of one outer pDCA step: an FP32 residual pass, then
// correction sweeps with BF16 pre-scaled weights and FP16 or BF16 storage of
// the correction, FP32 arithmetic, FP32 master iterate.
//
// The diagonal sweeps of Prop. nopre started from v^0 = u^t are, written for
// the correction e^s = v^s - u^t,
//   r    = b^t - T u^t                                  (once per outer step)
//   e^1  = G^{-1} r                                     (e^0 = 0)
//   e^{s+1} = e^s + G^{-1} (r - T e^s),   u^{t+1} = u^t + e^m,
// the same iteration up to rounding (L_s or, in the UN instances, L).  r is
// formed with the FP32 weights from the FP32 iterate and kept in FP32 (the
// FP32 residual correction of each outer step); only the correction e travels
// in 16-bit storage and only its sweeps use the BF16 weights, so their
// rounding errors are relative to |e|, not to |u|.  In
//   b - T u = eta Lambda (y - u) - (u^3 - u)/eps - eps (u - sum_j wt_ij u_j)
// the two c u terms cancel exactly and are never formed.
#include "mixed_body.cuh"

namespace pdca {

// this unit: L_s with FP16 correction storage; mixed_kernels_*.cu the other sets
PDCA_MIXED_SET(mixed_ls_f16, false, __half)

cudaError_t launch_mixed_residual(int K, bool bf16u, bool last, bool project, const SellView &A,
                                  const Coeffs &cf, const float *u, void *r, void *e, float *u_out,
                                  cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
    if (A.self)
        return bf16u ? mixed_un_b16_residual(K, last, project, A, cf, u, r, e, u_out, st)
                     : mixed_un_f16_residual(K, last, project, A, cf, u, r, e, u_out, st);
    return bf16u ? mixed_ls_b16_residual(K, last, project, A, cf, u, r, e, u_out, st)
                 : mixed_ls_f16_residual(K, last, project, A, cf, u, r, e, u_out, st);
}

cudaError_t launch_mixed_sweep(int K, bool bf16u, bool last, bool project, const SellView &A, const Coeffs &cf,
                               const void *e_src, const void *r, void *e_dst, const float *u, float *u_out,
                               cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
    if (A.self)
        return bf16u ? mixed_un_b16_sweep(K, last, project, A, cf, e_src, r, e_dst, u, u_out, st)
                     : mixed_un_f16_sweep(K, last, project, A, cf, e_src, r, e_dst, u, u_out, st);
    return bf16u ? mixed_ls_b16_sweep(K, last, project, A, cf, e_src, r, e_dst, u, u_out, st)
                 : mixed_ls_f16_sweep(K, last, project, A, cf, e_src, r, e_dst, u, u_out, st);
}

}  // namespace pdca
