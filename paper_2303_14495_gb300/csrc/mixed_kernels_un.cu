// Mixed-precision outer step for the unnormalized Laplacian L = D - W: the
// kernels of mixed_body.cuh with a_i = d_i read per row (launched through
// launch_mixed_residual / launch_mixed_sweep).
#include "mixed_body.cuh"

namespace pdca {

cudaError_t launch_mixed_residual_un(int K, bool bf16u, bool last, bool project, const SellView &A,
                                     const Coeffs &cf, const float *u, void *r, void *e, float *u_out,
                                     cudaStream_t st) {
    return mixed_residual_all<true>(K, bf16u, last, project, A, cf, u, r, e, u_out, st);
}

cudaError_t launch_mixed_sweep_un(int K, bool bf16u, bool last, bool project, const SellView &A,
                                  const Coeffs &cf, const void *e_src, const void *r, void *e_dst, const float *u,
                                  float *u_out, cudaStream_t st) {
    return mixed_sweep_all<true>(K, bf16u, last, project, A, cf, e_src, r, e_dst, u, u_out, st);
}

}  // namespace pdca
