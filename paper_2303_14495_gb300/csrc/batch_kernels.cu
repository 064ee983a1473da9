// Batched pass: many problems of the same K advanced by one pass (FP32 sweep,
// mixed residual or mixed correction sweep) in a single launch.  The table of
// per-problem descriptors is a __grid_constant__ kernel parameter, so a launch
// needs no device-side table and no copy.  Each warp handles one slice of one
// problem with exactly the device code of the single-problem kernels, so a
// problem's iterates are bit-identical alone and in a batch.  Problems on the
// unnormalized Laplacian go to their own launches (batch_kernels_un.cu).
#include "batch_body.cuh"

namespace pdca {

cudaError_t launch_batch_pass(int K, bool un, const BatchTable &t, cudaStream_t st) {
    if (t.n <= 0 || t.total_slices <= 0) return cudaSuccess;
    count_launches(1);
    return un ? launch_batch_pass_un(K, t, st) : batch_all<false>(K, t, st);
}

}  // namespace pdca
