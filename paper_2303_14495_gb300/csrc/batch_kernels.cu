// Batched pass: many problems of the same K advanced by one pass (FP32 sweep,
// mixed residual or mixed correction sweep) in a single launch.  The table of
// per-problem descriptors is a __grid_constant__ kernel parameter, so a launch
// needs no device-side table and no copy.  Each warp handles one slice of one
// problem with exactly the device code of the single-problem kernels, so a
// problem's iterates are bit-identical alone and in a batch.  This unit holds
// the L_s instances for K <= 8 and the dispatch; batch_kernels_*.cu the rest.
#include "batch_body.cuh"

namespace pdca {

cudaError_t batch_pass_ls_lo(int K, const BatchTable &t, cudaStream_t st) { return batch_set<false, true>(K, t, st); }

cudaError_t launch_batch_pass(int K, bool un, const BatchTable &t, cudaStream_t st) {
    if (t.n <= 0 || t.total_slices <= 0) return cudaSuccess;
    count_launches(1);
    if (un) return K <= 8 ? batch_pass_un_lo(K, t, st) : batch_pass_un_hi(K, t, st);
    return K <= 8 ? batch_pass_ls_lo(K, t, st) : batch_pass_ls_hi(K, t, st);
}

}  // namespace pdca
