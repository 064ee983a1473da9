// Batched passes of problems on the unnormalized Laplacian L = D - W (the
// kernels of batch_body.cuh with a_i = d_i read per row), launched through
// launch_batch_pass.
#include "batch_body.cuh"

namespace pdca {

cudaError_t launch_batch_pass_un(int K, const BatchTable &t, cudaStream_t st) { return batch_all<true>(K, t, st); }

}  // namespace pdca
