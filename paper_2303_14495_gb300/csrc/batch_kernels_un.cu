// Batched passes of problems on the unnormalized Laplacian L = D - W, K <= 8
// (the kernels of batch_body.cuh with a_i = d_i read per row).
#include "batch_body.cuh"

namespace pdca {

cudaError_t batch_pass_un_lo(int K, const BatchTable &t, cudaStream_t st) { return batch_set<true, true>(K, t, st); }

}  // namespace pdca
