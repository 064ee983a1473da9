// Batched passes of problems on L_s with K > 8 (the kernels of
// batch_body.cuh).
#include "batch_body.cuh"

namespace pdca {

cudaError_t batch_pass_ls_hi(int K, const BatchTable &t, cudaStream_t st) { return batch_set<false, false>(K, t, st); }

}  // namespace pdca
