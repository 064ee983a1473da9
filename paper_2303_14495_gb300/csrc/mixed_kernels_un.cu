// Mixed-precision outer step for the unnormalized Laplacian L = D - W with
// FP16 correction storage: the kernels of mixed_body.cuh with a_i = d_i read
// per row (launched through launch_mixed_residual / launch_mixed_sweep).
#include "mixed_body.cuh"

namespace pdca {

PDCA_MIXED_SET(mixed_un_f16, true, __half)

}  // namespace pdca
