// Mixed-precision outer step for the unnormalized Laplacian L = D - W with
// BF16 correction storage (the kernels of mixed_body.cuh with a_i = d_i read
// per row).
#include "mixed_body.cuh"

namespace pdca {

PDCA_MIXED_SET(mixed_un_b16, true, __nv_bfloat16)

}  // namespace pdca
