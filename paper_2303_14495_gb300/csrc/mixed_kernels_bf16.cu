// Mixed-precision outer step for L_s with BF16 correction storage (the
// kernels of mixed_body.cuh).
#include "mixed_body.cuh"

namespace pdca {

PDCA_MIXED_SET(mixed_ls_b16, false, __nv_bfloat16)

}  // namespace pdca
