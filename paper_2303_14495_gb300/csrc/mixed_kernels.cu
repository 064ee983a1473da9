// Mixed-precision form of one outer pDCA step: BF16 pre-scaled weights,
// FP16 or BF16 storage of the correction, FP32 arithmetic, FP32 master
// iterate.
//
// The diagonal sweeps of Prop. nopre started from v^0 = u^t are, written for
// the correction e^s = v^s - u^t,
//   r    = b^t - T u^t                                  (once per outer step)
//   e^1  = G^{-1} r                                     (e^0 = 0)
//   e^{s+1} = e^s + G^{-1} (r - T e^s),   u^{t+1} = u^t + e^m,
// the same iteration up to rounding.  r is formed in FP32 from the FP32
// iterate; only the small correction e and r travel in 16-bit storage, so
// their rounding error is relative to |e|, not to |u| (the FP32 residual
// correction of each outer step).  In
//   b - T u = eta Lambda (y - u) - (u^3 - u)/eps - eps (u - sum_j wt_ij u_j)
// the two c u terms cancel exactly and are never formed.
#include "device_common.cuh"

namespace pdca {
namespace {

using namespace dev;

template <int K, class HT, bool LAST, bool PROJECT>
__global__ void __launch_bounds__(kBlockThreads)
mixed_residual_kernel(const SellView A, const Coeffs cf, const float *__restrict__ u, HT *__restrict__ r_out,
                      HT *__restrict__ e_out, float *__restrict__ u_out) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (slice >= A.n_slices) return;
    mixed_residual_slice<K, HT, LAST, PROJECT>(A, cf, slice, threadIdx.x & 31, u, r_out, e_out, u_out);
}

template <int K, class HT, bool LAST, bool PROJECT>
__global__ void __launch_bounds__(kBlockThreads)
mixed_sweep_kernel(const SellView A, const Coeffs cf, const HT *__restrict__ e_src, const HT *__restrict__ rr,
                   HT *__restrict__ e_dst, const float *__restrict__ u, float *__restrict__ u_out) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (slice >= A.n_slices) return;
    mixed_sweep_slice<K, HT, LAST, PROJECT>(A, cf, slice, threadIdx.x & 31, e_src, rr, e_dst, u, u_out);
}

template <int K, class HT>
cudaError_t residual_k(bool last, bool project, const SellView &A, const Coeffs &cf, const float *u, void *r,
                       void *e, float *u_out, cudaStream_t st) {
    const int blocks = (A.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    HT *rh = static_cast<HT *>(r), *eh = static_cast<HT *>(e);
    if (!last)
        mixed_residual_kernel<K, HT, false, false><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh, u_out);
    else if (project && K >= 2)
        mixed_residual_kernel<K, HT, true, (K >= 2)><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh, u_out);
    else
        mixed_residual_kernel<K, HT, true, false><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh, u_out);
    return cudaGetLastError();
}

template <int K, class HT>
cudaError_t sweep_k(bool last, bool project, const SellView &A, const Coeffs &cf, const void *e_src,
                    const void *r, void *e_dst, const float *u, float *u_out, cudaStream_t st) {
    const int blocks = (A.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const HT *es = static_cast<const HT *>(e_src), *rh = static_cast<const HT *>(r);
    HT *ed = static_cast<HT *>(e_dst);
    if (!last)
        mixed_sweep_kernel<K, HT, false, false><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u, u_out);
    else if (project && K >= 2)
        mixed_sweep_kernel<K, HT, true, (K >= 2)><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u, u_out);
    else
        mixed_sweep_kernel<K, HT, true, false><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u, u_out);
    return cudaGetLastError();
}

}  // namespace

#define PDCA_DISPATCH_K(K, CALL)                                                      \
    switch (K) {                                                                      \
    case 1: return CALL(1); case 2: return CALL(2); case 3: return CALL(3);           \
    case 4: return CALL(4); case 5: return CALL(5); case 6: return CALL(6);           \
    case 7: return CALL(7); case 8: return CALL(8); case 9: return CALL(9);           \
    case 10: return CALL(10); case 11: return CALL(11); case 12: return CALL(12);     \
    case 13: return CALL(13); case 14: return CALL(14); case 15: return CALL(15);     \
    case 16: return CALL(16);                                                         \
    default: return cudaErrorInvalidValue;                                            \
    }

cudaError_t launch_mixed_residual(int K, bool bf16u, bool last, bool project, const SellView &A,
                                  const Coeffs &cf, const float *u, void *r, void *e, float *u_out,
                                  cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
    if (bf16u) {
#define CALL(KK) residual_k<KK, __nv_bfloat16>(last, project, A, cf, u, r, e, u_out, st)
        PDCA_DISPATCH_K(K, CALL)
#undef CALL
    }
#define CALL(KK) residual_k<KK, __half>(last, project, A, cf, u, r, e, u_out, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

cudaError_t launch_mixed_sweep(int K, bool bf16u, bool last, bool project, const SellView &A, const Coeffs &cf,
                               const void *e_src, const void *r, void *e_dst, const float *u, float *u_out,
                               cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
    if (bf16u) {
#define CALL(KK) sweep_k<KK, __nv_bfloat16>(last, project, A, cf, e_src, r, e_dst, u, u_out, st)
        PDCA_DISPATCH_K(K, CALL)
#undef CALL
    }
#define CALL(KK) sweep_k<KK, __half>(last, project, A, cf, e_src, r, e_dst, u, u_out, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

}  // namespace pdca
