// Kernels of the mixed-precision outer step, shared by the four translation
// units that instantiate them (L_s or L = D - W, FP16 or BF16 correction
// storage), compiled separately so the sets build in parallel.
#pragma once
#include "device_common.cuh"

namespace pdca {
namespace {

using namespace dev;

// A block owns iters x 8 consecutive slices, handed to its warps from a
// shared queue (as in the FP32 sweep).
template <int K, class HT, bool LAST, bool PROJECT, bool UN, bool OV>
__global__ void __launch_bounds__(kBlockThreads)
mixed_residual_kernel(const SellView A, const Coeffs cf, const float *__restrict__ u, float *__restrict__ r_out,
                      HT *__restrict__ e_out, float *__restrict__ u_out, int iters) {
    __shared__ int next_slot;
    const int count = kWarpsPerBlock * iters;
    for_block_slices_fmt(A, blockIdx.x * count, count, &next_slot, [&](int slice, auto fmt) {
        mixed_residual_slice<K, HT, LAST, PROJECT, UN, decltype(fmt)::value, OV>(A, cf, slice, threadIdx.x & 31, u,
                                                                                 r_out, e_out, u_out);
    });
}

template <int K, class HT, bool LAST, bool PROJECT, bool UN, bool OV>
__global__ void __launch_bounds__(kBlockThreads)
mixed_sweep_kernel(const SellView A, const Coeffs cf, const HT *__restrict__ e_src, const float *__restrict__ rr,
                   HT *__restrict__ e_dst, const float *__restrict__ u, float *__restrict__ u_out, int iters) {
    __shared__ int next_slot;
    const int count = kWarpsPerBlock * iters;
    for_block_slices_fmt(A, blockIdx.x * count, count, &next_slot, [&](int slice, auto fmt) {
        mixed_sweep_slice<K, HT, LAST, PROJECT, UN, decltype(fmt)::value, OV>(A, cf, slice, threadIdx.x & 31, e_src,
                                                                              rr, e_dst, u, u_out);
    });
}

template <int K, class HT, bool UN, bool OV>
cudaError_t residual_ku(bool last, bool project, const SellView &A, const Coeffs &cf, const float *u, void *r,
                        void *e, float *u_out, cudaStream_t st) {
    const int iters = view_iters(A);
    const int blocks = (A.n_slices + kWarpsPerBlock * iters - 1) / (kWarpsPerBlock * iters);
    float *rh = static_cast<float *>(r);
    HT *eh = static_cast<HT *>(e);
    if (!last)
        mixed_residual_kernel<K, HT, false, false, UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh, u_out, iters);
    else if (project && K >= 2)
        mixed_residual_kernel<K, HT, true, (K >= 2), UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh,
                                                                                          u_out, iters);
    else
        mixed_residual_kernel<K, HT, true, false, UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, u, rh, eh, u_out, iters);
    return cudaGetLastError();
}

template <int K, class HT, bool UN, bool OV>
cudaError_t sweep_ku(bool last, bool project, const SellView &A, const Coeffs &cf, const void *e_src,
                     const void *r, void *e_dst, const float *u, float *u_out, cudaStream_t st) {
    const int iters = view_iters(A);
    const int blocks = (A.n_slices + kWarpsPerBlock * iters - 1) / (kWarpsPerBlock * iters);
    const HT *es = static_cast<const HT *>(e_src);
    const float *rh = static_cast<const float *>(r);
    HT *ed = static_cast<HT *>(e_dst);
    if (!last)
        mixed_sweep_kernel<K, HT, false, false, UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u, u_out, iters);
    else if (project && K >= 2)
        mixed_sweep_kernel<K, HT, true, (K >= 2), UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u,
                                                                                       u_out, iters);
    else
        mixed_sweep_kernel<K, HT, true, false, UN, OV><<<blocks, kBlockThreads, 0, st>>>(A, cf, es, rh, ed, u, u_out, iters);
    return cudaGetLastError();
}

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

// One instance set per (Laplacian, correction storage type): the kernels
// for every K, with and without overflow sums.
template <bool UN, class HT>
cudaError_t mixed_residual_set(int K, bool last, bool project, const SellView &A, const Coeffs &cf, const float *u,
                               void *r, void *e, float *u_out, cudaStream_t st) {
    if (A.ov_index) {
#define CALL(KK) residual_ku<KK, HT, UN, true>(last, project, A, cf, u, r, e, u_out, st)
        PDCA_DISPATCH_K(K, CALL)
#undef CALL
    }
#define CALL(KK) residual_ku<KK, HT, UN, false>(last, project, A, cf, u, r, e, u_out, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

template <bool UN, class HT>
cudaError_t mixed_sweep_set(int K, bool last, bool project, const SellView &A, const Coeffs &cf, const void *e_src,
                            const void *r, void *e_dst, const float *u, float *u_out, cudaStream_t st) {
    if (A.ov_index) {
#define CALL(KK) sweep_ku<KK, HT, UN, true>(last, project, A, cf, e_src, r, e_dst, u, u_out, st)
        PDCA_DISPATCH_K(K, CALL)
#undef CALL
    }
#define CALL(KK) sweep_ku<KK, HT, UN, false>(last, project, A, cf, e_src, r, e_dst, u, u_out, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

}  // namespace

// Defines the two entry points of one instance set.
#define PDCA_MIXED_SET(NAME, UNV, HTV)                                                                           \
    cudaError_t NAME##_residual(int K, bool last, bool project, const SellView &A, const Coeffs &cf,             \
                                const float *u, void *r, void *e, float *u_out, cudaStream_t st) {              \
        return mixed_residual_set<UNV, HTV>(K, last, project, A, cf, u, r, e, u_out, st);                        \
    }                                                                                                            \
    cudaError_t NAME##_sweep(int K, bool last, bool project, const SellView &A, const Coeffs &cf,                \
                             const void *e_src, const void *r, void *e_dst, const float *u, float *u_out,        \
                             cudaStream_t st) {                                                                  \
        return mixed_sweep_set<UNV, HTV>(K, last, project, A, cf, e_src, r, e_dst, u, u_out, st);                \
    }

}  // namespace pdca
