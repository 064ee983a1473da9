// Overflow pre-pass: the sums of the entries that rows longer than the split
// length keep outside the sliced ELL.
//
// A row-per-lane sweep waits for its longest row, so a graph with hub rows
// (the k-NN graphs of high-dimensional point clouds have rows of several
// hundred entries) is as slow as its longest row.  Past the split length the
// entries are kept in a CSR of their own, and this pre-pass reduces each
// such row with one warp: the lanes take consecutive entries (coalesced
// column and weight loads, four gathers in flight per lane), then a fixed
// butterfly of shuffles adds the 32 partial sums.  The result, K floats per
// row, is added by the sweep-like kernel that runs next (add_overflow), after
// the row's sliced entries.  Fixed assignment and fixed summation order:
// the same bits on every run.
#include "device_common.cuh"

namespace pdca {
namespace {

using namespace dev;

constexpr int kOvThreads = 256;
constexpr int kOvWarps = kOvThreads / 32;

__device__ __forceinline__ float ov_weight(const OverflowView &O, int wkind, int64_t e) {
    if (wkind == kOvW16) return __bfloat162float(O.wb[e]);
    return __ldg(O.w + e);
}

// acc[0..K) += sum over the entries of overflow row q; whole warp, lane sums
// reduced by the fixed butterfly (every lane ends with the same values).
template <int K, class XT>
__device__ __forceinline__ void ov_row_sum(const OverflowView &O, int wkind, int32_t q, const XT *__restrict__ x,
                                           float (&acc)[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const int64_t e0 = O.rp[q], e1 = O.rp[q + 1];
    int64_t e = e0 + lane;
    for (; e + 96 < e1; e += 128) {   // four gathers in flight per lane
        int32_t c[4];
        float wv[4], rr[4][K];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            c[m] = __ldg(O.col + e + 32 * m);
            wv[m] = ov_weight(O, wkind, e + 32 * m);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) load_row_t<K, XT>(x + (size_t)c[m] * K, rr[m]);
#pragma unroll
        for (int m = 0; m < 4; ++m) fma_row<K>(acc, wv[m], rr[m]);
    }
    for (; e < e1; e += 32) {
        const int32_t ca = __ldg(O.col + e);
        const float wa = ov_weight(O, wkind, e);
        float ra[K];
        load_row_t<K, XT>(x + (size_t)ca * K, ra);
        fma_row<K>(acc, wa, ra);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = warp_sum_f(acc[k]);
}

template <int K, class XT>
__device__ __forceinline__ void ov_row(const OverflowView &O, int wkind, int32_t q, const XT *__restrict__ x,
                                       float *__restrict__ out) {
    float acc[K];
    ov_row_sum<K, XT>(O, wkind, q, x, acc);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) out[(size_t)q * K + k] = acc[k];
    }
}

template <int K, class XT>
__global__ void __launch_bounds__(kOvThreads)
overflow_kernel(const OverflowView O, int wkind, const XT *__restrict__ x, float *__restrict__ out) {
    for (int32_t q = blockIdx.x * kOvWarps + (threadIdx.x >> 5); q < O.n_rows; q += gridDim.x * kOvWarps)
        ov_row<K, XT>(O, wkind, q, x, out);
}

// Batched form: warp -> member by binary search over q_begin (member-uniform
// per warp, so the row-type branch does not diverge).
template <int K>
__global__ void __launch_bounds__(kOvThreads) batch_overflow_kernel(const __grid_constant__ BatchOvTable t) {
    for (int32_t gq = blockIdx.x * kOvWarps + (threadIdx.x >> 5); gq < t.total_rows; gq += gridDim.x * kOvWarps) {
        int lo = 0, hi = t.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t.d[mid].q_begin <= gq) lo = mid;
            else hi = mid - 1;
        }
        const BatchOvDesc &d = t.d[lo];
        const int32_t q = gq - d.q_begin;
        if (d.xkind == kOvXHalf) ov_row<K, __half>(d.O, d.wkind, q, static_cast<const __half *>(d.x), d.acc);
        else if (d.xkind == kOvXBf16)
            ov_row<K, __nv_bfloat16>(d.O, d.wkind, q, static_cast<const __nv_bfloat16 *>(d.x), d.acc);
        else ov_row<K, float>(d.O, d.wkind, q, static_cast<const float *>(d.x), d.acc);
    }
}

int ov_blocks(int32_t rows) {
    const int b = (rows + kOvWarps - 1) / kOvWarps;
    return b < 8 * kSmCount ? b : 8 * kSmCount;
}

template <int K>
cudaError_t overflow_k(int wkind, int xkind, const OverflowView &O, const void *x, float *acc, cudaStream_t st) {
    const int blocks = ov_blocks(O.n_rows);
    if (xkind == kOvXHalf)
        overflow_kernel<K, __half><<<blocks, kOvThreads, 0, st>>>(O, wkind, static_cast<const __half *>(x), acc);
    else if (xkind == kOvXBf16)
        overflow_kernel<K, __nv_bfloat16><<<blocks, kOvThreads, 0, st>>>(O, wkind,
                                                                       static_cast<const __nv_bfloat16 *>(x), acc);
    else
        overflow_kernel<K, float><<<blocks, kOvThreads, 0, st>>>(O, wkind, static_cast<const float *>(x), acc);
    return cudaGetLastError();
}

template <int K>
cudaError_t batch_overflow_k(const BatchOvTable &t, cudaStream_t st) {
    batch_overflow_kernel<K><<<ov_blocks(t.total_rows), kOvThreads, 0, st>>>(t);
    return cudaGetLastError();
}

}  // namespace

#define PDCA_OV_DISPATCH(K, CALL)                                                     \
    switch (K) {                                                                      \
    case 1: return CALL(1); case 2: return CALL(2); case 3: return CALL(3);           \
    case 4: return CALL(4); case 5: return CALL(5); case 6: return CALL(6);           \
    case 7: return CALL(7); case 8: return CALL(8); case 9: return CALL(9);           \
    case 10: return CALL(10); case 11: return CALL(11); case 12: return CALL(12);     \
    case 13: return CALL(13); case 14: return CALL(14); case 15: return CALL(15);     \
    case 16: return CALL(16);                                                         \
    default: return cudaErrorInvalidValue;                                            \
    }

cudaError_t launch_overflow(int K, int wkind, int xkind, const OverflowView &O, const void *x, float *acc,
                            cudaStream_t st) {
    if (O.n_rows <= 0) return cudaSuccess;
    count_launches(1);
#define CALL(KK) overflow_k<KK>(wkind, xkind, O, x, acc, st)
    PDCA_OV_DISPATCH(K, CALL)
#undef CALL
}

cudaError_t launch_batch_overflow(int K, const BatchOvTable &t, cudaStream_t st) {
    if (t.n <= 0 || t.total_rows <= 0) return cudaSuccess;
    count_launches(1);
#define CALL(KK) batch_overflow_k<KK>(t, st)
    PDCA_OV_DISPATCH(K, CALL)
#undef CALL
}

}  // namespace pdca
