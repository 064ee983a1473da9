// Batched pass: many problems of the same K advanced by one pass (FP32 sweep,
// mixed residual or mixed correction sweep) in a single launch.  The table of
// per-problem descriptors is a __grid_constant__ kernel parameter, so a launch
// needs no device-side table and no copy.  Each warp handles one slice of one
// problem with exactly the device code of the single-problem kernels, so a
// problem's iterates are bit-identical alone and in a batch.
#include "device_common.cuh"

static_assert(sizeof(pdca::BatchTable) <= 32000, "batch table exceeds the kernel parameter space");

namespace pdca {
namespace {

using namespace dev;

template <int K, class HT>
__device__ __forceinline__ void mixed_pass(const BatchDesc &d, int slice, int lane) {
    if (d.kind == kPassMixedResidual) {
        const float *u = static_cast<const float *>(d.src);
        HT *r = static_cast<HT *>(d.dst);
        HT *e = static_cast<HT *>(d.dst2);
        if (!d.last) mixed_residual_slice<K, HT, false, false>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
        else if (d.project) mixed_residual_slice<K, HT, true, (K >= 2)>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
        else mixed_residual_slice<K, HT, true, false>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
    } else {
        const HT *es = static_cast<const HT *>(d.src);
        const HT *rr = static_cast<const HT *>(d.aux);
        HT *ed = static_cast<HT *>(d.dst);
        if (!d.last) mixed_sweep_slice<K, HT, false, false>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
        else if (d.project) mixed_sweep_slice<K, HT, true, (K >= 2)>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
        else mixed_sweep_slice<K, HT, true, false>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
    }
}

template <int K>
__global__ void __launch_bounds__(kBlockThreads, 4) batch_pass_kernel(const __grid_constant__ BatchTable t) {
    const int gs = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (gs >= t.total_slices) return;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.d[mid].slice_begin <= gs) lo = mid;
        else hi = mid - 1;
    }
    const BatchDesc &d = t.d[lo];
    const int slice = gs - d.slice_begin;
    const int lane = threadIdx.x & 31;
    if (d.kind == kPassFp32) {
        const float *src = static_cast<const float *>(d.src);
        const float *ut = static_cast<const float *>(d.aux);
        float *dst = static_cast<float *>(d.dst);
        if (d.project) fp32_sweep_slice<K, (K >= 2)>(d.A, d.cf, slice, lane, src, ut, dst);
        else fp32_sweep_slice<K, false>(d.A, d.cf, slice, lane, src, ut, dst);
    } else if (d.bf16u) {
        mixed_pass<K, __nv_bfloat16>(d, slice, lane);
    } else {
        mixed_pass<K, __half>(d, slice, lane);
    }
}

template <int K>
cudaError_t batch_k(const BatchTable &t, cudaStream_t st) {
    const int blocks = (t.total_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    batch_pass_kernel<K><<<blocks, kBlockThreads, 0, st>>>(t);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_pass(int K, const BatchTable &t, cudaStream_t st) {
    if (t.n <= 0 || t.total_slices <= 0) return cudaSuccess;
    count_launches(1);
    switch (K) {
    case 1: return batch_k<1>(t, st); case 2: return batch_k<2>(t, st); case 3: return batch_k<3>(t, st);
    case 4: return batch_k<4>(t, st); case 5: return batch_k<5>(t, st); case 6: return batch_k<6>(t, st);
    case 7: return batch_k<7>(t, st); case 8: return batch_k<8>(t, st); case 9: return batch_k<9>(t, st);
    case 10: return batch_k<10>(t, st); case 11: return batch_k<11>(t, st); case 12: return batch_k<12>(t, st);
    case 13: return batch_k<13>(t, st); case 14: return batch_k<14>(t, st); case 15: return batch_k<15>(t, st);
    case 16: return batch_k<16>(t, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pdca
