// Batched pass kernels, shared by the four translation units that
// instantiate them (L_s or L = D - W, K <= 8 or K > 8), compiled separately
// so the sets build in parallel.  A launch holds problems of one K and one
// Laplacian.
#pragma once
#include "device_common.cuh"

static_assert(sizeof(pdca::BatchTable) <= 32000, "batch table exceeds the kernel parameter space");

namespace pdca {
namespace {

using namespace dev;

template <int K, class HT, bool UN, bool C16>
__device__ __forceinline__ void mixed_pass(const BatchDesc &d, int slice, int lane) {
    if (d.kind == kPassMixedResidual) {
        const float *u = static_cast<const float *>(d.src);
        float *r = static_cast<float *>(d.dst);
        HT *e = static_cast<HT *>(d.dst2);
        if (!d.last) mixed_residual_slice<K, HT, false, false, UN, C16>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
        else if (d.project)
            mixed_residual_slice<K, HT, true, (K >= 2), UN, C16>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
        else mixed_residual_slice<K, HT, true, false, UN, C16>(d.A, d.cf, slice, lane, u, r, e, d.u_out);
    } else {
        const HT *es = static_cast<const HT *>(d.src);
        const float *rr = static_cast<const float *>(d.aux);
        HT *ed = static_cast<HT *>(d.dst);
        if (!d.last)
            mixed_sweep_slice<K, HT, false, false, UN, C16>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
        else if (d.project)
            mixed_sweep_slice<K, HT, true, (K >= 2), UN, C16>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
        else mixed_sweep_slice<K, HT, true, false, UN, C16>(d.A, d.cf, slice, lane, es, rr, ed, d.u, d.u_out);
    }
}

// A problem's pass with the slice body of its Laplacian (UN: L = D - W) and
// of its column format.
template <int K, bool UN, bool C16>
__device__ __forceinline__ void member_pass(const BatchDesc &d, int slice, int lane) {
    if (d.kind == kPassFp32) {
        const float *src = static_cast<const float *>(d.src);
        const float *ut = static_cast<const float *>(d.aux);
        float *dst = static_cast<float *>(d.dst);
        if (d.project) fp32_sweep_slice<K, (K >= 2), UN, C16>(d.A, d.cf, slice, lane, src, ut, dst);
        else fp32_sweep_slice<K, false, UN, C16>(d.A, d.cf, slice, lane, src, ut, dst);
    } else if (d.bf16u) {
        mixed_pass<K, __nv_bfloat16, UN, C16>(d, slice, lane);
    } else {
        mixed_pass<K, __half, UN, C16>(d, slice, lane);
    }
}

// Every member's slices start at a multiple of 8 in the launch's slice range
// (slice_begin), so the 8 warps of a block work on 8 slices of one member,
// inside one format group: the member and the column format are uniform
// over the block.  Warps past the member's last slice return.
template <int K, bool UN>
__global__ void __launch_bounds__(kBlockThreads, 4) batch_pass_kernel(const __grid_constant__ BatchTable t) {
    const int b0 = blockIdx.x * kWarpsPerBlock;
    if (b0 >= t.total_slices) return;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.d[mid].slice_begin <= b0) lo = mid;
        else hi = mid - 1;
    }
    const BatchDesc &d = t.d[lo];
    const int first = b0 - d.slice_begin;
    const int slice = first + (threadIdx.x >> 5);
    if (slice >= d.A.n_slices) return;
    if (block_fmt16(d.A, first)) member_pass<K, UN, true>(d, slice, threadIdx.x & 31);
    else member_pass<K, UN, false>(d, slice, threadIdx.x & 31);
}

template <int K, bool UN>
cudaError_t batch_k(const BatchTable &t, cudaStream_t st) {
    const int blocks = (t.total_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    batch_pass_kernel<K, UN><<<blocks, kBlockThreads, 0, st>>>(t);
    return cudaGetLastError();
}

// K <= 8 (LO) or K > 8: the instance sets compile in separate translation
// units.
template <bool UN, bool LO>
cudaError_t batch_set(int K, const BatchTable &t, cudaStream_t st) {
    if constexpr (LO) {
        switch (K) {
        case 1: return batch_k<1, UN>(t, st); case 2: return batch_k<2, UN>(t, st);
        case 3: return batch_k<3, UN>(t, st); case 4: return batch_k<4, UN>(t, st);
        case 5: return batch_k<5, UN>(t, st); case 6: return batch_k<6, UN>(t, st);
        case 7: return batch_k<7, UN>(t, st); case 8: return batch_k<8, UN>(t, st);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (K) {
        case 9: return batch_k<9, UN>(t, st); case 10: return batch_k<10, UN>(t, st);
        case 11: return batch_k<11, UN>(t, st); case 12: return batch_k<12, UN>(t, st);
        case 13: return batch_k<13, UN>(t, st); case 14: return batch_k<14, UN>(t, st);
        case 15: return batch_k<15, UN>(t, st); case 16: return batch_k<16, UN>(t, st);
        default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace
}  // namespace pdca
