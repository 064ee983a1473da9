// Exclusive prefix sum of n int32 counts into n + 1 int64 offsets on the
// device (out[n] = total), in three launches: per-block scans of kScanBlock
// counts, a one-block scan of the block totals, and the block offsets added.
// Shared by the graph builders.
#pragma once

#include "pdca_internal.cuh"

namespace pdca {
namespace {

constexpr int kScanBlock = 1024;

// exclusive prefix sum of count into out (int64), per block of kScanBlock;
// block totals to bsum
__global__ void __launch_bounds__(kScanBlock)
scan_block_kernel(int64_t n, const int32_t *__restrict__ count, int64_t *__restrict__ out, int64_t *__restrict__ bsum) {
    __shared__ int64_t wsum[kScanBlock / 32];
    const int64_t g = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = g < n ? count[g] : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t s = v;   // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) wsum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        int64_t t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        wsum[lane] = t;   // inclusive scan of warp totals
    }
    __syncthreads();
    const int64_t before = warp > 0 ? wsum[warp - 1] : 0;
    if (g < n) out[g] = before + s - v;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = wsum[31];
}

// exclusive scan of the block totals in place (one block, chunked), total to *total
__global__ void __launch_bounds__(kScanBlock)
scan_totals_kernel(int64_t nb, int64_t *__restrict__ bsum, int64_t *__restrict__ total) {
    __shared__ int64_t wsum[kScanBlock / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t g = base + threadIdx.x;
        const int64_t v = g < nb ? bsum[g] : 0;
        int64_t s = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane == 31) wsum[warp] = s;
        __syncthreads();
        if (warp == 0) {
            int64_t t = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int64_t before = (warp > 0 ? wsum[warp - 1] : 0) + carry;
        if (g < nb) bsum[g] = before + s - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanBlock)
scan_add_kernel(int64_t n, const int64_t *__restrict__ bsum, const int64_t *__restrict__ total,
                int64_t *__restrict__ out) {
    const int64_t g = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (g < n) out[g] += bsum[blockIdx.x];
    if (g == 0) out[n] = *total;
}

// bsum: ceil(n / kScanBlock) int64; total: one int64 (device)
inline void exclusive_scan(int64_t n, const int32_t *count, int64_t *out, int64_t *bsum, int64_t *total,
                           cudaStream_t st) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    count_launches(3);
    scan_block_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(n, count, out, bsum);
    scan_totals_kernel<<<1, kScanBlock, 0, st>>>(nb, bsum, total);
    scan_add_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(n, bsum, total, out);
}

}  // namespace
}  // namespace pdca
