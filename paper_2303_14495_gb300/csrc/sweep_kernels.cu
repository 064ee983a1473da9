// Hot-path kernels of the pDCA solver on sm_103a.
//
// sweep_kernel   one preconditioned sweep (eq. general:diag:pre) with the DCA
//                linearisation (eq. bt:ut), the fidelity term and, on the last
//                sweep of an outer step, the simplex projection fused in;
// energy_kernel  F(u) (eqs. gl:functional:graph, functional:GL) and the
//                residual ||b^t - T u^{t+1}||, summed in two-float and FP64;
// power kernels  power method for lambda_max(L_s) (Sec. 3.1);
// labels / permutation kernels for the results.
//
// All of them walk the sliced-ELL operator the same way: one warp per 32-row
// slice, one lane per row, entry j of every lane read as one coalesced warp
// load of column indices (int32 or 16-bit) and one of weights (streamed
// without L1 allocation).  Neighbour rows of u come either from global memory through
// L1/L2 (plain form) or, in the tiled form, from shared memory: a block
// handles a tile of 16 slices and first copies the tile's halo rows (the distinct rows
// its entries reference) into shared memory, so every gather is a shared
// memory load addressed by a 16-bit local column.
#include "device_common.cuh"

#include <math.h>

#include <algorithm>
#include <type_traits>

namespace pdca {
namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// fused sweep
// ---------------------------------------------------------------------------
//   b    = eta Lambda_i y_i + c u_i - (u_i^3 - u_i)/eps          (u = u^t)
//   Tv   = eps (a_i v_i - sum_j w'_ij v_j) + (c + eta Lambda_i) v_i
//   v'_i = v_i + (b - Tv) / g_i,   then projected if PROJECT
// (a_i = 1 and w' = w / sqrt(d_i d_j) for L_s; a_i = d_i and w' = w for L,
// the UN instances).
//
// Latency hiding: the loads that depend on nothing (the row tag and length,
// the own rows of v^s and u^t, the first two entry groups) are issued first,
// and while a lane works on two entry groups the next two are already in
// flight.

// plain form: one warp per slice at a time; a block owns iters x 8
// consecutive slices (32 = one renumbering block of 1024 rows at the usual
// iters = 4) and its warps take them from a shared queue (the same slice
// body as the batched kernel)
// (OV: the problem has split rows whose overflow sums a pre-pass formed)
template <int K, bool PROJECT, bool UN, bool OV>
__global__ void __launch_bounds__(kBlockThreads, PDCA_SWEEP_MIN_BLOCKS)
sweep_kernel(const SellView A, const Coeffs cf, const float *__restrict__ v_src,
             const float *__restrict__ u_t, float *__restrict__ v_dst, int iters) {
    __shared__ int next_slot;
    const int count = kWarpsPerBlock * iters;
    for_block_slices_fmt(A, blockIdx.x * count, count, &next_slot, [&](int slice, auto fmt) {
        fp32_sweep_slice<K, PROJECT, UN, decltype(fmt)::value, OV>(A, cf, slice, threadIdx.x & 31, v_src, u_t,
                                                                   v_dst);
    });
}

// tiled form: one block per tile of 16 slices (one per warp); the halo of
// v^s goes to shared memory while the warps' own loads are in flight
template <int K, bool PROJECT>
__global__ void __launch_bounds__(kTileThreads, PDCA_TILE_MIN_BLOCKS)
sweep_tiled_kernel(const SellView A, const TileView T, const Coeffs cf, const float *__restrict__ v_src,
                   const float *__restrict__ u_t, float *__restrict__ v_dst) {
    extern __shared__ float4 smem_f4[];
    float *hs = reinterpret_cast<float *>(smem_f4);
    const int tile = blockIdx.x;
    const int slice = tile * kTileSlices + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const bool active = slice < A.n_slices;
    SliceRow<K, uint2> s;
    if (active) slice_prologue<K>(A, reinterpret_cast<const uint2 *>(T.lcol), slice, lane, v_src, u_t, s);
    const int64_t h0 = T.halo_off[tile];
    const bool staged = T.halo_off[tile + 1] - h0 <= T.smem_rows;
    if (staged) load_halo<K>(T, tile, v_src, hs);
    __syncthreads();
    if (!active) return;
    float acc[K];
    if (staged) slice_gather<K, kShared>(s, v_src, hs, nullptr, acc);
    else slice_gather<K, kIndirect>(s, v_src, nullptr, T.halo_idx + h0, acc);
    sweep_update<K, PROJECT>(cf, s.info, 1.0f, acc, s.v, s.u, v_dst + (size_t)(slice * kSliceRows + lane) * K);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Per-row contributions (FP32 inside a row, two-float across a warp's rows,
// FP64 across warps and blocks):
//   quad += u_i . (L u)_i  (L_s or L: a_i u_i - sum_j w'_ij u_j),  well += sum_k (u_ik^2 - 1)^2,
//   fid  += Lambda_i sum_k (u_ik - y_ik)^2,
//   rr   += ||b_i - (T u)_i||^2 with b from u_prev, bb += ||b_i||^2.
// b - T u is formed as c (u_prev - u) + eta Lambda (y - u)
//   - (u_prev^3 - u_prev)/eps - eps (L_s u), which avoids the cancellation
// of the two large terms c u_prev and c u.  x and xp are the row's own u and
// u_prev (xp unused without u_prev).
template <int K>
__device__ __forceinline__ void energy_row(const SellView &A, const Coeffs &cf, int r, uint32_t info,
                                           const float (&acc)[K], const float (&x)[K], const float (&xp)[K],
                                           bool has_prev, float (&red)[6]) {
    if (r >= A.n) return;
    const float a = A.self ? A.self[r] : 1.0f;
    const uint32_t tag = info & 0xFFu;
    const bool lab = tag != kTagUnlabelled;
    float q = 0.f, wl = 0.f, fd = 0.f, rr = 0.f, bb = 0.f, nf = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float ls = a * x[k] - acc[k];
        q = fmaf(x[k], ls, q);
        const float s = x[k] * x[k] - 1.0f;
        wl = fmaf(s, s, wl);
        const float y = lab ? prior_of<K>(tag, k) : 0.0f;
        if (lab) fd = fmaf(x[k] - y, x[k] - y, fd);
        if (!isfinite(x[k])) nf += 1.0f;
        if (has_prev) {
            const float up = xp[k];
            const float grad_w = (up * up * up - up) * cf.inv_eps;
            const float b = (lab ? cf.eta * y : 0.0f) + cf.c * up - grad_w;
            const float res = cf.c * (up - x[k]) + (lab ? cf.eta * (y - x[k]) : 0.0f) - grad_w - cf.eps * ls;
            rr = fmaf(res, res, rr);
            bb = fmaf(b, b, bb);
        }
    }
    red[0] += q; red[1] += wl; red[2] += fd; red[3] += rr; red[4] += bb; red[5] += nf;
}

// FP32 weights in both precisions (the mixed forms keep an FP32 copy of the
// operator for their residual passes), so F does not depend on the precision
// of the sweeps beyond the iterate itself.
template <int K>
__global__ void __launch_bounds__(kBlockThreads)
energy_kernel(const SellView A, const Coeffs cf, const float *__restrict__ u,
              const float *__restrict__ u_prev, double *__restrict__ partials, int iters) {
    // slices from the block's queue, sums per slice slot, added in slot order
    // (as in power_spmv_kernel)
    __shared__ int next_slot;
    __shared__ double slot_sum[kWarpsPerBlock * PDCA_SWEEP_MAX_ITERS][6];
    const int count = kWarpsPerBlock * iters;
    const int first = blockIdx.x * count;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < count * 6; i += blockDim.x) slot_sum[i / 6][i % 6] = 0.0;
    for_block_slices_fmt(A, first, count, &next_slot, [&](int slice, auto fmt) {
        constexpr bool C16 = decltype(fmt)::value;
        float red[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int r = slice * kSliceRows + lane;
        const uint32_t info = ld_stream(A.rowinfo + r);
        EntryStream<C16, float> s;
        stream_open(A, slice, lane, s);
        float x[K], xp[K];
        load_row<K>(u + (size_t)r * K, x);
        if (u_prev) load_own_row<K>(u_prev + (size_t)r * K, xp);
        float acc[K];
        stream_gather<K, C16, float, float>(A, s, info, r, u, acc);
        energy_row<K>(A, cf, r, info, acc, x, xp, u_prev != nullptr, red);
        const float red8[8] = {red[0], red[1], red[2], red[3], red[4], red[5], 0.f, 0.f};
        const double t = warp_sum8_df(red8);
        const int q = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if ((lane & 3) == 0 && q < 6) slot_sum[slice - first][q] = t;
    });
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int q = 0; q < count; ++q) t += slot_sum[q][threadIdx.x];
        partials[(size_t)blockIdx.x * kRedSlots + threadIdx.x] = t;
    }
}

template <int K>
__global__ void __launch_bounds__(kTileThreads, PDCA_TILE_MIN_BLOCKS)
energy_tiled_kernel(const SellView A, const TileView T, const Coeffs cf, const float *__restrict__ u,
                    const float *__restrict__ u_prev, double *__restrict__ partials) {
    extern __shared__ float4 smem_f4[];
    float *hs = reinterpret_cast<float *>(smem_f4);
    const int tile = blockIdx.x;
    const int64_t h0 = T.halo_off[tile];
    const bool staged = T.halo_off[tile + 1] - h0 <= T.smem_rows;
    if (staged) load_halo<K>(T, tile, u, hs);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float red[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = threadIdx.x >> 5; s < kTileSlices; s += kTileThreads / 32) {
        const int slice = tile * kTileSlices + s;
        if (slice >= A.n_slices) break;
        const int64_t base = A.slice_off[slice];
        float acc[K];
        tile_row_sum<K>(T, A, base, row_len(A, slice, lane), lane, staged, T.halo_idx + h0, hs, u, acc);
        const int r = slice * kSliceRows + lane;
        float x[K], xp[K];
        load_row<K>(u + (size_t)r * K, x);
        if (u_prev) load_row<K>(u_prev + (size_t)r * K, xp);
        energy_row<K>(A, cf, r, A.rowinfo[r], acc, x, xp, u_prev != nullptr, red);
    }
    block_sum_store<6, kTileThreads / 32>(red, partials + (size_t)blockIdx.x * kRedSlots);
}

// Single block: fixed-order sum of the block partials, then the scalars.
__global__ void __launch_bounds__(256)
energy_finalize_kernel(const double *__restrict__ partials, int n_parts, double eps_d, double eta_d,
                       int has_prev, RedOut *out, double *trace_F, double *trace_r) {
    __shared__ double sm[256][6];
    double t[6] = {0, 0, 0, 0, 0, 0};
    // unrolled so that the loads of several partials are in flight at once
    // (the additions keep their order)
#pragma unroll 8
    for (int i = threadIdx.x; i < n_parts; i += 256)
#pragma unroll
        for (int s = 0; s < 6; ++s) t[s] += partials[(size_t)i * kRedSlots + s];
#pragma unroll
    for (int s = 0; s < 6; ++s) sm[threadIdx.x][s] = t[s];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int s = 0; s < 6; ++s) sm[threadIdx.x][s] += sm[threadIdx.x + h][s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        RedOut o;
        o.quad = sm[0][0]; o.well = sm[0][1]; o.fid = sm[0][2];
        o.rr = sm[0][3]; o.bb = sm[0][4]; o.nonfinite = sm[0][5];
        o.F = 0.5 * eps_d * o.quad + o.well / (4.0 * eps_d) + 0.5 * eta_d * o.fid;
        o.rel_res = has_prev ? (o.bb > 0.0 ? sqrt(o.rr / o.bb) : sqrt(o.rr)) : nan("");
        *out = o;
        if (trace_F) *trace_F = o.F;
        if (trace_r) *trace_r = o.rel_res;
    }
}

// scale <- 1/sqrt(sum y.y); lambda <- sum (s x).y / sum (s x).(s x).
// Fixed-order sum over the partials by the NT threads of one block (a
// 256-thread block: the finalize kernel, or the last block of an SpMV).
template <int NT>
__device__ __forceinline__ void power_reduce(const double *partials, int n_parts, double *scale, double *lambda) {
    __shared__ double sm[NT][3];
    double t[3] = {0, 0, 0};
#pragma unroll 8
    for (int i = threadIdx.x; i < n_parts; i += NT)
#pragma unroll
        for (int s = 0; s < 3; ++s) t[s] += __ldcg(partials + (size_t)i * kRedSlots + s);
#pragma unroll
    for (int s = 0; s < 3; ++s) sm[threadIdx.x][s] = t[s];
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int s = 0; s < 3; ++s) sm[threadIdx.x][s] += sm[threadIdx.x + h][s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double yy = sm[0][0], xy = sm[0][1], xx = sm[0][2];
        *scale = yy > 0.0 ? 1.0 / sqrt(yy) : 0.0;
        *lambda = xx > 0.0 ? xy / xx : 0.0;
    }
}

__global__ void __launch_bounds__(256)
power_finalize_kernel(const double *__restrict__ partials, int n_parts, double *scale, double *lambda) {
    power_reduce<256>(partials, n_parts, scale, lambda);
}

// After the block's partial is stored: the last block to arrive reduces.
template <int NT>
__device__ __forceinline__ void power_last_block(const double *partials, unsigned *ticket, double *scale,
                                                 double *lambda) {
    __shared__ bool last;
    // the partial was stored by threads of warp 0 (block_sum_store): only
    // they fence, the other threads' stores of y need not drain first
    if (threadIdx.x < 32) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    power_reduce<NT>(partials, gridDim.x, scale, lambda);
    if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------------------------
// power method for lambda_max(L_s)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads)
power_init_kernel(const SellView A, const int32_t *__restrict__ perm, float *__restrict__ x,
                  double *__restrict__ partials) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    float red[3] = {0.f, 0.f, 0.f};
    if (slice < A.n_slices) {
        const int r = slice * kSliceRows + lane;
        float xi = 0.0f;
        if (r < A.n) xi = (float)(1.0 + 0.5 * sin((double)perm[r] + 1.0));
        x[r] = xi;
        red[0] = xi * xi;
    }
    block_sum_store<3>(red, partials + (size_t)blockIdx.x * kRedSlots);
}

// y = L (s x) with s = *scale (L_s, or L when A.self holds d_i); partial sums
// of y.y, (s x).y, (s x).(s x).
__device__ __forceinline__ void power_row(const SellView &A, int slice, int lane, float acc, float s,
                                          const float *__restrict__ x, float *__restrict__ y,
                                          float (&red)[3]) {
    const int r = slice * kSliceRows + lane;
    const float xs = s * __ldg(x + r);
    const float yi = (A.self ? __ldg(A.self + r) : 1.0f) * xs - s * acc;
    y[r] = yi;
    if (r < A.n) {
        red[0] = fmaf(yi, yi, red[0]);
        red[1] = fmaf(xs, yi, red[1]);
        red[2] = fmaf(xs, xs, red[2]);
    }
}

// A block owns iters x 8 consecutive slices, taken by its warps from a
// shared queue; each slice's three sums land in a slot of their own, and the
// block adds its slots in slot order, so the partial (and the estimate) does
// not depend on which warp took which slice.  Five blocks per SM (48
// registers, no spills): 127.5 against 131.4 us per SpMV at four (64
// registers); six (40 registers) spill and take 155 us.
__global__ void __launch_bounds__(kBlockThreads, 5)
power_spmv_kernel(const SellView A, const float *__restrict__ x, double *scale, float *__restrict__ y,
                  double *__restrict__ partials, unsigned *ticket, double *lambda, int iters) {
    __shared__ int next_slot;
    __shared__ double slot_sum[kWarpsPerBlock * PDCA_SWEEP_MAX_ITERS][3];
    const int count = kWarpsPerBlock * iters;
    const int first = blockIdx.x * count;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < count * 3; i += blockDim.x) slot_sum[i / 3][i % 3] = 0.0;
    const float s = (float)__ldcg(scale);
    // (the queue's opening barrier orders the zeroing before any slot store)
    for_block_slices_fmt(A, first, count, &next_slot, [&](int slice, auto fmt) {
        float acc[1];
        row_gather<1, float, float, decltype(fmt)::value>(A, slice, lane, x, acc);
        float red[3] = {0.f, 0.f, 0.f};
        power_row(A, slice, lane, acc[0], s, x, y, red);
        // FP32 inside the warp (the sums only normalise the iterate and
        // form the Rayleigh quotient), FP64 across warps and blocks
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float t = warp_sum_f(red[k]);
            if (lane == 0) slot_sum[slice - first][k] = (double)t;
        }
    });
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < count; ++q) t += slot_sum[q][threadIdx.x];
        partials[(size_t)blockIdx.x * kRedSlots + threadIdx.x] = t;
    }
    power_last_block<kBlockThreads>(partials, ticket, scale, lambda);
}

__global__ void __launch_bounds__(kTileThreads, PDCA_TILE_MIN_BLOCKS)
power_spmv_tiled_kernel(const SellView A, const TileView T, const float *__restrict__ x, double *scale,
                        float *__restrict__ y, double *__restrict__ partials, unsigned *ticket, double *lambda) {
    extern __shared__ float4 smem_f4[];
    float *hs = reinterpret_cast<float *>(smem_f4);
    const int tile = blockIdx.x;
    const int64_t h0 = T.halo_off[tile];
    const bool staged = T.halo_off[tile + 1] - h0 <= T.smem_rows;
    if (staged) load_halo<1>(T, tile, x, hs);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float s = (float)__ldcg(scale);
    float red[3] = {0.f, 0.f, 0.f};
    for (int sl = threadIdx.x >> 5; sl < kTileSlices; sl += kTileThreads / 32) {
        const int slice = tile * kTileSlices + sl;
        if (slice >= A.n_slices) break;
        const int64_t base = A.slice_off[slice];
        float acc[1];
        tile_row_sum<1>(T, A, base, row_len(A, slice, lane), lane, staged, T.halo_idx + h0, hs, x, acc);
        power_row(A, slice, lane, acc[0], s, x, y, red);
    }
    block_sum_store<3, kTileThreads / 32>(red, partials + (size_t)blockIdx.x * kRedSlots);
    power_last_block<kTileThreads>(partials, ticket, scale, lambda);
}

// ---------------------------------------------------------------------------
// results
// ---------------------------------------------------------------------------
template <int K>
__global__ void labels_kernel(int32_t n, const float *__restrict__ u, const int32_t *__restrict__ perm,
                              int32_t *__restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[K];
    load_row<K>(u + (size_t)r * K, x);
    int32_t lab;
    if (K == 1) {
        lab = x[0] >= 0.0f ? 1 : 0;
    } else {
        lab = 0;
        float best = x[0];
#pragma unroll
        for (int k = 1; k < K; ++k)
            if (x[k] > best) {
                best = x[k];
                lab = k;
            }
    }
    out[perm[r]] = lab;
}

__global__ void permute_out_kernel(int32_t n, int32_t K, const float *__restrict__ u,
                                   const int32_t *__restrict__ perm, float *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * K) return;
    const int64_t r = q / K;
    const int k = (int)(q - r * K);
    out[(int64_t)perm[r] * K + k] = u[q];
}

__global__ void permute_in_kernel(int32_t n, int32_t n_pad, int32_t K, const float *__restrict__ in,
                                  const int32_t *__restrict__ perm, float *__restrict__ u) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_pad * K) return;
    const int64_t r = q / K;
    const int k = (int)(q - r * K);
    u[q] = r < n ? in[(int64_t)perm[r] * K + k] : (K == 1 ? 0.0f : 2.0f / K - 1.0f);
}

// Dynamic shared memory above the default 48 KiB needs an opt-in per kernel.
template <class Kern>
cudaError_t allow_smem(Kern k, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K>
cudaError_t sweep_k(bool project, const SellView &A, const TileView *T, const Coeffs &cf, const float *v_src,
                    const float *u_t, float *v_dst, cudaStream_t st) {
    constexpr bool P = K >= 2;
    if (T) {
        if (A.self) return cudaErrorInvalidValue;   // the tiled kernels are L_s only
        const size_t sm = tile_smem_bytes(K, T->smem_rows);
        if (project && P) {
            cudaError_t e = allow_smem(sweep_tiled_kernel<K, P>, sm);
            if (e != cudaSuccess) return e;
            sweep_tiled_kernel<K, P><<<T->n_tiles, kTileThreads, sm, st>>>(A, *T, cf, v_src, u_t, v_dst);
        } else {
            cudaError_t e = allow_smem(sweep_tiled_kernel<K, false>, sm);
            if (e != cudaSuccess) return e;
            sweep_tiled_kernel<K, false><<<T->n_tiles, kTileThreads, sm, st>>>(A, *T, cf, v_src, u_t, v_dst);
        }
        return cudaGetLastError();
    }
    // keep at least 4 waves of resident blocks
    const int groups = (A.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int iters = view_iters(A);
    const int blocks = (groups + iters - 1) / iters;
    const bool ov = A.ov_index != nullptr;
#define PDCA_SWEEP(PR, UNL, OVL) \
    sweep_kernel<K, PR, UNL, OVL><<<blocks, kBlockThreads, 0, st>>>(A, cf, v_src, u_t, v_dst, iters)
    if (A.self) {
        if (project && P) { if (ov) PDCA_SWEEP(P, true, true); else PDCA_SWEEP(P, true, false); }
        else { if (ov) PDCA_SWEEP(false, true, true); else PDCA_SWEEP(false, true, false); }
    } else {
        if (project && P) { if (ov) PDCA_SWEEP(P, false, true); else PDCA_SWEEP(P, false, false); }
        else { if (ov) PDCA_SWEEP(false, false, true); else PDCA_SWEEP(false, false, false); }
    }
#undef PDCA_SWEEP
    return cudaGetLastError();
}

template <int K>
cudaError_t energy_k(const SellView &A, const TileView *T, const Coeffs &cf, const float *u, const float *u_prev,
                     double *partials, cudaStream_t st) {
    if (T) {
        const size_t sm = tile_smem_bytes(K, T->smem_rows);
        cudaError_t e = allow_smem(energy_tiled_kernel<K>, sm);
        if (e != cudaSuccess) return e;
        energy_tiled_kernel<K><<<T->n_tiles, kTileThreads, sm, st>>>(A, *T, cf, u, u_prev, partials);
    } else {
        const int iters = view_iters(A);
        energy_kernel<K><<<queue_blocks(A), kBlockThreads, 0, st>>>(A, cf, u, u_prev, partials, iters);
    }
    return cudaGetLastError();
}

template <int K>
cudaError_t labels_k(int32_t n, const float *u, const int32_t *perm, int32_t *out, cudaStream_t st) {
    labels_kernel<K><<<(n + 255) / 256, 256, 0, st>>>(n, u, perm, out);
    return cudaGetLastError();
}

}  // namespace

int energy_blocks(int32_t n_slices) { return (n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock; }

int queue_blocks(const SellView &A) {
    const int per_block = kWarpsPerBlock * view_iters(A);
    return (A.n_slices + per_block - 1) / per_block;
}

int reduce_parts(const SellView &A, const TileView *T) { return T ? T->n_tiles : queue_blocks(A); }


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

cudaError_t launch_sweep(int K, bool project, const SellView &A, const TileView *T, const Coeffs &cf,
                         const float *v_src, const float *u_t, float *v_dst, cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
#define CALL(KK) sweep_k<KK>(project, A, T, cf, v_src, u_t, v_dst, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

cudaError_t launch_energy(int K, const SellView &A, const TileView *T, const Coeffs &cf, const float *u,
                          const float *u_prev, double *partials, cudaStream_t st) {
    count_launches(1);
#define CALL(KK) energy_k<KK>(A, T, cf, u, u_prev, partials, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

cudaError_t launch_energy_finalize(const double *partials, int n_parts, double eps, double eta,
                                   int has_prev, RedOut *out, double *trace_F, double *trace_r,
                                   cudaStream_t st) {
    count_launches(1);
    energy_finalize_kernel<<<1, 256, 0, st>>>(partials, n_parts, eps, eta, has_prev, out, trace_F,
                                              trace_r);
    return cudaGetLastError();
}

cudaError_t launch_power_init(const SellView &A, const int32_t *perm, float *x, double *partials,
                              cudaStream_t st) {
    count_launches(1);
    power_init_kernel<<<energy_blocks(A.n_slices), kBlockThreads, 0, st>>>(A, perm, x, partials);
    return cudaGetLastError();
}

cudaError_t launch_power_spmv(const SellView &A, const TileView *T, const float *x, double *scale, float *y,
                              double *partials, unsigned *ticket, double *lambda, cudaStream_t st) {
    count_launches(1);
    if (T) {
        const size_t sm = tile_smem_bytes(1, T->smem_rows);
        cudaError_t e = allow_smem(power_spmv_tiled_kernel, sm);
        if (e != cudaSuccess) return e;
        power_spmv_tiled_kernel<<<T->n_tiles, kTileThreads, sm, st>>>(A, *T, x, scale, y, partials, ticket,
                                                                        lambda);
    } else {
        const int iters = view_iters(A);
        const int blocks = queue_blocks(A);
        power_spmv_kernel<<<blocks, kBlockThreads, 0, st>>>(A, x, scale, y, partials, ticket, lambda, iters);
    }
    return cudaGetLastError();
}

cudaError_t launch_power_finalize(const double *partials, int n_parts, double *scale, double *lambda,
                                  cudaStream_t st) {
    count_launches(1);
    power_finalize_kernel<<<1, 256, 0, st>>>(partials, n_parts, scale, lambda);
    return cudaGetLastError();
}

cudaError_t launch_labels(int K, int32_t n, const float *u, const int32_t *perm, int32_t *out,
                          cudaStream_t st) {
    count_launches(1);
#define CALL(KK) labels_k<KK>(n, u, perm, out, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

cudaError_t launch_permute_out(int K, int32_t n, const float *u, const int32_t *perm, float *out,
                               cudaStream_t st) {
    const int64_t tot = (int64_t)n * K;
    if (tot == 0) return cudaSuccess;
    count_launches(1);
    permute_out_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, K, u, perm, out);
    return cudaGetLastError();
}

cudaError_t launch_permute_in(int K, int32_t n, int32_t n_pad, const float *in, const int32_t *perm,
                              float *u, cudaStream_t st) {
    const int64_t tot = (int64_t)n_pad * K;
    if (tot == 0) return cudaSuccess;
    count_launches(1);
    permute_in_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, n_pad, K, in, perm, u);
    return cudaGetLastError();
}

}  // namespace pdca
