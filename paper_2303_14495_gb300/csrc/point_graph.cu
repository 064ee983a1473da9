// k-NN graph of a point cloud on the GPU (Sec. 2.3 for clustering: the
// k-nearest-neighbour indicator N_c times the Gaussian kernel with the
// local-scaling bandwidth of Zelnik-Manor and Perona), symmetrised by union:
//   w_ij = exp(-|x_i - x_j|^2 / (sigma_i sigma_j)),  sigma_i = distance of i
//   to its m-th nearest neighbour.
//
// Query rows go in tiles of T rows:
//   (the points are first centred on their mean, which leaves distances
//   unchanged and keeps the screening product accurate for data far from
//   the origin)
//   dist_mma_kernel   the product of the query tile with all points on the
//                     tensor cores (mma.sync m16n8k16, every FP32 value split
//                     into BF16 hi + lo, three products per pair, FP32
//                     accumulation; 128 x 128 outputs per block), turned into
//                     approximate squared distances |x|^2 + |y|^2 - 2 x.y in
//                     the epilogue;
//   candidate_fast_kernel  one warp per query: each lane keeps its 16
//                     smallest in registers and a c-round warp merge gives the
//                     query's c candidates (c = 3k + 8, a margin for the
//                     rounding of the screen); a query where a lane may have
//                     dropped one of them is flagged, and candidate_kernel
//                     (c kept per lane) does it again;
//   rerank_kernel     exact FP64 distances of the candidates (sums of squared
//                     coordinate differences, a warp per distance, the same
//                     bits from either end),
//                     the k smallest (d2, index) kept (ties to the lower index).
// Then sigma, and the union: in-degree counts, capacity offsets (scan), out-
// and in-edges placed, each row sorted by column and deduplicated, final
// offsets (scan) and the compacted CSR with the weights.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cmath>

#include "pdca_internal.cuh"
#include "scan.cuh"

namespace pdca {
namespace {

constexpr int kPgMaxK = 32;
constexpr int kPgMaxC = 3 * kPgMaxK + 8;
constexpr int kTB = 128;   // product tile: 128 x 128 outputs

// column means (FP64): block b sums the rows of chunk b for every coordinate
// (threads over coordinates, coalesced), then one thread per coordinate adds
// the chunk sums in chunk order
constexpr int kMeanChunks = 256;
__global__ void __launch_bounds__(256)
colsum_kernel(const float *__restrict__ X, int64_t n, int D, double *__restrict__ part) {
    const int64_t per = (n + kMeanChunks - 1) / kMeanChunks;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
    for (int d = threadIdx.x; d < D; d += 256) {
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += (double)__ldg(X + i * D + d);
        part[(int64_t)blockIdx.x * D + d] = s;
    }
}

__global__ void __launch_bounds__(256)
colmean_kernel(const double *__restrict__ part, int64_t n, int D, double *__restrict__ mean) {
    const int d = blockIdx.x * 256 + threadIdx.x;
    if (d >= D) return;
    double s = 0.0;
    for (int b = 0; b < kMeanChunks; ++b) s += part[(int64_t)b * D + d];
    mean[d] = s / (double)n;
}

// Xc = X - mean: distances are unchanged, and the screening product
// |x|^2 + |y|^2 - 2 x.y no longer loses the distances to large norms
__global__ void __launch_bounds__(256)
center_kernel(const float *__restrict__ X, int64_t n, int D, const double *__restrict__ mean, float *__restrict__ Xc) {
    const int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (q >= n * D) return;
    Xc[q] = (float)((double)X[q] - mean[q % D]);
}

__global__ void __launch_bounds__(256)
sqnorm_kernel(const float *__restrict__ X, int64_t n, int D, float *__restrict__ sq) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int d = 0; d < D; ++d) {
        const float v = __ldg(X + i * D + d);
        s = fmaf(v, v, s);
    }
    sq[i] = s;
}

// The screening product on the tensor cores (mma.sync, BF16 in, FP32
// accumulate), with each FP32 coordinate split into two BF16 parts,
// x = hi + lo + e (|e| <= 2^-17 |x|):  x.y ~ hi.hi' + hi.lo' + lo.hi'  (the
// lo.lo' term, <= 2^-16 |x||y|, is dropped).  Small integers (|x| < 256)
// split exactly, so lattice ties stay exact.
__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo_k, __nv_bfloat16 hi_k) {
    return (uint32_t)__bfloat16_as_ushort(lo_k) | ((uint32_t)__bfloat16_as_ushort(hi_k) << 16);
}

__device__ __forceinline__ void mma_bf16_16x8x16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kMK = 32;            // k-slab
constexpr int kMW = (kMK + 8) / 2; // shared row stride in 32-bit words (conflict-free fragment loads)

// out[t * n + j] = sq[q0 + t] + sq[j] - 2 x_{q0+t} . x_j  (+inf for j == q0 + t).
// Block: 128 query rows x 128 points, 8 warps of 64 x 32 outputs (4 x 4
// m16n8 tiles each).  A 32-wide k-slab of both operands is split into BF16
// hi/lo parts in shared memory (rows of kMW words: k pairs packed low k
// first, as the fragments want them); the next slab's global loads are
// issued before the current slab's products.  Fragment layouts are those of
// mma.m16n8k16 (A row-major, B column-major, i.e. both as [row][k]).
__global__ void __launch_bounds__(256)
dist_mma_kernel(const float *__restrict__ X, int64_t n, int D, int64_t q0, int T, const float *__restrict__ sq,
                float *__restrict__ out) {
    __shared__ uint32_t sm[4][kTB * kMW];   // A hi, A lo, B hi, B lo
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t row0 = (int64_t)blockIdx.y * kTB, col0 = (int64_t)blockIdx.x * kTB;
    // loader: value f = tid + 256 i of the 128 x 32 slab (a warp reads one
    // row's 32 consecutive floats); as k pairs: thread pairs (2p, 2p+1)
    float ra[16], rb[16];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int f = tid + 256 * i, r = f / kMK, kk = k0 + f % kMK;
            const int64_t qa = row0 + r, pb = col0 + r;
            ra[i] = (qa < T && kk < D) ? __ldg(X + (q0 + qa) * D + kk) : 0.0f;
            rb[i] = (pb < n && kk < D) ? __ldg(X + pb * D + kk) : 0.0f;
        }
    };
    float acc[4][4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[m][q][e] = 0.0f;
    fetch(0);
    for (int k0 = 0; k0 < D; k0 += kMK) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            // lanes 2p and 2p+1 hold k = 2p, 2p+1 of the same row: pair them
            const float xa = ra[i], xb = rb[i];
            const __nv_bfloat16 ah = __float2bfloat16_rn(xa), bh = __float2bfloat16_rn(xb);
            const __nv_bfloat16 al = __float2bfloat16_rn(xa - __bfloat162float(ah));
            const __nv_bfloat16 bl = __float2bfloat16_rn(xb - __bfloat162float(bh));
            const unsigned short o_ah = __shfl_xor_sync(0xffffffffu, __bfloat16_as_ushort(ah), 1);
            const unsigned short o_al = __shfl_xor_sync(0xffffffffu, __bfloat16_as_ushort(al), 1);
            const unsigned short o_bh = __shfl_xor_sync(0xffffffffu, __bfloat16_as_ushort(bh), 1);
            const unsigned short o_bl = __shfl_xor_sync(0xffffffffu, __bfloat16_as_ushort(bl), 1);
            if ((lane & 1) == 0) {
                const int f = tid + 256 * i, r = f / kMK, w = (f % kMK) / 2;
                sm[0][r * kMW + w] = pack_bf16x2(ah, __ushort_as_bfloat16(o_ah));
                sm[1][r * kMW + w] = pack_bf16x2(al, __ushort_as_bfloat16(o_al));
                sm[2][r * kMW + w] = pack_bf16x2(bh, __ushort_as_bfloat16(o_bh));
                sm[3][r * kMW + w] = pack_bf16x2(bl, __ushort_as_bfloat16(o_bl));
            }
        }
        __syncthreads();
        if (k0 + kMK < D) fetch(k0 + kMK);
#pragma unroll
        for (int s = 0; s < kMK / 16; ++s) {
            const int p = s * 8 + t4;
            uint32_t ah[4][4], al[4][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int r = wm * 64 + m * 16 + g;
                ah[m][0] = sm[0][r * kMW + p];
                ah[m][1] = sm[0][(r + 8) * kMW + p];
                ah[m][2] = sm[0][r * kMW + p + 4];
                ah[m][3] = sm[0][(r + 8) * kMW + p + 4];
                al[m][0] = sm[1][r * kMW + p];
                al[m][1] = sm[1][(r + 8) * kMW + p];
                al[m][2] = sm[1][r * kMW + p + 4];
                al[m][3] = sm[1][(r + 8) * kMW + p + 4];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = wn * 32 + q * 8 + g;
                bh[q][0] = sm[2][r * kMW + p];
                bh[q][1] = sm[2][r * kMW + p + 4];
                bl[q][0] = sm[3][r * kMW + p];
                bl[q][1] = sm[3][r * kMW + p + 4];
            }
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    mma_bf16_16x8x16(acc[m][q], ah[m], bh[q]);
                    mma_bf16_16x8x16(acc[m][q], ah[m], bl[q]);
                    mma_bf16_16x8x16(acc[m][q], al[m], bh[q]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t t = row0 + wm * 64 + m * 16 + g + (e >= 2 ? 8 : 0);
                const int64_t j = col0 + wn * 32 + q * 8 + t4 * 2 + (e & 1);
                if (t >= T || j >= n) continue;
                out[t * n + j] = (q0 + t == j) ? INFINITY : sq[q0 + t] + sq[j] - 2.0f * acc[m][q][e];
            }
}

// One warp per query row of the tile: the c smallest approximate distances
// (ties in order of the lanes' scans; the exact re-rank decides afterwards).
// Lane l scans j = l, l + 32, ...  The fast form keeps each lane's 16
// smallest in registers and merges them; the merge is exact unless some lane
// that dropped values had its 16th value at or below the merged c-th, and
// those rows (about 1 in 10^4 for c = 38) are flagged and done again by
// candidate_kernel, which keeps c per lane.
constexpr int kLaneKeep = 16;
__global__ void __launch_bounds__(256)
candidate_fast_kernel(const float *__restrict__ dist, int64_t n, int T, int c, int32_t *__restrict__ cand,
                      int32_t *__restrict__ redo) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= T) return;
    const int lane = threadIdx.x & 31;
    float bd[kLaneKeep];
    int32_t bj[kLaneKeep];
#pragma unroll
    for (int i = 0; i < kLaneKeep; ++i) {
        bd[i] = INFINITY;
        bj[i] = 0x7fffffff;
    }
    int64_t seen = 0;   // values this lane found below +inf
    const float *row = dist + (int64_t)t * n;
    auto consider = [&](float d, int64_t j) {
        if (!(d < bd[kLaneKeep - 1])) {
            seen += d < INFINITY ? 1 : 0;
            return;
        }
        ++seen;
        bd[kLaneKeep - 1] = d;
        bj[kLaneKeep - 1] = (int32_t)j;
#pragma unroll
        for (int i = kLaneKeep - 1; i > 0; --i) {
            if (bd[i] < bd[i - 1]) {
                const float x = bd[i];
                bd[i] = bd[i - 1];
                bd[i - 1] = x;
                const int32_t y = bj[i];
                bj[i] = bj[i - 1];
                bj[i - 1] = y;
            }
        }
    };
    int64_t j = lane;
    for (; j + 7 * 32 < n; j += 8 * 32) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(row + j + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) consider(v[u], j + 32 * u);
    }
    for (; j < n; j += 32) consider(row[j], j);
    const bool dropped = seen > kLaneKeep;
    const float last = bd[kLaneKeep - 1];
    float cth = INFINITY;
    for (int q = 0; q < c; ++q) {
        const float v = bd[0];
        const int32_t id = bj[0];
        float bv = v;
        int32_t bid = id;
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int32_t oid = __shfl_xor_sync(0xffffffffu, bid, o);
            if (ov < bv || (ov == bv && oid < bid)) {
                bv = ov;
                bid = oid;
            }
        }
        if (bid == id && id != 0x7fffffff) {   // the winning lane pops its head
#pragma unroll
            for (int i = 0; i + 1 < kLaneKeep; ++i) {
                bd[i] = bd[i + 1];
                bj[i] = bj[i + 1];
            }
            bd[kLaneKeep - 1] = INFINITY;
            bj[kLaneKeep - 1] = 0x7fffffff;
        }
        cth = bv;
        if (lane == 0) cand[(int64_t)t * c + q] = bid == 0x7fffffff ? -1 : bid;
    }
    const bool unsure = __any_sync(0xffffffffu, dropped && last <= cth);
    if (lane == 0) redo[t] = unsure ? 1 : 0;
}

__global__ void __launch_bounds__(256)
candidate_kernel(const float *__restrict__ dist, int64_t n, int T, int c, int32_t *__restrict__ cand,
                 const int32_t *__restrict__ redo) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= T) return;
    if (redo && !redo[t]) return;
    const int lane = threadIdx.x & 31;
    float bd[kPgMaxC];
    int32_t bj[kPgMaxC];
    int cnt = 0;
    float thr = INFINITY;   // the lane's current c-th smallest (kept in a register)
    const float *row = dist + (int64_t)t * n;
    auto consider = [&](float d, int64_t j) {
        if (!(d < thr) && cnt == c) return;
        int pos = cnt < c ? cnt : c - 1;
        while (pos > 0 && bd[pos - 1] > d) {
            bd[pos] = bd[pos - 1];
            bj[pos] = bj[pos - 1];
            --pos;
        }
        bd[pos] = d;
        bj[pos] = (int32_t)j;
        if (cnt < c) ++cnt;
        if (cnt == c) thr = bd[c - 1];
    };
    int64_t j = lane;
    // eight loads in flight per lane, then the (mostly rejecting) comparisons
    for (; j + 7 * 32 < n; j += 8 * 32) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(row + j + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) consider(v[u], j + 32 * u);
    }
    for (; j < n; j += 32) consider(row[j], j);
    // merge: c rounds, each takes the smallest head among the lanes
    int head = 0;
    for (int q = 0; q < c; ++q) {
        float v = head < cnt ? bd[head] : INFINITY;
        int32_t id = head < cnt ? bj[head] : 0x7fffffff;
        float bv = v;
        int32_t bid = id;
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int32_t oid = __shfl_xor_sync(0xffffffffu, bid, o);
            if (ov < bv || (ov == bv && oid < bid)) {
                bv = ov;
                bid = oid;
            }
        }
        if (bid == id && head < cnt) ++head;   // the winning lane advances
        if (lane == 0) cand[(int64_t)t * c + q] = bid == 0x7fffffff ? -1 : bid;
    }
}

// one warp per query: exact FP64 distances of the candidates, k smallest kept
__global__ void __launch_bounds__(256)
rerank_kernel(const float *__restrict__ X, int64_t n, int D, int64_t q0, int T, int c, int k,
              const int32_t *__restrict__ cand, int32_t *__restrict__ nbr, double *__restrict__ nd2) {
    __shared__ double sd[8][kPgMaxC];
    __shared__ int32_t sj[8][kPgMaxC];
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * 8 + wp;
    if (t >= T) return;
    const int64_t i = q0 + t;
    // one candidate at a time, the warp over the coordinates (coalesced):
    // lane l adds d = l, l + 32, ... in order, then lane 0's fixed tree adds
    // the lanes; each term depends only on |x_i[d] - x_j[d]|, so the sum has
    // the same bits for (i, j) and (j, i)
    // (four candidates at a time: four independent FP64 chains per lane)
    constexpr int kRr = 4;
    for (int q0 = 0; q0 < c; q0 += kRr) {
        int32_t j[kRr];
        double part[kRr];
#pragma unroll
        for (int u = 0; u < kRr; ++u) {
            j[u] = q0 + u < c ? cand[(int64_t)t * c + q0 + u] : -1;
            part[u] = 0.0;
        }
        for (int d = lane; d < D; d += 32) {
            const double xi = (double)__ldg(X + i * D + d);
#pragma unroll
            for (int u = 0; u < kRr; ++u)
                if (j[u] >= 0) {
                    const double diff = xi - (double)__ldg(X + (int64_t)j[u] * D + d);
                    part[u] = __fma_rn(diff, diff, part[u]);   // FP64 is slow here: one op per term
                }
        }
#pragma unroll
        for (int u = 0; u < kRr; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part[u] = __dadd_rn(part[u], __shfl_xor_sync(0xffffffffu, part[u], o));
            const double acc = j[u] >= 0 ? __shfl_sync(0xffffffffu, part[u], 0) : INFINITY;
            if (lane == 0 && q0 + u < c) {
                sd[wp][q0 + u] = acc;
                sj[wp][q0 + u] = j[u] >= 0 ? j[u] : 0x7fffffff;
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        // insertion sort by (d2, index), then the first k
        for (int a = 1; a < c; ++a) {
            const double v = sd[wp][a];
            const int32_t id = sj[wp][a];
            int b = a - 1;
            while (b >= 0 && (sd[wp][b] > v || (sd[wp][b] == v && sj[wp][b] > id))) {
                sd[wp][b + 1] = sd[wp][b];
                sj[wp][b + 1] = sj[wp][b];
                --b;
            }
            sd[wp][b + 1] = v;
            sj[wp][b + 1] = id;
        }
        for (int q = 0; q < k; ++q) {
            nbr[i * k + q] = sj[wp][q];
            nd2[i * k + q] = sd[wp][q];
        }
    }
}

__global__ void __launch_bounds__(256)
indegree_kernel(int64_t n, int k, int m, const int32_t *__restrict__ nbr, const double *__restrict__ nd2,
                int32_t *__restrict__ cnt, double *__restrict__ sigma, uint32_t *__restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const double s = sqrt(nd2[i * k + m - 1]);
    sigma[i] = s;
    if (!(s > 0.0) || !isfinite(s)) atomicOr(status, 1u);
    for (int q = 0; q < k; ++q) {
        const int32_t j = nbr[i * k + q];
        if (j < 0 || j >= n) {
            atomicOr(status, 2u);
            continue;
        }
        atomicAdd(cnt + j, 1);
    }
}

// out-edges at off[i] + q, in-edges after them (positions by atomic counter)
__global__ void __launch_bounds__(256)
place_kernel(int64_t n, int k, const int32_t *__restrict__ nbr, const double *__restrict__ nd2,
             const int64_t *__restrict__ off, int32_t *__restrict__ fillc, int32_t *__restrict__ ecol,
             double *__restrict__ ed2) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    for (int q = 0; q < k; ++q) {
        const int32_t j = nbr[i * k + q];
        if (j < 0 || j >= n) continue;
        const double d = nd2[i * k + q];
        ecol[off[i] + q] = j;
        ed2[off[i] + q] = d;
        const int64_t at = off[j] + k + atomicAdd(fillc + j, 1);
        ecol[at] = (int32_t)i;
        ed2[at] = d;
    }
}

// sort each row by column (equal columns carry equal distances) and drop repeats
__global__ void __launch_bounds__(256)
row_sort_kernel(int64_t n, const int64_t *__restrict__ off, int32_t *__restrict__ ecol, double *__restrict__ ed2,
                int32_t *__restrict__ len) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off[i], e = off[i + 1];
    for (int64_t a = b + 1; a < e; ++a) {
        const int32_t cj = ecol[a];
        const double dv = ed2[a];
        int64_t p = a - 1;
        while (p >= b && ecol[p] > cj) {
            ecol[p + 1] = ecol[p];
            ed2[p + 1] = ed2[p];
            --p;
        }
        ecol[p + 1] = cj;
        ed2[p + 1] = dv;
    }
    int64_t o = b;
    for (int64_t a = b; a < e; ++a)
        if (a == b || ecol[a] != ecol[o - 1]) {
            ecol[o] = ecol[a];
            ed2[o] = ed2[a];
            ++o;
        }
    len[i] = (int32_t)(o - b);
}

__global__ void __launch_bounds__(256)
compact_kernel(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ ecol,
               const double *__restrict__ ed2, const double *__restrict__ sigma, const int64_t *__restrict__ row_ptr,
               int32_t *__restrict__ col, float *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off[i], o = row_ptr[i], L = row_ptr[i + 1] - row_ptr[i];
    for (int64_t q = 0; q < L; ++q) {
        const int32_t j = ecol[b + q];
        col[o + q] = j;
        w[o + q] = (float)exp(-ed2[b + q] / (sigma[i] * sigma[j]));
    }
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct PgWs {
    float *sq, *dist, *xc;
    double *mean, *mpart;
    int32_t *redo;
    int32_t *cand, *nbr, *cnt, *fillc, *ecol, *len;
    double *nd2, *sigma, *ed2;
    int64_t *off, *bsum, *total;
    uint32_t *status;
    size_t bytes;
};

int tile_rows(int64_t n) { return (int)std::max<int64_t>(64, std::min<int64_t>(8192, ((int64_t)1 << 28) / n)); }

PgWs pg_ws(int64_t n, int k, int dim, char *base) {
    PgWs s{};
    const int T = tile_rows(n), c = (int)std::min<int64_t>(n - 1, 3 * k + 8);
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = al256(o + std::max<size_t>(b, 1)); return at; };
    const size_t nb = (size_t)((n + kScanBlock - 1) / kScanBlock);
    const size_t cap = (size_t)2 * n * k;
    const size_t o_sq = take(4 * (size_t)n), o_dist = take(4 * (size_t)T * n), o_cand = take(4 * (size_t)T * c);
    const size_t o_nbr = take(4 * (size_t)n * k), o_nd2 = take(8 * (size_t)n * k), o_sig = take(8 * (size_t)n);
    const size_t o_cnt = take(4 * (size_t)n), o_fill = take(4 * (size_t)n), o_len = take(4 * (size_t)n);
    const size_t o_off = take(8 * ((size_t)n + 1)), o_ecol = take(4 * cap), o_ed2 = take(8 * cap);
    const size_t o_bsum = take(8 * nb), o_tot = take(8), o_st = take(4);
    const size_t o_xc = take(4 * (size_t)n * dim), o_mean = take(8 * (size_t)dim);
    const size_t o_mpart = take(8 * (size_t)kMeanChunks * dim), o_redo = take(4 * (size_t)T);
    s.bytes = o;
    if (base) {
        s.sq = reinterpret_cast<float *>(base + o_sq);
        s.dist = reinterpret_cast<float *>(base + o_dist);
        s.cand = reinterpret_cast<int32_t *>(base + o_cand);
        s.nbr = reinterpret_cast<int32_t *>(base + o_nbr);
        s.nd2 = reinterpret_cast<double *>(base + o_nd2);
        s.sigma = reinterpret_cast<double *>(base + o_sig);
        s.cnt = reinterpret_cast<int32_t *>(base + o_cnt);
        s.fillc = reinterpret_cast<int32_t *>(base + o_fill);
        s.len = reinterpret_cast<int32_t *>(base + o_len);
        s.off = reinterpret_cast<int64_t *>(base + o_off);
        s.ecol = reinterpret_cast<int32_t *>(base + o_ecol);
        s.ed2 = reinterpret_cast<double *>(base + o_ed2);
        s.bsum = reinterpret_cast<int64_t *>(base + o_bsum);
        s.total = reinterpret_cast<int64_t *>(base + o_tot);
        s.status = reinterpret_cast<uint32_t *>(base + o_st);
        s.xc = reinterpret_cast<float *>(base + o_xc);
        s.mean = reinterpret_cast<double *>(base + o_mean);
        s.mpart = reinterpret_cast<double *>(base + o_mpart);
        s.redo = reinterpret_cast<int32_t *>(base + o_redo);
    }
    return s;
}

__global__ void fill_i32_kernel(int64_t n, int32_t v, int32_t *__restrict__ p) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n) p[i] = v;
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace pdca

using namespace pdca;

extern "C" pdca_status pdca_point_graph_workspace_size(int64_t n, int32_t dim, int32_t k, size_t *bytes) {
    if (!bytes || n < 2 || n > 0x7fffffffLL || dim < 1 || k < 1 || k > kPgMaxK || k > n - 1)
        return PDCA_ERR_INVALID_ARG;
    *bytes = pg_ws(n, k, dim, nullptr).bytes;
    return PDCA_OK;
}

extern "C" pdca_status pdca_point_graph(const float *X, int64_t n, int32_t dim, int32_t k, int32_t scale_nn,
                                        void *workspace, size_t ws_bytes, int64_t *row_ptr, int32_t *col, float *w,
                                        int64_t col_capacity, int64_t *nnz, void *stream) {
    if (!X || !workspace || !row_ptr || !col || !w || !nnz) return PDCA_ERR_INVALID_ARG;
    if (n < 2 || n > 0x7fffffffLL || dim < 1 || k < 1 || k > kPgMaxK || k > n - 1 || scale_nn < 1 || scale_nn > k)
        return PDCA_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return PDCA_ERR_INVALID_ARG;
    if (!dev_ptr(X) || !dev_ptr(workspace) || !dev_ptr(row_ptr) || !dev_ptr(col) || !dev_ptr(w))
        return PDCA_ERR_INVALID_ARG;
    const PgWs s = pg_ws(n, k, dim, static_cast<char *>(workspace));
    if (ws_bytes < s.bytes) return PDCA_ERR_OOM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int T = tile_rows(n), c = (int)std::min<int64_t>(n - 1, 3 * k + 8);
    const unsigned nblk = (unsigned)((n + 255) / 256);
    count_launches(4);
    colsum_kernel<<<kMeanChunks, 256, 0, st>>>(X, n, dim, s.mpart);
    colmean_kernel<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(s.mpart, n, dim, s.mean);
    center_kernel<<<(unsigned)((n * dim + 255) / 256), 256, 0, st>>>(X, n, dim, s.mean, s.xc);
    sqnorm_kernel<<<nblk, 256, 0, st>>>(s.xc, n, dim, s.sq);
    for (int64_t q0 = 0; q0 < n; q0 += T) {
        const int rows = (int)std::min<int64_t>(T, n - q0);
        const dim3 g((unsigned)((n + kTB - 1) / kTB), (unsigned)((rows + kTB - 1) / kTB));
        count_launches(4);
        dist_mma_kernel<<<g, 256, 0, st>>>(s.xc, n, dim, q0, rows, s.sq, s.dist);
        candidate_fast_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(s.dist, n, rows, c, s.cand, s.redo);
        candidate_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(s.dist, n, rows, c, s.cand, s.redo);
        rerank_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(X, n, dim, q0, rows, c, k, s.cand, s.nbr, s.nd2);
    }
    count_launches(5);
    fill_i32_kernel<<<nblk, 256, 0, st>>>(n, k, s.cnt);
    fill_i32_kernel<<<nblk, 256, 0, st>>>(n, 0, s.fillc);
    if (cudaMemsetAsync(s.status, 0, 4, st) != cudaSuccess) return PDCA_ERR_CUDA;
    indegree_kernel<<<nblk, 256, 0, st>>>(n, k, scale_nn, s.nbr, s.nd2, s.cnt, s.sigma, s.status);
    exclusive_scan(n, s.cnt, s.off, s.bsum, s.total, st);
    place_kernel<<<nblk, 256, 0, st>>>(n, k, s.nbr, s.nd2, s.off, s.fillc, s.ecol, s.ed2);
    row_sort_kernel<<<nblk, 256, 0, st>>>(n, s.off, s.ecol, s.ed2, s.len);
    exclusive_scan(n, s.len, row_ptr, s.bsum, s.total, st);
    int64_t tot = 0;
    uint32_t status = 0;
    if (cudaMemcpyAsync(&tot, s.total, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&status, s.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PDCA_ERR_CUDA;
    if (status & 2u) return PDCA_ERR_CUDA;        // never expected: a candidate index out of range
    if (status & 1u) return PDCA_ERR_BAD_GRAPH;   // sigma_i = 0: the m-th neighbour coincides with i
    *nnz = tot;
    if (tot > col_capacity) return PDCA_ERR_OOM;
    count_launches(1);
    compact_kernel<<<nblk, 256, 0, st>>>(n, s.off, s.ecol, s.ed2, s.sigma, row_ptr, col, w);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return PDCA_ERR_CUDA;
    return PDCA_OK;
}
