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
//   dist_tile_kernel  FP32 tiled product of the query tile with all points
//                     (128 x 128 outputs per block, 8 x 8 per thread, 8-wide
//                     k-slabs staged in shared memory), turned into approximate squared
//                     distances |x|^2 + |y|^2 - 2 x.y in the epilogue;
//   candidate_kernel  one warp per query: each lane keeps its c smallest, a
//                     c-round warp merge gives the query's c candidates
//                     (c = 3k + 8, a margin for the FP32 rounding);
//   rerank_kernel     exact FP64 distances of the candidates (sums of squared
//                     coordinate differences, the same bits from either end),
//                     the k smallest (d2, index) kept (ties to the lower index).
// Then sigma, and the union: in-degree counts, capacity offsets (scan), out-
// and in-edges placed, each row sorted by column and deduplicated, final
// offsets (scan) and the compacted CSR with the weights.
#include <math.h>

#include <algorithm>
#include <cmath>

#include "pdca_internal.cuh"
#include "scan.cuh"

namespace pdca {
namespace {

constexpr int kPgMaxK = 32;
constexpr int kPgMaxC = 3 * kPgMaxK + 8;
constexpr int kTB = 128, kTK = 8;   // product tile: 128 x 128 outputs, 8-wide slabs

// column means (FP64), one thread per coordinate (coalesced across threads)
__global__ void __launch_bounds__(256)
colmean_kernel(const float *__restrict__ X, int64_t n, int D, double *__restrict__ mean) {
    const int d = blockIdx.x * 256 + threadIdx.x;
    if (d >= D) return;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += (double)__ldg(X + i * D + d);
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

// out[t * n + j] = sq[q0 + t] + sq[j] - 2 x_{q0+t} . x_j  (+inf for j == q0 + t).
// Block: 128 query rows x 128 points, 256 threads with 8 x 8 outputs each;
// 8-wide k-slabs of both operands staged in shared memory (transposed, so
// each thread reads its 8 + 8 operands as float4 pairs), the next slab's
// global loads issued before the current slab's products.
__global__ void __launch_bounds__(256)
dist_tile_kernel(const float *__restrict__ X, int64_t n, int D, int64_t q0, int T, const float *__restrict__ sq,
                 float *__restrict__ out) {
    __shared__ __align__(16) float As[kTK][kTB];
    __shared__ __align__(16) float Bs[kTK][kTB];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t row0 = (int64_t)blockIdx.y * kTB, col0 = (int64_t)blockIdx.x * kTB;   // row: query t, col: point j
    // loader mapping: 128 rows x 8 columns per operand = 1024 values, 4 per thread
    const int lr = threadIdx.x / 2, lc = (threadIdx.x % 2) * 4;
    const int64_t qa = q0 + row0 + lr, pb = col0 + lr;
    const bool arow = row0 + lr < T, brow = pb < n;
    float ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int kk = k0 + lc + u;
            ra[u] = (arow && kk < D) ? __ldg(X + qa * D + kk) : 0.0f;
            rb[u] = (brow && kk < D) ? __ldg(X + pb * D + kk) : 0.0f;
        }
    };
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.0f;
    fetch(0);
    for (int k0 = 0; k0 < D; k0 += kTK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[lc + u][lr] = ra[u];
            Bs[lc + u][lr] = rb[u];
        }
        __syncthreads();
        if (k0 + kTK < D) fetch(k0 + kTK);
#pragma unroll
        for (int c = 0; c < kTK; ++c) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[c][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[c][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[c][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[c][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t t = row0 + (u < 4 ? ty * 4 + u : 64 + ty * 4 + u - 4);
        if (t >= T) continue;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int64_t j = col0 + (v < 4 ? tx * 4 + v : 64 + tx * 4 + v - 4);
            if (j >= n) continue;
            out[t * n + j] = (q0 + t == j) ? INFINITY : sq[q0 + t] + sq[j] - 2.0f * acc[u][v];
        }
    }
}

// one warp per query row of the tile: the c smallest approximate distances
// (ties in order of the lanes' scans; the exact re-rank decides afterwards)
__global__ void __launch_bounds__(256)
candidate_kernel(const float *__restrict__ dist, int64_t n, int T, int c, int32_t *__restrict__ cand) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= T) return;
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
    for (int q = lane; q < c; q += 32) {
        const int32_t j = cand[(int64_t)t * c + q];
        double acc = INFINITY;
        if (j >= 0) {
            acc = 0.0;
            for (int d = 0; d < D; ++d) {
                const double diff = (double)__ldg(X + i * D + d) - (double)__ldg(X + (int64_t)j * D + d);
                acc = __dadd_rn(acc, __dmul_rn(diff, diff));
            }
        }
        sd[wp][q] = acc;
        sj[wp][q] = j >= 0 ? j : 0x7fffffff;
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
    double *mean;
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
    count_launches(3);
    colmean_kernel<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(X, n, dim, s.mean);
    center_kernel<<<(unsigned)((n * dim + 255) / 256), 256, 0, st>>>(X, n, dim, s.mean, s.xc);
    sqnorm_kernel<<<nblk, 256, 0, st>>>(s.xc, n, dim, s.sq);
    for (int64_t q0 = 0; q0 < n; q0 += T) {
        const int rows = (int)std::min<int64_t>(T, n - q0);
        const dim3 g((unsigned)((n + kTB - 1) / kTB), (unsigned)((rows + kTB - 1) / kTB));
        count_launches(3);
        dist_tile_kernel<<<g, 256, 0, st>>>(s.xc, n, dim, q0, rows, s.sq, s.dist);
        candidate_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(s.dist, n, rows, c, s.cand);
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
