// Nonlocal image graph on the GPU (Sec. 2.3: w_ij = K(i,j) N(i,j), the
// Gaussian kernel of eq. kij on patch distances times the window indicator),
// restricted to the k window neighbours of smallest patch distance and
// symmetrised by union, the construction the image workloads use.
//
//   image_knn_kernel    one thread per pixel: patch distances to every window
//                       pixel in raster order, FP32 with each square and sum
//                       rounded separately (no FMA) and replicate padding;
//                       keeps the k smallest (d2, index) pairs (ties to the
//                       lower index); stops a candidate's sum as soon as it
//                       reaches the current k-th distance (terms are >= 0,
//                       so such a candidate can never be kept);
//   image_union_kernel  one thread per pixel: window pixel j is a neighbour
//                       iff j is among i's kept or i among j's kept; counts
//                       (first pass) or writes the sorted row with
//                       w = exp(-d2 / sigma^2) (second pass);
//   scan kernels        row offsets from the counts (exclusive prefix sum).
// The distance of a pair is the same bits from either end, so the weights
// are symmetric bit for bit and the CSR passes pdca_create's checks.
#include <math.h>

#include <algorithm>
#include <cmath>

#include "pdca_internal.cuh"
#include "scan.cuh"

namespace pdca {
namespace {

constexpr int kMaxK = 32;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void __launch_bounds__(128)
image_knn_kernel(const float *__restrict__ img, int H, int W, int C, int p, int r, int k, int32_t *__restrict__ nbr,
                 float *__restrict__ dist) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= (int64_t)H * W) return;
    const int y = (int)(i / W), x = (int)(i % W);
    float bd[kMaxK];
    int32_t bj[kMaxK];
    int cnt = 0;
    for (int dy = -r; dy <= r; ++dy) {
        const int yj = y + dy;
        if (yj < 0 || yj >= H) continue;
        for (int dx = -r; dx <= r; ++dx) {
            const int xj = x + dx;
            if (xj < 0 || xj >= W || (dy == 0 && dx == 0)) continue;
            const float worst = cnt == k ? bd[k - 1] : INFINITY;
            float acc = 0.0f;
            bool dead = false;
            for (int oy = -p; oy <= p && !dead; ++oy) {
                const int ya = clampi(y + oy, 0, H - 1), yb = clampi(yj + oy, 0, H - 1);
                for (int ox = -p; ox <= p; ++ox) {
                    const float *pa = img + ((int64_t)ya * W + clampi(x + ox, 0, W - 1)) * C;
                    const float *pb = img + ((int64_t)yb * W + clampi(xj + ox, 0, W - 1)) * C;
                    for (int c = 0; c < C; ++c) {
                        const float t = __fsub_rn(__ldg(pa + c), __ldg(pb + c));
                        acc = __fadd_rn(acc, __fmul_rn(t, t));
                    }
                }
                if (acc >= worst) dead = true;
            }
            if (dead || acc >= worst) continue;
            // insert (acc, j) after every kept entry with distance <= acc
            // (they have lower indices, since candidates come in index order)
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && bd[pos - 1] > acc) {
                bd[pos] = bd[pos - 1];
                bj[pos] = bj[pos - 1];
                --pos;
            }
            bd[pos] = acc;
            bj[pos] = yj * W + xj;
            if (cnt < k) ++cnt;
        }
    }
    for (int q = 0; q < k; ++q) {
        nbr[i * k + q] = q < cnt ? bj[q] : -1;
        dist[i * k + q] = q < cnt ? bd[q] : INFINITY;
    }
}

// w = exp(-d / sigma^2) as float32.  FP64 is slow on this GPU, so the
// exponential runs in FP32 wherever the result is a normal float32: with
// x = x_h + x_l (x_h = float32(x)), exp(-x) = exp(-x_h) (1 - x_l) to within a
// few float32 ulps (|x_l| <= 2^-24 x, so the dropped terms are below 2^-40).
// Near the underflow threshold, where FP32 would lose the subnormal digits,
// it runs in FP64.  Both ends of an edge see the same d, so w stays symmetric
// bit for bit.
__device__ __forceinline__ float edge_weight(float d, double inv_sigma2) {
    const double x = (double)d * inv_sigma2;   // within an ulp of d / sigma^2
    if (x < 80.0) {
        const float xh = (float)x;
        const float xl = (float)(x - (double)xh);
        return expf(-xh) * (1.0f - xl);
    }
    return (float)exp(-x);
}

// FILL = false: count[i] = row length; FILL = true: write the row at row_ptr[i].
template <bool FILL>
__global__ void __launch_bounds__(128)
image_union_kernel(int H, int W, int r, int k, const int32_t *__restrict__ nbr, const float *__restrict__ dist,
                   double inv_sigma2, int32_t *__restrict__ count, const int64_t *__restrict__ row_ptr,
                   int32_t *__restrict__ col, float *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= (int64_t)H * W) return;
    const int y = (int)(i / W), x = (int)(i % W);
    int32_t own[kMaxK];
    float ownd[kMaxK];
    for (int q = 0; q < k; ++q) {
        own[q] = __ldg(nbr + i * k + q);
        ownd[q] = __ldg(dist + i * k + q);
    }
    int64_t at = FILL ? row_ptr[i] : 0;
    int32_t len = 0;
    for (int yj = max(0, y - r); yj <= min(H - 1, y + r); ++yj)
        for (int xj = max(0, x - r); xj <= min(W - 1, x + r); ++xj) {
            const int32_t j = yj * W + xj;
            if (j == (int32_t)i) continue;
            float d = INFINITY;
            bool edge = false;
            for (int q = 0; q < k; ++q)
                if (own[q] == j) {
                    edge = true;
                    d = ownd[q];
                    break;
                }
            if (!edge) {
                const int32_t *lj = nbr + (int64_t)j * k;
                for (int q = 0; q < k; ++q)
                    if (__ldg(lj + q) == (int32_t)i) {
                        edge = true;
                        d = __ldg(dist + (int64_t)j * k + q);
                        break;
                    }
            }
            if (!edge) continue;
            if (FILL) {
                col[at] = j;
                w[at] = edge_weight(d, inv_sigma2);
                ++at;
            }
            ++len;
        }
    if (!FILL) count[i] = len;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct ImgWs {
    int32_t *nbr;
    float *dist;
    int32_t *count;
    int64_t *bsum, *total;
    size_t bytes;
};

ImgWs image_ws(int64_t n, int k, char *base) {
    ImgWs s{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align256(o + std::max<size_t>(b, 1)); return at; };
    const size_t o_nbr = take(sizeof(int32_t) * (size_t)n * k), o_dist = take(sizeof(float) * (size_t)n * k);
    const size_t o_cnt = take(sizeof(int32_t) * (size_t)n);
    const size_t nb = (size_t)((n + kScanBlock - 1) / kScanBlock);
    const size_t o_bsum = take(sizeof(int64_t) * nb), o_tot = take(sizeof(int64_t));
    s.bytes = o;
    if (base) {
        s.nbr = reinterpret_cast<int32_t *>(base + o_nbr);
        s.dist = reinterpret_cast<float *>(base + o_dist);
        s.count = reinterpret_cast<int32_t *>(base + o_cnt);
        s.bsum = reinterpret_cast<int64_t *>(base + o_bsum);
        s.total = reinterpret_cast<int64_t *>(base + o_tot);
    }
    return s;
}

bool args_ok(int32_t H, int32_t W, int32_t C, int32_t p, int32_t r, int32_t k) {
    if (H < 1 || W < 1 || C < 1 || C > 16 || p < 0 || p > 4 || r < 1 || k < 1 || k > kMaxK) return false;
    if ((int64_t)H * W > 0x7fffffffLL) return false;
    const int64_t wh = std::min<int64_t>(H, 2 * r + 1), ww = std::min<int64_t>(W, 2 * r + 1);
    return wh * ww - 1 >= k;   // every pixel has at least k window candidates
}

bool on_device(const void *p) {
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

extern "C" pdca_status pdca_image_graph_workspace_size(int32_t H, int32_t W, int32_t k, size_t *bytes) {
    if (!bytes || H < 1 || W < 1 || k < 1 || k > kMaxK || (int64_t)H * W > 0x7fffffffLL) return PDCA_ERR_INVALID_ARG;
    *bytes = image_ws((int64_t)H * W, k, nullptr).bytes;
    return PDCA_OK;
}

extern "C" pdca_status pdca_image_graph(const float *image, int32_t H, int32_t W, int32_t C, int32_t patch_radius,
                                        int32_t window_radius, int32_t k, double sigma, void *workspace,
                                        size_t ws_bytes, int64_t *row_ptr, int32_t *col, float *w,
                                        int64_t col_capacity, int64_t *nnz, void *stream) {
    if (!image || !workspace || !row_ptr || !col || !w || !nnz) return PDCA_ERR_INVALID_ARG;
    if (!args_ok(H, W, C, patch_radius, window_radius, k) || !(sigma > 0.0) || !std::isfinite(sigma))
        return PDCA_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return PDCA_ERR_INVALID_ARG;
    if (!on_device(image) || !on_device(workspace) || !on_device(row_ptr) || !on_device(col) || !on_device(w))
        return PDCA_ERR_INVALID_ARG;
    const int64_t n = (int64_t)H * W;
    const ImgWs s = image_ws(n, k, static_cast<char *>(workspace));
    if (ws_bytes < s.bytes) return PDCA_ERR_OOM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((n + 127) / 128);
    count_launches(3);
    image_knn_kernel<<<blocks, 128, 0, st>>>(image, H, W, C, patch_radius, window_radius, k, s.nbr, s.dist);
    const double s2 = 1.0 / ((double)sigma * sigma);   // 1 / sigma^2
    image_union_kernel<false><<<blocks, 128, 0, st>>>(H, W, window_radius, k, s.nbr, s.dist, s2, s.count,
                                                      nullptr, nullptr, nullptr);
    exclusive_scan(n, s.count, row_ptr, s.bsum, s.total, st);
    int64_t tot = 0;
    if (cudaMemcpyAsync(&tot, s.total, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PDCA_ERR_CUDA;
    *nnz = tot;
    if (tot > col_capacity) return PDCA_ERR_OOM;
    count_launches(1);
    image_union_kernel<true><<<blocks, 128, 0, st>>>(H, W, window_radius, k, s.nbr, s.dist, s2, nullptr, row_ptr,
                                                     col, w);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return PDCA_ERR_CUDA;
    return PDCA_OK;
}
