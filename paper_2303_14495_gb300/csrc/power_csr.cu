// Power method for lambda_max (Sec. 3.1) on the caller's CSR graph, run at
// create time while the host computes the node renumbering: the estimate
// needs no sliced-ELL operator, so the two overlap.
//
// Iterate x <- L x / ||L x|| (L_s or L = D - W) from x0_i = 1 + 0.5 sin(i + 1)
// (caller's index i), 150 iterations in the paper's setting, Rayleigh
// quotient of the last pair.  With s = 1 / ||x|| (kept on the device) one
// iteration forms, for every row,
//     y_i = a_i s x_i - b_i s sum_j w_ij z_j,
//     (L_s: a_i = 1, b_i = d_i^-1/2, z_j = d_j^-1/2 x_j;  L: a_i = d_i, b_i = 1, z_j = x_j)
// and writes y and z' = (y scaled as z), so the next iteration reads the
// neighbours' z directly.  c_i = d_i^-1/2 (L_s) or d_i (L) in FP32 is formed
// once by the init kernel.  Block partials of y.y, (s x).y and (s x).(s x)
// are summed by the block that finishes last (an atomic ticket), which
// updates s and the Rayleigh quotient (s x).y / (s x).(s x).
//
// Eight lanes share a row (a warp reads 4 rows' entries, 32 consecutive bytes
// of columns and of weights per row); a fixed grid walks the rows with a
// fixed stride, so every partial and the estimate are the same on every run.
#include "device_common.cuh"

#include <math.h>

namespace pdca {
namespace {

using namespace dev;

constexpr int kPcThreads = 256;
constexpr int kPcLanes = 8;                                   // lanes per row
constexpr int kPcRowsPerBlock = kPcThreads / kPcLanes;        // 32
constexpr int kPcBlocks = 8 * kSmCount;                       // fixed grid

__device__ __forceinline__ float sub_sum8(float v) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block partial of three sums: FP32 per thread and warp, FP64 across warps.
__device__ __forceinline__ void block_partial3(float (&v)[3], double *__restrict__ out) {
    __shared__ double sm[kPcThreads / 32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float t = warp_sum_f(v[s]);
        if (lane == 0) sm[warp][s] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kPcThreads / 32; ++q) t += sm[q][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// Last block to arrive: fixed-order sum of the partials, then s and lambda.
__device__ __forceinline__ void last_block_update(const double *partials, unsigned *ticket, double *scale,
                                                  double *lambda) {
    __shared__ bool last;
    if (threadIdx.x < 32) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double sm[kPcThreads][3];
    double t[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kPcThreads)
#pragma unroll
        for (int s = 0; s < 3; ++s) t[s] += __ldcg(partials + (size_t)i * kRedSlots + s);
#pragma unroll
    for (int s = 0; s < 3; ++s) sm[threadIdx.x][s] = t[s];
    __syncthreads();
    for (int h = kPcThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int s = 0; s < 3; ++s) sm[threadIdx.x][s] += sm[threadIdx.x + h][s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double yy = sm[0][0], xy = sm[0][1], xx = sm[0][2];
        *scale = yy > 0.0 ? 1.0 / sqrt(yy) : 0.0;
        if (xx > 0.0) *lambda = xy / xx;
        *ticket = 0u;
    }
}

// x0, z0 and the partial of x0.x0 (slots 0 and 2 hold it; s = 1/||x0||).
__global__ void __launch_bounds__(kPcThreads)
power_csr_init_kernel(int32_t n, const double *__restrict__ isd, const double *__restrict__ deg, int un,
                      float *__restrict__ c, float *__restrict__ x, float *__restrict__ z,
                      double *__restrict__ partials, unsigned *ticket, double *scale, double *lambda) {
    float red[3] = {0.f, 0.f, 0.f};
    for (int32_t i = blockIdx.x * kPcThreads + threadIdx.x; i < n; i += gridDim.x * kPcThreads) {
        const float xi = (float)(1.0 + 0.5 * sin((double)i + 1.0));
        const float ci = un ? (float)deg[i] : (float)isd[i];
        c[i] = ci;
        x[i] = xi;
        z[i] = un ? xi : ci * xi;
        red[0] = fmaf(xi, xi, red[0]);
    }
    block_partial3(red, partials + (size_t)blockIdx.x * kRedSlots);
    last_block_update(partials, ticket, scale, lambda);
}

__global__ void __launch_bounds__(kPcThreads)
power_csr_kernel(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                 const float *__restrict__ w, const float *__restrict__ c, int un, const float *__restrict__ x,
                 const float *__restrict__ z, float *__restrict__ y, float *__restrict__ z_out, double *scale,
                 double *__restrict__ partials, unsigned *ticket, double *lambda) {
    const float s = (float)__ldcg(scale);
    const int sub = threadIdx.x & (kPcLanes - 1);
    float red[3] = {0.f, 0.f, 0.f};
    const int32_t stride = gridDim.x * kPcRowsPerBlock;
    // every lane of a warp runs the same number of steps (row index rounded
    // up to whole warps of rows), so the shuffles below see full warps
    const int32_t n_up = (n + 3) / 4 * 4;
    for (int32_t i = blockIdx.x * kPcRowsPerBlock + (threadIdx.x / kPcLanes); i < n_up; i += stride) {
        float acc = 0.0f;
        const bool real = i < n;
        if (real) {
            const int64_t e0 = rp[i], e1 = rp[i + 1];
            for (int64_t e = e0 + sub; e < e1; e += kPcLanes) acc = fmaf(__ldg(w + e), __ldg(z + __ldg(col + e)), acc);
        }
        acc = sub_sum8(acc);
        if (real && sub == 0) {
            const float xs = s * x[i];
            const float ci = c[i];
            const float yi = un ? ci * xs - s * acc : xs - ci * (s * acc);
            y[i] = yi;
            z_out[i] = un ? yi : ci * yi;
            red[0] = fmaf(yi, yi, red[0]);
            red[1] = fmaf(xs, yi, red[1]);
            red[2] = fmaf(xs, xs, red[2]);
        }
    }
    block_partial3(red, partials + (size_t)blockIdx.x * kRedSlots);
    last_block_update(partials, ticket, scale, lambda);
}

}  // namespace

size_t power_csr_scratch_bytes(int32_t n) {
    return ((size_t)5 * (size_t)n * sizeof(float) + 255) / 256 * 256 + (size_t)kPcBlocks * kRedSlots * sizeof(double) +
           256;
}

cudaError_t launch_power_csr(int32_t n, const int64_t *rp, const int32_t *col, const float *w, const double *isd,
                             const double *deg, bool un, int32_t iters, void *scratch, double *scale, double *lambda,
                             cudaStream_t st) {
    float *c = static_cast<float *>(scratch);
    float *x = c + n, *y = c + 2 * (size_t)n, *z0 = c + 3 * (size_t)n, *z1 = c + 4 * (size_t)n;
    char *tail = static_cast<char *>(scratch) + ((size_t)5 * (size_t)n * sizeof(float) + 255) / 256 * 256;
    double *partials = reinterpret_cast<double *>(tail);
    unsigned *ticket = reinterpret_cast<unsigned *>(tail + (size_t)kPcBlocks * kRedSlots * sizeof(double));
    count_launches(1 + (uint64_t)iters + 1);
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    power_csr_init_kernel<<<kPcBlocks, kPcThreads, 0, st>>>(n, isd, deg, un ? 1 : 0, c, x, z0, partials, ticket,
                                                           scale, lambda);
    for (int32_t it = 0; it <= iters; ++it) {
        power_csr_kernel<<<kPcBlocks, kPcThreads, 0, st>>>(n, rp, col, w, c, un ? 1 : 0, x, z0, y, z1, scale,
                                                          partials, ticket, lambda);
        std::swap(x, y);
        std::swap(z0, z1);
    }
    return cudaGetLastError();
}

}  // namespace pdca
