// Hot-path kernels of the pDCA solver on sm_103a.
//
// sweep_kernel   one preconditioned sweep (eq. general:diag:pre) with the DCA
//                linearisation (eq. bt:ut), the fidelity term and, on the last
//                sweep of an outer step, the simplex projection fused in;
// energy_kernel  F(u) (eqs. gl:functional:graph, functional:GL) and the
//                residual ||b^t - T u^{t+1}|| with FP64 accumulation;
// power kernels  power method for lambda_max(L_s) (Sec. 3.1);
// labels / permutation kernels for the results.
//
// All of them walk the sliced-ELL operator the same way: one warp per 32-row
// slice, one lane per row, entry j of every lane read as one 128-byte
// coalesced load of column indices and one of weights (streamed with the
// evict-first hint), neighbour rows of u gathered through L1/L2.
#include "pdca_internal.cuh"

#include <math.h>

namespace pdca {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// row I/O: K floats per row, widest aligned vector access
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + q);
            x[4 * q + 0] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(p) + q);
            x[2 * q + 0] = t.x; x[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) x[q] = __ldg(p + q);
    }
}

template <int K>
__device__ __forceinline__ void store_row(float *__restrict__ p, const float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q)
            reinterpret_cast<float2 *>(p)[q] = make_float2(x[2 * q], x[2 * q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = x[q];
    }
}

// acc[k] = sum_j wt_ij * x_jk over the lane's row of the slice (padding
// entries carry weight 0 and point at the row itself).
template <int K>
__device__ __forceinline__ void gather_row_sum(const SellView &A, int64_t base, int width, int lane,
                                               const float *__restrict__ x, float (&acc)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const int32_t *__restrict__ cp = A.col + base + lane;
    const float *__restrict__ wp = A.w + base + lane;
    int j = 0;
    for (; j + 4 <= width; j += 4) {
        const int c0 = __ldcs(cp + 32 * (j + 0));
        const int c1 = __ldcs(cp + 32 * (j + 1));
        const int c2 = __ldcs(cp + 32 * (j + 2));
        const int c3 = __ldcs(cp + 32 * (j + 3));
        const float w0 = __ldcs(wp + 32 * (j + 0));
        const float w1 = __ldcs(wp + 32 * (j + 1));
        const float w2 = __ldcs(wp + 32 * (j + 2));
        const float w3 = __ldcs(wp + 32 * (j + 3));
        float x0[K], x1[K], x2[K], x3[K];
        load_row<K>(x + (size_t)c0 * K, x0);
        load_row<K>(x + (size_t)c1 * K, x1);
        load_row<K>(x + (size_t)c2 * K, x2);
        load_row<K>(x + (size_t)c3 * K, x3);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            acc[k] = fmaf(w0, x0[k], acc[k]);
            acc[k] = fmaf(w1, x1[k], acc[k]);
            acc[k] = fmaf(w2, x2[k], acc[k]);
            acc[k] = fmaf(w3, x3[k], acc[k]);
        }
    }
    for (; j < width; ++j) {
        const int c0 = __ldcs(cp + 32 * j);
        const float w0 = __ldcs(wp + 32 * j);
        float x0[K];
        load_row<K>(x + (size_t)c0 * K, x0);
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = fmaf(w0, x0[k], acc[k]);
    }
}

// prior y_ik in the +-1 coding from the row tag
template <int K>
__device__ __forceinline__ float prior_of(uint32_t tag, int k) {
    if (K == 1) return tag == 1u ? 1.0f : -1.0f;
    return tag == (uint32_t)k ? 1.0f : -1.0f;
}

// Euclidean projection of a row onto the simplex in the coding v = (u+1)/2
// (sort-and-threshold method of Held, Wolfe and Crowder), thresholds in FP64.
template <int K>
__device__ __forceinline__ void project_simplex(float (&u)[K]) {
    double v[K], mu[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = 0.5 * ((double)u[k] + 1.0);
        mu[k] = v[k];
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j + 1 < K - i; ++j) {
            const double a = mu[j], b = mu[j + 1];
            mu[j] = a > b ? a : b;
            mu[j + 1] = a > b ? b : a;
        }
    }
    double run = 0.0, theta = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        run += mu[j];
        const double t = (run - 1.0) / (double)(j + 1);
        if (mu[j] - t > 0.0) theta = t;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double vk = v[k] - theta;
        vk = vk < 0.0 ? 0.0 : vk;
        u[k] = (float)(2.0 * vk - 1.0);
    }
}

// ---------------------------------------------------------------------------
// fused sweep
// ---------------------------------------------------------------------------
//   b    = eta Lambda_i y_i + c u_i - (u_i^3 - u_i)/eps          (u = u^t)
//   Tv   = eps (v_i - sum_j wt_ij v_j) + (c + eta Lambda_i) v_i
//   v'_i = v_i + (b - Tv) / g_i,   then projected if PROJECT.
template <int K, bool PROJECT>
__global__ void __launch_bounds__(kBlockThreads)
sweep_kernel(const SellView A, const Coeffs cf, const float *__restrict__ v_src,
             const float *__restrict__ u_t, float *__restrict__ v_dst) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (slice >= A.n_slices) return;
    const int64_t base = A.slice_off[slice];
    const int width = (int)((A.slice_off[slice + 1] - base) >> 5);
    const int r = slice * kSliceRows + lane;
    const uint32_t info = A.rowinfo[r];

    float acc[K];
    gather_row_sum<K>(A, base, width, lane, v_src, acc);

    float v[K], u[K];
    load_row<K>(v_src + (size_t)r * K, v);
    if (u_t == v_src) {
#pragma unroll
        for (int k = 0; k < K; ++k) u[k] = v[k];
    } else {
        load_row<K>(u_t + (size_t)r * K, u);
    }
    const uint32_t tag = info & 0xFFu;
    const bool lab = tag != kTagUnlabelled;
    const float inv_g = lab ? cf.inv_g1 : cf.inv_g0;
    const float diag = cf.c + (lab ? cf.eta : 0.0f);
    float out[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float fid = lab ? cf.eta * prior_of<K>(tag, k) : 0.0f;
        const float uk = u[k];
        const float b = fid + cf.c * uk - (uk * uk * uk - uk) * cf.inv_eps;
        const float tv = cf.eps * (v[k] - acc[k]) + diag * v[k];
        out[k] = v[k] + (b - tv) * inv_g;
    }
    if constexpr (PROJECT) project_simplex<K>(out);
    store_row<K>(v_dst + (size_t)r * K, out);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum S values over the block in a fixed order and store them at out[0..S).
template <int S>
__device__ __forceinline__ void block_sum_store(double (&v)[S], double *__restrict__ out) {
    __shared__ double sm[kWarpsPerBlock][S];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double t = warp_sum(v[s]);
        if (lane == 0) sm[warp][s] = t;
    }
    __syncthreads();
    if (threadIdx.x < S) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kWarpsPerBlock; ++q) t += sm[q][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// Per-row contributions (FP32 inside a row, FP64 across rows):
//   quad += u_i . (L_s u)_i,  well += sum_k (u_ik^2 - 1)^2,
//   fid  += Lambda_i sum_k (u_ik - y_ik)^2,
//   rr   += ||b_i - (T u)_i||^2 with b from u_prev, bb += ||b_i||^2.
// b - T u is formed as c (u_prev - u) + eta Lambda (y - u)
//   - (u_prev^3 - u_prev)/eps - eps (L_s u), which avoids the cancellation
// of the two large terms c u_prev and c u.
template <int K>
__global__ void __launch_bounds__(kBlockThreads)
energy_kernel(const SellView A, const Coeffs cf, const float *__restrict__ u,
              const float *__restrict__ u_prev, double *__restrict__ partials) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    double red[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (slice < A.n_slices) {
        const int64_t base = A.slice_off[slice];
        const int width = (int)((A.slice_off[slice + 1] - base) >> 5);
        const int r = slice * kSliceRows + lane;
        const uint32_t info = A.rowinfo[r];
        float acc[K];
        gather_row_sum<K>(A, base, width, lane, u, acc);
        if (r < A.n) {
            float x[K];
            load_row<K>(u + (size_t)r * K, x);
            const uint32_t tag = info & 0xFFu;
            const bool lab = tag != kTagUnlabelled;
            float q = 0.f, wl = 0.f, fd = 0.f, rr = 0.f, bb = 0.f, nf = 0.f;
            float xp[K];
            if (u_prev) load_row<K>(u_prev + (size_t)r * K, xp);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float ls = x[k] - acc[k];
                q = fmaf(x[k], ls, q);
                const float s = x[k] * x[k] - 1.0f;
                wl = fmaf(s, s, wl);
                const float y = lab ? prior_of<K>(tag, k) : 0.0f;
                if (lab) fd = fmaf(x[k] - y, x[k] - y, fd);
                if (!isfinite(x[k])) nf += 1.0f;
                if (u_prev) {
                    const float up = xp[k];
                    const float grad_w = (up * up * up - up) * cf.inv_eps;
                    const float b = (lab ? cf.eta * y : 0.0f) + cf.c * up - grad_w;
                    const float res = cf.c * (up - x[k]) + (lab ? cf.eta * (y - x[k]) : 0.0f)
                                      - grad_w - cf.eps * ls;
                    rr = fmaf(res, res, rr);
                    bb = fmaf(b, b, bb);
                }
            }
            red[0] = q; red[1] = wl; red[2] = fd; red[3] = rr; red[4] = bb; red[5] = nf;
        }
    }
    block_sum_store<6>(red, partials + (size_t)blockIdx.x * kRedSlots);
}

// Single block: fixed-order sum of the block partials, then the scalars.
__global__ void __launch_bounds__(256)
energy_finalize_kernel(const double *__restrict__ partials, int n_parts, double eps_d, double eta_d,
                       int has_prev, RedOut *out, double *trace_F, double *trace_r) {
    __shared__ double sm[256][6];
    double t[6] = {0, 0, 0, 0, 0, 0};
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

// ---------------------------------------------------------------------------
// power method for lambda_max(L_s)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads)
power_init_kernel(const SellView A, const int32_t *__restrict__ perm, float *__restrict__ x,
                  double *__restrict__ partials) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    double red[3] = {0.0, 0.0, 0.0};
    if (slice < A.n_slices) {
        const int r = slice * kSliceRows + lane;
        float xi = 0.0f;
        if (r < A.n) xi = (float)(1.0 + 0.5 * sin((double)perm[r] + 1.0));
        x[r] = xi;
        red[0] = (double)xi * (double)xi;
    }
    block_sum_store<3>(red, partials + (size_t)blockIdx.x * kRedSlots);
}

// y = L_s (s x) with s = *scale; partial sums of y.y, (s x).y, (s x).(s x).
__global__ void __launch_bounds__(kBlockThreads)
power_spmv_kernel(const SellView A, const float *__restrict__ x, const double *__restrict__ scale,
                  float *__restrict__ y, double *__restrict__ partials) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    double red[3] = {0.0, 0.0, 0.0};
    if (slice < A.n_slices) {
        const int64_t base = A.slice_off[slice];
        const int width = (int)((A.slice_off[slice + 1] - base) >> 5);
        const int r = slice * kSliceRows + lane;
        const float s = (float)(*scale);
        float acc[1];
        gather_row_sum<1>(A, base, width, lane, x, acc);
        const float xs = s * __ldg(x + r);
        const float yi = xs - s * acc[0];
        y[r] = yi;
        if (r < A.n) {
            red[0] = (double)yi * (double)yi;
            red[1] = (double)xs * (double)yi;
            red[2] = (double)xs * (double)xs;
        }
    }
    block_sum_store<3>(red, partials + (size_t)blockIdx.x * kRedSlots);
}

// scale <- 1/sqrt(sum y.y); lambda <- sum (s x).y / sum (s x).(s x)
__global__ void __launch_bounds__(256)
power_finalize_kernel(const double *__restrict__ partials, int n_parts, double *scale,
                      double *lambda) {
    __shared__ double sm[256][3];
    double t[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < n_parts; i += 256)
#pragma unroll
        for (int s = 0; s < 3; ++s) t[s] += partials[(size_t)i * kRedSlots + s];
#pragma unroll
    for (int s = 0; s < 3; ++s) sm[threadIdx.x][s] = t[s];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
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

template <int K>
cudaError_t sweep_k(bool project, const SellView &A, const Coeffs &cf, const float *v_src,
                    const float *u_t, float *v_dst, cudaStream_t st) {
    const int blocks = (A.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (project && K >= 2)
        sweep_kernel<K, (K >= 2)><<<blocks, kBlockThreads, 0, st>>>(A, cf, v_src, u_t, v_dst);
    else
        sweep_kernel<K, false><<<blocks, kBlockThreads, 0, st>>>(A, cf, v_src, u_t, v_dst);
    return cudaGetLastError();
}

template <int K>
cudaError_t energy_k(const SellView &A, const Coeffs &cf, const float *u, const float *u_prev,
                     double *partials, cudaStream_t st) {
    energy_kernel<K><<<energy_blocks(A.n_slices), kBlockThreads, 0, st>>>(A, cf, u, u_prev, partials);
    return cudaGetLastError();
}

template <int K>
cudaError_t labels_k(int32_t n, const float *u, const int32_t *perm, int32_t *out, cudaStream_t st) {
    labels_kernel<K><<<(n + 255) / 256, 256, 0, st>>>(n, u, perm, out);
    return cudaGetLastError();
}

}  // namespace

int energy_blocks(int32_t n_slices) { return (n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock; }

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

cudaError_t launch_sweep(int K, bool project, const SellView &A, const Coeffs &cf,
                         const float *v_src, const float *u_t, float *v_dst, cudaStream_t st) {
    if (A.n_slices <= 0) return cudaSuccess;
    count_launches(1);
#define CALL(KK) sweep_k<KK>(project, A, cf, v_src, u_t, v_dst, st)
    PDCA_DISPATCH_K(K, CALL)
#undef CALL
}

cudaError_t launch_energy(int K, const SellView &A, const Coeffs &cf, const float *u,
                          const float *u_prev, double *partials, cudaStream_t st) {
    count_launches(1);
#define CALL(KK) energy_k<KK>(A, cf, u, u_prev, partials, st)
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

cudaError_t launch_power_spmv(const SellView &A, const float *x, const double *scale, float *y,
                              double *partials, cudaStream_t st) {
    count_launches(1);
    power_spmv_kernel<<<energy_blocks(A.n_slices), kBlockThreads, 0, st>>>(A, x, scale, y, partials);
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
