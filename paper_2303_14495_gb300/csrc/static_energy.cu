// pdca_energy_static: the GL energy F(u) of an iterate, computed straight
// from a device CSR graph, for callers that cannot allocate device memory.
//
// Such callers cannot give the library a workspace: for example a host
// framework that owns every device byte through its own fixed-budget pool
// and forbids other allocators, a plug-in loaded into such a process, or a
// latency-critical loop that must not pay cudaMalloc's implicit device-wide
// synchronisation.  This entry point therefore keeps its scratch (inverse
// square-root degrees, per-block partial sums, the result and a status word)
// in one file-scope __device__ array of fixed size.  Every process that
// loads the library holds that array on every GPU it uses until it exits.
//
// The graph is checked as far as one pass over it allows: row_ptr inside
// [0, nnz], columns in range, no self loop, finite non-negative weights,
// mask values 0/1 and prior labels in range on labelled rows (BAD_GRAPH).
// Symmetry and the column order are not checked.
//
// The array is shared by all calls: a call overwrites what the previous call
// left, and clears the status word before use.  Two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it and give wrong results; callers must serialise them.
#include "pdca_internal.cuh"

#include <math.h>

#include <cmath>
#include <mutex>

namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticBlocks = 1024;            // grid of the row pass (grid-stride)
constexpr int kStaticSlots = 8;                // doubles per block partial
constexpr size_t kOffInvSqrtDeg = 0;           // float[PDCA_STATIC_MAX_N]
constexpr size_t kOffPartials = (size_t)PDCA_STATIC_MAX_N * sizeof(float);
constexpr size_t kOffResult = kOffPartials + (size_t)kStaticBlocks * kStaticSlots * sizeof(double);
constexpr size_t kOffStatus = kOffResult + 8 * sizeof(double);
constexpr size_t kStaticScratchBytes = kOffStatus + 256;

// The scratch of pdca_energy_static (about 4.1 MiB).
static __device__ __align__(256) unsigned char g_pdca_static_scratch[kStaticScratchBytes];

constexpr unsigned kStBadGraph = 1u, kStIsolated = 2u;

// Address of the array on each device, looked up once per device.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};

// s_i = 1 / sqrt(d_i), d_i = sum_j w_ij in CSR order (FP64).
__global__ void static_degree_kernel(int32_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                     const float *__restrict__ w, unsigned char *__restrict__ scratch) {
    float *s = reinterpret_cast<float *>(scratch + kOffInvSqrtDeg);
    unsigned *status = reinterpret_cast<unsigned *>(scratch + kOffStatus);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
        if (e0 < 0 || e1 < e0 || e1 > nnz) {
            atomicOr(status, kStBadGraph);
            s[i] = 0.0f;
            continue;
        }
        double d = 0.0;
        bool bad = false;
        for (int64_t e = e0; e < e1; ++e) {
            const float wv = w[e];
            if (!(isfinite(wv) && wv >= 0.0f)) bad = true;
            d += (double)wv;
        }
        if (bad) atomicOr(status, kStBadGraph);
        if (!(d > 0.0)) atomicOr(status, kStIsolated);
        s[i] = d > 0.0 ? (float)(1.0 / sqrt(d)) : 0.0f;
    }
}

__device__ __forceinline__ double static_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per row: quad += u_i . (L_s u)_i, well += sum_k (u_ik^2 - 1)^2,
// fid += Lambda_i sum_k (u_ik - y_ik)^2, non-finite count; block partials.
template <int K>
__global__ void __launch_bounds__(kStaticThreads)
static_energy_kernel(int32_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                     const int32_t *__restrict__ col, const float *__restrict__ w,
                     const float *__restrict__ u, const uint8_t *__restrict__ mask,
                     const int32_t *__restrict__ labels, unsigned char *__restrict__ scratch) {
    const float *s = reinterpret_cast<const float *>(scratch + kOffInvSqrtDeg);
    double *partials = reinterpret_cast<double *>(scratch + kOffPartials);
    unsigned *status = reinterpret_cast<unsigned *>(scratch + kOffStatus);
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
        if (e0 < 0 || e1 < e0 || e1 > nnz) continue;   // flagged by the degree pass
        const float si = s[i];
        float acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0f;
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t j = col[e];
            if (j < 0 || j >= n || j == i) {
                atomicOr(status, kStBadGraph);
                continue;
            }
            const float wt = w[e] * si * s[j];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = fmaf(wt, u[(size_t)j * K + k], acc[k]);
        }
        const uint8_t m = mask[i];
        const int32_t lab = m ? labels[i] : 0;
        if (m > 1 || (m == 1 && (lab < 0 || lab >= (K == 1 ? 2 : K)))) atomicOr(status, kStBadGraph);
        float q = 0.f, wl = 0.f, fd = 0.f, nf = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float x = u[(size_t)i * K + k];
            const float ls = x - acc[k];
            q = fmaf(x, ls, q);
            const float t = x * x - 1.0f;
            wl = fmaf(t, t, wl);
            if (m) {
                const float y = (K == 1) ? (lab == 1 ? 1.0f : -1.0f) : (lab == k ? 1.0f : -1.0f);
                fd = fmaf(x - y, x - y, fd);
            }
            if (!isfinite(x)) nf += 1.0f;
        }
        red[0] += q;
        red[1] += wl;
        red[2] += fd;
        red[3] += nf;
    }
    __shared__ double sm[kStaticThreads / 32][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const double v = static_warp_sum(red[t]);
        if (lane == 0) sm[warp][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int q = 0; q < kStaticThreads / 32; ++q) v += sm[q][threadIdx.x];
        partials[(size_t)blockIdx.x * kStaticSlots + threadIdx.x] = v;
    }
}

// One block: fixed-order sum of the partials; result[0] = F, result[1] =
// non-finite count.  F_dev (device pointer or null) receives F when the
// status word is clear and F is finite, so a device output is written on
// success only, as a host one is.
__global__ void static_finalize_kernel(double eps, double eta, unsigned char *__restrict__ scratch,
                                       double *__restrict__ F_dev) {
    const double *partials = reinterpret_cast<const double *>(scratch + kOffPartials);
    double *result = reinterpret_cast<double *>(scratch + kOffResult);
    __shared__ double sm[kStaticThreads][4];
    double t[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < kStaticBlocks; b += kStaticThreads)
#pragma unroll
        for (int s = 0; s < 4; ++s) t[s] += partials[(size_t)b * kStaticSlots + s];
#pragma unroll
    for (int s = 0; s < 4; ++s) sm[threadIdx.x][s] = t[s];
    __syncthreads();
    for (int h = kStaticThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int s = 0; s < 4; ++s) sm[threadIdx.x][s] += sm[threadIdx.x + h][s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double F = 0.5 * eps * sm[0][0] + sm[0][1] / (4.0 * eps) + 0.5 * eta * sm[0][2];
        result[0] = F;
        result[1] = sm[0][3];
        const unsigned status = *reinterpret_cast<const unsigned *>(scratch + kOffStatus);
        if (F_dev && status == 0u && sm[0][3] == 0.0 && isfinite(F)) *F_dev = F;
    }
}

template <int K>
cudaError_t static_energy_k(int32_t n, int64_t nnz, const int64_t *rp, const int32_t *col, const float *w,
                            const float *u, const uint8_t *mask, const int32_t *lab, unsigned char *scr,
                            cudaStream_t st) {
    static_energy_kernel<K><<<kStaticBlocks, kStaticThreads, 0, st>>>(n, nnz, rp, col, w, u, mask, lab, scr);
    return cudaGetLastError();
}

cudaError_t launch_static_energy(int K, int32_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                                 const float *w, const float *u, const uint8_t *mask, const int32_t *lab,
                                 unsigned char *scr, cudaStream_t st) {
#define CALL(KK) static_energy_k<KK>(n, nnz, rp, col, w, u, mask, lab, scr, st)
    switch (K) {
    case 1: return CALL(1); case 2: return CALL(2); case 3: return CALL(3); case 4: return CALL(4);
    case 5: return CALL(5); case 6: return CALL(6); case 7: return CALL(7); case 8: return CALL(8);
    case 9: return CALL(9); case 10: return CALL(10); case 11: return CALL(11); case 12: return CALL(12);
    case 13: return CALL(13); case 14: return CALL(14); case 15: return CALL(15); case 16: return CALL(16);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array for the current device (set up once
// per device, with that device current).
pdca_status scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PDCA_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pdca_static_scratch) != cudaSuccess || !p) return PDCA_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return PDCA_OK;
}

}  // namespace

extern "C" pdca_status pdca_energy_static(const int64_t *row_ptr, const int32_t *col, const float *w,
                                          int32_t n, int64_t nnz, int32_t k, const float *u,
                                          const uint8_t *fid_mask, const int32_t *labels, double eps,
                                          double eta, void *stream, double *F_out) {
    if (!F_out || k < 1 || k > PDCA_MAX_K || n < 1 || nnz < 0) return PDCA_ERR_INVALID_ARG;
    if (!(std::isfinite(eps) && eps > 0) || !(std::isfinite(eta) && eta >= 0)) return PDCA_ERR_INVALID_ARG;
    if (n > PDCA_STATIC_MAX_N) return PDCA_ERR_TOO_LARGE;
    if (!on_device(row_ptr) || !on_device(u) || !on_device(fid_mask) || !on_device(labels) ||
        (nnz > 0 && (!on_device(col) || !on_device(w))))
        return PDCA_ERR_INVALID_ARG;
    unsigned char *scr = nullptr;
    pdca_status st = scratch_address(&scr);
    if (st != PDCA_OK) return st;
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    unsigned status = 0;
    double res[2] = {0.0, 0.0};
    if (cudaMemsetAsync(scr + kOffStatus, 0, sizeof(unsigned), sm) != cudaSuccess) return PDCA_ERR_CUDA;
    const int deg_blocks = (int)((n + kStaticThreads - 1) / kStaticThreads);
    static_degree_kernel<<<deg_blocks < kStaticBlocks ? deg_blocks : kStaticBlocks, kStaticThreads, 0, sm>>>(
        n, nnz, row_ptr, w, scr);
    if (cudaGetLastError() != cudaSuccess) return PDCA_ERR_CUDA;
    if (launch_static_energy(k, n, nnz, row_ptr, col, w, u, fid_mask, labels, scr, sm) != cudaSuccess)
        return PDCA_ERR_CUDA;
    const bool dev_out = on_device(F_out);
    static_finalize_kernel<<<1, kStaticThreads, 0, sm>>>(eps, eta, scr, dev_out ? F_out : nullptr);
    if (cudaGetLastError() != cudaSuccess) return PDCA_ERR_CUDA;
    pdca::count_launches(3);
    if (cudaMemcpyAsync(&status, scr + kOffStatus, sizeof(unsigned), cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaMemcpyAsync(res, scr + kOffResult, sizeof(res), cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaStreamSynchronize(sm) != cudaSuccess)
        return PDCA_ERR_CUDA;
    if (status & kStBadGraph) return PDCA_ERR_BAD_GRAPH;
    if (status & kStIsolated) return PDCA_ERR_ISOLATED_NODE;
    if (res[1] > 0 || !std::isfinite(res[0])) return PDCA_ERR_NONFINITE;
    if (!dev_out) *F_out = res[0];   // a device F_out was written by the finalize kernel
    return PDCA_OK;
}
