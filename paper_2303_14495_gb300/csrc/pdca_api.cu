// Host side of the C interface declared in include/pdca.h: argument checks,
// the workspace layout, problem creation and the outer pDCA loop.
#include "pdca_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

namespace pdca {
int host_workers();   // threads host_parallel_for uses (reorder.cpp)
}  // namespace pdca

using namespace pdca;

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr size_t kAlign = 256;
constexpr int kTraceCap = 1024;   // outer steps per trace chunk
constexpr double kPadTarget = 1.10;
constexpr int32_t kBfsChunk = 1 << 16;       // renumbering chunk (multiple of kBfsBlock)

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Everything about the device layout that depends only on the sizes and the
// row lengths; computed on the host from row_ptr.
struct Layout {
    int32_t n = 0, K = 0, n_pad = 0, n_slices = 0, sigma = 0, n_tiles = 0;
    bool host_order = false;           // BFS-block renumbering (widths known only at create)
    bool device_order = false;         // ... computed by the device kernels (else on a host thread)
    int64_t nnz = 0, sell_entries = 0, sell_cap = 0, halo_cap = 0;
    int32_t split = 0;                 // split length T (rows longer than T use the overflow CSR)
    int32_t n_ov = 0;                  // rows longer than T
    int64_t ov_entries = 0;            // their entries past T
    std::vector<int64_t> slice_off;    // n_slices + 1 (exact; filled at create for host order)
    size_t o_col, o_col16, o_fmt, o_w, o_wb, o_slice, o_rowinfo, o_perm, o_iperm, o_self, o_dsq, o_u[3], o_part,
        o_red, o_scal, o_trace;
    size_t o_hoff, o_hidx;
    size_t o_ovrp, o_ovcol, o_ovw, o_ovwb, o_ovidx, o_ovacc;   // overflow CSR and its pre-pass sums
    size_t o_mr, o_me[2];              // mixed precision: r (FP32) and the two corrections (16-bit)
    size_t o_srp, o_scol, o_sw, o_sdeg, o_sisd, o_smask, o_slab, o_scls, o_sscan = 0, o_skey = 0, o_sbfs = 0,
        o_status;
    size_t total = 0;
};

// Upper bound of the padded entries for any renumbering that sorts rows by
// degree inside windows of `sigma` rows: inside a window sorted descending,
// sum over slices of 32 * width <= (window nonzeros) + 32 * (window maximum),
// and the window maxima sum to at most the sum of the largest
// (number of windows) degrees; rounding each slice width up to kVec adds at
// most 32 (kVec - 1) per slice.  The top degrees are summed from a degree
// histogram (one pass) unless the largest degree makes it too big.
int64_t sell_bound(const int64_t *rp, int32_t n, int32_t sigma, int64_t max_deg) {
    const int64_t windows = ((int64_t)n + sigma - 1) / sigma;
    int64_t top = std::min<int64_t>(windows, n), s = 0;
    if (max_deg <= (1 << 20)) {
        // per-chunk histograms in parallel (few chunks when the degree range is wide)
        const int64_t nch = max_deg <= 4096 ? std::max<int64_t>(1, std::min<int64_t>(64, n / 65536)) : 1;
        std::vector<std::vector<uint32_t>> part((size_t)nch, std::vector<uint32_t>((size_t)max_deg + 1, 0u));
        host_parallel_for(nch, [&](int64_t c) {
            const int64_t i0 = (int64_t)n * c / nch, i1 = (int64_t)n * (c + 1) / nch;
            for (int64_t i = i0; i < i1; ++i) ++part[(size_t)c][(size_t)(rp[i + 1] - rp[i])];
        });
        std::vector<uint32_t> &hist = part[0];
        for (int64_t c = 1; c < nch; ++c)
            for (size_t d = 0; d < hist.size(); ++d) hist[d] += part[(size_t)c][d];
        for (int64_t d = max_deg; d >= 0 && top > 0; --d) {
            const int64_t take = std::min<int64_t>(top, hist[(size_t)d]);
            s += take * d;
            top -= take;
        }
    } else {
        std::vector<int32_t> d((size_t)n);
        for (int32_t i = 0; i < n; ++i) d[(size_t)i] = (int32_t)(rp[i + 1] - rp[i]);
        std::nth_element(d.begin(), d.begin() + (top - 1), d.end(), std::greater<int32_t>());
        for (int64_t i = 0; i < top; ++i) s += d[(size_t)i];
    }
    const int64_t n_slices = ((int64_t)n + kSliceRows - 1) / kSliceRows;
    return rp[n] + (int64_t)kSliceRows * s + n_slices * kSliceRows * (kVec - 1);
}

// Slice widths for one sort window: the degrees of the window sorted
// descending; a slice's width is the degree at its first position.
void window_widths(const int64_t *rp, int64_t base, int64_t end, int32_t split, std::vector<int32_t> &scratch,
                   std::vector<int64_t> &widths) {
    scratch.resize((size_t)(end - base));
    for (int64_t i = base; i < end; ++i)
        scratch[(size_t)(i - base)] = (int32_t)std::min<int64_t>(rp[i + 1] - rp[i], split);
    std::sort(scratch.begin(), scratch.end(), std::greater<int32_t>());
    for (int64_t p = 0; p < end - base; p += kSliceRows)
        widths[(size_t)((base + p) / kSliceRows)] = (scratch[(size_t)p] + kVec - 1) / kVec * kVec;
}

int64_t sell_entries_for(const int64_t *rp, int32_t n, int32_t sigma, int32_t split, std::vector<int64_t> &widths) {
    const int32_t n_slices = (n + kSliceRows - 1) / kSliceRows;
    widths.assign((size_t)n_slices, 0);
    const int64_t nwin = ((int64_t)n + sigma - 1) / sigma;
    host_parallel_for(nwin, [&](int64_t wdx) {
        std::vector<int32_t> scratch;
        const int64_t base = wdx * sigma;
        window_widths(rp, base, std::min<int64_t>(n, base + sigma), split, scratch, widths);
    });
    int64_t tot = 0;
    for (int64_t w : widths) tot += w * kSliceRows;
    return tot;
}

pdca_status check_params(const pdca_params &p) {
    auto fin = [](double x) { return std::isfinite(x); };
    if (!(fin(p.eps) && p.eps > 0) || !(fin(p.c) && p.c > 0) || !(fin(p.eta) && p.eta >= 0))
        return PDCA_ERR_INVALID_ARG;
    if (p.laplacian != PDCA_LAP_NORMALIZED && p.laplacian != PDCA_LAP_UNNORMALIZED) return PDCA_ERR_INVALID_ARG;
    if (!(fin(p.step_k) && p.step_k >= 0)) return PDCA_ERR_INVALID_ARG;
    if (p.laplacian == PDCA_LAP_UNNORMALIZED && p.tiling == PDCA_TILING_ON) return PDCA_ERR_INVALID_ARG;
    if (p.precision != PDCA_FP32 && p.precision != PDCA_MIXED_BF16W_FP16U && p.precision != PDCA_MIXED_BF16W_BF16U)
        return PDCA_ERR_INVALID_ARG;
    if (p.precision != PDCA_FP32 && p.tiling == PDCA_TILING_ON) return PDCA_ERR_INVALID_ARG;
    if (p.precond < PDCA_JACOBI_DAMPED || p.precond > PDCA_RICHARDSON) return PDCA_ERR_INVALID_ARG;
    if (!(fin(p.delta0) && p.delta0 >= 0) || !(fin(p.lambda_max) && p.lambda_max >= 0))
        return PDCA_ERR_INVALID_ARG;
    if (p.power_iters < 0) return PDCA_ERR_INVALID_ARG;
    if (p.sort_window != 0) {
        const int s = p.sort_window;
        if (s < 32 || s > 8192 || (s & (s - 1)) != 0) return PDCA_ERR_INVALID_ARG;
    }
    if (p.reorder != PDCA_REORDER_NONE && p.reorder != PDCA_REORDER_BFS) return PDCA_ERR_INVALID_ARG;
    if (p.tiling < PDCA_TILING_AUTO || p.tiling > PDCA_TILING_ON) return PDCA_ERR_INVALID_ARG;
    if (p.tiling == PDCA_TILING_ON && p.reorder != PDCA_REORDER_BFS) return PDCA_ERR_INVALID_ARG;
    if (p.entry_order != PDCA_ENTRIES_SPREAD && p.entry_order != PDCA_ENTRIES_CSR) return PDCA_ERR_INVALID_ARG;
    if (p.columns != PDCA_COLUMNS_AUTO && p.columns != PDCA_COLUMNS_32) return PDCA_ERR_INVALID_ARG;
    if (p.row_split < 0) return PDCA_ERR_INVALID_ARG;
    if (p.block_slices != 0 && p.block_slices != 8 && p.block_slices != 16 && p.block_slices != 32)
        return PDCA_ERR_INVALID_ARG;
    return PDCA_OK;
}

// Feasibility G > T of the diagonal preconditioners for L_s (Sec. 3.1):
// damped Jacobi G = diag(T)/omega needs omega in (0,1) and, for omega > 1/2,
// c > eps (2 omega - 1)/(1 - omega) (the spectrum of L_s lies in [0, 2]);
// perturbed Jacobi and Richardson need delta0 > 0 (Richardson also a
// lambda_max that bounds the spectrum, which the caller vouches for).
// c + 1/k: dividing the step-size-k system (I + kT, u^t + k b^t, G_k) by k
// gives the infinite-step system with this c and delta0/k.
double c_eff(const pdca_params &p) { return p.step_k > 0.0 ? p.c + 1.0 / p.step_k : p.c; }
double delta0_eff(const pdca_params &p) { return p.step_k > 0.0 ? p.delta0 / p.step_k : p.delta0; }

// Feasibility G > T (Sec. 3.1).  Damped Jacobi G = diag(T)/omega: for L_s the
// bound on c is exact for every graph (eigenvalues of D^{-1/2} W D^{-1/2} lie
// in [-1, 1]); for L, W >= -D gives G - T >= eps (1/omega - 2) D
// + (1/omega - 1)(c + eta Lambda), so c > eps d_max (2 omega - 1)/(1 - omega)
// suffices.  dmax = largest degree (used for L only).
pdca_status feasible(const pdca_params &p, double omega, double lambda, double dmax) {
    const double amax = p.laplacian == PDCA_LAP_UNNORMALIZED ? dmax : 1.0;
    switch (p.precond) {
    case PDCA_JACOBI_DAMPED:
        if (!(omega > 0.0 && omega < 1.0)) return PDCA_ERR_INFEASIBLE;
        if (omega > 0.5 && !(c_eff(p) > p.eps * amax * (2.0 * omega - 1.0) / (1.0 - omega)))
            return PDCA_ERR_INFEASIBLE;
        return PDCA_OK;
    case PDCA_JACOBI_PERTURBED:
        return p.delta0 > 0.0 ? PDCA_OK : PDCA_ERR_INFEASIBLE;
    default:
        return (p.delta0 > 0.0 && lambda > 0.0) ? PDCA_OK : PDCA_ERR_INFEASIBLE;
    }
}

// g_i = alpha a_i + beta_{Lambda_i} (a_i = 1 for L_s, d_i for L).
Coeffs make_coeffs(const pdca_params &p, double omega, double lambda) {
    const double c = c_eff(p), d0 = delta0_eff(p);
    double alpha, beta0;
    switch (p.precond) {
    case PDCA_JACOBI_DAMPED:
        alpha = p.eps / omega;
        beta0 = c / omega;
        break;
    case PDCA_JACOBI_PERTURBED:
        alpha = 2.0 * p.eps;
        beta0 = c + d0;
        break;
    default:
        alpha = 0.0;
        beta0 = p.eps * lambda + c + d0;
        break;
    }
    const double beta1 = beta0 + (p.precond == PDCA_JACOBI_DAMPED ? p.eta / omega : p.eta);
    Coeffs cf;
    cf.eps = (float)p.eps;
    cf.inv_eps = (float)(1.0 / p.eps);
    cf.c = (float)c;
    cf.eta = (float)p.eta;
    cf.inv_g0 = (float)(1.0 / (alpha + beta0));
    cf.inv_g1 = (float)(1.0 / (alpha + beta1));
    cf.alpha = (float)alpha;
    cf.beta0 = (float)beta0;
    cf.beta1 = (float)beta1;
    return cf;
}

// Host copy of row_ptr (copied from the device when it lives there) plus
// its structural checks.
pdca_status host_row_ptr(const int64_t *row_ptr, int32_t n, std::vector<int64_t> &keep,
                         const int64_t **view, int64_t *max_deg = nullptr) {
    if (!row_ptr || n < 1) return PDCA_ERR_INVALID_ARG;
    if (is_device_ptr(row_ptr)) {
        keep.resize((size_t)n + 1);
        if (cudaMemcpy(keep.data(), row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDefault) != cudaSuccess)
            return PDCA_ERR_CUDA;
        *view = keep.data();
    } else {
        *view = row_ptr;
    }
    const int64_t *rp = *view;
    if (rp[0] != 0) return PDCA_ERR_INVALID_ARG;
    // row lengths in range, and the largest, over chunks in parallel
    const int64_t chunk = 1 << 18, nch = ((int64_t)n + chunk - 1) / chunk;
    std::vector<int64_t> cmax((size_t)nch, 0);
    std::vector<uint8_t> cbad((size_t)nch, 0);
    host_parallel_for(nch, [&](int64_t c) {
        int64_t mx = 0;
        bool bad = false;
        for (int64_t i = c * chunk; i < std::min<int64_t>(n, (c + 1) * chunk); ++i) {
            const int64_t d = rp[i + 1] - rp[i];
            bad |= d < 0 || d >= (1 << 24);
            mx = d > mx ? d : mx;
        }
        cmax[(size_t)c] = mx;
        cbad[(size_t)c] = bad;
    });
    int64_t mx = 0;
    for (int64_t c = 0; c < nch; ++c) {
        if (cbad[(size_t)c]) return PDCA_ERR_INVALID_ARG;
        mx = std::max(mx, cmax[(size_t)c]);
    }
    if (max_deg) *max_deg = mx;
    return PDCA_OK;
}

// Split length T: a row longer than T keeps its first T entries in the
// sliced ELL and the rest in the overflow CSR, reduced one warp per row by a
// pre-pass.  A sweep waits for its longest row (one lane per row), so hub
// rows set its time on graphs whose rows are otherwise short.  Automatic
// choice: split only when some row is longer than max(256, t), with
// t = max(64, nnz / 200000) -- a row that a sweep over the whole graph
// would not hide -- and then at t.  Tiled kernels keep whole rows.
int32_t split_length(const pdca_params &p, int64_t nnz, int64_t max_deg) {
    if (p.tiling == PDCA_TILING_ON) return INT32_MAX;
    if (p.row_split > 0) return std::min<int32_t>(kSplitMax, (p.row_split + kVec - 1) / kVec * kVec);
    const int64_t t = std::max<int64_t>(64, (nnz / 200000 + kVec - 1) / kVec * kVec);
    if (max_deg > std::max<int64_t>(256, t)) return (int32_t)std::min<int64_t>(t, kSplitMax);
    return kSplitMax;
}

// The first regions of a problem's workspace: the create-time copies of the
// caller's CSR and fidelity data and the status words, at offsets that
// depend on n and nnz only, so that the copies can start before the host has
// checked the row offsets and worked out the layout.
struct StageHead {
    size_t o_srp, o_scol, o_sw, o_smask, o_slab, o_status, end;
};

StageHead stage_head(int32_t n, int64_t nnz) {
    StageHead S;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1)); return at; };
    S.o_srp = take(8 * ((size_t)n + 1));
    S.o_scol = take(4 * (size_t)nnz);
    S.o_sw = take(4 * (size_t)nnz);
    S.o_smask = take((size_t)n);
    S.o_slab = take(4 * (size_t)n);
    S.o_status = take(16);
    S.end = o;
    return S;
}

// The device renumbering pays off once the 65536-node chunks (serial work for
// one device block, or for one host thread) outnumber the host's threads by
// more than twice; the tiles' halo lists are built on the host.
bool use_device_order(const pdca_params &prm, int32_t n) {
    const int64_t chunks = ((int64_t)n + kBfsChunk - 1) / kBfsChunk;
    return prm.reorder == PDCA_REORDER_BFS && prm.tiling != PDCA_TILING_ON && chunks > 2 * (int64_t)host_workers();
}

pdca_status compute_layout(const int64_t *rp, int32_t n, int32_t K, const pdca_params &prm, int64_t max_deg,
                           Layout &L) {
    const int32_t sigma_req = prm.sort_window;
    L.n = n;
    L.K = K;
    L.nnz = rp[n];
    L.n_slices = (n + kSliceRows - 1) / kSliceRows;
    L.n_pad = L.n_slices * kSliceRows;
    L.n_tiles = (L.n_slices + kTileSlices - 1) / kTileSlices;
    L.split = split_length(prm, L.nnz, max_deg);
    if (max_deg > L.split) {
        const int64_t chunk = 1 << 18, nch = ((int64_t)n + chunk - 1) / chunk;
        std::vector<int64_t> cnt((size_t)nch, 0), ent((size_t)nch, 0);
        host_parallel_for(nch, [&](int64_t c) {
            for (int64_t i = c * chunk; i < std::min<int64_t>(n, (c + 1) * chunk); ++i) {
                const int64_t d = rp[i + 1] - rp[i];
                if (d > L.split) {
                    ++cnt[(size_t)c];
                    ent[(size_t)c] += d - L.split;
                }
            }
        });
        for (int64_t c = 0; c < nch; ++c) {
            L.n_ov += (int32_t)cnt[(size_t)c];
            L.ov_entries += ent[(size_t)c];
        }
    }
    std::vector<int64_t> widths;
    if (prm.reorder == PDCA_REORDER_BFS) {
        // the widths depend on the renumbering (computed at create); size for the bound
        L.host_order = true;
        L.device_order = use_device_order(prm, n);   // both forms give the same order
        L.sigma = sigma_req && sigma_req <= kBfsBlock ? sigma_req : kBfsBlock;
        L.sell_entries = 0;
        L.sell_cap = sell_bound(rp, n, L.sigma, max_deg);
        L.halo_cap = std::max<int64_t>(L.nnz, 1);
    } else if (sigma_req) {
        L.sigma = sigma_req;
        L.sell_entries = sell_entries_for(rp, n, L.sigma, L.split, widths);
    } else {
        // smallest window (from 128 rows up) whose slice padding is <= 10%
        for (int s = 128;; s <<= 1) {
            L.sigma = s;
            L.sell_entries = sell_entries_for(rp, n, s, L.split, widths);
            if (s >= 8192 || (double)L.sell_entries <= kPadTarget * (double)std::max<int64_t>(L.nnz, 1)) break;
        }
    }
    if (!L.host_order) {
        L.sell_cap = L.sell_entries;
        L.halo_cap = 1;
        L.slice_off.assign((size_t)L.n_slices + 1, 0);
        for (int32_t s = 0; s < L.n_slices; ++s) L.slice_off[s + 1] = L.slice_off[s] + widths[s] * kSliceRows;
    }

    const size_t P = (size_t)L.sell_cap, np = (size_t)L.n_pad, nn = (size_t)n;
    const size_t parts = (size_t)std::max(1, energy_blocks(L.n_slices)) * kRedSlots;
    const StageHead S = stage_head(n, L.nnz);
    L.o_srp = S.o_srp;
    L.o_scol = S.o_scol;
    L.o_sw = S.o_sw;
    L.o_smask = S.o_smask;
    L.o_slab = S.o_slab;
    L.o_status = S.o_status;
    size_t o = S.end;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1)); return at; };
    const bool mixed = prm.precision != PDCA_FP32;
    L.o_col = take(4 * P);
    L.o_col16 = take(prm.columns == PDCA_COLUMNS_AUTO ? 2 * P : 0);
    L.o_fmt = take((size_t)L.n_slices);
    L.o_w = take(4 * P);
    L.o_wb = take(mixed ? 2 * P : 0);
    L.o_slice = take(8 * ((size_t)L.n_slices + 1));
    L.o_rowinfo = take(4 * np);
    L.o_perm = take(4 * np);
    L.o_iperm = take(4 * nn);
    L.o_self = take(prm.laplacian == PDCA_LAP_UNNORMALIZED ? 4 * np : 0);
    L.o_dsq = take(prm.laplacian == PDCA_LAP_NORMALIZED ? 4 * np : 0);
    for (int b = 0; b < 3; ++b) L.o_u[b] = take(4 * np * (size_t)K);
    L.o_part = take(8 * parts);
    L.o_red = take(sizeof(RedOut));
    L.o_scal = take(8 * 8);
    L.o_trace = take(8 * 2 * (size_t)kTraceCap);
    L.o_hoff = take(8 * ((size_t)L.n_tiles + 1));
    L.o_hidx = take(4 * (size_t)L.halo_cap);
    const size_t nov = (size_t)L.n_ov, eov = (size_t)L.ov_entries;
    L.o_ovrp = take(nov ? 8 * (nov + 1) : 0);
    L.o_ovcol = take(4 * eov);
    L.o_ovw = take(4 * eov);
    L.o_ovwb = take(mixed ? 2 * eov : 0);
    L.o_ovidx = take(nov ? 4 * np : 0);
    L.o_ovacc = take(4 * nov * (size_t)std::max(K, 4));
    const size_t half_rows = mixed ? 2 * np * (size_t)K : 0;
    L.o_mr = take(mixed ? 4 * np * (size_t)K : 0);
    L.o_me[0] = take(half_rows);
    L.o_me[1] = take(half_rows);
    // the rest of the create-time staging
    L.o_sdeg = take(8 * nn);
    L.o_sisd = take(8 * nn);
    L.o_scls = take(4 * np);
    L.o_sscan = take(L.host_order ? 8 * (size_t)order_layout_scan_words(L.n_slices) : 0);
    L.o_skey = take(L.device_order ? 8 * nn : 0);
    L.o_sbfs = take(L.device_order ? 16 : 0);
    L.total = o;
    return PDCA_OK;
}

}  // namespace

namespace pdca {
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace pdca

struct pdca_problem {
    Layout L;
    pdca_params prm;
    double omega = 0.5;
    double lambda_used = 0.0, lambda_est = 0.0;
    double dmax = 0.0;         // largest degree
    float *self = nullptr;     // a_i = d_i per row (unnormalized L), else nullptr
    float *dsq = nullptr;      // sqrt(d_i) per row (normalized L_s: its null vector), else nullptr
    Coeffs cf;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    int32_t *sell_col = nullptr;
    uint16_t *col16 = nullptr;        // 16-bit columns (PDCA_COLUMNS_AUTO), else nullptr
    uint8_t *slice_fmt = nullptr;     // kFmt32 / kFmt16 per slice (with col16)
    int64_t slices16 = 0;             // slices stored with 16-bit columns
    float *sell_w = nullptr;          // FP32 weights (both precisions)
    __nv_bfloat16 *sell_wb = nullptr; // BF16 weights (mixed precision)
    OverflowView ov{};                // entries of the rows longer than the split length
    int32_t *ov_index = nullptr;      // overflow row of every split row (n_pad), or nullptr
    float *ov_acc = nullptr;          // the pre-pass sums (max(K, 4) floats per overflow row)
    int64_t *slice_off = nullptr;
    uint32_t *rowinfo = nullptr;
    int32_t *perm = nullptr, *iperm = nullptr;
    float *U[3] = {nullptr, nullptr, nullptr};
    double *partials = nullptr;
    RedOut *red = nullptr;
    double *scal = nullptr;    // [0] power scale, [1] power lambda
    double *trace = nullptr;   // [0, cap) energy, [cap, 2 cap) residual
    int cur = 0, prev = 1;
    bool has_prev = false;
    bool prof = false;
    bool tiled = false;
    bool slice_off_on_device = false;   // slice_off computed by the device renumbering
    uint32_t *fid_status = nullptr;     // fidelity check left on the device (pdca_create_like_async)
    TileView tv{};
    int64_t halo_rows = 0;
    bool mixed = false, bf16u = false;
    void *mr = nullptr, *me[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    // pdca_solve replay cache (pdca_graph_enable): one instantiated CUDA graph
    // per (outer, inner, starting buffers, coefficients)
    struct SolveGraph {
        int32_t outer, inner, cur, prev;
        bool has_prev;
        Coeffs cf;
        int end_cur, end_prev;
        uint64_t launches;
        cudaGraphExec_t exec;
    };
    bool graphs_on = false;
    std::vector<SolveGraph> graphs;
    void drop_graphs() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }

    SellView view() const {
        SellView A;
        A.col = sell_col;
        A.col16 = col16;
        A.slice_fmt = col16 ? slice_fmt : nullptr;
        A.w = sell_w;
        A.wb = mixed ? sell_wb : nullptr;
        A.slice_off = slice_off;
        A.rowinfo = rowinfo;
        A.self = self;
        A.ov_index = ov_index;
        A.ov_acc = ov_acc;
        A.n_slices = L.n_slices;
        A.n = L.n;
        // three n_pad x K FP32 iterates above half of the 129 MB L2
        A.stream_rows = 3.0 * 4.0 * (double)L.n_pad * (double)L.K > 64.0 * (1 << 20) ? 1 : 0;
        A.block_iters = prm.block_slices / kWarpsPerBlock;   // 0: automatic
        return A;
    }
    int spare() const { return has_prev ? 3 - cur - prev : (cur + 1) % 3; }
    const TileView *tiles() const { return tiled ? &tv : nullptr; }
};

namespace {

pdca_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PDCA_OK : PDCA_ERR_CUDA; }

#define PDCA_TRY(expr)                         \
    do {                                       \
        cudaError_t _e = (expr);               \
        if (_e != cudaSuccess) return PDCA_ERR_CUDA; \
    } while (0)

// Launch one sweep-like pass; with profiling on, bracket it with events.
template <class F>
pdca_status timed_pass(pdca_problem *h, F launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (h->prof) {
        while (h->ev.size() < h->ev_used + 2) {
            cudaEvent_t e;
            PDCA_TRY(cudaEventCreate(&e));
            h->ev.push_back(e);
        }
        a = h->ev[h->ev_used];
        b = h->ev[h->ev_used + 1];
        h->ev_used += 2;
        PDCA_TRY(cudaEventRecord(a, h->stream));
    }
    PDCA_TRY(launch());
    if (h->prof) PDCA_TRY(cudaEventRecord(b, h->stream));
    return PDCA_OK;
}

// The overflow pre-pass of the row sums over x (K columns; weights and row
// storage as given) into the handle's ov_acc; nothing without split rows.
cudaError_t overflow_pass(pdca_problem *h, int K, int wkind, int xkind, const void *x) {
    if (h->ov.n_rows <= 0) return cudaSuccess;
    return launch_overflow(K, wkind, xkind, h->ov, x, h->ov_acc, h->stream);
}

pdca_status sweep(pdca_problem *h, bool project, const float *src, const float *ut, float *dst) {
    return timed_pass(h, [&] {
        cudaError_t e = overflow_pass(h, h->L.K, kOvW32, kOvX32, src);
        if (e != cudaSuccess) return e;
        return launch_sweep(h->L.K, project, h->view(), h->tiles(), h->cf, src, ut, dst, h->stream);
    });
}

// Mixed-precision outer step: pass 0 forms r = b^t - T u^t and e^1 in FP32,
// the following passes update the 16-bit correction, the last one writes
// u^{t+1} = u^t + e^m in FP32 (projected for K >= 2).
pdca_status outer_step_mixed(pdca_problem *h, int32_t inner) {
    const int K = h->L.K;
    const SellView A = h->view();
    const int dst = (h->cur + 1) % 3;
    const float *u = h->U[h->cur];
    float *u_out = h->U[dst];
    const bool proj = K >= 2;
    const int xkind = h->bf16u ? kOvXBf16 : kOvXHalf;
    pdca_status st = timed_pass(h, [&] {
        cudaError_t e = overflow_pass(h, K, kOvW32, kOvX32, u);
        if (e != cudaSuccess) return e;
        return launch_mixed_residual(K, h->bf16u, inner == 1, proj, A, h->cf, u, h->mr, h->me[0], u_out, h->stream);
    });
    if (st != PDCA_OK) return st;
    for (int32_t s = 1; s < inner; ++s) {
        const bool last = s == inner - 1;
        void *src = h->me[(s - 1) % 2], *dstb = h->me[s % 2];
        st = timed_pass(h, [&] {
            cudaError_t e = overflow_pass(h, K, kOvW16, xkind, src);
            if (e != cudaSuccess) return e;
            return launch_mixed_sweep(K, h->bf16u, last, proj, A, h->cf, src, h->mr, dstb, u, u_out, h->stream);
        });
        if (st != PDCA_OK) return st;
    }
    h->prev = h->cur;
    h->cur = dst;
    h->has_prev = true;
    return PDCA_OK;
}

// One outer step (Prop. nopre): sweeps ping-pong between the two buffers
// that do not hold u^t; the last one projects rows for K >= 2.
pdca_status outer_step(pdca_problem *h, int32_t inner) {
    if (h->mixed) return outer_step_mixed(h, inner);
    const int a = (h->cur + 1) % 3, b = (h->cur + 2) % 3;
    const float *ut = h->U[h->cur];
    const float *src = ut;
    int last = h->cur;
    for (int32_t s = 0; s < inner; ++s) {
        const int dst = (s % 2 == 0) ? a : b;
        const bool project = (h->L.K >= 2) && (s == inner - 1);
        pdca_status st = sweep(h, project, src, ut, h->U[dst]);
        if (st != PDCA_OK) return st;
        src = h->U[dst];
        last = dst;
    }
    h->prev = h->cur;
    h->cur = last;
    h->has_prev = true;
    return PDCA_OK;
}

pdca_status reduce_energy(pdca_problem *h, double *trace_F, double *trace_r) {
    const SellView A = h->view();
    PDCA_TRY(overflow_pass(h, h->L.K, kOvW32, kOvX32, h->U[h->cur]));
    PDCA_TRY(launch_energy(h->L.K, A, h->tiles(), h->cf, h->U[h->cur], h->has_prev ? h->U[h->prev] : nullptr,
                           h->partials, h->stream));
    PDCA_TRY(launch_energy_finalize(h->partials, reduce_parts(A, h->tiles()), h->prm.eps, h->prm.eta,
                                    h->has_prev ? 1 : 0, h->red, trace_F, trace_r, h->stream));
    return PDCA_OK;
}

// Upper bound of lambda_max (Prop. diagonal:pre): 2 for L_s, 2 d_max for L.
double lambda_bound(const pdca_problem *h) {
    return h->prm.laplacian == PDCA_LAP_UNNORMALIZED ? 2.0 * h->dmax : 2.0;
}

// Enqueue the power method on stream st over the operator view A (tiles T);
// the estimate lands in scal[1].
pdca_status power_launch(pdca_problem *h, const SellView &A, const TileView *T, cudaStream_t st) {
    float *x = h->U[1], *y = h->U[2];
    double *scale = h->scal, *lam = h->scal + 1;
    unsigned *ticket = reinterpret_cast<unsigned *>(h->scal + 2);
    PDCA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
    PDCA_TRY(launch_power_init(A, h->perm, x, h->partials, st));
    PDCA_TRY(launch_power_finalize(h->partials, energy_blocks(A.n_slices), scale, lam, st));
    for (int it = 0; it <= h->prm.power_iters; ++it) {
        // the SpMV's last block reduces the partials and updates scale / lambda
        if (h->ov.n_rows > 0) PDCA_TRY(launch_overflow(1, kOvW32, kOvX32, h->ov, x, h->ov_acc, st));
        PDCA_TRY(launch_power_spmv(A, T, x, scale, y, h->partials, ticket, lam, st));
        std::swap(x, y);
    }
    return PDCA_OK;
}

// The estimate, once the power method's work on st is done.
pdca_status power_read(pdca_problem *h, cudaStream_t st) {
    double lam_h = 0.0;
    PDCA_TRY(cudaMemcpyAsync(&lam_h, h->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    PDCA_TRY(cudaStreamSynchronize(st));
    h->lambda_est = lam_h;
    h->lambda_used = std::min(lambda_bound(h), 1.001 * lam_h);
    return PDCA_OK;
}

pdca_status power_method(pdca_problem *h) {
    pdca_status st = power_launch(h, h->view(), h->tiles(), h->stream);
    return st != PDCA_OK ? st : power_read(h, h->stream);
}

// A stream of its own for work that overlaps the caller's stream at create
// time; synchronised and released on scope exit (also on the error paths,
// before the caller may reuse the workspace).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t in = nullptr, out = nullptr;
    ~SideStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        if (in) cudaEventDestroy(in);
        if (out) cudaEventDestroy(out);
    }
    cudaError_t open() {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out, cudaEventDisableTiming);
        return e;
    }
};

// Host symbolic analysis (BFS-block renumbering, degree sort, halo lists),
// then upload of perm / iperm / halo arrays and the exact slice offsets.
// The renumbering order of BFS mode, computed on a host thread while the
// device copies and validates the graph (the BFS reads only columns inside
// its own chunk, so an invalid column cannot make it read out of bounds; the
// order is used only once validation has passed).
struct OrderJob {
    std::vector<int32_t> col_keep, order;
    const int32_t *hc = nullptr;
    std::thread th;
    pdca_status st = PDCA_OK;
    ~OrderJob() {
        if (th.joinable()) th.join();
    }
    pdca_status start(const int64_t *rp, const int32_t *col, int64_t nnz, int32_t n, int32_t sigma) {
        hc = col;
        if (nnz > 0 && is_device_ptr(col)) {
            col_keep.resize((size_t)nnz);
            if (cudaMemcpy(col_keep.data(), col, 4 * (size_t)nnz, cudaMemcpyDefault) != cudaSuccess)
                return PDCA_ERR_CUDA;
            hc = col_keep.data();
        }
        order.resize((size_t)n);
        th = std::thread([this, rp, n, sigma] { locality_order(n, rp, hc, kBfsBlock, kBfsChunk, sigma, order.data()); });
        return PDCA_OK;
    }
    void join() {
        if (th.joinable()) th.join();
    }
};

// The overflow CSR's row offsets (rows longer than the split length, in new
// row order) and the overflow row of every such row, uploaded; the pack
// kernel fills the columns and weights.  perm: new row -> old row for the
// first `rows` rows (-1 on padding); the rows after them are padding.
pdca_status build_overflow(pdca_problem *h, const int64_t *rp, const int32_t *perm, int32_t rows) {
    Layout &L = h->L;
    if (L.n_ov == 0) return PDCA_OK;
    std::vector<int64_t> orp((size_t)L.n_ov + 1, 0);
    std::vector<int32_t> idx((size_t)L.n_pad, -1);
    int32_t q = 0;
    for (int32_t r = 0; r < rows; ++r) {
        const int32_t old = perm[r];
        if (old < 0) continue;
        const int64_t d = rp[old + 1] - rp[old];
        if (d <= L.split) continue;
        if (q >= L.n_ov) return PDCA_ERR_CUDA;   // the counts are a theorem; never expected
        idx[(size_t)r] = q;
        orp[(size_t)q + 1] = orp[(size_t)q] + (d - L.split);
        ++q;
    }
    if (q != L.n_ov || orp.back() != L.ov_entries) return PDCA_ERR_CUDA;
    int64_t *d_rp = reinterpret_cast<int64_t *>(h->ws + L.o_ovrp);
    PDCA_TRY(cudaMemcpyAsync(d_rp, orp.data(), 8 * orp.size(), cudaMemcpyHostToDevice, h->stream));
    PDCA_TRY(cudaMemcpyAsync(h->ov_index, idx.data(), 4 * idx.size(), cudaMemcpyHostToDevice, h->stream));
    // the copies read host vectors that go out of scope
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    return PDCA_OK;
}

// The device's BFS-block order of the nodes into iperm's storage, enqueued
// on st (structure only: it reads row_ptr, already checked on the host, and
// skips columns outside [0, n), so it may run beside the validation).
cudaError_t device_order_launch(pdca_problem *h, cudaStream_t st) {
    Layout &L = h->L;
    const int64_t *d_rp = reinterpret_cast<const int64_t *>(h->ws + L.o_srp);
    const int32_t *d_col = reinterpret_cast<const int32_t *>(h->ws + L.o_scol);
    int32_t *queue = reinterpret_cast<int32_t *>(h->ws + L.o_scls);   // rowcls later
    unsigned long long *key = reinterpret_cast<unsigned long long *>(h->ws + L.o_skey);
    uint32_t *err = reinterpret_cast<uint32_t *>(h->ws + L.o_sbfs);
    cudaError_t e = cudaMemsetAsync(err, 0, 4, st);
    if (e != cudaSuccess) return e;
    return launch_bfs_blocks(L.n, kBfsBlock, kBfsChunk, d_rp, d_col, queue, key, h->iperm, err, st);
}

// The renumbering (perm, iperm, slice offsets) from that order, on the
// handle's stream (which must follow the order's work): degree sort, perm,
// iperm and offsets on the device; the entry total, and the order where
// rows overflow, come back to the host.
pdca_status device_renumber(pdca_problem *h, const int64_t *rp) {
    Layout &L = h->L;
    const int32_t n = L.n;
    cudaStream_t st = h->stream;
    const int64_t *d_rp = reinterpret_cast<const int64_t *>(h->ws + L.o_srp);
    uint32_t *err = reinterpret_cast<uint32_t *>(h->ws + L.o_sbfs);
    int32_t *count = reinterpret_cast<int32_t *>(h->ws + L.o_scls);
    int64_t *tmp = reinterpret_cast<int64_t *>(h->ws + L.o_sscan);
    uint32_t err_h = 0;
    PDCA_TRY(cudaMemcpyAsync(&err_h, err, 4, cudaMemcpyDeviceToHost, st));
    PDCA_TRY(cudaStreamSynchronize(st));
    if (err_h) return PDCA_ERR_CUDA;   // the order is not a permutation; never expected
    PDCA_TRY(launch_order_sort(n, L.sigma, d_rp, h->iperm, h->perm, st));
    PDCA_TRY(launch_order_layout(n, L.n_pad, L.split, d_rp, h->perm, h->iperm, count, tmp, h->slice_off, st));
    int64_t entries = 0;   // the offsets stay on the device; their total comes back
    PDCA_TRY(cudaMemcpyAsync(&entries, h->slice_off + L.n_slices, 8, cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> perm_h(L.n_ov > 0 ? (size_t)n : 0);
    if (L.n_ov > 0) PDCA_TRY(cudaMemcpyAsync(perm_h.data(), h->perm, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
    PDCA_TRY(cudaStreamSynchronize(st));
    L.sell_entries = entries;
    if (L.sell_entries > L.sell_cap) return PDCA_ERR_CUDA;   // the bound is a theorem; never expected
    h->slice_off_on_device = true;
    return build_overflow(h, rp, perm_h.data(), L.n_ov > 0 ? n : 0);
}

pdca_status host_renumber(pdca_problem *h, const int64_t *rp, OrderJob &job) {
    Layout &L = h->L;
    const int32_t n = L.n;
    job.join();
    const int32_t *hc = job.hc;
    const std::vector<int32_t> &order = job.order;
    h->tiled = false;
    std::vector<int32_t> perm((size_t)L.n_pad, -1), iperm((size_t)n);
    const int64_t chunks = ((int64_t)n + 65535) / 65536;
    host_parallel_for(chunks, [&](int64_t c) {
        const int32_t r0 = (int32_t)(c * 65536), r1 = (int32_t)std::min<int64_t>(n, (c + 1) * 65536);
        for (int32_t r = r0; r < r1; ++r) {
            perm[(size_t)r] = order[(size_t)r];
            iperm[(size_t)order[(size_t)r]] = r;
        }
    });
    std::vector<int64_t> width((size_t)L.n_slices, 0);
    const int64_t schunks = ((int64_t)L.n_slices + 2047) / 2048;
    host_parallel_for(schunks, [&](int64_t c) {
        const int32_t s0 = (int32_t)(c * 2048), s1 = (int32_t)std::min<int64_t>(L.n_slices, (c + 1) * 2048);
        for (int32_t s = s0; s < s1; ++s) {
            int64_t wmax = 0;
            for (int32_t l = 0; l < kSliceRows; ++l) {
                const int32_t r = s * kSliceRows + l;
                if (r < n)
                    wmax = std::max<int64_t>(wmax, std::min<int64_t>(rp[perm[(size_t)r] + 1] - rp[perm[(size_t)r]],
                                                                     L.split));
            }
            width[(size_t)s] = (wmax + kVec - 1) / kVec * kVec;
        }
    });
    L.slice_off.assign((size_t)L.n_slices + 1, 0);
    for (int32_t s = 0; s < L.n_slices; ++s)
        L.slice_off[(size_t)s + 1] = L.slice_off[(size_t)s] + width[(size_t)s] * kSliceRows;
    L.sell_entries = L.slice_off.back();
    if (L.sell_entries > L.sell_cap) return PDCA_ERR_CUDA;   // the bound is a theorem; never expected
    // PDCA_TILING_ON (on every workload measured on GB300 the plain kernels
    // were faster than the shared-memory tiles, so AUTO uses the plain ones):
    // the tiles' halo lists on the host
    if (h->prm.tiling == PDCA_TILING_ON) {
        std::vector<int64_t> hoff;
        std::vector<int32_t> hidx;
        int32_t mx = 0;
        tile_halos(n, kTileRows, rp, hc, perm.data(), iperm.data(), hoff, hidx, &mx);
        // rows staged per block: the whole largest halo if it fits the budget,
        // else the budget (tiles above it gather through their halo list)
        const int32_t cap_rows = (int32_t)std::min<size_t>(65536, kTileSmemBudget / (sizeof(float) * L.K));
        const int32_t smem_rows = std::min(mx, cap_rows);
        int64_t over = 0;
        for (size_t t = 0; t + 1 < hoff.size(); ++t) over += (hoff[t + 1] - hoff[t]) > smem_rows ? 1 : 0;
        // tiles whose halo exceeds the staged rows take the halo-list path
        (void)over;
        const bool fits = mx >= 1 && mx <= 65536 && (int64_t)hidx.size() <= L.halo_cap &&
                          (int32_t)hoff.size() == L.n_tiles + 1;
        if (!fits) return PDCA_ERR_INVALID_ARG;
        if (fits) {
            int64_t *d_hoff = reinterpret_cast<int64_t *>(h->ws + L.o_hoff);
            int32_t *d_hidx = reinterpret_cast<int32_t *>(h->ws + L.o_hidx);
            PDCA_TRY(cudaMemcpyAsync(d_hoff, hoff.data(), 8 * hoff.size(), cudaMemcpyHostToDevice, h->stream));
            if (!hidx.empty())
                PDCA_TRY(cudaMemcpyAsync(d_hidx, hidx.data(), 4 * hidx.size(), cudaMemcpyHostToDevice, h->stream));
            h->tv.halo_off = d_hoff;
            h->tv.halo_idx = d_hidx;
            h->tv.lcol = reinterpret_cast<const uint16_t *>(h->sell_col);
            h->tv.n_tiles = L.n_tiles;
            h->tv.max_halo = mx;
            h->tv.smem_rows = smem_rows;
            h->halo_rows = (int64_t)hidx.size();
            h->tiled = true;
            // the copies above read host vectors that go out of scope
            PDCA_TRY(cudaStreamSynchronize(h->stream));
        }
    }
    PDCA_TRY(cudaMemcpyAsync(h->perm, perm.data(), 4 * perm.size(), cudaMemcpyHostToDevice, h->stream));
    PDCA_TRY(cudaMemcpyAsync(h->iperm, iperm.data(), 4 * iperm.size(), cudaMemcpyHostToDevice, h->stream));
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    return build_overflow(h, rp, perm.data(), L.n_pad);
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct BatchMember {
    pdca_problem *h;
    int32_t outer_left;
    int32_t inner;
    int32_t pass;   // pass index inside the current outer step
};

// Descriptor of member m's next pass (mirrors outer_step / outer_step_mixed).
void member_desc(const BatchMember &m, BatchDesc &d) {
    pdca_problem *h = m.h;
    const int K = h->L.K;
    d.A = h->view();
    d.cf = h->cf;
    d.last = m.pass == m.inner - 1;
    d.project = d.last && K >= 2;
    d.bf16u = h->bf16u ? 1 : 0;
    d.pad_ = 0;
    d.dst2 = nullptr;
    d.u = nullptr;
    d.u_out = nullptr;
    if (!h->mixed) {
        const int a = (h->cur + 1) % 3, b = (h->cur + 2) % 3;
        const int s = m.pass;
        d.kind = kPassFp32;
        d.src = s == 0 ? h->U[h->cur] : h->U[((s - 1) % 2 == 0) ? a : b];
        d.aux = h->U[h->cur];
        d.dst = h->U[(s % 2 == 0) ? a : b];
    } else {
        const int dst = (h->cur + 1) % 3;
        d.u_out = h->U[dst];
        if (m.pass == 0) {
            d.kind = kPassMixedResidual;
            d.src = h->U[h->cur];
            d.aux = nullptr;
            d.dst = h->mr;
            d.dst2 = h->me[0];
        } else {
            d.kind = kPassMixedSweep;
            d.src = h->me[(m.pass - 1) % 2];
            d.aux = h->mr;
            d.dst = h->me[m.pass % 2];
            d.u = h->U[h->cur];
        }
    }
}

// Host state after the pass was enqueued; true when the member finished.
bool member_advance(BatchMember &m) {
    pdca_problem *h = m.h;
    if (m.pass < m.inner - 1) {
        ++m.pass;
        return false;
    }
    int next;
    if (!h->mixed) {
        const int a = (h->cur + 1) % 3, b = (h->cur + 2) % 3;
        next = ((m.inner - 1) % 2 == 0) ? a : b;
    } else {
        next = (h->cur + 1) % 3;
    }
    h->prev = h->cur;
    h->cur = next;
    h->has_prev = true;
    m.pass = 0;
    return --m.outer_left == 0;
}

// Workspace of a problem that borrows another problem's operator: only the
// per-problem state (tags, iterates, reductions, mixed buffers, fidelity
// staging).
struct CloneLayout {
    size_t o_rowinfo, o_u[3], o_part, o_red, o_scal, o_trace, o_mr, o_me[2], o_ovacc, o_smask, o_slab, o_status,
        total;
};

CloneLayout clone_layout(const Layout &L, int32_t K, int32_t precision) {
    CloneLayout C;
    const size_t np = (size_t)L.n_pad, nn = (size_t)L.n;
    const size_t parts = (size_t)std::max(1, energy_blocks(L.n_slices)) * kRedSlots;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1)); return at; };
    C.o_rowinfo = take(4 * np);
    for (int b = 0; b < 3; ++b) C.o_u[b] = take(4 * np * (size_t)K);
    C.o_part = take(8 * parts);
    C.o_red = take(sizeof(RedOut));
    C.o_scal = take(8 * 8);
    C.o_trace = take(8 * 2 * (size_t)kTraceCap);
    const size_t half_rows = precision == PDCA_FP32 ? 0 : 2 * np * (size_t)K;
    C.o_mr = take(precision == PDCA_FP32 ? 0 : 4 * np * (size_t)K);
    C.o_me[0] = take(half_rows);
    C.o_me[1] = take(half_rows);
    C.o_ovacc = take(4 * (size_t)L.n_ov * (size_t)std::max(K, 4));
    C.o_smask = take(nn);
    C.o_slab = take(4 * nn);
    C.o_status = take(16);
    C.total = o;
    return C;
}

}  // namespace

struct pdca_batch {
    cudaStream_t stream = nullptr;
    int32_t max_problems = 0;
    std::vector<BatchMember> members;
    std::vector<pdca_problem *> done;
    BatchTable table;
    BatchOvTable ov_table;
};

extern "C" {

void pdca_default_params(pdca_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps = 1.0;
    p->c = 3.0;
    p->eta = 1.0;
    p->laplacian = PDCA_LAP_NORMALIZED;
    p->precond = PDCA_JACOBI_PERTURBED;
    p->damping = 0.5;
    p->delta0 = 1e-6;
    p->lambda_max = 0.0;
    p->power_iters = 150;
    p->precision = PDCA_FP32;
    p->sort_window = 0;
    p->reorder = PDCA_REORDER_BFS;
    p->tiling = PDCA_TILING_AUTO;
    p->entry_order = PDCA_ENTRIES_SPREAD;
    p->step_k = 0.0;
    p->columns = PDCA_COLUMNS_AUTO;
    p->row_split = 0;
    p->block_slices = 0;
}

const char *pdca_status_string(pdca_status s) {
    switch (s) {
    case PDCA_OK: return "ok";
    case PDCA_ERR_INVALID_ARG: return "invalid argument";
    case PDCA_ERR_NOT_SYMMETRIC: return "weight matrix is not symmetric";
    case PDCA_ERR_ISOLATED_NODE: return "isolated node (degree not > 0)";
    case PDCA_ERR_INFEASIBLE: return "preconditioner is not feasible (G > T fails)";
    case PDCA_ERR_NONFINITE: return "non-finite value in the iterate";
    case PDCA_ERR_OOM: return "workspace too small";
    case PDCA_ERR_CUDA: return "CUDA runtime error";
    case PDCA_ERR_TIMEOUT: return "reserved (no call waits on the device)";
    case PDCA_ERR_BAD_GRAPH: return "malformed graph or fidelity input";
    case PDCA_ERR_TOO_LARGE: return "graph larger than the fixed scratch of pdca_energy_static";
    case PDCA_ERR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
    }
    return "unknown status";
}

uint64_t pdca_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

pdca_status pdca_workspace_size(const int64_t *row_ptr, int32_t n, int32_t k, const pdca_params *p,
                                size_t *bytes) {
    if (!bytes || k < 1 || k > PDCA_MAX_K || n < 1) return PDCA_ERR_INVALID_ARG;
    pdca_params prm;
    pdca_default_params(&prm);
    if (p) prm = *p;
    pdca_status st = check_params(prm);
    if (st != PDCA_OK) return st;
    std::vector<int64_t> keep;
    const int64_t *rp = nullptr;
    int64_t max_deg = 0;
    st = host_row_ptr(row_ptr, n, keep, &rp, &max_deg);
    if (st != PDCA_OK) return st;
    Layout L;
    st = compute_layout(rp, n, k, prm, max_deg, L);
    if (st != PDCA_OK) return st;
    *bytes = L.total;
    return PDCA_OK;
}

pdca_status pdca_create(const int64_t *row_ptr, const int32_t *col, const float *w, int32_t n, int32_t k,
                        const uint8_t *fid_mask, const int32_t *labels, const pdca_params *p,
                        void *workspace, size_t ws_bytes, void *stream, pdca_problem **out) {
    if (!out) return PDCA_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 1 || k > PDCA_MAX_K || n < 1 || !fid_mask || !labels || !workspace) return PDCA_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PDCA_ERR_INVALID_ARG;
    pdca_params prm;
    pdca_default_params(&prm);
    if (p) prm = *p;
    pdca_status st = check_params(prm);
    if (st != PDCA_OK) return st;
    const double omega = prm.damping;
    if (prm.laplacian == PDCA_LAP_NORMALIZED && (prm.precond != PDCA_RICHARDSON || prm.lambda_max > 0)) {
        st = feasible(prm, omega, prm.lambda_max, 1.0);
        if (st != PDCA_OK) return st;
    }
    // With the row offsets in host memory, the copies of the CSR and
    // fidelity data start first, to fixed workspace offsets, and the host's
    // checks and layout work overlap them (the device renumbering waits for
    // the columns only).  Every return after this point first waits for the
    // copies, which read the caller's buffers.
    cudaStream_t sm0 = static_cast<cudaStream_t>(stream);
    SideStream order_side;
    bool early = false, order_ready = false;
    if (!is_device_ptr(row_ptr)) {
        const int64_t nnz0 = row_ptr[n];
        const StageHead S = stage_head(n, std::max<int64_t>(nnz0, 0));
        if (row_ptr[0] == 0 && nnz0 >= 0 && nnz0 < ((int64_t)1 << 40) && (nnz0 == 0 || (col && w)) &&
            ws_bytes >= S.end) {
            char *W0 = static_cast<char *>(workspace);
            auto cp0 = [&](size_t at, const void *src, size_t bytes) {
                return bytes ? cudaMemcpyAsync(W0 + at, src, bytes, cudaMemcpyDefault, sm0) : cudaSuccess;
            };
            early = true;
            cudaError_t e = cp0(S.o_srp, row_ptr, 8 * ((size_t)n + 1));
            if (e == cudaSuccess) e = cp0(S.o_scol, col, 4 * (size_t)nnz0);
            if (e == cudaSuccess && use_device_order(prm, n)) {
                e = order_side.open();
                if (e == cudaSuccess) e = cudaEventRecord(order_side.in, sm0);
                order_ready = e == cudaSuccess;
            }
            if (e == cudaSuccess) e = cp0(S.o_sw, w, 4 * (size_t)nnz0);
            if (e == cudaSuccess) e = cp0(S.o_smask, fid_mask, (size_t)n);
            if (e == cudaSuccess) e = cp0(S.o_slab, labels, 4 * (size_t)n);
            if (e == cudaSuccess) e = cudaMemsetAsync(W0 + S.o_status, 0, 16, sm0);
            if (e != cudaSuccess) {
                cudaStreamSynchronize(sm0);
                return PDCA_ERR_CUDA;
            }
        }
    }
    auto early_fail = [&](pdca_status s2) {
        if (early) cudaStreamSynchronize(sm0);
        return s2;
    };
    std::vector<int64_t> keep;
    const int64_t *rp = nullptr;
    int64_t max_deg = 0;
    st = host_row_ptr(row_ptr, n, keep, &rp, &max_deg);
    if (st != PDCA_OK) return early_fail(st);
    const int64_t nnz = rp[n];
    if (nnz > 0 && (!col || !w)) return early_fail(PDCA_ERR_INVALID_ARG);

    pdca_problem *h = new (std::nothrow) pdca_problem();
    if (!h) return early_fail(PDCA_ERR_INVALID_ARG);
    st = compute_layout(rp, n, k, prm, max_deg, h->L);
    if (st != PDCA_OK) { delete h; return early_fail(st); }
    if (ws_bytes < h->L.total) { delete h; return early_fail(PDCA_ERR_OOM); }
    h->prm = prm;
    h->omega = omega;
    h->stream = static_cast<cudaStream_t>(stream);
    h->ws = static_cast<char *>(workspace);
    const Layout &L = h->L;
    char *W = h->ws;
    h->sell_col = reinterpret_cast<int32_t *>(W + L.o_col);
    h->sell_w = reinterpret_cast<float *>(W + L.o_w);
    h->sell_wb = prm.precision != PDCA_FP32 ? reinterpret_cast<__nv_bfloat16 *>(W + L.o_wb) : nullptr;
    h->slice_fmt = reinterpret_cast<uint8_t *>(W + L.o_fmt);
    h->slice_off = reinterpret_cast<int64_t *>(W + L.o_slice);
    h->rowinfo = reinterpret_cast<uint32_t *>(W + L.o_rowinfo);
    h->perm = reinterpret_cast<int32_t *>(W + L.o_perm);
    h->iperm = reinterpret_cast<int32_t *>(W + L.o_iperm);
    h->self = prm.laplacian == PDCA_LAP_UNNORMALIZED ? reinterpret_cast<float *>(W + L.o_self) : nullptr;
    h->dsq = prm.laplacian == PDCA_LAP_NORMALIZED ? reinterpret_cast<float *>(W + L.o_dsq) : nullptr;
    for (int b = 0; b < 3; ++b) h->U[b] = reinterpret_cast<float *>(W + L.o_u[b]);
    if (L.n_ov > 0) {
        h->ov.rp = reinterpret_cast<const int64_t *>(W + L.o_ovrp);
        h->ov.col = reinterpret_cast<const int32_t *>(W + L.o_ovcol);
        h->ov.w = reinterpret_cast<const float *>(W + L.o_ovw);
        h->ov.wb = prm.precision != PDCA_FP32 ? reinterpret_cast<const __nv_bfloat16 *>(W + L.o_ovwb) : nullptr;
        h->ov.n_rows = L.n_ov;
        h->ov_index = reinterpret_cast<int32_t *>(W + L.o_ovidx);
        h->ov_acc = reinterpret_cast<float *>(W + L.o_ovacc);
    }
    h->mixed = prm.precision != PDCA_FP32;
    h->bf16u = prm.precision == PDCA_MIXED_BF16W_BF16U;
    h->mr = W + L.o_mr;
    h->me[0] = W + L.o_me[0];
    h->me[1] = W + L.o_me[1];
    h->partials = reinterpret_cast<double *>(W + L.o_part);
    h->red = reinterpret_cast<RedOut *>(W + L.o_red);
    h->scal = reinterpret_cast<double *>(W + L.o_scal);
    h->trace = reinterpret_cast<double *>(W + L.o_trace);
    int64_t *s_rp = reinterpret_cast<int64_t *>(W + L.o_srp);
    int32_t *s_col = reinterpret_cast<int32_t *>(W + L.o_scol);
    float *s_w = reinterpret_cast<float *>(W + L.o_sw);
    double *s_deg = reinterpret_cast<double *>(W + L.o_sdeg);
    double *s_isd = reinterpret_cast<double *>(W + L.o_sisd);
    uint8_t *s_mask = reinterpret_cast<uint8_t *>(W + L.o_smask);
    int32_t *s_lab = reinterpret_cast<int32_t *>(W + L.o_slab);
    uint32_t *s_status = reinterpret_cast<uint32_t *>(W + L.o_status);
    uint32_t *s_cls = reinterpret_cast<uint32_t *>(W + L.o_scls);
    cudaStream_t sm = h->stream;

    // BFS renumbering on a host thread, overlapping the copies and validation
    OrderJob job;
    if (L.host_order && !L.device_order) {
        st = job.start(rp, col, nnz, n, L.sigma);
        if (st != PDCA_OK) {
            delete h;
            return st;
        }
    }
    // the device's BFS order runs on a stream of its own beside the rest of
    // the copies and the validation (it needs only row_ptr and the columns)
    auto fail = [&](pdca_status s) { cudaStreamSynchronize(sm); delete h; return s; };
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, sm) : cudaSuccess;
    };
    if (!early &&
        (cp(s_rp, rp, 8 * ((size_t)n + 1)) != cudaSuccess || cp(s_col, col, 4 * (size_t)nnz) != cudaSuccess))
        return fail(PDCA_ERR_CUDA);
    if (L.device_order) {
        if (!order_ready &&
            (order_side.open() != cudaSuccess || cudaEventRecord(order_side.in, sm) != cudaSuccess))
            return fail(PDCA_ERR_CUDA);
        if (cudaStreamWaitEvent(order_side.s, order_side.in, 0) != cudaSuccess ||
            device_order_launch(h, order_side.s) != cudaSuccess ||
            cudaEventRecord(order_side.out, order_side.s) != cudaSuccess)
            return fail(PDCA_ERR_CUDA);
    }
    if (!early && (cp(s_w, w, 4 * (size_t)nnz) != cudaSuccess || cp(s_mask, fid_mask, (size_t)n) != cudaSuccess ||
                   cp(s_lab, labels, 4 * (size_t)n) != cudaSuccess ||
                   cudaMemsetAsync(s_status, 0, 16, sm) != cudaSuccess))
        return fail(PDCA_ERR_CUDA);
    if (launch_validate(n, k, s_rp, s_col, s_w, s_mask, s_lab, s_deg, s_isd, s_status, sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    uint32_t stat4[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(stat4, s_status, 16, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaStreamSynchronize(sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    uint32_t status = stat4[0];
    if (status & kBadGraph) return fail(PDCA_ERR_BAD_GRAPH);
    if (status & kNotSymmetric) return fail(PDCA_ERR_NOT_SYMMETRIC);
    if (status & kIsolated) return fail(PDCA_ERR_ISOLATED_NODE);
    std::memcpy(&h->dmax, stat4 + 2, sizeof(double));
    if (prm.precond != PDCA_RICHARDSON || prm.lambda_max > 0) {
        st = feasible(prm, omega, prm.lambda_max, h->dmax);
        if (st != PDCA_OK) return fail(st);
    }
    if (L.host_order) {
        if (L.device_order && cudaStreamWaitEvent(sm, order_side.out, 0) != cudaSuccess) return fail(PDCA_ERR_CUDA);
        st = L.device_order ? device_renumber(h, rp) : host_renumber(h, rp, job);
        if (st != PDCA_OK) return fail(st);
    } else {
        if (launch_window_sort(n, L.n_pad, L.sigma, s_rp, h->perm, h->iperm, sm) != cudaSuccess)
            return fail(PDCA_ERR_CUDA);
        if (L.n_ov > 0) {   // the overflow rows follow the device's renumbering
            std::vector<int32_t> perm_h((size_t)L.n_pad);
            if (cudaMemcpyAsync(perm_h.data(), h->perm, 4 * perm_h.size(), cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
                cudaStreamSynchronize(sm) != cudaSuccess)
                return fail(PDCA_ERR_CUDA);
            st = build_overflow(h, rp, perm_h.data(), L.n_pad);
            if (st != PDCA_OK) return fail(st);
        }
    }
    if (!h->slice_off_on_device && cp(h->slice_off, L.slice_off.data(), 8 * L.slice_off.size()) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    cudaError_t pe;
    if (h->tiled)
        pe = launch_pack_tiled(L.n_pad, s_rp, s_col, s_w, s_deg, s_isd, s_mask, s_lab, h->perm, h->iperm, h->slice_off,
                               h->tv.halo_off, h->tv.halo_idx, const_cast<uint16_t *>(h->tv.lcol), h->sell_w,
                               h->rowinfo, s_status, sm);
    else
        pe = launch_pack(n, L.n_pad, k, s_rp, s_col, s_w, s_deg, s_isd, s_mask, s_lab, h->perm, h->iperm, h->slice_off,
                         h->sell_col, h->sell_w, h->sell_wb, h->self, h->dsq, h->rowinfo,
                         prm.columns == PDCA_COLUMNS_AUTO ? s_cls : nullptr, L.split, h->ov_index,
                         h->ov.rp, const_cast<int32_t *>(h->ov.col), const_cast<float *>(h->ov.w),
                         const_cast<__nv_bfloat16 *>(h->ov.wb), s_status, sm);
    if (pe != cudaSuccess) return fail(PDCA_ERR_CUDA);
    const bool c16 = !h->tiled && prm.columns == PDCA_COLUMNS_AUTO;
    if (prm.entry_order == PDCA_ENTRIES_SPREAD &&
        launch_spread(L.n_pad, h->slice_off, h->rowinfo, h->tiled ? 0xFFFFFFu : kLenMask, c16 ? s_cls : nullptr,
                      h->tiled ? nullptr : h->sell_col,
                      h->tiled ? const_cast<uint16_t *>(h->tv.lcol) : nullptr, h->tv.halo_off, h->tv.halo_idx,
                      h->sell_w, h->sell_wb, sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    if (c16) {
        h->col16 = reinterpret_cast<uint16_t *>(W + L.o_col16);
        if (launch_compress(L.n_slices, h->slice_off, s_cls, h->sell_col, h->col16, h->rowinfo, h->slice_fmt, sm) !=
            cudaSuccess)
            return fail(PDCA_ERR_CUDA);
    }
    if (prm.precond == PDCA_RICHARDSON) {
        if (prm.lambda_max > 0) {
            h->lambda_used = prm.lambda_max;
        } else {
            st = power_method(h);
            if (st != PDCA_OK) return fail(st);
        }
        st = feasible(prm, omega, h->lambda_used, h->dmax);
        if (st != PDCA_OK) return fail(st);
    }
    h->cf = make_coeffs(prm, omega, h->lambda_used);
    if (launch_init_u(L.n_pad, k, h->rowinfo, h->U[0], sm) != cudaSuccess) return fail(PDCA_ERR_CUDA);
    h->cur = 0;
    h->prev = 1;
    h->has_prev = false;
    std::vector<uint8_t> fmt(c16 ? (size_t)L.n_slices : 0);
    if (cudaMemcpyAsync(&status, s_status, 4, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        (c16 && cudaMemcpyAsync(fmt.data(), h->slice_fmt, fmt.size(), cudaMemcpyDeviceToHost, sm) != cudaSuccess) ||
        cudaStreamSynchronize(sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    if (status & kLayoutMismatch) return fail(PDCA_ERR_CUDA);
    for (uint8_t f : fmt) h->slices16 += f == kFmt16 ? 1 : 0;
    *out = h;
    return PDCA_OK;
}

pdca_status pdca_workspace_size_like(const pdca_problem *base, int32_t k, const pdca_params *p, size_t *bytes) {
    if (!base || !bytes || k < 1 || k > PDCA_MAX_K) return PDCA_ERR_INVALID_ARG;
    pdca_params prm;
    pdca_default_params(&prm);
    if (p) prm = *p;
    pdca_status st = check_params(prm);
    if (st != PDCA_OK) return st;
    *bytes = clone_layout(base->L, k, prm.precision).total;
    return PDCA_OK;
}

}  // extern "C"

namespace {

// pdca_create_like and pdca_create_like_async: `wait` reads the fidelity
// check back before returning; without it the check's word stays on the
// device for pdca_labels / pdca_labels_async to report.
pdca_status create_like(const pdca_problem *base, int32_t k, const uint8_t *fid_mask, const int32_t *labels,
                        const pdca_params *p, void *workspace, size_t ws_bytes, pdca_problem **out, bool wait) {
    if (!out) return PDCA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!base || k < 1 || k > PDCA_MAX_K || !fid_mask || !labels || !workspace) return PDCA_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PDCA_ERR_INVALID_ARG;
    pdca_params prm;
    pdca_default_params(&prm);
    if (p) prm = *p;
    pdca_status st = check_params(prm);
    if (st != PDCA_OK) return st;
    // the shared operator fixes the weight format, the Laplacian and the kernel form
    if ((prm.precision != PDCA_FP32) != base->mixed) return PDCA_ERR_INVALID_ARG;
    if (prm.laplacian != base->prm.laplacian) return PDCA_ERR_INVALID_ARG;
    const double omega = prm.damping;
    if (prm.precond != PDCA_RICHARDSON || prm.lambda_max > 0) {
        st = feasible(prm, omega, prm.lambda_max, base->dmax);
        if (st != PDCA_OK) return st;
    }
    const CloneLayout CL = clone_layout(base->L, k, prm.precision);
    if (ws_bytes < CL.total) return PDCA_ERR_OOM;
    pdca_problem *h = new (std::nothrow) pdca_problem();
    if (!h) return PDCA_ERR_INVALID_ARG;
    h->L = base->L;
    h->L.K = k;
    h->prm = prm;
    h->omega = omega;
    h->stream = base->stream;
    h->ws = static_cast<char *>(workspace);
    h->sell_col = base->sell_col;
    h->col16 = base->col16;
    h->slice_fmt = base->slice_fmt;
    h->slices16 = base->slices16;
    h->sell_w = base->sell_w;
    h->sell_wb = base->sell_wb;
    h->ov = base->ov;
    h->ov_index = base->ov_index;
    h->slice_off = base->slice_off;
    h->perm = base->perm;
    h->iperm = base->iperm;
    h->self = base->self;
    h->dsq = base->dsq;
    h->dmax = base->dmax;
    h->tiled = base->tiled;
    h->tv = base->tv;
    h->halo_rows = base->halo_rows;
    h->mixed = base->mixed;
    h->bf16u = prm.precision == PDCA_MIXED_BF16W_BF16U;
    char *W = h->ws;
    h->rowinfo = reinterpret_cast<uint32_t *>(W + CL.o_rowinfo);
    for (int b = 0; b < 3; ++b) h->U[b] = reinterpret_cast<float *>(W + CL.o_u[b]);
    h->partials = reinterpret_cast<double *>(W + CL.o_part);
    h->red = reinterpret_cast<RedOut *>(W + CL.o_red);
    h->scal = reinterpret_cast<double *>(W + CL.o_scal);
    h->trace = reinterpret_cast<double *>(W + CL.o_trace);
    h->mr = W + CL.o_mr;
    h->me[0] = W + CL.o_me[0];
    h->me[1] = W + CL.o_me[1];
    h->ov_acc = base->L.n_ov > 0 ? reinterpret_cast<float *>(W + CL.o_ovacc) : nullptr;
    uint8_t *s_mask = reinterpret_cast<uint8_t *>(W + CL.o_smask);
    int32_t *s_lab = reinterpret_cast<int32_t *>(W + CL.o_slab);
    uint32_t *s_status = reinterpret_cast<uint32_t *>(W + CL.o_status);
    cudaStream_t sm = h->stream;
    auto fail = [&](pdca_status s2) { cudaStreamSynchronize(sm); delete h; return s2; };
    const int32_t n = h->L.n;
    if (cudaMemcpyAsync(s_mask, fid_mask, (size_t)n, cudaMemcpyDefault, sm) != cudaSuccess ||
        cudaMemcpyAsync(s_lab, labels, 4 * (size_t)n, cudaMemcpyDefault, sm) != cudaSuccess ||
        cudaMemsetAsync(s_status, 0, 16, sm) != cudaSuccess ||
        launch_retag(h->L.n_pad, k, base->rowinfo, h->perm, s_mask, s_lab, h->rowinfo, s_status, sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    if (prm.precond == PDCA_RICHARDSON) {
        if (prm.lambda_max > 0) {
            h->lambda_used = prm.lambda_max;
        } else if (base->lambda_est > 0) {   // same operator: reuse its estimate
            h->lambda_est = base->lambda_est;
            h->lambda_used = std::min(lambda_bound(h), 1.001 * base->lambda_est);
        } else {
            st = power_method(h);
            if (st != PDCA_OK) return fail(st);
        }
        st = feasible(prm, omega, h->lambda_used, h->dmax);
        if (st != PDCA_OK) return fail(st);
    }
    h->cf = make_coeffs(prm, omega, h->lambda_used);
    if (launch_init_u(h->L.n_pad, k, h->rowinfo, h->U[0], sm) != cudaSuccess) return fail(PDCA_ERR_CUDA);
    h->cur = 0;
    h->prev = 1;
    h->has_prev = false;
    if (!wait) {
        h->fid_status = s_status;
        *out = h;
        return PDCA_OK;
    }
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, s_status, 4, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaStreamSynchronize(sm) != cudaSuccess)
        return fail(PDCA_ERR_CUDA);
    if (status) return fail(PDCA_ERR_BAD_GRAPH);
    *out = h;
    return PDCA_OK;
}

}  // namespace

extern "C" {

pdca_status pdca_create_like(const pdca_problem *base, int32_t k, const uint8_t *fid_mask, const int32_t *labels,
                             const pdca_params *p, void *workspace, size_t ws_bytes, pdca_problem **out) {
    return create_like(base, k, fid_mask, labels, p, workspace, ws_bytes, out, true);
}

pdca_status pdca_create_like_async(const pdca_problem *base, int32_t k, const uint8_t *fid_mask,
                                   const int32_t *labels, const pdca_params *p, void *workspace, size_t ws_bytes,
                                   pdca_problem **out) {
    return create_like(base, k, fid_mask, labels, p, workspace, ws_bytes, out, false);
}

pdca_status pdca_set_u(pdca_problem *h, const float *u) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    const Layout &L = h->L;
    const int stage = (h->cur + 1) % 3, target = (h->cur + 2) % 3;
    if (!u) {
        PDCA_TRY(launch_init_u(L.n_pad, L.K, h->rowinfo, h->U[target], h->stream));
    } else {
        const float *src = u;
        if (!is_device_ptr(u)) {
            PDCA_TRY(cudaMemcpyAsync(h->U[stage], u, sizeof(float) * (size_t)L.n * L.K, cudaMemcpyHostToDevice,
                                     h->stream));
            src = h->U[stage];
        }
        PDCA_TRY(launch_permute_in(L.K, L.n, L.n_pad, src, h->perm, h->U[target], h->stream));
    }
    h->cur = target;
    h->prev = stage;
    h->has_prev = false;
    return PDCA_OK;
}

pdca_status pdca_spectral_workspace_size(const pdca_problem *h, size_t *bytes) {
    if (!h || !bytes) return PDCA_ERR_INVALID_ARG;
    *bytes = align_up(spectral_workspace_bytes(h->L.n_pad)) + align_up(sizeof(float) * (size_t)h->L.n);
    return PDCA_OK;
}

pdca_status pdca_spectral_init(pdca_problem *h, void *workspace, size_t ws_bytes, int32_t max_iters, double tol,
                               double *lambda2, float *u0_out, int32_t *iters_done) {
    if (!h || !workspace || max_iters < 0 || !(tol > 0.0) || !std::isfinite(tol)) return PDCA_ERR_INVALID_ARG;
    if (h->L.K != 1 || h->tiled) return PDCA_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return PDCA_ERR_INVALID_ARG;
    size_t need = 0;
    pdca_spectral_workspace_size(h, &need);
    if (ws_bytes < need) return PDCA_ERR_OOM;
    float *vec = reinterpret_cast<float *>(static_cast<char *>(workspace) + align_up(spectral_workspace_bytes(h->L.n_pad)));
    // the tolerance is relative to the bound of the spectrum
    const double bound = h->self ? 2.0 * h->dmax : 2.0;
    const pdca_status st = spectral_eigvec(h->view(), h->ov, h->self != nullptr, h->self ? nullptr : h->dsq, h->perm,
                                           h->L.n, h->L.n_pad, h->stream, workspace, max_iters, tol * bound,
                                           lambda2, vec, iters_done);
    if (st != PDCA_OK && st != PDCA_ERR_NOT_CONVERGED) return st;
    pdca_status s2 = pdca_set_u(h, vec);
    if (s2 != PDCA_OK) return s2;
    if (u0_out) PDCA_TRY(cudaMemcpyAsync(u0_out, vec, sizeof(float) * (size_t)h->L.n, cudaMemcpyDefault, h->stream));
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    return st;
}

pdca_status pdca_step(pdca_problem *h, int32_t inner_sweeps) {
    if (!h || inner_sweeps < 1) return PDCA_ERR_INVALID_ARG;
    return outer_step(h, inner_sweeps);
}

}  // extern "C"

namespace {

// pdca_solve through a cached CUDA graph: the launches of `outer` outer steps
// are captured once per starting state (which of the three iterate buffers
// hold u^t and u^{t-1}) and coefficient set, then replayed; the replay runs
// exactly the kernels and arguments of the direct path.
pdca_status solve_graph(pdca_problem *h, int32_t outer, int32_t inner) {
    for (auto &g : h->graphs)
        if (g.outer == outer && g.inner == inner && g.cur == h->cur && g.prev == h->prev &&
            g.has_prev == h->has_prev && std::memcmp(&g.cf, &h->cf, sizeof(Coeffs)) == 0) {
            PDCA_TRY(cudaGraphLaunch(g.exec, h->stream));
            count_launches(g.launches);
            h->cur = g.end_cur;
            h->prev = g.end_prev;
            h->has_prev = true;
            return PDCA_OK;
        }
    pdca_problem::SolveGraph g{};
    g.outer = outer;
    g.inner = inner;
    g.cur = h->cur;
    g.prev = h->prev;
    g.has_prev = h->has_prev;
    g.cf = h->cf;
    const uint64_t l0 = pdca_kernel_launches();
    PDCA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    pdca_status st = PDCA_OK;
    for (int32_t t = 0; t < outer && st == PDCA_OK; ++t) st = outer_step(h, inner);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (st != PDCA_OK || ce != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return st != PDCA_OK ? st : PDCA_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return PDCA_ERR_CUDA;
    g.launches = pdca_kernel_launches() - l0;   // counted once at capture: they run at this first launch
    g.end_cur = h->cur;
    g.end_prev = h->prev;
    if (h->graphs.size() >= 6) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(g);
    PDCA_TRY(cudaGraphLaunch(g.exec, h->stream));
    return PDCA_OK;
}

}  // namespace

extern "C" {

pdca_status pdca_solve(pdca_problem *h, int32_t outer_iters, int32_t inner_sweeps, double damping,
                       double *energy_trace, double *residual_trace) {
    if (!h || outer_iters < 0 || inner_sweeps < 1 || !(damping >= 0.0)) return PDCA_ERR_INVALID_ARG;
    if (damping > 0.0 && h->prm.precond == PDCA_JACOBI_DAMPED && damping != h->omega) {
        pdca_status st = feasible(h->prm, damping, h->lambda_used, h->dmax);
        if (st != PDCA_OK) return st;
        h->omega = damping;
        h->prm.damping = damping;
        h->cf = make_coeffs(h->prm, h->omega, h->lambda_used);
    }
    const bool tracing = energy_trace || residual_trace;
    if (h->graphs_on && !tracing && !h->prof && !h->tiled && outer_iters > 0 && h->stream != nullptr) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PDCA_TRY(cudaStreamIsCapturing(h->stream, &cs));
        if (cs == cudaStreamCaptureStatusNone) return solve_graph(h, outer_iters, inner_sweeps);
    }
    int chunk0 = 0;
    for (int32_t t = 0; t < outer_iters; ++t) {
        pdca_status st = outer_step(h, inner_sweeps);
        if (st != PDCA_OK) return st;
        if (tracing) {
            const int slot = t - chunk0;
            st = reduce_energy(h, h->trace + slot, h->trace + kTraceCap + slot);
            if (st != PDCA_OK) return st;
            if (slot == kTraceCap - 1 || t == outer_iters - 1) {
                const size_t cnt = (size_t)slot + 1;
                if (energy_trace)
                    PDCA_TRY(cudaMemcpyAsync(energy_trace + chunk0, h->trace, 8 * cnt, cudaMemcpyDefault, h->stream));
                if (residual_trace)
                    PDCA_TRY(cudaMemcpyAsync(residual_trace + chunk0, h->trace + kTraceCap, 8 * cnt,
                                             cudaMemcpyDefault, h->stream));
                PDCA_TRY(cudaStreamSynchronize(h->stream));
                chunk0 = t + 1;
            }
        }
    }
    return PDCA_OK;
}

pdca_status pdca_energy(pdca_problem *h, double *F, double *rel_residual) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    pdca_status st = reduce_energy(h, nullptr, nullptr);
    if (st != PDCA_OK) return st;
    RedOut o;
    PDCA_TRY(cudaMemcpyAsync(&o, h->red, sizeof(RedOut), cudaMemcpyDeviceToHost, h->stream));
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    if (F) *F = o.F;
    if (rel_residual) *rel_residual = o.rel_res;
    if (o.nonfinite > 0 || !std::isfinite(o.F)) return PDCA_ERR_NONFINITE;
    return PDCA_OK;
}

pdca_status pdca_get_u(pdca_problem *h, float *u_out) {
    if (!h || !u_out) return PDCA_ERR_INVALID_ARG;
    const Layout &L = h->L;
    if (is_device_ptr(u_out)) {
        PDCA_TRY(launch_permute_out(L.K, L.n, h->U[h->cur], h->perm, u_out, h->stream));
        PDCA_TRY(cudaStreamSynchronize(h->stream));
        return PDCA_OK;
    }
    float *stage = h->U[h->spare()];
    PDCA_TRY(launch_permute_out(L.K, L.n, h->U[h->cur], h->perm, stage, h->stream));
    PDCA_TRY(cudaMemcpyAsync(u_out, stage, sizeof(float) * (size_t)L.n * L.K, cudaMemcpyDeviceToHost, h->stream));
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    return PDCA_OK;
}

pdca_status pdca_labels(pdca_problem *h, int32_t *labels_out) {
    if (!h || !labels_out) return PDCA_ERR_INVALID_ARG;
    const Layout &L = h->L;
    uint32_t fid = 0;
    if (is_device_ptr(labels_out)) {
        PDCA_TRY(launch_labels(L.K, L.n, h->U[h->cur], h->perm, labels_out, h->stream));
    } else {
        int32_t *stage = reinterpret_cast<int32_t *>(h->U[h->spare()]);
        PDCA_TRY(launch_labels(L.K, L.n, h->U[h->cur], h->perm, stage, h->stream));
        PDCA_TRY(cudaMemcpyAsync(labels_out, stage, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost,
                                 h->stream));
    }
    if (h->fid_status) PDCA_TRY(cudaMemcpyAsync(&fid, h->fid_status, 4, cudaMemcpyDeviceToHost, h->stream));
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    return fid ? PDCA_ERR_BAD_GRAPH : PDCA_OK;
}

pdca_status pdca_labels_async(pdca_problem *h, int32_t *labels_out, uint32_t *fid_status_out) {
    if (!h || !labels_out) return PDCA_ERR_INVALID_ARG;
    const Layout &L = h->L;
    if (is_device_ptr(labels_out)) {
        PDCA_TRY(launch_labels(L.K, L.n, h->U[h->cur], h->perm, labels_out, h->stream));
    } else {
        int32_t *stage = reinterpret_cast<int32_t *>(h->U[h->spare()]);
        PDCA_TRY(launch_labels(L.K, L.n, h->U[h->cur], h->perm, stage, h->stream));
        PDCA_TRY(cudaMemcpyAsync(labels_out, stage, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToHost,
                                 h->stream));
    }
    if (!fid_status_out) return PDCA_OK;
    if (h->fid_status) {
        PDCA_TRY(cudaMemcpyAsync(fid_status_out, h->fid_status, 4, cudaMemcpyDefault, h->stream));
    } else if (is_device_ptr(fid_status_out)) {
        PDCA_TRY(cudaMemsetAsync(fid_status_out, 0, 4, h->stream));
    } else {
        *fid_status_out = 0;   // checked when the problem was created
    }
    return PDCA_OK;
}

pdca_status pdca_lambda_max(pdca_problem *h, double *lambda_used, double *lambda_estimate) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    if (lambda_used) *lambda_used = h->lambda_used;
    if (lambda_estimate) *lambda_estimate = h->lambda_est;
    return PDCA_OK;
}

pdca_status pdca_layout(pdca_problem *h, int64_t *sell_entries, int64_t *n_slices, int32_t *sort_window,
                        int32_t *tiled, int64_t *halo_rows, int32_t *max_halo, int64_t *slices16,
                        int32_t *split_len, int64_t *split_rows) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    if (split_len) *split_len = h->tiled ? 0 : h->L.split;
    if (split_rows) *split_rows = h->L.n_ov;
    if (slices16) *slices16 = h->slices16;
    if (sell_entries) *sell_entries = h->L.sell_entries;
    if (n_slices) *n_slices = h->L.n_slices;
    if (sort_window) *sort_window = h->L.sigma;
    if (tiled) *tiled = h->tiled ? 1 : 0;
    if (halo_rows) *halo_rows = h->tiled ? h->halo_rows : 0;
    if (max_halo) *max_halo = h->tiled ? h->tv.max_halo : 0;
    return PDCA_OK;
}

pdca_status pdca_locality_order(const int64_t *row_ptr, const int32_t *col, int32_t n, int32_t sort_window,
                                int32_t device, int32_t *order, void *stream) {
    if (!row_ptr || !order || n < 1 || (device != 0 && device != 1)) return PDCA_ERR_INVALID_ARG;
    const int32_t sigma = sort_window == 0 ? kBfsBlock : sort_window;
    if (sigma < 32 || sigma > kBfsBlock || (sigma & (sigma - 1)) != 0) return PDCA_ERR_INVALID_ARG;
    std::vector<int64_t> keep;
    const int64_t *rp = nullptr;
    pdca_status st = host_row_ptr(row_ptr, n, keep, &rp);
    if (st != PDCA_OK) return st;
    if (rp[n] > 0 && !col) return PDCA_ERR_INVALID_ARG;
    if (device == 0) {
        if (is_device_ptr(row_ptr) || is_device_ptr(col) || is_device_ptr(order)) return PDCA_ERR_INVALID_ARG;
        locality_order(n, rp, col, kBfsBlock, kBfsChunk, sigma, order);
        return PDCA_OK;
    }
    if (!is_device_ptr(row_ptr) || (rp[n] > 0 && !is_device_ptr(col)) || !is_device_ptr(order))
        return PDCA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    const size_t nn = (size_t)n;
    if (cudaMalloc(&scratch, 16 * nn + 16) != cudaSuccess) {
        cudaGetLastError();
        return PDCA_ERR_OOM;
    }
    char *b = static_cast<char *>(scratch);
    unsigned long long *key = reinterpret_cast<unsigned long long *>(b);
    int32_t *queue = reinterpret_cast<int32_t *>(b + 8 * nn);
    int32_t *tmp = reinterpret_cast<int32_t *>(b + 12 * nn);
    uint32_t *err = reinterpret_cast<uint32_t *>(b + 16 * nn);
    uint32_t err_h = 0;
    st = PDCA_OK;
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess ||
        launch_bfs_blocks(n, kBfsBlock, kBfsChunk, row_ptr, col, queue, key, tmp, err, s) != cudaSuccess ||
        cudaMemcpyAsync(&err_h, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        st = PDCA_ERR_CUDA;
    else if (err_h)
        st = PDCA_ERR_CUDA;
    else if (launch_order_sort(n, sigma, row_ptr, tmp, order, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        st = PDCA_ERR_CUDA;
    cudaFree(scratch);
    return st;
}

pdca_status pdca_profile_enable(pdca_problem *h, int32_t on) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    h->prof = on != 0;
    return PDCA_OK;
}

pdca_status pdca_profile_read(pdca_problem *h, double *sweep_ms, int64_t *sweep_launches) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    PDCA_TRY(cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.f;
        PDCA_TRY(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
        tot += ms;
    }
    if (sweep_ms) *sweep_ms = tot;
    if (sweep_launches) *sweep_launches = (int64_t)(h->ev_used / 2);
    h->ev_used = 0;
    return PDCA_OK;
}

pdca_status pdca_batch_create(int32_t max_problems, void *stream, pdca_batch **out) {
    if (!out || max_problems < 1) return PDCA_ERR_INVALID_ARG;
    pdca_batch *b = new (std::nothrow) pdca_batch();
    if (!b) return PDCA_ERR_INVALID_ARG;
    b->stream = static_cast<cudaStream_t>(stream);
    b->max_problems = max_problems;
    *out = b;
    return PDCA_OK;
}

pdca_status pdca_batch_add(pdca_batch *b, pdca_problem *h, int32_t outer_iters, int32_t inner_sweeps) {
    if (!b || !h || outer_iters < 1 || inner_sweeps < 1) return PDCA_ERR_INVALID_ARG;
    if (h->stream != b->stream || h->tiled) return PDCA_ERR_INVALID_ARG;
    if ((int32_t)b->members.size() >= b->max_problems) return PDCA_ERR_INVALID_ARG;
    for (const BatchMember &m : b->members)
        if (m.h == h) return PDCA_ERR_INVALID_ARG;
    for (const pdca_problem *d : b->done)
        if (d == h) return PDCA_ERR_INVALID_ARG;
    b->members.push_back(BatchMember{h, outer_iters, inner_sweeps, 0});
    return PDCA_OK;
}

pdca_status pdca_batch_step(pdca_batch *b, int32_t passes, int32_t *active_after) {
    if (!b || passes < 0) return PDCA_ERR_INVALID_ARG;
    for (int32_t p = 0; p < passes && !b->members.empty(); ++p) {
        // one launch per class (K, Laplacian) and per kBatchMax members
        bool used[2][PDCA_MAX_K + 1] = {};
        for (const BatchMember &m : b->members) used[m.h->self ? 1 : 0][m.h->L.K] = true;
        for (int un = 0; un < 2; ++un)
            for (int K = 1; K <= PDCA_MAX_K; ++K) {
                if (!used[un][K]) continue;
                BatchTable &t = b->table;
                BatchOvTable &o = b->ov_table;
                t.n = 0;
                t.total_slices = 0;
                o.n = 0;
                o.total_rows = 0;
                // the overflow pre-pass of the members gathered so far, then their pass
                auto flush = [&]() -> cudaError_t {
                    if (t.n == 0) return cudaSuccess;
                    cudaError_t e = launch_batch_overflow(K, o, b->stream);
                    if (e != cudaSuccess) return e;
                    e = launch_batch_pass(K, un == 1, t, b->stream);
                    t.n = 0;
                    t.total_slices = 0;
                    o.n = 0;
                    o.total_rows = 0;
                    return e;
                };
                for (size_t i = 0; i < b->members.size(); ++i) {
                    const BatchMember &m = b->members[i];
                    if (m.h->L.K != K || (m.h->self ? 1 : 0) != un) continue;
                    BatchDesc &d = t.d[t.n++];
                    member_desc(m, d);
                    d.slice_begin = t.total_slices;
                    // members start at multiples of 8 slices (one block never spans two)
                    t.total_slices += (m.h->L.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock * kWarpsPerBlock;
                    if (m.h->ov.n_rows > 0) {
                        BatchOvDesc &q = o.d[o.n++];
                        q.O = m.h->ov;
                        q.x = d.src;
                        q.acc = m.h->ov_acc;
                        q.q_begin = o.total_rows;
                        q.wkind = d.kind == kPassMixedSweep ? kOvW16 : kOvW32;
                        q.xkind = d.kind == kPassMixedSweep ? (m.h->bf16u ? kOvXBf16 : kOvXHalf) : kOvX32;
                        q.pad_ = 0;
                        o.total_rows += m.h->ov.n_rows;
                    }
                    if (t.n == kBatchMax) PDCA_TRY(flush());
                }
                PDCA_TRY(flush());
            }
        std::vector<BatchMember> keep;
        keep.reserve(b->members.size());
        for (BatchMember &m : b->members) {
            if (member_advance(m)) b->done.push_back(m.h);
            else keep.push_back(m);
        }
        b->members.swap(keep);
    }
    if (active_after) *active_after = (int32_t)b->members.size();
    return PDCA_OK;
}

pdca_status pdca_batch_poll(pdca_batch *b, pdca_problem **done, int32_t capacity, int32_t *count) {
    if (!b || !count || capacity < 0 || (capacity > 0 && !done)) return PDCA_ERR_INVALID_ARG;
    const int32_t k = std::min<int32_t>(capacity, (int32_t)b->done.size());
    for (int32_t i = 0; i < k; ++i) done[i] = b->done[(size_t)i];
    b->done.erase(b->done.begin(), b->done.begin() + k);
    *count = k;
    return PDCA_OK;
}

pdca_status pdca_batch_remove(pdca_batch *b, pdca_problem *h) {
    if (!b || !h) return PDCA_ERR_INVALID_ARG;
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i].h == h) {
            b->members.erase(b->members.begin() + (ptrdiff_t)i);
            return PDCA_OK;
        }
    for (size_t i = 0; i < b->done.size(); ++i)
        if (b->done[i] == h) {
            b->done.erase(b->done.begin() + (ptrdiff_t)i);
            return PDCA_OK;
        }
    return PDCA_ERR_INVALID_ARG;
}

void pdca_batch_destroy(pdca_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    delete b;
}

pdca_status pdca_graph_enable(pdca_problem *h, int32_t on) {
    if (!h) return PDCA_ERR_INVALID_ARG;
    if (!on) {
        PDCA_TRY(cudaStreamSynchronize(h->stream));
        h->drop_graphs();
    }
    h->graphs_on = on != 0;
    return PDCA_OK;
}

void pdca_destroy(pdca_problem *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->drop_graphs();
    delete h;
}

void pdca_release(pdca_problem *h) {
    if (!h) return;
    if (!h->graphs.empty()) cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);   // a pending event is freed once it completes
    h->drop_graphs();
    delete h;
}

}  // extern "C"
