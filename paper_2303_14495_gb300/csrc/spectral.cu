// Spectral initial iterate of the unsupervised model: the second eigenvector
// of L_s (or L) scaled to max |u_i| = 1 (the unsupervised clustering
// experiments of Sec. 5.3 initialise with the second eigenvector of the
// normalized graph Laplacian).  "Second" is the smallest eigenpair on the
// orthogonal complement of the null vector q (D^1/2 1 for L_s, 1 for L),
// which stays unique when the graph has several components.
//
// The eigenpair comes from a block LOBPCG (Knyazev's locally optimal block
// preconditioned conjugate gradient, without preconditioner) on the same
// sliced-ELL operator the sweeps use, with every block kept orthogonal to q
// (A maps that complement to itself).  The block holds the m = 4 lowest
// eigenpairs of the complement.  Every iteration:
//   R = A X - X Theta, deflated against q;
//   Rayleigh-Ritz on S = [X R P] (P the previous search direction) from the
//   Gram blocks G = S^T S and H = S^T A S, all formed in one batch: with
//   D = diag(G)^-1/2 and D G D = L L^T, the m smallest eigenpairs of
//   L^-1 D H D L^-T give the coefficients C (without P when D G D is not
//   numerically positive definite);
//   X <- S C, P <- [R P] C_{R,P}, with A X, A P updated by the same
//   coefficients (one SpMM per iteration, for A R).
// Every 10 iterations X and P are deflated again and X re-orthonormalised.
// Device work: the SpMM, 4x4 Gram blocks U^T V (FP64 accumulation, fixed
// block order, the block partials added on the device, so results are
// deterministic) and linear combinations of n x 4 blocks.  Host work: the
// small dense symmetric eigenproblems (cyclic Jacobi rotations) and Cholesky
// factors, in FP64; two waits for the device per iteration.
#include "device_common.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace pdca {

namespace {

using namespace dev;

constexpr int kM = 4;                       // block size
constexpr int kGramBlocks = 2 * kSmCount;   // fixed grid of the Gram kernel
constexpr int kGramSlots = 16;              // Gram products per launch slot
constexpr int kMaxGrams = 16;               // Gram launches per synchronisation

// Y = L X for n_pad x 4 FP32 blocks (renumbered rows; padding rows stay 0).
// (FP32 weights, which every problem keeps whatever its precision.)
template <bool UN>
__global__ void __launch_bounds__(kBlockThreads)
spmm4_kernel(const SellView A, const float *__restrict__ x, float *__restrict__ y) {
    const int slice = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (slice >= A.n_slices) return;
    const int lane = threadIdx.x & 31;
    const int r = slice * kSliceRows + lane;
    float acc[kM], v[kM];
    if (block_fmt16(A, blockIdx.x * kWarpsPerBlock)) row_gather<kM, float, float, true>(A, slice, lane, x, acc);
    else row_gather<kM, float, float, false>(A, slice, lane, x, acc);
    load_row<kM>(x + (size_t)r * kM, v);
    const float a = UN ? __ldg(A.self + r) : 1.0f;
    float out[kM];
#pragma unroll
    for (int k = 0; k < kM; ++k) out[k] = a * v[k] - acc[k];
    store_row<kM>(y + (size_t)r * kM, out);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// The Gram products queued before a wait, launched together: product s of
// the table in blockIdx.y.
struct GramTable {
    const float *u[kMaxGrams];
    const float *v[kMaxGrams];
};

// partial[s][block][4 i + j] = sum over this block's rows of U_s[r][i] V_s[r][j]
__global__ void __launch_bounds__(256)
gram4_kernel(int32_t rows, const __grid_constant__ GramTable t, double *__restrict__ partial_all) {
    const float *__restrict__ u = t.u[blockIdx.y];
    const float *__restrict__ v = t.v[blockIdx.y];
    double *__restrict__ partial = partial_all + (size_t)blockIdx.y * kGramBlocks * kGramSlots;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int32_t r = blockIdx.x * 256 + threadIdx.x; r < rows; r += gridDim.x * 256) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(u) + r);
        const float4 b = __ldg(reinterpret_cast<const float4 *>(v) + r);
        const double ai[4] = {a.x, a.y, a.z, a.w}, bj[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[4 * i + j] = fma(ai[i], bj[j], acc[4 * i + j]);
    }
    __shared__ double sm[8][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const double t = warp_sum_d(acc[q]);
        if (lane == 0) sm[warp][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += sm[w][threadIdx.x];
        partial[(size_t)blockIdx.x * kGramSlots + threadIdx.x] = t;
    }
}

// sums[s][q] = the kGramBlocks block partials of Gram slot s added in block
// order (one thread per entry, the order of a plain loop)
__global__ void __launch_bounds__(kGramSlots)
gram_sum_kernel(const double *__restrict__ partial, double *__restrict__ sums) {
    const double *p = partial + (size_t)blockIdx.x * kGramBlocks * kGramSlots + threadIdx.x;
    double t = 0.0;
    for (int b = 0; b < kGramBlocks; ++b) t += p[(size_t)b * kGramSlots];
    sums[(size_t)blockIdx.x * kGramSlots + threadIdx.x] = t;
}

struct Coef3 {
    float c[3][16];   // row-major 4 x 4 blocks
};

// out[r] = U0[r] C0 + U1[r] C1 + U2[r] C2 (rows as 1 x 4 vectors; U1, U2 nullable)
__global__ void __launch_bounds__(256)
combine4_kernel(int32_t rows, float *__restrict__ out, const float *__restrict__ u0, const float *__restrict__ u1,
                const float *__restrict__ u2, const Coef3 cf) {
    const int32_t r = blockIdx.x * 256 + threadIdx.x;
    if (r >= rows) return;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
    const float *src[3] = {u0, u1, u2};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (!src[b]) continue;
        const float4 t = __ldg(reinterpret_cast<const float4 *>(src[b]) + r);
        const float x[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = fmaf(x[i], cf.c[b][4 * i + j], o[j]);
    }
    reinterpret_cast<float4 *>(out)[r] = make_float4(o[0], o[1], o[2], o[3]);
}

// Up to four combinations of up to four blocks each in one launch (output o
// in blockIdx.y).
struct Coef4 {
    float c[4][16];   // row-major 4 x 4 blocks
};

struct CombTable {
    float *out[4];
    const float *u[4][4];
    Coef4 cf[4];
};

__global__ void __launch_bounds__(256)
combine4_multi_kernel(int32_t rows, const __grid_constant__ CombTable t) {
    const int32_t r = blockIdx.x * 256 + threadIdx.x;
    if (r >= rows) return;
    const int o_ix = blockIdx.y;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float *src = t.u[o_ix][b];
        if (!src) continue;
        const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + r);
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = fmaf(x[i], t.cf[o_ix].c[b][4 * i + j], o[j]);
    }
    reinterpret_cast<float4 *>(t.out[o_ix])[r] = make_float4(o[0], o[1], o[2], o[3]);
}

// Start block: column j of row r is a fixed function of the caller's node
// index (so the start does not depend on the renumbering); padding rows 0.
// The null-vector block: q in column 0 (the constant on real rows when q is
// null), zeros elsewhere.
__global__ void __launch_bounds__(256)
spectral_start_kernel(int32_t n, int32_t n_pad, const int32_t *__restrict__ perm, const float *__restrict__ q,
                      float *__restrict__ x, float *__restrict__ qb) {
    const int32_t r = blockIdx.x * 256 + threadIdx.x;
    if (r >= n_pad) return;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
    float qr = 0.0f;
    if (r < n) {
        const double i = (double)perm[r] + 1.0;
        o[0] = (float)sin(0.9238795325112867 * i + 0.3);
        o[1] = (float)sin(0.7548776662466927 * i);
        o[2] = (float)sin(0.5698402909980532 * i + 1.0);
        o[3] = (float)cos(0.3247179572447460 * i + 2.0);
        qr = q ? q[r] : 1.0f;
    }
    reinterpret_cast<float4 *>(x)[r] = make_float4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<float4 *>(qb)[r] = make_float4(qr, 0.f, 0.f, 0.f);
}

// Largest |x[r][col]| of each block and the smallest caller index attaining it.
__global__ void __launch_bounds__(256)
absmax_kernel(int32_t n, const float *__restrict__ x, int col, const int32_t *__restrict__ perm,
              float *__restrict__ bmax, int32_t *__restrict__ bidx, int32_t *__restrict__ brow) {
    float best = -1.0f;
    int32_t at = 0x7fffffff, row = -1;
    for (int32_t r = blockIdx.x * 256 + threadIdx.x; r < n; r += gridDim.x * 256) {
        const float a = fabsf(x[(size_t)r * kM + col]);
        const int32_t i = perm[r];
        if (a > best || (a == best && i < at)) {
            best = a;
            at = i;
            row = r;
        }
    }
    __shared__ float sb[256];
    __shared__ int32_t si[256], sr[256];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = at;
    sr[threadIdx.x] = row;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const float b2 = sb[threadIdx.x + h];
            const int32_t i2 = si[threadIdx.x + h];
            if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
                sb[threadIdx.x] = b2;
                si[threadIdx.x] = i2;
                sr[threadIdx.x] = sr[threadIdx.x + h];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bmax[blockIdx.x] = sb[0];
        bidx[blockIdx.x] = si[0];
        brow[blockIdx.x] = sr[0];
    }
}

// out[perm[r]] = scale * x[r][col] for the n real rows (caller order)
__global__ void __launch_bounds__(256)
extract_kernel(int32_t n, const float *__restrict__ x, int col, const int32_t *__restrict__ perm, float scale,
               float *__restrict__ out) {
    const int32_t r = blockIdx.x * 256 + threadIdx.x;
    if (r >= n) return;
    out[perm[r]] = scale * x[(size_t)r * kM + col];
}

// ---------------------------------------------------------------------------
// host: small dense linear algebra in FP64
// ---------------------------------------------------------------------------

// Symmetric eigenproblem by cyclic Jacobi rotations: a (n x n, row-major) is
// destroyed; eigenvalues ascending in w, eigenvectors as columns of v.
void jacobi_eigen(int n, std::vector<double> a, std::vector<double> &w, std::vector<double> &v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
                tot += x;
                if (i != j) off += x;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                // rotation angle that zeroes a_pq: tan(2 phi) = 2 a_pq / (a_qq - a_pp)
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[(size_t)x * n + x] < a[(size_t)y * n + y]; });
    std::vector<double> vs((size_t)n * n);
    w.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        w[k] = a[(size_t)idx[k] * n + idx[k]];
        for (int i = 0; i < n; ++i) vs[(size_t)i * n + k] = v[(size_t)i * n + idx[k]];
    }
    v.swap(vs);
}

// g (4 x 4 SPD) = R^T R; returns R^{-1} (upper triangular) or false when g is
// not numerically positive definite relative to its largest diagonal entry.
bool chol_inv_upper(const double *g, double *rinv) {
    double r[16] = {0};
    double dmax = 0.0;
    for (int i = 0; i < 4; ++i) dmax = std::max(dmax, g[5 * i]);
    if (!(dmax > 0.0)) return false;
    for (int j = 0; j < 4; ++j) {
        double s = g[4 * j + j];
        for (int k = 0; k < j; ++k) s -= r[4 * k + j] * r[4 * k + j];
        if (!(s > 1e-10 * dmax)) return false;
        r[4 * j + j] = sqrt(s);
        for (int i = j + 1; i < 4; ++i) {
            double t = g[4 * j + i];
            for (int k = 0; k < j; ++k) t -= r[4 * k + j] * r[4 * k + i];
            r[4 * j + i] = t / r[4 * j + j];
        }
    }
    // invert the upper triangle by back substitution, column by column
    for (int i = 0; i < 16; ++i) rinv[i] = 0.0;
    for (int j = 0; j < 4; ++j) {
        rinv[4 * j + j] = 1.0 / r[4 * j + j];
        for (int i = j - 1; i >= 0; --i) {
            double t = 0.0;
            for (int k = i + 1; k <= j; ++k) t += r[4 * i + k] * rinv[4 * k + j];
            rinv[4 * i + j] = -t / r[4 * i + i];
        }
    }
    return true;
}

// C = D R'^{-1} with D = diag(g_ii^{-1/2}) and D g D = R'^T R': U C has
// orthonormal columns.  False when the columns are (numerically) dependent.
bool ortho_coeffs(const double *g, double *cmat) {
    double dsc[4], gs[16], ri[16];
    for (int i = 0; i < 4; ++i) {
        if (!(g[5 * i] > 0.0) || !std::isfinite(g[5 * i])) return false;
        dsc[i] = 1.0 / sqrt(g[5 * i]);
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) gs[4 * i + j] = dsc[i] * g[4 * i + j] * dsc[j];
    if (!chol_inv_upper(gs, ri)) return false;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) cmat[4 * i + j] = dsc[i] * ri[4 * i + j];
    return true;
}

// Rayleigh-Ritz on the basis S = [X R P] (nb blocks of 4 columns) from the
// Gram blocks G = S^T S and H = S^T A S: with D = diag(G)^-1/2, a Cholesky
// factorisation L L^T of D G D that leaves out, in column order, every
// column of norm below 1e-12 (a zero residual column of a converged Ritz
// vector) or whose pivot falls below 1e-8 (a direction already in the span
// of the earlier ones), the m smallest eigenpairs (y, theta) of L^-1 D H D L^-T on the kept
// columns give the coefficients D L^-T y of the new X in S (0 for the left
// out columns).  False when fewer than m columns are kept.
bool ritz_coeffs(const std::vector<std::vector<double>> &g, const int (&gs)[3][3], const int (&hs)[3][3], int nb,
                 std::vector<double> &cb, std::vector<double> &theta) {
    const int ns = 4 * nb;
    std::vector<double> G((size_t)ns * ns), H((size_t)ns * ns);
    for (int bi = 0; bi < nb; ++bi)
        for (int bj = bi; bj < nb; ++bj) {
            const std::vector<double> &gg = g[gs[bi][bj]], &hh = g[hs[bi][bj]];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    const double x = bi == bj ? 0.5 * (gg[4 * i + j] + gg[4 * j + i]) : gg[4 * i + j];
                    const double y = bi == bj ? 0.5 * (hh[4 * i + j] + hh[4 * j + i]) : hh[4 * i + j];
                    G[(size_t)(4 * bi + i) * ns + 4 * bj + j] = G[(size_t)(4 * bj + j) * ns + 4 * bi + i] = x;
                    H[(size_t)(4 * bi + i) * ns + 4 * bj + j] = H[(size_t)(4 * bj + j) * ns + 4 * bi + i] = y;
                }
        }
    std::vector<double> d(ns, 0.0);
    for (int k = 0; k < ns; ++k) {
        const double gk = G[(size_t)k * ns + k];
        if (gk > 1e-24 && std::isfinite(gk)) d[k] = 1.0 / sqrt(gk);   // X columns have unit norm
    }
    // Cholesky of D G D over the kept columns (act), in column order
    std::vector<int> act;
    std::vector<double> L;   // row-major over kept columns, grown as kept
    for (int k = 0; k < ns; ++k) {
        if (d[k] == 0.0) continue;
        const int na = (int)act.size();
        std::vector<double> row(na + 1, 0.0);
        double t = 1.0;   // the scaled diagonal
        for (int m = 0; m < na; ++m) {
            double u = G[(size_t)k * ns + act[m]] * d[k] * d[act[m]];
            for (int p2 = 0; p2 < m; ++p2) u -= row[p2] * L[(size_t)m * ns + p2];
            row[m] = u / L[(size_t)m * ns + m];
            t -= row[m] * row[m];
        }
        if (!(t > 1e-8)) continue;
        row[na] = sqrt(t);
        L.resize((size_t)(na + 1) * ns, 0.0);
        for (int m = 0; m <= na; ++m) L[(size_t)na * ns + m] = row[m];
        act.push_back(k);
    }
    const int na = (int)act.size();
    if (na < kM) return false;
    // Li = L^-1 (lower), by forward substitution column by column
    std::vector<double> Li((size_t)na * na, 0.0);
    for (int j = 0; j < na; ++j) {
        Li[(size_t)j * na + j] = 1.0 / L[(size_t)j * ns + j];
        for (int i = j + 1; i < na; ++i) {
            double u = 0.0;
            for (int k = j; k < i; ++k) u += L[(size_t)i * ns + k] * Li[(size_t)k * na + j];
            Li[(size_t)i * na + j] = -u / L[(size_t)i * ns + i];
        }
    }
    // M = Li (D H D)_act Li^T
    std::vector<double> Hs((size_t)na * na), T1((size_t)na * na, 0.0), M((size_t)na * na, 0.0);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < na; ++j)
            Hs[(size_t)i * na + j] = H[(size_t)act[i] * ns + act[j]] * d[act[i]] * d[act[j]];
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < na; ++j) {
            double u = 0.0;
            for (int k = 0; k <= i; ++k) u += Li[(size_t)i * na + k] * Hs[(size_t)k * na + j];
            T1[(size_t)i * na + j] = u;
        }
    for (int i = 0; i < na; ++i)
        for (int j = 0; j <= i; ++j) {
            double u = 0.0;
            for (int k = 0; k <= j; ++k) u += T1[(size_t)i * na + k] * Li[(size_t)j * na + k];
            M[(size_t)i * na + j] = M[(size_t)j * na + i] = u;
        }
    std::vector<double> w, v;
    jacobi_eigen(na, M, w, v);
    // coefficients D Li^T y for the m smallest, on the kept columns
    cb.assign((size_t)ns * kM, 0.0);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < kM; ++j) {
            double u = 0.0;
            for (int k = i; k < na; ++k) u += Li[(size_t)k * na + i] * v[(size_t)k * na + j];
            cb[(size_t)act[i] * kM + j] = d[act[i]] * u;
        }
    for (int j = 0; j < kM; ++j) theta[j] = w[j];
    return true;
}

struct Ctx {
    SellView A;
    OverflowView O;
    cudaStream_t st;
    int32_t n, n_pad;
    bool un;
    double *partial;          // kMaxGrams x kGramBlocks x 16 (device)
    double *sums;             // kMaxGrams x 16 (device)
    GramTable table{};        // the products queued since the last wait
    std::vector<double> host; // the sums on the host
    int pending = 0;
    bool overflow = false;
};

cudaError_t spmm(Ctx &c, const float *x, float *y) {
    const int blocks = (c.A.n_slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
    // the split rows' remaining entries first (kM columns per overflow row)
    cudaError_t e = launch_overflow(kM, kOvW32, kOvX32, c.O, x, const_cast<float *>(c.A.ov_acc), c.st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    if (c.un) spmm4_kernel<true><<<blocks, kBlockThreads, 0, c.st>>>(c.A, x, y);
    else spmm4_kernel<false><<<blocks, kBlockThreads, 0, c.st>>>(c.A, x, y);
    return cudaGetLastError();
}

// queue U^T V (launched at the next wait); returns its slot
int gram(Ctx &c, const float *u, const float *v) {
    if (c.pending >= kMaxGrams) {   // never expected: every step queues at most 12
        c.overflow = true;
        return 0;
    }
    const int slot = c.pending++;
    c.table.u[slot] = u;
    c.table.v[slot] = v;
    return slot;
}

// wait for the queued Grams; g[slot] = 4 x 4 result (row-major)
cudaError_t gram_wait(Ctx &c, std::vector<std::vector<double>> &g) {
    if (c.overflow) return cudaErrorInvalidValue;
    if (c.pending == 0) {
        g.clear();
        return cudaSuccess;
    }
    count_launches(2);
    gram4_kernel<<<dim3(kGramBlocks, c.pending), 256, 0, c.st>>>(c.n_pad, c.table, c.partial);
    gram_sum_kernel<<<c.pending, kGramSlots, 0, c.st>>>(c.partial, c.sums);
    cudaError_t e = cudaGetLastError();
    const size_t cnt = (size_t)c.pending * kGramSlots;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.host.data(), c.sums, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return e;
    g.assign(c.pending, std::vector<double>(16, 0.0));
    for (int s = 0; s < c.pending; ++s)
        for (int q = 0; q < 16; ++q) g[s][q] = c.host[(size_t)s * kGramSlots + q];
    c.pending = 0;
    return cudaSuccess;
}

cudaError_t combine(Ctx &c, float *out, const float *u0, const double *c0, const float *u1 = nullptr,
                    const double *c1 = nullptr, const float *u2 = nullptr, const double *c2 = nullptr) {
    Coef3 cf{};
    const double *cs[3] = {c0, c1, c2};
    for (int b = 0; b < 3; ++b)
        for (int q = 0; q < 16; ++q) cf.c[b][q] = cs[b] ? (float)cs[b][q] : 0.0f;
    count_launches(1);
    combine4_kernel<<<(c.n_pad + 255) / 256, 256, 0, c.st>>>(c.n_pad, out, u0, u1, u2, cf);
    return cudaGetLastError();
}

// The four updates of an iteration (new X, A X, P, A P) in one launch; each
// entry: output, up to three inputs and their coefficient blocks.
struct CombSpec {
    float *out;
    const float *u[4];
    const double *c[4];
};

cudaError_t combine_four(Ctx &c, const CombSpec (&sp)[4]) {
    CombTable t{};
    for (int o = 0; o < 4; ++o) {
        t.out[o] = sp[o].out;
        for (int b = 0; b < 4; ++b) {
            t.u[o][b] = sp[o].u[b];
            for (int q = 0; q < 16; ++q) t.cf[o].c[b][q] = sp[o].c[b] ? (float)sp[o].c[b][q] : 0.0f;
        }
    }
    count_launches(1);
    combine4_multi_kernel<<<dim3((c.n_pad + 255) / 256, 4), 256, 0, c.st>>>(c.n_pad, t);
    return cudaGetLastError();
}

void neg(double *m) {
    for (int q = 0; q < 16; ++q) m[q] = -m[q];
}

const double kIdentity[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};

}  // namespace

// ---------------------------------------------------------------------------

constexpr int kBufs = 13;

size_t spectral_workspace_bytes(int32_t n_pad) {
    const size_t blk = ((size_t)n_pad * kM * sizeof(float) + 255) / 256 * 256;
    return kBufs * blk + (size_t)kMaxGrams * (kGramBlocks + 1) * kGramSlots * sizeof(double) + 3 * 256 * 4;
}

pdca_status spectral_eigvec(const SellView &A, const OverflowView &O, bool un, const float *q, const int32_t *perm, int32_t n,
                            int32_t n_pad, cudaStream_t st, void *workspace, int32_t max_iters, double tol,
                            double *lambda2, float *out_caller_order, int32_t *iters_done) {

    char *W = static_cast<char *>(workspace);
    const size_t blk = ((size_t)n_pad * kM * sizeof(float) + 255) / 256 * 256;
    float *buf[kBufs];
    for (int b = 0; b < kBufs; ++b) buf[b] = reinterpret_cast<float *>(W + (size_t)b * blk);
    Ctx c;
    c.A = A;
    c.O = O;
    c.st = st;
    c.n = n;
    c.n_pad = n_pad;
    c.un = un;
    c.partial = reinterpret_cast<double *>(W + kBufs * blk);
    c.sums = c.partial + (size_t)kMaxGrams * kGramBlocks * kGramSlots;
    c.host.assign((size_t)kMaxGrams * kGramSlots, 0.0);
    float *bmax = reinterpret_cast<float *>(W + kBufs * blk + (size_t)kMaxGrams * (kGramBlocks + 1) * kGramSlots * 8);
    int32_t *bidx = reinterpret_cast<int32_t *>(bmax + 256);
    int32_t *brow = bidx + 256;
    float *X = buf[0], *AX = buf[1], *Wb = buf[2], *AW = buf[3], *P = buf[4], *AP = buf[5];
    float *T[6] = {buf[6], buf[7], buf[8], buf[9], buf[10], buf[11]};
    float *Qb = buf[12];
    std::vector<std::vector<double>> g;
#define SP_TRY(e)                                   \
    do {                                            \
        if ((e) != cudaSuccess) return PDCA_ERR_CUDA; \
    } while (0)

    // X: start block, deflated and orthonormalised (twice)
    count_launches(1);
    spectral_start_kernel<<<(n_pad + 255) / 256, 256, 0, st>>>(n, n_pad, perm, q, X, Qb);
    SP_TRY(cudaGetLastError());
    gram(c, Qb, Qb);
    SP_TRY(gram_wait(c, g));
    const double qq = g[0][0];
    if (!(qq > 0.0)) return PDCA_ERR_NONFINITE;
    // U <- U - q (q^T U) / (q^T q), in place through a temporary
    auto deflate = [&](float *&U, float *&tmp) -> cudaError_t {
        gram(c, Qb, U);
        cudaError_t e = gram_wait(c, g);
        if (e != cudaSuccess) return e;
        double cq[16] = {0};
        for (int j = 0; j < 4; ++j) cq[j] = -g[0][j] / qq;
        e = combine(c, tmp, U, kIdentity, Qb, cq);
        if (e != cudaSuccess) return e;
        std::swap(U, tmp);
        return cudaSuccess;
    };
    for (int pass = 0; pass < 2; ++pass) {
        SP_TRY(deflate(X, T[0]));
        gram(c, X, X);
        SP_TRY(gram_wait(c, g));
        double ri[16];
        if (!ortho_coeffs(g[0].data(), ri)) return PDCA_ERR_NONFINITE;
        SP_TRY(combine(c, T[0], X, ri));
        std::swap(X, T[0]);
    }
    SP_TRY(spmm(c, X, AX));
    bool hasP = false;
    std::vector<double> theta(kM, 0.0);
    int it = 0;
    bool converged = false;
    for (; it <= max_iters; ++it) {
        // Rayleigh-Ritz on X alone only at the start (later X is the Ritz block)
        if (it == 0) {
            gram(c, X, AX);
            SP_TRY(gram_wait(c, g));
            std::vector<double> a(16), w, v;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) a[4 * i + j] = 0.5 * (g[0][4 * i + j] + g[0][4 * j + i]);
            jacobi_eigen(4, a, w, v);
            SP_TRY(combine(c, T[0], X, v.data()));
            SP_TRY(combine(c, T[1], AX, v.data()));
            std::swap(X, T[0]);
            std::swap(AX, T[1]);
            theta = w;
        }
        // keep X, P orthogonal to q and X orthonormal against FP32 drift every
        // 10 iterations (A q = 0, so A X and A P need no deflation)
        if (it % 10 == 9) {
            SP_TRY(deflate(X, T[0]));
            if (hasP) SP_TRY(deflate(P, T[0]));
            gram(c, X, X);
            SP_TRY(gram_wait(c, g));
            double rx[16];
            if (!ortho_coeffs(g[0].data(), rx)) return PDCA_ERR_NONFINITE;
            SP_TRY(combine(c, T[0], X, rx));
            SP_TRY(combine(c, T[1], AX, rx));
            std::swap(X, T[0]);
            std::swap(AX, T[1]);
        }
        // residual block R = AX - X diag(theta) (into W) and A R
        double mth[16] = {0};
        for (int i = 0; i < 4; ++i) mth[5 * i] = -theta[i];
        SP_TRY(combine(c, Wb, AX, kIdentity, X, mth));
        SP_TRY(deflate(Wb, T[0]));
        SP_TRY(spmm(c, Wb, AW));
        // every Gram block of S = [X R P] and S^T A S in one batch
        const int nb = hasP ? 3 : 2;
        const float *S[3] = {X, Wb, P}, *AS[3] = {AX, AW, AP};
        int gs[3][3], hs[3][3];
        for (int i = 0; i < nb; ++i)
            for (int j = i; j < nb; ++j) {
                gs[i][j] = gram(c, S[i], S[j]);
                hs[i][j] = gram(c, S[i], AS[j]);
            }
        SP_TRY(gram_wait(c, g));
        const double r0 = sqrt(std::max(0.0, g[gs[1][1]][0]));
        if (r0 <= tol) {
            converged = true;
            break;
        }
        if (it == max_iters) break;
        std::vector<double> cb;   // (4 nb) x 4 coefficients of the new X
        int nbu = nb;
        for (; nbu >= 2; --nbu) {   // with P, else without it when [X R P] is numerically dependent
            if (ritz_coeffs(g, gs, hs, nbu, cb, theta)) break;
        }
        if (nbu < 2) break;   // R lies in span X numerically: as converged as FP32 allows
        double cx[3][16] = {{0}};
        for (int bb = 0; bb < nbu; ++bb)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) cx[bb][4 * i + j] = cb[(size_t)(4 * bb + i) * 4 + j];
        const bool useP = nbu == 3;
        // new X, A X, P, A P
        const CombSpec sp[4] = {
            {T[0], {X, Wb, useP ? P : nullptr, nullptr}, {cx[0], cx[1], useP ? cx[2] : nullptr, nullptr}},
            {T[1], {AX, AW, useP ? AP : nullptr, nullptr}, {cx[0], cx[1], useP ? cx[2] : nullptr, nullptr}},
            {T[2], {Wb, useP ? P : nullptr, nullptr, nullptr}, {cx[1], useP ? cx[2] : nullptr, nullptr, nullptr}},
            {T[3], {AW, useP ? AP : nullptr, nullptr, nullptr}, {cx[1], useP ? cx[2] : nullptr, nullptr, nullptr}}};
        SP_TRY(combine_four(c, sp));
        std::swap(X, T[0]);
        std::swap(AX, T[1]);
        std::swap(P, T[2]);
        std::swap(AP, T[3]);
        hasP = true;
    }
    if (!std::isfinite(theta[0])) return PDCA_ERR_NONFINITE;
    if (lambda2) *lambda2 = theta[0];
    if (iters_done) *iters_done = it;
    // u^0: column 0 scaled to max |u| = 1, largest-magnitude entry positive
    count_launches(1);
    absmax_kernel<<<256, 256, 0, st>>>(n, X, 0, perm, bmax, bidx, brow);
    SP_TRY(cudaGetLastError());
    std::vector<float> hb(256);
    std::vector<int32_t> hi(256), hr(256);
    SP_TRY(cudaMemcpyAsync(hb.data(), bmax, 256 * sizeof(float), cudaMemcpyDeviceToHost, st));
    SP_TRY(cudaMemcpyAsync(hi.data(), bidx, 256 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SP_TRY(cudaMemcpyAsync(hr.data(), brow, 256 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SP_TRY(cudaStreamSynchronize(st));
    float best = -1.0f;
    int32_t at = 0x7fffffff, row = -1;
    for (int b = 0; b < 256; ++b)
        if (hb[b] > best || (hb[b] == best && hi[b] < at)) {
            best = hb[b];
            at = hi[b];
            row = hr[b];
        }
    if (!(best > 0.0f) || row < 0 || row >= n) return PDCA_ERR_NONFINITE;
    float val = 0.0f;   // the entry of largest magnitude fixes the sign
    SP_TRY(cudaMemcpyAsync(&val, X + (size_t)row * kM, sizeof(float), cudaMemcpyDeviceToHost, st));
    SP_TRY(cudaStreamSynchronize(st));
    const float scale = (val < 0.0f ? -1.0f : 1.0f) / best;
    count_launches(1);
    extract_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, X, 0, perm, scale, out_caller_order);
    SP_TRY(cudaGetLastError());
    return converged ? PDCA_OK : PDCA_ERR_NOT_CONVERGED;
#undef SP_TRY
}

}  // namespace pdca
