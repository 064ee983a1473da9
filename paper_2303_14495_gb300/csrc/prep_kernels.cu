// Operator preparation on the GPU (create time, Sec. 2.2):
//   validate_kernel     CSR checks (range, no self loop, strictly increasing
//                       columns, finite non-negative weights, w_ij == w_ji)
//                       and the degrees d_i = sum_j w_ij (FP64, CSR order);
//   window_sort_kernel  renumbering: rows sorted by degree inside windows;
//   pack_kernel         sliced-ELL with w_ij d_i^-1/2 d_j^-1/2 (L_s; the
//                       factors d_i^-1/2 come from validate_kernel) or w_ij plus
//                       the per-row d_i (L), and the row tags; entries in
//                       chunk bands where 16-bit columns are possible;
//   spread_kernel       entry order inside rows for conflict-light gathers;
//   compress_kernel     16-bit columns for the slices that allow them;
//   init_u_kernel       u^0 (prior on labelled rows, centre elsewhere).
#include "pdca_internal.cuh"
#include "scan.cuh"

#include <cuda_bf16.h>
#include <math.h>

namespace pdca {
namespace {

// kValLanes lanes per row: each lane checks one entry at a time (range, no
// self loop, strictly increasing columns, a finite non-negative weight, and
// w_ji stored with the same value, by binary search in row j); the row's
// first lane adds the weights into d_i in CSR order (FP64).  One atomic per
// warp for the flags and for the largest degree.
constexpr int kValLanes = 8;

__global__ void __launch_bounds__(256)
validate_kernel(int32_t n, int32_t K, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                const float *__restrict__ w, const uint8_t *__restrict__ mask, const int32_t *__restrict__ labels,
                double *__restrict__ deg, double *__restrict__ isd, uint32_t *__restrict__ status) {
    constexpr unsigned kAll = 0xffffffffu;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((t & ~31ll) >= (int64_t)n * kValLanes) return;   // whole warps past the last row
    const int32_t i = (int32_t)(t / kValLanes);
    const int sub = (int)(t % kValLanes);
    const int g0 = (threadIdx.x & 31) & ~(kValLanes - 1);
    const bool live = i < n;
    uint32_t bad = 0;
    double d = 0.0;
    int64_t e0 = 0, e1 = 0;
    if (live) {
        e0 = row_ptr[i];
        e1 = row_ptr[i + 1];
    }
    const int32_t chunks = live ? (int32_t)((e1 - e0 + kValLanes - 1) / kValLanes) : 0;
    const int32_t cmax = __reduce_max_sync(kAll, chunks);
    for (int32_t c = 0; c < cmax; ++c) {
        const int64_t e = e0 + (int64_t)c * kValLanes + sub;
        float wv = 0.0f;
        if (e < e1) {
            const int32_t j = col[e];
            wv = w[e];
            if (j < 0 || j >= n) {
                bad |= kBadGraph;
            } else {
                if (j == i || (e > e0 && j <= col[e - 1])) bad |= kBadGraph;
                if (!(isfinite(wv) && wv >= 0.0f)) bad |= kBadGraph;
                int64_t lo = row_ptr[j], hi = row_ptr[j + 1] - 1;
                bool ok = false;
                while (lo <= hi) {
                    const int64_t mid = lo + ((hi - lo) >> 1);
                    const int32_t cm = col[mid];
                    if (cm == i) {
                        ok = (w[mid] == wv);
                        break;
                    }
                    if (cm < i) lo = mid + 1;
                    else hi = mid - 1;
                }
                if (!ok) bad |= kNotSymmetric;
            }
        }
#pragma unroll
        for (int k = 0; k < kValLanes; ++k) {
            const float wk = __shfl_sync(kAll, wv, g0 + k);
            if (sub == 0 && e0 + (int64_t)c * kValLanes + k < e1) d += (double)wk;
        }
    }
    unsigned long long dbits = 0;
    if (live && sub == 0) {
        if (!(d > 0.0)) bad |= kIsolated;
        const uint8_t m = mask[i];
        if (m > 1) bad |= kBadGraph;
        if (m == 1) {
            const int32_t l = labels[i];
            const int32_t hiK = K == 1 ? 2 : K;
            if (l < 0 || l >= hiK) bad |= kBadGraph;
        }
        deg[i] = d;
        isd[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
        // non-negative doubles order like their bit patterns
        dbits = (unsigned long long)__double_as_longlong(d);
    }
    bad = __reduce_or_sync(kAll, bad);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(kAll, dbits, o);
        dbits = x > dbits ? x : dbits;
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(status, bad);
        atomicMax(reinterpret_cast<unsigned long long *>(status + 2), dbits);
    }
}

// One block per window of `sigma` rows: bitonic sort of keys
// ((2^32-1 - degree) << 32 | position), i.e. degree descending, ties by the
// original index.  Rows past n sort last and become padding (perm = -1).
__global__ void window_sort_kernel(int32_t n, int32_t n_pad, int32_t sigma,
                                   const int64_t *__restrict__ row_ptr, int32_t *__restrict__ perm,
                                   int32_t *__restrict__ iperm) {
    extern __shared__ unsigned long long keys[];
    const int64_t base = (int64_t)blockIdx.x * sigma;
    for (int p = threadIdx.x; p < sigma; p += blockDim.x) {
        const int64_t i = base + p;
        unsigned long long key = ~0ull;
        if (i < n) {
            const uint32_t dgr = (uint32_t)(row_ptr[i + 1] - row_ptr[i]);
            key = ((unsigned long long)(0xFFFFFFFFu - dgr) << 32) | (uint32_t)p;
        }
        keys[p] = key;
    }
    __syncthreads();
    for (int k = 2; k <= sigma; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int p = threadIdx.x; p < sigma; p += blockDim.x) {
                const int q = p ^ jj;
                if (q > p) {
                    const unsigned long long a = keys[p], b = keys[q];
                    const bool up = (p & k) == 0;
                    if ((a > b) == up) {
                        keys[p] = b;
                        keys[q] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < sigma; p += blockDim.x) {
        const int64_t r = base + p;
        if (r >= n_pad) continue;
        const unsigned long long key = keys[p];
        if (key == ~0ull) {
            perm[r] = -1;
        } else {
            const int32_t old = (int32_t)(base + (int64_t)(key & 0xFFFFFFFFull));
            perm[r] = old;
            iperm[old] = (int32_t)r;
        }
    }
}

// Renumbering from a node order (position -> node, in perm[0, n)): padding
// rows of perm set to -1, iperm the inverse.
__global__ void order_perm_kernel(int32_t n, int32_t n_pad, int32_t *__restrict__ perm,
                                  int32_t *__restrict__ iperm) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    if (r >= n) {
        perm[r] = -1;
        return;
    }
    iperm[perm[r]] = r;
}

// Entries of every slice: 32 x (its longest row, capped at the split
// length, rounded up to kVec).  One warp per slice, lane = row.
__global__ void slice_count_kernel(int32_t n, int32_t n_slices, int32_t split, const int64_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ perm, int32_t *__restrict__ count) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = t >> 5;
    if (s >= n_slices) return;   // warp-uniform
    const int64_t r = t;
    int32_t d = 0;
    if (r < n) {
        const int32_t v = perm[r];
        const int64_t dv = row_ptr[v + 1] - row_ptr[v];
        d = dv < split ? (int32_t)dv : split;
    }
    const int32_t wmax = __reduce_max_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0) count[s] = (wmax + kVec - 1) / kVec * kVec * kSliceRows;
}

// One thread per row.  With rowcls, a row's entries are ordered in three
// bands -- columns in the previous 65536-node chunk, in the next one, in the
// row's own chunk (each band in CSR order) -- otherwise kept in CSR order.
// The first split_len entries of that order go to the sliced ELL, the rest
// to the row's overflow CSR row ov_index[r] (kOvFlag in rowinfo).  rowcls[r]
// records the bands of the sliced entries, n_prev | n_next << 8, and
// 1 << 16 when they can take 16-bit columns (no column further than one
// chunk away, the band limits met); 0 for a row whose columns reach further
// (its entries then stay in CSR order).  Padding rows count as able.
__global__ void pack_kernel(int32_t n_pad, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, const float *__restrict__ w,
                            const double *__restrict__ deg, const double *__restrict__ isd,
                            const uint8_t *__restrict__ mask,
                            const int32_t *__restrict__ labels, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ iperm, const int64_t *__restrict__ slice_off,
                            int32_t *__restrict__ sell_col, float *__restrict__ sell_w,
                            __nv_bfloat16 *__restrict__ sell_wb, float *__restrict__ self,
                            float *__restrict__ dsq, uint32_t *__restrict__ rowinfo,
                            uint32_t *__restrict__ rowcls, int32_t split_len, const int32_t *__restrict__ ov_index,
                            const int64_t *__restrict__ ov_rp, int32_t *__restrict__ ov_col,
                            float *__restrict__ ov_w, __nv_bfloat16 *__restrict__ ov_wb,
                            uint32_t *__restrict__ status) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int32_t s = r >> 5, lane = r & 31;
    const int64_t base = slice_off[s];
    const int32_t width = (int32_t)((slice_off[s + 1] - base) >> 5);
    const int32_t old = perm[r];
    int32_t len = 0, kept = 0;
    uint32_t tag = kTagUnlabelled, ovf = 0u;
    uint32_t cls = 1u << 16;
    auto at = [&](int32_t j) { return base + 32 * kVec * (int64_t)(j / kVec) + kVec * lane + (j % kVec); };
    if (old >= 0) {
        const int64_t e0 = row_ptr[old];
        len = (int32_t)(row_ptr[old + 1] - e0);
        kept = len < split_len ? len : split_len;
        int64_t o0 = 0;
        if (len > split_len) {
            const int32_t q = ov_index ? ov_index[r] : -1;
            if (q < 0 || ov_rp[q + 1] - ov_rp[q] != (int64_t)(len - split_len)) {
                // host and device layouts disagree: keep the row inside its slice
                atomicOr(status, kLayoutMismatch);
                len = kept;
            } else {
                o0 = ov_rp[q];
                ovf = kOvFlag;
            }
        }
        if (kept > width) {  // never write past the slice
            atomicOr(status, kLayoutMismatch);
            kept = width;
            len = len < width ? len : width;
            ovf = 0u;
        }
        const double di = deg[old];
        if (self) self[r] = (float)di;
        if (dsq) dsq[r] = (float)sqrt(di);
        // chunk distance of every column: band counts
        const int32_t hr = r >> kChunkShift;
        int32_t np = 0, nn = 0;
        bool banded = rowcls != nullptr;
        if (banded) {
            for (int32_t j = 0; j < len; ++j) {
                const int32_t d = (iperm[col[e0 + j]] >> kChunkShift) - hr;
                np += d == -1;
                nn += d == 1;
                if (d < -1 || d > 1) banded = false;
            }
        }
        int32_t p_prev = 0, p_next = np, p_own = np + nn;
        for (int32_t j = 0; j < len; ++j) {
            const int32_t oj = col[e0 + j];
            const int32_t cj = iperm[oj];
            int32_t pos = j;
            if (banded) {
                const int32_t d = (cj >> kChunkShift) - hr;
                pos = d < 0 ? p_prev++ : (d > 0 ? p_next++ : p_own++);
            }
            const double wt = self ? (double)w[e0 + j] : (double)w[e0 + j] * isd[old] * isd[oj];
            if (pos < kept) {
                const int64_t a = at(pos);
                sell_col[a] = cj;
                sell_w[a] = (float)wt;
                if (sell_wb) sell_wb[a] = __double2bfloat16(wt);
            } else if (ovf) {
                const int64_t a = o0 + (pos - kept);
                ov_col[a] = cj;
                ov_w[a] = (float)wt;
                if (ov_wb) ov_wb[a] = __double2bfloat16(wt);
            }
        }
        if (mask[old]) tag = (uint32_t)labels[old];
        // bands of the sliced entries (the first `kept` of the banded order)
        const int32_t np_k = np < kept ? np : kept;
        const int32_t nb_k = np + nn < kept ? np + nn : kept;
        const int32_t nn_k = nb_k - np_k;
        const bool ok16 = banded && (uint32_t)np_k <= kBandMax && (uint32_t)nn_k <= kBandMax;
        // counts above 255 are kept at 255 (such a row is not 16-bit capable
        // anyway); the fields must not run into the capability bit
        cls = banded ? ((uint32_t)min(np_k, 255) | ((uint32_t)min(nn_k, 255) << 8) | (ok16 ? 1u << 16 : 0u)) : 0u;
    } else {
        if (self) self[r] = 0.0f;
        if (dsq) dsq[r] = 0.0f;
    }
    for (int32_t j = kept; j < width; ++j) {
        const int64_t a = at(j);
        sell_col[a] = r;
        sell_w[a] = 0.0f;
        if (sell_wb) sell_wb[a] = __float2bfloat16(0.0f);
    }
    rowinfo[r] = ((uint32_t)kept << 8) | tag | ovf;
    if (rowcls) rowcls[r] = cls;
}

// One block per group of kFmtGroupSlices slices, one warp per slice: when
// every row of the group can take 16-bit columns (rowcls), store the low 16
// bits of the group's columns in col16, rewrite its rowinfo words in the
// 16-bit form (tag | len << 8 | n_prev << 20 | n_next << 26) and mark its
// slices kFmt16; otherwise mark them kFmt32.  The kernels pick the column
// format once per block, and no block range crosses a group.
__global__ void __launch_bounds__(kFmtGroupSlices * 32)
compress_kernel(int32_t n_slices, const int64_t *__restrict__ slice_off, const uint32_t *__restrict__ rowcls,
                const int32_t *__restrict__ sell_col, uint16_t *__restrict__ col16, uint32_t *__restrict__ rowinfo,
                uint8_t *__restrict__ slice_fmt) {
    const int32_t s = blockIdx.x * kFmtGroupSlices + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const bool real = s < n_slices;   // slices past the end count as able
    const int32_t r = s * kSliceRows + lane;
    const uint32_t cls = real ? rowcls[r] : (1u << 16);
    const bool ok = __syncthreads_and((int)((cls >> 16) & 1u)) != 0;
    if (!real) return;
    if (lane == 0) slice_fmt[s] = ok ? kFmt16 : kFmt32;
    if (!ok) return;
    const int64_t base = slice_off[s];
    const int32_t width = (int32_t)((slice_off[s + 1] - base) >> 5);
    for (int32_t j = 0; j < width; ++j) {
        const int64_t a = base + 32 * kVec * (int64_t)(j / kVec) + kVec * lane + (j % kVec);
        col16[a] = (uint16_t)((uint32_t)sell_col[a] & 0xFFFFu);
    }
    const uint32_t info = rowinfo[r];   // len <= kSplitMax: bits 20..31 are free
    rowinfo[r] = info | ((cls & 0xFFu) << 20) | (((cls >> 8) & 0xFFu) << 26);
}

// Tiled form: the column of every entry becomes its position in the tile's
// sorted halo list (binary search); padding entries use position 0.
__global__ void pack_tiled_kernel(int32_t n_pad, const int64_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col, const float *__restrict__ w,
                                  const double *__restrict__ deg, const double *__restrict__ isd,
                            const uint8_t *__restrict__ mask,
                                  const int32_t *__restrict__ labels, const int32_t *__restrict__ perm,
                                  const int32_t *__restrict__ iperm, const int64_t *__restrict__ slice_off,
                                  const int64_t *__restrict__ halo_off, const int32_t *__restrict__ halo_idx,
                                  uint16_t *__restrict__ lcol, float *__restrict__ sell_w,
                                  uint32_t *__restrict__ rowinfo, uint32_t *__restrict__ status) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int32_t s = r >> 5, lane = r & 31;
    const int64_t base = slice_off[s];
    const int32_t width = (int32_t)((slice_off[s + 1] - base) >> 5);
    const int32_t tile = r / kTileRows;
    const int64_t h0 = halo_off[tile], h1 = halo_off[tile + 1];
    if (h1 <= h0 || h1 - h0 > 65536) {
        atomicOr(status, kLayoutMismatch);
        return;
    }
    const int32_t old = perm[r];
    int32_t len = 0;
    uint32_t tag = kTagUnlabelled;
    if (old >= 0) {
        const int64_t e0 = row_ptr[old];
        len = (int32_t)(row_ptr[old + 1] - e0);
        if (len > width) {
            atomicOr(status, kLayoutMismatch);
            len = width;
        }
        for (int32_t j = 0; j < len; ++j) {
            const int32_t oj = col[e0 + j];
            const int32_t cj = iperm[oj];
            int64_t lo = h0, hi = h1 - 1, pos = -1;
            while (lo <= hi) {
                const int64_t mid = lo + ((hi - lo) >> 1);
                const int32_t v = halo_idx[mid];
                if (v == cj) { pos = mid; break; }
                if (v < cj) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0) {
                atomicOr(status, kLayoutMismatch);
                pos = h0;
            }
            const int64_t at = base + 32 * kVec * (int64_t)(j / kVec) + kVec * lane + (j % kVec);
            lcol[at] = (uint16_t)(pos - h0);
            sell_w[at] = (float)((double)w[e0 + j] * isd[old] * isd[oj]);
        }
        if (mask[old]) tag = (uint32_t)labels[old];
    }
    for (int32_t j = len; j < width; ++j) {
        const int64_t at = base + 32 * kVec * (int64_t)(j / kVec) + kVec * lane + (j % kVec);
        lcol[at] = 0;
        sell_w[at] = 0.0f;
    }
    rowinfo[r] = ((uint32_t)len << 8) | tag;
}

// One thread per quarter of a slice (S = 8 lanes: the rows whose 16-byte
// neighbour rows one L1 wavefront serves).  Neighbour row c lies in group
// c / S of S consecutive rows at slot c % S; two rows of the quarter read at
// the same position conflict when they use the same slot of different groups.
// Position by position, each row (in lane order) takes its first remaining
// entry, looking at most kSpreadLook ahead, whose slot is free or holds the
// same group; without one it keeps its entry.  Rows are permuted in place
// (column and weight together); padding entries stay where they are.  The
// choice reads global columns only, so the plain and tiled forms get the same
// order, and it does not depend on K or the precision.
constexpr int kSpreadLook = 64;
constexpr int kSpreadLanes = 8;   // S

// Quarter lane0 / S of slice s, entries in global memory.
__device__ void spread_quarter(int64_t s, int32_t lane0, const int64_t *__restrict__ slice_off,
                               const uint32_t *__restrict__ rowinfo, uint32_t len_mask,
                               const uint32_t *__restrict__ rowcls, int32_t *__restrict__ sell_col,
                               uint16_t *__restrict__ lcol, const int64_t *__restrict__ halo_off,
                               const int32_t *__restrict__ halo_idx, float *__restrict__ sell_w,
                               __nv_bfloat16 *__restrict__ sell_wb) {
    constexpr int S = kSpreadLanes;
    const int64_t base = slice_off[s];
    const int64_t h0 = lcol ? halo_off[(s * kSliceRows) / kTileRows] : 0;
    int32_t len[S], np[S], nb[S];
    int32_t maxlen = 0;
#pragma unroll
    for (int32_t l = 0; l < S; ++l) {
        const int64_t r = s * kSliceRows + lane0 + l;
        len[l] = (int32_t)((rowinfo[r] >> 8) & len_mask);
        const uint32_t c = rowcls ? rowcls[r] : 0u;
        np[l] = (int32_t)(c & 0xFFu);
        nb[l] = np[l] + (int32_t)((c >> 8) & 0xFFu);
        maxlen = max(maxlen, len[l]);
    }
    auto at = [&](int32_t lane, int32_t j) {
        return base + 32 * kVec * (int64_t)(j / kVec) + kVec * lane + (j % kVec);
    };
    auto gcol = [&](int64_t a) { return lcol ? halo_idx[h0 + lcol[a]] : sell_col[a]; };
    int32_t group_at[S];
    for (int32_t p = 0; p < maxlen; ++p) {
        uint32_t used = 0;
#pragma unroll
        for (int32_t l = 0; l < S; ++l) {
            if (p >= len[l]) continue;
            const int32_t lane = lane0 + l;
            // the entry stays inside its band (previous, next, own chunk)
            const int32_t band_end = p < np[l] ? np[l] : (p < nb[l] ? nb[l] : len[l]);
            const int32_t lim = min(band_end, p + kSpreadLook);
            int32_t pick = -1, slot = 0, grp = 0;
            for (int32_t j = p; j < lim; ++j) {
                const int32_t c = gcol(at(lane, j));
                slot = c % S;
                grp = c / S;
                if (!((used >> slot) & 1u) || group_at[slot] == grp) {
                    pick = j;
                    break;
                }
            }
            if (pick < 0) continue;   // every candidate conflicts: keep the entry at p
            if (!((used >> slot) & 1u)) {
                used |= 1u << slot;
                group_at[slot] = grp;
            }
            if (pick == p) continue;
            const int64_t a = at(lane, p), b = at(lane, pick);
            if (lcol) {
                const uint16_t x = lcol[a];
                lcol[a] = lcol[b];
                lcol[b] = x;
            } else {
                const int32_t x = sell_col[a];
                sell_col[a] = sell_col[b];
                sell_col[b] = x;
            }
            if (sell_wb) {
                const __nv_bfloat16 x = sell_wb[a];
                sell_wb[a] = sell_wb[b];
                sell_wb[b] = x;
            }
            if (sell_w) {
                const float x = sell_w[a];
                sell_w[a] = sell_w[b];
                sell_w[b] = x;
            }
        }
    }
}

__global__ void spread_kernel(int32_t n_slices, const int64_t *__restrict__ slice_off,
                              const uint32_t *__restrict__ rowinfo, uint32_t len_mask,
                              const uint32_t *__restrict__ rowcls,
                              int32_t *__restrict__ sell_col,
                              uint16_t *__restrict__ lcol, const int64_t *__restrict__ halo_off,
                              const int32_t *__restrict__ halo_idx, float *__restrict__ sell_w,
                              __nv_bfloat16 *__restrict__ sell_wb) {
    constexpr int groups = kSliceRows / kSpreadLanes;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_slices * groups) return;
    spread_quarter(t / groups, (int32_t)(t % groups) * kSpreadLanes, slice_off, rowinfo, len_mask, rowcls,
                   sell_col, lcol, halo_off, halo_idx, sell_w, sell_wb);
}

// Row tags of a problem that shares another problem's operator: the row
// lengths come from the base's rowinfo, the tags from the new fidelity data
// (original node order, checked like the validation kernel does).
__global__ void retag_kernel(int32_t n_pad, int32_t K, const uint32_t *__restrict__ base_rowinfo,
                             const int32_t *__restrict__ perm, const uint8_t *__restrict__ mask,
                             const int32_t *__restrict__ labels, uint32_t *__restrict__ rowinfo,
                             uint32_t *__restrict__ status) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const uint32_t len = base_rowinfo[r] >> 8;
    const int32_t old = perm[r];
    uint32_t tag = kTagUnlabelled;
    if (old >= 0) {
        const uint8_t m = mask[old];
        if (m > 1) atomicOr(status, kBadGraph);
        if (m == 1) {
            const int32_t l = labels[old];
            const int32_t hiK = K == 1 ? 2 : K;
            if (l < 0 || l >= hiK) atomicOr(status, kBadGraph);
            else tag = (uint32_t)l;
        }
    }
    rowinfo[r] = (len << 8) | tag;
}

__global__ void init_u_kernel(int32_t n_pad, int32_t K, const uint32_t *__restrict__ rowinfo,
                              float *__restrict__ u) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_pad * K) return;
    const int64_t r = q / K;
    const int32_t k = (int32_t)(q - r * K);
    const uint32_t tag = rowinfo[r] & 0xFFu;
    float v;
    if (tag == kTagUnlabelled) v = K == 1 ? 0.0f : 2.0f / K - 1.0f;
    else if (K == 1) v = tag == 1u ? 1.0f : -1.0f;
    else v = tag == (uint32_t)k ? 1.0f : -1.0f;
    u[q] = v;
}

}  // namespace

cudaError_t launch_validate(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col,
                            const float *w, const uint8_t *mask, const int32_t *labels, double *deg, double *isd,
                            uint32_t *status, cudaStream_t st) {
    count_launches(1);
    const int64_t threads = (int64_t)n * kValLanes;
    validate_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, K, row_ptr, col, w, mask, labels, deg, isd,
                                                                        status);
    return cudaGetLastError();
}

cudaError_t launch_order_layout(int32_t n, int32_t n_pad, int32_t split, const int64_t *row_ptr, int32_t *perm,
                                int32_t *iperm, int32_t *count, int64_t *scan_tmp, int64_t *slice_off,
                                cudaStream_t st) {
    const int32_t n_slices = n_pad / kSliceRows;
    count_launches(2);
    order_perm_kernel<<<(n_pad + 255) / 256, 256, 0, st>>>(n, n_pad, perm, iperm);
    slice_count_kernel<<<(unsigned)(((int64_t)n_slices * 32 + 255) / 256), 256, 0, st>>>(n, n_slices, split, row_ptr,
                                                                                         perm, count);
    const int64_t nb = (n_slices + kScanBlock - 1) / kScanBlock;
    exclusive_scan(n_slices, count, slice_off, scan_tmp, scan_tmp + nb, st);
    return cudaGetLastError();
}

int64_t order_layout_scan_words(int32_t n_slices) { return (n_slices + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t launch_window_sort(int32_t n, int32_t n_pad, int32_t sigma, const int64_t *row_ptr,
                               int32_t *perm, int32_t *iperm, cudaStream_t st) {
    const size_t smem = (size_t)sigma * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(window_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int windows = (int)(((int64_t)n + sigma - 1) / sigma);
    const int threads = sigma / 2 < 1024 ? sigma / 2 : 1024;
    count_launches(1);
    window_sort_kernel<<<windows, threads, smem, st>>>(n, n_pad, sigma, row_ptr, perm, iperm);
    return cudaGetLastError();
}

cudaError_t launch_pack(int32_t n, int32_t n_pad, int32_t K, const int64_t *row_ptr, const int32_t *col,
                        const float *w, const double *deg, const double *isd, const uint8_t *mask,
                        const int32_t *labels,
                        const int32_t *perm, const int32_t *iperm, const int64_t *slice_off,
                        int32_t *sell_col, float *sell_w, __nv_bfloat16 *sell_wb, float *self, float *dsq,
                        uint32_t *rowinfo, uint32_t *rowcls, int32_t split_len, const int32_t *ov_index,
                        const int64_t *ov_rp, int32_t *ov_col, float *ov_w, __nv_bfloat16 *ov_wb, uint32_t *status,
                        cudaStream_t st) {
    (void)n;
    (void)K;
    count_launches(1);
    pack_kernel<<<(n_pad + 255) / 256, 256, 0, st>>>(n_pad, row_ptr, col, w, deg, isd, mask, labels, perm,
                                                     iperm, slice_off, sell_col, sell_w, sell_wb, self, dsq,
                                                     rowinfo, rowcls, split_len, ov_index, ov_rp, ov_col, ov_w,
                                                     ov_wb, status);
    return cudaGetLastError();
}

cudaError_t launch_compress(int32_t n_slices, const int64_t *slice_off, const uint32_t *rowcls,
                            const int32_t *sell_col, uint16_t *col16, uint32_t *rowinfo, uint8_t *slice_fmt,
                            cudaStream_t st) {
    if (n_slices <= 0) return cudaSuccess;
    count_launches(1);
    compress_kernel<<<(n_slices + kFmtGroupSlices - 1) / kFmtGroupSlices, kFmtGroupSlices * 32, 0, st>>>(
        n_slices, slice_off, rowcls, sell_col, col16, rowinfo, slice_fmt);
    return cudaGetLastError();
}

cudaError_t launch_pack_tiled(int32_t n_pad, const int64_t *row_ptr, const int32_t *col, const float *w,
                              const double *deg, const double *isd, const uint8_t *mask, const int32_t *labels,
                              const int32_t *perm, const int32_t *iperm, const int64_t *slice_off,
                              const int64_t *halo_off, const int32_t *halo_idx, uint16_t *lcol,
                              float *sell_w, uint32_t *rowinfo, uint32_t *status, cudaStream_t st) {
    count_launches(1);
    pack_tiled_kernel<<<(n_pad + 255) / 256, 256, 0, st>>>(n_pad, row_ptr, col, w, deg, isd, mask, labels, perm,
                                                           iperm, slice_off, halo_off, halo_idx, lcol, sell_w,
                                                           rowinfo, status);
    return cudaGetLastError();
}

cudaError_t launch_spread(int32_t n_pad, const int64_t *slice_off, const uint32_t *rowinfo, uint32_t len_mask,
                          const uint32_t *rowcls, int32_t *sell_col, uint16_t *lcol, const int64_t *halo_off,
                          const int32_t *halo_idx, float *sell_w, __nv_bfloat16 *sell_wb, cudaStream_t st) {
    const int32_t n_slices = n_pad / kSliceRows;
    const int64_t threads = (int64_t)n_slices * (kSliceRows / kSpreadLanes);
    if (threads == 0) return cudaSuccess;
    count_launches(1);
    spread_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(n_slices, slice_off, rowinfo, len_mask, rowcls,
                                                                     sell_col, lcol, halo_off, halo_idx, sell_w,
                                                                     sell_wb);
    return cudaGetLastError();
}

cudaError_t launch_retag(int32_t n_pad, int32_t K, const uint32_t *base_rowinfo, const int32_t *perm,
                         const uint8_t *mask, const int32_t *labels, uint32_t *rowinfo, uint32_t *status,
                         cudaStream_t st) {
    count_launches(1);
    retag_kernel<<<(n_pad + 255) / 256, 256, 0, st>>>(n_pad, K, base_rowinfo, perm, mask, labels, rowinfo,
                                                      status);
    return cudaGetLastError();
}

cudaError_t launch_init_u(int32_t n_pad, int32_t K, const uint32_t *rowinfo, float *u, cudaStream_t st) {
    const int64_t tot = (int64_t)n_pad * K;
    count_launches(1);
    init_u_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_pad, K, rowinfo, u);
    return cudaGetLastError();
}

}  // namespace pdca
