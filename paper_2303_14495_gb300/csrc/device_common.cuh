// Device helpers shared by the kernels of the library: row I/O in FP32 and in
// 16-bit storage types, the sliced-ELL gathers, the simplex projection and
// the block reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <string.h>

#include <type_traits>

#include "pdca_internal.cuh"

namespace pdca {
namespace dev {

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

// The same with st.global.cs, for problems whose iterates exceed L2: a pass
// writes each row once and reads it only in the next pass, after the whole
// graph has streamed through the caches.
template <int K>
__device__ __forceinline__ void store_row_cs(float *__restrict__ p, const float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            __stcs(reinterpret_cast<float4 *>(p) + q, make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]));
    } else {
        store_row<K>(p, x);
    }
}

template <int K>
__device__ __forceinline__ void load_row_smem(const float *p, float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = reinterpret_cast<const float4 *>(p)[q];
            x[4 * q + 0] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const float2 t = reinterpret_cast<const float2 *>(p)[q];
            x[2 * q + 0] = t.x; x[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) x[q] = p[q];
    }
}

template <int K>
__device__ __forceinline__ void store_row_smem(float *p, const float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) reinterpret_cast<float2 *>(p)[q] = make_float2(x[2 * q], x[2 * q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = x[q];
    }
}

// acc[k] = sum_j wt_ij * x_jk over the lane's row of the slice (padding
// entries carry weight 0 and point at a valid row).  `len` is the lane's own
// row length: the lane reads only its ceil(len / kVec) groups (kVec
// consecutive entries per 128-bit load, two groups per iteration), so the
// slice padding beyond a row's end is never fetched.  Plain form: global columns, rows gathered from global
// memory through L1/L2.
template <int K>
__device__ __forceinline__ void fma_row(float (&acc)[K], float w, const float (&x)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fmaf(w, x[k], acc[k]);
}

// 16-bit storage types (FP16 / BF16) of u in the mixed-precision path.
template <class T>
__device__ __forceinline__ float2 unpack2(unsigned v) {
    if constexpr (std::is_same_v<T, __half>) {
        __half2 h;
        memcpy(&h, &v, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 h;
        memcpy(&h, &v, 4);
        return __bfloat1622float2(h);
    }
}
template <class T>
__device__ __forceinline__ unsigned pack2(float a, float b) {
    unsigned v;
    if constexpr (std::is_same_v<T, __half>) {
        const __half2 h = __floats2half2_rn(a, b);
        memcpy(&v, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        memcpy(&v, &h, 4);
    }
    return v;
}

// K values of type T at p (row start, aligned to K * sizeof(T)) as floats.
template <int K, class T>
__device__ __forceinline__ void load_row_t(const T *__restrict__ p, float (&x)[K]) {
    if constexpr (std::is_same_v<T, float>) {
        load_row<K>(p, x);
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p) + q);
            const float2 a = unpack2<T>(t.x), b = unpack2<T>(t.y);
            x[4 * q + 0] = a.x; x[4 * q + 1] = a.y; x[4 * q + 2] = b.x; x[4 * q + 3] = b.y;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const float2 a = unpack2<T>(__ldg(reinterpret_cast<const unsigned *>(p) + q));
            x[2 * q + 0] = a.x; x[2 * q + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p) + q);
            const float2 a = unpack2<T>((unsigned)b);
            x[q] = a.x;
        }
    }
}

template <int K, class T>
__device__ __forceinline__ void store_row_t(T *__restrict__ p, const float (&x)[K]) {
    if constexpr (std::is_same_v<T, float>) {
        store_row<K>(p, x);
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            reinterpret_cast<uint2 *>(p)[q] =
                make_uint2(pack2<T>(x[4 * q], x[4 * q + 1]), pack2<T>(x[4 * q + 2], x[4 * q + 3]));
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) reinterpret_cast<unsigned *>(p)[q] = pack2<T>(x[2 * q], x[2 * q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if constexpr (std::is_same_v<T, __half>) p[q] = __float2half_rn(x[q]);
            else p[q] = __float2bfloat16_rn(x[q]);
        }
    }
}

// Entry-stream loads that bypass L1 allocation: every column index and
// weight is read exactly once per pass, so L1 keeps its capacity for the
// gathered rows of the iterate.
__device__ __forceinline__ int4 ld_stream(const int4 *p) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_stream(const uint2 *p) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) {
    uint32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

// the four weights of one entry group
template <class WT>
__device__ __forceinline__ float4 load_w_group(const WT *p) {
    if constexpr (std::is_same_v<WT, float>) {
        return ld_stream(reinterpret_cast<const float4 *>(p));
    } else {
        const uint2 t = ld_stream(reinterpret_cast<const uint2 *>(p));
        const float2 a = unpack2<__nv_bfloat16>(t.x), b = unpack2<__nv_bfloat16>(t.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
}
template <class WT>
__device__ __forceinline__ const WT *weights_of(const SellView &A) {
    if constexpr (std::is_same_v<WT, float>) return A.w;
    else return A.wb;
}

// ---------------------------------------------------------------------------
// plain gathers: acc[k] = sum_j wt_ij x_jk over the lane's row, in either
// column format of the slice (int32 columns, or 16-bit columns whose chunk
// follows from the entry's band).  `info` is the row's rowinfo word.  The
// lane reads only its own ceil(len / kVec) groups, so the slice padding
// beyond a row's end is never fetched; the padding inside a row's last
// group points at the row itself with weight 0.
// ---------------------------------------------------------------------------
template <bool C16> struct ColFmt { using G = int4; };          // four int32 columns
template <> struct ColFmt<true> { using G = uint2; };           // four 16-bit columns
template <class WT> struct WFmt { using G = float4; };          // four FP32 weights
template <> struct WFmt<__nv_bfloat16> { using G = uint2; };    // four BF16 weights

template <class WT>
__device__ __forceinline__ float4 wgroup(const typename WFmt<WT>::G &g) {
    if constexpr (std::is_same_v<WT, float>) {
        return g;
    } else {
        const float2 a = unpack2<__nv_bfloat16>(g.x), b = unpack2<__nv_bfloat16>(g.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// the row's entries in the sliced ELL (plain kernels, either format)
__device__ __forceinline__ int info_len(uint32_t info, bool) { return (int)((info >> 8) & kLenMask); }

// A row longer than the split length continues in the overflow CSR: add the
// pre-pass's sum of its remaining entries (after the sliced entries, so the
// order of the additions is fixed).
template <int K>
__device__ __forceinline__ void add_overflow(const SellView &A, int r, uint32_t info, float (&acc)[K]) {
    if (info & kOvFlag) {
        const float *p = A.ov_acc + (size_t)__ldg(A.ov_index + r) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += __ldg(p + k);
    }
}

// Bands of a row with 16-bit columns: entries j < np lie in the previous
// 65536-node chunk, np <= j < nb in the next one, the rest (and the padding)
// in the row's own chunk, which starts at node `own`.
struct Bands {
    int own, np, nb;
};
template <bool C16>
__device__ __forceinline__ Bands bands_of(uint32_t info, int r) {
    Bands b{0, 0, 0};
    if constexpr (C16) {
        b.own = r & ~((1 << kChunkShift) - 1);
        b.np = (int)((info >> 20) & kBandMax);
        b.nb = b.np + (int)((info >> 26) & kBandMax);
    }
    return b;
}

__device__ __forceinline__ int group_col(const int4 &c, int i);
__device__ __forceinline__ int group_col(const uint2 &c, int i);
// column i of entry group g
__device__ __forceinline__ int entry_col(const int4 &c, int i, int, const Bands &) { return group_col(c, i); }
__device__ __forceinline__ int entry_col(const uint2 &c, int i, int g, const Bands &b) {
    const int j = kVec * g + i;
    const int hi = j < b.np ? b.own - (1 << kChunkShift) : (j < b.nb ? b.own + (1 << kChunkShift) : b.own);
    return hi + group_col(c, i);
}

// Entry streams of one lane's row, with the first two groups loaded ahead.
template <bool C16, class WT>
struct EntryStream {
    using CG = typename ColFmt<C16>::G;
    using WG = typename WFmt<WT>::G;
    const CG *cp;
    const WG *wp;
    CG c0, c1;
    WG w0, w1;
    int wg;   // entry groups of the slice (its width / kVec)
};

// Issue the loads of the first two entry groups (they depend only on the
// slice) -- before the row's own data, so their latency overlaps it.  Group
// 0 always exists (every slice is at least kVec wide); group 1 is loaded when
// the slice has it.
template <bool C16, class WT>
__device__ __forceinline__ void stream_open(const SellView &A, int slice, int lane, EntryStream<C16, WT> &s) {
    const int64_t base = A.slice_off[slice];
    s.wg = (int)((A.slice_off[slice + 1] - base) >> 5) / kVec;
    if constexpr (C16) s.cp = reinterpret_cast<const uint2 *>(A.col16 + base) + lane;
    else s.cp = reinterpret_cast<const int4 *>(A.col + base) + lane;
    s.wp = reinterpret_cast<const typename WFmt<WT>::G *>(weights_of<WT>(A) + base) + lane;
    const int width_groups = (int)((A.slice_off[slice + 1] - base) >> 5) / kVec;
    s.c0 = ld_stream(s.cp);
    s.w0 = ld_stream(s.wp);
    if (width_groups > 1) {
        s.c1 = ld_stream(s.cp + 32);
        s.w1 = ld_stream(s.wp + 32);
    }
}

template <int K, class XT, class CG>
__device__ __forceinline__ void fma_entry_group(float (&acc)[K], const CG &c, const float4 &w, int g,
                                                const Bands &b, const XT *__restrict__ x) {
    float r0[K], r1[K], r2[K], r3[K];
    load_row_t<K, XT>(x + (size_t)entry_col(c, 0, g, b) * K, r0);
    load_row_t<K, XT>(x + (size_t)entry_col(c, 1, g, b) * K, r1);
    load_row_t<K, XT>(x + (size_t)entry_col(c, 2, g, b) * K, r2);
    load_row_t<K, XT>(x + (size_t)entry_col(c, 3, g, b) * K, r3);
    fma_row<K>(acc, w.x, r0);
    fma_row<K>(acc, w.y, r1);
    fma_row<K>(acc, w.z, r2);
    fma_row<K>(acc, w.w, r3);
}

// The gather proper: while a lane works on two entry groups the next two are
// in flight; products are added in entry order.
// OV = false leaves out the overflow sums (problems without split rows; the
// check alone costs the FP32 sweep about 3% on GB300).
template <int K, bool C16, class WT, class XT, bool OV = true>
__device__ __forceinline__ void stream_gather(const SellView &A, EntryStream<C16, WT> &s, uint32_t info, int r,
                                              const XT *__restrict__ x, float (&acc)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const Bands b = bands_of<C16>(info, r);
    // every lane walks the slice's whole width: a padding entry holds the
    // lane's own row with weight 0 and adds nothing, and with one trip count
    // for the warp the loads of consecutive groups overlap better than with
    // a trip count per lane (2% on the FP32 sweep, measured)
    const int groups = s.wg;
    for (int g = 0; g < groups; g += 2) {
        typename ColFmt<C16>::G n0 = s.c0, n1 = s.c1;
        typename WFmt<WT>::G nw0 = s.w0, nw1 = s.w1;
        if (g + 2 < groups) {
            n0 = ld_stream(s.cp + 32 * (g + 2));
            nw0 = ld_stream(s.wp + 32 * (g + 2));
        }
        if (g + 3 < groups) {
            n1 = ld_stream(s.cp + 32 * (g + 3));
            nw1 = ld_stream(s.wp + 32 * (g + 3));
        }
        fma_entry_group<K, XT>(acc, s.c0, wgroup<WT>(s.w0), g, b, x);
        if (g + 1 < groups) fma_entry_group<K, XT>(acc, s.c1, wgroup<WT>(s.w1), g + 1, b, x);
        s.c0 = n0;
        s.w0 = nw0;
        s.c1 = n1;
        s.w1 = nw1;
    }
    if constexpr (OV) add_overflow<K>(A, r, info, acc);
}

// The gather without look-ahead: each step loads two entry groups, then
// their eight rows, then adds the products in entry order.  It holds fewer
// registers than stream_gather; the mixed-precision passes use it and keep
// six blocks per SM.
template <int K, bool C16, class WT, class XT, bool OV = true>
__device__ __forceinline__ void short_gather(const SellView &A, int slice, int lane, uint32_t info, int r,
                                             const XT *__restrict__ x, float (&acc)[K]) {
    using CG = typename ColFmt<C16>::G;
    using WG = typename WFmt<WT>::G;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const int64_t base = A.slice_off[slice];
    const CG *cp;
    if constexpr (C16) cp = reinterpret_cast<const uint2 *>(A.col16 + base) + lane;
    else cp = reinterpret_cast<const int4 *>(A.col + base) + lane;
    const WG *wp = reinterpret_cast<const WG *>(weights_of<WT>(A) + base) + lane;
    const Bands b = bands_of<C16>(info, r);
    // this lane's own groups (walking the slice's whole width, as
    // stream_gather does, made the mixed passes 9% slower)
    const int groups = (info_len(info, C16) + kVec - 1) / kVec;
    int g = 0;
    for (; g + 2 <= groups; g += 2) {
        const CG ca = ld_stream(cp + 32 * g), cb = ld_stream(cp + 32 * (g + 1));
        const float4 wa = wgroup<WT>(ld_stream(wp + 32 * g)), wb = wgroup<WT>(ld_stream(wp + 32 * (g + 1)));
        float x0[K], x1[K], x2[K], x3[K], y0[K], y1[K], y2[K], y3[K];   // all eight rows in flight
        load_row_t<K, XT>(x + (size_t)entry_col(ca, 0, g, b) * K, x0);
        load_row_t<K, XT>(x + (size_t)entry_col(ca, 1, g, b) * K, x1);
        load_row_t<K, XT>(x + (size_t)entry_col(ca, 2, g, b) * K, x2);
        load_row_t<K, XT>(x + (size_t)entry_col(ca, 3, g, b) * K, x3);
        load_row_t<K, XT>(x + (size_t)entry_col(cb, 0, g + 1, b) * K, y0);
        load_row_t<K, XT>(x + (size_t)entry_col(cb, 1, g + 1, b) * K, y1);
        load_row_t<K, XT>(x + (size_t)entry_col(cb, 2, g + 1, b) * K, y2);
        load_row_t<K, XT>(x + (size_t)entry_col(cb, 3, g + 1, b) * K, y3);
        fma_row<K>(acc, wa.x, x0); fma_row<K>(acc, wa.y, x1);
        fma_row<K>(acc, wa.z, x2); fma_row<K>(acc, wa.w, x3);
        fma_row<K>(acc, wb.x, y0); fma_row<K>(acc, wb.y, y1);
        fma_row<K>(acc, wb.z, y2); fma_row<K>(acc, wb.w, y3);
    }
    if (g < groups) {
        const CG ca = ld_stream(cp + 32 * g);
        const float4 wa = wgroup<WT>(ld_stream(wp + 32 * g));
        fma_entry_group<K, XT>(acc, ca, wa, g, b, x);
    }
    if constexpr (OV) add_overflow<K>(A, r, info, acc);
}

// Column format of the slices one block handles.  The format is decided per
// group of kFmtGroupSlices slices, and every block of the plain kernels works
// inside one group (queue ranges of 8, 16 or 32 slices aligned to their size;
// 8 slices in the batched and spectral kernels), so the branch is uniform over
// the block and the two forms of a kernel body never share registers.
__device__ __forceinline__ bool block_fmt16(const SellView &A, int first_slice) {
    return A.slice_fmt != nullptr && __ldg(A.slice_fmt + first_slice) == kFmt16;
}

// One row's gather with nothing else overlapped; returns its rowinfo word.
template <int K, class WT, class XT, bool C16>
__device__ __forceinline__ uint32_t row_gather(const SellView &A, int slice, int lane, const XT *__restrict__ x,
                                               float (&acc)[K]) {
    const int r = slice * kSliceRows + lane;
    const uint32_t info = ld_stream(A.rowinfo + r);
    EntryStream<C16, WT> s;
    stream_open(A, slice, lane, s);
    stream_gather<K, C16, WT, XT>(A, s, info, r, x, acc);
    return info;
}

// Tiled form: 16-bit local columns (four per 64-bit load) into the halo rows
// held in shared memory.
template <int K>
__device__ __forceinline__ void gather_row_sum_smem(const TileView &T, const SellView &A, int64_t base,
                                                    int len, int lane, const float *hs, float (&acc)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const uint2 *__restrict__ cp = reinterpret_cast<const uint2 *>(T.lcol + base) + lane;
    const float4 *__restrict__ wp = reinterpret_cast<const float4 *>(A.w + base) + lane;
    const int groups = (len + kVec - 1) / kVec;
    int g = 0;
    for (; g + 2 <= groups; g += 2) {
        const uint2 ca = __ldcs(cp + 32 * g), cb = __ldcs(cp + 32 * (g + 1));
        const float4 wa = __ldcs(wp + 32 * g), wb = __ldcs(wp + 32 * (g + 1));
        float x0[K], x1[K], x2[K], x3[K];
        load_row_smem<K>(hs + (ca.x & 0xFFFFu) * K, x0);
        load_row_smem<K>(hs + (ca.x >> 16) * K, x1);
        load_row_smem<K>(hs + (ca.y & 0xFFFFu) * K, x2);
        load_row_smem<K>(hs + (ca.y >> 16) * K, x3);
        fma_row<K>(acc, wa.x, x0); fma_row<K>(acc, wa.y, x1);
        fma_row<K>(acc, wa.z, x2); fma_row<K>(acc, wa.w, x3);
        load_row_smem<K>(hs + (cb.x & 0xFFFFu) * K, x0);
        load_row_smem<K>(hs + (cb.x >> 16) * K, x1);
        load_row_smem<K>(hs + (cb.y & 0xFFFFu) * K, x2);
        load_row_smem<K>(hs + (cb.y >> 16) * K, x3);
        fma_row<K>(acc, wb.x, x0); fma_row<K>(acc, wb.y, x1);
        fma_row<K>(acc, wb.z, x2); fma_row<K>(acc, wb.w, x3);
    }
    if (g < groups) {
        const uint2 ca = __ldcs(cp + 32 * g);
        const float4 wa = __ldcs(wp + 32 * g);
        float x0[K], x1[K], x2[K], x3[K];
        load_row_smem<K>(hs + (ca.x & 0xFFFFu) * K, x0);
        load_row_smem<K>(hs + (ca.x >> 16) * K, x1);
        load_row_smem<K>(hs + (ca.y & 0xFFFFu) * K, x2);
        load_row_smem<K>(hs + (ca.y >> 16) * K, x3);
        fma_row<K>(acc, wa.x, x0); fma_row<K>(acc, wa.y, x1);
        fma_row<K>(acc, wa.z, x2); fma_row<K>(acc, wa.w, x3);
    }
}

// Tiled form for a tile whose halo exceeds the shared-memory allocation: the
// local column indexes the tile's halo list, which gives the global row.
template <int K>
__device__ __forceinline__ void gather_row_sum_indirect(const TileView &T, const SellView &A, int64_t base,
                                                        int len, int lane, const int32_t *__restrict__ hidx,
                                                        const float *__restrict__ x, float (&acc)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const uint2 *__restrict__ cp = reinterpret_cast<const uint2 *>(T.lcol + base) + lane;
    const float4 *__restrict__ wp = reinterpret_cast<const float4 *>(A.w + base) + lane;
    const int groups = (len + kVec - 1) / kVec;
    for (int g = 0; g < groups; ++g) {
        const uint2 ca = __ldcs(cp + 32 * g);
        const float4 wa = __ldcs(wp + 32 * g);
        float x0[K], x1[K], x2[K], x3[K];
        load_row<K>(x + (size_t)__ldg(hidx + (ca.x & 0xFFFFu)) * K, x0);
        load_row<K>(x + (size_t)__ldg(hidx + (ca.x >> 16)) * K, x1);
        load_row<K>(x + (size_t)__ldg(hidx + (ca.y & 0xFFFFu)) * K, x2);
        load_row<K>(x + (size_t)__ldg(hidx + (ca.y >> 16)) * K, x3);
        fma_row<K>(acc, wa.x, x0); fma_row<K>(acc, wa.y, x1);
        fma_row<K>(acc, wa.z, x2); fma_row<K>(acc, wa.w, x3);
    }
}

// Gather for one row of a tile: from shared memory when the tile's halo is
// staged there, through the halo list otherwise.
template <int K>
__device__ __forceinline__ void tile_row_sum(const TileView &T, const SellView &A, int64_t base, int len,
                                             int lane, bool staged, const int32_t *__restrict__ hidx,
                                             const float *hs, const float *__restrict__ x, float (&acc)[K]) {
    if (staged) gather_row_sum_smem<K>(T, A, base, len, lane, hs, acc);
    else gather_row_sum_indirect<K>(T, A, base, len, lane, hidx, x, acc);
}

// Copy the tile's halo rows of x into shared memory (rows in halo order).
// Batches of four rows per thread: the four index loads, then the four row
// loads, then the four shared-memory stores, so a batch costs one index and
// one row latency whatever the halo size.
template <int K>
__device__ __forceinline__ void load_halo(const TileView &T, int tile, const float *__restrict__ x, float *hs) {
    const int64_t h0 = T.halo_off[tile];
    const int h = (int)(T.halo_off[tile + 1] - h0);
    const int32_t *__restrict__ idx = T.halo_idx + h0;
    const int bd = blockDim.x;
    for (int q0 = threadIdx.x; q0 < h; q0 += 4 * bd) {
        int32_t i[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) i[m] = (q0 + m * bd < h) ? __ldcs(idx + q0 + m * bd) : -1;
        float r[4][K];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (i[m] >= 0) load_row<K>(x + (size_t)i[m] * K, r[m]);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (i[m] >= 0) store_row_smem<K>(hs + (q0 + m * bd) * K, r[m]);
    }
}

__device__ __forceinline__ int row_len(const SellView &A, int slice, int lane) {
    return (int)(__ldg(A.rowinfo + slice * kSliceRows + lane) >> 8);
}

// prior y_ik in the +-1 coding from the row tag
template <int K>
__device__ __forceinline__ float prior_of(uint32_t tag, int k) {
    if (K == 1) return tag == 1u ? 1.0f : -1.0f;
    return tag == (uint32_t)k ? 1.0f : -1.0f;
}

// Euclidean projection of a row onto the simplex in the coding v = (u+1)/2
// (sort-and-threshold method of Held, Wolfe and Crowder), written directly in
// u: with u sorted descending and S_j = sum_{i<=j} u_(i), rho is the largest
// j with j u_(j) - S_j + 2 > 0, lambda = (S_rho + rho - 2)/rho (twice the
// threshold theta of the v coding) and u' = max(u - lambda, -1).
// The threshold sums S_j are kept as an unevaluated pair hi + lo of floats
// (Knuth's TwoSum), about 48 significant bits, so no FP64 unit is needed.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

template <int K>
__device__ __forceinline__ void project_simplex(float (&u)[K]) {
    float mu[K];
#pragma unroll
    for (int k = 0; k < K; ++k) mu[k] = u[k];
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j + 1 < K - i; ++j) {
            const float a = mu[j], b = mu[j + 1];
            mu[j] = fmaxf(a, b);
            mu[j + 1] = fminf(a, b);
        }
    }
    float hi = 0.0f, lo = 0.0f, s_hi = mu[0], s_lo = 0.0f;
    int rho = 1;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float e;
        two_sum(hi, mu[j], hi, e);
        lo += e;
        if (((float)(j + 1) * mu[j] - hi) - lo + 2.0f > 0.0f) {
            rho = j + 1;
            s_hi = hi;
            s_lo = lo;
        }
    }
    const float lam = (((s_hi - 2.0f) + (float)rho) + s_lo) / (float)rho;
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] = fmaxf(u[k] - lam, -1.0f);
}


// Reductions.  Per-row terms are formed in FP32; sums over rows are kept as
// an unevaluated pair hi + lo of floats (TwoSum of every addition, about 48
// significant bits: compensated summation in the FP32 pipe, because FP64
// throughput on GB300 is a small fraction of FP32's) inside a warp, and in
// FP64 across warps and blocks.  Fixed shuffle tree, fixed order.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// (hi, lo) += (bhi, blo) for two-float numbers (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ void df_add(float &hi, float &lo, float bhi, float blo) {
    float sum, err;
    two_sum(hi, bhi, sum, err);
    err += lo + blo;
    hi = sum + err;
    lo = err - (hi - sum);
}

// Sum of v over the warp's 32 lanes in two-float arithmetic, as a double
// (the value lane 0 holds is the one used).
__device__ __forceinline__ double warp_sum_df(float v) {
    float hi = v, lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bhi = __shfl_xor_sync(kFull, hi, o), blo = __shfl_xor_sync(kFull, lo, o);
        df_add(hi, lo, bhi, blo);
    }
    return (double)hi + (double)lo;
}

// Sums of eight per-lane values over the warp's 32 lanes in two-float
// arithmetic, with 9 shuffle pairs instead of 40: at each of the first three
// levels a lane keeps half of its values and sends the other half to its
// partner (lane ^ 16, ^ 8, ^ 4), the last two levels add whole values.  The
// pattern is fixed, so the result is too.  On return lane l holds the total
// of value q(l) = 4 [l & 16] + 2 [l & 8] + [l & 4] (four lanes per value).
__device__ __forceinline__ double warp_sum8_df(const float (&v)[8]) {
    const int lane = threadIdx.x & 31;
    float hi[4], lo[4];
    {
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float keep = up ? v[i + 4] : v[i], send = up ? v[i] : v[i + 4];
            hi[i] = keep;
            lo[i] = 0.0f;
            df_add(hi[i], lo[i], __shfl_xor_sync(kFull, send, 16), 0.0f);
        }
    }
    {
        const bool up = (lane & 8) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            float khi = up ? hi[i + 2] : hi[i], klo = up ? lo[i + 2] : lo[i];
            const float shi = up ? hi[i] : hi[i + 2], slo = up ? lo[i] : lo[i + 2];
            df_add(khi, klo, __shfl_xor_sync(kFull, shi, 8), __shfl_xor_sync(kFull, slo, 8));
            hi[i] = khi;
            lo[i] = klo;
        }
    }
    {
        const bool up = (lane & 4) != 0;
        float khi = up ? hi[1] : hi[0], klo = up ? lo[1] : lo[0];
        const float shi = up ? hi[0] : hi[1], slo = up ? lo[0] : lo[1];
        df_add(khi, klo, __shfl_xor_sync(kFull, shi, 4), __shfl_xor_sync(kFull, slo, 4));
        hi[0] = khi;
        lo[0] = klo;
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
        const float bhi = __shfl_xor_sync(kFull, hi[0], o), blo = __shfl_xor_sync(kFull, lo[0], o);
        df_add(hi[0], lo[0], bhi, blo);
    }
    return (double)hi[0] + (double)lo[0];
}

// Sum S values over the block (WARPS warps) in a fixed order and store them
// at out[0..S): each warp sums its 32 lanes in two-float arithmetic, the
// warp totals are summed in FP64.
template <int S, int WARPS = kWarpsPerBlock>
__device__ __forceinline__ void block_sum_store(float (&v)[S], double *__restrict__ out) {
    __shared__ double sm[WARPS][S];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double t = warp_sum_df(v[s]);
        if (lane == 0) sm[warp][s] = t;
    }
    __syncthreads();
    if (threadIdx.x < S) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < WARPS; ++q) t += sm[q][threadIdx.x];
        out[threadIdx.x] = t;
    }
}


// ---------------------------------------------------------------------------
// One pass over one slice (lane = row), shared by the single-problem kernels
// and the batched kernel.
// ---------------------------------------------------------------------------
// 1/g_i: precomputed per tag for L_s; alpha a_i + beta per row for L
template <bool UN>
__device__ __forceinline__ float inv_g_of(const Coeffs &cf, bool lab, float a) {
    if constexpr (UN) return __frcp_rn(fmaf(cf.alpha, a, lab ? cf.beta1 : cf.beta0));
    else return lab ? cf.inv_g1 : cf.inv_g0;
}

// (L x)_i = a_i x_i - acc with a_i = 1 for L_s
template <bool UN>
__device__ __forceinline__ float lap_row(float a, float x, float acc) {
    if constexpr (UN) return a * x - acc;
    else return x - acc;
}

template <int K, bool PROJECT, bool UN = false>
__device__ __forceinline__ void sweep_update(const Coeffs &cf, uint32_t info, float a, const float (&acc)[K],
                                             const float (&v)[K], const float (&u)[K], float *__restrict__ dst,
                                             bool stream = false) {
    const uint32_t tag = info & 0xFFu;
    const bool lab = tag != kTagUnlabelled;
    const float inv_g = inv_g_of<UN>(cf, lab, a);
    const float diag = cf.c + (lab ? cf.eta : 0.0f);
    float out[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float fid = lab ? cf.eta * prior_of<K>(tag, k) : 0.0f;
        const float uk = u[k];
        const float b = fid + cf.c * uk - (uk * uk * uk - uk) * cf.inv_eps;
        const float tv = cf.eps * lap_row<UN>(a, v[k], acc[k]) + diag * v[k];
        out[k] = v[k] + (b - tv) * inv_g;
    }
    if constexpr (PROJECT) project_simplex<K>(out);
    if (stream) store_row_cs<K>(dst, out);
    else store_row<K>(dst, out);
}

// column i (0..3) of an entry group: int32 global columns or 16-bit locals
__device__ __forceinline__ int group_col(const int4 &c, int i) {
    return i == 0 ? c.x : i == 1 ? c.y : i == 2 ? c.z : c.w;
}
__device__ __forceinline__ int group_col(const uint2 &c, int i) {
    return (int)(i == 0 ? (c.x & 0xFFFFu) : i == 1 ? (c.x >> 16) : i == 2 ? (c.y & 0xFFFFu) : (c.y >> 16));
}

enum GatherMode { kGlobal = 0, kShared = 1, kIndirect = 2 };

template <int K, int MODE>
__device__ __forceinline__ void source_row(int c, const float *__restrict__ x, const float *hs,
                                           const int32_t *__restrict__ hidx, float (&r)[K]) {
    if constexpr (MODE == kGlobal) load_row<K>(x + (size_t)c * K, r);
    else if constexpr (MODE == kShared) load_row_smem<K>(hs + c * K, r);
    else load_row<K>(x + (size_t)__ldg(hidx + c) * K, r);
}

template <int K, int MODE, class IdxT>
__device__ __forceinline__ void fma_group(float (&acc)[K], const IdxT &c, const float4 &w,
                                          const float *__restrict__ x, const float *hs,
                                          const int32_t *__restrict__ hidx) {
    float r0[K], r1[K], r2[K], r3[K];
    source_row<K, MODE>(group_col(c, 0), x, hs, hidx, r0);
    source_row<K, MODE>(group_col(c, 1), x, hs, hidx, r1);
    source_row<K, MODE>(group_col(c, 2), x, hs, hidx, r2);
    source_row<K, MODE>(group_col(c, 3), x, hs, hidx, r3);
    fma_row<K>(acc, w.x, r0);
    fma_row<K>(acc, w.y, r1);
    fma_row<K>(acc, w.z, r2);
    fma_row<K>(acc, w.w, r3);
}

// Slices of a block's range, handed out to its warps in order: a warp takes
// the next untaken slot when it finishes one (a shared-memory counter), so a
// warp with short rows does not idle while another works on long ones, and
// the block retires as soon as the range is done.  The first slot of warp w
// is w; f(slice) runs for every slice of [first, first + count) that exists.
template <class F>
__device__ __forceinline__ void for_block_slices(int first, int count, int n_slices, int *next_slot, F &&f) {
    if (threadIdx.x == 0) *next_slot = kWarpsPerBlock;
    __syncthreads();
    int slot = threadIdx.x >> 5;
#pragma unroll 1
    while (slot < count) {
        const int slice = first + slot;
        if (slice >= n_slices) return;
        f(slice);
        int nxt = 0;
        if ((threadIdx.x & 31) == 0) nxt = atomicAdd(next_slot, 1);
        slot = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// The same, with the body told the block's column format:
// f(slice, std::true_type) for 16-bit columns, f(slice, std::false_type)
// for int32 columns.
template <class F>
__device__ __forceinline__ void for_block_slices_fmt(const SellView &A, int first, int count, int *next_slot,
                                                     F &&f) {
    if (block_fmt16(A, first))
        for_block_slices(first, count, A.n_slices, next_slot, [&](int slice) { f(slice, std::true_type{}); });
    else
        for_block_slices(first, count, A.n_slices, next_slot, [&](int slice) { f(slice, std::false_type{}); });
}

// Per-lane state of one slice row, loaded before the gather (tiled form).
template <int K, class IdxT>
struct SliceRow {
    uint32_t info;
    float a;       // a_i (unnormalized L only)
    int groups;
    const IdxT *cp;
    const float4 *wp;
    float v[K], u[K];
    IdxT c0, c1;
    float4 w0, w1;
};

template <int K, bool UN = false, class IdxT>
__device__ __forceinline__ void slice_prologue(const SellView &A, const IdxT *cols, int slice, int lane,
                                               const float *__restrict__ v_src, const float *__restrict__ u_t,
                                               SliceRow<K, IdxT> &s) {
    const int r = slice * kSliceRows + lane;
    const int64_t base = A.slice_off[slice];
    s.cp = cols + base / kVec + lane;
    s.wp = reinterpret_cast<const float4 *>(A.w + base) + lane;
    // the row's own data is read by this lane only: keep L1 for the gathers
    s.info = ld_stream(A.rowinfo + r);
    s.a = UN ? __ldg(A.self + r) : 1.0f;
    // every real row has an entry and every slice is at least kVec wide, so
    // group 0 always exists; group 1 is loaded when the slice has it
    const int width_groups = (int)((A.slice_off[slice + 1] - base) >> 5) / kVec;
    s.c0 = ld_stream(s.cp);
    s.w0 = ld_stream(s.wp);
    if (width_groups > 1) {
        s.c1 = ld_stream(s.cp + 32);
        s.w1 = ld_stream(s.wp + 32);
    }
    load_row<K>(v_src + (size_t)r * K, s.v);
    if (u_t == v_src) {
#pragma unroll
        for (int k = 0; k < K; ++k) s.u[k] = s.v[k];
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = ld_stream(reinterpret_cast<const float4 *>(u_t + (size_t)r * K) + q);
            s.u[4 * q + 0] = t.x; s.u[4 * q + 1] = t.y; s.u[4 * q + 2] = t.z; s.u[4 * q + 3] = t.w;
        }
    } else {
        load_row<K>(u_t + (size_t)r * K, s.u);
    }
}

template <int K, int MODE, class IdxT>
__device__ __forceinline__ void slice_gather(SliceRow<K, IdxT> &s, const float *__restrict__ x, const float *hs,
                                             const int32_t *__restrict__ hidx, float (&acc)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0f;
    const int groups = (int)((s.info >> 8) + kVec - 1) / kVec;   // this lane's own groups
    for (int g = 0; g < groups; g += 2) {
        IdxT n0 = s.c0, n1 = s.c1;
        float4 nw0 = s.w0, nw1 = s.w1;
        if (g + 2 < groups) {
            n0 = ld_stream(s.cp + 32 * (g + 2));
            nw0 = ld_stream(s.wp + 32 * (g + 2));
        }
        if (g + 3 < groups) {
            n1 = ld_stream(s.cp + 32 * (g + 3));
            nw1 = ld_stream(s.wp + 32 * (g + 3));
        }
        fma_group<K, MODE>(acc, s.c0, s.w0, x, hs, hidx);
        if (g + 1 < groups) fma_group<K, MODE>(acc, s.c1, s.w1, x, hs, hidx);
        s.c0 = n0;
        s.w0 = nw0;
        s.c1 = n1;
        s.w1 = nw1;
    }
}

// The row's own data, read by this lane only (L1 is kept for the gathers).
template <int K>
__device__ __forceinline__ void load_own_row(const float *__restrict__ p, float (&x)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = ld_stream(reinterpret_cast<const float4 *>(p) + q);
            x[4 * q + 0] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    } else {
        load_row<K>(p, x);
    }
}

// FP32 sweep of one slice: the loads that depend on nothing (the row tag and
// length, the first two entry groups, the own rows of v^s and u^t) first,
// then the pipelined gather, then the update.
template <int K, bool PROJECT, bool UN, bool C16, bool OV = true>
__device__ __forceinline__ void fp32_sweep_slice(const SellView &A, const Coeffs &cf, int slice, int lane,
                                                 const float *__restrict__ v_src, const float *__restrict__ u_t,
                                                 float *__restrict__ v_dst) {
    const int r = slice * kSliceRows + lane;
    const uint32_t info = ld_stream(A.rowinfo + r);
    EntryStream<C16, float> s;
    stream_open(A, slice, lane, s);
    const float a = UN ? __ldg(A.self + r) : 1.0f;
    float v[K], u[K];
    load_row<K>(v_src + (size_t)r * K, v);
    if (u_t == v_src) {
#pragma unroll
        for (int k = 0; k < K; ++k) u[k] = v[k];
    } else {
        load_own_row<K>(u_t + (size_t)r * K, u);
    }
    float acc[K];
    stream_gather<K, C16, float, float, OV>(A, s, info, r, v_src, acc);
    sweep_update<K, PROJECT, UN>(cf, info, a, acc, v, u, v_dst + (size_t)r * K, A.stream_rows != 0);
}

// Mixed precision, pass 0 of an outer step: r = b^t - T u^t with FP32
// weights and the FP32 iterate (the FP32 residual correction), stored in
// FP32, and e^1 = G^-1 r in 16-bit storage (or, with a single sweep,
// u^{t+1} = u^t + e^1).
template <int K, class HT, bool LAST, bool PROJECT, bool UN, bool C16, bool OV = true>
__device__ __forceinline__ void mixed_residual_slice(const SellView &A, const Coeffs &cf, int slice, int lane,
                                                     const float *__restrict__ u, float *__restrict__ r_out,
                                                     HT *__restrict__ e_out, float *__restrict__ u_out) {
    const int r = slice * kSliceRows + lane;
    const uint32_t info = ld_stream(A.rowinfo + r);
    const float a = UN ? __ldg(A.self + r) : 1.0f;
    float acc[K];
    short_gather<K, C16, float, float, OV>(A, slice, lane, info, r, u, acc);
    float x[K];
    load_row<K>(u + (size_t)r * K, x);
    const uint32_t tag = info & 0xFFu;
    const bool lab = tag != kTagUnlabelled;
    const float inv_g = inv_g_of<UN>(cf, lab, a);
    float res[K], e[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float fid = lab ? cf.eta * (prior_of<K>(tag, k) - x[k]) : 0.0f;
        res[k] = fid - (x[k] * x[k] * x[k] - x[k]) * cf.inv_eps - cf.eps * lap_row<UN>(a, x[k], acc[k]);
        e[k] = res[k] * inv_g;
    }
    if constexpr (LAST) {
        float out[K];
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = x[k] + e[k];
        if constexpr (PROJECT) project_simplex<K>(out);
        store_row<K>(u_out + (size_t)r * K, out);
    } else {
        store_row<K>(r_out + (size_t)r * K, res);
        store_row_t<K, HT>(e_out + (size_t)r * K, e);
    }
}

// Mixed precision correction sweep with BF16 weights: e' = e + G^-1 (r - T e)
// (r in FP32, e in 16-bit storage); the last one writes u^{t+1} = u^t + e' in
// FP32 (projected for K >= 2).
template <int K, class HT, bool LAST, bool PROJECT, bool UN, bool C16, bool OV = true>
__device__ __forceinline__ void mixed_sweep_slice(const SellView &A, const Coeffs &cf, int slice, int lane,
                                                  const HT *__restrict__ e_src, const float *__restrict__ rr,
                                                  HT *__restrict__ e_dst, const float *__restrict__ u,
                                                  float *__restrict__ u_out) {
    const int r = slice * kSliceRows + lane;
    const uint32_t info = ld_stream(A.rowinfo + r);
    const float a = UN ? __ldg(A.self + r) : 1.0f;
    float acc[K];
    short_gather<K, C16, __nv_bfloat16, HT, OV>(A, slice, lane, info, r, e_src, acc);
    float e[K], res[K];
    load_row_t<K, HT>(e_src + (size_t)r * K, e);
    load_own_row<K>(rr + (size_t)r * K, res);   // the residual row: read by this lane only
    const uint32_t tag = info & 0xFFu;
    const bool lab = tag != kTagUnlabelled;
    const float inv_g = inv_g_of<UN>(cf, lab, a);
    const float diag = cf.c + (lab ? cf.eta : 0.0f);
    float en[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float te = cf.eps * lap_row<UN>(a, e[k], acc[k]) + diag * e[k];
        en[k] = e[k] + (res[k] - te) * inv_g;
    }
    if constexpr (LAST) {
        float x[K];
        load_own_row<K>(u + (size_t)r * K, x);
#pragma unroll
        for (int k = 0; k < K; ++k) x[k] += en[k];
        if constexpr (PROJECT) project_simplex<K>(x);
        store_row<K>(u_out + (size_t)r * K, x);
    } else {
        store_row_t<K, HT>(e_dst + (size_t)r * K, en);
    }
}

}  // namespace dev
}  // namespace pdca
