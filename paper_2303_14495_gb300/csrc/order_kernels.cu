// Locality renumbering on the device (structure only, no arithmetic of the
// method): the BFS-block order of reorder.cpp, computed by CUDA kernels.
//
// The node range is cut into chunks of kBfsChunk nodes; one block of
// kBfsThreads threads renumbers a chunk.  Inside a chunk, searches start at
// the lowest node not yet placed; a search visits nodes breadth-first
// (edges leaving the chunk are ignored) and places them in visiting order
// until the current block of `block` nodes is full; the nodes a search has
// queued but not placed when the block fills become free again, and a
// search that runs dry before the block is full is followed by a new one
// that continues the same block.  The visiting order is the order of a FIFO
// queue: the nodes of a level in the order of their first discovery, by the
// earliest node of the previous level, through its earliest edge.
//
// Two ways of expanding a level give that order:
//   * warp mode (small frontiers): warp 0 takes the frontier nodes one at a
//     time, its lanes over the node's edges (a column repeated inside a row
//     counts at its first lane); a ballot and a prefix count append the free
//     neighbours in edge order;
//   * block mode (frontiers of kBfsWide nodes or more): kBfsLanes lanes per
//     frontier node, up to kBfsSeg nodes per round.  Every free neighbour
//     gets the smallest key (frontier position << 32 | edge index) among its
//     discoverers (atomicMin); each frontier node counts the neighbours whose
//     key is its own, a block scan of the counts gives every node its place,
//     and the nodes are appended in edge order.  Rounds go in frontier order,
//     so a neighbour claimed in an earlier round is no longer free.
// A level stops early once the queue holds the nodes the block still needs:
// the nodes in front of them are final by then.
//
// Then, inside windows of sigma positions, nodes are sorted by degree
// (descending, ties in place order), as the host implementation does.
#include "pdca_internal.cuh"

namespace pdca {
namespace {

constexpr int kBfsThreads = 1024;
constexpr int kBfsLanes = 8;                          // lanes per frontier node (block mode)
constexpr int kBfsSeg = kBfsThreads / kBfsLanes;      // frontier nodes per round
constexpr int kBfsWide = 8;                           // frontier size that takes block mode
constexpr unsigned kAll = 0xffffffffu;

// Search state of a chunk, in shared memory.  qlen == 0: no search open.
struct BfsCtl {
    int32_t pos;    // nodes placed in the chunk
    int32_t cnt;    // nodes placed in the current block
    int32_t seed;   // every node below it is placed
    int32_t qlen;   // queue length of the open search
    int32_t lb, le; // frontier = queue[lb, le)
    int32_t need;   // nodes the open search may still place
    int32_t done;
    int32_t total;  // nodes appended by a round (block mode)
};

// Place the first min(need, qlen) queued nodes, free the rest (lanes of the
// calling group: `stride` threads starting at `t`).
__device__ __forceinline__ void bfs_finish(const BfsCtl &c, int t, int stride, uint8_t *state,
                                           const int32_t *queue, int32_t *order, int64_t c0) {
    const int32_t take = min(c.need, c.qlen);
    for (int32_t i = t; i < c.qlen; i += stride) {
        const int32_t v = queue[i];
        state[v] = i < take ? 2 : 0;
        if (i < take) order[c0 + c.pos + i] = (int32_t)(c0 + v);
    }
}

// Warp 0: searches and levels while frontiers stay small.  Returns with
// c.done set, or with an open search whose next level has kBfsWide or more
// nodes.
__device__ void bfs_warp(BfsCtl &c, int32_t m, int32_t block, int64_t c0, const int64_t *__restrict__ rp,
                         const int32_t *__restrict__ col, uint8_t *state, int32_t *queue, int32_t *order,
                         uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    BfsCtl s = c;   // kept alike in all lanes
    while (true) {
        if (s.qlen == 0) {   // open a search
            if (s.pos >= m) {
                s.done = 1;
                break;
            }
            if (s.cnt == block) s.cnt = 0;
            int32_t at = s.seed;
            while (at < m) {   // the lowest node not placed (one exists: pos < m)
                const int32_t i = at + lane;
                const unsigned b = __ballot_sync(kAll, i < m && state[i] != 2);
                if (b) {
                    at += __ffs(b) - 1;
                    break;
                }
                at += 32;
            }
            if (at >= m) {   // never expected: the counts say a node is left
                if (lane == 0) atomicOr(err, 1u);
                s.done = 1;
                break;
            }
            s.seed = at;
            if (lane == 0) {
                queue[0] = at;
                state[at] = 1;
            }
            __syncwarp();
            s.qlen = 1;
            s.lb = 0;
            s.le = 1;
            s.need = min(block - s.cnt, m - s.pos);
        }
        if (s.qlen >= s.need || s.lb == s.le) {   // the search is over
            bfs_finish(s, lane, 32, state, queue, order, c0);
            __syncwarp();
            const int32_t take = min(s.need, s.qlen);
            s.pos += take;
            s.cnt += take;
            s.qlen = 0;
            continue;
        }
        if (s.le - s.lb >= kBfsWide) break;   // a wide level: the whole block expands it
        for (int32_t f = s.lb; f < s.le && s.qlen < s.need && !s.done; ++f) {
            const int32_t v = queue[f];
            const int64_t e0 = rp[c0 + v], e1 = rp[c0 + v + 1];
            for (int64_t eb = e0; eb < e1; eb += 32) {
                const int64_t e = eb + lane;
                uint32_t lj = 0;
                bool fresh = false;
                if (e < e1) {
                    lj = (uint32_t)((int64_t)col[e] - c0);
                    fresh = lj < (uint32_t)m && state[lj] == 0;
                }
                // a column repeated inside one row counts once (its first lane)
                const unsigned same = __match_any_sync(kAll, fresh ? lj : 0xFFFFFFFFu);
                fresh = fresh && (__ffs(same) - 1) == lane;
                const unsigned b = __ballot_sync(kAll, fresh);
                if (s.qlen + __popc(b) > m) {   // never expected: a node is queued once
                    if (lane == 0) atomicOr(err, 1u);
                    s.done = 1;
                    break;
                }
                if (fresh) {
                    queue[s.qlen + __popc(b & lt)] = (int32_t)lj;
                    state[lj] = 1;
                }
                s.qlen += __popc(b);
                __syncwarp();
            }
        }
        if (s.done) break;
        s.lb = s.le;
        s.le = s.qlen;
    }
    if (lane == 0) c = s;
}

// The whole block: one wide level [lb, le) (early stop once qlen >= need).
__device__ void bfs_block_level(BfsCtl &c, int32_t m, int64_t c0, const int64_t *__restrict__ rp,
                                const int32_t *__restrict__ col, uint8_t *state, int32_t *queue,
                                unsigned long long *key, int32_t *s_cnt, uint32_t *err) {
    const int g = threadIdx.x / kBfsLanes, sub = threadIdx.x % kBfsLanes;
    const int lane = threadIdx.x & 31;
    const unsigned gshift = (unsigned)(lane & ~(kBfsLanes - 1));
    const int32_t lb = c.lb, le = c.le;
    for (int32_t s0 = lb; s0 < le; s0 += kBfsSeg) {
        const int32_t f = s0 + g;
        const bool act = f < le;
        int64_t e0 = 0, e1 = 0;
        if (act) {
            const int32_t v = queue[f];
            e0 = rp[c0 + v];
            e1 = rp[c0 + v + 1];
        }
        const int32_t rounds = __reduce_max_sync(kAll, act ? (int32_t)((e1 - e0 + kBfsLanes - 1) / kBfsLanes) : 0);
        // claims
        for (int32_t k = 0; k < rounds; ++k) {
            const int64_t e = e0 + (int64_t)k * kBfsLanes + sub;
            if (e < e1) {
                const uint32_t lj = (uint32_t)((int64_t)col[e] - c0);
                if (lj < (uint32_t)m && state[lj] == 0)
                    atomicMin(key + lj, ((unsigned long long)(uint32_t)f << 32) | (uint32_t)(e - e0));
            }
        }
        __syncthreads();
        // neighbours whose key is this node's, per node
        int32_t won = 0;
        for (int32_t k = 0; k < rounds; ++k) {
            const int64_t e = e0 + (int64_t)k * kBfsLanes + sub;
            if (e < e1) {
                const uint32_t lj = (uint32_t)((int64_t)col[e] - c0);
                if (lj < (uint32_t)m && state[lj] == 0 &&
                    __ldcg(key + lj) == (((unsigned long long)(uint32_t)f << 32) | (uint32_t)(e - e0)))
                    ++won;
            }
        }
        for (int o = kBfsLanes / 2; o > 0; o >>= 1) won += __shfl_xor_sync(kAll, won, o);
        if (sub == 0) s_cnt[g] = won;
        __syncthreads();
        if (threadIdx.x < 32) {   // exclusive scan of the kBfsSeg counts, 4 per lane
            int32_t v[kBfsSeg / 32], sum = 0;
#pragma unroll
            for (int q = 0; q < kBfsSeg / 32; ++q) {
                v[q] = s_cnt[lane * (kBfsSeg / 32) + q];
                sum += v[q];
            }
            int32_t incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(kAll, incl, o);
                if (lane >= o) incl += t;
            }
            int32_t run = incl - sum;
#pragma unroll
            for (int q = 0; q < kBfsSeg / 32; ++q) {
                s_cnt[lane * (kBfsSeg / 32) + q] = run;
                run += v[q];
            }
            if (lane == 31) c.total = incl;
        }
        __syncthreads();
        if (c.qlen + c.total > m) {   // never expected: a node is queued once
            if (threadIdx.x == 0) {
                atomicOr(err, 1u);
                c.done = 1;
            }
            __syncthreads();
            return;
        }
        // append in edge order
        int32_t at = c.qlen + s_cnt[g];
        for (int32_t k = 0; k < rounds; ++k) {
            const int64_t e = e0 + (int64_t)k * kBfsLanes + sub;
            bool win = false;
            uint32_t lj = 0;
            if (e < e1) {
                lj = (uint32_t)((int64_t)col[e] - c0);
                win = lj < (uint32_t)m && state[lj] == 0 &&
                      __ldcg(key + lj) == (((unsigned long long)(uint32_t)f << 32) | (uint32_t)(e - e0));
            }
            const unsigned bits = (__ballot_sync(kAll, win) >> gshift) & ((1u << kBfsLanes) - 1u);
            if (win) queue[at + __popc(bits & ((1u << sub) - 1u))] = (int32_t)lj;
            at += __popc(bits);
        }
        __syncthreads();
        // the new nodes are queued; their keys are free again
        const int32_t q0 = c.qlen, q1 = c.qlen + c.total;
        for (int32_t i = q0 + (int32_t)threadIdx.x; i < q1; i += kBfsThreads) {
            const int32_t v = queue[i];
            state[v] = 1;
            key[v] = ~0ull;
        }
        __syncthreads();
        if (threadIdx.x == 0) c.qlen = q1;
        __syncthreads();
        if (c.qlen >= c.need) break;
    }
    if (threadIdx.x == 0) {
        c.lb = le;
        c.le = c.qlen;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBfsThreads, 1)
bfs_blocks_kernel(int32_t n, int32_t chunk, int32_t block, const int64_t *__restrict__ rp,
                  const int32_t *__restrict__ col, int32_t *__restrict__ queue_all,
                  unsigned long long *__restrict__ key_all, int32_t *__restrict__ order, uint32_t *err) {
    extern __shared__ uint8_t state[];   // chunk bytes: 0 free, 1 queued, 2 placed
    __shared__ BfsCtl c;
    __shared__ int32_t s_cnt[kBfsSeg];
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int32_t m = (int32_t)min((int64_t)chunk, (int64_t)n - c0);
    int32_t *queue = queue_all + c0;
    unsigned long long *key = key_all + c0;
    for (int32_t i = threadIdx.x; i < m; i += kBfsThreads) state[i] = 0;
    if (threadIdx.x == 0) c = BfsCtl{0, 0, 0, 0, 0, 0, 0, 0, 0};
    __syncthreads();
    while (true) {
        if (threadIdx.x < 32) bfs_warp(c, m, block, c0, rp, col, state, queue, order, err);
        __syncthreads();
        if (c.done) break;
        bfs_block_level(c, m, c0, rp, col, state, queue, key, s_cnt, err);
        if (c.done) break;
        if (c.qlen >= c.need || c.lb == c.le) {   // the search is over: place its nodes together
            bfs_finish(c, threadIdx.x, kBfsThreads, state, queue, order, c0);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int32_t take = min(c.need, c.qlen);
                c.pos += take;
                c.cnt += take;
                c.qlen = 0;
            }
            __syncthreads();
        }
    }
}

// Degree sort inside windows of sigma positions of `order` (bitonic, keys
// (2^32-1 - degree) << 32 | position): descending degree, ties in order.
__global__ void order_sort_kernel(int32_t n, int32_t sigma, const int64_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ order, int32_t *__restrict__ out) {
    extern __shared__ unsigned long long keys[];
    const int64_t base = (int64_t)blockIdx.x * sigma;
    for (int p = threadIdx.x; p < sigma; p += blockDim.x) {
        const int64_t i = base + p;
        unsigned long long k = ~0ull;
        if (i < n) {
            const int32_t v = order[i];
            const uint32_t dgr = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
            k = ((unsigned long long)(0xFFFFFFFFu - dgr) << 32) | (uint32_t)p;
        }
        keys[p] = k;
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
        if (r < n) out[r] = order[base + (int64_t)(keys[p] & 0xFFFFFFFFull)];
    }
}

}  // namespace

cudaError_t launch_bfs_blocks(int32_t n, int32_t block, int32_t chunk, const int64_t *row_ptr, const int32_t *col,
                              int32_t *queue, unsigned long long *key, int32_t *order, uint32_t *err,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (chunk <= 0 || chunk > 65536 || block <= 0 || chunk % block != 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)chunk;
    cudaError_t e = cudaFuncSetAttribute(bfs_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(key, 0xFF, sizeof(unsigned long long) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    const int chunks = (int)(((int64_t)n + chunk - 1) / chunk);
    count_launches(1);
    bfs_blocks_kernel<<<chunks, kBfsThreads, smem, st>>>(n, chunk, block, row_ptr, col, queue, key, order, err);
    return cudaGetLastError();
}

cudaError_t launch_order_sort(int32_t n, int32_t sigma, const int64_t *row_ptr, const int32_t *order, int32_t *out,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (sigma <= 0 || sigma > 1024 || (sigma & (sigma - 1)) != 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(order_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sigma * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    const int windows = (int)(((int64_t)n + sigma - 1) / sigma);
    const int threads = sigma / 2 < 1024 ? (sigma / 2 > 32 ? sigma / 2 : 32) : 1024;
    count_launches(1);
    order_sort_kernel<<<windows, threads, sigma * sizeof(unsigned long long), st>>>(n, sigma, row_ptr, order, out);
    return cudaGetLastError();
}

}  // namespace pdca
