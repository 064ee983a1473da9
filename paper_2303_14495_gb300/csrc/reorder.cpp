// Host-side symbolic analysis of the graph at create time (structure only, no
// arithmetic of the method):
//   * locality renumbering: nodes are grouped into blocks of `block` nodes by
//     breadth-first search over the graph, so that a block is a compact
//     region (for image graphs: a blob of pixels rather than a strip of a
//     scan line);
//   * inside every block, rows are sorted by degree (descending) so the 32
//     rows of a slice have similar lengths;
//   * per tile of `tile_rows` renumbered rows, the sorted list of distinct
//     neighbour rows (the tile's halo), which the tiled kernels stage in
//     shared memory.
// The node range is cut into fixed chunks that are processed independently
// (in parallel), so the result does not depend on the number of threads.
#include "pdca_internal.cuh"

#include <algorithm>
#include <functional>
#include <thread>
#include <vector>

namespace pdca {

namespace {

int worker_count() {
    unsigned hc = std::thread::hardware_concurrency();
    if (hc == 0) hc = 4;
    return (int)std::min<unsigned>(hc, 64);
}

template <class F>
void parallel_for(int64_t count, F &&f) {
    const int nt = (int)std::min<int64_t>(worker_count(), std::max<int64_t>(count, 1));
    if (nt <= 1) {
        for (int64_t i = 0; i < count; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int64_t i = t; i < count; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

// BFS blocks inside [c0, c1): repeatedly take the first unvisited node as a
// seed and visit nodes breadth-first (edges leaving the chunk are ignored),
// appending them to the current block; a block closes after `block` nodes,
// and a new seed continues the same block if a search runs dry first.
// Node state: 0 fresh, 1 queued by the current search, 2 visited.  When a
// block closes, the nodes still queued (the tail of the queue) become fresh
// again for the next search.
void chunk_blocks(int64_t c0, int64_t c1, const int64_t *rp, const int32_t *col, int32_t block,
                  int32_t *order) {
    const int64_t m = c1 - c0;
    std::vector<uint8_t> state((size_t)m, 0);
    std::vector<int32_t> queue;
    queue.reserve((size_t)block * 4);
    int64_t pos = c0, seed = c0;
    while (pos < c1) {
        int64_t cnt = 0;
        while (cnt < block && pos < c1) {
            while (state[(size_t)(seed - c0)] == 2) ++seed;
            queue.clear();
            queue.push_back((int32_t)seed);
            state[(size_t)(seed - c0)] = 1;
            size_t qh = 0;
            while (qh < queue.size() && cnt < block) {
                // the rows of queued nodes are scattered in memory: start
                // fetching the edge list of a node a few places ahead
                if (qh + 8 < queue.size()) {
                    const int32_t a = queue[qh + 8];
                    __builtin_prefetch(col + rp[a]);
                }
                const int32_t v = queue[qh++];
                state[(size_t)(v - c0)] = 2;
                order[pos++] = v;
                ++cnt;
                const int64_t e1 = rp[v + 1];
                for (int64_t e = rp[v]; e < e1; ++e) {
                    const uint64_t lj = (uint64_t)((int64_t)col[e] - c0);
                    if (lj >= (uint64_t)m) continue;
                    if (state[lj] == 0) {
                        state[lj] = 1;
                        queue.push_back((int32_t)(lj + c0));
                        __builtin_prefetch(rp + lj + c0);
                    }
                }
            }
            for (size_t q = qh; q < queue.size(); ++q) state[(size_t)(queue[q] - c0)] = 0;
        }
    }
}

}  // namespace

void host_parallel_for(int64_t count, const std::function<void(int64_t)> &f) { parallel_for(count, f); }

int host_workers() { return worker_count(); }

void locality_order(int32_t n, const int64_t *rp, const int32_t *col, int32_t block, int32_t chunk,
                    int32_t sort_window, int32_t *order) {
    const int64_t nchunks = ((int64_t)n + chunk - 1) / chunk;
    parallel_for(nchunks, [&](int64_t c) {
        const int64_t c0 = c * chunk, c1 = std::min<int64_t>(n, c0 + chunk);
        chunk_blocks(c0, c1, rp, col, block, order);
    });
    // degree sort (descending, stable) inside every window of `sort_window`
    // positions (a divisor of `block`): a counting sort on the degrees, which
    // are read once per node; degrees above kMaxBucket share the top bucket
    // and are ordered among themselves by a stable comparison sort.
    constexpr int64_t kMaxBucket = 255;
    const int64_t nwin = ((int64_t)n + sort_window - 1) / sort_window;
    parallel_for(nwin, [&](int64_t wdx) {
        int32_t *b = order + wdx * sort_window;
        const int64_t len = std::min<int64_t>(n, (wdx + 1) * sort_window) - wdx * sort_window;
        std::vector<int64_t> dg((size_t)len);
        std::vector<int32_t> tmp(b, b + len);
        int64_t count[kMaxBucket + 2] = {0};
        for (int64_t i = 0; i < len; ++i) {
            dg[(size_t)i] = rp[tmp[(size_t)i] + 1] - rp[tmp[(size_t)i]];
            ++count[kMaxBucket - std::min(dg[(size_t)i], kMaxBucket) + 1];
        }
        for (int64_t k = 1; k <= kMaxBucket + 1; ++k) count[k] += count[k - 1];
        for (int64_t i = 0; i < len; ++i) b[count[kMaxBucket - std::min(dg[(size_t)i], kMaxBucket)]++] = tmp[(size_t)i];
        const int64_t top = count[0];   // nodes of degree >= kMaxBucket sit first
        if (top > 1)
            std::stable_sort(b, b + top, [&](int32_t x, int32_t y) { return (rp[x + 1] - rp[x]) > (rp[y + 1] - rp[y]); });
    });
}

void tile_halos(int32_t n, int32_t tile_rows, const int64_t *rp, const int32_t *col, const int32_t *perm,
                const int32_t *iperm, std::vector<int64_t> &halo_off, std::vector<int32_t> &halo_idx,
                int32_t *max_halo) {
    const int64_t ntiles = ((int64_t)n + tile_rows - 1) / tile_rows;
    std::vector<std::vector<int32_t>> per((size_t)ntiles);
    parallel_for(ntiles, [&](int64_t t) {
        std::vector<int32_t> &h = per[(size_t)t];
        const int64_t r0 = t * tile_rows, r1 = std::min<int64_t>(n, r0 + tile_rows);
        for (int64_t r = r0; r < r1; ++r) {
            const int32_t old = perm[r];
            for (int64_t e = rp[old]; e < rp[old + 1]; ++e) h.push_back(iperm[col[e]]);
        }
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
    });
    halo_off.assign((size_t)ntiles + 1, 0);
    int32_t mx = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        halo_off[(size_t)t + 1] = halo_off[(size_t)t] + (int64_t)per[(size_t)t].size();
        mx = std::max<int32_t>(mx, (int32_t)per[(size_t)t].size());
    }
    halo_idx.resize((size_t)halo_off.back());
    parallel_for(ntiles, [&](int64_t t) {
        std::copy(per[(size_t)t].begin(), per[(size_t)t].end(), halo_idx.begin() + halo_off[(size_t)t]);
    });
    *max_halo = mx;
}

}  // namespace pdca
