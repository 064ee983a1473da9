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
void chunk_blocks(int64_t c0, int64_t c1, const int64_t *rp, const int32_t *col, int32_t block,
                  int32_t *order) {
    const int64_t m = c1 - c0;
    std::vector<uint8_t> vis((size_t)m, 0), inq((size_t)m, 0);
    std::vector<int32_t> queue, touched;
    queue.reserve((size_t)block * 4);
    touched.reserve((size_t)block * 4);
    int64_t pos = c0, seed = c0;
    while (pos < c1) {
        int64_t cnt = 0;
        while (cnt < block && pos < c1) {
            while (vis[(size_t)(seed - c0)]) ++seed;
            queue.clear();
            touched.clear();
            queue.push_back((int32_t)seed);
            inq[(size_t)(seed - c0)] = 1;
            touched.push_back((int32_t)seed);
            size_t qh = 0;
            while (qh < queue.size() && cnt < block) {
                // the rows of queued nodes are scattered in memory: start
                // fetching the edge list of a node a few places ahead
                if (qh + 8 < queue.size()) {
                    const int32_t a = queue[qh + 8];
                    __builtin_prefetch(col + rp[a]);
                }
                const int32_t v = queue[qh++];
                vis[(size_t)(v - c0)] = 1;
                order[pos++] = v;
                ++cnt;
                for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                    const int64_t j = col[e];
                    if (j < c0 || j >= c1) continue;
                    const size_t lj = (size_t)(j - c0);
                    if (!vis[lj] && !inq[lj]) {
                        inq[lj] = 1;
                        queue.push_back((int32_t)j);
                        touched.push_back((int32_t)j);
                        __builtin_prefetch(rp + j);
                    }
                }
            }
            for (int32_t t : touched) inq[(size_t)(t - c0)] = 0;
        }
    }
}

}  // namespace

void host_parallel_for(int64_t count, const std::function<void(int64_t)> &f) { parallel_for(count, f); }

void locality_order(int32_t n, const int64_t *rp, const int32_t *col, int32_t block, int32_t chunk,
                    int32_t sort_window, int32_t *order) {
    const int64_t nchunks = ((int64_t)n + chunk - 1) / chunk;
    parallel_for(nchunks, [&](int64_t c) {
        const int64_t c0 = c * chunk, c1 = std::min<int64_t>(n, c0 + chunk);
        chunk_blocks(c0, c1, rp, col, block, order);
    });
    // degree sort (descending, stable) inside every window of `sort_window`
    // positions (a divisor of `block`)
    const int64_t nwin = ((int64_t)n + sort_window - 1) / sort_window;
    parallel_for(nwin, [&](int64_t wdx) {
        int32_t *b = order + wdx * sort_window;
        int32_t *e = order + std::min<int64_t>(n, (wdx + 1) * sort_window);
        std::stable_sort(b, e, [&](int32_t x, int32_t y) { return (rp[x + 1] - rp[x]) > (rp[y + 1] - rp[y]); });
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
