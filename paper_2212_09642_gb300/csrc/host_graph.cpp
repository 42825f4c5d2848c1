// Host-side graph utilities of libvne: greedy distance-d colouring
// (Algorithm 1 of Section 3.1), the degree-descending and reverse
// Cuthill-McKee relabellings, and the O(n) passes of the matrix assembly
// (threads over row ranges).
#include <stdint.h>

#include <algorithm>
#include <vector>
#include <thread>
#include <climits>

#include "host_graph.h"

namespace vne {

namespace {
// Threads for an O(n) host pass: one per 2^17 rows, at most 8.
int pass_threads(int64_t n) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t by_n = n >> 17;
    int t = (int)std::min<int64_t>(std::min<int64_t>(8, hw ? (int64_t)hw : 1), std::max<int64_t>(1, by_n));
    return std::max(1, t);
}
// Runs f(t, lo, hi) on T contiguous ranges of [0, n).
template <typename F>
void run_ranges(int64_t n, int T, F f) {
    if (T <= 1) {
        f(0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; t++) th.emplace_back(f, t, n * t / T, n * (t + 1) / T);
    for (auto& x : th) x.join();
}
}  // namespace

int64_t check_row_offsets(int64_t n, const int64_t* rph, int32_t* rp32, int64_t* maxdeg_out) {
    const int T = pass_threads(n);
    std::vector<int64_t> mx(T, 0), bad(T, -1);
    rp32[0] = (int32_t)rph[0];
    run_ranges(n, T, [&](int t, int64_t lo, int64_t hi) {
        int64_t m = 0;
        for (int64_t i = lo; i < hi; i++) {
            const int64_t d = rph[i + 1] - rph[i];
            if (d < 0 || rph[i + 1] >= (int64_t)INT32_MAX) {
                bad[t] = i;
                return;
            }
            m = std::max(m, d);
            rp32[i + 1] = (int32_t)rph[i + 1];
        }
        mx[t] = m;
    });
    int64_t m = 0;
    for (int t = 0; t < T; t++) {
        if (bad[t] >= 0) return bad[t];  // ranges are in row order: the first bad row
        m = std::max(m, mx[t]);
    }
    *maxdeg_out = m;
    return -1;
}

void degree_relabel(int64_t n, const int32_t* rp32, int64_t maxdeg, int32_t* order, int64_t* rp2, int32_t* rp2_32) {
    const int64_t C = maxdeg + 1;  // class c = maxdeg - degree
    int T = pass_threads(n);
    if (C * T > 4 * n) T = 1;  // per-thread class counts would outweigh the pass
    // class counts per thread range, then the offset of each (class, thread):
    // classes in order, threads in row order within a class (stable in the id)
    std::vector<int64_t> cnt((size_t)T * C, 0);
    run_ranges(n, T, [&](int t, int64_t lo, int64_t hi) {
        int64_t* c = cnt.data() + (size_t)t * C;
        for (int64_t i = lo; i < hi; i++) c[maxdeg - (rp32[i + 1] - rp32[i])]++;
    });
    std::vector<int64_t> cls_start(C + 1, 0), cls_base(C + 1, 0);  // first position, first packed offset
    {
        int64_t pos = 0, off = 0;
        for (int64_t c = 0; c < C; c++) {
            cls_start[c] = pos;
            cls_base[c] = off;
            int64_t k = 0;
            for (int t = 0; t < T; t++) {
                const int64_t v = cnt[(size_t)t * C + c];
                cnt[(size_t)t * C + c] = pos + k;  // becomes the thread's cursor in class c
                k += v;
            }
            pos += k;
            off += k * (maxdeg - c);
        }
        cls_start[C] = pos;
        cls_base[C] = off;
    }
    run_ranges(n, T, [&](int t, int64_t lo, int64_t hi) {
        int64_t* cur = cnt.data() + (size_t)t * C;
        for (int64_t i = lo; i < hi; i++) order[cur[maxdeg - (rp32[i + 1] - rp32[i])]++] = (int32_t)i;
    });
    // packed offsets: position p of class c starts at cls_base[c] + (p - cls_start[c]) * degree
    rp2[0] = 0;
    rp2_32[0] = 0;
    run_ranges(n, T, [&](int, int64_t lo, int64_t hi) {
        int64_t c = std::upper_bound(cls_start.begin(), cls_start.end(), lo) - cls_start.begin() - 1;
        for (int64_t p = lo; p < hi; p++) {
            while (p >= cls_start[c + 1]) c++;
            const int64_t v = cls_base[c] + (p + 1 - cls_start[c]) * (maxdeg - c);
            rp2[p + 1] = v;
            rp2_32[p + 1] = (int32_t)v;
        }
    });
}

// Order of Algorithm 1: nodes by descending degree, ties by ascending id.
std::vector<int32_t> degree_order(int64_t n, const int64_t* rowptr) {
    std::vector<int32_t> order(n);
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; i++) maxdeg = std::max(maxdeg, rowptr[i + 1] - rowptr[i]);
    // counting sort on degree (descending), stable in the node id
    std::vector<int64_t> cnt(maxdeg + 2, 0);
    for (int64_t i = 0; i < n; i++) cnt[maxdeg - (rowptr[i + 1] - rowptr[i]) + 1]++;
    for (int64_t d = 0; d <= maxdeg; d++) cnt[d + 1] += cnt[d];
    for (int64_t i = 0; i < n; i++) order[cnt[maxdeg - (rowptr[i + 1] - rowptr[i])]++] = (int32_t)i;
    return order;
}

std::vector<int32_t> rcm_order(int64_t n, const int64_t* rowptr, const int32_t* col) {
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> seen(n, 0);
    // component seeds in ascending degree, ties by id
    std::vector<int32_t> by_degree = degree_order(n, rowptr);  // descending degree
    std::vector<int32_t> nbr;
    for (int64_t s = n - 1; s >= 0; s--) {
        const int32_t seed = by_degree[s];
        if (seen[seed]) continue;
        seen[seed] = 1;
        size_t head = order.size();
        order.push_back(seed);
        while (head < order.size()) {
            const int32_t u = order[head++];
            nbr.clear();
            for (int64_t k = rowptr[u]; k < rowptr[u + 1]; k++) {
                const int32_t w = col[k];
                if (!seen[w]) {
                    seen[w] = 1;
                    nbr.push_back(w);
                }
            }
            std::sort(nbr.begin(), nbr.end(), [&](int32_t a, int32_t b) {
                const int64_t da = rowptr[a + 1] - rowptr[a], db = rowptr[b + 1] - rowptr[b];
                return da != db ? da < db : a < b;
            });
            order.insert(order.end(), nbr.begin(), nbr.end());
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Greedy distance-d colouring: each node in `order` takes the smallest colour
// not used by an already coloured node within geodesic distance d (found by
// a depth-limited breadth-first search).
int32_t greedy_coloring(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t d, int32_t* colors) {
    std::vector<int32_t> order = degree_order(n, rowptr);
    for (int64_t i = 0; i < n; i++) colors[i] = -1;
    std::vector<int64_t> seen(n, -1);      // BFS stamp per node
    std::vector<int32_t> depth(n, 0);
    std::vector<int64_t> used;             // stamp per colour
    std::vector<int32_t> queue;
    queue.reserve(1024);
    int32_t ncol = 0;
    for (int64_t t = 0; t < n; t++) {
        const int32_t src = order[t];
        queue.clear();
        queue.push_back(src);
        seen[src] = t;
        depth[src] = 0;
        for (size_t h = 0; h < queue.size(); h++) {
            int32_t u = queue[h];
            if (depth[u] == d) continue;
            for (int64_t k = rowptr[u]; k < rowptr[u + 1]; k++) {
                int32_t w = col[k];
                if (seen[w] == t) continue;
                seen[w] = t;
                depth[w] = depth[u] + 1;
                queue.push_back(w);
                if (colors[w] >= 0) {
                    if ((size_t)colors[w] >= used.size()) used.resize(colors[w] + 1, -1);
                    used[colors[w]] = t;
                }
            }
        }
        int32_t c = 0;
        while ((size_t)c < used.size() && used[c] == t) c++;
        colors[src] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    return ncol;
}

}  // namespace vne
