// Host-side graph utilities of libvne: greedy distance-d colouring
// (Algorithm 1 of Section 3.1) and the degree-descending and reverse
// Cuthill-McKee relabellings.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "host_graph.h"

namespace vne {

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
