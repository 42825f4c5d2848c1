// Host logic of the matrix assembly: the threaded row-offset check and the
// threaded degree relabelling against the serial counting sort (degree
// descending, stable in the node id) and a serial prefix sum of the
// permuted degrees.  Built and run by test_host_relabel.py.
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>
#include <climits>
#include "host_graph.h"
using namespace vne;
int main() {
    std::mt19937_64 g(7);
    int fails = 0;
    for (int trial = 0; trial < 40; trial++) {
        int64_t n = (trial < 10) ? (1 + g() % 50) : (trial < 30 ? (100000 + g() % 900000) : (1 << 20));
        int mode = trial % 3;
        std::vector<int64_t> rp(n + 1, 0);
        for (int64_t i = 0; i < n; i++) {
            int64_t d;
            if (mode == 0) d = g() % 9;                        // small degrees incl. 0
            else if (mode == 1) d = (g() % 16 == 0) ? g() % 3000 : 1 + g() % 6;  // heavy tail
            else d = (i == 0) ? n - 1 : 1;                    // star: maxdeg ~ n (serial fallback)
            rp[i + 1] = rp[i] + d;
        }
        if (rp[n] >= INT32_MAX) continue;
        std::vector<int32_t> rp32(n + 1), order(n), rp2_32(n + 1);
        std::vector<int64_t> rp2(n + 1);
        int64_t maxdeg = -1;
        if (check_row_offsets(n, rp.data(), rp32.data(), &maxdeg) != -1) { printf("unexpected bad row\n"); return 1; }
        int64_t md = 0; for (int64_t i = 0; i < n; i++) md = std::max(md, rp[i+1]-rp[i]);
        if (md != maxdeg) { printf("maxdeg mismatch\n"); fails++; }
        for (int64_t i = 0; i <= n; i++) if (rp32[i] != (int32_t)rp[i]) { printf("rp32 mismatch\n"); fails++; break; }
        degree_relabel(n, rp32.data(), maxdeg, order.data(), rp2.data(), rp2_32.data());
        std::vector<int32_t> ref = degree_order(n, rp.data());
        for (int64_t i = 0; i < n; i++) if (ref[i] != order[i]) { printf("order mismatch trial %d at %lld\n", trial, (long long)i); fails++; break; }
        int64_t acc = 0;
        if (rp2[0] != 0 || rp2_32[0] != 0) fails++;
        for (int64_t i = 0; i < n; i++) { acc += rp[ref[i] + 1] - rp[ref[i]]; if (rp2[i + 1] != acc || rp2_32[i + 1] != (int32_t)acc) { printf("rp2 mismatch trial %d at %lld\n", trial, (long long)i); fails++; break; } }
    }
    // bad rows: non-monotone in the middle of a large array
    {
        int64_t n = 1 << 20; std::vector<int64_t> rp(n + 1); for (int64_t i = 0; i <= n; i++) rp[i] = 2 * i;
        rp[700001] = rp[700000] - 1; for (int64_t i = 700002; i <= n; i++) rp[i] = rp[i-1] + 2;
        rp[900001] = rp[900000] - 5;
        std::vector<int32_t> rp32(n + 1); int64_t md;
        int64_t b = check_row_offsets(n, rp.data(), rp32.data(), &md);
        if (b != 700000) { printf("bad row %lld\n", (long long)b); fails++; }
    }
    printf(fails ? "FAIL %d\n" : "ALL OK\n", fails);
    return fails != 0;
}
