// Host-side graph utilities of libvne.
#pragma once
#include <stdint.h>

#include <vector>

namespace vne {
std::vector<int32_t> degree_order(int64_t n, const int64_t* rowptr);
// One pass over the caller's row offsets (threads over row ranges): writes
// the int32 copy rp32[0..n] and the largest degree; returns the first row i
// with rowptr[i + 1] < rowptr[i] or rowptr[i + 1] >= 2^31 - 1, else -1.
int64_t check_row_offsets(int64_t n, const int64_t* rowptr, int32_t* rp32, int64_t* maxdeg);
// Degree-descending order stable in the node id (order: new -> old, a
// counting sort over the degree classes with per-thread cursors) and the
// packed row offsets rp2 / rp2_32 [0..n] of the relabelled matrix.
void degree_relabel(int64_t n, const int32_t* rp32, int64_t maxdeg, int32_t* order, int64_t* rp2, int32_t* rp2_32);
// Reverse Cuthill-McKee order (new -> old): breadth-first search from a
// minimum-degree node of each connected component, neighbours in ascending
// degree (ties by id), the whole sequence reversed.
std::vector<int32_t> rcm_order(int64_t n, const int64_t* rowptr, const int32_t* col);
int32_t greedy_coloring(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t d, int32_t* colors);
}  // namespace vne
