// Host-side graph utilities of libvne.
#pragma once
#include <stdint.h>

#include <vector>

namespace vne {
std::vector<int32_t> degree_order(int64_t n, const int64_t* rowptr);
// Reverse Cuthill-McKee order (new -> old): breadth-first search from a
// minimum-degree node of each connected component, neighbours in ascending
// degree (ties by id), the whole sequence reversed.
std::vector<int32_t> rcm_order(int64_t n, const int64_t* rowptr, const int32_t* col);
int32_t greedy_coloring(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t d, int32_t* colors);
}  // namespace vne
