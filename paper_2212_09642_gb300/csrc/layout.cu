// Layout conversions of probe blocks: the engine's panel-major layout
// ([K / ks][n][ks], rows in the packed, possibly relabelled order) to and
// from row-major [n][k] blocks in the caller's node numbering, and the
// selection of a subset of a block's columns.  One thread per element; the
// row-major side is read or written contiguously along a row.
#include "common.cuh"
#include "kernels.h"

namespace vne {

// out[id][c] = in column col0 + c of packed row r, id the caller's number of r
template <typename T>
__global__ void k_panel_to_rows(const T* __restrict__ in, int n, int ks, int col0, int k,
                                const int32_t* __restrict__ node_id, T* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * k) return;
    const int r = (int)(idx / k), c = (int)(idx % k);
    const int gc = col0 + c;
    const int id = node_id ? node_id[r] : r;
    out[(size_t)id * k + c] = in[(size_t)(gc / ks) * n * ks + (size_t)r * ks + (gc % ks)];
}

// panel-major out with Kp columns: column c < k of packed row r from in[id][c],
// columns k..Kp-1 zero
template <typename T>
__global__ void k_rows_to_panel(const T* __restrict__ in, int n, int ks, int k, int Kp,
                                const int32_t* __restrict__ node_id, T* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * Kp) return;
    const int r = (int)(idx / Kp), c = (int)(idx % Kp);
    const int id = node_id ? node_id[r] : r;
    out[(size_t)(c / ks) * n * ks + (size_t)r * ks + (c % ks)] = c < k ? in[(size_t)id * k + c] : (T)0;
}

// panel-major out with Kp columns: column c < k is column src_cols[c] of the
// panel-major in (same n and ks), columns k..Kp-1 zero
template <typename T>
__global__ void k_select_columns(const T* __restrict__ in, int n, int ks, const int32_t* __restrict__ src_cols,
                                 int k, int Kp, T* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * Kp) return;
    const int r = (int)(idx / Kp), c = (int)(idx % Kp);
    T v = (T)0;
    if (c < k) {
        const int s = src_cols[c];
        v = in[(size_t)(s / ks) * n * ks + (size_t)r * ks + (s % ks)];
    }
    out[(size_t)(c / ks) * n * ks + (size_t)r * ks + (c % ks)] = v;
}

static unsigned blocks_for(int64_t total) { return (unsigned)((total + 255) / 256); }

template <typename T>
cudaError_t launch_panel_to_rows(const T* in, int n, int ks, int col0, int k, const int32_t* node_id, T* out,
                                 cudaStream_t st) {
    const int64_t total = (int64_t)n * k;
    if (total == 0) return cudaSuccess;
    k_panel_to_rows<T><<<blocks_for(total), 256, 0, st>>>(in, n, ks, col0, k, node_id, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_to_panel(const T* in, int n, int ks, int k, int Kp, const int32_t* node_id, T* out,
                                 cudaStream_t st) {
    const int64_t total = (int64_t)n * Kp;
    if (total == 0) return cudaSuccess;
    k_rows_to_panel<T><<<blocks_for(total), 256, 0, st>>>(in, n, ks, k, Kp, node_id, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_select_columns(const T* in, int n, int ks, const int32_t* src_cols, int k, int Kp, T* out,
                                  cudaStream_t st) {
    const int64_t total = (int64_t)n * Kp;
    if (total == 0) return cudaSuccess;
    k_select_columns<T><<<blocks_for(total), 256, 0, st>>>(in, n, ks, src_cols, k, Kp, out);
    return cudaGetLastError();
}

#define VNE_LAYOUT_INST(T)                                                                                     \
    template cudaError_t launch_panel_to_rows<T>(const T*, int, int, int, int, const int32_t*, T*, cudaStream_t); \
    template cudaError_t launch_rows_to_panel<T>(const T*, int, int, int, int, const int32_t*, T*, cudaStream_t); \
    template cudaError_t launch_select_columns<T>(const T*, int, int, const int32_t*, int, int, T*, cudaStream_t);
VNE_LAYOUT_INST(float)
VNE_LAYOUT_INST(double)

}  // namespace vne
