// Device-side assembly of the stored operator from the caller's CSR pattern
// (Section 2: rho = L / tr L with L = D - W of the graph).  Validation of the
// column indices and the degree-order relabelling run here, one warp per
// row, so that building a matrix costs one pass over the nonzeros in HBM
// instead of a host pass.  The relabelling is a symmetric permutation
// rho -> P rho P^T, which leaves the spectrum (and S(rho)) unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace vne {

namespace {

constexpr int kWarps = 8;

// Offending nonzeros: bad[0] = smallest index k with a column outside
// [0, n), bad[1] = smallest k with col[k] == row (pattern matrices only).
__global__ void __launch_bounds__(kWarps * 32) k_validate(const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, int64_t n, int pattern,
                                                          unsigned long long* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t r = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); r < n; r += warps) {
        const int32_t b = rowptr[r], e = rowptr[r + 1];
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t c = __ldcs(col + k);
            if (c < 0 || (int64_t)c >= n) atomicMin(bad, (unsigned long long)k);
            else if (pattern && (int64_t)c == r) atomicMin(bad + 1, (unsigned long long)k);
        }
    }
}

// New row i is old row order[i]; its columns are renamed by inv (old -> new)
// and keep the order of the old row.
template <typename V>
__global__ void __launch_bounds__(kWarps * 32) k_relabel(const int32_t* __restrict__ rp_old,
                                                         const int32_t* __restrict__ col_old,
                                                         const double* __restrict__ val_old,
                                                         const int32_t* __restrict__ rp_new,
                                                         const int32_t* __restrict__ order,
                                                         const int32_t* __restrict__ inv, int64_t n,
                                                         int32_t* __restrict__ col_new, V* __restrict__ val_new) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); i < n; i += warps) {
        const int32_t o = order[i];
        const int32_t b = rp_old[o], len = rp_old[o + 1] - b, d = rp_new[i];
        for (int32_t q = lane; q < len; q += 32) {
            col_new[d + q] = inv[__ldcs(col_old + b + q)];
            if (val_old) val_new[d + q] = (V)__ldcs(val_old + b + q);
        }
    }
}

// inv[order[i]] = i
__global__ void k_invert_perm(const int32_t* __restrict__ order, int64_t n, int32_t* __restrict__ inv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        inv[order[i]] = (int32_t)i;
}

template <typename V>
__global__ void k_convert(const double* __restrict__ in, int64_t count, V* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (V)in[k];
}

int grid_for(int64_t rows) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    int64_t want = (rows + kWarps - 1) / kWarps;
    int64_t cap = (int64_t)sms * 16;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int64_t n, int pattern,
                            unsigned long long* bad, cudaStream_t st) {
    // all bytes 0xff: no offending index yet
    cudaError_t e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_validate<<<grid_for(n), kWarps * 32, 0, st>>>(rowptr, col, n, pattern, bad);
    return cudaGetLastError();
}

cudaError_t launch_relabel(const int32_t* rp_old, const int32_t* col_old, const double* val_old,
                           const int32_t* rp_new, const int32_t* order, const int32_t* inv, int64_t n,
                           int32_t* col_new, void* val_new, int fp64, cudaStream_t st) {
    if (fp64)
        k_relabel<double><<<grid_for(n), kWarps * 32, 0, st>>>(rp_old, col_old, val_old, rp_new, order, inv, n,
                                                                col_new, (double*)val_new);
    else
        k_relabel<float><<<grid_for(n), kWarps * 32, 0, st>>>(rp_old, col_old, val_old, rp_new, order, inv, n,
                                                               col_new, (float*)val_new);
    return cudaGetLastError();
}

cudaError_t launch_invert_perm(const int32_t* order, int64_t n, int32_t* inv, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_invert_perm<<<grid_for((n + 31) / 32), kWarps * 32, 0, st>>>(order, n, inv);
    return cudaGetLastError();
}

cudaError_t launch_convert_values(const double* in, int64_t count, void* out, int fp64, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int blocks = grid_for((count + 31) / 32);  // 256 threads: 8 x 32 elements per pass
    if (fp64) k_convert<double><<<blocks, 256, 0, st>>>(in, count, (double*)out);
    else k_convert<float><<<blocks, 256, 0, st>>>(in, count, (float*)out);
    return cudaGetLastError();
}

}  // namespace vne
