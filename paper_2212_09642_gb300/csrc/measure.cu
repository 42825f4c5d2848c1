// Measurement kernel of libvne: random row gathers from a table of a given
// size, optionally with a concurrent streaming read.  It measures the
// throughput ceiling of the SpMM step kernel's access pattern (neighbour rows
// of one panel, gathered from L2 while the CSR and vector streams pass
// through), which lies above the HBM copy bandwidth for tables that fit in
// L2.  Not part of the method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace vne {

namespace {

__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// LPR lanes (16 bytes each) per row; row r = hash(i) mod rows for gather i.
template <int LPR>
__global__ void __launch_bounds__(256) k_gather_probe(const float4* __restrict__ table, uint32_t rows,
                                                     uint64_t count, uint32_t seed,
                                                     const float4* __restrict__ stream, uint64_t stream_vec,
                                                     float* __restrict__ sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t sub = (uint32_t)(tid % LPR);
    float acc = 0.f;
    for (uint64_t i = tid / LPR; i < count; i += nthreads / LPR) {
        const uint32_t r = probe_hash((uint32_t)i ^ seed) % rows;
        const float4 v = __ldg(table + (size_t)r * LPR + sub);
        acc += (v.x + v.y) + (v.z + v.w);
    }
    for (uint64_t k = tid; k < stream_vec; k += nthreads) acc += __ldcs(stream + k).x;
    // the tables are zero: the sum stays 0 and the store never happens, but
    // the compiler cannot drop the loads
    if (acc != 0.f) sink[0] = acc;
}

}  // namespace

cudaError_t launch_gather_probe(const void* table, uint64_t table_bytes, int row_bytes, uint64_t count, uint32_t seed,
                                const void* stream, uint64_t stream_bytes, float* sink, cudaStream_t st) {
    if (row_bytes != 32 && row_bytes != 64 && row_bytes != 128) return cudaErrorInvalidValue;
    const uint64_t rows = table_bytes / (uint64_t)row_bytes;
    if (rows < 1 || rows > 0xffffffffull) return cudaErrorInvalidValue;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const dim3 grid(sms * 8), block(256);
    const float4* t = static_cast<const float4*>(table);
    const float4* s = static_cast<const float4*>(stream);
    const uint64_t sv = stream_bytes / 16;
    if (row_bytes == 32) k_gather_probe<2><<<grid, block, 0, st>>>(t, (uint32_t)rows, count, seed, s, sv, sink);
    else if (row_bytes == 64) k_gather_probe<4><<<grid, block, 0, st>>>(t, (uint32_t)rows, count, seed, s, sv, sink);
    else k_gather_probe<8><<<grid, block, 0, st>>>(t, (uint32_t)rows, count, seed, s, sv, sink);
    return cudaGetLastError();
}

}  // namespace vne
