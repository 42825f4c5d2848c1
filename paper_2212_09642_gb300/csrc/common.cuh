// Shared device-side definitions of libvne (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define VNE_WARPS 8                 // warps per CTA of the step kernels
#define VNE_THREADS (VNE_WARPS * 32)

namespace vne {

// 16-byte lane vectors: each lane owns CPL consecutive columns of a row.
template <typename T> struct LaneVec;
template <> struct LaneVec<float> { typedef float4 type; static constexpr int CPL = 4; };
template <> struct LaneVec<double> { typedef double2 type; static constexpr int CPL = 2; };

template <typename T>
__device__ __forceinline__ void load_lane(const T* p, T (&v)[LaneVec<T>::CPL]) {
    typedef typename LaneVec<T>::type V;
    V x = *reinterpret_cast<const V*>(p);
    const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int q = 0; q < LaneVec<T>::CPL; q++) v[q] = e[q];
}

// streaming load (read once; do not keep in L1)
template <typename T>
__device__ __forceinline__ void load_lane_stream(const T* p, T (&v)[LaneVec<T>::CPL]) {
    typedef typename LaneVec<T>::type V;
    V x = __ldcs(reinterpret_cast<const V*>(p));
    const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
    for (int q = 0; q < LaneVec<T>::CPL; q++) v[q] = e[q];
}

template <typename T>
__device__ __forceinline__ void store_lane(T* p, const T (&v)[LaneVec<T>::CPL]) {
    typedef typename LaneVec<T>::type V;
    V x;
    T* e = reinterpret_cast<T*>(&x);
#pragma unroll
    for (int q = 0; q < LaneVec<T>::CPL; q++) e[q] = v[q];
    *reinterpret_cast<V*>(p) = x;
}

template <typename T>
__device__ __forceinline__ void store_lane_stream(T* p, const T (&v)[LaneVec<T>::CPL]) {
    typedef typename LaneVec<T>::type V;
    V x;
    T* e = reinterpret_cast<T*>(&x);
#pragma unroll
    for (int q = 0; q < LaneVec<T>::CPL; q++) e[q] = v[q];
    __stcs(reinterpret_cast<V*>(p), x);
}

// Gathered loads with an L2 evict_last cache policy (HINT 1) and, for
// HINT 2, without allocating in L1: the gathered panel is reused by every
// row that has a neighbour in it, the streams around it are read once.
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

template <int HINT>
__device__ __forceinline__ void load_lane_hint(const float* p, float (&v)[4], uint64_t pol) {
    if (HINT == 0) {
        float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if (HINT == 1) {
        asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "l"(p), "l"(pol));
    }
}

template <int HINT>
__device__ __forceinline__ void load_lane_hint(const double* p, double (&v)[2], uint64_t pol) {
    if (HINT == 0) {
        double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = x.x; v[1] = x.y;
    } else if (HINT == 1) {
        asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                     : "=d"(v[0]), "=d"(v[1])
                     : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                     : "=d"(v[0]), "=d"(v[1])
                     : "l"(p), "l"(pol));
    }
}

// L2-coherent load of a value another CTA wrote in this kernel (bypasses L1).
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }

// Work unit of the step kernels: either `rows > 0` consecutive short rows
// starting at `row`, or (rows < 0) chunk number (-rows - 1) of long row
// number `row` of the hub table, covering nonzeros [nnz_begin, nnz_end).
// rows == 0 is padding.
struct WorkItem {
    int32_t row;
    int32_t rows;
    int32_t nnz_begin;
    int32_t nnz_end;
};

// A long row split into `chunks` warp items; chunk partial sums live at
// slots [slot, slot + chunks) of the hub scratch.
struct HubRow {
    int32_t row;
    int32_t chunks;
    int32_t slot;
    int32_t seg;
};

// Row tile of the elementwise kernels: rows [row_begin, row_end) of one segment.
struct RowTile {
    int32_t row_begin;
    int32_t row_end;
    int32_t seg;
    int32_t pad;
};

// Per-segment constants (a segment is one graph of a block-diagonal batch).
struct SegInfo {
    int32_t row_begin;   // first row of the segment in the packed numbering
    int32_t rows;        // n of the graph
    int32_t cta_begin;   // first CTA (within a panel) of the step kernel
    int32_t cta_count;
    int32_t tile_begin;  // first row tile (within a panel)
    int32_t tile_count;
    int32_t hub_begin;   // long rows of the segment: hubs [hub_begin, hub_begin + hub_count)
    int32_t hub_count;
    double scale;        // A = scale * M for the stored operator M
    double tau;          // breakdown threshold on beta (for M)
};

}  // namespace vne
