// Allocation-free Lanczos quadrature entry point (vne_quadform_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// quadratic form: code running under another framework's memory pool that
// must not be bypassed, real-time loops that forbid allocator calls, or
// embedding hosts that hand the library only the buffers they own.  This
// entry point serves them: the caller passes the CSR pattern, the probe
// vectors and the output array (all device memory it owns), and every
// intermediate (Lanczos vectors, alpha/beta, cross-CTA partial sums and their
// counters) lives in one fixed static device array defined below.  The host
// side allocates nothing either (no cudaMalloc/cudaFree, no host containers).
//
// Limits and sharing:
//  - The scratch array holds VNE_NOALLOC_SCRATCH_BYTES (32 MiB) on every GPU
//    that loads the library, for the life of the process.
//  - All calls share that one array and it keeps the previous call's
//    contents; each call clears the parts that must start at zero.  Calls
//    whose work overlaps on a GPU (different streams, or host threads) race
//    on the array and give wrong results: serialise them.
//  - The first call on each device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
//
// The kernels are plan-free variants of the main engine's step and update
// kernels: a warp takes a fixed run of 32 consecutive rows instead of a
// precomputed work-item schedule, so no schedule has to be uploaded.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/vne.h"
#include "kernels.h"

namespace vne {
namespace noalloc {

constexpr size_t kScratchBytes = VNE_NOALLOC_SCRATCH_BYTES;
constexpr int KS = 8;          // columns per panel (FP64: 4 lanes per row)
constexpr int CPL = 2;         // doubles per lane (16 bytes)
constexpr int LPR = KS / CPL;  // lanes per row
constexpr int G = 32 / LPR;    // row groups per warp
constexpr int ROWS_PER_WARP = 32;
constexpr int ROWS_PER_CTA = ROWS_PER_WARP * VNE_WARPS;
constexpr int TILE_ROWS = 4096;
constexpr int kMaxDevices = 64;

// The scratch array.  Host code never dereferences this symbol: on the host
// it is only a stand-in, and its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Layout {
    double* w;        // 3 vector slots (w_j, w_{j-1} / w_{j+1}, u): 3 * n * Kp
    double* alpha;    // [m][Kp]
    double* beta;     // [m][Kp]
    double* sigma;    // [m+1][Kp]
    double* norm2;    // [Kp]
    double* mean;     // [Kp]
    double* scale;    // [Kp]
    double* part;     // [P][max(ctas, tiles)][KS]
    uint32_t* counter;  // [P]  (zeroed per call)
    int32_t* maxdeg;    // [1]  (zeroed per call)
    int32_t* bad;       // [1]  (zeroed per call): set when the CSR input is invalid
    size_t bytes;       // total bytes used
    size_t zero_offset; // byte offset of the region that must start at zero
    size_t zero_bytes;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

inline Layout make_layout(unsigned char* base, int n, int Kp, int m, int P, int parts) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return base + at;
    };
    L.w = (double*)take(3 * (size_t)n * Kp * sizeof(double));
    L.alpha = (double*)take((size_t)m * Kp * sizeof(double));
    L.beta = (double*)take((size_t)m * Kp * sizeof(double));
    L.sigma = (double*)take((size_t)(m + 1) * Kp * sizeof(double));
    L.norm2 = (double*)take((size_t)Kp * sizeof(double));
    L.mean = (double*)take((size_t)Kp * sizeof(double));
    L.scale = (double*)take((size_t)Kp * sizeof(double));
    L.part = (double*)take((size_t)P * parts * KS * sizeof(double));
    L.zero_offset = o;
    L.counter = (uint32_t*)take((size_t)P * sizeof(uint32_t));
    L.maxdeg = (int32_t*)take(sizeof(int32_t));
    L.bad = (int32_t*)take(sizeof(int32_t));
    L.zero_bytes = o - L.zero_offset;
    L.bytes = o;
    return L;
}

// Last-arriving-CTA reduction of KS partials per CTA (fixed order).
__device__ bool last_cta(const double* part, uint32_t* counter, int panel, int nparts, double* tot) {
    __shared__ int s_last;
    __shared__ double red[VNE_THREADS];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == (unsigned)(nparts - 1));
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    constexpr int NS = VNE_THREADS / KS;
    const int c = threadIdx.x % KS, s = threadIdx.x / KS;
    double acc = 0.0;
    for (int i = s; i < nparts; i += NS) acc += __ldcg(&part[((size_t)panel * nparts + i) * KS + c]);
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < KS) {
        double t = 0.0;
        for (int q = 0; q < NS; q++) t += red[q * KS + threadIdx.x];
        tot[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

__device__ void cta_partial(double v, int panel, int idx, int nparts, double* part) {
    // v: this thread's partial for column threadIdx.x % KS
    __shared__ double red[VNE_THREADS];
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < KS) {
        double s = 0.0;
        for (int q = threadIdx.x; q < VNE_THREADS; q += KS) s += red[q];
        part[((size_t)panel * nparts + idx) * KS + threadIdx.x] = s;
    }
}

// Largest degree and the trace scale; rows that are not a CSR (a negative
// offset, a decreasing pair of offsets, no stored entry at all) mark the
// input invalid instead.
__global__ void k_init(const int32_t* rowptr, int n, int Kp, Layout L) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t a = rowptr[i], b = rowptr[i + 1];
        if (a < 0 || b < a) atomicExch(L.bad, 1);
        else atomicMax(L.maxdeg, b - a);
    }
    const int32_t nnz = rowptr[n];
    if (i == 0 && nnz <= 0) atomicExch(L.bad, 1);
    if (i < Kp) L.scale[i] = nnz > 0 ? 1.0 / (double)nnz : 0.0;
}

// psi = NaN for every column when the input was found invalid.
__global__ void k_mark_invalid(const Layout L, int k, double* psi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k && *L.bad) psi[c] = __longlong_as_double(0x7ff8000000000000LL);
}

// pass 1: column means; pass 2 (center = 1): w_1 = b - mean, ||c||^2, sigma_1
__global__ void __launch_bounds__(VNE_THREADS) k_start(const double* X, int n, int k, int Kp, int tiles, int center,
                                                       Layout L) {
    const int panel = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int c = threadIdx.x % KS, rs = threadIdx.x / KS;
    const int gc = panel * KS + c;
    const int r0 = tile * TILE_ROWS, r1 = min(n, r0 + TILE_ROWS);
    const double mu = center ? L.mean[gc] : 0.0;
    double* w1 = L.w + (size_t)panel * n * KS;
    double acc = 0.0;
    for (int r = r0 + rs; r < r1; r += VNE_THREADS / KS) {
        double v = (gc < k) ? X[(size_t)r * k + gc] : 0.0;
        if (center) {
            v = (gc < k) ? v - mu : 0.0;
            w1[(size_t)r * KS + c] = v;
            acc += v * v;
        } else {
            acc += v;
        }
    }
    cta_partial(acc, panel, tile, tiles, L.part);
    __shared__ double tot[KS];
    if (last_cta(L.part, L.counter + panel, panel, tiles, tot) && threadIdx.x < KS) {
        int col = panel * KS + threadIdx.x;
        if (center) {
            L.norm2[col] = tot[threadIdx.x];
            L.sigma[col] = tot[threadIdx.x] > 0.0 ? 1.0 / sqrt(tot[threadIdx.x]) : 0.0;
        } else {
            L.mean[col] = tot[threadIdx.x] / (double)n;
        }
    }
}

// u = sigma_j L w_j - beta_{j-1} sigma_{j-1} w_{j-1};  alpha_j = sigma_j (w_j . u)
__global__ void __launch_bounds__(VNE_THREADS) k_step_rows(const int32_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ col, int n, int Kp, int ctas,
                                                           int j, int s_cur, int s_prev, int s_u, Layout L) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPR, sub = lane % LPR, cofs = sub * CPL;
    const int panel = blockIdx.x / ctas, cta = blockIdx.x % ctas;
    const size_t slot = (size_t)n * Kp, pofs = (size_t)panel * n * KS;
    const double* W = L.w + s_cur * slot + pofs;
    const double* Wp = L.w + s_prev * slot + pofs;
    double* U = L.w + s_u * slot + pofs;
    const int colg = panel * KS + cofs;
    double sig[CPL], cp[CPL], dot[CPL];
    for (int q = 0; q < CPL; q++) {
        sig[q] = L.sigma[(size_t)(j - 1) * Kp + colg + q];
        cp[q] = (j > 1) ? L.beta[(size_t)(j - 2) * Kp + colg + q] * L.sigma[(size_t)(j - 2) * Kp + colg + q] : 0.0;
        dot[q] = 0.0;
    }
    const int r0 = cta * ROWS_PER_CTA + warp * ROWS_PER_WARP;
    const int r1 = min(n, r0 + ROWS_PER_WARP);
    const int nnz = rowptr[n];
    for (int r = r0 + g; r < r1; r += G) {
        int kb = rowptr[r], ke = rowptr[r + 1];
        if (kb < 0 || ke < kb || ke > nnz) {  // not a CSR row: no entry is read
            atomicExch(L.bad, 1);
            kb = ke = 0;
        }
        double acc[CPL] = {0.0, 0.0};
        for (int e = kb; e < ke; e++) {
            const int cc = col[e];
            if (cc < 0 || cc >= n) {  // outside the matrix: skipped, the input is marked invalid
                atomicExch(L.bad, 1);
                continue;
            }
            const double2 x = *reinterpret_cast<const double2*>(W + (size_t)cc * KS + cofs);
            acc[0] += x.x;
            acc[1] += x.y;
        }
        const double2 xs = *reinterpret_cast<const double2*>(W + (size_t)r * KS + cofs);
        double2 xp = make_double2(0.0, 0.0);
        if (j > 1) xp = *reinterpret_cast<const double2*>(Wp + (size_t)r * KS + cofs);
        const double deg = (double)(ke - kb);
        double2 u;
        u.x = sig[0] * (deg * xs.x - acc[0]) - cp[0] * xp.x;
        u.y = sig[1] * (deg * xs.y - acc[1]) - cp[1] * xp.y;
        *reinterpret_cast<double2*>(U + (size_t)r * KS + cofs) = u;
        dot[0] += xs.x * u.x;
        dot[1] += xs.y * u.y;
    }
    // reduce over the row groups of the warp, then over warps
    for (int q = 0; q < CPL; q++)
        for (int off = LPR; off < 32; off <<= 1) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], off);
    __shared__ double sred[VNE_WARPS][KS];
    if (g == 0)
        for (int q = 0; q < CPL; q++) sred[warp][cofs + q] = dot[q];
    __syncthreads();
    if (threadIdx.x < KS) {
        double s = 0.0;
        for (int w = 0; w < VNE_WARPS; w++) s += sred[w][threadIdx.x];
        L.part[((size_t)panel * ctas + cta) * KS + threadIdx.x] = s;
    }
    __shared__ double tot[KS];
    if (last_cta(L.part, L.counter + panel, panel, ctas, tot) && threadIdx.x < KS) {
        int c = panel * KS + threadIdx.x;
        L.alpha[(size_t)(j - 1) * Kp + c] = L.sigma[(size_t)(j - 1) * Kp + c] * tot[threadIdx.x];
    }
}

// w_{j+1} = u - alpha_j sigma_j w_j;  beta_j = ||w_{j+1}||;  sigma_{j+1} = 1 / beta_j
__global__ void __launch_bounds__(VNE_THREADS) k_update_rows(int n, int Kp, int tiles, int j, int s_cur, int s_u,
                                                             int s_next, Layout L) {
    const int panel = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int c = threadIdx.x % KS, rs = threadIdx.x / KS;
    const int gc = panel * KS + c;
    const size_t slot = (size_t)n * Kp, pofs = (size_t)panel * n * KS;
    const double* W = L.w + s_cur * slot + pofs;
    const double* U = L.w + s_u * slot + pofs;
    double* Wn = L.w + s_next * slot + pofs;
    const double a = L.alpha[(size_t)(j - 1) * Kp + gc] * L.sigma[(size_t)(j - 1) * Kp + gc];
    const int r0 = tile * TILE_ROWS, r1 = min(n, r0 + TILE_ROWS);
    double acc = 0.0;
    for (int r = r0 + rs; r < r1; r += VNE_THREADS / KS) {
        double v = U[(size_t)r * KS + c] - a * W[(size_t)r * KS + c];
        Wn[(size_t)r * KS + c] = v;
        acc += v * v;
    }
    cta_partial(acc, panel, tile, tiles, L.part);
    __shared__ double tot[KS];
    if (last_cta(L.part, L.counter + panel, panel, tiles, tot) && threadIdx.x < KS) {
        int col = panel * KS + threadIdx.x;
        double b = sqrt(tot[threadIdx.x]);
        double tau = 1e-13 * 2.0 * (double)(*L.maxdeg);
        if (!(b > tau) || L.sigma[(size_t)(j - 1) * Kp + col] == 0.0) {
            L.beta[(size_t)(j - 1) * Kp + col] = 0.0;
            L.sigma[(size_t)j * Kp + col] = 0.0;
        } else {
            L.beta[(size_t)(j - 1) * Kp + col] = b;
            L.sigma[(size_t)j * Kp + col] = 1.0 / b;
        }
    }
}

// per-device cache of the scratch array's device address (no allocation)
static void* g_addr[kMaxDevices];
static bool g_ready[kMaxDevices];

}  // namespace noalloc
}  // namespace vne

using namespace vne::noalloc;

extern "C" vne_status vne_quadform_noalloc(void* stream, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                           const double* vectors, int32_t k, int32_t krylov_steps, double* psi) {
    if (n < 1 || k < 1 || krylov_steps < 1 || krylov_steps > 128 || !row_ptr || !col_idx || !vectors || !psi)
        return VNE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VNE_EDEVICE;
    if (!g_ready[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return VNE_EDEVICE;
        g_addr[dev] = p;
        g_ready[dev] = true;
    }
    // an error already pending on this thread belongs to earlier work: leave
    // it for its owner and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return VNE_EDEVICE;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = krylov_steps;
    const int P = (k + KS - 1) / KS, Kp = P * KS;
    const int ctas = (n + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
    const int tiles = (n + TILE_ROWS - 1) / TILE_ROWS;
    const int parts = ctas > tiles ? ctas : tiles;
    Layout L = make_layout((unsigned char*)g_addr[dev], n, Kp, m, P, parts);
    if (L.bytes > kScratchBytes) return VNE_EINVAL;  // n * k too large for the fixed scratch
    if (cudaMemsetAsync((unsigned char*)g_addr[dev] + L.zero_offset, 0, L.zero_bytes, st) != cudaSuccess)
        return VNE_EDEVICE;
    if (cudaMemsetAsync(L.alpha, 0, (size_t)m * Kp * sizeof(double), st) != cudaSuccess) return VNE_EDEVICE;
    if (cudaMemsetAsync(L.beta, 0, (size_t)m * Kp * sizeof(double), st) != cudaSuccess) return VNE_EDEVICE;
    if (cudaMemsetAsync(L.sigma, 0, (size_t)(m + 1) * Kp * sizeof(double), st) != cudaSuccess) return VNE_EDEVICE;
    // every launch is checked right after it is made (the pending-error
    // check above makes the status this call's own)
    const int nb = (n > Kp ? n : Kp);
    k_init<<<(nb + 255) / 256, 256, 0, st>>>(row_ptr, n, Kp, L);
    if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
    k_start<<<P * tiles, VNE_THREADS, 0, st>>>(vectors, n, k, Kp, tiles, 0, L);
    if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
    k_start<<<P * tiles, VNE_THREADS, 0, st>>>(vectors, n, k, Kp, tiles, 1, L);
    if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
    // slots: w_j in slot (j-1) % 2, u in slot 2
    for (int j = 1; j <= m; j++) {
        const int s_cur = (j - 1) & 1, s_other = j & 1;
        k_step_rows<<<P * ctas, VNE_THREADS, 0, st>>>(row_ptr, col_idx, n, Kp, ctas, j, s_cur, s_other, 2, L);
        if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
        k_update_rows<<<P * tiles, VNE_THREADS, 0, st>>>(n, Kp, tiles, j, s_cur, 2, s_other, L);
        if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
    }
    if (vne::launch_tridiag_quad(L.alpha, L.beta, L.norm2, L.scale, k, m, Kp, psi, st) != cudaSuccess)
        return VNE_EDEVICE;
    k_mark_invalid<<<(k + 127) / 128, 128, 0, st>>>(L, k, psi);
    if (cudaGetLastError() != cudaSuccess) return VNE_EDEVICE;
    return VNE_OK;
}
