// The dense contractions of the Hutch++ sketch (Section 3.2) on the
// fifth-generation tensor cores (tcgen05): the Grams C = X^T Y of FP32
// panel-major blocks (the Cholesky-QR of Y = f(A) Omega, and Q^T G for the
// projection G - Q Q^T G) and the block products Out = In2 + coef In M
// (Q = Y R^{-1}, G' = G - Q (Q^T G)).  The block product is described
// above its kernel below; the Gram first.
//
// The contraction runs over the n rows of the blocks; the output is at most
// 128 x 128.  Each CTA owns a contiguous range of rows and accumulates its
// partial Gram in tensor memory (TMEM, FP32, one column per output column)
// over groups of slabs, and the groups in FP32 registers; the partials are
// summed in FP64 across CTAs by the caller's reduction.
//
// Pipeline per CTA (one CTA per SM, 256 threads):
//   * raw slabs of 32 rows are copied into shared memory with cp.async,
//     several slabs ahead (zero-filled past the CTA's last row);
//   * all threads split each raw value x into TF32 parts x = hi + lo
//     (hi = rna(x), lo = rna(x - hi)) and store them transposed into the
//     K-major operand layout without swizzling: 8-row x 16-byte core
//     matrices, 128 contiguous bytes each, core matrices 128 B apart along
//     K (the slab's rows) and 1024 B apart along M / N (the block columns);
//     the operand buffers are double-buffered, so the conversion of a slab
//     overlaps the tensor-core work on the previous one;
//   * one thread issues, per 8-row step of the slab, three kind::tf32 MMAs
//     (hi.hi + hi.lo + lo.hi: products at FP32 accuracy; for the Gram of a
//     block with itself two, E = (hi / 2) hi^T + hi lo^T, and the caller's
//     reduction forms E + E^T) of shape
//     M = 128 (columns of X, zero-padded) x N = ky rounded up to 16, and
//     commits them to the buffer's mbarrier; the threads wait on that
//     mbarrier before they overwrite the buffer two slabs later;
//   * the tensor core's FP32 accumulation drifts over long chains (about
//     7e-5 of sum |x_i y_i| after 2,500 accumulations), so the MMAs of 8
//     slabs go into one of two TMEM accumulators, and once they are done the
//     threads add that accumulator into FP32 registers (tcgen05.ld) while
//     the next group runs into the other one.
// Every wait is bounded: a wait that runs out sets *err, and the CTA stops,
// waits for its copies and (bounded) for the last MMA commit on each
// mbarrier, frees its TMEM and returns.
#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace vne {
namespace {

constexpr int kSlab = 32;                       // rows per slab (the contraction dimension)
constexpr int kRawLd = 128;                     // raw row in floats (a warp reads 32 consecutive columns of a row)
constexpr int kRawFloats = kSlab * kRawLd;      // one raw slab of one block
constexpr int kOpBytes = 128 * kSlab * 4;       // one TF32 operand slab: 128 rows x 32 K x 4 B
constexpr uint32_t kLbo = 128;                  // byte step between core matrices along K
constexpr uint32_t kSbo = (kSlab / 4) * 128;    // byte step between 8-row groups (1024)
constexpr uint32_t kWaitPolls = 1u << 20;       // mbarrier polls before a wait is abandoned
constexpr int kTmemCols = 256;                  // two accumulators of 128 FP32 columns (N <= 128)
constexpr int kGroup = 8;                       // slabs accumulated in TMEM before a flush to registers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Shared-memory matrix descriptor of a K-major operand without swizzling:
// start address, leading (K) and stride (M/N) byte offsets, all >> 4;
// bits 46-47 hold the descriptor version (1), swizzle mode 0 (none).
__device__ __forceinline__ uint64_t op_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kLbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kSbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5), A = B = TF32
// (bits 7-9, 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t polls = kWaitPolls) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < polls; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// After a wait gave up: let every MMA already issued finish before the TMEM
// is released.  Work unit t commits to mbarrier t & 1 (phase t >> 1), and a
// unit is committed only after the previous commit to the same barrier has
// completed, so each barrier has at most one phase outstanding: that of the
// last unit committed to it.  The waits use the full poll limit.
__device__ __forceinline__ void drain_commits(uint64_t* mbar, int committed) {
    for (int b = 0; b < 2; b++) {
        const int t = ((committed - 1) & 1) == b ? committed - 1 : committed - 2;
        if (t >= 0) mbar_wait(mbar + b, (uint32_t)(t >> 1) & 1u);
    }
}

// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool SAME>
struct GramSmem {
    static constexpr int kOps = SAME ? 3 : 4;     // per buffer: A hi, A lo, then hi / 2 or B hi, B lo
    static constexpr int kStages = SAME ? 6 : 3;  // raw slab buffers (kStages - 1 slabs in flight)
    static constexpr int kRawBlocks = SAME ? 1 : 2;
    static constexpr int kOpRegion = 2 * kOps * kOpBytes;
    static constexpr int kRawRegion = kStages * kRawBlocks * kRawFloats * 4;
    static constexpr int kBytes = kOpRegion + kRawRegion + 32;  // + 2 mbarriers + TMEM address slot
};

// Split and transpose one raw slab (rows x columns, kRawLd stride) into the
// K-major TF32 hi / lo operand buffers (and hi / 2, exact, when half is
// given); columns >= k are written as zeros.
__device__ __forceinline__ void convert_slab(const float* raw, int k, unsigned char* hi, unsigned char* lo,
                                             unsigned char* half) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int q = threadIdx.x + 256 * i;  // 128 rows of the operand x 8 groups of 4 slab rows
        const int m = q & 127, kg = q >> 7;
        uint4 h = make_uint4(0u, 0u, 0u, 0u), l = make_uint4(0u, 0u, 0u, 0u);
        if (m < k) {
            const float x0 = raw[(4 * kg + 0) * kRawLd + m], x1 = raw[(4 * kg + 1) * kRawLd + m];
            const float x2 = raw[(4 * kg + 2) * kRawLd + m], x3 = raw[(4 * kg + 3) * kRawLd + m];
            h.x = tf32_rna(x0);
            h.y = tf32_rna(x1);
            h.z = tf32_rna(x2);
            h.w = tf32_rna(x3);
            l.x = tf32_rna(x0 - __uint_as_float(h.x));
            l.y = tf32_rna(x1 - __uint_as_float(h.y));
            l.z = tf32_rna(x2 - __uint_as_float(h.z));
            l.w = tf32_rna(x3 - __uint_as_float(h.w));
        }
        const uint32_t off = (uint32_t)(m >> 3) * kSbo + (uint32_t)kg * kLbo + (uint32_t)(m & 7) * 16;
        *reinterpret_cast<uint4*>(hi + off) = h;
        *reinterpret_cast<uint4*>(lo + off) = l;
        if (half)
            *reinterpret_cast<float4*>(half + off) =
                make_float4(0.5f * __uint_as_float(h.x), 0.5f * __uint_as_float(h.y), 0.5f * __uint_as_float(h.z),
                            0.5f * __uint_as_float(h.w));
    }
}

template <int KS, bool SAME>
__global__ void __launch_bounds__(256, 1)
    k_gram_tc5(const float* __restrict__ X, int kx, const float* __restrict__ Y, int ky, int n, int rows_per_chunk,
               double* __restrict__ part, int* __restrict__ err, uint32_t polls) {
    using L = GramSmem<SAME>;
    constexpr int V = KS / 4;  // 16-byte pieces per row of one panel
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ops = smem;  // [buffer][A hi, A lo, B hi, B lo]
    float* raw = reinterpret_cast<float*>(smem + L::kOpRegion);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L::kOpRegion + L::kRawRegion);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x;
    const int r_begin = chunk * rows_per_chunk;
    const int r_end = min(n, r_begin + rows_per_chunk);
    const int nslab = r_end > r_begin ? (r_end - r_begin + kSlab - 1) / kSlab : 0;
    const int ky16 = (ky + 15) & ~15;
    const int px = kx / KS, py = ky / KS;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    auto issue = [&](int s) {
        if (s < nslab) {
            const int rt = r_begin + s * kSlab;
            float* rx = raw + (s % L::kStages) * L::kRawBlocks * kRawFloats;
            const int nx = px * kSlab * V, ny = SAME ? 0 : py * kSlab * V;
            for (int idx = tid; idx < nx + ny; idx += 256) {
                const bool isx = idx < nx;
                const int e = isx ? idx : idx - nx;
                const int p = e / (kSlab * V), rem = e % (kSlab * V);
                const int rl = rem / V, c = (rem % V) * 4;
                const int r = rt + rl;
                const bool in = r < r_end;
                const float* src = (isx ? X : Y) + (size_t)p * n * KS + (size_t)(in ? r : r_begin) * KS + c;
                float* dst = rx + (isx ? 0 : kRawFloats) + rl * kRawLd + p * KS + c;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                             "r"(in ? 16 : 0)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const uint32_t idesc = idesc_tf32(128, ky16);
    // this warp's share of the output: TMEM lanes 32 * quarter .. + 31 (one
    // output row per lane), column blocks c0 = 32 * ((warp >> 2) + 2 i)
    const int quarter = warp & 3;
    float acc[2][32];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 32; j++) acc[i][j] = 0.f;
    auto flush = [&](int g) {  // add accumulator g & 1 (all its MMAs done) into acc
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int c0 = ((warp >> 2) + 2 * i) * 32;
            if (c0 < ky16) {  // warp-uniform
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((g & 1) * 128 + c0), v);
#pragma unroll
                for (int j = 0; j < 32; j++) acc[i][j] += __uint_as_float(v[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };
    int next_flush = 0;  // first group not yet added into acc
    bool failed = false;
    int committed = nslab;  // slabs whose MMAs were issued
    for (int s = 0; s < L::kStages - 1; s++) issue(s);
    for (int s = 0; s < nslab; s++) {
        // slabs s .. s + kStages - 2 are in flight: wait for slab s
        asm volatile("cp.async.wait_group %0;" ::"n"(L::kStages - 2) : "memory");
        const int b = s & 1;
        // the MMAs of slab s - 2 read operand buffer b
        const bool ready = s < 2 || mbar_wait(mbar + b, (uint32_t)((s - 2) >> 1) & 1u, polls);
        if (__syncthreads_or(!ready)) {  // also: slab s has landed for every thread's copies
            failed = true;
            committed = s;
            break;
        }
        // the groups whose last slab is <= s - 2 are complete
        while (next_flush < (s - 1) / kGroup) flush(next_flush++);
        unsigned char* buf = ops + b * L::kOps * kOpBytes;
        convert_slab(raw + (s % L::kStages) * L::kRawBlocks * kRawFloats, kx, buf, buf + kOpBytes,
                     SAME ? buf + 2 * kOpBytes : nullptr);
        if (!SAME) convert_slab(raw + (s % L::kStages) * L::kRawBlocks * kRawFloats + kRawFloats, ky,
                                buf + 2 * kOpBytes, buf + 3 * kOpBytes, nullptr);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(buf), a_lo = a_hi + kOpBytes;
            const uint32_t d = tmem + (uint32_t)(((s / kGroup) & 1) * 128);
            const bool first = (s % kGroup) == 0;
#pragma unroll
            for (int t = 0; t < kSlab / 8; t++) {
                const uint32_t o = (uint32_t)t * 2 * kLbo;  // two core matrices of K per MMA
                if (SAME) {
                    // E = (H / 2) H^T + H L^T, so that E + E^T = H H^T + H L^T + L H^T
                    const uint32_t a_half = a_hi + 2 * kOpBytes;
                    mma_tf32(d, op_desc(a_half + o), op_desc(a_hi + o), idesc, (!first || t > 0) ? 1u : 0u);
                    mma_tf32(d, op_desc(a_hi + o), op_desc(a_lo + o), idesc, 1u);
                } else {
                    const uint32_t b_hi = a_hi + 2 * kOpBytes, b_lo = b_hi + kOpBytes;
                    mma_tf32(d, op_desc(a_hi + o), op_desc(b_hi + o), idesc, (!first || t > 0) ? 1u : 0u);
                    mma_tf32(d, op_desc(a_hi + o), op_desc(b_lo + o), idesc, 1u);
                    mma_tf32(d, op_desc(a_lo + o), op_desc(b_hi + o), idesc, 1u);
                }
            }
            mma_commit(mbar + b);
        }
        // the next prefetch goes into the stage converted in the previous
        // iteration; it is issued after the proxy fence above, so that the
        // fence does not wait for it
        issue(s + L::kStages - 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (nslab > 0 && !failed) {
        const int sl = nslab - 1;
        const bool done = mbar_wait(mbar + (sl & 1), (uint32_t)(sl >> 1) & 1u, polls);
        failed = __syncthreads_or(!done);
    }
    if (failed) {
        if (tid == 0) atomicExch(err, 1);
        drain_commits(mbar, committed);  // bounded; the outcome is already an error
    } else {
        const int ngroups = (nslab + kGroup - 1) / kGroup;
        while (next_flush < ngroups) flush(next_flush++);
        const int row = quarter * 32 + lane;  // output row = column of X
        double* dst = part + (size_t)chunk * kx * ky + (size_t)row * ky;
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int c0 = ((warp >> 2) + 2 * i) * 32;
            if (row < kx && c0 < ky16) {
#pragma unroll
                for (int j = 0; j < 32; j++)
                    if (c0 + j < ky) dst[c0 + j] = (double)acc[i][j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Poll limit of the main-loop waits of both kernels (kWaitPolls unless a
// failure-injection test lowered it); the drain after a failure always uses
// kWaitPolls.
uint32_t g_main_polls = kWaitPolls;

template <int KS, bool SAME>
cudaError_t gram_tc5_launch(const float* X, int kx, const float* Y, int ky, int n, int rpc, int chunks, double* part,
                            int* err, cudaStream_t st) {
    const int smem = GramSmem<SAME>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc5<KS, SAME>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_gram_tc5<KS, SAME><<<chunks, 256, smem, st>>>(X, kx, Y, ky, n, rpc, part, err, g_main_polls);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_tc5(const float* X, int kx, const float* Y, int ky, int ks, int n, double* part, int max_chunks,
                            int* err, int* chunks_out, int* sym_out, cudaStream_t st) {
    if (kx < 1 || ky < 1 || kx > 128 || ky > 128 || n < 1 || max_chunks < 1 || !err || !chunks_out || !sym_out)
        return cudaErrorInvalidValue;
    if ((ks != 8 && ks != 16 && ks != 32) || kx % ks || ky % ks) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one CTA per SM, each over an equal share of the rows (a multiple of the slab)
    const int want = std::max(1, std::min(max_chunks, sms));
    int rpc = (n + want - 1) / want;
    rpc = ((rpc + kSlab - 1) / kSlab) * kSlab;
    const int chunks = (n + rpc - 1) / rpc;
    *chunks_out = chunks;
    const bool same = (X == Y) && (kx == ky);
    *sym_out = same ? 1 : 0;  // the partials of a block with itself hold E, the Gram is E + E^T
#define VNE_TC5(KSV)                                                                                      \
    if (ks == KSV)                                                                                        \
        return same ? gram_tc5_launch<KSV, true>(X, kx, Y, ky, n, rpc, chunks, part, err, st)             \
                    : gram_tc5_launch<KSV, false>(X, kx, Y, ky, n, rpc, chunks, part, err, st);
    VNE_TC5(8)
    VNE_TC5(16)
    VNE_TC5(32)
#undef VNE_TC5
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Block product Out = (In2 ? In2 : 0) + coef In M for FP32 panel-major blocks
// In [n x kin], Out [n x kout] (kin, kout <= 128) and M FP64 [kin x kout].
// The MMA's M dimension is a tile of 128 rows of In, N = kout rounded up to
// 16 and K = kin, taken in chunks of 32 columns.  B = coef M^T is split
// into TF32 hi / lo once per CTA and stays in shared memory (K-major, one
// 32-column region per chunk).  For each (tile, chunk) unit the threads load
// the chunk from HBM into registers one unit ahead (16-byte loads, rows in
// order) and store its hi / lo parts into one of two A buffers; one thread
// issues hi.hi + hi.lo + lo.hi per 8 columns of K into the tile's TMEM
// accumulator (two, alternating between tiles) and commits to the buffer's
// mbarrier.  Once a tile's last unit is done, the threads read its
// accumulator (tcgen05.ld, one row per lane), add In2 and store Out, while
// the next tile accumulates into the other one.  Persistent grid, one CTA
// per SM; bounded waits as in the Gram.
namespace {

constexpr int kApplyChunk = 32;  // K columns per unit

template <int KS>
__global__ void __launch_bounds__(256, 1)
    k_apply_tc5(const float* __restrict__ In, int kin, const double* __restrict__ Mat, int kout,
                const float* __restrict__ In2, float* __restrict__ Out, int n, double coef, int* __restrict__ err,
                uint32_t polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nk = (kin + kApplyChunk - 1) / kApplyChunk;  // K chunks
    const int kout16 = (kout + 15) & ~15;
    const int bchunk = (kout16 / 8) * (int)kSbo;            // bytes of one B chunk (N rows x 32 K)
    unsigned char* b_hi = smem;
    unsigned char* b_lo = smem + nk * bchunk;
    unsigned char* a_ops = smem + 2 * nk * bchunk;          // [2 buffers][hi, lo] x 16 KB
    uint64_t* mbar = reinterpret_cast<uint64_t*>(a_ops + 4 * kOpBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (n + 127) / 128;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nunits = my_tiles * nk;

    // B = coef M^T, TF32 hi / lo, K-major per 32-column chunk
    for (int idx = tid; idx < nk * kApplyChunk * kout16; idx += 256) {
        const int k = idx / kout16, c = idx % kout16;
        const float x = (k < kin && c < kout) ? (float)(coef * Mat[(size_t)k * kout + c]) : 0.f;
        const uint32_t h = tf32_rna(x), l = tf32_rna(x - __uint_as_float(h));
        const uint32_t off = (uint32_t)(k / kApplyChunk) * bchunk + (uint32_t)(c >> 3) * kSbo +
                             (uint32_t)((k % kApplyChunk) >> 2) * kLbo + (uint32_t)(c & 7) * 16 + (uint32_t)(k & 3) * 4;
        *reinterpret_cast<uint32_t*>(b_hi + off) = h;
        *reinterpret_cast<uint32_t*>(b_lo + off) = l;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B, written by the generic proxy
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_tf32(128, kout16);

    // unit u = (local tile u / nk, chunk u % nk); this thread's four
    // 16-byte pieces: operand row m, 4-column group kg of the chunk
    auto load_unit = [&](int u, float4 (&v)[4]) {
        const int tile = (int)blockIdx.x + (u / nk) * (int)gridDim.x, kc = u % nk;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int q = tid + 256 * i;
            const int m = (q & 7) + 8 * (q >> 6), kg = (q >> 3) & 7;
            const int r = tile * 128 + m, col = kc * kApplyChunk + 4 * kg;
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < n && col < kin)
                v[i] = __ldcs(reinterpret_cast<const float4*>(In + (size_t)(col / KS) * n * KS + (size_t)r * KS +
                                                              (col % KS)));
        }
    };
    auto store_unit = [&](const float4 (&v)[4], unsigned char* hi, unsigned char* lo) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int q = tid + 256 * i;
            const int m = (q & 7) + 8 * (q >> 6), kg = (q >> 3) & 7;
            uint4 h, l;
            h.x = tf32_rna(v[i].x);
            h.y = tf32_rna(v[i].y);
            h.z = tf32_rna(v[i].z);
            h.w = tf32_rna(v[i].w);
            l.x = tf32_rna(v[i].x - __uint_as_float(h.x));
            l.y = tf32_rna(v[i].y - __uint_as_float(h.y));
            l.z = tf32_rna(v[i].z - __uint_as_float(h.z));
            l.w = tf32_rna(v[i].w - __uint_as_float(h.w));
            const uint32_t off = (uint32_t)(m >> 3) * kSbo + (uint32_t)kg * kLbo + (uint32_t)(m & 7) * 16;
            *reinterpret_cast<uint4*>(hi + off) = h;
            *reinterpret_cast<uint4*>(lo + off) = l;
        }
    };
    const int quarter = warp & 3;
    auto epilogue = [&](int i) {  // local tile i: accumulator i & 1 holds coef In M for its 128 rows
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        const int r = tile * 128 + quarter * 32 + lane;
#pragma unroll 1
        for (int j = 0; j < 2; j++) {
            const int c0 = ((warp >> 2) + 2 * j) * 32;
            if (c0 >= kout16) continue;  // warp-uniform
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((i & 1) * 128 + c0), v);
            if (r < n) {
#pragma unroll
                for (int g = 0; g < 8; g++) {
                    const int c = c0 + 4 * g;
                    if (c < kout) {
                        const size_t o = (size_t)(c / KS) * n * KS + (size_t)r * KS + (c % KS);
                        float4 y = make_float4(__uint_as_float(v[4 * g]), __uint_as_float(v[4 * g + 1]),
                                               __uint_as_float(v[4 * g + 2]), __uint_as_float(v[4 * g + 3]));
                        if (In2) {
                            const float4 z = __ldcs(reinterpret_cast<const float4*>(In2 + o));
                            y.x += z.x, y.y += z.y, y.z += z.z, y.w += z.w;
                        }
                        __stcs(reinterpret_cast<float4*>(Out + o), y);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    bool failed = false;
    int committed = nunits;  // units whose MMAs were issued
    int next_epi = 0;
    float4 cur[4], nxt[4];
    if (nunits > 0) load_unit(0, cur);
    for (int u = 0; u < nunits; u++) {
        if (u + 1 < nunits) load_unit(u + 1, nxt);
        const int b = u & 1;
        const bool ready = u < 2 || mbar_wait(mbar + b, (uint32_t)((u - 2) >> 1) & 1u, polls);
        if (__syncthreads_or(!ready)) {
            failed = true;
            committed = u;
            break;
        }
        // tiles whose last unit is <= u - 2 are complete
        while (next_epi < my_tiles && (next_epi + 1) * nk - 1 <= u - 2) epilogue(next_epi++);
        unsigned char* hi = a_ops + b * 2 * kOpBytes;
        store_unit(cur, hi, hi + kOpBytes);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int i = u / nk, kc = u % nk;
            const uint32_t d = tmem + (uint32_t)((i & 1) * 128);
            const uint32_t ah = smem_u32(hi), al = ah + kOpBytes;
            const uint32_t bh = smem_u32(b_hi) + (uint32_t)(kc * bchunk), bl = smem_u32(b_lo) + (uint32_t)(kc * bchunk);
            const int steps = min(kApplyChunk / 8, (kin - kc * kApplyChunk + 7) / 8);
            for (int t = 0; t < steps; t++) {
                const uint32_t o = (uint32_t)t * 2 * kLbo;
                mma_tf32(d, op_desc(ah + o), op_desc(bh + o), idesc, (kc > 0 || t > 0) ? 1u : 0u);
                mma_tf32(d, op_desc(ah + o), op_desc(bl + o), idesc, 1u);
                mma_tf32(d, op_desc(al + o), op_desc(bh + o), idesc, 1u);
            }
            mma_commit(mbar + b);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) cur[i] = nxt[i];
    }
    if (nunits > 0 && !failed) {
        const int ul = nunits - 1;
        const bool done = mbar_wait(mbar + (ul & 1), (uint32_t)(ul >> 1) & 1u, polls);
        failed = __syncthreads_or(!done);
    }
    if (failed) {
        if (tid == 0) atomicExch(err, 1);
        drain_commits(mbar, committed);  // bounded; the outcome is already an error
    } else {
        while (next_epi < my_tiles) epilogue(next_epi++);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

cudaError_t launch_apply_tc5(const float* In, int kin, const double* M, int kout, const float* In2, float* Out, int ks,
                             int n, double coef, int* err, cudaStream_t st) {
    if (kin < 1 || kout < 1 || kin > 128 || kout > 128 || n < 1 || !err) return cudaErrorInvalidValue;
    if ((ks != 8 && ks != 16 && ks != 32) || kin % ks || kout % ks) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nk = (kin + kApplyChunk - 1) / kApplyChunk;
    const int kout16 = (kout + 15) & ~15;
    const int smem = 2 * nk * (kout16 / 8) * (int)kSbo + 4 * kOpBytes + 32;
    const int ntiles = (n + 127) / 128;
    const int grid = std::max(1, std::min(ntiles, sms));
#define VNE_APPLY5(KSV)                                                                                       \
    if (ks == KSV) {                                                                                          \
        e = cudaFuncSetAttribute(k_apply_tc5<KSV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);         \
        if (e != cudaSuccess) return e;                                                                       \
        k_apply_tc5<KSV><<<grid, 256, smem, st>>>(In, kin, M, kout, In2, Out, n, coef, err, g_main_polls);     \
        return cudaGetLastError();                                                                            \
    }
    VNE_APPLY5(8)
    VNE_APPLY5(16)
    VNE_APPLY5(32)
#undef VNE_APPLY5
    return cudaErrorInvalidValue;
}

void set_tensor_wait_polls(int64_t polls) {
    g_main_polls = polls < 0 ? kWaitPolls : (uint32_t)std::min<int64_t>(polls, kWaitPolls);
}

}  // namespace vne
