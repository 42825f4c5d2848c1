// Lanczos hot-path kernels of libvne: start vectors (probe generation and
// implicit desingularisation), the fused SpMM step, the three-term update,
// full reorthogonalisation and the Lanczos matvec recovery.
//
// Vector layout ("panel-major"): a block of K = P * KS columns over the
// packed rows is stored as P panels, each [n_total][KS] row-major, so one row
// of a panel is KS contiguous values (32-128 bytes) and a neighbour gather
// reads whole sectors.  Panels are processed in blockIdx order, which keeps
// the panel being gathered resident in L2 while the others stream.
//
// Lanczos in scaled form (Section 4, polynomial Krylov).  Slot j holds an
// unnormalised basis vector w_j with v_j = sigma_j w_j (sigma_1 = 1/||c||,
// sigma_{j+1} = 1/beta_j), so normalisation never needs its own pass:
//   step kernel   u     = sigma_j M w_j - beta_{j-1} sigma_{j-1} w_{j-1}
//                 alpha_j = sigma_j (w_j . u)
//   update kernel w_{j+1} = u - alpha_j sigma_j w_j,  beta_j = ||w_{j+1}||
// M is the stored operator (the Laplacian L for a graph, kept implicit) and
// A = scale * M; alpha and beta here belong to M and are scaled in FP64 by
// the quadrature.  Inner products are accumulated per lane in the vector
// precision over at most a few rows, then in FP64 across lanes, warps and
// CTAs; the cross-CTA sums are done by the last CTA to arrive for each
// (panel, segment), in a fixed order, so results are bit-reproducible.
#include "common.cuh"
#include "kernels.h"

namespace vne {

// ---------------------------------------------------------------------------
// fixed-order cross-CTA reduction
//
// Every CTA writes NQ*KS partial values at part[(panel*nparts + idx)*W + c]
// (W = NQ*KS) and calls this; the CTA that arrives last for the counter sums
// the `count` partials starting at `begin` in index order and returns true
// with the totals in s_out[0..W).  The counter is reset for the next launch.
template <int W>
__device__ bool last_cta_reduce(const double* part, uint32_t* counter, int panel, int nparts,
                                int begin, int count, double* s_out) {
    __shared__ int s_last;
    __shared__ double red[VNE_THREADS];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned old = atomicAdd(counter, 1u);
        s_last = (old == (unsigned)(count - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    constexpr int NS = VNE_THREADS / W;
    const int c = threadIdx.x % W, s = threadIdx.x / W;
    // four independent accumulators, so that four loads are in flight at
    // once (the order of the additions is still fixed)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (s < NS) {
        const double* src = part + ((size_t)panel * nparts + begin) * W + c;
        int i = s;
        for (; i + 3 * NS < count; i += 4 * NS) {
#pragma unroll
            for (int u = 0; u < 4; u++) acc[u] += ld_cg(src + (size_t)(i + u * NS) * W);
        }
#pragma unroll
        for (int u = 0; u < 3; u++)
            if (i + u * NS < count) acc[u] += ld_cg(src + (size_t)(i + u * NS) * W);
    }
    red[threadIdx.x] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    __syncthreads();
    if (threadIdx.x < W) {
        double t = 0.0;
        for (int q = 0; q < NS; q++) t += red[q * W + threadIdx.x];
        s_out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// counter-based Rademacher entries (SplitMix64 mixer; see the header of
// abi.cu for the definition)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double rademacher_entry(uint64_t s, uint64_t col, uint64_t node) {
    uint64_t h = mix64((((col << 32) | node) ^ s) + 0x9E3779B97F4A7C15ULL);
    return (h >> 63) ? -1.0 : 1.0;
}

// Standard normal entries from the same counters (Box & Muller 1958): with
// h1 = h(col, node) and h2 = mix64(h1 + gamma), u1 = ((h1 >> 11) + 1/2) 2^-53
// and u2 = (h2 >> 11) 2^-53, x = sqrt(-2 log u1) cos(2 pi u2) in FP64.
__device__ __forceinline__ double gaussian_entry(uint64_t s, uint64_t col, uint64_t node) {
    const uint64_t h1 = mix64((((col << 32) | node) ^ s) + 0x9E3779B97F4A7C15ULL);
    const uint64_t h2 = mix64(h1 + 0x9E3779B97F4A7C15ULL);
    const double u1 = ((double)(h1 >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = (double)(h2 >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Start-vector source value for packed row r (local node id `id`, segment
// seg) and block column gc (global within the block).
__device__ __forceinline__ double source_value(const StartSource& S, int r, int id, int gc, int seg) {
    if (gc >= S.ncols) return 0.0;
    switch (S.kind) {
        case SRC_RADEMACHER: {
            const uint64_t sd = S.seg_seed ? S.seg_seed[seg] : S.seed_mixed;
            const uint64_t col = S.seg_seed ? (uint64_t)(S.seg_col0[seg] + gc) : (uint64_t)(S.col_begin + gc);
            return S.gaussian ? gaussian_entry(sd, col, (uint64_t)id) : rademacher_entry(sd, col, (uint64_t)id);
        }
        case SRC_INDICATOR:
            return (S.colors[id] == S.col_begin + gc) ? 1.0 : 0.0;
        case SRC_DENSE64:
            return S.dense[(size_t)id * S.ld + gc];
        default:
            return 0.0;
    }
}

template <typename T, int KS>
__device__ __forceinline__ double source_value_panel(const StartSource& S, const T* panel_src, int r,
                                                     int id, int gc, int n_total, int seg) {
    if (S.kind == SRC_PANEL) {
        if (gc >= S.ncols) return 0.0;
        const T* base = panel_src + (size_t)(gc / KS) * n_total * KS;
        return (double)base[(size_t)r * KS + (gc % KS)];
    }
    return source_value(S, r, id, gc, seg);
}

// Source value in the vector precision: FP32 blocks take the value in FP32
// (exact for Rademacher and indicator entries), so the start passes do no
// FP64 arithmetic per entry.
template <typename T, int KS>
__device__ __forceinline__ T source_value_t(const StartSource& S, const T* panel_src, int r, int id, int gc,
                                            int n_total, int seg) {
    if (sizeof(T) == 8) return (T)source_value_panel<T, KS>(S, panel_src, r, id, gc, n_total, seg);
    if (gc >= S.ncols) return (T)0;
    switch (S.kind) {
        case SRC_RADEMACHER: {
            const uint64_t s = S.seg_seed ? S.seg_seed[seg] : S.seed_mixed;
            const uint64_t col = S.seg_seed ? (uint64_t)(S.seg_col0[seg] + gc) : (uint64_t)(S.col_begin + gc);
            if (S.gaussian) return (T)gaussian_entry(s, col, (uint64_t)id);
            const uint64_t h = mix64((((col << 32) | (uint64_t)id) ^ s) + 0x9E3779B97F4A7C15ULL);
            return (h >> 63) ? (T)-1 : (T)1;
        }
        case SRC_INDICATOR:
            return (S.colors[id] == S.col_begin + gc) ? (T)1 : (T)0;
        case SRC_DENSE64:
            return (T)S.dense[(size_t)id * S.ld + gc];
        case SRC_PANEL:
            return panel_src[(size_t)(gc / KS) * n_total * KS + (size_t)r * KS + (gc % KS)];
        default:
            return (T)0;
    }
}

// Per-thread sum over its rows: FP64 throughout for FP64 blocks; for FP32
// blocks FP32 partial sums of 16 rows, added in FP64 (a Rademacher column's
// partial sums are exact).
template <typename T>
struct RowSum {
    double acc = 0.0;
    T part = (T)0;
    int cnt = 0;
    __device__ __forceinline__ void add(T v) {
        if (sizeof(T) == 8) {
            acc += (double)v;
            return;
        }
        part += v;
        if (++cnt == 16) {
            acc += (double)part;
            part = (T)0;
            cnt = 0;
        }
    }
    __device__ __forceinline__ double total() const { return acc + (double)part; }
};

// Four consecutive entries of one row of a panel (16-byte aligned: the
// column offset is a multiple of 4 and a panel row holds KS >= 4 entries).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
    } else {
        const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
        v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
    }
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
}

// Rademacher entries of four block columns for one tile: key_j = (probe
// column << 32) ^ seed, so that the hash input ((col << 32) | node) ^ seed
// is key_j ^ node (the node id occupies the low 32 bits).
struct RadQuad {
    uint64_t key[4];
    bool live[4];
    __device__ __forceinline__ RadQuad(const StartSource& S, int seg, int gc0) {
        const uint64_t sd = S.seg_seed ? S.seg_seed[seg] : S.seed_mixed;
        const int cb = S.seg_seed ? S.seg_col0[seg] : S.col_begin;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            live[j] = gc0 + j < S.ncols;
            key[j] = ((uint64_t)(cb + gc0 + j) << 32) ^ sd;
        }
    }
    // the four entries of node id; neg[j] counts the -1 entries of live columns
    template <typename T>
    __device__ __forceinline__ void row(uint32_t id, T (&v)[4], int (&neg)[4]) const {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint64_t h = mix64((key[j] ^ (uint64_t)id) + 0x9E3779B97F4A7C15ULL);
            const int sgn = (int)(h >> 63);
            neg[j] += live[j] ? sgn : 0;
            v[j] = live[j] ? (sgn ? (T)-1 : (T)1) : (T)0;
        }
    }
};

// Per-column totals of a CTA: each thread holds four columns' partial sums;
// sum them over the threads of the same columns in a fixed order and write
// the CTA's partial for the segment reduction.
template <int KS>
__device__ __forceinline__ void cta_column_partials(const double (&sum)[4], int rsub, int c0, double* part_out) {
    constexpr int RPP = VNE_THREADS / (KS / 4);
    __shared__ double red[RPP][KS];
#pragma unroll
    for (int j = 0; j < 4; j++) red[rsub][c0 + j] = sum[j];
    __syncthreads();
    if (threadIdx.x < KS) {
        double s = 0.0;
        for (int q = 0; q < RPP; q++) s += red[q][threadIdx.x];
        part_out[threadIdx.x] = s;
    }
}

// The Rademacher entries of this thread's four columns for the rows of a
// tile (stored as they are generated if STORE); the node ids of four rows
// are loaded before their hashes.  Returns the rows taken, counts the -1
// entries.
template <typename T, int KS, bool STORE>
__device__ __forceinline__ int rad_rows(const StartParams<T>& p, const RowTile& t, const SegInfo& sg,
                                        const RadQuad& rq, int rsub, int c0, T* out, int (&neg)[4]) {
    constexpr int RPP = VNE_THREADS / (KS / 4);
    int rows = 0;
    for (int r0 = t.row_begin + rsub; r0 < t.row_end; r0 += 4 * RPP) {
        uint32_t ids[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int r = r0 + u * RPP;
            ids[u] = r < t.row_end ? (p.node_id ? (uint32_t)__ldg(p.node_id + r) : (uint32_t)(r - sg.row_begin)) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int r = r0 + u * RPP;
            if (r < t.row_end) {
                T v[4];
                rq.row(ids[u], v, neg);
                if (STORE) st4(out + (size_t)r * KS + c0, v);
                rows++;
            }
        }
    }
    return rows;
}

// Pass 1: column sums per segment -> mean (only when desingularising).  A
// thread covers four consecutive columns of a row.  Rademacher sources take
// a dedicated path: four hashes per row and integer counts of the -1
// entries, so the column sums are exact (as the FP32 partial sums of +-1
// entries are); pass 2 generates them again (cheaper than a store and a
// read of the block).  Other sources are stored in w_1 on the way (16-byte
// stores) and pass 2 reads them back.
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS, 4) k_start_mean(StartParams<T> p) {
    const int panel = blockIdx.x / p.tiles_per_panel, tile = blockIdx.x % p.tiles_per_panel;
    const RowTile t = p.tiles[tile];
    const SegInfo sg = p.seg[t.seg];
    constexpr int QPR = KS / 4, RPP = VNE_THREADS / QPR;
    const int c0 = (threadIdx.x % QPR) * 4, rsub = threadIdx.x / QPR;
    const int gc0 = panel * KS + c0;
    T* out = p.w1 + (size_t)panel * p.n_total * KS;
    double sum[4];
    if (p.src.kind == SRC_RADEMACHER && !p.src.gaussian) {
        const RadQuad rq(p.src, t.seg, gc0);
        int neg[4] = {0, 0, 0, 0};
        const int rows = rad_rows<T, KS, false>(p, t, sg, rq, rsub, c0, out, neg);
#pragma unroll
        for (int j = 0; j < 4; j++) sum[j] = rq.live[j] ? (double)(rows - 2 * neg[j]) : 0.0;
    } else {
        RowSum<T> rs[4];
        for (int r = t.row_begin + rsub; r < t.row_end; r += RPP) {
            const int id = p.node_id ? __ldg(p.node_id + r) : r - sg.row_begin;
            T v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                v[j] = source_value_t<T, KS>(p.src, p.panel_src, r, id, gc0 + j, p.n_total, t.seg);
                rs[j].add(v[j]);
            }
            st4(out + (size_t)r * KS + c0, v);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) sum[j] = rs[j].total();
    }
    cta_column_partials<KS>(sum, rsub, c0, p.part + ((size_t)panel * p.tiles_per_panel + tile) * KS);
    __shared__ double tot[KS];
    if (last_cta_reduce<KS>(p.part, p.counter + (size_t)panel * p.nseg + t.seg, panel, p.tiles_per_panel,
                            sg.tile_begin, sg.tile_count, tot)) {
        if (threadIdx.x < KS)
            p.mean[(size_t)t.seg * p.K + panel * KS + threadIdx.x] = tot[threadIdx.x] / (double)sg.rows;
    }
}

// Pass 2: w_1 = b - mean (stored in T), ||w_1||^2 (FP64 across partial sums),
// sigma_1 = 1/||w_1||.  Rademacher entries are generated as in pass 1 and
// their squared norms follow in closed form (rows, or rows (1 - mean^2) for
// b - mean); other sources are read back from w_1, where pass 1 stored them
// (16-byte loads, four rows in flight per thread), or, without
// desingularisation, taken from the source.
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS, 3) k_start_center(StartParams<T> p) {
    const int panel = blockIdx.x / p.tiles_per_panel, tile = blockIdx.x % p.tiles_per_panel;
    const RowTile t = p.tiles[tile];
    const SegInfo sg = p.seg[t.seg];
    constexpr int QPR = KS / 4, RPP = VNE_THREADS / QPR;
    const int c0 = (threadIdx.x % QPR) * 4, rsub = threadIdx.x / QPR;
    const int gc0 = panel * KS + c0;
    T* out = p.w1 + (size_t)panel * p.n_total * KS;
    double sum[4];
    if (p.desing) {
        T mu[4];
        bool live[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            live[j] = gc0 + j < p.src.ncols;
            mu[j] = (T)p.mean[(size_t)t.seg * p.K + gc0 + j];
        }
        if (p.src.kind == SRC_RADEMACHER && !p.src.gaussian) {
            // generated again (pass 1 did not store them); with b_i^2 = 1 and
            // sum_i b_i = rows * mean, the squared norm of b - mean is
            // rows (1 - mean^2), so no per-entry accumulation is needed
            const RadQuad rq(p.src, t.seg, gc0);
            int neg[4] = {0, 0, 0, 0}, rows = 0;
            for (int r0 = t.row_begin + rsub; r0 < t.row_end; r0 += 4 * RPP) {
                uint32_t ids[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = r0 + u * RPP;
                    ids[u] = r < t.row_end ? (p.node_id ? (uint32_t)__ldg(p.node_id + r)
                                                         : (uint32_t)(r - sg.row_begin))
                                           : 0u;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = r0 + u * RPP;
                    if (r < t.row_end) {
                        T v[4];
                        rq.row(ids[u], v, neg);
#pragma unroll
                        for (int j = 0; j < 4; j++) v[j] = live[j] ? v[j] - mu[j] : (T)0;
                        st4(out + (size_t)r * KS + c0, v);
                        rows++;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const double m = p.mean[(size_t)t.seg * p.K + gc0 + j];
                sum[j] = live[j] ? (double)rows * (1.0 - m * m) : 0.0;
            }
        } else {
            RowSum<T> rs[4];
            for (int r0 = t.row_begin + rsub; r0 < t.row_end; r0 += 4 * RPP) {
                T v[4][4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = r0 + u * RPP;
                    if (r < t.row_end) ld4(out + (size_t)r * KS + c0, v[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = r0 + u * RPP;
                    if (r < t.row_end) {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            v[u][j] = live[j] ? v[u][j] - mu[j] : (T)0;
                            rs[j].add(v[u][j] * v[u][j]);
                        }
                        st4(out + (size_t)r * KS + c0, v[u]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) sum[j] = rs[j].total();
        }
    } else if (p.src.kind == SRC_RADEMACHER && !p.src.gaussian) {
        const RadQuad rq(p.src, t.seg, gc0);
        int neg[4] = {0, 0, 0, 0};
        const int rows = rad_rows<T, KS, true>(p, t, sg, rq, rsub, c0, out, neg);
#pragma unroll
        for (int j = 0; j < 4; j++) sum[j] = rq.live[j] ? (double)rows : 0.0;
    } else {
        RowSum<T> rs[4];
        for (int r = t.row_begin + rsub; r < t.row_end; r += RPP) {
            const int id = p.node_id ? __ldg(p.node_id + r) : r - sg.row_begin;
            T v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                v[j] = source_value_t<T, KS>(p.src, p.panel_src, r, id, gc0 + j, p.n_total, t.seg);
                rs[j].add(v[j] * v[j]);
            }
            st4(out + (size_t)r * KS + c0, v);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) sum[j] = rs[j].total();
    }
    cta_column_partials<KS>(sum, rsub, c0, p.part + ((size_t)panel * p.tiles_per_panel + tile) * KS);
    __shared__ double tot[KS];
    if (last_cta_reduce<KS>(p.part, p.counter + (size_t)panel * p.nseg + t.seg, panel, p.tiles_per_panel,
                            sg.tile_begin, sg.tile_count, tot)) {
        if (threadIdx.x < KS) {
            size_t o = (size_t)t.seg * p.K + panel * KS + threadIdx.x;
            double nrm2 = tot[threadIdx.x];
            p.norm2[o] = nrm2;
            p.sig1[o] = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// Served blocks: deflated start vectors (see kernels.h).  One CTA per listed
// tile; thread t handles block column t % 64 (and t % 64 + 64, ..) of the
// tile's rows t / 64, t / 64 + 4, ...; partials of the CTA are summed over
// its four row groups, and the last CTA of a segment adds the segment's
// tile partials in list order.

// The last-arriving CTA of segment s sums the W-value partials of its tiles
// (list entries tb .. tb + tc - 1) in order; true in that CTA, with the
// totals in out[0 .. W).
__device__ bool srv_last_reduce(const double* part, uint32_t* counter, int tb, int tc, int W, double* out) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == (unsigned)(tc - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < tc; i++) acc += ld_cg(&part[(size_t)(tb + i) * W + w]);
        out[w] = acc;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

template <typename T>
__device__ __forceinline__ T srv_probe(const SrvStartParams<T>& p, int s, int c, int r) {
    const uint64_t sd = p.seg_seed[s];
    const uint64_t col = (uint64_t)(p.seg_col0[s] + c);
    const uint64_t id = (uint64_t)p.node_id[r];
    return (T)(p.gaussian ? gaussian_entry(sd, col, id) : rademacher_entry(sd, col, id));
}

// pass 1: coef[s][i][c] = q_i . g_c over the segment's rows
template <typename T>
__global__ void __launch_bounds__(VNE_THREADS) k_srv_coef(SrvStartParams<T> p) {
    const RowTile t = p.tiles[p.tile_list[blockIdx.x]];
    const int s = t.seg, c0 = threadIdx.x % 64, rs = threadIdx.x / 64;
    __shared__ double red[VNE_THREADS / 64][4 * 256];
    for (int c = c0; c < p.K; c += 64) {
        // products in the vector precision, runs of 16 rows summed in FP64
        RowSum<T> acc[4];
        for (int r = t.row_begin + rs; r < t.row_end; r += VNE_THREADS / 64) {
            const T g = srv_probe(p, s, c, r);
#pragma unroll
            for (int i = 0; i < 4; i++) acc[i].add(p.q[(size_t)r * 4 + i] * g);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) red[rs][i * p.K + c] = acc[i].total();
    }
    __syncthreads();
    const int W = 4 * p.K;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < VNE_THREADS / 64; q++) v += red[q][w];
        p.part[(size_t)blockIdx.x * W + w] = v;
    }
    __shared__ double tot[4 * 256];
    if (srv_last_reduce(p.part, p.counter + s, p.seg_tb[s], p.seg_tc[s], W, tot))
        for (int w = threadIdx.x; w < W; w += blockDim.x) p.coef[(size_t)s * W + w] = tot[w];
}

// pass 2 (center = 0): column sums of g' = g - Q coef -> mean; pass 3
// (center = 1): c = g' - mean written to w1, ||c||^2 -> norm2, sigma_1
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_srv_pass(SrvStartParams<T> p, int center) {
    const RowTile t = p.tiles[p.tile_list[blockIdx.x]];
    const int s = t.seg, c0 = threadIdx.x % 64, rs = threadIdx.x / 64;
    __shared__ double red[VNE_THREADS / 64][256];
    for (int c = c0; c < p.K; c += 64) {
        T cf[4];
#pragma unroll
        for (int i = 0; i < 4; i++) cf[i] = (T)p.coef[((size_t)s * 4 + i) * p.K + c];
        const T mu = center ? (T)p.mean[(size_t)s * p.K + c] : (T)0;
        T* out = p.w1 + (size_t)(c / KS) * p.n_total * KS + (c % KS);
        RowSum<T> acc;
        for (int r = t.row_begin + rs; r < t.row_end; r += VNE_THREADS / 64) {
            T v = srv_probe(p, s, c, r);
#pragma unroll
            for (int i = 0; i < 4; i++) v -= p.q[(size_t)r * 4 + i] * cf[i];
            if (center) {
                v -= mu;
                out[(size_t)r * KS] = v;
                acc.add(v * v);
            } else {
                acc.add(v);
            }
        }
        red[rs][c] = acc.total();
    }
    __syncthreads();
    for (int w = threadIdx.x; w < p.K; w += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < VNE_THREADS / 64; q++) v += red[q][w];
        p.part[(size_t)blockIdx.x * p.K + w] = v;
    }
    __shared__ double tot[256];
    if (srv_last_reduce(p.part, p.counter + s, p.seg_tb[s], p.seg_tc[s], p.K, tot)) {
        for (int w = threadIdx.x; w < p.K; w += blockDim.x) {
            const size_t o = (size_t)s * p.K + w;
            if (center) {
                p.norm2[o] = tot[w];
                p.sig1[o] = tot[w] > 0.0 ? 1.0 / sqrt(tot[w]) : 0.0;
            } else {
                p.mean[o] = tot[w] / (double)p.seg[s].rows;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The per-step pointers of one segment: the launch's own (one step j for
// every segment), or, with per-segment step counters, those of the
// segment's step j_s (false: the segment is idle in this launch).
template <typename T>
struct StepView {
    const T* w_cur;
    const T* w_prev;
    T* w_next;
    const double* sig_cur;
    const double* sig_prev;
    const double* beta_prev;
    double* alpha;
    double* beta;
    double* sig_next;
    int first;
};

template <bool SEGJ, typename T>
__device__ __forceinline__ bool step_view(const StepParams<T>& p, int seg, StepView<T>& v) {
    if (!SEGJ) {
        v.w_cur = p.w_cur;
        v.w_prev = p.w_prev;
        v.w_next = p.w_next;
        v.sig_cur = p.sig_cur;
        v.sig_prev = p.sig_prev;
        v.beta_prev = p.beta_prev;
        v.alpha = p.alpha;
        v.beta = p.beta;
        v.sig_next = p.sig_next;
        v.first = p.first;
        return true;
    }
    const int j = p.segj[seg];
    if (j <= 0) return false;
    const size_t SK = (size_t)p.nseg * p.K;
    v.w_cur = ((j - 1) & 1) ? p.slot1 : p.slot0;
    v.w_prev = (j & 1) ? p.slot1 : p.slot0;
    v.w_next = (j & 1) ? p.slot1 : p.slot0;
    v.sig_cur = p.sigma0 + (size_t)(j - 1) * SK;
    v.sig_prev = j > 1 ? p.sigma0 + (size_t)(j - 2) * SK : p.sigma0;
    v.beta_prev = j > 1 ? p.beta0 + (size_t)(j - 2) * SK : p.beta0;
    v.alpha = p.alpha0 + (size_t)(j - 1) * SK;
    v.beta = p.beta0 + (size_t)(j - 1) * SK;
    v.sig_next = p.sigma0 + (size_t)j * SK;
    v.first = j == 1;
    return true;
}

// ---------------------------------------------------------------------------
// Step kernel: u = sigma_j M w_j - beta_{j-1} sigma_{j-1} w_{j-1},
// alpha_j = sigma_j (w_j . u).  One warp per work item.
// Variants (selected by the schedule autotuner): MINB = CTAs per SM the
// register allocation must allow, UNR = independent neighbour gathers in
// flight per row group, STREAM = write u with an evict-first hint, STAGE =
// copy the work item's column indices and row offsets into shared memory
// with coalesced loads first, so each gather waits on a shared-memory read
// instead of a dependent global index load (dynamic smem: item_nnz ints per
// warp + kStageRp row offsets per warp; a warp takes p.ipw items in turn, so
// a CTA covers VNE_WARPS * ipw items and its reduction tail is amortised over
// them), PTAIL = issue a row's last (fewer than
// UNR) gathers at once under predicates instead of one per latency round,
// and load the row's own entries of w_j and w_{j-1} before its gathers.
template <typename T, int KS, bool VALUED, int MINB, int UNR, bool STREAM, bool STAGE, int HINT = 0,
          bool PTAIL = false, bool SEGJ = false>
__global__ void __launch_bounds__(VNE_THREADS, MINB) k_step(StepParams<T> p) {
    constexpr int CPL = LaneVec<T>::CPL;
    constexpr int LPR = KS / CPL;  // lanes per row
    constexpr int G = 32 / LPR;    // row groups per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPR, sub = lane % LPR;
    const int panel = p.panel_base + blockIdx.x / p.ctas_per_panel, cta = blockIdx.x % p.ctas_per_panel;
    const int seg = p.cta_seg[cta];
    StepView<T> sv;
    if (!step_view<SEGJ>(p, seg, sv)) return;  // idle segment: every CTA of it returns here
    const size_t pofs = (size_t)panel * p.n_total * KS;
    const T* __restrict__ W = sv.w_cur + pofs;
    const T* __restrict__ Wp = sv.w_prev + pofs;
    T* __restrict__ U = p.u + pofs;
    const int cofs = sub * CPL;

    // per-column coefficients staged in shared memory (keeps registers for gathers)
    __shared__ T s_sig[KS], s_cp[KS];
    if (threadIdx.x < KS) {
        const size_t o = (size_t)seg * p.K + panel * KS + threadIdx.x;
        s_sig[threadIdx.x] = (T)sv.sig_cur[o];
        s_cp[threadIdx.x] = sv.first ? (T)0 : (T)(sv.beta_prev[o] * sv.sig_prev[o]);
    }
    __syncthreads();
    T dot[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) dot[q] = (T)0;
    const uint64_t pol = HINT ? policy_evict_last() : 0ull;

    auto epilogue_x = [&](int r, const T (&acc)[CPL], int deg, T (&dt)[CPL], const T (&x)[CPL],
                          const T (&xp)[CPL]) {
        T uu[CPL];
#pragma unroll
        for (int q = 0; q < CPL; q++) {
            T ax = VALUED ? acc[q] : ((T)deg * x[q] - acc[q]);
            T v = s_sig[cofs + q] * ax;
            if (!sv.first) v -= s_cp[cofs + q] * xp[q];
            uu[q] = v;
            dt[q] += x[q] * v;
        }
        if (STREAM) store_lane_stream(U + (size_t)r * KS + cofs, uu);
        else store_lane(U + (size_t)r * KS + cofs, uu);
    };
    auto epilogue = [&](int r, const T (&acc)[CPL], int deg, T (&dt)[CPL]) {
        T x[CPL], xp[CPL];
        load_lane(W + (size_t)r * KS + cofs, x);
        if (!sv.first) load_lane_stream(Wp + (size_t)r * KS + cofs, xp);
        epilogue_x(r, acc, deg, dt, x, xp);
    };

    extern __shared__ int32_t s_stage[];
    int32_t* s_col = s_stage + warp * (p.stage_nnz + kStageRp);
    int32_t* s_rp = s_col + p.stage_nnz;
    for (int ii = 0; ii < p.ipw; ii++) {
    const WorkItem it = p.items[((size_t)cta * p.ipw + ii) * VNE_WARPS + warp];
    int nb_item = it.nnz_begin;
    if (STAGE && ii > 0) __syncwarp();  // the previous item's reads of the staging are done
    if (STAGE && it.rows != 0) {
        const int cnt = it.nnz_end - it.nnz_begin;
        for (int i = lane; i < cnt; i += 32) s_col[i] = __ldcs(p.col + nb_item + i);
        if (it.rows > 0)
            for (int i = lane; i <= it.rows; i += 32) s_rp[i] = p.rowptr[it.row + i];
        __syncwarp();
    }
    auto colidx = [&](int k) -> int { return STAGE ? s_col[k - nb_item] : __ldg(p.col + k); };
    if (it.rows > 0) {
        for (int r = it.row + g; r < it.row + it.rows; r += G) {
            const int kb = STAGE ? s_rp[r - it.row] : p.rowptr[r];
            const int ke = STAGE ? s_rp[r - it.row + 1] : p.rowptr[r + 1];
            T x[CPL], xp[CPL];
            if (PTAIL) {  // the row's own entries, in flight while it gathers
                load_lane(W + (size_t)r * KS + cofs, x);
                if (!sv.first) load_lane_stream(Wp + (size_t)r * KS + cofs, xp);
            }
            T acc[CPL];
#pragma unroll
            for (int q = 0; q < CPL; q++) acc[q] = (T)0;
            int k = kb;
            for (; k + UNR <= ke; k += UNR) {
                int cc[UNR];
#pragma unroll
                for (int u = 0; u < UNR; u++) cc[u] = colidx(k + u);
                T a[UNR][CPL];
#pragma unroll
                for (int u = 0; u < UNR; u++) load_lane_hint<HINT>(W + (size_t)cc[u] * KS + cofs, a[u], pol);
                if (VALUED) {
                    T v[UNR];
#pragma unroll
                    for (int u = 0; u < UNR; u++) v[u] = __ldg(p.vals + k + u);
#pragma unroll
                    for (int u = 0; u < UNR; u++)
#pragma unroll
                        for (int q = 0; q < CPL; q++) acc[q] += v[u] * a[u][q];
                } else {
#pragma unroll
                    for (int u = 0; u < UNR; u += 2)
#pragma unroll
                        for (int q = 0; q < CPL; q++) acc[q] += a[u][q] + a[u + 1][q];
                }
            }
            if (PTAIL) {
                if (k < ke) {  // the last ke - k < UNR gathers, all in flight at once
                    T a[UNR][CPL];
#pragma unroll
                    for (int u = 0; u < UNR; u++) {
                        if (k + u < ke) {
                            load_lane_hint<HINT>(W + (size_t)colidx(k + u) * KS + cofs, a[u], pol);
                        } else {
#pragma unroll
                            for (int q = 0; q < CPL; q++) a[u][q] = (T)0;
                        }
                    }
                    if (VALUED) {
#pragma unroll
                        for (int u = 0; u < UNR; u++) {
                            const T v = (k + u < ke) ? __ldg(p.vals + k + u) : (T)0;
#pragma unroll
                            for (int q = 0; q < CPL; q++) acc[q] += v * a[u][q];
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < UNR; u += 2)
#pragma unroll
                            for (int q = 0; q < CPL; q++) acc[q] += a[u][q] + a[u + 1][q];
                    }
                }
                epilogue_x(r, acc, ke - kb, dot, x, xp);
            } else {
                for (; k < ke; k++) {
                    int c0 = colidx(k);
                    T a0[CPL];
                    load_lane_hint<HINT>(W + (size_t)c0 * KS + cofs, a0, pol);
                    T v0 = VALUED ? __ldg(p.vals + k) : (T)1;
#pragma unroll
                    for (int q = 0; q < CPL; q++) acc[q] += VALUED ? v0 * a0[q] : a0[q];
                }
                epilogue(r, acc, ke - kb, dot);
            }
        }
    } else if (it.rows < 0) {
        // one chunk of a long row, all groups of the warp share it
        const HubRow h = p.hubs[it.row];
        const int chunk = -it.rows - 1;
        T acc[CPL];
#pragma unroll
        for (int q = 0; q < CPL; q++) acc[q] = (T)0;
        for (int k = it.nnz_begin + g; k < it.nnz_end; k += G) {
            int c0 = colidx(k);
            T a0[CPL];
            load_lane_hint<HINT>(W + (size_t)c0 * KS + cofs, a0, pol);
            T v0 = VALUED ? __ldg(p.vals + k) : (T)1;
#pragma unroll
            for (int q = 0; q < CPL; q++) acc[q] += VALUED ? v0 * a0[q] : a0[q];
        }
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
            for (int q = 0; q < CPL; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        T* hp = p.hub_part + ((size_t)panel * p.hub_slots + h.slot) * KS;
        if (g == 0) store_lane(hp + (size_t)chunk * KS + cofs, acc);
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            unsigned old = atomicAdd(p.hub_cnt + (size_t)panel * p.nhubs + it.row, 1u);
            last = (old == (unsigned)(h.chunks - 1));
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            if (g == 0) {
                T tot[CPL], hd[CPL];
#pragma unroll
                for (int q = 0; q < CPL; q++) {
                    tot[q] = (T)0;
                    hd[q] = (T)0;
                }
                for (int c = 0; c < h.chunks; c++)
#pragma unroll
                    for (int q = 0; q < CPL; q++) tot[q] += ld_cg(hp + (size_t)c * KS + cofs + q);
                const int r = h.row;
                epilogue(r, tot, p.rowptr[r + 1] - p.rowptr[r], hd);
                // the long row's share of w_j . u goes to its own slot, summed
                // in hub order by the reducing CTA (independent of which CTA
                // finished the row)
#pragma unroll
                for (int q = 0; q < CPL; q++)
                    p.hub_dot[((size_t)panel * p.nhubs + it.row) * KS + cofs + q] = (double)hd[q];
            }
            if (lane == 0) p.hub_cnt[(size_t)panel * p.nhubs + it.row] = 0u;
        }
    }
    }  // work items of this warp

    // CTA partial of w_j . u per column: FP64 across groups, warps, CTAs
    __shared__ double sred[VNE_WARPS][KS];
    double d[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        d[q] = (double)dot[q];
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], off);
    }
    if (g == 0)
#pragma unroll
        for (int q = 0; q < CPL; q++) sred[warp][cofs + q] = d[q];
    __syncthreads();
    if (threadIdx.x < KS) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < VNE_WARPS; w++) s += sred[w][threadIdx.x];
        p.part[((size_t)panel * p.ctas_per_panel + cta) * KS + threadIdx.x] = s;
    }
    __shared__ double tot[KS];
    const SegInfo sg = p.seg[seg];
    if (last_cta_reduce<KS>(p.part, p.counter + (size_t)panel * p.nseg + seg, panel, p.ctas_per_panel,
                            sg.cta_begin, sg.cta_count, tot)) {
        // add the long rows' shares in a fixed order (strided over the CTA)
        __shared__ double hred[VNE_THREADS];
        constexpr int NS = VNE_THREADS / KS;
        const int c = threadIdx.x % KS, s = threadIdx.x / KS;
        double hacc = 0.0;
        for (int h = s; h < sg.hub_count; h += NS)
            hacc += ld_cg(&p.hub_dot[((size_t)panel * p.nhubs + sg.hub_begin + h) * KS + c]);
        hred[threadIdx.x] = hacc;
        __syncthreads();
        if (threadIdx.x < KS) {
            double t = tot[threadIdx.x];
            for (int q = 0; q < NS; q++) t += hred[q * KS + threadIdx.x];
            size_t o = (size_t)seg * p.K + panel * KS + threadIdx.x;
            sv.alpha[o] = sv.sig_cur[o] * t;
        }
    }
}

// ---------------------------------------------------------------------------
// Update kernel: w_{j+1} = u - alpha_j sigma_j w_j (or, with `renorm`, just
// the norm of w_{j+1} in place), beta_j = ||w_{j+1}||, sigma_{j+1} = 1/beta_j
// unless beta_j <= tau (breakdown: beta_j = sigma_{j+1} = 0, column done).
template <typename T, int KS, bool SEGJ = false>
__global__ void __launch_bounds__(VNE_THREADS) k_update(StepParams<T> p) {
    constexpr int CPL = LaneVec<T>::CPL;
    constexpr int LPR = KS / CPL;
    constexpr int RPI = VNE_THREADS / LPR;  // rows per iteration
    // panels in reverse order: the step kernel walked them forwards, so the
    // first panels updated are the ones it touched last (still partly in L2),
    // and the next step starts on the panel updated last
    const int np = gridDim.x / p.tiles_per_panel;
    const int panel = p.panel_base + (np - 1 - (int)(blockIdx.x / p.tiles_per_panel)),
              tile = blockIdx.x % p.tiles_per_panel;
    if (p.renorm && p.panel_active && !p.panel_active[panel]) return;  // nothing changed in this panel
    const RowTile t = p.tiles[tile];
    StepView<T> sv;
    if (!step_view<SEGJ>(p, t.seg, sv)) return;  // idle segment: every CTA of it returns here
    const int sub = threadIdx.x % LPR, rsub = threadIdx.x / LPR;
    const int cofs = sub * CPL;
    const size_t pofs = (size_t)panel * p.n_total * KS;
    const size_t so = (size_t)t.seg * p.K + panel * KS + cofs;
    T a[CPL], nrm[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        a[q] = p.renorm ? (T)0 : (T)(sv.alpha[so + q] * sv.sig_cur[so + q]);
        nrm[q] = (T)0;
    }
    const T* __restrict__ Uu = p.u + pofs;
    const T* __restrict__ W = sv.w_cur + pofs;
    T* __restrict__ Wn = sv.w_next + pofs;
    for (int r = t.row_begin + rsub; r < t.row_end; r += RPI) {
        T uu[CPL], x[CPL], wn[CPL];
        if (p.renorm) {
            load_lane(Wn + (size_t)r * KS + cofs, wn);
        } else {
            load_lane_stream(Uu + (size_t)r * KS + cofs, uu);
            load_lane(W + (size_t)r * KS + cofs, x);
#pragma unroll
            for (int q = 0; q < CPL; q++) wn[q] = uu[q] - a[q] * x[q];
            store_lane(Wn + (size_t)r * KS + cofs, wn);
        }
#pragma unroll
        for (int q = 0; q < CPL; q++) nrm[q] += wn[q] * wn[q];
    }
    __shared__ double red[VNE_THREADS / LPR][KS];
#pragma unroll
    for (int q = 0; q < CPL; q++) red[rsub][cofs + q] = (double)nrm[q];
    __syncthreads();
    if (threadIdx.x < KS) {
        double s = 0.0;
        for (int i = 0; i < RPI; i++) s += red[i][threadIdx.x];
        p.part[((size_t)panel * p.tiles_per_panel + tile) * KS + threadIdx.x] = s;
    }
    __shared__ double tot[KS];
    const SegInfo sg = p.seg[t.seg];
    if (last_cta_reduce<KS>(p.part, p.counter + (size_t)panel * p.nseg + t.seg, panel, p.tiles_per_panel,
                            sg.tile_begin, sg.tile_count, tot)) {
        if (threadIdx.x < KS) {
            size_t o = (size_t)t.seg * p.K + panel * KS + threadIdx.x;
            double b = sqrt(tot[threadIdx.x]);
            if (!(b > sg.tau) || sv.sig_cur[o] == 0.0) {
                sv.beta[o] = 0.0;
                sv.sig_next[o] = 0.0;
            } else {
                sv.beta[o] = b;
                sv.sig_next[o] = 1.0 / b;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Full reorthogonalisation (classical Gram-Schmidt pass) of w_{j+1} against
// v_i = sigma_i w_i, i = 1..j, all stored in consecutive slots.
// The passes stream a row tile of one panel, which is a contiguous run of
// (rows x KS) elements, in 16-byte chunks: thread t takes chunks t, t + 256,
// ..., all of them in the same column group (t mod KS/V, V elements a chunk).
// Pass A: coef_i = sigma_i^2 (w_i . w_{j+1}) for every (i, column).  Products
// are formed in the vector precision and summed in runs of 16 chunks before
// the FP64 sum (GB300 retires FP64 at a small fraction of the FP32 rate; a
// run keeps the FP32 error near 16 units of the run's magnitude).  With a
// selection, a (panel, i) whose columns all skip basis vector i does nothing:
// pass B sets its coefficients to zero without its partials.
constexpr int kReorthMaxJ = 136;  // basis vectors per pass (m <= 128 Lanczos steps)

template <typename T>
struct Chunk16 {
    static constexpr int V = 16 / (int)sizeof(T);
    T x[V];
};

template <typename T>
__device__ __forceinline__ Chunk16<T> load_chunk(const T* p) {
    Chunk16<T> c;
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        c.x[0] = v.x; c.x[1] = v.y; c.x[2] = v.z; c.x[3] = v.w;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        c.x[0] = v.x; c.x[1] = v.y;
    }
    return c;
}

template <typename T>
__device__ __forceinline__ void store_chunk(T* p, const Chunk16<T>& c) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(c.x[0], c.x[1], c.x[2], c.x[3]);
    else *reinterpret_cast<double2*>(p) = make_double2(c.x[0], c.x[1]);
}

template <typename T, int KS>
__device__ __forceinline__ bool reorth_panel_uses(const ReorthParams<T>& p, int panel, int i) {
    if (!p.sel) return true;
    const uint8_t* s = p.sel + (size_t)i * p.K + (size_t)panel * KS;
    int any = 0;
#pragma unroll
    for (int c = 0; c < KS; c++) any |= s[c];
    return any != 0;
}

template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_reorth_dots(ReorthParams<T> p) {
    constexpr int V = Chunk16<T>::V, G = KS / V;
    static_assert(KS % V == 0 && VNE_THREADS % G == 0, "chunk layout");
    // grid: panel * tiles * j ; each CTA: one tile, one i
    const int i = blockIdx.x % p.j;
    const int pt = blockIdx.x / p.j;
    const int panel = pt / p.tiles_per_panel, tile = pt % p.tiles_per_panel;
    if (p.panel_active && !p.panel_active[panel]) return;
    if (!reorth_panel_uses<T, KS>(p, panel, i)) return;
    const RowTile t = p.tiles[tile];
    const size_t base = (size_t)panel * p.n_total * KS + (size_t)t.row_begin * KS;
    const T* Wi = p.basis + (size_t)i * p.slot_stride + base;
    const T* Wn = p.w + base;
    const int nchunks = (t.row_end - t.row_begin) * G;
    const size_t opart = (((size_t)panel * p.j + i) * p.tiles_per_panel + tile) * KS;
    if constexpr (sizeof(T) == 8) {
        // FP64 inner products are bound by the FP64 pipe, so the partial sums
        // take as few FP64 additions as possible: each thread accumulates its
        // chunks directly (exact trip count: a predicated-off iteration would
        // still take FP64 issue slots), then 8 partials per (column,
        // sub-sum) and the 8 sub-sums per column are added in index order
        double acc[V];
#pragma unroll
        for (int e = 0; e < V; e++) acc[e] = 0.0;
#pragma unroll 4
        for (int q = threadIdx.x; q < nchunks; q += VNE_THREADS) {
            const Chunk16<T> a = load_chunk(Wi + (size_t)q * V), b = load_chunk(Wn + (size_t)q * V);
#pragma unroll
            for (int e = 0; e < V; e++) acc[e] += a.x[e] * b.x[e];
        }
        constexpr int PER = VNE_THREADS / G;  // partials per column
        constexpr int SUB = PER >= 8 ? 8 : PER;
        __shared__ double red[VNE_THREADS * V];
        __shared__ double sub[KS * SUB];
#pragma unroll
        for (int e = 0; e < V; e++) red[threadIdx.x * V + e] = acc[e];
        __syncthreads();
        if (threadIdx.x < KS * SUB) {
            const int c = threadIdx.x % KS, sidx = threadIdx.x / KS, g = c / V, e = c % V;
            double x = 0.0;
            for (int k = sidx; k < PER; k += SUB) x += red[(g + k * G) * V + e];
            sub[sidx * KS + c] = x;
        }
        __syncthreads();
        if (threadIdx.x < KS) {
            double x = 0.0;
#pragma unroll
            for (int k = 0; k < SUB; k++) x += sub[k * KS + threadIdx.x];
            p.part[opart + threadIdx.x] = x;
        }
    } else {
        double acc[V];
#pragma unroll
        for (int e = 0; e < V; e++) acc[e] = 0.0;
        for (int q0 = threadIdx.x; q0 < nchunks; q0 += 16 * VNE_THREADS) {
            T run[V];
#pragma unroll
            for (int e = 0; e < V; e++) run[e] = (T)0;
            // a fixed run of 16 with predicated tails (measured faster for FP32)
#pragma unroll 4
            for (int u = 0; u < 16; u++) {
                const int q = q0 + u * VNE_THREADS;
                if (q < nchunks) {
                    const Chunk16<T> a = load_chunk(Wi + (size_t)q * V), b = load_chunk(Wn + (size_t)q * V);
#pragma unroll
                    for (int e = 0; e < V; e++) run[e] += a.x[e] * b.x[e];
                }
            }
#pragma unroll
            for (int e = 0; e < V; e++) acc[e] += (double)run[e];
        }
        // lanes of one column group (lane mod G) combine by a fixed shuffle
        // tree, then the warps' sums are added in warp order
#pragma unroll
        for (int off = G; off < 32; off <<= 1)
#pragma unroll
            for (int e = 0; e < V; e++) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
        constexpr int NW = VNE_THREADS / 32;
        __shared__ double red[NW][KS];
        const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
        if (lane < G)
#pragma unroll
            for (int e = 0; e < V; e++) red[warp][lane * V + e] = acc[e];
        __syncthreads();
        if (threadIdx.x < KS) {
            double x = 0.0;
#pragma unroll
            for (int w = 0; w < NW; w++) x += red[w][threadIdx.x];
            p.part[opart + threadIdx.x] = x;
        }
    }
}

// Pass B: fixed-order sum of the tile partials -> coefficients.
template <int KS>
__global__ void k_reorth_coef(ReorthCoefParams p) {
    // one thread per (panel, i, c)
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int total = p.panels * p.j * KS;
    if (idx >= total) return;
    int c = idx % KS, i = (idx / KS) % p.j, panel = idx / (KS * p.j);
    int col = panel * KS + c;
    if ((p.panel_active && !p.panel_active[panel]) || (p.sel && !p.sel[(size_t)i * p.K + col])) {
        p.coef[(size_t)i * p.K + col] = 0.0;
        return;
    }
    double s = 0.0;
    for (int t = 0; t < p.tiles_per_panel; t++)
        s += p.part[(((size_t)panel * p.j + i) * p.tiles_per_panel + t) * KS + c];
    double sig = p.sig[(size_t)i * p.K + col];
    p.coef[(size_t)i * p.K + col] = sig * sig * s;
}

// Pass C: w_{j+1} -= sum_i coef_i w_i in the vector precision.  Warp 0 of each
// CTA lists the basis vectors with a nonzero coefficient in its panel (in
// index order, by ballots), their coefficients are staged in shared memory
// rounded to the vector precision, and only those vectors are read; a thread
// keeps four chunks in flight.
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_reorth_apply(ReorthParams<T> p) {
    constexpr int V = Chunk16<T>::V, G = KS / V, U = 4;
    static_assert(KS % V == 0 && VNE_THREADS % G == 0, "chunk layout");
    const int panel = blockIdx.x / p.tiles_per_panel, tile = blockIdx.x % p.tiles_per_panel;
    if (p.panel_active && !p.panel_active[panel]) return;
    __shared__ int16_t act[kReorthMaxJ];
    __shared__ T cf[kReorthMaxJ * KS];
    __shared__ int nact;
    const double* cp = p.coef + (size_t)panel * KS;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int count = 0;
        for (int b0 = 0; b0 < p.j; b0 += 32) {
            const int i = b0 + lane;
            int u = 0;
            if (i < p.j)
#pragma unroll 8
                for (int c = 0; c < KS; c++) u |= cp[(size_t)i * p.K + c] != 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, u);
            if (u) act[count + __popc(m & ((1u << lane) - 1u))] = (int16_t)i;
            count += __popc(m);
        }
        if (lane == 0) nact = count;
    }
    __syncthreads();
    const int na = nact;
    for (int x = threadIdx.x; x < na * KS; x += VNE_THREADS) cf[x] = (T)cp[(size_t)act[x / KS] * p.K + x % KS];
    __syncthreads();
    if (na == 0) return;
    const RowTile t = p.tiles[tile];
    const size_t base = (size_t)panel * p.n_total * KS + (size_t)t.row_begin * KS;
    T* Wn = p.w + base;
    const T* B = p.basis + base;
    const int nchunks = (t.row_end - t.row_begin) * G;
    const int g = threadIdx.x % G;
    if constexpr (sizeof(T) == 8) {
        // full groups of U chunks, then the remaining chunks one at a time (a
        // predicated-off FMA would still take an issue slot of the FP64 pipe)
        int q0 = threadIdx.x;
        for (; q0 + (U - 1) * VNE_THREADS < nchunks; q0 += U * VNE_THREADS) {
            Chunk16<T> v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = load_chunk(Wn + (size_t)(q0 + u * VNE_THREADS) * V);
#pragma unroll 2
            for (int k = 0; k < na; k++) {
                const T* bk = B + (size_t)act[k] * p.slot_stride;
                const T* c = cf + k * KS + g * V;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const Chunk16<T> b = load_chunk(bk + (size_t)(q0 + u * VNE_THREADS) * V);
#pragma unroll
                    for (int e = 0; e < V; e++) v[u].x[e] -= c[e] * b.x[e];
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) store_chunk(Wn + (size_t)(q0 + u * VNE_THREADS) * V, v[u]);
        }
        for (; q0 < nchunks; q0 += VNE_THREADS) {
            Chunk16<T> v = load_chunk(Wn + (size_t)q0 * V);
#pragma unroll 2
            for (int k = 0; k < na; k++) {
                const Chunk16<T> b = load_chunk(B + (size_t)act[k] * p.slot_stride + (size_t)q0 * V);
                const T* c = cf + k * KS + g * V;
#pragma unroll
                for (int e = 0; e < V; e++) v.x[e] -= c[e] * b.x[e];
            }
            store_chunk(Wn + (size_t)q0 * V, v);
        }
    } else {
        // groups of U chunks with predicated tails (measured faster for FP32)
        for (int q0 = threadIdx.x; q0 < nchunks; q0 += U * VNE_THREADS) {
            Chunk16<T> v[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int q = q0 + u * VNE_THREADS;
                if (q < nchunks) v[u] = load_chunk(Wn + (size_t)q * V);
            }
#pragma unroll 2
            for (int k = 0; k < na; k++) {
                const T* bk = B + (size_t)act[k] * p.slot_stride;
                const T* c = cf + k * KS + g * V;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int q = q0 + u * VNE_THREADS;
                    if (q < nchunks) {
                        const Chunk16<T> b = load_chunk(bk + (size_t)q * V);
#pragma unroll
                        for (int e = 0; e < V; e++) v[u].x[e] -= c[e] * b.x[e];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int q = q0 + u * VNE_THREADS;
                if (q < nchunks) store_chunk(Wn + (size_t)q * V, v[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Partial reorthogonalisation (Simon 1984): the loss of orthogonality
// omega_{j+1,k} ~ v_{j+1} . v_k, k = 1..j, follows from the alpha's and
// beta's alone,
//   beta_j omega_{j+1,k} = beta_k omega_{j,k+1} + (alpha_k - alpha_j) omega_{j,k}
//                          + beta_{k-1} omega_{j,k-1} - beta_{j-1} omega_{j-1,k} +- 2 eps ||M||,
// with omega_{j,j} = 1 and omega_{j+1,j} = eps.  Once max_{k<j} |omega_{j+1,k}|
// reaches sqrt(eps), w_{j+1} is orthogonalised against the v_k with
// |omega_{j+1,k}| >= eps^(3/4) (those estimates are reset to eps), and the
// next vector against the same set.  One thread per column; the rows
// omega_{j-1,.} and omega_{j,.} are rolled in place.
__device__ __forceinline__ int m2_row(int j) { return j & 1; }  // rolling buffer of omega_{j,.}

__global__ void k_pro_omega(ProParams p) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.SK) return;
    const int j = p.j, SK = p.SK;
    double* om_old = p.omega + (size_t)m2_row(j + 1) * (p.m + 2) * SK;  // omega_{j-1,.}, becomes omega_{j+1,.}
    const double* om = p.omega + (size_t)m2_row(j) * (p.m + 2) * SK;     // omega_{j,.}
    for (int k = 0; k <= j; k++) p.sel[(size_t)k * SK + c] = 0;
    const double bj = p.beta[(size_t)(j - 1) * SK + c];
    if (j == 1) {  // a new block: omega_{0,.} = 0, omega_{1,.} = e_1, no pending set
        double* om1 = p.omega + (size_t)(m2_row(1)) * (p.m + 2) * SK;
        for (int k = 0; k < p.m + 2; k++) {
            om_old[(size_t)k * SK + c] = 0.0;
            om1[(size_t)k * SK + c] = k == 1 ? 1.0 : 0.0;
        }
        p.pend[c] = 0;
    }
    if (!(bj > 0.0) || p.sig[(size_t)j * SK + c] == 0.0) {  // finished column: nothing to estimate
        p.pend[c] = 0;
        return;
    }
    const double aj = p.alpha[(size_t)(j - 1) * SK + c];
    const double bjm1 = j > 1 ? p.beta[(size_t)(j - 2) * SK + c] : 0.0;
    const double noise = 2.0 * p.eps * p.normM;
    // omega_{j+1,k} for k = 1..j-1 (1-based), written over omega_{j-1,k}
    // after it is read
    double om_jm1_prev = 0.0;  // omega_{j,k-1}
    double mx = 0.0;
    for (int k = 1; k <= j - 1; k++) {
        const double ok = (k == j) ? 1.0 : om[(size_t)k * SK + c];
        const double okp1 = (k + 1 == j) ? 1.0 : om[(size_t)(k + 1) * SK + c];
        double t = p.beta[(size_t)(k - 1) * SK + c] * okp1 + (p.alpha[(size_t)(k - 1) * SK + c] - aj) * ok -
                   bjm1 * om_old[(size_t)k * SK + c];
        if (k > 1) t += p.beta[(size_t)(k - 2) * SK + c] * om_jm1_prev;
        t += copysign(noise, t);
        const double v = t / bj;
        om_jm1_prev = ok;
        om_old[(size_t)k * SK + c] = v;
        mx = fmax(mx, fabs(v));
    }
    om_old[(size_t)j * SK + c] = p.eps;
    om_old[(size_t)(j + 1) * SK + c] = 1.0;
    const double sq = sqrt(p.eps), eta = pow(p.eps, 0.75);
    int any = 0;
    if (p.pend[c]) {  // the second vector of a pair: the previous step's set (k <= j - 1)
        p.pend[c] = 0;
        for (int k = 1; k <= j - 1; k++)
            if (p.pend_sel[(size_t)k * SK + c]) {
                p.sel[(size_t)(k - 1) * SK + c] = 1;
                om_old[(size_t)k * SK + c] = p.eps;
                any = 1;
            }
    } else if (j > 1 && mx >= sq) {
        for (int k = 1; k <= j; k++) {
            const int s = fabs(om_old[(size_t)k * SK + c]) >= eta;
            p.pend_sel[(size_t)k * SK + c] = (uint8_t)s;
            if (s) {
                p.sel[(size_t)(k - 1) * SK + c] = 1;
                om_old[(size_t)k * SK + c] = p.eps;
                any = 1;
            }
        }
        p.pend[c] = 1;
    }
    if (any) atomicOr(p.panel_active + (c % p.K) / p.ks, 1);
}

cudaError_t launch_pro_omega(const ProParams& p, cudaStream_t st) {
    k_pro_omega<<<(p.SK + 127) / 128, 128, 0, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lanczos matvec recovery (eq. rational-krylov-approximation-matvec):
// y = ||c|| V_m f(T_m) e1 = sum_j gamma_j w_j with gamma_j = ||c|| sigma_j z_j.
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_recover(RecoverParams<T> p) {
    constexpr int CPL = LaneVec<T>::CPL;
    constexpr int LPR = KS / CPL;
    constexpr int RPI = VNE_THREADS / LPR;
    const int panel = blockIdx.x / p.tiles_per_panel, tile = blockIdx.x % p.tiles_per_panel;
    const RowTile t = p.tiles[tile];
    const int sub = threadIdx.x % LPR, rsub = threadIdx.x / LPR;
    const int cofs = sub * CPL;
    extern __shared__ __align__(16) unsigned char s_raw[];
    T* s_gamma = reinterpret_cast<T*>(s_raw);  // [m][KS], converted once to the data precision
    for (int idx = threadIdx.x; idx < p.m * KS; idx += blockDim.x) {
        int j = idx / KS, c = idx % KS;
        s_gamma[idx] = (T)p.gamma[(size_t)j * p.K + panel * KS + c];
    }
    __syncthreads();
    const size_t pofs = (size_t)panel * p.n_total * KS;
    for (int r = t.row_begin + rsub; r < t.row_end; r += RPI) {
        T acc[CPL];
#pragma unroll
        for (int q = 0; q < CPL; q++) acc[q] = (T)0;
        const T* b = p.basis + pofs + (size_t)r * KS + cofs;
        int j = 0;
        // eight independent streaming loads in flight per thread
        for (; j + 8 <= p.m; j += 8) {
            T x[8][CPL];
#pragma unroll
            for (int u = 0; u < 8; u++) load_lane_stream(b + (size_t)(j + u) * p.slot_stride, x[u]);
#pragma unroll
            for (int u = 0; u < 8; u++)
#pragma unroll
                for (int q = 0; q < CPL; q++) acc[q] += s_gamma[(j + u) * KS + cofs + q] * x[u][q];
        }
        for (; j < p.m; j++) {
            T x[CPL];
            load_lane_stream(b + (size_t)j * p.slot_stride, x);
#pragma unroll
            for (int q = 0; q < CPL; q++) acc[q] += s_gamma[j * KS + cofs + q] * x[q];
        }
        store_lane(p.y + pofs + (size_t)r * KS + cofs, acc);
    }
}

// ---------------------------------------------------------------------------
// Plain SpMM Y = scale * M X for the kernel-level entry point (X, Y row-major
// [n][k] in the caller's numbering; perm maps packed rows to caller rows).
template <typename T, bool VALUED>
__global__ void k_spmm_plain(const int32_t* rowptr, const int32_t* col, const T* vals, int n, int k,
                             const int32_t* node_id, double scale, const T* X, T* Y) {
    int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (r >= n) return;
    int kb = rowptr[r], ke = rowptr[r + 1];
    int rid = node_id ? node_id[r] : r;
    for (int c = lane; c < k; c += 32) {
        double acc = 0.0;
        for (int e = kb; e < ke; e++) {
            int cc = col[e];
            int cid = node_id ? node_id[cc] : cc;
            double x = (double)X[(size_t)cid * k + c];
            acc += VALUED ? (double)vals[e] * x : -x;
        }
        if (!VALUED) acc += (double)(ke - kb) * (double)X[(size_t)rid * k + c];
        Y[(size_t)rid * k + c] = (T)(scale * acc);
    }
}

__global__ void k_rademacher_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, int fp64, void* out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    int64_t i = idx / k;
    int c = (int)(idx % k);
    double v = rademacher_entry(seed_mixed, (uint64_t)(col_begin + c), (uint64_t)i);
    if (fp64) ((double*)out)[idx] = v;
    else ((float*)out)[idx] = (float)v;
}

__global__ void k_gaussian_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, double* out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    out[idx] = gaussian_entry(seed_mixed, (uint64_t)(col_begin + (int)(idx % k)), (uint64_t)(idx / k));
}

// ---------------------------------------------------------------------------
// host-side launchers

template <typename T>
static int panel_width_ok(int ks) {
    if (sizeof(T) == 4) return ks == 8 || ks == 16 || ks == 32;
    return ks == 4 || ks == 8 || ks == 16;
}

#define VNE_DISPATCH_KS(T, ks, CALL)                                   \
    do {                                                               \
        if (sizeof(T) == 4) {                                          \
            if ((ks) == 8) { constexpr int KS = 8; CALL; }             \
            else if ((ks) == 16) { constexpr int KS = 16; CALL; }      \
            else if ((ks) == 32) { constexpr int KS = 32; CALL; }      \
            else return cudaErrorInvalidValue;                         \
        } else {                                                       \
            if ((ks) == 4) { constexpr int KS = 4; CALL; }             \
            else if ((ks) == 8) { constexpr int KS = 8; CALL; }        \
            else if ((ks) == 16) { constexpr int KS = 16; CALL; }      \
            else return cudaErrorInvalidValue;                         \
        }                                                              \
    } while (0)

template <typename T>
cudaError_t launch_start(const StartParams<T>& p, int ks, int panels, cudaStream_t st) {
    dim3 grid(panels * p.tiles_per_panel);
    if (p.desing) VNE_DISPATCH_KS(T, ks, (k_start_mean<T, KS><<<grid, VNE_THREADS, 0, st>>>(p)));
    VNE_DISPATCH_KS(T, ks, (k_start_center<T, KS><<<grid, VNE_THREADS, 0, st>>>(p)));
    return cudaGetLastError();
}

// Step-kernel variants: {MINB, UNR, STREAM, STAGE, HINT, PTAIL}.  FP64 uses variant 0 only.
#define VNE_STEP_VARIANTS(T, KS, VALUED, v, st, grid, p, smem)                                                   \
    switch (sizeof(T) == 8 ? 0 : (v)) {                                                                          \
        case 1: k_step<T, KS, VALUED, 6, 4, true, false><<<grid, VNE_THREADS, 0, st>>>(p); break;               \
        case 2: k_step<T, KS, VALUED, 6, 8, true, false><<<grid, VNE_THREADS, 0, st>>>(p); break;               \
        case 3: k_step<T, KS, VALUED, 8, 4, true, false><<<grid, VNE_THREADS, 0, st>>>(p); break;               \
        case 4: k_step<T, KS, VALUED, 6, 4, true, true><<<grid, VNE_THREADS, smem, st>>>(p); break;             \
        case 5: k_step<T, KS, VALUED, 4, 8, true, true><<<grid, VNE_THREADS, smem, st>>>(p); break;             \
        case 6: k_step<T, KS, VALUED, 6, 4, true, true, 1><<<grid, VNE_THREADS, smem, st>>>(p); break;          \
        case 7: k_step<T, KS, VALUED, 6, 4, true, true, 2><<<grid, VNE_THREADS, smem, st>>>(p); break;          \
        case 8: k_step<T, KS, VALUED, 6, 8, true, true, 0, true><<<grid, VNE_THREADS, smem, st>>>(p); break;    \
        case 9: k_step<T, KS, VALUED, 6, 4, true, true, 0, true><<<grid, VNE_THREADS, smem, st>>>(p); break;    \
        case 10: k_step<T, KS, VALUED, 4, 8, true, true, 0, true><<<grid, VNE_THREADS, smem, st>>>(p); break;   \
        case 11: k_step<T, KS, VALUED, 6, 8, true, false, 0, true><<<grid, VNE_THREADS, 0, st>>>(p); break;     \
        case 12: k_step<T, KS, VALUED, 5, 4, true, true, 0, true><<<grid, VNE_THREADS, smem, st>>>(p); break;   \
        case 13: k_step<T, KS, VALUED, 5, 8, true, true, 0, true><<<grid, VNE_THREADS, smem, st>>>(p); break;   \
        default: k_step<T, KS, VALUED, 4, 4, false, false><<<grid, VNE_THREADS, 0, st>>>(p); break;             \
    }

template <typename T>
cudaError_t launch_step(const StepParams<T>& p, int ks, int panels, bool valued, int variant, cudaStream_t st) {
    dim3 grid(panels * p.ctas_per_panel);
    const size_t smem = (size_t)VNE_WARPS * (p.stage_nnz + kStageRp) * sizeof(int32_t);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;  // items above 1024 nonzeros are not staged
    if (valued) VNE_DISPATCH_KS(T, ks, VNE_STEP_VARIANTS(T, KS, true, variant, st, grid, p, smem));
    else VNE_DISPATCH_KS(T, ks, VNE_STEP_VARIANTS(T, KS, false, variant, st, grid, p, smem));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const StepParams<T>& p, int ks, int panels, cudaStream_t st) {
    dim3 grid(panels * p.tiles_per_panel);
    VNE_DISPATCH_KS(T, ks, (k_update<T, KS><<<grid, VNE_THREADS, 0, st>>>(p)));
    return cudaGetLastError();
}

// One Lanczos step (step kernel, then update kernel) of a pattern operator
// with per-segment step counters (p.segj): segment s runs its step
// p.segj[s], idle segments (0) are skipped.  The step kernel is the
// predicated-tail staged variant with four CTAs per SM.
template <typename T>
cudaError_t launch_srv_start(const SrvStartParams<T>& p, int ks, cudaStream_t st) {
    if (p.ntiles == 0) return cudaSuccess;
    if (p.K < 1 || p.K > 64 || p.K % ks) return cudaErrorInvalidValue;
    k_srv_coef<T><<<p.ntiles, VNE_THREADS, 0, st>>>(p);
    VNE_DISPATCH_KS(T, ks, (k_srv_pass<T, KS><<<p.ntiles, VNE_THREADS, 0, st>>>(p, 0)));
    VNE_DISPATCH_KS(T, ks, (k_srv_pass<T, KS><<<p.ntiles, VNE_THREADS, 0, st>>>(p, 1)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_update_segj(const StepParams<T>& p, int ks, int panels, cudaStream_t st) {
    if (!p.segj) return cudaErrorInvalidValue;
    const size_t smem = (size_t)VNE_WARPS * (p.stage_nnz + kStageRp) * sizeof(int32_t);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    dim3 gs(panels * p.ctas_per_panel), gu(panels * p.tiles_per_panel);
    VNE_DISPATCH_KS(T, ks, (k_step<T, KS, false, 4, 8, true, true, 0, true, true><<<gs, VNE_THREADS, smem, st>>>(p)));
    VNE_DISPATCH_KS(T, ks, (k_update<T, KS, true><<<gu, VNE_THREADS, 0, st>>>(p)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reorth(const ReorthParams<T>& p, const ReorthCoefParams& c, int ks, cudaStream_t st) {
    if (p.j <= 0) return cudaSuccess;
    if (p.j > kReorthMaxJ) return cudaErrorInvalidValue;
    VNE_DISPATCH_KS(T, ks, (k_reorth_dots<T, KS><<<dim3(p.panels * p.tiles_per_panel * p.j), VNE_THREADS, 0, st>>>(p)));
    int total = c.panels * c.j * ks;
    VNE_DISPATCH_KS(T, ks, (k_reorth_coef<KS><<<dim3((total + 255) / 256), 256, 0, st>>>(c)));
    VNE_DISPATCH_KS(T, ks, (k_reorth_apply<T, KS><<<dim3(p.panels * p.tiles_per_panel), VNE_THREADS, 0, st>>>(p)));
    return cudaGetLastError();
}

// coef[i][col] = sig_i^2 (basis_i . w) per column, without the update pass
template <typename T>
cudaError_t launch_col_dots(const ReorthParams<T>& p, const ReorthCoefParams& c, int ks, cudaStream_t st) {
    if (p.j <= 0) return cudaSuccess;
    VNE_DISPATCH_KS(T, ks, (k_reorth_dots<T, KS><<<dim3(p.panels * p.tiles_per_panel * p.j), VNE_THREADS, 0, st>>>(p)));
    int total = c.panels * c.j * ks;
    VNE_DISPATCH_KS(T, ks, (k_reorth_coef<KS><<<dim3((total + 255) / 256), 256, 0, st>>>(c)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_recover(const RecoverParams<T>& p, int ks, int panels, cudaStream_t st) {
    size_t smem = (size_t)p.m * ks * sizeof(T);
    dim3 grid(panels * p.tiles_per_panel);
    VNE_DISPATCH_KS(T, ks, (k_recover<T, KS><<<grid, VNE_THREADS, smem, st>>>(p)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmm_plain(const int32_t* rowptr, const int32_t* col, const T* vals, int n, int k,
                              const int32_t* node_id, double scale, const T* X, T* Y, cudaStream_t st) {
    dim3 grid((n + 7) / 8);
    if (vals) k_spmm_plain<T, true><<<grid, 256, 0, st>>>(rowptr, col, vals, n, k, node_id, scale, X, Y);
    else k_spmm_plain<T, false><<<grid, 256, 0, st>>>(rowptr, col, vals, n, k, node_id, scale, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_rademacher_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, int fp64, void* out,
                                   cudaStream_t st) {
    int64_t total = n * (int64_t)k;
    if (total == 0) return cudaSuccess;
    k_rademacher_fill<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed_mixed, n, col_begin, k, fp64, out);
    return cudaGetLastError();
}

cudaError_t launch_gaussian_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, double* out, cudaStream_t st) {
    const int64_t total = n * (int64_t)k;
    if (total == 0) return cudaSuccess;
    k_gaussian_fill<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed_mixed, n, col_begin, k, out);
    return cudaGetLastError();
}

#define VNE_INST(T)                                                                                        \
    template cudaError_t launch_start<T>(const StartParams<T>&, int, int, cudaStream_t);                   \
    template cudaError_t launch_step<T>(const StepParams<T>&, int, int, bool, int, cudaStream_t);          \
    template cudaError_t launch_update<T>(const StepParams<T>&, int, int, cudaStream_t);                   \
    template cudaError_t launch_step_update_segj<T>(const StepParams<T>&, int, int, cudaStream_t);         \
    template cudaError_t launch_srv_start<T>(const SrvStartParams<T>&, int, cudaStream_t);                 \
    template cudaError_t launch_reorth<T>(const ReorthParams<T>&, const ReorthCoefParams&, int, cudaStream_t); \
    template cudaError_t launch_col_dots<T>(const ReorthParams<T>&, const ReorthCoefParams&, int, cudaStream_t); \
    template cudaError_t launch_recover<T>(const RecoverParams<T>&, int, int, cudaStream_t);               \
    template cudaError_t launch_spmm_plain<T>(const int32_t*, const int32_t*, const T*, int, int,          \
                                              const int32_t*, double, const T*, T*, cudaStream_t);
VNE_INST(float)
VNE_INST(double)

}  // namespace vne
