// Serving loop of libvne: continuous batching of entropy queries.
//
// A query asks for S(rho) of one graph to a relative accuracy eps.  The
// server answers with Hutch++ (Section 3.2, eq. Hutch++_formula) in an
// adaptive form: a fixed sketch of N_r = 4 columns when the query is
// admitted (Q = orth(f(A) Omega) and psi(q_i), computed for the query alone),
// then blocks of K deflated Hutchinson probes g' = (I - Q Q^T) g until
// 2.576 * stderr <= (eps / 2) * |estimate| (at least two blocks) or the
// probe cap; estimate = sum_i psi(q_i) + mean psi(g').  The adaptive
// algorithm the paper cites is not printed in it; this is the stated proxy.
// With a Krylov tolerance tau (Section 5.2 keeps the Krylov error of the
// adaptive estimator within half the requested accuracy), the Lanczos runs of
// a block -- the basis vectors' quadratic forms at admission, then each
// block of deflated probes -- stop together at the first multiple of
// check_every below m at which every column's Theorem 4.4 estimate is at most
// tau |psi| (lam_min half the column's smallest positive Ritz value, lam_max
// the Gershgorin bound).  The sketch f(A) Omega takes opt.sketch_steps steps
// (any sketch keeps Hutch++ unbiased; it sets only the variance removed).
//
// Device layout: an arena of fixed capacity (rows, nonzeros) holds the
// packed CSR of every admitted query and the Lanczos vectors of its current
// block (two slots and u, panel-major, K columns) at a row range that the
// query keeps from admission to completion; its CSR is copied there once.
// Per-query scalars live in segment slot s (0 .. max_active - 1) of
// [m][(max_active + 1) * K] arrays; segment max_active is never active.  The
// work tables of the packed operator (work items and their CTA-to-segment
// map, long-row chunks, row tiles) are device tables whose ranges a query
// takes at admission, first fit, its own schedule shifted to its arena rows
// and nonzeros; at completion its CTAs and tiles are handed to the idle
// segment and the ranges are freed.  No tick rebuilds the tables.
//
// A tick (vne_server_step) is one Lanczos step of every active query, each
// at its own step j: queries whose block starts get their deflated start
// vectors, one step and one update kernel run over all active segments with
// per-segment step counters, and the queries whose block ends get their
// Gauss quadratures and update their statistics.  Admission happens at every
// tick, FIFO, while a segment slot and arena space are free.  A query's
// numbers depend only on its own graph, seed and schedule, so they are the
// same whatever runs beside it.
#include "engine.h"

namespace {

__global__ void k_pack_rowptr(const int32_t* src, int n, int32_t e0, int32_t* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) dst[i] = src[i] + e0;
}
__global__ void k_pack_col(const int32_t* src, int64_t nnz, int32_t r0, int32_t* dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) dst[i] = src[i] + r0;
}
__global__ void k_pack_ids(const int32_t* perm, int n, int32_t* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = perm ? perm[i] : i;
}

// First-fit allocator of [begin, end) ranges of a fixed capacity.
struct Ranges {
    std::vector<std::pair<int64_t, int64_t>> free;  // sorted, disjoint
    void reset(int64_t cap) {
        free.clear();
        if (cap > 0) free.push_back({0, cap});
    }
    int64_t take(int64_t size) {
        for (size_t i = 0; i < free.size(); i++) {
            const int64_t b = free[i].first, e = free[i].second;
            if (e - b >= size) {
                if (e - b == size) free.erase(free.begin() + i);
                else free[i].first = b + size;
                return b;
            }
        }
        return -1;
    }
    void give(int64_t b, int64_t size) {
        auto it = std::lower_bound(free.begin(), free.end(), std::make_pair(b, (int64_t)0));
        it = free.insert(it, {b, b + size});
        const size_t i = it - free.begin();
        if (i + 1 < free.size() && free[i].second == free[i + 1].first) {
            free[i].second = free[i + 1].second;
            free.erase(free.begin() + i + 1);
        }
        if (i > 0 && free[i - 1].second == free[i].first) {
            free[i - 1].second = free[i].second;
            free.erase(free.begin() + i);
        }
    }
};

constexpr int kSketchCols = 4;  // N_r of the served Hutch++

// Device records with first-fit ranges; a table grows (keeping its
// contents, the new part filled with `fill`) when a range does not fit.
// `per` records per range unit.
template <typename R>
struct DevTable {
    R* d = nullptr;
    int64_t cap = 0;  // range units
    int per = 1;
    R fill{};
    Ranges free;
    int64_t take(vne_ctx* ctx, int64_t n) {
        if (n <= 0) return 0;
        int64_t b = free.take(n);
        if (b >= 0) return b;
        const int64_t ncap = std::max<int64_t>({2 * cap, cap + n, 1024});
        R* nd = nullptr;
        VNE_TRY_CUDA(ctx, dev_malloc((void**)&nd, (size_t)ncap * per * sizeof(R)));
        cudaError_t e = cap ? cudaMemcpyAsync(nd, d, (size_t)cap * per * sizeof(R), cudaMemcpyDeviceToDevice,
                                              ctx->stream)
                            : cudaSuccess;
        if (e == cudaSuccess) {
            const std::vector<R> tail((size_t)(ncap - cap) * per, fill);
            e = cudaMemcpyAsync(nd + (size_t)cap * per, tail.data(), tail.size() * sizeof(R),
                                cudaMemcpyHostToDevice, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            dev_free(nd);
            VNE_TRY_CUDA(ctx, e);
        }
        dev_free(d);
        d = nd;
        free.give(cap, ncap - cap);
        cap = ncap;
        return free.take(n);
    }
    void give(int64_t b, int64_t n) {
        if (n > 0) free.give(b, n);
    }
    void put(vne_ctx* ctx, int64_t b, const std::vector<R>& v) {
        if (!v.empty())
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d + (size_t)b * per, v.data(), v.size() * sizeof(R),
                                              cudaMemcpyHostToDevice, ctx->stream));
    }
};

}  // namespace

struct vne_server {
    vne_ctx* ctx = nullptr;
    vne_options opt;
    size_t budget = 0, used = 0;
    int max_active = 64, m = 40, K = 64, ks = 16, max_vectors = 8192;
    double quad_tol = 0.0;  // > 0: Krylov tolerance; < 0: half of each query's accuracy; 0: m steps
    int check = 5, grid = 256;  // Theorem 4.4 estimate over 256 geometric + 256 linear points
    int precision = -1;  // -1 not yet known, 0 FP32, 1 FP64 (all queries share it)
    // arena
    int64_t rows_cap = 0, nnz_cap = 0;
    Ranges rows, nnz;
    int32_t *a_rowptr = nullptr, *a_col = nullptr, *a_nid = nullptr;
    void *slot0 = nullptr, *slot1 = nullptr, *u = nullptr, *q = nullptr;
    double *alpha = nullptr, *beta = nullptr, *sigma = nullptr, *norm2 = nullptr, *mean = nullptr, *psi = nullptr,
           *coef = nullptr, *scale = nullptr, *est = nullptr;
    std::vector<void*> owned;
    // segment slots (segment max_active: the idle one)
    int nseg = 65;
    std::vector<int> slot_req;  // request index, -1 free
    Problem P;                  // packed operator of the active set (tables below, not owned by P)
    DevTable<WorkItem> items;   // range unit: one CTA (VNE_WARPS items)
    DevTable<int32_t> cta_seg;  // range unit: one CTA
    DevTable<HubRow> hubs;
    DevTable<RowTile> tiles;
    Ranges hub_slots;           // partial-sum slots of the long-row chunks
    int64_t hub_slot_cap = 0;
    SegInfo* d_segs = nullptr;
    cudaEvent_t stage_ev = nullptr;  // recorded after each tick's staging copy
    char* pin = nullptr;             // pinned staging of a tick's host arrays
    size_t pin_cap = 0;
    struct Req {
        vne_matrix* M;
        double eps;
        uint64_t seed, seed_mixed;
        int max_vectors;
        int state;  // 0 queued, 1 active, 2 done
        int slot = -1;
        int64_t r0 = -1, e0 = -1;
        int j = 0;  // Lanczos step of the current block, 0 = the block has not started
        int blocks = 0;
        int64_t nvec = 0;
        double mean = 0.0, m2 = 0.0, low = 0.0, est = 0.0, se = 0.0;
        double tau = 0.0, lam_max = 0.0;  // Krylov tolerance (0: m steps), Gershgorin bound of A
        int rank = 0;
        size_t footprint = 0;
        // ranges of the work tables: CTAs, long rows, their slots, tiles
        int64_t cta_b = 0, cta_n = 0, hub_b = 0, hub_n = 0, hs_b = 0, hs_n = 0, tile_b = 0, tile_n = 0;
        int64_t submit_tick = 0, admit_tick = -1, done_tick = -1;
    };
    std::vector<Req> reqs;
    std::vector<int> pending;  // FIFO (front = pend_head)
    size_t pend_head = 0;
    std::vector<int> active;
    int64_t tick = 0;
    ~vne_server() {
        for (void* p : owned) dev_free(p);
        dev_free(items.d);
        dev_free(cta_seg.d);
        dev_free(hubs.d);
        dev_free(tiles.d);
        dev_free(d_segs);
        if (stage_ev) cudaEventDestroy(stage_ev);
        pinned_free(pin);
    }
};

namespace {

size_t row_bytes(const vne_server* S, size_t es) {
    // CSR offsets and node ids, two vector slots and u, the deflation basis
    return 8 + 3 * (size_t)S->K * es + kSketchCols * es;
}

// Allocate the arena for the precision of the first query.
void arena_alloc(vne_server* S, bool fp64) {
    vne_ctx* ctx = S->ctx;
    const size_t es = fp64 ? 8 : 4;
    S->nseg = S->max_active + 1;
    const int SK = S->nseg * S->K;
    const size_t fixed = (size_t)(3 * S->m + 8 + 4 + 3) * SK * 8 + ((size_t)1 << 20);
    VNE_REQUIRE(ctx, S->budget > fixed, VNE_ENOMEM, "HBM budget %zu too small for the server's scalars", S->budget);
    // rows and nonzeros share the budget: up to 12 nonzeros per row
    const size_t per_row = row_bytes(S, es) + 12 * 4;
    S->rows_cap = (int64_t)std::min<size_t>((S->budget - fixed) / per_row, (size_t)INT32_MAX - 1);
    S->nnz_cap = std::min<int64_t>(12 * S->rows_cap, INT32_MAX - 1);
    auto take = [&](size_t bytes) {
        void* p = nullptr;
        VNE_TRY_CUDA(ctx, dev_malloc(&p, std::max<size_t>(bytes, 256)));
        S->owned.push_back(p);
        return p;
    };
    S->a_rowptr = (int32_t*)take((S->rows_cap + 1) * 4);
    S->a_col = (int32_t*)take(std::max<int64_t>(S->nnz_cap, 1) * 4);
    S->a_nid = (int32_t*)take(S->rows_cap * 4);
    S->slot0 = take((size_t)S->rows_cap * S->K * es);
    S->slot1 = take((size_t)S->rows_cap * S->K * es);
    S->u = take((size_t)S->rows_cap * S->K * es);
    S->q = take((size_t)S->rows_cap * kSketchCols * es);
    S->alpha = (double*)take((size_t)S->m * SK * 8);
    S->beta = (double*)take((size_t)S->m * SK * 8);
    S->sigma = (double*)take((size_t)(S->m + 1) * SK * 8);
    S->norm2 = (double*)take((size_t)SK * 8);
    S->mean = (double*)take((size_t)SK * 8);
    S->psi = (double*)take((size_t)SK * 8);
    S->est = (double*)take((size_t)3 * SK * 8);
    S->scale = (double*)take((size_t)SK * 8);
    S->coef = (double*)take((size_t)kSketchCols * SK * 8);
    if (fp64 && S->ks > 16) {  // FP64 panels hold 4, 8 or 16 columns
        S->ks = 16;
        S->K = ((S->K + 15) / 16) * 16;
    }
    S->rows.reset(S->rows_cap);
    S->nnz.reset(S->nnz_cap);
    S->slot_req.assign(S->max_active, -1);
    S->precision = fp64 ? 1 : 0;
    // the packed operator: the arena, and tables filled per query
    Problem& P = S->P;
    P.owns_tables = false;
    P.fp64 = fp64;
    P.valued = false;
    P.ipw = 1;
    P.n_total = (int32_t)S->rows_cap;
    P.nnz_total = S->nnz_cap;
    P.nseg = S->nseg;
    P.rowptr = S->a_rowptr;
    P.col = S->a_col;
    P.node_id = S->a_nid;
    P.vals = nullptr;
    P.stage_nnz = 1;
    P.segs.assign(S->nseg, SegInfo{});
    S->items.per = VNE_WARPS;
    // never-used parts of the tables: empty items, CTAs and tiles of the idle segment
    S->items.fill = WorkItem{0, 0, 0, 0};
    S->cta_seg.fill = S->max_active;
    S->tiles.fill = RowTile{0, 0, S->max_active, 0};
    S->hubs.fill = HubRow{0, 0, 0, S->max_active};
    VNE_TRY_CUDA(ctx, dev_malloc((void**)&S->d_segs, (size_t)S->nseg * sizeof(SegInfo)));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(S->d_segs, P.segs.data(), (size_t)S->nseg * sizeof(SegInfo),
                                      cudaMemcpyHostToDevice, ctx->stream));
}

// Place a query's schedule in the work tables: its CTAs, long rows, their
// partial-sum slots and row tiles get ranges of their own (first fit), its
// items and tiles shifted to its arena rows and nonzeros and mapped to its
// segment slot s.
void place_tables(vne_server* S, vne_server::Req& rq, int s) {
    vne_ctx* ctx = S->ctx;
    Problem& P = S->P;
    Problem* MP = matrix_problem(rq.M, &S->opt);
    rq.cta_n = (int64_t)(MP->items.size() / VNE_WARPS);
    rq.hub_n = (int64_t)MP->hubs.size();
    rq.hs_n = MP->hub_slots;
    rq.tile_n = (int64_t)MP->tiles.size();
    rq.cta_b = S->items.take(ctx, rq.cta_n);
    if (S->cta_seg.take(ctx, rq.cta_n) != rq.cta_b)  // the two CTA tables share their ranges
        VNE_REQUIRE(ctx, false, VNE_EDEVICE, "server CTA tables out of step");
    rq.hub_b = S->hubs.take(ctx, rq.hub_n);
    rq.tile_b = S->tiles.take(ctx, rq.tile_n);
    rq.hs_b = 0;
    if (rq.hs_n > 0) {
        rq.hs_b = S->hub_slots.take(rq.hs_n);
        if (rq.hs_b < 0) {  // grow the slot space
            const int64_t grow = std::max<int64_t>(rq.hs_n, S->hub_slot_cap + 1024);
            S->hub_slots.give(S->hub_slot_cap, grow);
            S->hub_slot_cap += grow;
            rq.hs_b = S->hub_slots.take(rq.hs_n);
        }
    }
    const int32_t r0 = (int32_t)rq.r0, e0 = (int32_t)rq.e0, hb = (int32_t)rq.hub_b;
    std::vector<WorkItem> it = MP->items;
    for (WorkItem& w : it) {
        if (w.rows > 0) w.row += r0;
        else if (w.rows < 0) w.row += hb;
        if (w.rows != 0) {
            w.nnz_begin += e0;
            w.nnz_end += e0;
        }
    }
    std::vector<HubRow> hubs = MP->hubs;
    for (HubRow& h : hubs) {
        h.row += r0;
        h.slot += (int32_t)rq.hs_b;
        h.seg = s;
    }
    std::vector<RowTile> tiles = MP->tiles;
    for (RowTile& t : tiles) {
        t.row_begin += r0;
        t.row_end += r0;
        t.seg = s;
    }
    S->items.put(ctx, rq.cta_b, it);
    S->cta_seg.put(ctx, rq.cta_b, std::vector<int32_t>((size_t)rq.cta_n, s));
    S->hubs.put(ctx, rq.hub_b, hubs);
    S->tiles.put(ctx, rq.tile_b, tiles);
    SegInfo sg = MP->segs[0];
    sg.row_begin = r0;
    sg.cta_begin = (int32_t)rq.cta_b;
    sg.cta_count = (int32_t)rq.cta_n;
    sg.tile_begin = (int32_t)rq.tile_b;
    sg.hub_begin = hb;
    P.segs[s] = sg;
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(S->d_segs + s, &P.segs[s], sizeof(SegInfo), cudaMemcpyHostToDevice,
                                      ctx->stream));
    std::vector<double> hscale((size_t)S->K, sg.scale);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(S->scale + (size_t)s * S->K, hscale.data(), hscale.size() * 8,
                                      cudaMemcpyHostToDevice, ctx->stream));
    P.stage_nnz = std::max(P.stage_nnz, MP->stage_nnz);
}

// Hand a finished query's CTAs and tiles to the idle segment and free its
// ranges (its items and long rows are no longer reachable).
void clear_tables(vne_server* S, vne_server::Req& rq) {
    vne_ctx* ctx = S->ctx;
    const int32_t idle = S->max_active;
    S->cta_seg.put(ctx, rq.cta_b, std::vector<int32_t>((size_t)rq.cta_n, idle));
    S->tiles.put(ctx, rq.tile_b, std::vector<RowTile>((size_t)rq.tile_n, RowTile{0, 0, idle, 0}));
    S->P.segs[rq.slot] = SegInfo{};
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(S->d_segs + rq.slot, &S->P.segs[rq.slot], sizeof(SegInfo),
                                      cudaMemcpyHostToDevice, ctx->stream));
    S->items.give(rq.cta_b, rq.cta_n);
    S->cta_seg.give(rq.cta_b, rq.cta_n);
    S->hubs.give(rq.hub_b, rq.hub_n);
    S->tiles.give(rq.tile_b, rq.tile_n);
    if (rq.hs_n > 0) S->hub_slots.give(rq.hs_b, rq.hs_n);
}

// Admit the query at the head of the queue if a slot and arena space are
// free: copy its CSR into the arena and compute its deflation basis.
template <typename T>
bool admit_one(vne_server* S, int ri) {
    vne_ctx* ctx = S->ctx;
    cudaStream_t st = ctx->stream;
    vne_server::Req& rq = S->reqs[ri];
    vne_matrix* M = rq.M;
    int s = -1;
    for (int i = 0; i < S->max_active && s < 0; i++)
        if (S->slot_req[i] < 0) s = i;
    if (s < 0) return false;
    const int64_t r0 = S->rows.take(M->n + 1);  // one spare row holds the end offset
    if (r0 < 0) return false;
    const int64_t e0 = S->nnz.take(std::max<int64_t>(M->nnz, 1));
    if (e0 < 0) {
        S->rows.give(r0, M->n + 1);
        return false;
    }
    const int n = (int)M->n;
    k_pack_rowptr<<<(n + 256) / 256, 256, 0, st>>>(M->d_rowptr, n, (int32_t)e0, S->a_rowptr + r0);
    if (M->nnz) k_pack_col<<<(unsigned)((M->nnz + 255) / 256), 256, 0, st>>>(M->d_col, M->nnz, (int32_t)r0, S->a_col + e0);
    k_pack_ids<<<(n + 255) / 256, 256, 0, st>>>(M->d_node_id, n, S->a_nid + r0);
    VNE_TRY_CUDA(ctx, cudaGetLastError());
    ctx->launches += 3;
    std::vector<double> psi_q;
    int rank = 0;
    vne_options o = S->opt;
    o.probe_offset = 0;
    o.panel = sizeof(T) == 4 ? 8 : 4;  // the narrowest panel holding the 4 sketch columns
    Adaptive ad;  // the Krylov rule of the blocks, on the basis vectors' quadratic forms
    ad.tol = rq.tau;
    ad.check = S->check;
    ad.lam_min = 0.0;
    ad.lam_max = rq.lam_max;
    ad.grid = S->grid;
    const int ms = S->opt.sketch_steps > 0 ? std::min(S->opt.sketch_steps, S->m) : S->m;
    hutchpp_deflation<T>(M, &o, kSketchCols, S->m, ms, rq.seed, (T*)S->q + r0 * kSketchCols, psi_q, rank,
                         rq.tau > 0.0 ? &ad : nullptr);
    rq.low = 0.0;
    for (int i = 0; i < rank; i++) rq.low += psi_q[i];
    rq.rank = rank;
    rq.slot = s;
    rq.r0 = r0;
    rq.e0 = e0;
    place_tables(S, rq, s);
    rq.j = 0;
    rq.state = 1;
    rq.admit_tick = S->tick;
    S->slot_req[s] = ri;
    S->used += rq.footprint;
    S->active.push_back(ri);
    return true;
}

void release(vne_server* S, vne_server::Req& rq) {
    clear_tables(S, rq);
    S->rows.give(rq.r0, rq.M->n + 1);
    S->nnz.give(rq.e0, std::max<int64_t>(rq.M->nnz, 1));
    S->slot_req[rq.slot] = -1;
    S->used -= rq.footprint;
}

template <typename T>
int tick_impl(vne_server* S) {
    vne_ctx* ctx = S->ctx;
    cudaStream_t st = ctx->stream;
    // admission, FIFO
    while (S->pend_head < S->pending.size() && (int)S->active.size() < S->max_active) {
        const int ri = S->pending[S->pend_head];
        if (S->used + S->reqs[ri].footprint > S->budget) break;
        if (!admit_one<T>(S, ri)) break;
        S->pend_head++;
    }
    S->tick++;
    if (S->active.empty()) return 0;
    Problem& P = S->P;
    P.d_segs = S->d_segs;
    P.d_items = S->items.d;
    P.d_cta_seg = S->cta_seg.d;
    P.d_hubs = S->hubs.d;
    P.d_tiles = S->tiles.d;
    // the tables' extent: the ends of the ranges in use
    int64_t cta_high = 0, tile_high = 0, hub_high = 0, slot_high = 0;
    for (int ri : S->active) {
        const vne_server::Req& rq = S->reqs[ri];
        cta_high = std::max(cta_high, rq.cta_b + rq.cta_n);
        tile_high = std::max(tile_high, rq.tile_b + rq.tile_n);
        hub_high = std::max(hub_high, rq.hub_b + rq.hub_n);
        slot_high = std::max(slot_high, rq.hs_b + rq.hs_n);
    }
    const int K = S->K, SK = S->nseg * K, ks = S->ks, panels = K / ks;
    // Every host array of the tick's launches is known before the first of
    // them; they go to the device in one asynchronous copy from one pinned
    // buffer (a copy from pageable memory would synchronise the stream).
    // blocks that start now: deflated start vectors
    std::vector<int32_t> tlist, tb(S->nseg, 0), tc(S->nseg, 0), col0(S->nseg, 0);
    std::vector<uint64_t> seeds(S->nseg, 0);
    for (int ri : S->active) {
        vne_server::Req& rq = S->reqs[ri];
        const SegInfo& sg = P.segs[rq.slot];
        seeds[rq.slot] = rq.seed_mixed;
        if (rq.j != 0) continue;
        tb[rq.slot] = (int32_t)tlist.size();
        tc[rq.slot] = sg.tile_count;
        col0[rq.slot] = kSketchCols + rq.blocks * K;
        for (int t = 0; t < sg.tile_count; t++) tlist.push_back(sg.tile_begin + t);
        rq.j = 1;
    }
    // one Lanczos step of every active segment, each at its own step
    std::vector<int32_t> segj(S->nseg, 0);  // the idle segment max_active stays 0
    for (int ri : S->active) segj[S->reqs[ri].slot] = S->reqs[ri].j;
    // blocks that end after this step (step m) or check their Krylov error (a
    // multiple of check_every below m, with a tolerance).  A check needs
    // every column's Theorem 4.4 estimate within tau |psi|; it is evaluated
    // on the first kFirst columns of each checking query, and on the others
    // only for the queries whose first columns all pass (the same decision,
    // without the FP64 work of estimates that cannot change it)
    std::vector<int> ending, checking;
    for (int ri : S->active) {
        const vne_server::Req& rq = S->reqs[ri];
        if (rq.j == S->m) ending.push_back(ri);
        else if (rq.tau > 0.0 && rq.j % S->check == 0) checking.push_back(ri);
    }
    const int kFirst = std::min(K, 8);
    struct Lists {
        std::vector<int32_t> qcols, qm, bcols, bm;
        std::vector<double> blam;
    };
    auto make_lists = [&](const std::vector<int>& quad_all, const std::vector<int>& est_q, int c_begin, int c_end) {
        // quadratures of all columns of quad_all, quadratures and estimates
        // of columns [c_begin, c_end) of est_q
        Lists L;
        for (int ri : quad_all) {
            const vne_server::Req& rq = S->reqs[ri];
            for (int c = 0; c < K; c++) {
                L.qcols.push_back(rq.slot * K + c);
                L.qm.push_back(rq.j);
            }
        }
        for (int ri : est_q) {
            const vne_server::Req& rq = S->reqs[ri];
            for (int c = c_begin; c < c_end; c++) {
                L.qcols.push_back(rq.slot * K + c);
                L.qm.push_back(rq.j);
                L.bcols.push_back(rq.slot * K + c);
                L.bm.push_back(rq.j);
                L.blam.push_back(rq.lam_max);
            }
        }
        return L;
    };
    Lists LA = make_lists(ending, checking, 0, kFirst);
    // the staging copy (after the previous tick's copy has read the buffer)
    struct Part {
        const void* src;
        size_t bytes, off;
    };
    std::vector<Part> parts;
    size_t total = 0;
    auto add = [&](const void* src, size_t bytes) {
        const size_t off = (total + 15) & ~(size_t)15;
        parts.push_back({src, bytes, off});
        total = off + std::max<size_t>(bytes, 16);
        return parts.size() - 1;
    };
    const size_t i_tl = add(tlist.data(), tlist.size() * 4), i_tb = add(tb.data(), tb.size() * 4),
                 i_tc = add(tc.data(), tc.size() * 4), i_sd = add(seeds.data(), seeds.size() * 8),
                 i_c0 = add(col0.data(), col0.size() * 4), i_sj = add(segj.data(), segj.size() * 4),
                 i_qc = add(LA.qcols.data(), LA.qcols.size() * 4), i_qm = add(LA.qm.data(), LA.qm.size() * 4),
                 i_bc = add(LA.bcols.data(), LA.bcols.size() * 4), i_bm = add(LA.bm.data(), LA.bm.size() * 4),
                 i_bl = add(LA.blam.data(), LA.blam.size() * 8);
    if (S->stage_ev) VNE_TRY_CUDA(ctx, cudaEventSynchronize(S->stage_ev));
    if (S->pin_cap < total) {
        pinned_free(S->pin);
        S->pin = nullptr;
        S->pin_cap = 0;
        VNE_TRY_CUDA(ctx, pinned_malloc((void**)&S->pin, 2 * total));
        S->pin_cap = 2 * total;
    }
    char* pin = S->pin;
    for (const Part& q : parts)
        if (q.bytes) memcpy(pin + q.off, q.src, q.bytes);
    char* dstage = (char*)ws_get(ctx, "srv.stage", total);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(dstage, pin, total, cudaMemcpyHostToDevice, st));
    if (!S->stage_ev) VNE_TRY_CUDA(ctx, cudaEventCreateWithFlags(&S->stage_ev, cudaEventDisableTiming));
    VNE_TRY_CUDA(ctx, cudaEventRecord(S->stage_ev, st));
    auto dptr = [&](size_t i) { return (void*)(dstage + parts[i].off); };
    if (!tlist.empty()) {
        SrvStartParams<T> sp{};
        sp.tile_list = (const int32_t*)dptr(i_tl);
        sp.tiles = P.d_tiles;
        sp.seg = P.d_segs;
        sp.seg_tb = (const int32_t*)dptr(i_tb);
        sp.seg_tc = (const int32_t*)dptr(i_tc);
        sp.node_id = P.node_id;
        sp.seg_seed = (const uint64_t*)dptr(i_sd);
        sp.seg_col0 = (const int32_t*)dptr(i_c0);
        sp.q = (const T*)S->q;
        sp.coef = S->coef;
        sp.mean = S->mean;
        sp.norm2 = S->norm2;
        sp.sig1 = S->sigma;
        sp.w1 = (T*)S->slot0;
        sp.part = ws_get_t<double>(ctx, "srv.part", tlist.size() * kSketchCols * K);
        sp.counter = ws_get_t<uint32_t>(ctx, "srv.counter", S->nseg);
        sp.ntiles = (int32_t)tlist.size();
        sp.K = K;
        sp.n_total = P.n_total;
        sp.gaussian = S->opt.gaussian_probes != 0;
        VNE_TRY_CUDA(ctx, launch_srv_start<T>(sp, ks, st));
        ctx->launches += 3;
    }
    StepParams<T> p;
    memset(&p, 0, sizeof(p));
    p.rowptr = P.rowptr;
    p.col = P.col;
    p.n_total = P.n_total;
    p.K = K;
    p.nseg = P.nseg;
    p.seg = P.d_segs;
    p.items = P.d_items;
    p.ctas_per_panel = (int32_t)cta_high;
    p.cta_seg = P.d_cta_seg;
    p.hubs = P.d_hubs;
    p.nhubs = (int32_t)std::max<int64_t>(hub_high, 1);
    p.hub_slots = (int32_t)std::max<int64_t>(slot_high, 1);
    p.hub_part = ws_get_t<T>(ctx, "srv.hub_part", (size_t)panels * p.hub_slots * ks);
    p.hub_cnt = ws_get_t<uint32_t>(ctx, "srv.hub_cnt", (size_t)panels * p.nhubs);
    p.hub_dot = ws_get_t<double>(ctx, "srv.hub_dot", (size_t)panels * p.nhubs * ks);
    p.stage_nnz = std::max(P.stage_nnz, 1);
    p.ipw = 1;
    p.tiles = P.d_tiles;
    p.tiles_per_panel = (int32_t)tile_high;
    p.u = (T*)S->u;
    p.part = ws_get_t<double>(ctx, "srv.step_part", (size_t)panels * std::max(cta_high, tile_high) * ks);
    p.counter = ws_get_t<uint32_t>(ctx, "srv.step_counter", (size_t)panels * P.nseg);
    p.segj = (const int32_t*)dptr(i_sj);
    p.slot0 = (T*)S->slot0;
    p.slot1 = (T*)S->slot1;
    p.alpha0 = S->alpha;
    p.beta0 = S->beta;
    p.sigma0 = S->sigma;
    if (cta_high > 0) {
        VNE_TRY_CUDA(ctx, launch_step_update_segj<T>(p, ks, panels, st));
        ctx->launches += 2;
    }
    std::vector<double> hp, he;
    auto evaluate = [&](const Lists& L, const int32_t* qc, const int32_t* qm, const int32_t* bc, const int32_t* bm,
                        const double* bl) {
        if (L.qcols.empty()) return;
        // the kernels' step bucket from the largest step count listed
        const int mx = *std::max_element(L.qm.begin(), L.qm.end());
        VNE_TRY_CUDA(ctx, launch_tridiag_quad_list(S->alpha, S->beta, S->norm2, S->scale, (int)L.qcols.size(), qc,
                                                   qm, mx, SK, S->psi, st));
        ctx->launches += 1;
        if (!L.bcols.empty()) {
            VNE_TRY_CUDA(ctx, launch_tridiag_bounds_list(S->alpha, S->beta, S->norm2, S->scale, (int)L.bcols.size(),
                                                         bc, bm, bl, mx, SK, 0.0, 1.0, S->grid, S->est,
                                                         S->est + SK, S->est + 2 * SK, st));
            ctx->launches += 1;
            he = download(ctx, S->est + 2 * SK, SK);
        }
        hp = download(ctx, S->psi, SK);
    };
    auto passes = [&](const vne_server::Req& rq, int c_begin, int c_end) {
        for (int c = c_begin; c < c_end; c++) {
            const size_t o = (size_t)rq.slot * K + c;
            if (!(he[o] <= rq.tau * fabs(hp[o]))) return false;
        }
        return true;
    };
    evaluate(LA, (const int32_t*)dptr(i_qc), (const int32_t*)dptr(i_qm), (const int32_t*)dptr(i_bc),
             (const int32_t*)dptr(i_bm), (const double*)dptr(i_bl));
    std::vector<int> candidates;
    for (int ri : checking)
        if (passes(S->reqs[ri], 0, kFirst)) candidates.push_back(ri);
    std::vector<char> block_done(S->reqs.size(), 0);
    for (int ri : ending) block_done[ri] = 1;
    // the rest of the candidates' columns (the device arrays keep the values
    // of the first evaluation for every other column)
    if (!candidates.empty() && kFirst < K) {
        Lists LB = make_lists({}, candidates, kFirst, K);
        evaluate(LB, upload(ctx, "srv.qcols", LB.qcols), upload(ctx, "srv.qm", LB.qm),
                 upload(ctx, "srv.bcols", LB.bcols), upload(ctx, "srv.bm", LB.bm), upload(ctx, "srv.blam", LB.blam));
    }
    for (int ri : candidates)
        if (passes(S->reqs[ri], kFirst, K)) block_done[ri] = 1;
    int completed = 0;
    std::vector<int> still;
    for (int ri : S->active) {
        vne_server::Req& rq = S->reqs[ri];
        if (!block_done[ri]) {
            rq.j++;
            still.push_back(ri);
            continue;
        }
        for (int c = 0; c < K; c++) {  // Welford update
            const double x = hp[(size_t)rq.slot * K + c];
            rq.nvec++;
            const double d = x - rq.mean;
            rq.mean += d / (double)rq.nvec;
            rq.m2 += d * (x - rq.mean);
        }
        rq.blocks++;
        rq.est = rq.low + rq.mean;
        rq.se = rq.nvec > 1 ? sqrt(rq.m2 / (double)(rq.nvec - 1) / (double)rq.nvec) : 0.0;
        const bool converged = rq.blocks >= 2 && 2.576 * rq.se <= 0.5 * rq.eps * fabs(rq.est);
        if (converged || rq.nvec >= rq.max_vectors) {
            rq.state = 2;
            rq.done_tick = S->tick;
            release(S, rq);
            completed++;
        } else {
            rq.j = 0;  // the next block starts at the next tick
            still.push_back(ri);
        }
    }
    S->active.swap(still);
    return completed;
}

}  // namespace

extern "C" vne_status vne_server_create(vne_ctx* ctx, uint64_t hbm_budget_bytes, int32_t max_active,
                                        int32_t krylov_steps, int32_t block_vectors, const vne_options* opt,
                                        vne_server** out) {
    if (!ctx || !out) return VNE_EINVAL;
    *out = nullptr;
    if (max_active < 1 || max_active > 1024 || krylov_steps < 1 || krylov_steps > 128 || block_vectors < 8 ||
        block_vectors > 64)
        return VNE_EINVAL;
    vne_server* S = new (std::nothrow) vne_server();
    if (!S) return VNE_ENOMEM;
    S->ctx = ctx;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->m = krylov_steps;
    if (opt) S->opt = *opt;
    else vne_options_default(&S->opt);
    S->opt.reorth = 0;
    S->quad_tol = S->opt.quad_tol;
    S->check = S->opt.check_every > 0 ? S->opt.check_every : 5;
    S->ks = S->opt.panel > 0 ? S->opt.panel : 16;
    if (S->ks != 8 && S->ks != 16 && S->ks != 32) S->ks = 16;
    S->K = ((block_vectors + S->ks - 1) / S->ks) * S->ks;
    if (S->K > 64) {
        delete S;
        return VNE_EINVAL;
    }
    *out = S;
    return VNE_OK;
}

extern "C" vne_status vne_server_destroy(vne_server* S) {
    if (!S) return VNE_EINVAL;
    cudaSetDevice(S->ctx->device);
    if (S->ctx->stream) cudaStreamSynchronize(S->ctx->stream);
    else cudaDeviceSynchronize();
    delete S;
    return VNE_OK;
}

extern "C" vne_status vne_server_submit(vne_server* S, vne_matrix* M, double rel_eps, uint64_t seed,
                                        int32_t max_vectors, int32_t* ticket) {
    if (!S || !M || !ticket || !(rel_eps > 0.0) || max_vectors < 2) return VNE_EINVAL;
    vne_ctx* ctx = S->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, M->ctx == ctx && M->pattern && M->desing, VNE_EINVAL,
                "serving takes graph (pattern) matrices of the server's context");
    VNE_REQUIRE(ctx, S->precision < 0 || S->precision == (M->fp64 ? 1 : 0), VNE_EINVAL,
                "all queries of a server share one precision");
    if (S->precision < 0) arena_alloc(S, M->fp64);
    const size_t es = M->fp64 ? 8 : 4;
    vne_server::Req r{};
    r.M = M;
    r.eps = rel_eps;
    r.seed = seed;
    r.seed_mixed = seed_mix(seed);
    r.max_vectors = max_vectors;
    r.tau = S->quad_tol > 0.0 ? S->quad_tol : (S->quad_tol < 0.0 ? 0.5 * rel_eps : 0.0);
    r.lam_max = M->normM * M->scale;
    r.footprint = (size_t)(M->n + 1) * row_bytes(S, es) + (size_t)4 * M->nnz;
    VNE_REQUIRE(ctx, M->n + 1 <= S->rows_cap && M->nnz <= S->nnz_cap && r.footprint <= S->budget, VNE_ENOMEM,
                "query of %lld rows and %lld nonzeros exceeds the server's capacity", (long long)M->n,
                (long long)M->nnz);
    r.submit_tick = S->tick;
    *ticket = (int32_t)S->reqs.size();
    S->reqs.push_back(r);
    S->pending.push_back(*ticket);
    VNE_API_END(ctx)
}

extern "C" vne_status vne_server_step(vne_server* S, int32_t* completed, int32_t* active_count) {
    if (!S) return VNE_EINVAL;
    vne_ctx* ctx = S->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    int done = 0;
    if (S->precision == 1) done = tick_impl<double>(S);
    else if (S->precision == 0) done = tick_impl<float>(S);
    if (completed) *completed = done;
    if (active_count) *active_count = (int32_t)S->active.size();
    VNE_API_END(ctx)
}

extern "C" vne_status vne_server_result(const vne_server* S, int32_t ticket, int32_t* state, double* estimate,
                                        double* std_error, int64_t* vectors_used, int64_t* ticks) {
    if (!S || ticket < 0 || ticket >= (int32_t)S->reqs.size()) return VNE_EINVAL;
    const vne_server::Req& r = S->reqs[ticket];
    if (state) *state = r.state;
    if (estimate) *estimate = r.est;
    if (std_error) *std_error = r.se;
    if (vectors_used) *vectors_used = r.nvec;
    if (ticks) {
        ticks[0] = r.submit_tick;
        ticks[1] = r.admit_tick;
        ticks[2] = r.done_tick;
    }
    return VNE_OK;
}

extern "C" vne_status vne_server_info(const vne_server* S, int32_t* queued, int32_t* active, uint64_t* used_bytes) {
    if (!S) return VNE_EINVAL;
    if (queued) *queued = (int32_t)(S->pending.size() - S->pend_head);
    if (active) *active = (int32_t)S->active.size();
    if (used_bytes) *used_bytes = S->used;
    return VNE_OK;
}
