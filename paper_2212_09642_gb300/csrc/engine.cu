// Block Krylov engine of libvne: workspace and error helpers, the warp-level
// schedule of a packed CSR operator, the block Lanczos step loop with CUDA
// graph capture and replay, blocked quadratic forms and operator application.
//
// Engine overview.  A "problem" is a packed CSR operator M (one graph, or
// several graphs block-diagonally, each a segment) with a warp-level work
// schedule.  A block of K probe columns runs m Lanczos steps at once: per
// step one fused SpMM kernel and one update kernel (kernels_lanczos.cu), all
// launched back to back on the context stream with no host synchronisation;
// then one FP64 tridiagonal-quadrature kernel gives psi for every column.
#include "engine.h"

namespace vne_engine {

namespace {
std::atomic<int64_t> g_live_dev{0}, g_live_pinned{0};
std::atomic<int64_t> g_fail_countdown{0};  // > 0: the allocation that brings it to 0 fails

bool inject_failure() {
    int64_t v = g_fail_countdown.load();
    while (v > 0) {
        if (g_fail_countdown.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
    *p = nullptr;
    if (inject_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_dev++;
    else *p = nullptr;
    return e;
}

void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_dev--;
}

cudaError_t pinned_malloc(void** p, size_t bytes) {
    *p = nullptr;
    if (inject_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_live_pinned++;
    else *p = nullptr;
    return e;
}

void pinned_free(void* p) {
    if (!p) return;
    cudaFreeHost(p);
    g_live_pinned--;
}

int64_t live_device_buffers() { return g_live_dev.load(); }
int64_t live_pinned_buffers() { return g_live_pinned.load(); }
void fail_allocation_after(int64_t k) { g_fail_countdown.store(k); }

void set_err(vne_ctx* ctx, const char* fmt, ...) {
    if (!ctx) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
}

void* ws_get(vne_ctx* ctx, const std::string& name, size_t bytes, bool zero) {
    WsBuf& b = ctx->ws[name];
    if (b.bytes < bytes) {
        dev_free(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        size_t alloc = std::max<size_t>(bytes, 256);
        VNE_TRY_CUDA(ctx, dev_malloc(&b.ptr, alloc));
        VNE_TRY_CUDA(ctx, cudaMemsetAsync(b.ptr, 0, alloc, ctx->stream));
        b.bytes = alloc;
    }
    if (zero && bytes) VNE_TRY_CUDA(ctx, cudaMemsetAsync(b.ptr, 0, bytes, ctx->stream));
    return b.ptr;
}

void* pinned_bytes(vne_ctx* ctx, const std::string& name, size_t bytes) {
    auto& b = ctx->pinned[name];
    if (b.second < bytes) {
        pinned_free(b.first);
        b.first = nullptr;
        b.second = 0;
        if (pinned_malloc(&b.first, bytes) != cudaSuccess) {
            b.first = nullptr;
            return nullptr;
        }
        b.second = bytes;
    }
    return b.first;
}

const std::vector<int32_t>& host_cols(vne_matrix* M) {
    if ((int64_t)M->h_col.size() != M->nnz) {
        M->h_col.resize(M->nnz);
        if (M->nnz) {
            VNE_TRY_CUDA(M->ctx, cudaMemcpyAsync(M->h_col.data(), M->d_col, M->nnz * sizeof(int32_t),
                                                 cudaMemcpyDeviceToHost, M->ctx->stream));
            VNE_TRY_CUDA(M->ctx, cudaStreamSynchronize(M->ctx->stream));
        }
    }
    return M->h_col;
}

cudaEvent_t ctx_event(vne_ctx* ctx) {
    if (ctx->ev_next == ctx->ev_pool.size()) {
        cudaEvent_t e;
        VNE_TRY_CUDA(ctx, cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_next++];
}

void ctx_flush_profile(vne_ctx* ctx) {
    for (auto& p : ctx->pending) {
        if (!p.a) {  // bytes-only record (work measured after the launches ran)
            ctx->stat[p.kind].bytes += p.bytes;
            continue;
        }
        float ms = 0.f;
        VNE_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->stat[p.kind].launches++;
        ctx->stat[p.kind].ms += ms;
        ctx->stat[p.kind].bytes += p.bytes;
    }
    ctx->pending.clear();
    ctx->ev_next = 0;
}

uint64_t mix64_host(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t seed_mix(uint64_t seed) { return mix64_host(seed + 0x9E3779B97F4A7C15ULL); }

extern const int kTileRows = 4096;

// Work items of one segment (rows [row_begin, row_begin + rows) of the packed
// CSR): runs of short rows with about `target` nonzeros (at most 64 rows),
// and rows longer than `long_thresh` split into chunks of `chunk` nonzeros.
void plan_segment(const int64_t* rowptr, int32_t row_begin, int32_t rows, int32_t seg, int target, Problem& P) {
    // every item holds at most `target` nonzeros: short rows are packed into
    // runs (at most 64 rows), rows longer than `target` are split into chunks
    const int64_t chunk = std::max(target, 32);
    // at most 64 rows per item, 128 for items of 1024 nonzeros or more (fewer
    // CTAs, so less of the per-CTA reduction tail per row)
    const int max_rows = target >= 1024 ? kItemMaxRows : 64;
    const size_t first_item = P.items.size();
    SegInfo& sg0 = P.segs[seg];
    sg0.hub_begin = (int32_t)P.hubs.size();
    int32_t blk_start = -1, blk_rows = 0;
    int64_t blk_nnz = 0;
    auto flush = [&]() {
        if (blk_rows > 0)
            P.items.push_back(WorkItem{blk_start, blk_rows, (int32_t)rowptr[blk_start],
                                       (int32_t)rowptr[blk_start + blk_rows]});
        blk_start = -1;
        blk_rows = 0;
        blk_nnz = 0;
    };
    for (int32_t r = row_begin; r < row_begin + rows; r++) {
        int64_t deg = rowptr[r + 1] - rowptr[r];
        if (deg > chunk) {
            flush();
            int32_t nch = (int32_t)((deg + chunk - 1) / chunk);
            int32_t h = (int32_t)P.hubs.size();
            P.hubs.push_back(HubRow{r, nch, P.hub_slots, seg});
            P.hub_slots += nch;
            for (int32_t c = 0; c < nch; c++) {
                int64_t b = rowptr[r] + c * chunk, e = std::min<int64_t>(rowptr[r + 1], b + chunk);
                P.items.push_back(WorkItem{h, -(c + 1), (int32_t)b, (int32_t)e});
            }
            continue;
        }
        if (blk_rows > 0 && (blk_nnz + deg > chunk || blk_rows >= max_rows)) flush();
        if (blk_rows == 0) blk_start = r;
        blk_rows++;
        blk_nnz += deg;
    }
    flush();
    while ((P.items.size() - first_item) % ((size_t)VNE_WARPS * P.ipw)) P.items.push_back(WorkItem{0, 0, 0, 0});
    for (size_t i = first_item; i < P.items.size(); i++)
        P.stage_nnz = std::max<int32_t>(P.stage_nnz, P.items[i].nnz_end - P.items[i].nnz_begin);
    SegInfo& sg = P.segs[seg];
    sg.hub_count = (int32_t)P.hubs.size() - sg.hub_begin;
    sg.cta_begin = (int32_t)(first_item / ((size_t)VNE_WARPS * P.ipw));
    sg.cta_count = (int32_t)((P.items.size() - first_item) / ((size_t)VNE_WARPS * P.ipw));
    for (int32_t c = 0; c < sg.cta_count; c++) P.cta_seg.push_back(seg);
    sg.tile_begin = (int32_t)P.tiles.size();
    // row tiles of the streaming kernels: 4096 rows, fewer for small
    // segments (at least 16 tiles down to 256 rows) so that their update and
    // reorthogonalisation passes still spread over several SMs
    const int32_t trows = std::max<int32_t>(256, std::min<int32_t>(kTileRows, ((rows / 16) + 31) & ~31));
    for (int32_t r = row_begin; r < row_begin + rows; r += trows)
        P.tiles.push_back(RowTile{r, std::min(row_begin + rows, r + trows), seg, 0});
    sg.tile_count = (int32_t)P.tiles.size() - sg.tile_begin;
}


void problem_upload(vne_ctx* ctx, Problem& P) {
    P.d_segs = dev_copy(ctx, P.segs);
    P.d_items = dev_copy(ctx, P.items);
    P.d_hubs = dev_copy(ctx, P.hubs);
    P.d_cta_seg = dev_copy(ctx, P.cta_seg);
    P.d_tiles = dev_copy(ctx, P.tiles);
}

double default_tau(bool fp64) { return fp64 ? 1e-13 : 1e-10; }

int default_item_nnz(const vne_options* o) { return (o && o->item_nnz > 0) ? o->item_nnz : 256; }


Sched resolve_sched(const vne_matrix* M, const vne_options* o) {
    Sched s;
    s.ks = (o && o->panel > 0) ? o->panel : (M->tuned ? M->tuned_panel : choose_panel(M->fp64, o, M->n));
    s.item_nnz = (o && o->item_nnz > 0) ? o->item_nnz : (M->tuned ? M->tuned_item_nnz : 256);
    s.variant = (o && o->step_variant >= 0) ? o->step_variant : (M->tuned ? M->tuned_variant : 4);
    if (M->fp64) s.variant = 0;
    s.ipw = (o && o->items_per_warp > 0) ? o->items_per_warp : (M->tuned ? M->tuned_ipw : 1);
    s.interleave = (o && o->interleave >= 0) ? (o->interleave != 0) : (M->tuned ? M->tuned_interleave : false);
    s.graph = !(o && o->graphs == 0);
    return s;
}

Problem* matrix_problem(vne_matrix* M, const vne_options* opt) {
    const Sched sc = resolve_sched(M, opt);
    int target = sc.item_nnz;
    double taurel = (opt && opt->breakdown_tol > 0) ? opt->breakdown_tol : default_tau(M->fp64);
    if (M->prob && M->prob_item_nnz == target && M->prob->ipw == sc.ipw && M->prob->segs[0].tau == taurel * M->normM)
        return M->prob;
    delete M->prob;
    M->prob = nullptr;
    std::unique_ptr<Problem> P(new Problem());
    P->fp64 = M->fp64;
    P->valued = !M->pattern;
    P->n_total = (int32_t)M->n;
    P->nnz_total = M->nnz;
    P->nseg = 1;
    P->rowptr = M->d_rowptr;
    P->col = M->d_col;
    P->vals = M->d_vals;
    P->node_id = M->d_node_id;
    P->ipw = sc.ipw;
    P->norm_m = M->normM;
    SegInfo s{};
    s.row_begin = 0;
    s.rows = (int32_t)M->n;
    s.scale = M->scale;
    s.tau = taurel * M->normM;
    P->segs.push_back(s);
    plan_segment(M->h_rowptr.data(), 0, (int32_t)M->n, 0, target, *P);
    problem_upload(M->ctx, *P);
    M->prob = P.release();
    M->prob_item_nnz = target;
    return M->prob;
}

int choose_panel(bool fp64, const vne_options* opt, int64_t n) {
    if (opt && opt->panel > 0) return opt->panel;
    if (fp64) return 8;
    // keep one panel (n * KS * 4 bytes) comfortably inside L2
    if (n * 16 * 4 <= (int64_t)64 << 20) return 16;
    return 8;
}

// ---------------------------------------------------------------------------
// block Krylov engine



template <typename T>
void run_block(vne_ctx* ctx, Problem& P, const StartSource& src, const T* panel_src, int K, int ks, int m,
               int reorth, bool keep_basis, bool desing, const std::string& tag, BlockOut& out, int variant,
               bool interleave, bool graph, bool want_psi, const Adaptive* ad) {
    cudaStream_t st = ctx->stream;
    const int panels = (K + ks - 1) / ks;
    const int Kp = panels * ks;
    const int S = P.nseg;
    const int SK = S * Kp;
    const size_t slot_elems = (size_t)Kp * P.n_total;
    const bool store_all = keep_basis || reorth != 0;
    const int nslots = store_all ? m + 1 : 2;
    VNE_REQUIRE(ctx, reorth == 0 || S == 1, VNE_EUNSUPPORTED, "reorthogonalisation needs a single matrix");
    T* slots = ws_get_t<T>(ctx, tag + ".slots", slot_elems * nslots);
    T* u = ws_get_t<T>(ctx, "u", slot_elems);
    double* alpha = ws_get_t<double>(ctx, tag + ".alpha", (size_t)m * SK, true);
    double* beta = ws_get_t<double>(ctx, tag + ".beta", (size_t)m * SK, true);
    double* sigma = ws_get_t<double>(ctx, tag + ".sigma", (size_t)(m + 1) * SK, true);
    double* norm2 = ws_get_t<double>(ctx, tag + ".norm2", SK);
    double* mean = ws_get_t<double>(ctx, "mean", SK);
    double* psi = ws_get_t<double>(ctx, tag + ".psi", SK);
    const int ctas = P.ctas_per_panel(), tiles = P.tiles_per_panel();
    double* part = ws_get_t<double>(ctx, "part", (size_t)panels * std::max(ctas, tiles) * ks);
    uint32_t* counter = ws_get_t<uint32_t>(ctx, "counter", (size_t)panels * S, true);
    const int nh = (int)P.hubs.size();
    const int64_t nnz_total = P.nnz_total;
    T* hub_part = ws_get_t<T>(ctx, "hub_part", (size_t)panels * std::max(P.hub_slots, 1) * ks);
    uint32_t* hub_cnt = ws_get_t<uint32_t>(ctx, "hub_cnt", (size_t)panels * std::max(nh, 1), true);
    double* hub_dot = ws_get_t<double>(ctx, "hub_dot", (size_t)panels * std::max(nh, 1) * ks);
    // per-column scale (segment scale) for the quadrature
    std::vector<double> hscale(SK);
    for (int s = 0; s < S; s++)
        for (int c = 0; c < Kp; c++) hscale[(size_t)s * Kp + c] = P.segs[s].scale;
    double* dscale = upload(ctx, tag + ".scale", hscale);

    auto slot = [&](int j) -> T* {  // slot holding w_j, j >= 1
        int idx = store_all ? (j - 1) : ((j - 1) & 1);
        return slots + (size_t)idx * slot_elems;
    };

    StartParams<T> sp{};
    sp.src = src;
    sp.panel_src = panel_src;
    sp.node_id = P.node_id;
    sp.seg = P.d_segs;
    sp.nseg = S;
    sp.K = Kp;
    sp.n_total = P.n_total;
    sp.tiles_per_panel = tiles;
    sp.tiles = P.d_tiles;
    sp.desing = desing ? 1 : 0;
    sp.w1 = slot(1);
    sp.mean = mean;
    sp.norm2 = norm2;
    sp.sig1 = sigma;
    sp.part = part;
    sp.counter = counter;
    VNE_TRY_CUDA(ctx, launch_start<T>(sp, ks, panels, st));
    ctx->launches += desing ? 2 : 1;

    StepParams<T> p;
    memset(&p, 0, sizeof(p));  // the bytes of p are part of the graph key
    p.rowptr = P.rowptr;
    p.col = P.col;
    p.vals = (const T*)P.vals;
    p.n_total = P.n_total;
    p.K = Kp;
    p.nseg = S;
    p.seg = P.d_segs;
    p.items = P.d_items;
    p.ctas_per_panel = ctas;
    p.cta_seg = P.d_cta_seg;
    p.hubs = P.d_hubs;
    p.nhubs = std::max(nh, 1);
    p.hub_slots = std::max(P.hub_slots, 1);
    p.hub_part = hub_part;
    p.hub_cnt = hub_cnt;
    p.hub_dot = hub_dot;
    p.stage_nnz = std::max(P.stage_nnz, 1);
    p.ipw = P.ipw;
    p.tiles = P.d_tiles;
    p.tiles_per_panel = tiles;
    p.u = u;
    p.part = part;
    p.counter = counter;
    double* rcoef = nullptr;
    double* rpart = nullptr;
    if (reorth) {
        rcoef = ws_get_t<double>(ctx, "reorth.coef", (size_t)m * Kp);
        rpart = ws_get_t<double>(ctx, "reorth.part", (size_t)panels * m * tiles * ks);
    }
    // partial reorthogonalisation state (Simon's omega recurrence)
    ProParams pro{};
    if (reorth == 2) {
        pro.alpha = alpha;
        pro.beta = beta;
        pro.sig = sigma;
        pro.omega = ws_get_t<double>(ctx, tag + ".pro.omega", (size_t)2 * (m + 2) * SK);
        pro.sel = ws_get_t<uint8_t>(ctx, tag + ".pro.sel", (size_t)(m + 1) * SK);
        pro.pend_sel = ws_get_t<uint8_t>(ctx, tag + ".pro.psel", (size_t)(m + 2) * SK);
        pro.pend = ws_get_t<int32_t>(ctx, tag + ".pro.pend", SK);
        pro.panel_active = ws_get_t<int32_t>(ctx, tag + ".pro.active", panels);
        pro.SK = SK;
        pro.ks = ks;
        pro.K = Kp;
        pro.m = m;
        pro.eps = sizeof(T) == 4 ? 0x1.0p-24 : 0x1.0p-53;
        pro.normM = P.norm_m;
    }
    // The step loop, enqueued on stream `s`; `prof` brackets the launches
    // with events (never while capturing).
    auto enqueue_loop = [&](cudaStream_t s, bool prof, int j_begin, int j_end) {
        for (int j = j_begin; j <= j_end; j++) {
            p.first = (j == 1);
            p.renorm = 0;
            p.w_cur = slot(j);
            p.w_prev = (j > 1) ? slot(j - 1) : slot(j);
            p.w_next = slot(j + 1);
            p.sig_cur = sigma + (size_t)(j - 1) * SK;
            p.sig_prev = (j > 1) ? sigma + (size_t)(j - 2) * SK : sigma;
            p.beta_prev = (j > 1) ? beta + (size_t)(j - 2) * SK : beta;
            p.alpha = alpha + (size_t)(j - 1) * SK;
            p.beta = beta + (size_t)(j - 1) * SK;
            p.sig_next = sigma + (size_t)j * SK;
            cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
            if (prof) {
                e0 = ctx_event(ctx);
                VNE_TRY_CUDA(ctx, cudaEventRecord(e0, s));
            }
            if (interleave && !reorth) {
                // per-panel launches, step then update of the same panel: the
                // update finds u and w_j of that panel still in L2
                for (int pn = 0; pn < panels; pn++) {
                    p.panel_base = pn;
                    VNE_TRY_CUDA(ctx, launch_step<T>(p, ks, 1, P.valued, variant, s));
                    VNE_TRY_CUDA(ctx, launch_update<T>(p, ks, 1, s));
                }
                p.panel_base = 0;
                ctx->launches += 2 * panels;
                if (prof) {
                    e1 = ctx_event(ctx);
                    VNE_TRY_CUDA(ctx, cudaEventRecord(e1, s));
                }
            } else {
                p.panel_base = 0;
                VNE_TRY_CUDA(ctx, launch_step<T>(p, ks, panels, P.valued, variant, s));
                if (prof) {
                    e1 = ctx_event(ctx);
                    VNE_TRY_CUDA(ctx, cudaEventRecord(e1, s));
                }
                VNE_TRY_CUDA(ctx, launch_update<T>(p, ks, panels, s));
                ctx->launches += 2;
            }
            if (prof) {
                e2 = ctx_event(ctx);
                VNE_TRY_CUDA(ctx, cudaEventRecord(e2, s));
                // algorithmic (compulsory) bytes: the CSR structure (+ values)
                // once per launch, the gathered block w_j once, w_{j-1} (j > 1)
                // and u once each; the re-reads of the CSR for every further
                // panel are the design's own traffic, not counted here
                const double es = sizeof(T);
                double csr = 4.0 * (P.n_total + 1) + (double)nnz_total * (4.0 + (P.valued ? es : 0.0));
                double vec = (double)P.n_total * ks * es;
                double step_bytes = (interleave && !reorth ? panels : 1) * csr + panels * vec * (j > 1 ? 3.0 : 2.0);
                double upd_bytes = panels * vec * 3.0;
                if (interleave && !reorth) {
                    // one timed span covers the interleaved step and update launches
                    ctx->pending.push_back({0, e0, e1, step_bytes + upd_bytes});
                } else {
                    ctx->pending.push_back({0, e0, e1, step_bytes});
                    ctx->pending.push_back({1, e1, e2, upd_bytes});
                }
            }
            if (reorth == 2) {
                // estimate the loss of orthogonality of w_{j+1}; orthogonalise
                // the columns that need it (twice) against their selected
                // basis vectors and renormalise; panels with nothing to do
                // skip every pass
                pro.j = j;
                VNE_TRY_CUDA(ctx, cudaMemsetAsync(pro.panel_active, 0, panels * sizeof(int32_t), s));
                VNE_TRY_CUDA(ctx, launch_pro_omega(pro, s));
                ReorthParams<T> rp{};
                rp.basis = slots;
                rp.slot_stride = slot_elems;
                rp.w = slot(j + 1);
                rp.j = j;
                rp.K = Kp;
                rp.n_total = P.n_total;
                rp.panels = panels;
                rp.tiles_per_panel = tiles;
                rp.tiles = P.d_tiles;
                rp.part = rpart;
                rp.coef = rcoef;
                rp.panel_active = pro.panel_active;
                rp.sel = pro.sel;
                ReorthCoefParams cp{};
                cp.part = rpart;
                cp.sig = sigma;
                cp.coef = rcoef;
                cp.j = j;
                cp.K = Kp;
                cp.panels = panels;
                cp.tiles_per_panel = tiles;
                cp.sel = pro.sel;
                cp.panel_active = pro.panel_active;
                for (int pass = 0; pass < 2; pass++) VNE_TRY_CUDA(ctx, launch_reorth<T>(rp, cp, ks, s));
                p.renorm = 1;
                p.panel_active = pro.panel_active;
                VNE_TRY_CUDA(ctx, launch_update<T>(p, ks, panels, s));
                p.panel_active = nullptr;
                ctx->launches += 8;
            } else if (reorth && j < m + 1) {
                ReorthParams<T> rp{};
                rp.basis = slots;
                rp.slot_stride = slot_elems;
                rp.w = slot(j + 1);
                rp.j = j;
                rp.K = Kp;
                rp.n_total = P.n_total;
                rp.panels = panels;
                rp.tiles_per_panel = tiles;
                rp.tiles = P.d_tiles;
                rp.part = rpart;
                rp.coef = rcoef;
                ReorthCoefParams cp{};
                cp.part = rpart;
                cp.sig = sigma;
                cp.coef = rcoef;
                cp.j = j;
                cp.K = Kp;
                cp.panels = panels;
                cp.tiles_per_panel = tiles;
                for (int pass = 0; pass < 2; pass++) VNE_TRY_CUDA(ctx, launch_reorth<T>(rp, cp, ks, s));
                p.renorm = 1;
                VNE_TRY_CUDA(ctx, launch_update<T>(p, ks, panels, s));
                ctx->launches += 7;
            }
        }
    };
    if (ctx->time_steps) VNE_TRY_CUDA(ctx, cudaEventRecord(ctx->loop_ev[0], st));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    int m_run = m;  // steps actually taken
    if (ad && ad->tol > 0.0 && want_psi) {
        // adaptive: chunks of `check` steps launched directly, each followed
        // by the quadratures and error estimates of all columns
        double* est = ws_get_t<double>(ctx, tag + ".est", 3 * (size_t)SK);
        int j = 0;
        m_run = 0;
        while (j < m) {
            const int j1 = std::min(m, j + std::max(1, ad->check));
            enqueue_loop(st, ctx->profile, j + 1, j1);
            j = j1;
            m_run = j;
            if (j >= m) break;
            VNE_TRY_CUDA(ctx, launch_tridiag_quad(alpha, beta, norm2, dscale, SK, j, SK, psi, st));
            VNE_TRY_CUDA(ctx, launch_tridiag_bounds(alpha, beta, norm2, dscale, SK, j, SK, ad->lam_min, ad->lam_max,
                                                    ad->grid, est, est + SK, est + 2 * SK, st));
            ctx->launches += 2;
            std::vector<double> hp = download(ctx, psi, SK), he = download(ctx, est + 2 * SK, SK);
            bool done = true;
            if (ad->abs)
                for (int c = 0; c < ad->ncols && done; c++) done = he[c] <= ad->abs[c];
            else
                for (int c = 0; c < SK && done; c++) done = he[c] <= ad->tol * fabs(hp[c]);
            if (done) break;
        }
    } else if (!graph || ctx->profile || cap != cudaStreamCaptureStatusNone) {
        enqueue_loop(st, ctx->profile, 1, m);
    } else {
        // Graph key: every value the loop's launches depend on.
        std::string key;
        auto put = [&key](const void* v, size_t b) { key.append(reinterpret_cast<const char*>(v), b); };
        const int ints[] = {(int)sizeof(T), ks, panels, m, variant, (int)interleave, (int)reorth, (int)store_all,
                            (int)P.valued, SK};
        put(ints, sizeof(ints));
        const void* ptrs[] = {slots,     alpha,    beta,         sigma,    rcoef,          rpart,
                              pro.omega, pro.sel,     pro.pend_sel, pro.pend, pro.panel_active};
        put(ptrs, sizeof(ptrs));
        put(&slot_elems, sizeof(slot_elems));
        put(&p, sizeof(p));
        auto it = ctx->graphs.find(key);
        if (it == ctx->graphs.end()) {
            if (ctx->graph_seen.size() > 4096) ctx->graph_seen.clear();
            if (++ctx->graph_seen[key] >= 2) {
                if (ctx->graphs.size() >= 64) {
                    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
                    ctx->graphs.clear();
                }
                if (!ctx->cap_stream)
                    VNE_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
                const int64_t l0 = ctx->launches;
                cudaGraph_t g = nullptr;
                VNE_TRY_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
                try {
                    enqueue_loop(ctx->cap_stream, false, 1, m);
                } catch (...) {
                    cudaStreamEndCapture(ctx->cap_stream, &g);
                    if (g) cudaGraphDestroy(g);
                    ctx->launches = l0;
                    throw;
                }
                VNE_TRY_CUDA(ctx, cudaStreamEndCapture(ctx->cap_stream, &g));
                cudaGraphExec_t ex = nullptr;
                cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                VNE_TRY_CUDA(ctx, e);
                it = ctx->graphs.emplace(key, vne_ctx::LoopGraph{ex, ctx->launches - l0}).first;
                ctx->launches = l0;
                ctx->graphs_captured++;
            }
        }
        if (it != ctx->graphs.end()) {
            VNE_TRY_CUDA(ctx, cudaGraphLaunch(it->second.exec, st));
            ctx->launches += it->second.kernels;
            ctx->graphs_replayed++;
        } else {
            enqueue_loop(st, false, 1, m);
        }
    }
    if (ctx->time_steps) VNE_TRY_CUDA(ctx, cudaEventRecord(ctx->loop_ev[1], st));
    if (want_psi) {
        VNE_TRY_CUDA(ctx, launch_tridiag_quad(alpha, beta, norm2, dscale, SK, m_run, SK, psi, st));
        ctx->launches += 1;
    }
    ctx->last_steps = std::max(ctx->last_steps, m_run);
    out.K = K;
    out.Kp = Kp;
    out.ks = ks;
    out.panels = panels;
    out.m = m_run;
    out.SK = SK;
    out.alpha = alpha;
    out.beta = beta;
    out.sigma = sigma;
    out.norm2 = norm2;
    out.psi = psi;
    out.scale = dscale;
    out.basis = slots;
    out.slot_stride = slot_elems;
}

std::vector<double> download(vne_ctx* ctx, const double* d, size_t count) {
    std::vector<double> h(count);
    if (count) VNE_TRY_CUDA(ctx, cudaMemcpyAsync(h.data(), d, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!ctx->pending.empty()) ctx_flush_profile(ctx);
    return h;
}

int want_reorth(const vne_matrix* M, const vne_options* o) {
    int r = o ? o->reorth : -1;
    if (r < 0) return M->fp64 ? 1 : 0;
    return r == 2 ? 2 : (r != 0 ? 1 : 0);
}

int block_limit(const vne_options* o) { return (o && o->block > 0) ? o->block : 256; }

vne_options defaults() {
    vne_options o;
    vne_options_default(&o);
    return o;
}


template <typename T>
std::vector<double> quadforms(vne_matrix* M, const vne_options* o, StartSource src, int ncols, int m,
                              const double* abs_tol) {
    vne_ctx* ctx = M->ctx;
    Problem* P = matrix_problem(M, o);
    Sched sc = resolve_sched(M, o);
    int ks = sc.ks;
    check_ks<T>(ctx, ks);
    int lim = block_limit(o);
    const int reorth = want_reorth(M, o);
    std::vector<double> psi(ncols);
    ctx->last_steps = 0;
    Adaptive ad;
    if (o && o->quad_tol > 0.0) {
        ad.tol = o->quad_tol;
        ad.check = o->check_every > 0 ? o->check_every : 5;
        ad.lam_min = o->spectrum_min;
        ad.lam_max = M->normM * M->scale;
    }
    if (abs_tol) {
        ad.tol = 1.0;  // enables the adaptive loop; the per-column tolerances decide
        ad.check = o && o->check_every > 0 ? o->check_every : 5;
        ad.lam_min = o ? o->spectrum_min : 0.0;
        ad.lam_max = M->normM * M->scale;
    }
    for (int b0 = 0; b0 < ncols; b0 += lim) {
        int K = std::min(lim, ncols - b0);
        if (abs_tol) {
            ad.abs = abs_tol + b0;
            ad.ncols = K;
        }
        StartSource s = src;
        s.ncols = K;
        if (s.kind == SRC_RADEMACHER || s.kind == SRC_INDICATOR) s.col_begin = src.col_begin + b0;
        if (s.kind == SRC_DENSE64) s.dense = src.dense + b0;
        BlockOut out;
        run_block<T>(ctx, *P, s, nullptr, K, ks, m, reorth, false, M->desing, "q", out, sc.variant, sc.interleave,
                     sc.graph, true, ad.tol > 0.0 ? &ad : nullptr);
        std::vector<double> h = download(ctx, out.psi, K);
        std::copy(h.begin(), h.end(), psi.begin() + b0);
    }
    return psi;
}


// Apply the operator to a panel-major block with the Lanczos step kernel:
// out = A in + shift * in (A = scale M), and dq[c] = scale * (in . out).
template <typename T>
void apply_operator(vne_ctx* ctx, Problem& P, int ks, int Kp, const T* in, T* out, double shift, double* dq,
                    int variant, const std::string& tag) {
    cudaStream_t st = ctx->stream;
    const int panels = Kp / ks;
    const int ctas = P.ctas_per_panel(), tiles = P.tiles_per_panel();
    const int nh = (int)P.hubs.size();
    const double scale = P.segs[0].scale;
    std::vector<double> hs(Kp, scale), hc(Kp, -shift), h1(Kp, 1.0);
    StepParams<T> p{};
    p.rowptr = P.rowptr;
    p.col = P.col;
    p.vals = (const T*)P.vals;
    p.n_total = P.n_total;
    p.K = Kp;
    p.nseg = 1;
    p.seg = P.d_segs;
    p.items = P.d_items;
    p.ctas_per_panel = ctas;
    p.cta_seg = P.d_cta_seg;
    p.hubs = P.d_hubs;
    p.nhubs = std::max(nh, 1);
    p.hub_slots = std::max(P.hub_slots, 1);
    p.hub_part = ws_get_t<T>(ctx, "hub_part", (size_t)panels * std::max(P.hub_slots, 1) * ks);
    p.hub_cnt = ws_get_t<uint32_t>(ctx, "op.hub_cnt", (size_t)panels * std::max(nh, 1));
    p.hub_dot = ws_get_t<double>(ctx, "hub_dot", (size_t)panels * std::max(nh, 1) * ks);
    p.stage_nnz = std::max(P.stage_nnz, 1);
    p.ipw = P.ipw;
    p.tiles = P.d_tiles;
    p.tiles_per_panel = tiles;
    p.first = (shift == 0.0) ? 1 : 0;
    p.renorm = 0;
    p.w_cur = in;
    p.w_prev = in;
    p.u = out;
    p.w_next = out;
    p.sig_cur = upload(ctx, tag + ".sig", hs);
    p.beta_prev = upload(ctx, tag + ".cp", hc);
    p.sig_prev = upload(ctx, tag + ".one", h1);
    p.alpha = dq;
    p.part = ws_get_t<double>(ctx, "op.part", (size_t)panels * std::max(ctas, tiles) * ks);
    p.counter = ws_get_t<uint32_t>(ctx, "op.counter", (size_t)panels);
    cudaEvent_t e0 = nullptr;
    if (ctx->profile) {
        e0 = ctx_event(ctx);
        VNE_TRY_CUDA(ctx, cudaEventRecord(e0, st));
    }
    VNE_TRY_CUDA(ctx, launch_step<T>(p, ks, panels, P.valued, variant, st));
    ctx->launches += 1;
    if (ctx->profile) {
        cudaEvent_t e1 = ctx_event(ctx);
        VNE_TRY_CUDA(ctx, cudaEventRecord(e1, st));
        const double es = sizeof(T);
        double csr = 4.0 * (P.n_total + 1) + (double)P.nnz_total * (4.0 + (P.valued ? es : 0.0));
        double vec = (double)P.n_total * ks * es;
        ctx->pending.push_back({0, e0, e1, csr + panels * vec * (shift != 0.0 ? 3.0 : 2.0)});
    }
}

#define VNE_ENGINE_INSTANTIATE(T)                                                                                \
    template void run_block<T>(vne_ctx*, Problem&, const StartSource&, const T*, int, int, int, int, bool, bool,  \
                               const std::string&, BlockOut&, int, bool, bool, bool, const Adaptive*);          \
    template std::vector<double> quadforms<T>(vne_matrix*, const vne_options*, StartSource, int, int,             \
                                              const double*);                                                    \
    template void apply_operator<T>(vne_ctx*, Problem&, int, int, const T*, T*, double, double*, int,             \
                                    const std::string&);
VNE_ENGINE_INSTANTIATE(float)
VNE_ENGINE_INSTANTIATE(double)

}  // namespace vne_engine

vne_matrix::~vne_matrix() {
    delete prob;
    vne_engine::dev_free(d_rowptr);
    vne_engine::dev_free(d_col);
    vne_engine::dev_free(d_vals);
    vne_engine::dev_free(d_node_id);
}
