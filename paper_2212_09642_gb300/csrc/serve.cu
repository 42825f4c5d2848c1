// Serving loop of libvne: continuous batching of entropy queries.
#include "engine.h"

// ---------------------------------------------------------------------------
// serving: continuous batching of entropy queries
//
// Each tick admits queued requests (FIFO) while the active set fits the HBM
// budget and the slot limit, packs the active graphs block-diagonally on the
// device (their CSR stays resident from vne_create_density_matrix), and runs
// one Lanczos block of `block` Rademacher probes per request in one batched
// launch sequence.  A request's probes for tick t are its columns
// t*block .. (t+1)*block-1, so its numbers do not depend on its neighbours.
// After the block each request updates its running mean and variance and
// retires once 2.576 * stderr <= (eps / 2) * |mean| (at least two blocks) or
// its vector cap is reached.

namespace {

__global__ void k_pack_rowptr(const int32_t* src, int n, int32_t e0, int32_t* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + e0;
}
__global__ void k_pack_col(const int32_t* src, int64_t nnz, int32_t r0, int32_t* dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) dst[i] = src[i] + r0;
}
__global__ void k_pack_ids(const int32_t* perm, int n, int32_t* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = perm ? perm[i] : i;
}

}  // namespace

struct vne_server {
    vne_ctx* ctx = nullptr;
    size_t budget = 0, used = 0;
    int max_active = 64, m = 40, block = 64, max_vectors = 8192;
    vne_options opt;
    struct Req {
        vne_matrix* M;
        double eps;
        uint64_t seed_mixed;
        int max_vectors;
        int state;  // 0 queued, 1 active, 2 done
        int64_t nvec;
        double mean, m2, est, se;
        size_t footprint;
        int64_t submit_tick, admit_tick, done_tick;
        int blocks;
    };
    std::vector<Req> reqs;
    std::vector<int> pending;  // FIFO (front = index pend_head)
    size_t pend_head = 0;
    std::vector<int> active;
    int64_t tick = 0;
};

extern "C" vne_status vne_server_create(vne_ctx* ctx, uint64_t hbm_budget_bytes, int32_t max_active,
                                        int32_t krylov_steps, int32_t block_vectors, const vne_options* opt,
                                        vne_server** out) {
    if (!ctx || !out) return VNE_EINVAL;
    *out = nullptr;
    if (max_active < 1 || krylov_steps < 1 || krylov_steps > 128 || block_vectors < 2 || block_vectors > 256)
        return VNE_EINVAL;
    vne_server* S = new (std::nothrow) vne_server();
    if (!S) return VNE_ENOMEM;
    S->ctx = ctx;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->m = krylov_steps;
    S->block = block_vectors;
    if (opt) S->opt = *opt;
    else vne_options_default(&S->opt);
    *out = S;
    return VNE_OK;
}

extern "C" vne_status vne_server_destroy(vne_server* S) {
    if (!S) return VNE_EINVAL;
    delete S;
    return VNE_OK;
}

extern "C" vne_status vne_server_submit(vne_server* S, vne_matrix* M, double rel_eps, uint64_t seed,
                                        int32_t max_vectors, int32_t* ticket) {
    if (!S || !M || !ticket || !(rel_eps > 0.0) || max_vectors < 2) return VNE_EINVAL;
    vne_ctx* ctx = S->ctx;
    if (M->ctx != ctx || M->fp64 || !M->pattern) {
        set_err(ctx, "serving takes FP32 graph (pattern) matrices of the server's context");
        return VNE_EINVAL;
    }
    vne_server::Req r{};
    r.M = M;
    r.eps = rel_eps;
    r.seed_mixed = seed_mix(seed);
    r.max_vectors = max_vectors;
    const int ks = resolve_sched(M, &S->opt).ks;
    const int Kp = ((S->block + ks - 1) / ks) * ks;
    // resident CSR + the block's Lanczos vectors (2 slots + u) + scalars
    r.footprint = (size_t)4 * (M->n + 1 + M->nnz) + (size_t)3 * M->n * Kp * 4 + (size_t)(3 * S->m + 8) * Kp * 8;
    if (r.footprint > S->budget) {
        set_err(ctx, "request footprint %zu exceeds the HBM budget %zu", r.footprint, S->budget);
        return VNE_ENOMEM;
    }
    r.submit_tick = S->tick;
    *ticket = (int32_t)S->reqs.size();
    S->reqs.push_back(r);
    S->pending.push_back(*ticket);
    return VNE_OK;
}

extern "C" vne_status vne_server_step(vne_server* S, int32_t* completed, int32_t* active_count) {
    if (!S) return VNE_EINVAL;
    vne_ctx* ctx = S->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    if (completed) *completed = 0;
    // admission
    while (S->pend_head < S->pending.size() && (int)S->active.size() < S->max_active) {
        vne_server::Req& r = S->reqs[S->pending[S->pend_head]];
        if (S->used + r.footprint > S->budget) break;
        S->used += r.footprint;
        r.state = 1;
        r.admit_tick = S->tick;
        S->active.push_back(S->pending[S->pend_head]);
        S->pend_head++;
    }
    if (active_count) *active_count = (int32_t)S->active.size();
    S->tick++;
    if (S->active.empty()) return VNE_OK;
    const vne_options& o = S->opt;
    // all active matrices share the schedule knobs of the server options
    const int target = default_item_nnz(&o);
    int ks = 0, variant = 0;
    Problem P;
    P.owns_tables = false;
    P.fp64 = false;
    P.valued = false;
    int64_t ntot = 0, nnztot = 0;
    for (int idx : S->active) {
        ntot += S->reqs[idx].M->n;
        nnztot += S->reqs[idx].M->nnz;
    }
    VNE_REQUIRE(ctx, ntot < INT32_MAX && nnztot < INT32_MAX, VNE_EINVAL, "active set too large");
    int32_t* prp = ws_get_t<int32_t>(ctx, "srv.rowptr", ntot + 1);
    int32_t* pci = ws_get_t<int32_t>(ctx, "srv.col", std::max<int64_t>(nnztot, 1));
    int32_t* pid = ws_get_t<int32_t>(ctx, "srv.ids", ntot);
    std::vector<uint64_t> seeds;
    std::vector<int32_t> col0;
    int64_t r0 = 0, e0 = 0;
    cudaStream_t st = ctx->stream;
    for (size_t sidx = 0; sidx < S->active.size(); sidx++) {
        vne_server::Req& rq = S->reqs[S->active[sidx]];
        vne_matrix* M = rq.M;
        Sched sc = resolve_sched(M, &o);
        if (sidx == 0) {
            ks = sc.ks;
            variant = sc.variant;
        }
        Problem* MP = matrix_problem(M, &o);  // the matrix's own (cached) schedule
        const int n = (int)M->n;
        k_pack_rowptr<<<(n + 255) / 256, 256, 0, st>>>(M->d_rowptr, n, (int32_t)e0, prp + r0);
        if (M->nnz) k_pack_col<<<(unsigned)((M->nnz + 255) / 256), 256, 0, st>>>(M->d_col, M->nnz, (int32_t)r0, pci + e0);
        k_pack_ids<<<(n + 255) / 256, 256, 0, st>>>(M->d_node_id, n, pid + r0);
        ctx->launches += 3;
        SegInfo sg = MP->segs[0];
        const int32_t seg = (int32_t)sidx;
        const int32_t hub_base = (int32_t)P.hubs.size(), slot_base = P.hub_slots;
        sg.row_begin = (int32_t)r0;
        sg.cta_begin = (int32_t)(P.items.size() / VNE_WARPS);  // the packed problem takes one item per warp
        sg.cta_count = (int32_t)(MP->items.size() / VNE_WARPS);
        sg.tile_begin = (int32_t)P.tiles.size();
        sg.hub_begin = hub_base;
        for (WorkItem it : MP->items) {
            if (it.rows > 0) it.row += (int32_t)r0;
            else if (it.rows < 0) it.row += hub_base;
            if (it.rows != 0) {
                it.nnz_begin += (int32_t)e0;
                it.nnz_end += (int32_t)e0;
            }
            P.items.push_back(it);
        }
        for (HubRow h : MP->hubs) {
            h.row += (int32_t)r0;
            h.slot += slot_base;
            h.seg = seg;
            P.hubs.push_back(h);
        }
        P.hub_slots += MP->hub_slots;
        for (int32_t c = 0; c < sg.cta_count; c++) P.cta_seg.push_back(seg);
        for (RowTile t : MP->tiles) {
            t.row_begin += (int32_t)r0;
            t.row_end += (int32_t)r0;
            t.seg = seg;
            P.tiles.push_back(t);
        }
        P.stage_nnz = std::max(P.stage_nnz, MP->stage_nnz);
        P.segs.push_back(sg);
        seeds.push_back(rq.seed_mixed);
        col0.push_back(rq.blocks * S->block);
        r0 += M->n;
        e0 += M->nnz;
    }
    const int32_t last = (int32_t)nnztot;
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(prp + ntot, &last, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    VNE_TRY_CUDA(ctx, cudaGetLastError());
    P.n_total = (int32_t)ntot;
    P.nnz_total = nnztot;
    P.nseg = (int32_t)S->active.size();
    P.rowptr = prp;
    P.col = pci;
    P.node_id = pid;
    P.d_segs = upload(ctx, "srv.segs", P.segs);
    P.d_items = upload(ctx, "srv.items", P.items);
    P.d_hubs = upload(ctx, "srv.hubs", P.hubs);
    P.d_cta_seg = upload(ctx, "srv.ctaseg", P.cta_seg);
    P.d_tiles = upload(ctx, "srv.tiles", P.tiles);
    StartSource src{};
    src.kind = SRC_RADEMACHER;
    src.gaussian = S->opt.gaussian_probes != 0;
    src.ncols = S->block;
    src.seg_seed = upload(ctx, "srv.seeds", seeds);
    src.seg_col0 = upload(ctx, "srv.col0", col0);
    BlockOut out;
    check_ks<float>(ctx, ks);
    ctx->last_steps = 0;
    run_block<float>(ctx, P, src, nullptr, S->block, ks, S->m, false, false, true, "srv", out, variant, false,
                     S->opt.graphs != 0);
    std::vector<double> psi = download(ctx, out.psi, out.SK);
    // statistics and retirement
    std::vector<int> still;
    for (size_t sidx = 0; sidx < S->active.size(); sidx++) {
        const int idx = S->active[sidx];
        vne_server::Req& rq = S->reqs[idx];
        for (int c = 0; c < S->block; c++) {  // Welford update
            const double x = psi[sidx * out.Kp + c];
            rq.nvec++;
            const double d = x - rq.mean;
            rq.mean += d / (double)rq.nvec;
            rq.m2 += d * (x - rq.mean);
        }
        rq.blocks++;
        rq.est = rq.mean;
        rq.se = rq.nvec > 1 ? sqrt(rq.m2 / (double)(rq.nvec - 1) / (double)rq.nvec) : 0.0;
        const bool converged = rq.blocks >= 2 && 2.576 * rq.se <= 0.5 * rq.eps * fabs(rq.mean);
        if (converged || rq.nvec >= rq.max_vectors) {
            rq.state = 2;
            rq.done_tick = S->tick;
            S->used -= rq.footprint;
            if (completed) (*completed)++;
        } else {
            still.push_back(idx);
        }
    }
    S->active.swap(still);
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
