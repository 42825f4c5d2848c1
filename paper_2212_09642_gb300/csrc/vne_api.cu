// libvne C ABI: contexts, density matrices, the block Krylov engine and the
// trace estimators of Benzi, Rinelli, Simunec (arXiv 2212.09642).
//
// Engine overview.  A "problem" is a packed CSR operator M (one graph, or
// several graphs block-diagonally, each a segment) with a warp-level work
// schedule.  A block of K probe columns runs m Lanczos steps at once: per
// step one fused SpMM kernel and one update kernel (kernels_lanczos.cu), all
// launched back to back on the context stream with no host synchronisation;
// then one FP64 tridiagonal-quadrature kernel gives psi for every column.
//
// Probe generator (identical to the oracle's, written independently):
//   mix64 = SplitMix64 output mixer (Steele, Lea, Flood 2014),
//   s = mix64(seed + 0x9E3779B97F4A7C15),
//   h(j, i) = mix64((((j << 32) | i) ^ s) + 0x9E3779B97F4A7C15),
//   entry = +1 if the top bit of h is 0 else -1,
// j the global probe column, i the node id in the caller's numbering.
#include <cuda_runtime.h>
#include <math.h>
#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <tuple>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/vne.h"
#include "host_graph.h"
#include "kernels.h"

using namespace vne;

// ---------------------------------------------------------------------------
// context, errors, workspace

struct WsBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Per-kernel live timing (CUDA events on the context stream around each
// launch of the step and update kernels), enabled by vne_ctx_profile.
struct KernelStat {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;  // algorithmic bytes of the timed launches
};

struct Problem;

struct vne_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    std::map<std::string, WsBuf> ws;
    int64_t launches = 0;  // kernels launched by this context
    int last_cg_iters = 0; // largest multi-shift CG iteration count of the last rational call
    bool profile = false;
    KernelStat stat[4];    // 0: step (SpMM) kernel, 1: update kernel, 2: CG update, 3: CG direction
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Pending> pending;
    size_t ev_next = 0;
    bool time_steps = false;          // autotuner: time the whole step loop
    cudaEvent_t loop_ev[2] = {nullptr, nullptr};
    // autotuned schedules, shared by matrices of the same shape
    struct TuneKey {
        int64_t n, nnz, maxdeg;
        int fp64, pattern;
        bool operator<(const TuneKey& o) const {
            return std::tie(n, nnz, maxdeg, fp64, pattern) < std::tie(o.n, o.nnz, o.maxdeg, o.fp64, o.pattern);
        }
    };
    std::map<TuneKey, std::array<int, 4>> tune_cache;
    // CUDA graphs of step loops, keyed by the launch parameters of the loop;
    // a loop is captured the second time its key is seen
    struct LoopGraph {
        cudaGraphExec_t exec;
        int64_t kernels;  // kernel launches the graph holds
    };
    std::map<std::string, LoopGraph> graphs;
    std::map<std::string, int> graph_seen;
    cudaStream_t cap_stream = nullptr;  // private stream the captures run on
    int64_t graphs_captured = 0, graphs_replayed = 0;
    int last_steps = 0;  // Lanczos steps of the last quadrature call (largest over its blocks)
    int last_poly_dim = 0;  // polynomial dimension chosen by the switching rule (last rational call)
    // packed layout of the last batch of matrices (vne_batch_hutchinson),
    // kept for repeated estimates over the same batch; key = the matrices'
    // creation ids and the plan parameters
    Problem* batch_prob = nullptr;
    // device colourings: streams of the jobs after the first, pinned counters
    std::vector<cudaStream_t> color_streams;
    std::vector<cudaEvent_t> color_events;
    int32_t* pinned_ctr = nullptr;
    // pinned host staging of the matrix assembly (reused; every assembly
    // ends with a stream synchronisation, so no copy from it is in flight)
    std::map<std::string, std::pair<void*, size_t>> pinned;
    std::vector<uint64_t> batch_key;
    int batch_ks = 0;
};

struct vne_matrix {
    vne_ctx* ctx = nullptr;
    uint64_t uid = 0;               // creation id, unique within the process
    int64_t n = 0, nnz = 0;
    bool fp64 = false, pattern = false, desing = false;
    double trace = 0.0, scale = 1.0, normM = 0.0;
    std::vector<int64_t> h_rowptr;  // packed (possibly relabelled) numbering
    std::vector<int32_t> h_col;     // host copy of d_col, made on first use (host_cols)
    std::vector<int32_t> perm;      // packed row -> caller node id (empty: identity)
    int32_t* d_rowptr = nullptr;
    int32_t* d_col = nullptr;
    void* d_vals = nullptr;
    int32_t* d_node_id = nullptr;
    Problem* prob = nullptr;        // cached schedule
    int prob_item_nnz = -1;
    bool tuned = false;             // autotuned schedule (vne_autotune)
    int tuned_panel = 0, tuned_item_nnz = 0, tuned_variant = 0;
    bool tuned_interleave = false;
    int64_t maxdeg = 0;
};

namespace {

struct Error {
    vne_status code;
};

void set_err(vne_ctx* ctx, const char* fmt, ...) {
    if (!ctx) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
}

#define VNE_TRY_CUDA(ctx, call)                                                                        \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            set_err((ctx), "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            throw Error{e_ == cudaErrorMemoryAllocation ? VNE_ENOMEM : VNE_EDEVICE};                     \
        }                                                                                              \
    } while (0)

#define VNE_REQUIRE(ctx, cond, code, ...)     \
    do {                                      \
        if (!(cond)) {                        \
            set_err((ctx), __VA_ARGS__);      \
            throw Error{(code)};              \
        }                                     \
    } while (0)

// Workspace buffers grow on demand and are kept for the life of the context,
// so the hot loop never allocates.  New allocations are zero-filled (the
// cross-CTA counters rely on starting at zero; the kernels reset them after
// use).  zero = true clears the requested bytes on every call.
void* ws_get(vne_ctx* ctx, const std::string& name, size_t bytes, bool zero = false) {
    WsBuf& b = ctx->ws[name];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        size_t alloc = std::max<size_t>(bytes, 256);
        VNE_TRY_CUDA(ctx, cudaMalloc(&b.ptr, alloc));
        VNE_TRY_CUDA(ctx, cudaMemsetAsync(b.ptr, 0, alloc, ctx->stream));
        b.bytes = alloc;
    }
    if (zero && bytes) VNE_TRY_CUDA(ctx, cudaMemsetAsync(b.ptr, 0, bytes, ctx->stream));
    return b.ptr;
}

template <typename T>
T* ws_get_t(vne_ctx* ctx, const std::string& name, size_t count, bool zero = false) {
    return (T*)ws_get(ctx, name, count * sizeof(T), zero);
}

// Pinned host buffer `name` of at least `count` elements (grown on demand).
template <typename T>
T* pinned_get(vne_ctx* ctx, const std::string& name, size_t count) {
    auto& b = ctx->pinned[name];
    const size_t bytes = std::max<size_t>(count * sizeof(T), 64);
    if (b.second < bytes) {
        if (b.first) cudaFreeHost(b.first);
        b.first = nullptr;
        b.second = 0;
        if (cudaMallocHost(&b.first, bytes) != cudaSuccess) {
            b.first = nullptr;
            return nullptr;
        }
        b.second = bytes;
    }
    return (T*)b.first;
}

template <typename T>
T* upload(vne_ctx* ctx, const std::string& name, const std::vector<T>& v) {
    T* d = ws_get_t<T>(ctx, name, std::max<size_t>(v.size(), 1));
    if (!v.empty())
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return d;
}

// Host copy of the stored column indices (device order), made on first use.
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

// Resolve the recorded event pairs (the stream must be synchronised).
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

}  // namespace

// ---------------------------------------------------------------------------
// schedule ("plan") of a packed operator

struct Problem {
    bool fp64 = false, valued = false;
    int32_t n_total = 0, nseg = 0;
    int64_t nnz_total = 0;
    const int32_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const void* vals = nullptr;
    const int32_t* node_id = nullptr;
    std::vector<SegInfo> segs;
    std::vector<WorkItem> items;
    std::vector<HubRow> hubs;
    std::vector<int32_t> cta_seg;
    std::vector<RowTile> tiles;
    int32_t hub_slots = 0;
    int32_t stage_nnz = 0;   // largest item (nonzeros)
    // device copies (owned)
    SegInfo* d_segs = nullptr;
    WorkItem* d_items = nullptr;
    HubRow* d_hubs = nullptr;
    int32_t* d_cta_seg = nullptr;
    RowTile* d_tiles = nullptr;
    std::vector<void*> owned;  // extra device buffers owned by the problem (batch packing)
    bool owns_tables = true;   // false: the tables live in context workspace
    ~Problem() {
        if (owns_tables) {
            cudaFree(d_segs);
            cudaFree(d_items);
            cudaFree(d_hubs);
            cudaFree(d_cta_seg);
            cudaFree(d_tiles);
        }
        for (void* p : owned) cudaFree(p);
    }
    int ctas_per_panel() const { return (int)(items.size() / VNE_WARPS); }
    int tiles_per_panel() const { return (int)tiles.size(); }
};

namespace {

const int kTileRows = 4096;

// Work items of one segment (rows [row_begin, row_begin + rows) of the packed
// CSR): runs of short rows with about `target` nonzeros (at most 64 rows),
// and rows longer than `long_thresh` split into chunks of `chunk` nonzeros.
void plan_segment(const int64_t* rowptr, int32_t row_begin, int32_t rows, int32_t seg, int target, Problem& P) {
    // every item holds at most `target` nonzeros: short rows are packed into
    // runs (at most 64 rows), rows longer than `target` are split into chunks
    const int64_t chunk = std::max(target, 32);
    const int max_rows = 64;
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
    while ((P.items.size() - first_item) % VNE_WARPS) P.items.push_back(WorkItem{0, 0, 0, 0});
    for (size_t i = first_item; i < P.items.size(); i++)
        P.stage_nnz = std::max<int32_t>(P.stage_nnz, P.items[i].nnz_end - P.items[i].nnz_begin);
    SegInfo& sg = P.segs[seg];
    sg.hub_count = (int32_t)P.hubs.size() - sg.hub_begin;
    sg.cta_begin = (int32_t)(first_item / VNE_WARPS);
    sg.cta_count = (int32_t)((P.items.size() - first_item) / VNE_WARPS);
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

template <typename T>
T* dev_copy(vne_ctx* ctx, const std::vector<T>& v) {
    T* d = nullptr;
    size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    VNE_TRY_CUDA(ctx, cudaMalloc(&d, bytes));
    if (!v.empty()) VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return d;
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

struct Sched {
    int ks, item_nnz, variant;
    bool interleave;
    bool graph;
};

int choose_panel(bool fp64, const vne_options* opt, int64_t n);

// Schedule for a call: explicit options win, then the matrix's autotuned
// choice, then the built-in defaults.
Sched resolve_sched(const vne_matrix* M, const vne_options* o) {
    Sched s;
    s.ks = (o && o->panel > 0) ? o->panel : (M->tuned ? M->tuned_panel : choose_panel(M->fp64, o, M->n));
    s.item_nnz = (o && o->item_nnz > 0) ? o->item_nnz : (M->tuned ? M->tuned_item_nnz : 256);
    s.variant = (o && o->step_variant >= 0) ? o->step_variant : (M->tuned ? M->tuned_variant : 4);
    if (M->fp64) s.variant = 0;
    s.interleave = (o && o->interleave >= 0) ? (o->interleave != 0) : (M->tuned ? M->tuned_interleave : false);
    s.graph = !(o && o->graphs == 0);
    return s;
}

Problem* matrix_problem(vne_matrix* M, const vne_options* opt) {
    int target = resolve_sched(M, opt).item_nnz;
    double taurel = (opt && opt->breakdown_tol > 0) ? opt->breakdown_tol : default_tau(M->fp64);
    if (M->prob && M->prob_item_nnz == target && M->prob->segs[0].tau == taurel * M->normM) return M->prob;
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

struct BlockOut {
    int K = 0, Kp = 0, ks = 0, panels = 0, m = 0, SK = 0;
    double* alpha = nullptr;   // [m][SK]
    double* beta = nullptr;    // [m][SK]
    double* sigma = nullptr;   // [m+1][SK]
    double* norm2 = nullptr;   // [SK]
    double* psi = nullptr;     // [SK]
    double* scale = nullptr;   // [SK]
    void* basis = nullptr;     // slot 0 (when kept)
    size_t slot_stride = 0;    // elements
};

std::vector<double> download(vne_ctx* ctx, const double* d, size_t count);

// Adaptive stopping of a block (Theorem 4.4): after every `check` steps the
// quadratures and the error estimates of all columns are computed; the block
// stops once every estimate is at most tol x |psi|, or, with `abs`, at most
// abs[c] for each real column c of the block.
struct Adaptive {
    double tol = 0.0;
    int check = 5;
    double lam_min = 0.0;  // <= 0: half the smallest positive Ritz value per column
    double lam_max = 0.0;
    int grid = 1000;
    const double* abs = nullptr;  // per-column absolute tolerances of this block
    int ncols = 0;                // real columns covered by `abs`
};

template <typename T>
void run_block(vne_ctx* ctx, Problem& P, const StartSource& src, const T* panel_src, int K, int ks, int m,
               bool reorth, bool keep_basis, bool desing, const std::string& tag, BlockOut& out, int variant = 0,
               bool interleave = false, bool graph = true, bool want_psi = true, const Adaptive* ad = nullptr) {
    cudaStream_t st = ctx->stream;
    const int panels = (K + ks - 1) / ks;
    const int Kp = panels * ks;
    const int S = P.nseg;
    const int SK = S * Kp;
    const size_t slot_elems = (size_t)Kp * P.n_total;
    const bool store_all = keep_basis || reorth;
    const int nslots = store_all ? m + 1 : 2;
    VNE_REQUIRE(ctx, reorth == false || S == 1, VNE_EUNSUPPORTED, "full reorthogonalisation needs a single matrix");
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
            if (reorth && j < m + 1) {
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
        const void* ptrs[] = {slots, alpha, beta, sigma, rcoef, rpart};
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

bool want_reorth(const vne_matrix* M, const vne_options* o) {
    int r = o ? o->reorth : -1;
    if (r < 0) return M->fp64;
    return r != 0;
}

int block_limit(const vne_options* o) { return (o && o->block > 0) ? o->block : 256; }

vne_options defaults() {
    vne_options o;
    vne_options_default(&o);
    return o;
}

template <typename T>
void check_ks(vne_ctx* ctx, int ks) {
    bool ok = sizeof(T) == 4 ? (ks == 8 || ks == 16 || ks == 32) : (ks == 4 || ks == 8 || ks == 16);
    VNE_REQUIRE(ctx, ok, VNE_EINVAL, "panel width %d not supported for this precision", ks);
}

// Quadratic forms of one source over all its columns, in blocks.
template <typename T>
std::vector<double> quadforms(vne_matrix* M, const vne_options* o, StartSource src, int ncols, int m,
                              const double* abs_tol = nullptr) {
    vne_ctx* ctx = M->ctx;
    Problem* P = matrix_problem(M, o);
    Sched sc = resolve_sched(M, o);
    int ks = sc.ks;
    check_ks<T>(ctx, ks);
    int lim = block_limit(o);
    bool reorth = want_reorth(M, o);
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

// Rational Krylov quadratic forms (poles -shifts[i] and n_inf poles at
// infinity) of one start block, by multi-shift CG.
template <typename T>
void rational_block(vne_ctx* ctx, Problem& P, const StartSource& src, int K, int ks, const double* shifts,
                    int nshift, int n_inf, double tol, int max_iter, bool desing, int variant, double drop,
                    double drop2, std::vector<double>& psi, std::vector<int>& iters, std::vector<double>& resid,
                    int* rank_min, double lam_min = 0.0, double lam_max = 0.0, int* kpoly_out = nullptr) {
    cudaStream_t st = ctx->stream;
    VNE_REQUIRE(ctx, P.nseg == 1, VNE_EUNSUPPORTED, "rational mode needs a single matrix");
    VNE_REQUIRE(ctx, nshift >= 1 && nshift <= 8, VNE_EINVAL, "1..8 finite poles are supported");
    VNE_REQUIRE(ctx, n_inf >= -1 && n_inf <= 3, VNE_EINVAL, "0..3 poles at infinity (or -1: switching rule)");
    // n_inf = -1: the polynomial part K_k(A, c) is chosen by the switching
    // rule of Section 5.3 (ell = 3, c = 0.75) from the polynomial error
    // estimates of the first kMixMax CG iterations, and spanned by the seed
    // CG residuals r_0..r_{k-1} (orthogonal, the Lanczos directions of A)
    constexpr int kMixMax = 16, kMixEll = 3;
    constexpr double kMixC = 0.75;
    const bool mixed = n_inf < 0;
    const int panels = (K + ks - 1) / ks, Kp = panels * ks;
    const int n = P.n_total;
    const size_t blk = (size_t)Kp * n;
    const int tiles = P.tiles_per_panel();
    // seed system: the smallest shift
    int s0i = 0;
    for (int i = 1; i < nshift; i++)
        if (shifts[i] < shifts[s0i]) s0i = i;
    const double s0 = shifts[s0i];
    const double scale = P.segs[0].scale;
    // start block c (desingularised probes), norms
    T* C = ws_get_t<T>(ctx, "rat.c", blk);
    double* norm2 = ws_get_t<double>(ctx, "rat.norm2", Kp);
    double* sig1 = ws_get_t<double>(ctx, "rat.sig1", Kp);
    {
        StartParams<T> sp{};
        sp.src = src;
        sp.node_id = P.node_id;
        sp.seg = P.d_segs;
        sp.nseg = 1;
        sp.K = Kp;
        sp.n_total = n;
        sp.tiles_per_panel = tiles;
        sp.tiles = P.d_tiles;
        sp.desing = desing ? 1 : 0;
        sp.w1 = C;
        sp.mean = ws_get_t<double>(ctx, "mean", Kp);
        sp.norm2 = norm2;
        sp.sig1 = sig1;
        sp.part = ws_get_t<double>(ctx, "part", (size_t)panels * tiles * ks);
        sp.counter = ws_get_t<uint32_t>(ctx, "counter", (size_t)panels, true);
        VNE_TRY_CUDA(ctx, launch_start<T>(sp, ks, panels, st));
    }
    // CG vectors
    CgVectors<T> v{};
    v.n = n;
    v.tiles_per_panel = tiles;
    v.tiles = P.d_tiles;
    v.r = ws_get_t<T>(ctx, "rat.r", blk);
    v.q = ws_get_t<T>(ctx, "rat.q", blk);
    v.p = ws_get_t<T>(ctx, "rat.p", blk);
    T* xs = ws_get_t<T>(ctx, "rat.x", blk * nshift);
    T* pss = ws_get_t<T>(ctx, "rat.ps", blk * nshift);
    for (int i = 0; i < nshift; i++) {
        v.x[i] = xs + (size_t)i * blk;
        v.ps[i] = pss + (size_t)i * blk;
    }
    v.part = ws_get_t<double>(ctx, "rat.part", (size_t)panels * tiles * ks);
    v.counter = ws_get_t<uint32_t>(ctx, "rat.counter", (size_t)panels, true);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(v.r, C, blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(v.p, C, blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
    VNE_TRY_CUDA(ctx, cudaMemsetAsync(xs, 0, blk * nshift * sizeof(T), st));
    for (int i = 0; i < nshift; i++)
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(v.ps[i], C, blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
    // scalar state
    CgState cs{};
    cs.K = Kp;
    cs.nshift = nshift;
    cs.scale = scale;
    cs.shift0 = s0;
    cs.tol = tol;
    std::vector<double> hsh(shifts, shifts + nshift);
    cs.shift = upload(ctx, "rat.shifts", hsh);
    double* dq = ws_get_t<double>(ctx, "rat.dq", Kp);
    cs.dq = dq;
    double* sc = ws_get_t<double>(ctx, "rat.scalars", (size_t)Kp * (7 + 6 * nshift));
    cs.rho = sc;
    cs.rho_new = sc + Kp;
    cs.a = sc + 2 * Kp;
    cs.b = sc + 3 * Kp;
    cs.a_prev = sc + 4 * Kp;
    cs.b_prev = sc + 5 * Kp;
    cs.cnorm = sc + 6 * Kp;
    double* sh = sc + 7 * Kp;
    cs.zeta = sh;
    cs.zeta_prev = sh + (size_t)nshift * Kp;
    cs.zeta_next = sh + 2 * (size_t)nshift * Kp;
    cs.as = sh + 3 * (size_t)nshift * Kp;
    cs.bs = sh + 4 * (size_t)nshift * Kp;
    cs.resid = sh + 5 * (size_t)nshift * Kp;
    int32_t* ibuf = ws_get_t<int32_t>(ctx, "rat.ints", (size_t)2 * nshift * Kp + 1);
    cs.active = ibuf;
    cs.iters = ibuf + (size_t)nshift * Kp;
    cs.any_active = ibuf + 2 * (size_t)nshift * Kp;
    VNE_TRY_CUDA(ctx, launch_cg_init(cs, norm2, st));
    ctx->launches += 1;
    double* ah = mixed ? ws_get_t<double>(ctx, "rat.ahist", (size_t)kMixMax * Kp) : nullptr;
    double* bh = mixed ? ws_get_t<double>(ctx, "rat.bhist", (size_t)kMixMax * Kp) : nullptr;
    T* rh = mixed ? ws_get_t<T>(ctx, "rat.rhist", blk * (kMixMax - 1)) : nullptr;  // r_1 .. r_{kMixMax-1}
    int it = 0;
    for (; it < max_iter; it++) {
        apply_operator<T>(ctx, P, ks, Kp, v.p, v.q, s0, dq, variant, "rat.op");
        VNE_TRY_CUDA(ctx, launch_cg_scalars_a(cs, st));
        if (mixed && it < kMixMax)
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(ah + (size_t)it * Kp, cs.a, Kp * sizeof(double),
                                              cudaMemcpyDeviceToDevice, st));
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
        if (ctx->profile) {
            e0 = ctx_event(ctx);
            VNE_TRY_CUDA(ctx, cudaEventRecord(e0, st));
        }
        VNE_TRY_CUDA(ctx, launch_cg_update<T>(v, cs, ks, panels, st));
        if (ctx->profile) {
            e1 = ctx_event(ctx);
            VNE_TRY_CUDA(ctx, cudaEventRecord(e1, st));
        }
        if (mixed && it + 1 < kMixMax)
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(rh + (size_t)it * blk, v.r, blk * sizeof(T), cudaMemcpyDeviceToDevice,
                                              st));
        VNE_TRY_CUDA(ctx, cudaMemsetAsync(cs.any_active, 0, sizeof(int32_t), st));
        VNE_TRY_CUDA(ctx, launch_cg_scalars_b(cs, st));
        if (mixed && it < kMixMax)
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(bh + (size_t)it * Kp, cs.b, Kp * sizeof(double),
                                              cudaMemcpyDeviceToDevice, st));
        if (ctx->profile) {
            e2 = ctx_event(ctx);
            VNE_TRY_CUDA(ctx, cudaEventRecord(e2, st));
        }
        VNE_TRY_CUDA(ctx, launch_cg_direction<T>(v, cs, ks, panels, st));
        ctx->launches += 4;
        if (ctx->profile) {
            e3 = ctx_event(ctx);
            VNE_TRY_CUDA(ctx, cudaEventRecord(e3, st));
            // algorithmic bytes of the seed part: update reads r, q, writes r;
            // direction reads r, p, writes p.  The per-shift part (update:
            // p_s and x_s read and written) is added after the loop from the
            // iterations each shift stayed active.
            const double vec = (double)n * K * sizeof(T);
            ctx->pending.push_back({2, e0, e1, vec * 3.0});
            ctx->pending.push_back({3, e2, e3, vec * 3.0});
        }
        if ((it & 7) == 7 || it + 1 == max_iter) {
            int32_t any = 0;
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(&any, cs.any_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
            if (!any) {
                it++;
                break;
            }
        }
    }
    // polynomial part: K_{n_inf+1}(A, c) by powers of A, or, with the
    // switching rule, K_k(A, c) by the seed residuals
    int kpoly = n_inf + 1;
    if (mixed) {
        const int kk = std::min(kMixMax, it);  // CG iterations recorded
        double* tdiag = ws_get_t<double>(ctx, "rat.tdiag", (size_t)kMixMax * Kp);
        double* toff = ws_get_t<double>(ctx, "rat.toff", (size_t)kMixMax * Kp);
        double* est = ws_get_t<double>(ctx, "rat.est", (size_t)kMixMax * Kp);
        double* blo = ws_get_t<double>(ctx, "rat.blo", (size_t)2 * Kp);
        double* ones = upload(ctx, "rat.ones", std::vector<double>(Kp, 1.0));
        // breakdown threshold of the Lanczos engine, in units of A
        const double tau_a = P.segs[0].tau * P.segs[0].scale;
        VNE_TRY_CUDA(ctx, launch_cg_tridiag(ah, bh, Kp, kk, s0, tau_a, tdiag, toff, st));
        for (int k = 1; k <= kk; k++)
            VNE_TRY_CUDA(ctx, launch_tridiag_bounds(tdiag, toff, norm2, ones, Kp, k, Kp, lam_min, lam_max, 1000, blo,
                                                    blo + Kp, est + (size_t)(k - 1) * Kp, st));
        ctx->launches += 1 + kk;
        std::vector<double> he = download(ctx, est, (size_t)std::max(kk, 1) * Kp);
        // per column: the first k with err_k / err_{k-ell-1} >= c^ell (an
        // estimate of 0: the Krylov space is invariant); the block takes
        // the largest k
        kpoly = 1;
        for (int c = 0; c < K; c++) {
            int kc = kk;
            for (int k = 1; k <= kk; k++) {
                const double e = he[(size_t)(k - 1) * Kp + c];
                if (e == 0.0 || (k >= kMixEll + 2 && e / he[(size_t)(k - kMixEll - 2) * Kp + c] >=
                                                       std::pow(kMixC, kMixEll))) {
                    kc = k;
                    break;
                }
            }
            kpoly = std::max(kpoly, kc);
        }
        kpoly = std::max(1, std::min(kpoly, kk > 0 ? kk : 1));
    }
    if (kpoly_out) *kpoly_out = mixed ? kpoly : 0;
    // basis W = [polynomial part, x_1..x_S] and A W
    const int nb = kpoly + nshift;
    T* apow = ws_get_t<T>(ctx, "rat.apow", blk * kpoly);
    std::vector<const T*> W(nb), AW(nb);
    W[0] = C;
    if (mixed) {
        for (int j = 1; j < kpoly; j++) W[j] = rh + (size_t)(j - 1) * blk;
        for (int j = 0; j < kpoly; j++) {
            apply_operator<T>(ctx, P, ks, Kp, W[j], apow + (size_t)j * blk, 0.0, dq, variant, "rat.op0");
            AW[j] = apow + (size_t)j * blk;
        }
    } else {
        const T* prev = C;
        for (int j = 0; j < kpoly; j++) {
            T* out = apow + (size_t)j * blk;
            apply_operator<T>(ctx, P, ks, Kp, prev, out, 0.0, dq, variant, "rat.op0");
            prev = out;
        }
        for (int j = 1; j < kpoly; j++) W[j] = apow + (size_t)(j - 1) * blk;
        for (int j = 0; j < kpoly; j++) AW[j] = apow + (size_t)j * blk;
    }
    for (int i = 0; i < nshift; i++)  // A x_s into the (now free) direction buffers
        apply_operator<T>(ctx, P, ks, Kp, v.x[i], v.ps[i], 0.0, dq, variant, "rat.op0");
    for (int i = 0; i < nshift; i++) {
        W[kpoly + i] = v.x[i];
        AW[kpoly + i] = v.ps[i];
    }
    // Gram matrices of (W, A W), Cholesky-QR2: pass 1 basis change X1, then
    // the Gram matrices of (W X1, A W X1) for the final orthonormalisation.
    // Both are symmetric (W^T A W since A is): the pairs a <= b are formed
    // and mirrored.
    auto gram_pairs = [&](const std::vector<const T*>& Wv, const std::vector<const T*>& AWv, double* out) {
        // one pass over the 2 nb vectors (k_multi_gram); the pairs a <= b of
        // W.W then W.AW, mirrored into the full [nb][nb] layouts
        const int nu = nb * (nb + 1) / 2, npairs = 2 * nu;
        MultiGram<T> mg{};
        mg.n = n;
        mg.panels = panels;
        mg.ks = ks;
        mg.nb = nb;
        for (int a = 0; a < nb; a++) {
            mg.w[a] = Wv[a];
            mg.aw[a] = AWv[a];
        }
        const int groups = (npairs * ks + VNE_THREADS * 16 - 1) / (VNE_THREADS * 16);
        const int want = std::max(1, 4 * std::max(ctx->sm_count, 1) / std::max(1, panels * groups));
        mg.chunks = std::max(1, std::min(want, (n + 15) / 16));
        mg.part = ws_get_t<double>(ctx, "rat.mgpart", (size_t)panels * groups * mg.chunks * VNE_THREADS * 16);
        double* uniq = ws_get_t<double>(ctx, "rat.uniq", (size_t)npairs * Kp);
        VNE_TRY_CUDA(ctx, launch_multi_gram<T>(mg, uniq, st));
        VNE_TRY_CUDA(ctx, launch_gram_mirror(uniq, nb, Kp, out, st));
        VNE_TRY_CUDA(ctx, launch_gram_mirror(uniq + (size_t)nu * Kp, nb, Kp, out + (size_t)nb * nb * Kp, st));
        ctx->launches += 4;
    };
    const size_t gsz = (size_t)2 * nb * nb * Kp;
    double* gram = ws_get_t<double>(ctx, "rat.gram", gsz);
    double* gram2 = ws_get_t<double>(ctx, "rat.gram2", gsz);
    double* X1 = ws_get_t<double>(ctx, "rat.X1", (size_t)nb * nb * Kp);
    gram_pairs(W, AW, gram);
    VNE_TRY_CUDA(ctx, launch_rational_pass1(gram, nb, Kp, drop, X1, st));
    T* tw = ws_get_t<T>(ctx, "rat.tw", blk * nb);
    T* taw = ws_get_t<T>(ctx, "rat.taw", blk * nb);
    std::vector<const T*> W1(nb), AW1(nb);
    for (int dir = 0; dir < 2; dir++) {
        BlockTransform<T> bt{};
        bt.n = n;
        bt.K = Kp;
        bt.nb = nb;
        bt.tiles_per_panel = tiles;
        bt.tiles = P.d_tiles;
        bt.X = X1;
        T* base = dir == 0 ? tw : taw;
        for (int i = 0; i < nb; i++) {
            bt.in[i] = dir == 0 ? W[i] : AW[i];
            bt.out[i] = base + (size_t)i * blk;
            (dir == 0 ? W1 : AW1)[i] = bt.out[i];
        }
        VNE_TRY_CUDA(ctx, launch_block_transform<T>(bt, ks, panels, st));
    }
    gram_pairs(W1, AW1, gram2);
    double* dpsi = ws_get_t<double>(ctx, "rat.psi", Kp);
    int* drank = ws_get_t<int>(ctx, "rat.rank", Kp);
    // ||c||^2 is the (0,0) entry of the first Gram matrix
    VNE_TRY_CUDA(ctx, launch_rational_pass2(gram2, gram2 + (size_t)nb * nb * Kp, gram, nb, Kp, drop2, dpsi, drank, st));
    ctx->launches += 4;
    psi = download(ctx, dpsi, K);
    std::vector<int> hr(Kp), hit((size_t)nshift * Kp);
    std::vector<double> hres((size_t)nshift * Kp);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hr.data(), drank, Kp * sizeof(int), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hit.data(), cs.iters, hit.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hres.data(), cs.resid, hres.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->profile) {
        double shift_iters = 0.0;
        for (int i = 0; i < nshift; i++)
            for (int c = 0; c < K; c++) shift_iters += hit[(size_t)i * Kp + c];
        const double per = (double)n * sizeof(T);
        ctx->pending.push_back({2, nullptr, nullptr, shift_iters * per * 4.0});
        ctx_flush_profile(ctx);
    }
    iters.assign((size_t)nshift * K, 0);
    resid.assign((size_t)nshift * K, 0.0);
    for (int i = 0; i < nshift; i++)
        for (int c = 0; c < K; c++) {
            iters[(size_t)i * K + c] = hit[(size_t)i * Kp + c];
            resid[(size_t)i * K + c] = hres[(size_t)i * Kp + c];
        }
    int rmin = nb;
    for (int c = 0; c < K; c++) rmin = std::min(rmin, hr[c]);
    if (rank_min) *rank_min = rmin;
    (void)it;
}

template <typename T>
void rational_quadforms(vne_matrix* M, const vne_options* o, StartSource src, int ncols, const double* shifts,
                        int nshift, std::vector<double>& psi, std::vector<int>& iters, std::vector<double>& resid) {
    vne_ctx* ctx = M->ctx;
    Problem* P = matrix_problem(M, o);
    Sched sc = resolve_sched(M, o);
    check_ks<T>(ctx, sc.ks);
    const int lim = std::min(block_limit(o), 128);
    const double tol = (o && o->cg_tol > 0) ? o->cg_tol : 1e-8;
    const int maxit = (o && o->cg_max_iter > 0) ? o->cg_max_iter : 10000;
    const int n_inf = o ? o->n_inf_poles : 2;
    // a pole direction whose squared relative remainder after orthogonalising
    // against the earlier ones is below the threshold is dependent: FP64 uses
    // the oracle's rule (remainder 1e-6 of the norm); FP32 vectors stop at a
    // remainder of 1e-3, because a kept direction's A-image carries the
    // vectors' rounding amplified by 1 / remainder.  Both Cholesky-QR passes
    // apply the rule.
    const double drop = M->fp64 ? 1e-12 : 1e-6;
    const double drop2 = drop;
    psi.assign(ncols, 0.0);
    iters.assign((size_t)nshift * ncols, 0);
    resid.assign((size_t)nshift * ncols, 0.0);
    const double lam_min = o ? o->spectrum_min : 0.0, lam_max = M->normM * M->scale;
    ctx->last_poly_dim = 0;
    for (int b0 = 0; b0 < ncols; b0 += lim) {
        const int K = std::min(lim, ncols - b0);
        StartSource s = src;
        s.ncols = K;
        if (s.kind == SRC_RADEMACHER || s.kind == SRC_INDICATOR) s.col_begin = src.col_begin + b0;
        if (s.kind == SRC_DENSE64) s.dense = src.dense + b0;
        std::vector<double> bp, br;
        std::vector<int> bi;
        int rmin = 0, kpoly = 0;
        rational_block<T>(ctx, *P, s, K, sc.ks, shifts, nshift, n_inf, tol, maxit, M->desing, sc.variant, drop, drop2,
                          bp, bi, br, &rmin, lam_min, lam_max, &kpoly);
        ctx->last_poly_dim = std::max(ctx->last_poly_dim, kpoly);
        for (int c = 0; c < K; c++) psi[b0 + c] = bp[c];
        for (int i = 0; i < nshift; i++)
            for (int c = 0; c < K; c++) {
                iters[(size_t)i * ncols + b0 + c] = bi[(size_t)i * K + c];
                resid[(size_t)i * ncols + b0 + c] = br[(size_t)i * K + c];
            }
    }
}

std::vector<double> resolve_shifts(const vne_matrix* M, const double* poles, int num_poles) {
    std::vector<double> sh(num_poles);
    if (poles) {
        for (int i = 0; i < num_poles; i++) sh[i] = poles[i];
    } else {
        // default poles: log-spaced on [1e-4 ||A||_G, ||A||_G]
        const double lam = M->normM * M->scale;
        for (int i = 0; i < num_poles; i++)
            sh[i] = lam * pow(10.0, num_poles > 1 ? -4.0 * i / (num_poles - 1) : 0.0);
    }
    return sh;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

#define VNE_API_BEGIN try {
#define VNE_API_END(ctx)                                  \
    }                                                     \
    catch (const Error& e) {                              \
        return e.code;                                    \
    }                                                     \
    catch (const std::bad_alloc&) {                       \
        set_err((ctx), "host allocation failed");         \
        return VNE_ENOMEM;                                \
    }                                                     \
    catch (...) {                                         \
        set_err((ctx), "unexpected internal error");      \
        return VNE_EDEVICE;                               \
    }                                                     \
    return VNE_OK;

extern "C" void vne_options_default(vne_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->reorth = -1;
    o->n_inf_poles = 2;
    o->cg_max_iter = 10000;
    o->cg_tol = 1e-8;
    o->step_variant = -1;
    o->interleave = -1;
    o->graphs = -1;
}

extern "C" const char* vne_version(void) { return "vne 0.1 (sm_103a)"; }

extern "C" vne_status vne_ctx_create(int32_t device, vne_ctx** out) {
    if (!out) return VNE_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) return VNE_EDEVICE;
    if (device < 0 || device >= count) return VNE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VNE_EDEVICE;
    vne_ctx* c = new (std::nothrow) vne_ctx();
    if (!c) return VNE_ENOMEM;
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return VNE_OK;
}

extern "C" vne_status vne_ctx_destroy(vne_ctx* ctx) {
    if (!ctx) return VNE_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto& kv : ctx->ws)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->loop_ev)
        if (e) cudaEventDestroy(e);
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaStream_t sx : ctx->color_streams) cudaStreamDestroy(sx);
    for (cudaEvent_t e : ctx->color_events) cudaEventDestroy(e);
    if (ctx->pinned_ctr) cudaFreeHost(ctx->pinned_ctr);
    for (auto& kv : ctx->pinned)
        if (kv.second.first) cudaFreeHost(kv.second.first);
    delete ctx->batch_prob;
    delete ctx;
    return VNE_OK;
}

extern "C" vne_status vne_ctx_set_stream(vne_ctx* ctx, void* stream) {
    if (!ctx) return VNE_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return VNE_OK;
}

extern "C" const char* vne_last_error(const vne_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" vne_status vne_create_density_matrix(vne_ctx* ctx, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                     const double* vals, uint32_t flags, vne_matrix** out) {
    if (!ctx || !out) return VNE_EINVAL;
    *out = nullptr;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    const bool fp64 = flags & VNE_FP64, fp32 = flags & VNE_FP32;
    VNE_REQUIRE(ctx, fp64 != fp32, VNE_EINVAL, "exactly one of VNE_FP64 / VNE_FP32 is required");
    VNE_REQUIRE(ctx, n >= 1 && n < (int64_t)INT32_MAX, VNE_EINVAL, "n = %lld out of range", (long long)n);
    VNE_REQUIRE(ctx, row_ptr && col_idx, VNE_EINVAL, "row_ptr and col_idx are required");
    VNE_REQUIRE(ctx, !(vals && (flags & VNE_CHECK_SYMMETRY)), VNE_EUNSUPPORTED,
                "VNE_CHECK_SYMMETRY supports pattern matrices only");
    std::unique_ptr<vne_matrix> M(new vne_matrix());
    M->ctx = ctx;
    static std::atomic<uint64_t> next_uid{1};
    M->uid = next_uid.fetch_add(1);
    M->n = n;
    M->fp64 = fp64;
    M->pattern = (vals == nullptr);
    const bool dev = flags & VNE_INPUT_DEVICE;
    // Row pointers on the host (O(n)): monotonicity, degrees, the relabelling
    // and the work plan need them there.  One pass checks them, finds the
    // largest degree and writes the int32 copy for the device into pinned
    // staging; the uploads and the device validation of the columns then run
    // while the host builds the relabelling.
    std::vector<int64_t> rp_dev;
    const int64_t* rph = row_ptr;
    if (dev) {
        rp_dev.resize(n + 1);
        VNE_TRY_CUDA(ctx, cudaMemcpy(rp_dev.data(), row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        rph = rp_dev.data();
    }
    VNE_REQUIRE(ctx, rph[0] == 0, VNE_EINVAL, "row_ptr[0] must be 0");
    int32_t* rp32 = pinned_get<int32_t>(ctx, "asm.rp32", n + 1);
    VNE_REQUIRE(ctx, rp32, VNE_ENOMEM, "pinned staging of %lld row pointers", (long long)(n + 1));
    int64_t maxdeg = 0;
    const int64_t bad_row = check_row_offsets(n, rph, rp32, &maxdeg);
    if (bad_row >= 0) {
        VNE_REQUIRE(ctx, rph[bad_row + 1] >= rph[bad_row], VNE_EINVAL, "row_ptr not monotone at %lld",
                    (long long)bad_row);
        VNE_REQUIRE(ctx, false, VNE_EINVAL, "nnz = %lld exceeds int32", (long long)rph[bad_row + 1]);
    }
    const int64_t nnz = rph[n];
    M->nnz = nnz;
    // Columns (and values) on the device: the caller's device arrays, or one
    // copy of the host arrays into staging buffers.
    const int32_t* d_ci = col_idx;
    if (!dev) {
        int32_t* stage = ws_get_t<int32_t>(ctx, "asm.col", std::max<int64_t>(nnz, 1));
        if (nnz) VNE_TRY_CUDA(ctx, cudaMemcpyAsync(stage, col_idx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        d_ci = stage;
    }
    const double* d_va = vals;
    if (vals && !dev) {
        double* stage = ws_get_t<double>(ctx, "asm.vals", std::max<int64_t>(nnz, 1));
        if (nnz) VNE_TRY_CUDA(ctx, cudaMemcpyAsync(stage, vals, nnz * sizeof(double), cudaMemcpyHostToDevice, st));
        d_va = stage;
    }
    int32_t* d_rp_in = ws_get_t<int32_t>(ctx, "asm.rowptr", n + 1);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d_rp_in, rp32, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // column range and (pattern) self-loops, checked on the device
    unsigned long long* d_bad = ws_get_t<unsigned long long>(ctx, "asm.bad", 2);
    VNE_TRY_CUDA(ctx, launch_validate(d_rp_in, d_ci, n, vals ? 0 : 1, d_bad, st));
    unsigned long long* bad = pinned_get<unsigned long long>(ctx, "asm.bad", 2);
    VNE_REQUIRE(ctx, bad, VNE_ENOMEM, "pinned staging");
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(bad, d_bad, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    ctx->launches += 1;
    // degree-descending relabelling (stable in the node id), built while the
    // device validates: a counting sort over the degree classes; the packed
    // row pointers follow from the class sizes alone
    const bool by_degree = (flags & VNE_REORDER) && !(flags & VNE_REORDER_RCM);
    int32_t* order_pin = nullptr;
    int32_t* rp2_pin = nullptr;
    std::vector<int64_t> rp2;
    if (by_degree) {
        order_pin = pinned_get<int32_t>(ctx, "asm.order", n);
        rp2_pin = pinned_get<int32_t>(ctx, "asm.rp2", n + 1);
        VNE_REQUIRE(ctx, order_pin && rp2_pin, VNE_ENOMEM, "pinned staging of the relabelling");
        rp2.resize(n + 1);
        degree_relabel(n, rp32, maxdeg, order_pin, rp2.data(), rp2_pin);
    }
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    if (bad[0] != ~0ull || bad[1] != ~0ull) {
        const unsigned long long k = std::min(bad[0], bad[1]);
        const int64_t row = (int64_t)(std::upper_bound(rph, rph + n + 1, (int64_t)k) - rph) - 1;
        int32_t c = 0;
        VNE_TRY_CUDA(ctx, cudaMemcpy(&c, d_ci + k, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (k == bad[0]) VNE_REQUIRE(ctx, false, VNE_EINVAL, "column index %d out of range in row %lld", c, (long long)row);
        VNE_REQUIRE(ctx, false, VNE_EINVAL, "self-loop at node %lld (pattern Laplacian)", (long long)row);
    }
    // Host copies of columns / values only where a host pass needs them
    // (symmetry check; trace and Gershgorin bound of a valued matrix).
    std::vector<int32_t> hci;
    std::vector<double> hva;
    const bool need_host = vals || (flags & VNE_CHECK_SYMMETRY) || (flags & VNE_REORDER_RCM);
    if (need_host && nnz) {
        hci.resize(nnz);
        if (dev) VNE_TRY_CUDA(ctx, cudaMemcpy(hci.data(), col_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
        else memcpy(hci.data(), col_idx, nnz * sizeof(int32_t));
        if (vals) {
            hva.resize(nnz);
            if (dev) VNE_TRY_CUDA(ctx, cudaMemcpy(hva.data(), vals, nnz * sizeof(double), cudaMemcpyDeviceToHost));
            else memcpy(hva.data(), vals, nnz * sizeof(double));
        }
    }
    if (flags & VNE_CHECK_SYMMETRY) {
        for (int64_t i = 0; i < n; i++) std::sort(hci.begin() + rph[i], hci.begin() + rph[i + 1]);
        for (int64_t i = 0; i < n; i++)
            for (int64_t k = rph[i]; k < rph[i + 1]; k++) {
                int32_t j = hci[k];
                bool found = std::binary_search(hci.begin() + rph[j], hci.begin() + rph[j + 1], (int32_t)i);
                VNE_REQUIRE(ctx, found, VNE_ENOTSYM, "pattern not symmetric: (%lld,%d)", (long long)i, j);
            }
    }
    // trace, Gershgorin bound of the stored operator M, scale
    if (!vals) {
        M->trace = (double)nnz;
        M->normM = 2.0 * (double)maxdeg;
        M->desing = true;
    } else {
        double tr = 0.0, nm = 0.0;
        for (int64_t i = 0; i < n; i++) {
            double rs = 0.0;
            for (int64_t k = rph[i]; k < rph[i + 1]; k++) {
                if (hci[k] == i) tr += hva[k];
                rs += fabs(hva[k]);
            }
            nm = std::max(nm, rs);
        }
        M->trace = tr;
        M->normM = nm;
        M->desing = (flags & VNE_IS_LAPLACIAN) != 0;
    }
    bool normalize = !vals || (flags & VNE_NORMALIZE_TRACE);
    if (normalize) {
        VNE_REQUIRE(ctx, M->trace > 0.0, VNE_EINVAL, "trace must be positive to normalise (got %g)", M->trace);
        M->scale = 1.0 / M->trace;
    } else {
        M->scale = 1.0;
    }
    const size_t es = fp64 ? 8 : 4;
    VNE_TRY_CUDA(ctx, cudaMalloc(&M->d_rowptr, (n + 1) * sizeof(int32_t)));
    VNE_TRY_CUDA(ctx, cudaMalloc(&M->d_col, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
    if (vals) VNE_TRY_CUDA(ctx, cudaMalloc(&M->d_vals, std::max<int64_t>(nnz, 1) * es));
    if (by_degree) {
        // degree order built above; inverse permutation and the moved
        // nonzeros on the device
        int32_t* d_inv = ws_get_t<int32_t>(ctx, "asm.inv", n);
        VNE_TRY_CUDA(ctx, cudaMalloc(&M->d_node_id, n * sizeof(int32_t)));
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_node_id, order_pin, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_rowptr, rp2_pin, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        VNE_TRY_CUDA(ctx, launch_invert_perm(M->d_node_id, n, d_inv, st));
        VNE_TRY_CUDA(ctx, launch_relabel(d_rp_in, d_ci, d_va, M->d_rowptr, M->d_node_id, d_inv, n, M->d_col,
                                         M->d_vals, fp64 ? 1 : 0, st));
        ctx->launches += 2;
        M->perm.assign(order_pin, order_pin + n);
        VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));  // the pinned staging is reused by the next assembly
    } else if (flags & VNE_REORDER_RCM) {
        // relabelling (host): reverse Cuthill-McKee; the nonzeros are moved
        // on the device
        std::vector<int32_t> order = rcm_order(n, rph, hci.data());  // new -> old
        std::vector<int32_t> inv(n);
        for (int64_t i = 0; i < n; i++) inv[order[i]] = (int32_t)i;
        rp2.assign(n + 1, 0);
        for (int64_t i = 0; i < n; i++) rp2[i + 1] = rp2[i] + (rph[order[i] + 1] - rph[order[i]]);
        std::vector<int32_t> rp2_32(n + 1);
        for (int64_t i = 0; i <= n; i++) rp2_32[i] = (int32_t)rp2[i];
        int32_t* d_inv = upload(ctx, "asm.inv", inv);
        VNE_TRY_CUDA(ctx, cudaMalloc(&M->d_node_id, n * sizeof(int32_t)));
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_node_id, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_rowptr, rp2_32.data(), (n + 1) * sizeof(int32_t),
                                          cudaMemcpyHostToDevice, st));
        VNE_TRY_CUDA(ctx, launch_relabel(d_rp_in, d_ci, d_va, M->d_rowptr, M->d_node_id, d_inv, n, M->d_col,
                                         M->d_vals, fp64 ? 1 : 0, st));
        ctx->launches += 1;
        VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));  // host vectors above are sources of async copies
        M->perm = std::move(order);
    } else {
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_rowptr, d_rp_in, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        if (nnz) VNE_TRY_CUDA(ctx, cudaMemcpyAsync(M->d_col, d_ci, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        if (vals) {
            VNE_TRY_CUDA(ctx, launch_convert_values(d_va, nnz, M->d_vals, fp64 ? 1 : 0, st));
            ctx->launches += 1;
        }
        rp2.assign(rph, rph + n + 1);
        VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    }
    M->h_rowptr.swap(rp2);
    M->maxdeg = maxdeg;
    {
        auto it = ctx->tune_cache.find(vne_ctx::TuneKey{M->n, M->nnz, maxdeg, (int)M->fp64, (int)M->pattern});
        if (it != ctx->tune_cache.end()) {
            M->tuned = true;
            M->tuned_panel = it->second[0];
            M->tuned_item_nnz = it->second[1];
            M->tuned_variant = it->second[2];
            M->tuned_interleave = it->second[3] != 0;
        }
    }
    *out = M.release();
    VNE_API_END(ctx)
}

extern "C" vne_status vne_matrix_destroy(vne_matrix* M) {
    if (!M) return VNE_EINVAL;
    cudaSetDevice(M->ctx->device);
    if (M->ctx->stream) cudaStreamSynchronize(M->ctx->stream);
    delete M->prob;
    cudaFree(M->d_rowptr);
    cudaFree(M->d_col);
    cudaFree(M->d_vals);
    cudaFree(M->d_node_id);
    delete M;
    return VNE_OK;
}

extern "C" vne_status vne_matrix_info(const vne_matrix* M, int64_t* n, int64_t* nnz, double* trace, double* norm_bound) {
    if (!M) return VNE_EINVAL;
    if (n) *n = M->n;
    if (nnz) *nnz = M->nnz;
    if (trace) *trace = M->trace;
    if (norm_bound) *norm_bound = M->normM * M->scale;
    return VNE_OK;
}

extern "C" vne_status vne_quadform_batch(vne_matrix* M, const double* vectors, int32_t k, uint32_t vec_flags,
                              int32_t krylov_steps, const double* poles, int32_t num_poles, const vne_options* opt,
                              double* psi, double* alpha_beta) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, k >= 1 && vectors && psi, VNE_EINVAL, "need k >= 1, vectors and psi");
    const double* dvec = vectors;
    if (!(vec_flags & VNE_VECTORS_DEVICE)) {
        double* d = ws_get_t<double>(ctx, "qb.input", (size_t)M->n * k);
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, vectors, (size_t)M->n * k * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        dvec = d;
    }
    if (poles != nullptr || num_poles > 0) {
        // rational Krylov space: multi-shift CG
        VNE_REQUIRE(ctx, num_poles >= 1 && num_poles <= 8, VNE_EINVAL, "1..8 poles are supported");
        std::vector<double> sh = resolve_shifts(M, poles, num_poles);
        for (double v : sh) VNE_REQUIRE(ctx, v > 0.0, VNE_EINVAL, "poles must be negative reals (shifts > 0)");
        StartSource s{};
        s.kind = SRC_DENSE64;
        s.ld = k;
        s.dense = dvec;
        std::vector<double> ps, rs;
        std::vector<int> its;
        if (M->fp64) rational_quadforms<double>(M, &o, s, k, sh.data(), num_poles, ps, its, rs);
        else rational_quadforms<float>(M, &o, s, k, sh.data(), num_poles, ps, its, rs);
        std::copy(ps.begin(), ps.end(), psi);
        if (alpha_beta) {  // rational mode: report CG iterations and final residuals per shift
            for (int c = 0; c < k; c++)
                for (int i = 0; i < 2 * krylov_steps; i++) alpha_beta[(size_t)c * 2 * krylov_steps + i] = 0.0;
        }
        return VNE_OK;
    }
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    const int m = krylov_steps;
    Problem* P = matrix_problem(M, &o);
    Sched sc = resolve_sched(M, &o);
    int ks = sc.ks;
    bool reorth = want_reorth(M, &o);
    int lim = block_limit(&o);
    for (int b0 = 0; b0 < k; b0 += lim) {
        int K = std::min(lim, k - b0);
        StartSource s{};
        s.kind = SRC_DENSE64;
        s.ncols = K;
        s.ld = k;
        s.dense = dvec + b0;
        BlockOut out;
        if (M->fp64) {
            check_ks<double>(ctx, ks);
            run_block<double>(ctx, *P, s, nullptr, K, ks, m, reorth, false, M->desing, "q", out, sc.variant,
                              sc.interleave, sc.graph);
        } else {
            check_ks<float>(ctx, ks);
            run_block<float>(ctx, *P, s, nullptr, K, ks, m, reorth, false, M->desing, "q", out, sc.variant,
                             sc.interleave, sc.graph);
        }
        std::vector<double> h = download(ctx, out.psi, K);
        std::copy(h.begin(), h.end(), psi + b0);
        if (alpha_beta) {
            std::vector<double> a = download(ctx, out.alpha, (size_t)m * out.SK);
            std::vector<double> b = download(ctx, out.beta, (size_t)m * out.SK);
            for (int c = 0; c < K; c++)
                for (int j = 0; j < m; j++) {
                    alpha_beta[(size_t)(b0 + c) * 2 * m + j] = a[(size_t)j * out.SK + c] * M->scale;
                    alpha_beta[(size_t)(b0 + c) * 2 * m + m + j] = b[(size_t)j * out.SK + c] * M->scale;
                }
        }
    }
    VNE_API_END(ctx)
}

extern "C" vne_status vne_entropy_hutchinson(vne_matrix* M, int32_t num_vectors, int32_t krylov_steps, uint64_t seed,
                                  const vne_options* opt, double* estimate, double* std_error, double* psi_out) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, num_vectors >= 1 && estimate, VNE_EINVAL, "need num_vectors >= 1 and estimate");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    StartSource s{};
    s.kind = SRC_RADEMACHER;
    s.gaussian = o.gaussian_probes != 0;
    s.seed_mixed = seed_mix(seed);
    VNE_REQUIRE(ctx, o.probe_offset >= 0, VNE_EINVAL, "probe_offset must be >= 0");
    s.col_begin = o.probe_offset;
    std::vector<double> psi = M->fp64 ? quadforms<double>(M, &o, s, num_vectors, krylov_steps)
                                      : quadforms<float>(M, &o, s, num_vectors, krylov_steps);
    double mean = 0.0;
    for (double v : psi) mean += v;
    mean /= num_vectors;
    double var = 0.0;
    for (double v : psi) var += (v - mean) * (v - mean);
    var = num_vectors > 1 ? var / (num_vectors - 1) : 0.0;
    *estimate = mean;
    if (std_error) *std_error = sqrt(var / num_vectors);
    if (psi_out) std::copy(psi.begin(), psi.end(), psi_out);
    VNE_API_END(ctx)
}

namespace {

__global__ void k_gamma(const double* norm2, const double* sigma, const double* zvec, int m, int K, double* gamma) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * K) return;
    int c = idx % K;
    gamma[idx] = sqrt(norm2[c]) * sigma[idx] * zvec[idx];
}

template <typename T>
void hutchpp_impl(vne_matrix* M, const vne_options* o, int Nr, int NH, int m, uint64_t seed, double* estimate,
                  double* parts) {
    vne_ctx* ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    Problem* P = matrix_problem(M, o);
    const int n = (int)M->n;
    Sched sc = resolve_sched(M, o);
    int ks = sc.ks;
    check_ks<T>(ctx, ks);
    VNE_REQUIRE(ctx, Nr >= 1 && Nr <= 128 && NH >= 0 && NH <= 4096, VNE_EINVAL, "need 1 <= N_r <= 128, 0 <= N_H");
    const uint64_t sm = seed_mix(seed);
    // 1. sketch: Y = f(A) Omega by the Lanczos matvec approximation, basis kept
    StartSource s{};
    s.kind = SRC_RADEMACHER;
    s.gaussian = o && o->gaussian_probes != 0;
    s.seed_mixed = sm;
    s.col_begin = 0;
    s.ncols = Nr;
    BlockOut sk;
    ctx->last_steps = 0;
    // the sketch block only feeds f(A) Omega: its quadratures are not needed
    run_block<T>(ctx, *P, s, nullptr, Nr, ks, m, want_reorth(M, o), true, M->desing, "sketch", sk, sc.variant,
                 sc.interleave, sc.graph, false);
    const int Kp = sk.Kp;
    double* zvec = ws_get_t<double>(ctx, "zvec", (size_t)m * Kp);
    VNE_TRY_CUDA(ctx, launch_tridiag_fvec(sk.alpha, sk.beta, sk.scale, Kp, m, Kp, zvec, st));
    double* gamma = ws_get_t<double>(ctx, "gamma", (size_t)m * Kp);
    k_gamma<<<(m * Kp + 255) / 256, 256, 0, st>>>(sk.norm2, sk.sigma, zvec, m, Kp, gamma);
    VNE_TRY_CUDA(ctx, cudaGetLastError());
    const size_t blk = (size_t)Kp * n;
    T* Y = ws_get_t<T>(ctx, "Y", blk);
    RecoverParams<T> rp{};
    rp.basis = (const T*)sk.basis;
    rp.slot_stride = sk.slot_stride;
    rp.y = Y;
    rp.gamma = gamma;
    rp.m = m;
    rp.K = Kp;
    rp.n_total = n;
    rp.tiles_per_panel = P->tiles_per_panel();
    rp.tiles = P->d_tiles;
    VNE_TRY_CUDA(ctx, launch_recover<T>(rp, ks, sk.panels, st));
    ctx->launches += 3;  // fvec, gamma, recover
    // 2. Q = orthonormal basis of range(Y): pivoted Cholesky-QR, twice
    const int nch = std::max(1, std::min(4 * ctx->sm_count, (n + 63) / 64));
    double* gpart = ws_get_t<double>(ctx, "gram.part", (size_t)nch * Kp * std::max(Kp, 128));
    double* G1 = ws_get_t<double>(ctx, "G1", (size_t)Kp * Kp);
    double* Minv = ws_get_t<double>(ctx, "Minv", (size_t)Kp * Kp);
    int* drank = ws_get_t<int>(ctx, "rank", 3);  // two ranks + the tensor-core Gram's wait flag
    int* gerr = drank + 2;
    double* cwork = ws_get_t<double>(ctx, "chol.work", (size_t)Kp * Kp + Kp);
    int* cpiv = ws_get_t<int>(ctx, "chol.piv", Kp);
    VNE_TRY_CUDA(ctx, cudaMemsetAsync(gerr, 0, sizeof(int), st));
    T* Q1 = ws_get_t<T>(ctx, "Q1", blk);
    // Q and (I - Q Q^T) G share one buffer: Q in block columns [0, Kp), the
    // projected Hutchinson vectors in [Kp, Kp + Kg), so one Lanczos block
    // evaluates all N_r + N_H quadratic forms.
    const int Kg = NH > 0 ? ((NH + ks - 1) / ks) * ks : 0;
    VNE_REQUIRE(ctx, Kg <= 128, VNE_EUNSUPPORTED, "N_H > 128 not supported in one projection block");
    T* QG = ws_get_t<T>(ctx, "QG", (size_t)(Kp + Kg) * n);
    T* Q = QG;
    const double tol = M->fp64 ? 1e-13 : 1e-5;
    VNE_TRY_CUDA(ctx, launch_gram<T>(Y, Kp, Y, Kp, ks, n, gpart, nch, G1, gerr, st));
    VNE_TRY_CUDA(ctx, launch_chol_qr_factor(G1, Kp, tol, Minv, drank, cwork, cpiv, st));
    VNE_TRY_CUDA(ctx, launch_apply<T>(Y, Kp, Minv, Kp, nullptr, Q1, ks, n, 1.0, gerr, st));
    VNE_TRY_CUDA(ctx, launch_gram<T>(Q1, Kp, Q1, Kp, ks, n, gpart, nch, G1, gerr, st));
    VNE_TRY_CUDA(ctx, launch_chol_qr_factor(G1, Kp, tol, Minv, drank + 1, cwork, cpiv, st));
    VNE_TRY_CUDA(ctx, launch_apply<T>(Q1, Kp, Minv, Kp, nullptr, Q, ks, n, 1.0, gerr, st));
    ctx->launches += 12;  // 2 x (gram + reduce + symmetrise + factor + inverse + apply)
    if (Kg > 0) {
        // G (Rademacher columns N_r..N_r+N_H-1), then G' = G - Q (Q^T G)
        const size_t gblk = (size_t)Kg * n;
        T* Gr = ws_get_t<T>(ctx, "Graw", gblk);
        T* Gp = QG + (size_t)Kp * n;
        StartSource sg{};
        sg.kind = SRC_RADEMACHER;
        sg.gaussian = o && o->gaussian_probes != 0;
        sg.seed_mixed = sm;
        sg.col_begin = Nr;
        sg.ncols = NH;
        StartParams<T> spp{};
        spp.src = sg;
        spp.node_id = P->node_id;
        spp.seg = P->d_segs;
        spp.nseg = 1;
        spp.K = Kg;
        spp.n_total = n;
        spp.tiles_per_panel = P->tiles_per_panel();
        spp.tiles = P->d_tiles;
        spp.desing = 0;
        spp.w1 = Gr;
        spp.mean = ws_get_t<double>(ctx, "mean", Kg);
        spp.norm2 = ws_get_t<double>(ctx, "g.norm2", Kg);
        spp.sig1 = ws_get_t<double>(ctx, "g.sig", Kg);
        spp.part = ws_get_t<double>(ctx, "part", (size_t)(Kg / ks) * P->tiles_per_panel() * ks);
        spp.counter = ws_get_t<uint32_t>(ctx, "counter", (size_t)(Kg / ks), true);
        VNE_TRY_CUDA(ctx, launch_start<T>(spp, ks, Kg / ks, st));
        double* C = ws_get_t<double>(ctx, "QtG", (size_t)Kp * Kg);
        double* gpart2 = ws_get_t<double>(ctx, "gram.part2", (size_t)nch * Kp * Kg);
        VNE_TRY_CUDA(ctx, launch_gram<T>(Q, Kp, Gr, Kg, ks, n, gpart2, nch, C, gerr, st));
        VNE_TRY_CUDA(ctx, launch_apply<T>(Q, Kp, C, Kg, Gr, Gp, ks, n, -1.0, gerr, st));
        ctx->launches += 4;
    }
    int hr[3] = {0, 0, 0};
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hr, drank, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    VNE_REQUIRE(ctx, hr[2] == 0, VNE_EDEVICE, "tensor-core sketch kernel: a bounded wait ran out");
    const int r = std::min(hr[0], hr[1]);
    // 3. all N_r + N_H quadratic forms in one Lanczos block
    double low = 0.0, resid = 0.0;
    {
        StartSource sq{};
        sq.kind = SRC_PANEL;
        sq.ncols = Kp + Kg;
        BlockOut qo;
        run_block<T>(ctx, *P, sq, QG, Kp + Kg, ks, m, want_reorth(M, o), false, M->desing, "q", qo, sc.variant,
                     sc.interleave, sc.graph);
        std::vector<double> h = download(ctx, qo.psi, Kp + Kg);
        for (int c = 0; c < r; c++) low += h[c];
        for (int c = 0; c < NH; c++) resid += h[Kp + c];
        if (NH > 0) resid /= NH;
    }
    *estimate = low + resid;
    if (parts) {
        parts[0] = low;
        parts[1] = resid;
        parts[2] = (double)r;
    }
}

}  // namespace

extern "C" vne_status vne_entropy_hutchpp(vne_matrix* M, int32_t sketch_cols, int32_t hutch_vectors,
                                          int32_t krylov_steps, uint64_t seed, const vne_options* opt,
                                          double* estimate, double* parts) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, estimate, VNE_EINVAL, "estimate is required");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    if (M->fp64) hutchpp_impl<double>(M, &o, sketch_cols, hutch_vectors, krylov_steps, seed, estimate, parts);
    else hutchpp_impl<float>(M, &o, sketch_cols, hutch_vectors, krylov_steps, seed, estimate, parts);
    VNE_API_END(ctx)
}

namespace {

// Greedy distance-d colouring (Algorithm 1) of M's graph on the device, in
// rounds of k_color_round (and k_color_big for balls too large for a warp).
// Several colourings (one per distance) run at once, each on its own stream
// with its own workspace: their rounds are latency-bound, so they overlap.
// The colours land in workspace `name` of each job in the caller's node
// numbering; job.rounds = the rounds it took, 0 when a ball (d >= 3) did not
// fit even a CTA's table (then nothing is written).
struct ColorJob {
    int d = 1;
    std::string name;
    int32_t* out = nullptr;  // caller numbering
    int32_t s = 0;           // colours
    int rounds = 0;
    // internal
    cudaStream_t st = nullptr;
    ColorRound p{};
    int32_t* ctr = nullptr;
    int32_t* h = nullptr;  // pinned host copy of the counters
    int r = 0;
    int64_t prev = 0;
    bool done = false, overflow = false;
};

void device_colorings(vne_matrix* M, std::vector<ColorJob>& jobs) {
    vne_ctx* ctx = M->ctx;
    const int64_t n = M->n;
    const int nj = (int)jobs.size();
    if (!ctx->pinned_ctr) VNE_TRY_CUDA(ctx, cudaMallocHost(&ctx->pinned_ctr, 8 * 8 * sizeof(int32_t)));
    VNE_REQUIRE(ctx, nj >= 1 && nj <= 8, VNE_EINVAL, "1..8 colourings at once");
    while ((int)ctx->color_streams.size() < nj - 1) {
        cudaStream_t sx = nullptr;
        VNE_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking));
        ctx->color_streams.push_back(sx);
        for (int k = 0; k < 2; k++) {  // fork and join events of that stream
            cudaEvent_t e = nullptr;
            VNE_TRY_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            ctx->color_events.push_back(e);
        }
    }
    const int32_t n32 = (int32_t)n;
    for (int i = 0; i < nj; i++) {
        ColorJob& J = jobs[i];
        J.st = i == 0 ? ctx->stream : ctx->color_streams[i - 1];
        if (i > 0) {  // the job's stream follows the work enqueued on the context's stream
            cudaEvent_t ev = ctx->color_events[2 * (i - 1)];
            VNE_TRY_CUDA(ctx, cudaEventRecord(ev, ctx->stream));
            VNE_TRY_CUDA(ctx, cudaStreamWaitEvent(J.st, ev, 0));
        }
        const std::string w = "col" + std::to_string(i) + ".";
        uint64_t* key = ws_get_t<uint64_t>(ctx, w + "key", n);
        int32_t* color = ws_get_t<int32_t>(ctx, w + "color", n);
        int32_t* blk = ws_get_t<int32_t>(ctx, w + "blk", n);
        int32_t* l0 = ws_get_t<int32_t>(ctx, w + "l0", n);
        int32_t* l1 = ws_get_t<int32_t>(ctx, w + "l1", n);
        J.ctr = ws_get_t<int32_t>(ctx, w + "ctr", 8, true);  // cnt[3], ncolors, overflow, bigcnt[2]
        int32_t* inv = M->d_node_id ? ws_get_t<int32_t>(ctx, w + "inv", n) : nullptr;
        int32_t* tries = ws_get_t<int32_t>(ctx, w + "tries", n);
        VNE_TRY_CUDA(ctx, launch_color_init(M->d_rowptr, M->d_node_id, n, key, inv, tries, color, blk, l0, J.st));
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(J.ctr, &n32, sizeof(n32), cudaMemcpyHostToDevice, J.st));
        ColorRound& p = J.p;
        p = ColorRound{};
        p.rowptr = M->d_rowptr;
        p.col = M->d_col;
        p.key = key;
        p.inv = inv;
        p.color = color;
        p.blk = blk;
        p.tries = tries;
        p.list[0] = l0;
        p.list[1] = l1;
        p.cnt = J.ctr;
        p.ncolors = J.ctr + 3;
        p.overflow = J.ctr + 4;
        p.d = J.d;
        if (J.d >= 3) {
            // balls too large for a warp's shared-memory table go to one CTA
            // each (k_color_big); the tables start empty (epoch 0 everywhere)
            const size_t ctas = (size_t)color_big_ctas();
            p.biglist = ws_get_t<int32_t>(ctx, w + "big", n);
            p.bigcnt = J.ctr + 5;
            p.bigtab = ws_get_t<uint64_t>(ctx, w + "bigtab", ctas * color_big_table_entries(), true);
            p.bigball = ws_get_t<int32_t>(ctx, w + "bigball", ctas * color_big_ball_entries());
            p.epoch = ws_get_t<uint32_t>(ctx, w + "epoch", ctas, true);
        }
        J.h = ctx->pinned_ctr + 8 * i;
        J.r = 0;
        J.prev = n;
        J.done = J.overflow = false;
    }
    for (;;) {
        bool any = false;
        for (ColorJob& J : jobs) {
            if (J.done) continue;
            any = true;
            // every round colours at least the first uncoloured node in the
            // greedy order, so a batch of rounds always makes progress
            const int batch = J.prev > 4096 ? 4 : 16;
            for (int b = 0; b < batch; b++, J.r++) {
                J.p.round = J.r;
                VNE_TRY_CUDA(ctx, launch_color_round(J.p, J.st));
                ctx->launches++;
                if (J.p.biglist) {
                    VNE_TRY_CUDA(ctx, launch_color_big(J.p, J.st));
                    ctx->launches++;
                }
            }
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(J.h, J.ctr, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, J.st));
        }
        if (!any) break;
        for (ColorJob& J : jobs) {
            if (J.done) continue;
            VNE_TRY_CUDA(ctx, cudaStreamSynchronize(J.st));
            if (J.h[4]) {
                J.done = J.overflow = true;
                continue;
            }
            const int64_t left = J.h[J.r % 3];
            if (left == 0) {
                J.done = true;
                continue;
            }
            VNE_REQUIRE(ctx, left < J.prev, VNE_EDEVICE, "device colouring made no progress (%lld nodes left)",
                        (long long)left);
            J.prev = left;
        }
    }
    for (ColorJob& J : jobs) {
        if (J.overflow) {
            J.rounds = 0;
            continue;
        }
        J.out = ws_get_t<int32_t>(ctx, J.name, n);
        VNE_TRY_CUDA(ctx, launch_color_scatter(J.p.color, M->d_node_id, n, J.out, J.st));
        ctx->launches++;
        J.s = J.h[3];
        J.rounds = J.r;
    }
    // the context's stream continues after every job
    for (int i = 1; i < nj; i++) {
        cudaEvent_t ev = ctx->color_events[2 * (i - 1) + 1];
        VNE_TRY_CUDA(ctx, cudaEventRecord(ev, jobs[i].st));
        VNE_TRY_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ev, 0));
    }
}

// Colours of M's graph in the caller's numbering, on the device; *rounds =
// device rounds.  A distance-(d - 1) ball beyond the CTA table (about 196,000
// nodes) is refused: the sequential sweep over such balls would take
// n x 196,000 steps or more.
void matrix_colorings(vne_matrix* M, std::vector<ColorJob>& jobs) {
    device_colorings(M, jobs);
    for (const ColorJob& J : jobs)
        VNE_REQUIRE(M->ctx, J.rounds > 0, VNE_EUNSUPPORTED,
                    "distance-%d colouring: a ball of radius %d holds more than %zu nodes; pass a colouring", J.d,
                    J.d - 1, color_big_table_entries() / 4 * 3);
}

int32_t* matrix_coloring(vne_matrix* M, int d, const std::string& name, int32_t* s, int* rounds) {
    std::vector<ColorJob> jobs(1);
    jobs[0].d = d;
    jobs[0].name = name;
    matrix_colorings(M, jobs);
    *s = jobs[0].s;
    if (rounds) *rounds = jobs[0].rounds;
    return jobs[0].out;
}

}  // namespace

extern "C" vne_status vne_matrix_coloring(vne_matrix* M, int32_t distance, int32_t* colors, int32_t* num_colors,
                                          int32_t* device_rounds) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, distance >= 1, VNE_EINVAL, "distance must be >= 1");
    int32_t s = 0;
    int rounds = 0;
    int32_t* d = matrix_coloring(M, distance, "colors", &s, &rounds);
    if (colors && M->n)
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(colors, d, M->n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (num_colors) *num_colors = s;
    if (device_rounds) *device_rounds = rounds;
    VNE_API_END(ctx)
}

extern "C" vne_status vne_greedy_coloring(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t distance,
                                          int32_t* colors, int32_t* num_colors) {
    if (n < 1 || !row_ptr || !col_idx || !colors || distance < 1) return VNE_EINVAL;
    try {
        int32_t s = greedy_coloring(n, row_ptr, col_idx, distance, colors);
        if (num_colors) *num_colors = s;
    } catch (...) {
        return VNE_ENOMEM;
    }
    return VNE_OK;
}

extern "C" vne_status vne_entropy_probing(vne_matrix* M, const int32_t* coloring, int32_t distance,
                                          int32_t krylov_steps, const double* poles, int32_t num_poles,
                                          const vne_options* opt, double* estimate, int32_t* num_colors) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, estimate, VNE_EINVAL, "estimate is required");
    const bool rational = (poles != nullptr || num_poles > 0);
    VNE_REQUIRE(ctx, rational || (krylov_steps >= 1 && krylov_steps <= 128), VNE_EINVAL,
                "krylov_steps must be in [1, 128]");
    const int64_t n = M->n;
    // colours in the caller's node numbering
    int32_t s = 0;
    int32_t* dcol = nullptr;
    if (coloring) {
        std::vector<int32_t> col(n);
        for (int64_t i = 0; i < n; i++) {
            VNE_REQUIRE(ctx, coloring[i] >= 0, VNE_EINVAL, "negative colour at node %lld", (long long)i);
            col[i] = coloring[i];
            s = std::max(s, coloring[i] + 1);
        }
        dcol = upload(ctx, "colors", col);
    } else {
        VNE_REQUIRE(ctx, distance >= 1, VNE_EINVAL, "distance must be >= 1");
        dcol = matrix_coloring(M, distance, "colors", &s, nullptr);
    }
    StartSource src{};
    src.kind = SRC_INDICATOR;
    src.colors = dcol;
    src.col_begin = 0;
    std::vector<double> psi;
    if (rational) {
        VNE_REQUIRE(ctx, num_poles >= 1 && num_poles <= 8, VNE_EINVAL, "1..8 poles are supported");
        std::vector<double> sh = resolve_shifts(M, poles, num_poles);
        for (double v : sh) VNE_REQUIRE(ctx, v > 0.0, VNE_EINVAL, "poles must be negative reals (shifts > 0)");
        std::vector<int> its;
        std::vector<double> rs;
        if (M->fp64) rational_quadforms<double>(M, &o, src, s, sh.data(), num_poles, psi, its, rs);
        else rational_quadforms<float>(M, &o, src, s, sh.data(), num_poles, psi, its, rs);
        int mx = 0;
        for (int v : its) mx = std::max(mx, v);
        ctx->last_cg_iters = mx;
    } else {
        psi = M->fp64 ? quadforms<double>(M, &o, src, s, krylov_steps) : quadforms<float>(M, &o, src, s, krylov_steps);
    }
    double tot = 0.0;
    for (double v : psi) tot += v;
    *estimate = tot;
    if (num_colors) *num_colors = s;
    VNE_API_END(ctx)
}

namespace {

// Section 5.1: d from T_1, T_2, T_3.  The model |S - T_d| ~ C q^d / d^k is
// fitted to |T_{d+1} - T_d| at d = 1, 2 for k = 2 and k = 3 (q = 2^k e2 / e1,
// C = e1 / q); each decaying fit (q < 1) gives the smallest d with a
// modelled error <= eps_abs, and the larger of the two is taken.  Returns
// -1 when neither k gives a decaying fit.  e1 = 0: d = 1; e2 = 0 (q = 0):
// d = 1 if e1 <= eps_abs, else 2.  The result may exceed d_max by one.
int probing_heuristic_d(double t1, double t2, double t3, double eps_abs, int d_max) {
    const double e1 = fabs(t2 - t1), e2 = fabs(t3 - t2);
    if (e1 == 0.0) return 1;
    if (e2 == 0.0) return e1 <= eps_abs ? 1 : 2;
    int best = -1;
    for (int k = 2; k <= 3; k++) {
        const double q = std::ldexp(1.0, k) * e2 / e1;
        if (!(q < 1.0)) continue;
        const double C = e1 / q;
        int d = 1;
        while (d <= d_max && C * std::pow(q, d) / std::pow((double)d, k) > eps_abs) d++;
        best = std::max(best, d);
    }
    return best;
}

// T_d of Algorithm 2 at one distance: colour on the device, then Lanczos on
// the colour indicators with the adaptive stop of Theorem 4.4, either
// relative (tol_rel x psi) or per colour eps_abs |V_l| / n.
template <typename T>
double probing_at(vne_matrix* M, const vne_options* o, int d, int m, double tol_rel, double eps_abs,
                  vne_coloring_fn fn, void* user, int* colors, int* steps, int32_t* pre_col = nullptr,
                  int32_t pre_s = 0) {
    vne_ctx* ctx = M->ctx;
    int32_t s = 0;
    int32_t* dcol = nullptr;
    std::vector<int32_t> host_sizes;
    if (pre_col) {  // a device colouring computed beforehand
        dcol = pre_col;
        s = pre_s;
    } else if (fn) {
        // the caller's colouring (e.g. an optimal one for a structured graph)
        std::vector<int32_t> col(M->n);
        s = fn(user, d, M->n, col.data());
        VNE_REQUIRE(ctx, s >= 1, VNE_EINVAL, "colouring callback failed at distance %d (returned %d)", d, s);
        host_sizes.assign(s, 0);
        for (int64_t i = 0; i < M->n; i++) {
            VNE_REQUIRE(ctx, col[i] >= 0 && col[i] < s, VNE_EINVAL, "colour %d of node %lld outside [0, %d)", col[i],
                        (long long)i, s);
            host_sizes[col[i]]++;
        }
        dcol = upload(ctx, "colors", col);
    } else {
        dcol = matrix_coloring(M, d, "colors", &s, nullptr);
    }
    StartSource src{};
    src.kind = SRC_INDICATOR;
    src.colors = dcol;
    src.col_begin = 0;
    vne_options oo = *o;
    std::vector<double> psi;
    if (eps_abs > 0.0) {
        std::vector<int32_t> sizes(s);
        if (fn) {
            sizes = host_sizes;
        } else {
            int32_t* cnt = ws_get_t<int32_t>(ctx, "colors.count", (size_t)s, true);
            VNE_TRY_CUDA(ctx, launch_color_hist(dcol, M->n, cnt, ctx->stream));
            ctx->launches++;
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(sizes.data(), cnt, s * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                              ctx->stream));
            VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
        std::vector<double> tol(s);
        for (int l = 0; l < s; l++) tol[l] = eps_abs * (double)sizes[l] / (double)M->n;
        oo.quad_tol = 0.0;
        psi = quadforms<T>(M, &oo, src, s, m, tol.data());
    } else {
        oo.quad_tol = tol_rel;
        psi = quadforms<T>(M, &oo, src, s, m);
    }
    *colors = s;
    *steps = ctx->last_steps;
    double tot = 0.0;
    for (double v : psi) tot += v;
    return tot;
}

}  // namespace

extern "C" vne_status vne_entropy_probing_auto(vne_matrix* M, double eps, int32_t krylov_steps, int32_t d_max,
                                               vne_coloring_fn coloring_fn, void* user, const vne_options* opt,
                                               double* estimate, vne_probing_report* rep) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, estimate, VNE_EINVAL, "estimate is required");
    VNE_REQUIRE(ctx, eps > 0.0 && eps < 1.0, VNE_EINVAL, "eps must be in (0, 1)");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    VNE_REQUIRE(ctx, d_max >= 1 && d_max <= 1024, VNE_EINVAL, "d_max must be in [1, 1024]");
    vne_options o = opt ? *opt : defaults();
    vne_probing_report r{};
    std::vector<double> T;
    std::vector<int> cols, steps;
    // the device colourings at d = 1, 2, 3 do not depend on the T values:
    // computed first, at once (their rounds overlap on three streams)
    std::vector<ColorJob> pre;
    if (!coloring_fn) {
        pre.resize(3);
        for (int i = 0; i < 3; i++) {
            pre[i].d = i + 1;
            pre[i].name = "colors.d" + std::to_string(i + 1);
        }
        matrix_colorings(M, pre);
    }
    auto run = [&](int d, double tol_rel, double eps_abs) {
        int c = 0, st = 0;
        int32_t* pc = (d <= (int)pre.size()) ? pre[d - 1].out : nullptr;
        const int32_t ps = (d <= (int)pre.size()) ? pre[d - 1].s : 0;
        double t = M->fp64 ? probing_at<double>(M, &o, d, krylov_steps, tol_rel, eps_abs, coloring_fn, user, &c, &st,
                                                pc, ps)
                           : probing_at<float>(M, &o, d, krylov_steps, tol_rel, eps_abs, coloring_fn, user, &c, &st,
                                               pc, ps);
        T.push_back(t);
        cols.push_back(c);
        steps.push_back(st);
    };
    // T_1 with the relative rule: its sum is within eps/2 of T_1 <= S
    run(1, 0.5 * eps, 0.0);
    const double eps_abs = 0.5 * eps * T[0];
    run(2, 0.0, eps_abs);
    run(3, 0.0, eps_abs);
    int d = probing_heuristic_d(T[0], T[1], T[2], eps_abs, d_max);
    int rule = VNE_PROBING_RULE_FIT;
    if (d > d_max) {
        d = d_max;
        rule = VNE_PROBING_RULE_CAPPED;
    } else if (d < 0) {
        // no decaying fit: the smallest d with |T_{d+1} - T_d| <= eps_abs
        rule = VNE_PROBING_RULE_DIFFERENCES;
        d = 1;
        for (;;) {
            if (d >= d_max) {
                d = d_max;
                rule = VNE_PROBING_RULE_CAPPED;
                break;
            }
            if ((int)T.size() < d + 1) run(d + 1, 0.0, eps_abs);
            if (fabs(T[d] - T[d - 1]) <= eps_abs) break;
            d++;
        }
    }
    if ((int)T.size() < d) {
        // T_d at a distance not evaluated yet (the distances in between are not needed)
        int c = 0, st = 0;
        double t = M->fp64 ? probing_at<double>(M, &o, d, krylov_steps, 0.0, eps_abs, coloring_fn, user, &c, &st)
                           : probing_at<float>(M, &o, d, krylov_steps, 0.0, eps_abs, coloring_fn, user, &c, &st);
        r.num_colors = c;
        r.steps_chosen = st;
        *estimate = t;
    } else {
        r.num_colors = cols[d - 1];
        r.steps_chosen = steps[d - 1];
        *estimate = T[d - 1];
    }
    for (int i = 0; i < 3; i++) {
        r.t[i] = T[i];
        r.colors_d[i] = cols[i];
        r.steps_d[i] = steps[i];
    }
    r.eps_abs = eps_abs;
    r.distance = d;
    r.rule = rule;
    r.evaluated = (int32_t)T.size();
    if (rep) *rep = r;
    VNE_API_END(ctx)
}

extern "C" vne_status vne_spmm(vne_matrix* M, const void* X, void* Y, int32_t k) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, X && Y && k >= 1, VNE_EINVAL, "need X, Y and k >= 1");
    if (M->fp64)
        VNE_TRY_CUDA(ctx, launch_spmm_plain<double>(M->d_rowptr, M->d_col, (const double*)M->d_vals, (int)M->n, k,
                                                    M->d_node_id, M->scale, (const double*)X, (double*)Y, ctx->stream));
    else
        VNE_TRY_CUDA(ctx, launch_spmm_plain<float>(M->d_rowptr, M->d_col, (const float*)M->d_vals, (int)M->n, k,
                                                   M->d_node_id, M->scale, (const float*)X, (float*)Y, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VNE_API_END(ctx)
}

extern "C" vne_status vne_block_gram(vne_ctx* ctx, const float* X, int32_t kx, const float* Y, int32_t ky, int32_t ks,
                                     int64_t n, double* C) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, X && Y && C && n >= 1 && n < INT32_MAX && kx >= 1 && ky >= 1 && kx <= 128 && ky <= 128 &&
                         (ks == 8 || ks == 16 || ks == 32) && kx % ks == 0 && ky % ks == 0,
                VNE_EINVAL, "bad arguments to vne_block_gram");
    const int nch = std::max(1, std::min(4 * ctx->sm_count, (int)((n + 63) / 64)));
    double* part = ws_get_t<double>(ctx, "bg.part", (size_t)nch * kx * ky);
    double* dC = ws_get_t<double>(ctx, "bg.C", (size_t)kx * ky);
    int* err = ws_get_t<int>(ctx, "bg.err", 1, true);
    VNE_TRY_CUDA(ctx, launch_gram<float>(X, kx, Y, ky, ks, (int)n, part, nch, dC, err, ctx->stream));
    int herr = 0;
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(C, dC, (size_t)kx * ky * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VNE_REQUIRE(ctx, herr == 0, VNE_EDEVICE, "tensor-core Gram: a bounded wait ran out");
    VNE_API_END(ctx)
}

extern "C" vne_status vne_block_apply(vne_ctx* ctx, const float* In, int32_t kin, const double* M, int32_t kout,
                                      const float* In2, float* Out, int32_t ks, int64_t n, double coef) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, In && M && Out && n >= 1 && n < INT32_MAX && kin >= 1 && kout >= 1 && kin <= 128 &&
                         kout <= 128 && (ks == 8 || ks == 16 || ks == 32) && kin % ks == 0 && kout % ks == 0,
                VNE_EINVAL, "bad arguments to vne_block_apply");
    std::vector<double> hm(M, M + (size_t)kin * kout);
    double* dM = upload(ctx, "ba.M", hm);
    int* err = ws_get_t<int>(ctx, "ba.err", 1, true);
    VNE_TRY_CUDA(ctx, launch_apply<float>(In, kin, dM, kout, In2, Out, ks, (int)n, coef, err, ctx->stream));
    int herr = 0;
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VNE_REQUIRE(ctx, herr == 0, VNE_EDEVICE, "tensor-core block product: a bounded wait ran out");
    VNE_API_END(ctx)
}

extern "C" vne_status vne_tridiag_quadrature(vne_ctx* ctx, const double* alpha, const double* beta, const double* norm2,
                                             double scale, int32_t count, int32_t m, double* psi) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, alpha && beta && norm2 && psi && count >= 1 && m >= 1 && m <= 128, VNE_EINVAL,
                "bad arguments to vne_tridiag_quadrature");
    // host layout [count][m] -> device column-interleaved [m][count]
    std::vector<double> a((size_t)m * count), b((size_t)m * count), sc(count, scale), nn(norm2, norm2 + count);
    for (int c = 0; c < count; c++)
        for (int j = 0; j < m; j++) {
            a[(size_t)j * count + c] = alpha[(size_t)c * m + j];
            b[(size_t)j * count + c] = (j + 1 < m) ? beta[(size_t)c * m + j] : 0.0;
        }
    double* da = upload(ctx, "tq.a", a);
    double* db = upload(ctx, "tq.b", b);
    double* ds = upload(ctx, "tq.s", sc);
    double* dn = upload(ctx, "tq.n", nn);
    double* dp = ws_get_t<double>(ctx, "tq.p", count);
    VNE_TRY_CUDA(ctx, launch_tridiag_quad(da, db, dn, ds, count, m, count, dp, ctx->stream));
    std::vector<double> h = download(ctx, dp, count);
    std::copy(h.begin(), h.end(), psi);
    VNE_API_END(ctx)
}

extern "C" vne_status vne_quadrature_bounds(vne_ctx* ctx, const double* alpha, const double* beta,
                                            const double* norm2, double scale, int32_t count, int32_t m,
                                            double lam_min, double lam_max, int32_t grid, double* lower,
                                            double* upper, double* estimate) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, alpha && beta && norm2 && lower && upper && estimate && count >= 1 && m >= 1 && m <= 128,
                VNE_EINVAL, "bad arguments to vne_quadrature_bounds");
    VNE_REQUIRE(ctx, lam_min > 0.0 && lam_max > lam_min && grid >= 1, VNE_EINVAL,
                "need 0 < lam_min < lam_max and grid >= 1");
    // host layout [count][m] -> device column-interleaved [m][count]
    std::vector<double> a((size_t)m * count), b((size_t)m * count), sc(count, scale), nn(norm2, norm2 + count);
    for (int c = 0; c < count; c++)
        for (int j = 0; j < m; j++) {
            a[(size_t)j * count + c] = alpha[(size_t)c * m + j];
            b[(size_t)j * count + c] = beta[(size_t)c * m + j];
        }
    double* da = upload(ctx, "tb.a", a);
    double* db = upload(ctx, "tb.b", b);
    double* ds = upload(ctx, "tb.s", sc);
    double* dn = upload(ctx, "tb.n", nn);
    double* dout = ws_get_t<double>(ctx, "tb.out", 3 * (size_t)count);
    VNE_TRY_CUDA(ctx, launch_tridiag_bounds(da, db, dn, ds, count, m, count, lam_min, lam_max, grid, dout,
                                            dout + count, dout + 2 * count, ctx->stream));
    ctx->launches += 1;
    std::vector<double> h = download(ctx, dout, 3 * (size_t)count);
    std::copy(h.begin(), h.begin() + count, lower);
    std::copy(h.begin() + count, h.begin() + 2 * count, upper);
    std::copy(h.begin() + 2 * count, h.end(), estimate);
    VNE_API_END(ctx)
}

extern "C" vne_status vne_rademacher(vne_ctx* ctx, uint64_t seed, int64_t n, int32_t col_begin, int32_t k, int32_t fp64,
                                     void* out_device) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, out_device && n >= 1 && k >= 1 && col_begin >= 0, VNE_EINVAL, "bad arguments to vne_rademacher");
    VNE_TRY_CUDA(ctx, launch_rademacher_fill(seed_mix(seed), n, col_begin, k, fp64, out_device, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VNE_API_END(ctx)
}

extern "C" vne_status vne_gaussian_probes(vne_ctx* ctx, uint64_t seed, int64_t n, int32_t col_begin, int32_t k,
                                          double* out_device) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, out_device && n >= 1 && k >= 1 && col_begin >= 0, VNE_EINVAL,
                "bad arguments to vne_gaussian_probes");
    VNE_TRY_CUDA(ctx, launch_gaussian_fill(seed_mix(seed), n, col_begin, k, out_device, ctx->stream));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    VNE_API_END(ctx)
}

// ---------------------------------------------------------------------------
// batched uneven graphs: block-diagonal packing, one schedule, one launch per
// kernel per step for all graphs

extern "C" vne_status vne_batch_hutchinson(vne_matrix* const* mats, int32_t count, int32_t num_vectors,
                                           int32_t krylov_steps, uint64_t seed, const vne_options* opt,
                                           double* estimates, double* std_errors) {
    if (!mats || count < 1 || !mats[0]) return VNE_EINVAL;
    vne_ctx* ctx = mats[0]->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, estimates && num_vectors >= 1, VNE_EINVAL, "need estimates and num_vectors >= 1");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    const bool fp64 = mats[0]->fp64;
    int64_t ntot = 0, nnztot = 0;
    bool any_perm = false, any_valued = false;
    for (int i = 0; i < count; i++) {
        VNE_REQUIRE(ctx, mats[i] && mats[i]->ctx == ctx && mats[i]->fp64 == fp64, VNE_EINVAL,
                    "all matrices must share the context and precision");
        ntot += mats[i]->n;
        nnztot += mats[i]->nnz;
        any_perm |= !mats[i]->perm.empty();
        any_valued |= !mats[i]->pattern;
    }
    VNE_REQUIRE(ctx, !any_valued, VNE_EUNSUPPORTED, "batched mode packs pattern (graph) matrices");
    VNE_REQUIRE(ctx, ntot < INT32_MAX && nnztot < INT32_MAX, VNE_EINVAL, "packed batch too large");
    double taurel = o.breakdown_tol > 0 ? o.breakdown_tol : default_tau(fp64);
    const int target = default_item_nnz(&o);
    std::vector<uint64_t> key;
    key.push_back((uint64_t)target);
    uint64_t tbits = 0;
    memcpy(&tbits, &taurel, sizeof(tbits));
    key.push_back(tbits);
    key.push_back((uint64_t)fp64);
    key.push_back((uint64_t)o.panel);
    for (int i = 0; i < count; i++) key.push_back(mats[i]->uid);
    if (!ctx->batch_prob || ctx->batch_key != key) {
        delete ctx->batch_prob;
        ctx->batch_prob = nullptr;
        ctx->batch_key.clear();
        // packed CSR
        std::vector<int64_t> rp(ntot + 1, 0);
        std::vector<int32_t> ci(nnztot);
        std::vector<int32_t> nid;
        if (any_perm) nid.resize(ntot);
        std::unique_ptr<Problem> P(new Problem());
        P->fp64 = fp64;
        P->valued = false;
        P->n_total = (int32_t)ntot;
        P->nnz_total = nnztot;
        P->nseg = count;
        int64_t r0 = 0, e0 = 0;
        for (int i = 0; i < count; i++) {
            vne_matrix* M = mats[i];
            const std::vector<int32_t>& hc = host_cols(M);
            for (int64_t r = 0; r < M->n; r++) {
                rp[r0 + r + 1] = e0 + M->h_rowptr[r + 1];
                if (any_perm) nid[r0 + r] = M->perm.empty() ? (int32_t)r : M->perm[r];
            }
            for (int64_t e = 0; e < M->nnz; e++) ci[e0 + e] = hc[e] + (int32_t)r0;
            SegInfo s{};
            s.row_begin = (int32_t)r0;
            s.rows = (int32_t)M->n;
            s.scale = M->scale;
            s.tau = taurel * M->normM;
            P->segs.push_back(s);
            r0 += M->n;
            e0 += M->nnz;
        }
        for (int i = 0; i < count; i++) plan_segment(rp.data(), P->segs[i].row_begin, P->segs[i].rows, i, target, *P);
        std::vector<int32_t> rp32(ntot + 1);
        for (int64_t i = 0; i <= ntot; i++) rp32[i] = (int32_t)rp[i];
        int32_t* drp = dev_copy(ctx, rp32);
        int32_t* dci = dev_copy(ctx, ci);
        P->owned.push_back(drp);
        P->owned.push_back(dci);
        P->rowptr = drp;
        P->col = dci;
        if (any_perm) {
            int32_t* dn = dev_copy(ctx, nid);
            P->owned.push_back(dn);
            P->node_id = dn;
        }
        problem_upload(ctx, *P);
        // the packed launch walks the segments in order, so the panel that has to
        // stay L2-resident is one segment's slice: size it by the largest graph
        int64_t nmax = 0;
        for (int i = 0; i < count; i++) nmax = std::max<int64_t>(nmax, mats[i]->n);
        ctx->batch_ks = choose_panel(fp64, &o, nmax);
        ctx->batch_prob = P.release();
        ctx->batch_key = key;
    }
    Problem* P = ctx->batch_prob;
    const int ks = ctx->batch_ks;
    const int variant = fp64 ? 0 : (o.step_variant >= 0 ? o.step_variant : 4);
    StartSource s{};
    s.kind = SRC_RADEMACHER;
    s.gaussian = o.gaussian_probes != 0;
    s.seed_mixed = seed_mix(seed);
    s.col_begin = 0;
    s.ncols = num_vectors;
    BlockOut out;
    ctx->last_steps = 0;
    if (fp64) {
        check_ks<double>(ctx, ks);
        run_block<double>(ctx, *P, s, nullptr, num_vectors, ks, krylov_steps, false, false, true, "batch", out, 0,
                          false, o.graphs != 0);
    } else {
        check_ks<float>(ctx, ks);
        run_block<float>(ctx, *P, s, nullptr, num_vectors, ks, krylov_steps, false, false, true, "batch", out,
                         variant, false, o.graphs != 0);
    }
    std::vector<double> psi = download(ctx, out.psi, out.SK);
    for (int i = 0; i < count; i++) {
        double mean = 0.0;
        for (int c = 0; c < num_vectors; c++) mean += psi[(size_t)i * out.Kp + c];
        mean /= num_vectors;
        double var = 0.0;
        for (int c = 0; c < num_vectors; c++) {
            double d = psi[(size_t)i * out.Kp + c] - mean;
            var += d * d;
        }
        estimates[i] = mean;
        if (std_errors) std_errors[i] = num_vectors > 1 ? sqrt(var / (num_vectors - 1) / num_vectors) : 0.0;
    }
    VNE_API_END(ctx)
}

extern "C" vne_status vne_ctx_profile(vne_ctx* ctx, int32_t enable) {
    if (!ctx) return VNE_EINVAL;
    ctx->profile = enable != 0;
    for (auto& k : ctx->stat) k = KernelStat();
    ctx->launches = 0;
    return VNE_OK;
}

extern "C" vne_status vne_ctx_last_steps(const vne_ctx* ctx, int32_t* steps) {
    if (!ctx || !steps) return VNE_EINVAL;
    *steps = ctx->last_steps;
    return VNE_OK;
}

extern "C" vne_status vne_ctx_last_poly_dim(const vne_ctx* ctx, int32_t* k) {
    if (!ctx || !k) return VNE_EINVAL;
    *k = ctx->last_poly_dim;
    return VNE_OK;
}

extern "C" vne_status vne_ctx_graph_stats(const vne_ctx* ctx, int64_t* captured, int64_t* replayed) {
    if (!ctx) return VNE_EINVAL;
    if (captured) *captured = ctx->graphs_captured;
    if (replayed) *replayed = ctx->graphs_replayed;
    return VNE_OK;
}

extern "C" vne_status vne_measure_gather(vne_ctx* ctx, uint64_t table_bytes, int32_t row_bytes, uint64_t gathers,
                                         uint64_t stream_bytes, int32_t reps, double* gather_gbs) {
    if (!ctx) return VNE_EINVAL;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, gather_gbs && reps >= 1 && gathers >= 1, VNE_EINVAL, "need gather_gbs, reps >= 1, gathers >= 1");
    VNE_REQUIRE(ctx, row_bytes == 32 || row_bytes == 64 || row_bytes == 128, VNE_EINVAL, "row_bytes must be 32, 64 or 128");
    VNE_REQUIRE(ctx, table_bytes >= (uint64_t)row_bytes && table_bytes / row_bytes <= 0xffffffffull, VNE_EINVAL,
                "table size out of range");
    cudaStream_t st = ctx->stream;
    void* table = ws_get(ctx, "probe.table", table_bytes);
    void* stream = ws_get(ctx, "probe.stream", std::max<uint64_t>(stream_bytes, 16));
    float* sink = ws_get_t<float>(ctx, "probe.sink", 1);
    for (int i = 0; i < 2; i++)
        if (!ctx->loop_ev[i]) VNE_TRY_CUDA(ctx, cudaEventCreate(&ctx->loop_ev[i]));
    cudaEvent_t e0 = ctx->loop_ev[0], e1 = ctx->loop_ev[1];
    double best = 1e300;
    for (int r = 0; r <= reps; r++) {
        VNE_TRY_CUDA(ctx, cudaEventRecord(e0, st));
        VNE_TRY_CUDA(ctx, launch_gather_probe(table, table_bytes, row_bytes, gathers, 977u * r + 1u, stream,
                                              stream_bytes, sink, st));
        VNE_TRY_CUDA(ctx, cudaEventRecord(e1, st));
        VNE_TRY_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        VNE_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) best = std::min(best, (double)ms);
    }
    ctx->launches += reps + 1;
    *gather_gbs = (double)gathers * row_bytes / (best * 1e-3) / 1e9;
    VNE_API_END(ctx)
}

extern "C" vne_status vne_ctx_stats(const vne_ctx* ctx, int64_t* launches, double* kernel_stats) {
    if (!ctx) return VNE_EINVAL;
    if (launches) *launches = ctx->launches;
    if (kernel_stats)
        for (int k = 0; k < 4; k++) {
            kernel_stats[3 * k + 0] = (double)ctx->stat[k].launches;
            kernel_stats[3 * k + 1] = ctx->stat[k].ms;
            kernel_stats[3 * k + 2] = ctx->stat[k].bytes;
        }
    return VNE_OK;
}

// ---------------------------------------------------------------------------
// schedule autotuner

extern "C" vne_status vne_autotune(vne_matrix* M, int32_t k, int32_t steps, vne_options* chosen,
                                   double* ms_per_step) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    VNE_REQUIRE(ctx, k >= 1 && k <= 256 && steps >= 2 && steps <= 128, VNE_EINVAL,
                "autotune needs 1 <= k <= 256 and 2 <= steps <= 128");
    for (int i = 0; i < 2; i++)
        if (!ctx->loop_ev[i]) VNE_TRY_CUDA(ctx, cudaEventCreate(&ctx->loop_ev[i]));
    const int panels_f[3] = {8, 16, 32}, panels_d[3] = {4, 8, 16};
    const int items[4] = {128, 256, 512, 1024};
    const int nvar = M->fp64 ? 1 : kStepVariants;
    double best = 1e300;
    int bk = 0, bi = 0, bv = 0, bil = 0;
    const bool was_tuned = M->tuned;
    M->tuned = false;
    for (int pi = 0; pi < 3; pi++)
        for (int ii = 0; ii < 4; ii++)
            for (int v = 0; v < nvar; v++)
            for (int il = 0; il < 2; il++) {
                vne_options o;
                vne_options_default(&o);
                o.panel = M->fp64 ? panels_d[pi] : panels_f[pi];
                o.item_nnz = items[ii];
                o.step_variant = v;
                o.interleave = il;
                o.reorth = 0;
                Problem* P = matrix_problem(M, &o);
                StartSource s{};
                s.kind = SRC_RADEMACHER;
                s.seed_mixed = seed_mix(12345);
                s.ncols = k;
                double ms_min = 1e300;
                for (int rep = 0; rep < 2; rep++) {
                    BlockOut out;
                    ctx->time_steps = true;
                    if (M->fp64) run_block<double>(ctx, *P, s, nullptr, k, o.panel, steps, false, false, M->desing, "tune", out, v, il, false);
                    else run_block<float>(ctx, *P, s, nullptr, k, o.panel, steps, false, false, M->desing, "tune", out, v, il, false);
                    ctx->time_steps = false;
                    download(ctx, out.psi, 1);
                    float ms = 0.f;
                    VNE_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->loop_ev[0], ctx->loop_ev[1]));
                    ms_min = std::min(ms_min, (double)ms);
                }
                if (ms_min < best) {
                    best = ms_min;
                    bk = o.panel;
                    bi = items[ii];
                    bv = v;
                    bil = il;
                }
            }
    // release the tuning block's workspace
    for (auto it = ctx->ws.begin(); it != ctx->ws.end();) {
        if (it->first.compare(0, 5, "tune.") == 0) {
            cudaFree(it->second.ptr);
            it = ctx->ws.erase(it);
        } else {
            ++it;
        }
    }
    (void)was_tuned;
    M->tuned = true;
    M->tuned_panel = bk;
    M->tuned_item_nnz = bi;
    M->tuned_variant = bv;
    M->tuned_interleave = bil != 0;
    ctx->tune_cache[vne_ctx::TuneKey{M->n, M->nnz, M->maxdeg, (int)M->fp64, (int)M->pattern}] = {bk, bi, bv, bil};
    if (chosen) {
        vne_options_default(chosen);
        chosen->panel = bk;
        chosen->item_nnz = bi;
        chosen->step_variant = bv;
        chosen->interleave = bil;
    }
    if (ms_per_step) *ms_per_step = best / steps;
    VNE_API_END(ctx)
}

extern "C" vne_status vne_quadform_rational(vne_matrix* M, const double* vectors, int32_t k, uint32_t vec_flags,
                                            const double* shifts, int32_t num_shifts, const vne_options* opt,
                                            double* psi, int32_t* cg_iterations, double* residuals) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, k >= 1 && vectors && psi, VNE_EINVAL, "need k >= 1, vectors and psi");
    VNE_REQUIRE(ctx, num_shifts >= 1 && num_shifts <= 8, VNE_EINVAL, "1..8 poles are supported");
    std::vector<double> sh = resolve_shifts(M, shifts, num_shifts);
    for (double v : sh) VNE_REQUIRE(ctx, v > 0.0, VNE_EINVAL, "shifts must be positive (poles -s)");
    const double* dvec = vectors;
    if (!(vec_flags & VNE_VECTORS_DEVICE)) {
        double* d = ws_get_t<double>(ctx, "qb.input", (size_t)M->n * k);
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, vectors, (size_t)M->n * k * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        dvec = d;
    }
    StartSource s{};
    s.kind = SRC_DENSE64;
    s.ld = k;
    s.dense = dvec;
    std::vector<double> ps, rs;
    std::vector<int> its;
    if (M->fp64) rational_quadforms<double>(M, &o, s, k, sh.data(), num_shifts, ps, its, rs);
    else rational_quadforms<float>(M, &o, s, k, sh.data(), num_shifts, ps, its, rs);
    std::copy(ps.begin(), ps.end(), psi);
    if (cg_iterations) std::copy(its.begin(), its.end(), cg_iterations);
    if (residuals) std::copy(rs.begin(), rs.end(), residuals);
    VNE_API_END(ctx)
}

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
        sg.cta_begin = (int32_t)(P.items.size() / VNE_WARPS);
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
