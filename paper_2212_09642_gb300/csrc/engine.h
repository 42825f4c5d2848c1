// Internal header of libvne: the context and matrix handles, the packed
// operator ("problem") with its warp-level schedule, the workspace and error
// helpers, and the block Krylov engine shared by the estimator drivers.
//
// File map of the host side:
//   engine.cu          workspace, schedules, the block Lanczos engine
//                      (run_block, CUDA-graph capture and replay), blocked
//                      quadratic forms, operator application
//   abi.cu             contexts, matrix assembly, quadform_batch, Hutchinson,
//                      kernel-level and measurement entry points
//   hutchpp.cu         Hutch++ (sketch, orthonormalisation, projection)
//   rational_driver.cu rational Krylov quadratures by multi-shift CG
//   probing.cu         colourings, probing, probing with the choice of d
//   batch.cu           batched uneven graphs
//   autotune.cu        the SpMM schedule autotuner
//   serve.cu           the serving loop (continuous batching)
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/vne.h"
#include "host_graph.h"
#include "kernels.h"

using namespace vne;

// ---------------------------------------------------------------------------
// context, matrix handle

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
    std::map<TuneKey, std::array<int, 5>> tune_cache;
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
    int tuned_panel = 0, tuned_item_nnz = 0, tuned_variant = 0, tuned_ipw = 1;
    bool tuned_interleave = false;
    int64_t maxdeg = 0;
    ~vne_matrix();  // frees the device arrays and the cached schedule (engine.cu)
};

namespace vne_engine {
void dev_free(void* p);
}

// ---------------------------------------------------------------------------
// schedule ("plan") of a packed operator

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
    int32_t ipw = 1;         // work items per warp (CTA = VNE_WARPS * ipw items)
    double norm_m = 0.0;     // Gershgorin bound of the stored operator (single matrix)
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
            vne_engine::dev_free(d_segs);
            vne_engine::dev_free(d_items);
            vne_engine::dev_free(d_hubs);
            vne_engine::dev_free(d_cta_seg);
            vne_engine::dev_free(d_tiles);
        }
        for (void* p : owned) vne_engine::dev_free(p);
    }
    int ctas_per_panel() const { return (int)(items.size() / ((size_t)VNE_WARPS * ipw)); }
    int tiles_per_panel() const { return (int)tiles.size(); }
};

namespace vne_engine {

// Every device and pinned host allocation of the library goes through these
// wrappers: they count live allocations (vne_debug_live_allocations) and,
// for failure-injection tests, make the k-th next allocation fail as if the
// memory were exhausted (vne_debug_fail_allocation).
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t pinned_malloc(void** p, size_t bytes);
void pinned_free(void* p);
int64_t live_device_buffers();
int64_t live_pinned_buffers();
void fail_allocation_after(int64_t k);  // 0: off

struct Error {
    vne_status code;
};

void set_err(vne_ctx* ctx, const char* fmt, ...);

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
void* ws_get(vne_ctx* ctx, const std::string& name, size_t bytes, bool zero = false);

template <typename T>
T* ws_get_t(vne_ctx* ctx, const std::string& name, size_t count, bool zero = false) {
    return (T*)ws_get(ctx, name, count * sizeof(T), zero);
}

// Pinned host buffer `name` of at least `bytes` bytes (grown on demand);
// nullptr if the allocation fails.
void* pinned_bytes(vne_ctx* ctx, const std::string& name, size_t bytes);
template <typename T>
T* pinned_get(vne_ctx* ctx, const std::string& name, size_t count) {
    return (T*)pinned_bytes(ctx, name, std::max<size_t>(count * sizeof(T), 64));
}

template <typename T>
T* upload(vne_ctx* ctx, const std::string& name, const std::vector<T>& v) {
    T* d = ws_get_t<T>(ctx, name, std::max<size_t>(v.size(), 1));
    if (!v.empty())
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return d;
}

// Host copy of the stored column indices (device order), made on first use.
const std::vector<int32_t>& host_cols(vne_matrix* M);
cudaEvent_t ctx_event(vne_ctx* ctx);
// Resolve the recorded event pairs (the stream must be synchronised).
void ctx_flush_profile(vne_ctx* ctx);
uint64_t mix64_host(uint64_t z);
uint64_t seed_mix(uint64_t seed);

extern const int kTileRows;
// Work items and row tiles of one segment of a packed CSR.
void plan_segment(const int64_t* rowptr, int32_t row_begin, int32_t rows, int32_t seg, int target, Problem& P);

// Device copy of a host vector, owned by the caller (dev_free).
template <typename T>
T* dev_copy(vne_ctx* ctx, const std::vector<T>& v) {
    T* d = nullptr;
    size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    VNE_TRY_CUDA(ctx, dev_malloc((void**)&d, bytes));
    if (!v.empty())
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return d;
}

void problem_upload(vne_ctx* ctx, Problem& P);
double default_tau(bool fp64);
int default_item_nnz(const vne_options* o);

struct Sched {
    int ks, item_nnz, variant, ipw;
    bool interleave;
    bool graph;
};

int choose_panel(bool fp64, const vne_options* opt, int64_t n);
// Schedule for a call: explicit options win, then the matrix's autotuned
// choice, then the built-in defaults.
Sched resolve_sched(const vne_matrix* M, const vne_options* o);
Problem* matrix_problem(vne_matrix* M, const vne_options* opt);

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

// m Lanczos steps of a block of K columns (see engine.cu).
template <typename T>
void run_block(vne_ctx* ctx, Problem& P, const StartSource& src, const T* panel_src, int K, int ks, int m,
               int reorth, bool keep_basis, bool desing, const std::string& tag, BlockOut& out, int variant = 0,
               bool interleave = false, bool graph = true, bool want_psi = true, const Adaptive* ad = nullptr);

// Reorthogonalisation policy of a call: 0 none, 1 full, 2 partial.
int want_reorth(const vne_matrix* M, const vne_options* o);
int block_limit(const vne_options* o);
vne_options defaults();

template <typename T>
void check_ks(vne_ctx* ctx, int ks) {
    bool ok = sizeof(T) == 4 ? (ks == 8 || ks == 16 || ks == 32) : (ks == 4 || ks == 8 || ks == 16);
    VNE_REQUIRE(ctx, ok, VNE_EINVAL, "panel width %d not supported for this precision", ks);
}

// Quadratic forms of one source over all its columns, in blocks.
template <typename T>
std::vector<double> quadforms(vne_matrix* M, const vne_options* o, StartSource src, int ncols, int m,
                              const double* abs_tol = nullptr);

// out = A in + shift * in (A = scale M) and dq[c] = scale * (in . out), with
// the Lanczos step kernel.
template <typename T>
void apply_operator(vne_ctx* ctx, Problem& P, int ks, int Kp, const T* in, T* out, double shift, double* dq,
                    int variant, const std::string& tag);

// Rational Krylov quadratic forms (rational_driver.cu).
template <typename T>
void rational_quadforms(vne_matrix* M, const vne_options* o, StartSource src, int ncols, const double* shifts,
                        int nshift, std::vector<double>& psi, std::vector<int>& iters, std::vector<double>& resid);
std::vector<double> resolve_shifts(const vne_matrix* M, const double* poles, int num_poles);

// Hutch++ deflation basis of one query (hutchpp.cu): the sketch of probe
// columns 0..Nr-1, Q = orth(f(A) Omega) copied to q_rows ([n][Nr] row-major
// in M's packed row order, zero columns beyond the rank), psi(q_i) for
// i < Nr (0 beyond the rank) and the rank.
// The sketch takes sketch_steps Lanczos steps, the quadratic forms m, or
// fewer with `ad` (stopped by the Theorem 4.4 estimate).
template <typename T>
void hutchpp_deflation(vne_matrix* M, const vne_options* o, int Nr, int m, int sketch_steps, uint64_t seed,
                       T* q_rows, std::vector<double>& psi_q, int& rank, const Adaptive* ad = nullptr);

}  // namespace vne_engine

using namespace vne_engine;

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
