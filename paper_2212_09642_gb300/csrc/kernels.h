// Internal kernel launch interface of libvne (host <-> device parameter blocks).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace vne {

enum SourceKind { SRC_RADEMACHER = 0, SRC_INDICATOR = 1, SRC_DENSE64 = 2, SRC_PANEL = 3 };

struct StartSource {
    int32_t kind;
    int32_t ncols;      // real columns (the rest of the block is zero padding)
    int32_t col_begin;  // global probe index of block column 0 (Rademacher) or colour of column 0
    int32_t ld;         // leading dimension of `dense`
    uint64_t seed_mixed;
    const int32_t* colors;  // SRC_INDICATOR: colour per local node id
    const double* dense;    // SRC_DENSE64: [n][ld] in caller numbering
    const uint64_t* seg_seed;  // SRC_RADEMACHER, optional: per-segment mixed seed
    const int32_t* seg_col0;   //   and per-segment first probe column
    int32_t gaussian;          // SRC_RADEMACHER: 1 = standard normal entries (Box-Muller on the counters)
};

template <typename T>
struct StartParams {
    StartSource src;
    const T* panel_src;        // SRC_PANEL: panel-major block
    const int32_t* node_id;    // packed row -> local node id (NULL: identity within segment)
    const SegInfo* seg;
    int32_t nseg, K, n_total, tiles_per_panel;
    const RowTile* tiles;
    int32_t desing;
    T* w1;
    double* mean;   // [nseg*K]
    double* norm2;  // [nseg*K]
    double* sig1;   // [nseg*K]
    double* part;
    uint32_t* counter;
};

template <typename T>
struct StepParams {
    const int32_t* rowptr;
    const int32_t* col;
    const T* vals;
    int32_t n_total, K, nseg;
    const SegInfo* seg;
    const WorkItem* items;
    int32_t ctas_per_panel;
    const int32_t* cta_seg;
    const HubRow* hubs;
    int32_t nhubs, hub_slots;
    T* hub_part;
    uint32_t* hub_cnt;
    double* hub_dot;   // [panels][nhubs][KS]: w_j . u of each long row (added in fixed order)
    const RowTile* tiles;
    int32_t tiles_per_panel;
    int32_t stage_nnz;  // largest work item in nonzeros (staged variants)
    int32_t ipw;        // work items per warp (a CTA covers VNE_WARPS * ipw consecutive items)
    // per-segment step counters (serving): with segj set, segment s runs its
    // own step segj[s] (0: idle this launch); w_j lives in slot (j - 1) & 1,
    // the scalars in row j - 1 of [m][nseg * K] arrays (sigma: [m + 1][...])
    const int32_t* segj;
    T* slot0;
    T* slot1;
    double* alpha0;
    double* beta0;
    double* sigma0;
    const int32_t* panel_active;  // update kernel with renorm: nullable, inactive panels are skipped
    int32_t panel_base; // first panel of this launch (per-panel launches)
    int32_t first;   // j == 1: no previous vector
    int32_t renorm;  // update kernel: only recompute the norm of w_next in place
    const T* w_cur;
    const T* w_prev;
    T* u;
    T* w_next;
    const double* sig_cur;
    const double* sig_prev;
    const double* beta_prev;
    double* alpha;
    double* beta;
    double* sig_next;
    double* part;
    uint32_t* counter;
};

template <typename T>
struct ReorthParams {
    const T* basis;       // slot 0
    size_t slot_stride;   // elements between consecutive slots
    T* w;                 // vector being orthogonalised (slot j)
    int32_t j, K, n_total, panels, tiles_per_panel;
    const RowTile* tiles;
    double* part;         // [panels][j][tiles][KS]
    const double* coef;   // [j][K]
    const int32_t* panel_active;  // nullable: panels with no column to orthogonalise are skipped
    const uint8_t* sel;   // nullable [j][K]: a (panel, i) with no selected column is skipped
};

struct ReorthCoefParams {
    const double* part;
    const double* sig;    // [j][K] sigma_i of each basis vector
    double* coef;
    int32_t j, K, panels, tiles_per_panel;
    const uint8_t* sel;           // nullable [j][K]: orthogonalise column c against basis vector i
    const int32_t* panel_active;  // nullable, as in ReorthParams
};

// Partial reorthogonalisation (Simon's omega recurrence), one thread per
// column, after the update of step j (1-based) has formed w_{j+1} and beta_j.
struct ProParams {
    const double* alpha;  // [m][SK], M units
    const double* beta;   // [m][SK]
    const double* sig;    // [m+1][SK]: sigma_{j+1} = 0 marks a finished column
    double* omega;        // [2][m+2][SK]: omega_{j-1,.} and omega_{j,.}, rolled in place
    uint8_t* sel;         // [m+1][SK]: this step's set (row i: basis vector i+1)
    uint8_t* pend_sel;    // [m+1][SK]: the set the next step repeats
    int32_t* pend;        // [SK]
    int32_t* panel_active;  // [panels], zeroed before the kernel
    int32_t j, SK, ks, K, m;
    double eps, normM;
};
cudaError_t launch_pro_omega(const ProParams& p, cudaStream_t st);

template <typename T>
struct RecoverParams {
    const T* basis;
    size_t slot_stride;
    T* y;
    const double* gamma;  // [m][K]
    int32_t m, K, n_total, tiles_per_panel;
    const RowTile* tiles;
};

template <typename T> cudaError_t launch_start(const StartParams<T>&, int ks, int panels, cudaStream_t);
template <typename T>
cudaError_t launch_step(const StepParams<T>&, int ks, int panels, bool valued, int variant, cudaStream_t);
constexpr int kStepVariants = 14;
// A work item spans at most kItemMaxRows rows (64 for items of fewer than
// 1024 nonzeros); the staged variants keep its row offsets in kStageRp ints
// of shared memory per warp.
constexpr int kItemMaxRows = 128;
constexpr int kStageRp = kItemMaxRows + 4;
template <typename T> cudaError_t launch_update(const StepParams<T>&, int ks, int panels, cudaStream_t);
// Start vectors of a served block (Hutch++ with a deflation basis Q per
// segment): for the segments listed, g = probe columns col0[s] ..
// col0[s] + K - 1 (Rademacher, or Gaussian), g' = g - Q_s (Q_s^T g),
// c = g' - mean(g') 1 written to w1 (panel-major, K columns), with
// ||c||^2 and sigma_1 = 1 / ||c||.  Three passes with fixed-order
// per-segment reductions.
template <typename T>
struct SrvStartParams {
    const int32_t* tile_list;  // [ntiles] tiles of the starting segments, grouped by segment
    const RowTile* tiles;
    const SegInfo* seg;        // rows of each segment
    const int32_t* seg_tb;     // [nseg] first entry of the segment in tile_list
    const int32_t* seg_tc;     // [nseg] its number of tiles
    const int32_t* node_id;    // packed row -> node id in the query's own numbering
    const uint64_t* seg_seed;  // [nseg] mixed seed
    const int32_t* seg_col0;   // [nseg] first probe column of the block
    const T* q;                // [n_total][4] deflation basis, zero columns beyond the rank
    double* coef;              // [nseg][4][K]
    double* mean;              // [nseg][K]
    double* norm2;             // [nseg][K]
    double* sig1;              // [nseg][K]: row 0 of the sigma array
    T* w1;                     // panel-major [K / KS][n_total][KS]
    double* part;              // [ntiles][4 * K]
    uint32_t* counter;         // [nseg], zero between launches
    int32_t ntiles, K, n_total, gaussian;
};
template <typename T> cudaError_t launch_srv_start(const SrvStartParams<T>& p, int ks, cudaStream_t st);
// Step and update kernels for per-segment step counters (p.segj, pattern operators only).
template <typename T> cudaError_t launch_step_update_segj(const StepParams<T>&, int ks, int panels, cudaStream_t);
template <typename T> cudaError_t launch_reorth(const ReorthParams<T>&, const ReorthCoefParams&, int ks, cudaStream_t);
// The first two passes of launch_reorth only: coef[i][col] = sig_i^2
// (basis_i . w) for i < j (fixed-order sums, deterministic).
template <typename T> cudaError_t launch_col_dots(const ReorthParams<T>&, const ReorthCoefParams&, int ks, cudaStream_t);
template <typename T> cudaError_t launch_recover(const RecoverParams<T>&, int ks, int panels, cudaStream_t);
template <typename T>
cudaError_t launch_spmm_plain(const int32_t* rowptr, const int32_t* col, const T* vals, int n, int k,
                              const int32_t* node_id, double scale, const T* X, T* Y, cudaStream_t);
cudaError_t launch_rademacher_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, int fp64, void* out,
                                   cudaStream_t);
// FP64 standard normal probes from the same counters (Box-Muller).
cudaError_t launch_gaussian_fill(uint64_t seed_mixed, int64_t n, int col_begin, int k, double* out, cudaStream_t st);

// ---- block layouts (layout.cu) ----
// Columns col0 .. col0 + k - 1 of a panel-major block (n rows, panel width
// ks) to row-major [n][k] in the caller's numbering (node_id: packed row ->
// caller id, NULL for the identity).
template <typename T>
cudaError_t launch_panel_to_rows(const T* in, int n, int ks, int col0, int k, const int32_t* node_id, T* out,
                                 cudaStream_t st);
// Row-major [n][k] (caller numbering) to a panel-major block of Kp >= k
// columns, the columns beyond k zero.
template <typename T>
cudaError_t launch_rows_to_panel(const T* in, int n, int ks, int k, int Kp, const int32_t* node_id, T* out,
                                 cudaStream_t st);
// Panel-major block of Kp >= k columns whose column c < k is column
// src_cols[c] (device int32) of the panel-major `in`; columns beyond k zero.
template <typename T>
cudaError_t launch_select_columns(const T* in, int n, int ks, const int32_t* src_cols, int k, int Kp, T* out,
                                  cudaStream_t st);

// ---- multi-shift CG and rational projection (rational.cu) ----
// v *= 1 / sqrt(rem2[col]) where rem2 > drop^2 orig2 (a kept direction),
// else v = 0 (a dependent one): the last step of one Gram-Schmidt
// orthonormalisation, for a panel-major block of K columns.
template <typename T>
cudaError_t launch_cgs_scale(T* v, const double* orig2, const double* rem2, double drop, int n, int K, int ks,
                             int tiles_per_panel, const RowTile* tiles, cudaStream_t st);
struct CgState {
    int32_t K, nshift;
    double scale, shift0, tol;
    const double* shift;  // [nshift] (device)
    const double* dq;     // step-kernel output: scale * (p . q) per column
    double *rho, *rho_new, *a, *b, *a_prev, *b_prev, *cnorm;
    double *zeta, *zeta_prev, *zeta_next, *as, *bs, *resid;  // [nshift][K]
    int32_t *active, *iters;                                  // [nshift][K]
    int32_t* any_active;
};

template <typename T>
struct CgVectors {
    int32_t n, tiles_per_panel;
    const RowTile* tiles;
    T *r, *q, *p;
    T* x[8];
    T* ps[8];
    double* part;
    uint32_t* counter;
};

// Both Gram matrices of a basis W and its image A W in one pass over the
// vectors: for every column, W_a . W_b and W_a . (A W)_b for a <= b, pairs
// numbered row by row (W.W first, then W.AW), written to out[pair][col].
template <typename T>
struct MultiGram {
    int32_t n, panels, ks, nb;
    const T* w[24];
    const T* aw[24];
    int32_t chunks;   // row ranges per panel (grid x)
    int32_t groups;   // output groups per chunk (grid y)
    double* part;     // [panels][groups][chunks][outputs of a group]
};
template <typename T> cudaError_t launch_multi_gram(MultiGram<T> g, double* out, cudaStream_t);


cudaError_t launch_cg_scalars_a(const CgState&, cudaStream_t);
cudaError_t launch_cg_scalars_b(const CgState&, cudaStream_t);
template <typename T> cudaError_t launch_cg_update(const CgVectors<T>&, const CgState&, int ks, int panels, cudaStream_t);
template <typename T> cudaError_t launch_cg_direction(const CgVectors<T>&, const CgState&, int ks, int panels, cudaStream_t);
template <typename T>
struct BlockTransform {
    int32_t n, K, nb, tiles_per_panel;
    const RowTile* tiles;
    const T* in[24];
    T* out[24];
    const double* X;  // [nb][nb][K]
};
// Seed-CG scalars -> Lanczos tridiagonal of A (k rows, column-interleaved).
cudaError_t launch_cg_tridiag(const double* a_hist, const double* b_hist, int K, int k, double s0, double tau,
                              double* diag, double* off, cudaStream_t);
// Full [nb][nb][K] Gram matrices from their upper triangles (pairs a <= b).
cudaError_t launch_gram_mirror(const double* uniq, int nb, int K, double* full, cudaStream_t);
cudaError_t launch_rational_pass1(const double* M, int nb, int ncols, double drop, double* X, cudaStream_t);
cudaError_t launch_rational_pass2(const double* M, const double* K, const double* c2, int nb, int ncols, double drop,
                                  double* psi, int* rank, cudaStream_t);
template <typename T> cudaError_t launch_block_transform(const BlockTransform<T>&, int ks, int panels, cudaStream_t);
cudaError_t launch_cg_init(CgState st, const double* norm2, cudaStream_t);

// ---- dense / small kernels (kernels_dense.cu) ----
// Measurement (measure.cu): `count` random gathers of row_bytes-byte rows
// (32, 64 or 128) from the first table_bytes of `table`, plus one streaming
// read of stream_bytes from `stream`; both buffers must be zero-filled.
cudaError_t launch_gather_probe(const void* table, uint64_t table_bytes, int row_bytes, uint64_t count, uint32_t seed,
                                const void* stream, uint64_t stream_bytes, float* sink, cudaStream_t st);

// Greedy distance-d colouring on the device (coloring.cu).  key[v] orders the
// nodes as Algorithm 1 does (descending degree, then ascending caller id);
// color[v] = -1 until coloured; blk[v] = last blocker seen.
struct ColorRound {
    const int32_t* rowptr;
    const int32_t* col;
    const uint64_t* key;
    const int32_t* inv;  // caller id -> stored node (NULL: identity)
    int32_t* color;
    int32_t* blk;
    int32_t* tries;     // searches that ended at a blocker, per node
    int32_t* list[2];   // uncoloured nodes: read list[r & 1], append to list[(r + 1) & 1]
    int32_t* cnt;       // [3] rotating list lengths
    int32_t* ncolors;   // max colour + 1
    int32_t* overflow;  // set when a d-ball (d >= 3) does not fit even the per-CTA table
    int32_t* biglist;   // d >= 3: nodes whose ball does not fit a warp's table (NULL: set overflow instead)
    int32_t* bigcnt;    // [2] rotating lengths of biglist
    uint64_t* bigtab;   // per CTA of k_color_big: open-addressing table (epoch << 32 | node)
    int32_t* bigball;   // per CTA: frontier storage
    uint32_t* epoch;    // per CTA: search counter (table entries of older searches count as empty)
    int32_t d, round;
};
cudaError_t launch_color_init(const int32_t* rowptr, const int32_t* node_id, int64_t n, uint64_t* key,
                              int32_t* inv, int32_t* tries, int32_t* color, int32_t* blk, int32_t* list,
                              cudaStream_t st);
cudaError_t launch_color_round(const ColorRound& p, cudaStream_t st);
// d >= 3: the nodes of biglist, one CTA each, with a table in global memory.
cudaError_t launch_color_big(const ColorRound& p, cudaStream_t st);
int color_big_ctas();
size_t color_big_table_entries();
size_t color_big_ball_entries();
// out[node_id[v]] = color[v] (caller numbering); counts[c] += |{v : color[v] = c}|
cudaError_t launch_color_scatter(const int32_t* color, const int32_t* node_id, int64_t n, int32_t* out,
                                 cudaStream_t st);
cudaError_t launch_color_hist(const int32_t* color, int64_t n, int32_t* counts, cudaStream_t st);

// Matrix assembly (assemble.cu).  bad[0] / bad[1]: smallest nonzero index
// with an out-of-range column / a self-loop (pattern matrices), ~0 if none.
cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int64_t n, int pattern,
                            unsigned long long* bad, cudaStream_t st);
// New row i = old row order[i], columns renamed by inv; values (optional,
// FP64 in) converted to the path precision.
// inv[order[i]] = i for a permutation of 0 .. n-1 (device arrays).
cudaError_t launch_invert_perm(const int32_t* order, int64_t n, int32_t* inv, cudaStream_t st);
cudaError_t launch_relabel(const int32_t* rp_old, const int32_t* col_old, const double* val_old,
                           const int32_t* rp_new, const int32_t* order, const int32_t* inv, int64_t n,
                           int32_t* col_new, void* val_new, int fp64, cudaStream_t st);
cudaError_t launch_convert_values(const double* in, int64_t count, void* out, int fp64, cudaStream_t st);

// Gauss quadrature of `count` tridiagonals stored column-interleaved:
// alpha[j*ld + c], beta[j*ld + c] for j < m.  psi[c] = norm2[c] * sum u1^2 f(scale[c] theta).
// With zvec != NULL also z[j*ld + c] = (U f(scale Theta) U^T e1)_j (warp-per-column kernel).
cudaError_t launch_tridiag_quad(const double* alpha, const double* beta, const double* norm2,
                                const double* scale_per_col, int count, int m, int ld, double* psi,
                                cudaStream_t);
// Theorem 4.4 bounds (lower, upper) and the geometric-mean estimate of the
// quadrature error after m steps; beta row m-1 holds beta_m.  A = scale * T.
cudaError_t launch_tridiag_bounds(const double* alpha, const double* beta, const double* norm2, const double* scale,
                                  int count, int m, int ld, double lam_min, double lam_max, int grid, double* lower,
                                  double* upper, double* estimate, cudaStream_t st);
// The same for a list of columns: entry k is column cols[k] of the ld-strided
// arrays after mcol[k] <= m steps (outputs at that column); the bounds take
// lam_max_col[k] as the upper end of the interval when lam_max_col is given.
cudaError_t launch_tridiag_quad_list(const double* alpha, const double* beta, const double* norm2,
                                     const double* scale_per_col, int count, const int32_t* cols,
                                     const int32_t* mcol, int m, int ld, double* psi, cudaStream_t);
cudaError_t launch_tridiag_bounds_list(const double* alpha, const double* beta, const double* norm2,
                                       const double* scale, int count, const int32_t* cols, const int32_t* mcol,
                                       const double* lam_max_col, int m, int ld, double lam_min, double lam_max,
                                       int grid, double* lower, double* upper, double* estimate, cudaStream_t st);
cudaError_t launch_tridiag_fvec(const double* alpha, const double* beta, const double* scale_per_col,
                                int count, int m, int ld, double* zvec, cudaStream_t);

// Gram C = X^T Y of two panel-major blocks (FP32/FP64 data, FP64 result [Kx][Ky]).
// FP32 blocks of at most 128 columns run on the tcgen05 tensor cores; err
// (device int) is set to 1 if one of that kernel's bounded waits ran out.
template <typename T>
cudaError_t launch_gram(const T* X, int kx, const T* Y, int ky, int ks, int n, double* part, int nchunks,
                        double* C, int* err, cudaStream_t);
// Per-CTA partial Grams of the tcgen05 kernel: part [chunks][kx][ky], at
// most max_chunks (one CTA per SM); *chunks_out = the CTAs launched;
// *sym_out = 1 when the partials hold E with X^T X = E + E^T (X == Y).
cudaError_t launch_gram_tc5(const float* X, int kx, const float* Y, int ky, int ks, int n, double* part,
                            int max_chunks, int* err, int* chunks_out, int* sym_out, cudaStream_t st);
// Out = (In2 ? In2 : 0) + coef * In * M, M double [kin][kout] row-major; panel-major blocks.
// FP32 blocks with err given run on the tcgen05 tensor cores (err as for
// launch_gram).
template <typename T>
cudaError_t launch_apply(const T* In, int kin, const double* M, int kout, const T* In2, T* Out, int ks, int n,
                         double coef, int* err, cudaStream_t);
cudaError_t launch_apply_tc5(const float* In, int kin, const double* M, int kout, const float* In2, float* Out, int ks,
                             int n, double coef, int* err, cudaStream_t st);
// Poll limit of the main-loop mbarrier waits of the tcgen05 kernels (< 0:
// the built-in limit); for failure-injection tests only.
void set_tensor_wait_polls(int64_t polls);
// Pivoted Cholesky of a k x k SPD matrix G (FP64) with rank cut-off tol * max diag.
// Writes Minv [k][k] (rows permuted: Q = Y Minv spans range(Y)) and rank.
// work: k * k + k doubles (R and 1 / R_jj), piv: k ints (device).  pivot =
// false takes the columns in order (piv the identity).
cudaError_t launch_chol_qr_factor(const double* G, int k, double tol, double* Minv, int* rank, double* work,
                                  int* piv, cudaStream_t, bool pivot = true);

}  // namespace vne
