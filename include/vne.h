/*
 * vne.h -- C ABI of the GB300 von Neumann entropy library (libvne.so).
 *
 * The library estimates S(A) = tr f(A), f(x) = -x log x, for a sparse
 * symmetric positive semidefinite density matrix A (normally A = L / tr L with
 * L a graph Laplacian), following Benzi, Rinelli, Simunec, "Computation of
 * the von Neumann entropy of large matrices via trace estimators and rational
 * Krylov methods" (arXiv 2212.09642).  Every trace estimator reduces to many
 * quadratic forms v^T f(A) v, which the library evaluates at once, one probe
 * vector per column of a block, on the GPU.
 *
 * Conventions shared by every call:
 *  - Every function returns a vne_status; VNE_OK (0) on success.  On failure
 *    vne_last_error(ctx) returns a human-readable message.  No C++ exception
 *    crosses the ABI.
 *  - All arrays are plain pointers with explicit sizes.  Unless a flag or the
 *    argument's description says "device", pointers are host pointers; host
 *    outputs are written before the call returns (the call synchronises its
 *    stream).
 *  - The caller owns every array it passes.  A vne_matrix owns its device
 *    copy of the matrix until vne_matrix_destroy; the context owns the
 *    device workspace it grows on demand and frees in vne_ctx_destroy.
 *  - Work is enqueued on the context's stream (vne_ctx_set_stream; default
 *    the legacy default stream).  Calls on one context are not thread safe.
 *  - Node indices are int32 on the device: n < 2^31 and nnz < 2^31.
 */
#ifndef VNE_H
#define VNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vne_status;
#define VNE_OK 0
#define VNE_EINVAL 1        /* invalid argument (size, pointer, flag, option) */
#define VNE_ENOMEM 2        /* a device or host allocation failed */
#define VNE_ENOTSYM 3       /* the CSR pattern is not symmetric */
#define VNE_ENOCONVERGE 4   /* an iterative solve did not reach its tolerance */
#define VNE_ETIMEOUT 5      /* a bounded device wait gave up */
#define VNE_EDEVICE 6       /* a CUDA runtime call or kernel failed */
#define VNE_EUNSUPPORTED 7  /* valid request that this build does not handle */

typedef struct vne_ctx vne_ctx;
typedef struct vne_matrix vne_matrix;

/* ---- flags of vne_create_density_matrix ------------------------------ */
#define VNE_FP64 0x1u            /* vectors, SpMM and Lanczos vectors in FP64 */
#define VNE_FP32 0x2u            /* vectors and SpMM in FP32; alpha, beta,
                                    inner products and the tridiagonal
                                    eigensolve stay FP64 (mixed path) */
#define VNE_NORMALIZE_TRACE 0x4u /* divide the given values by their trace */
#define VNE_IS_LAPLACIAN 0x8u    /* A 1 = 0: use implicit desingularisation */
#define VNE_INPUT_DEVICE 0x10u   /* row_ptr / col_idx / vals are device pointers */
#define VNE_REORDER 0x20u        /* relabel nodes by descending degree */
#define VNE_CHECK_SYMMETRY 0x40u /* verify the pattern is symmetric (host, O(nnz log)) */
#define VNE_REORDER_RCM 0x80u    /* relabel nodes by reverse Cuthill-McKee (host BFS, O(nnz log)):
                                    neighbours get nearby labels, so the SpMM's gathers stay local
                                    on graphs with geometric structure; wins over VNE_REORDER */

/* ---- options ---------------------------------------------------------- */
typedef struct vne_options {
    int32_t reorth;       /* 0: plain three-term Lanczos; 1: full
                             reorthogonalisation (classical Gram-Schmidt
                             twice) against the stored basis; 2: partial
                             reorthogonalisation (Simon's omega recurrence
                             estimates the loss of orthogonality from alpha
                             and beta, in FP64, with the rounding unit of the
                             vector precision; once it reaches sqrt(eps) the
                             new vector and the next one are orthogonalised,
                             twice, against the basis vectors whose estimate
                             is at least eps^(3/4)).  Reorthogonalisation
                             keeps all m + 1 Lanczos vectors of a block.
                             -1: default (full for FP64 matrices, none for
                             FP32). */
    int32_t block;        /* probe columns per device block, 0 = auto (<= 256) */
    int32_t panel;        /* columns per panel of the panel-major vector
                             layout (FP32: 8, 16, 32; FP64: 4, 8, 16), 0 = auto */
    int32_t item_nnz;     /* target nonzeros per warp work item, 0 = auto */
    int32_t n_inf_poles;  /* rational mode: poles at infinity, 0..3 (default
                             2); -1: chosen per block by the switching rule of
                             Section 5.3 (polynomial iterations until
                             err_k / err_{k-4} >= 0.75^3 for the Theorem 4.4
                             estimate, at most 16; the largest k over the
                             block's columns), the polynomial part K_k(A, c)
                             spanned by the seed CG residuals */
    int32_t cg_max_iter;  /* rational mode: multi-shift CG iteration cap */
    double cg_tol;        /* rational mode: relative residual (default 1e-8) */
    double breakdown_tol; /* Lanczos stops when beta_j <= tol * ||A||_G;
                             0 = default (1e-13 FP64, 1e-10 FP32) */
    int32_t step_variant; /* SpMM step-kernel variant 0..13 (occupancy,
                             gathers in flight, shared-memory staging, L2
                             cache policy of the gathers), -1 = auto */
    int32_t interleave;   /* 1: launch step and update panel by panel so the
                             update reads the panel while it is in L2; 0: one
                             launch each over all panels; -1 = auto */
    int32_t graphs;       /* 1: replay the Lanczos step loop of a block as a
                             CUDA graph, captured on the second call with the
                             same shape and buffers and cached in the context;
                             0: launch every kernel directly; -1 = auto (1).
                             Calls with profiling on launch directly. */
    int32_t probe_offset; /* Hutchinson: index of the first probe column of
                             the seeded Rademacher stream (probes
                             probe_offset .. probe_offset + N - 1), so that
                             ranks splitting [0, N) into ranges evaluate
                             exactly the probes of one single run; 0 default */
    int32_t check_every;  /* adaptive Lanczos (quad_tol > 0): steps between
                             checks of the error estimate, 0 = 5 */
    double quad_tol;      /* > 0: Lanczos quadratures stop once every column
                             of a block has the error estimate of Theorem 4.4
                             (geometric mean of its bounds) below quad_tol x
                             |psi|, or at krylov_steps; checks after at least
                             check_every steps.  0 = fixed krylov_steps.
                             Servers: < 0 takes half of each query's
                             rel_eps (see the serving section). */
    double spectrum_min;  /* adaptive mode: lower end of the spectral interval
                             of A for the bounds; 0 = half the smallest
                             positive Ritz value of each column (the upper end
                             is the Gershgorin bound of A) */
    int32_t gaussian_probes; /* 1: Hutchinson / Hutch++ / batched / served
                                probes are standard normal (the paper's
                                choice, Section 3.2): Box-Muller on the same
                                counters as the Rademacher entries, see
                                vne_gaussian_probes; 0 (default): Rademacher */
    int32_t items_per_warp; /* SpMM step kernel: work items a warp takes in
                               turn (1, 2 or 4; a CTA covers 8 x this many
                               items, so its reduction tail is amortised over
                               more rows), 0 = auto */
    int32_t sketch_steps;   /* servers: Lanczos steps of a query's sketch
                               f(A) Omega (any sketch keeps Hutch++ unbiased,
                               so this sets only how much variance it
                               removes), 0 = krylov_steps */
} vne_options;

/* Fill *opt with the defaults described above. */
void vne_options_default(vne_options *opt);

/* ---- context ---------------------------------------------------------- */
/* Create a context on CUDA device `device` (no allocation beyond small
 * bookkeeping).  EINVAL for a bad device index, EDEVICE if CUDA fails. */
vne_status vne_ctx_create(int32_t device, vne_ctx **ctx);
/* Free the context and its workspace.  Matrices must be destroyed first. */
vne_status vne_ctx_destroy(vne_ctx *ctx);
/* Enqueue all further work on `stream` (a cudaStream_t, may be NULL). */
vne_status vne_ctx_set_stream(vne_ctx *ctx, void *stream);
/* Message of the last failing call on this context ("" if none).  The
 * pointer stays valid until the next call on the context. */
const char *vne_last_error(const vne_ctx *ctx);
/* Library version string. */
const char *vne_version(void);
/* Measurement support.  vne_ctx_profile(ctx, 1) resets the counters and, from
 * then on, brackets every launch of the Lanczos step (SpMM) and update
 * kernels with CUDA events on the context stream; vne_ctx_stats returns the
 * number of kernels this context launched since the reset and, per kernel
 * kind (0 = step / SpMM, 1 = Lanczos update, 2 = CG update, 3 = CG
 * direction), {timed launches, total milliseconds, total algorithmic bytes}.
 * kernel_stats must hold 12 doubles (or be NULL). */
vne_status vne_ctx_profile(vne_ctx *ctx, int32_t enable);
vne_status vne_ctx_stats(const vne_ctx *ctx, int64_t *launches, double *kernel_stats);
/* CUDA-graph use of the context since its creation: step loops captured into
 * a new graph (*captured) and step loops replayed from a cached graph
 * (*replayed, including the replay right after a capture).  Either pointer
 * may be NULL.  EINVAL for a null context. */
vne_status vne_ctx_graph_stats(const vne_ctx *ctx, int64_t *captured, int64_t *replayed);
/* Lanczos steps taken by the last quadrature call on the context (the
 * largest over its blocks; krylov_steps unless quad_tol stopped earlier). */
vne_status vne_ctx_last_steps(const vne_ctx *ctx, int32_t *steps);
/* Dimension k of the polynomial part K_k(A, c) the switching rule chose in the
 * last rational call with n_inf_poles = -1 (largest over its blocks); 0 after
 * a call with a fixed number of poles at infinity. */
vne_status vne_ctx_last_poly_dim(const vne_ctx *ctx, int32_t *k);
/* Throughput ceiling of the SpMM step's access pattern (a measurement aid, not
 * part of the method): `gathers` reads of random row_bytes-byte rows (32, 64
 * or 128) from a device table of table_bytes, plus one streaming read of
 * stream_bytes, on the context's stream; *gather_gbs = gathered bytes per
 * second (GB/s), best of `reps` >= 1 launches after one warm-up.  The buffers
 * are context workspace (kept until vne_ctx_destroy).  EINVAL for bad sizes. */
vne_status vne_measure_gather(vne_ctx *ctx, uint64_t table_bytes, int32_t row_bytes, uint64_t gathers,
                              uint64_t stream_bytes, int32_t reps, double *gather_gbs);

/* ---- density matrix (Section 2, eq. graph_laplacian) ------------------ */
/* Copy a symmetric CSR matrix to the device.
 *   n        number of rows (= columns), 1 <= n < 2^31
 *   row_ptr  int64[n+1], row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz < 2^31
 *   col_idx  int32[nnz], 0 <= col < n
 *   vals     double[nnz] or NULL.  NULL: the matrix is the graph Laplacian
 *            L = D - W of the pattern (off-diagonal entries = -1, no
 *            self-loops or duplicates allowed; diagonal = degree), and the
 *            density matrix is rho = L / tr(L) (VNE_NORMALIZE_TRACE and
 *            VNE_IS_LAPLACIAN implied).  The Laplacian is kept implicit:
 *            only the pattern is stored on the device.
 *            Non-NULL: entries of a general symmetric matrix (diagonal
 *            included), stored in the path precision.
 *   flags    exactly one of VNE_FP64 / VNE_FP32, plus optional flags above.
 * Errors: EINVAL (bad sizes, indices, flags; zero trace), ENOTSYM (with
 * VNE_CHECK_SYMMETRY), ENOMEM, EDEVICE.  *out is NULL on failure. */
vne_status vne_create_density_matrix(vne_ctx *ctx, int64_t n, const int64_t *row_ptr,
                                     const int32_t *col_idx, const double *vals,
                                     uint32_t flags, vne_matrix **out);
vne_status vne_matrix_destroy(vne_matrix *mat);
/* n, stored nnz, trace of the matrix before normalisation, Gershgorin bound
 * ||A||_G of the normalised matrix.  Any output pointer may be NULL. */
vne_status vne_matrix_info(const vne_matrix *mat, int64_t *n, int64_t *nnz, double *trace,
                           double *norm_bound);

/* ---- quadratic forms (Section 4, eq. rational-krylov-approximation-quadform)
 * psi_j ~ b_j^T f(A) b_j for the k columns b_j of `vectors`.
 *   vectors       double[n][k] row-major (host, or device with
 *                 VNE_INPUT_DEVICE in `vec_flags`)
 *   krylov_steps  m >= 1 Lanczos steps (polynomial mode) or, with poles,
 *                 ignored (the space is fixed by the poles)
 *   poles         NULL: polynomial Krylov (Lanczos Gauss quadrature).
 *                 Otherwise num_poles positive shifts s (poles xi = -s):
 *                 rational Krylov space span{c, Ac, .., A^l c,
 *                 (A + s_i I)^{-1} c}, l = opt->n_inf_poles, solved by
 *                 multi-shift CG (Sections 4.2, 5.3).
 *   psi           double[k] output (host)
 *   alpha_beta    NULL or double[k][2m] output (host): per column the
 *                 Lanczos alpha_1..alpha_m then beta_1..beta_m of the
 *                 normalised matrix (zeros after a breakdown).  Polynomial
 *                 mode only.
 * With VNE_IS_LAPLACIAN (or a pattern matrix) each b is replaced by
 * b - mean(b) 1 (implicit desingularisation, Remark graph-laplacian-krylov),
 * which leaves b^T f(A) b unchanged. */
#define VNE_VECTORS_DEVICE 0x1u
vne_status vne_quadform_batch(vne_matrix *mat, const double *vectors, int32_t k, uint32_t vec_flags,
                              int32_t krylov_steps, const double *poles, int32_t num_poles,
                              const vne_options *opt, double *psi, double *alpha_beta);

/* ---- rational Krylov quadratic forms (Sections 4, 4.2, 5.3) -----------
 * psi_j ~ b_j^T f(A) b_j in the rational Krylov space with poles -shifts[i]
 * (i < num_shifts <= 8) and opt->n_inf_poles poles at infinity:
 * span{c, A c, .., A^l c, (A + s_i I)^{-1} c}, c the (desingularised) b_j.
 * The shifted systems are solved together by multi-shift conjugate
 * gradients seeded on the smallest shift, each shift retired once its
 * recursive relative residual is <= opt->cg_tol (default 1e-8) or after
 * opt->cg_max_iter iterations; the basis is orthonormalised in pole order
 * (first vector c / ||c||) and psi = ||c||^2 e1^T f(V^T A V) e1.
 *   shifts        NULL: default log-spaced shifts on [1e-4 ||A||_G, ||A||_G]
 *   cg_iterations NULL or int32[num_shifts][k]: iterations until each shift converged
 *   residuals     NULL or double[num_shifts][k]: final recursive relative residuals
 * vne_quadform_batch and vne_entropy_probing take the same path when they
 * are given poles. */
vne_status vne_quadform_rational(vne_matrix *mat, const double *vectors, int32_t k, uint32_t vec_flags,
                                 const double *shifts, int32_t num_shifts, const vne_options *opt, double *psi,
                                 int32_t *cg_iterations, double *residuals);

/* ---- Hutchinson (Section 3.2, eq. hutchinson-stochastic-trace-estimator)
 * estimate = (1/N) sum_j psi_m(x_j), x_j Rademacher columns 0..N-1 of the
 * counter-based generator with `seed`; std_error = sample std / sqrt(N);
 * psi_out = the N quadratic forms.  std_error, psi_out may be NULL. */
vne_status vne_entropy_hutchinson(vne_matrix *mat, int32_t num_vectors, int32_t krylov_steps,
                                  uint64_t seed, const vne_options *opt, double *estimate,
                                  double *std_error, double *psi_out);

/* ---- Hutch++ (Section 3.2, eq. Hutch++_formula)
 * Omega = Rademacher columns 0..N_r-1, G = columns N_r..N_r+N_H-1.
 * Y = f(A) Omega by the Lanczos matvec approximation
 * (eq. rational-krylov-approximation-matvec), Q = orth(Y) = the
 * column-pivoted QR factor of Y (a pivoted Cholesky-QR pass, then an
 * unpivoted one), estimate = sum_i psi(q_i) + (1/N_H) sum_j psi((I - Q Q^T)
 * g_j).  parts (NULL ok) receives {low-rank part, residual part, rank of Q}.
 * N_r in [1, 128], N_H in [0, 128].  ETIMEOUT if a bounded wait of the
 * tensor-core sketch kernels ran out. */
vne_status vne_entropy_hutchpp(vne_matrix *mat, int32_t sketch_cols, int32_t hutch_vectors,
                               int32_t krylov_steps, uint64_t seed, const vne_options *opt,
                               double *estimate, double *parts);

/* ---- Hutch++ in two stages (Section 3.2, eq. Hutch++_formula), for
 * callers that split one estimate over several GPUs (the quadratic forms are
 * independent: remark after eq. rational-krylov-approximation-matvec) or
 * inspect its parts.  vne_entropy_hutchpp is stage 1 over all N_r columns
 * followed by stage 2 over all N_r + N_H quadratic forms, with the same
 * results column for column.
 *
 * Stage 1: columns [col_begin, col_begin + ncols) of the sketch Y = f(A)
 * Omega (eq. rational-krylov-approximation-matvec), Omega the probe columns
 * 0..N_r-1 of `seed` (Rademacher, or Gaussian with opt->gaussian_probes).
 * Every column is its own Lanczos recurrence: a column's value does not
 * depend on the range it is computed in.
 *   Y      [n][ncols] row-major, rows in the caller's node numbering, in the
 *          matrix's precision (float for VNE_FP32, double for VNE_FP64); a
 *          device pointer with VNE_VECTORS_DEVICE in flags, else host.
 * ncols in [1, 256].  The call synchronises the context stream. */
vne_status vne_hutchpp_sketch(vne_matrix *mat, int32_t col_begin, int32_t ncols, int32_t krylov_steps,
                              uint64_t seed, const vne_options *opt, uint32_t flags, void *Y);

/* Stage 2: from the whole sketch Y ([n][N_r], layout and flags as in stage
 * 1), Q = orth(Y) as in vne_entropy_hutchpp, G' = (I - Q Q^T) G with G the
 * probe columns N_r..N_r+N_H-1, and the quadratic forms psi_m of the columns
 * [q_1 .. q_{N_r} | g'_1 .. g'_{N_H}] with index in
 * [col_begin, col_begin + ncols): index i < N_r is q_{i+1} (psi = 0 for
 * i >= rank), index N_r + j is g'_{j+1}.
 *   psi     host double[ncols]
 *   pivots  host int32[N_r] or NULL: the sketch column chosen as the i-th
 *           pivot of Q (q_{i+1}), -1 beyond the rank
 *   rank    host int32 or NULL: the numerical rank of Y (pivots above
 *           1e-13 (FP64) / 1e-5 (FP32) of the largest diagonal of Y^T Y)
 * The estimate is sum_{i < rank} psi[i] + (1/N_H) sum_j psi[N_r + j].
 * EINVAL for a column range outside [0, N_r + N_H), N_r outside [1, 128] or
 * N_H outside [0, 128]; ETIMEOUT as for vne_entropy_hutchpp. */
vne_status vne_hutchpp_project(vne_matrix *mat, const void *Y, uint32_t flags, int32_t sketch_cols,
                               int32_t hutch_vectors, int32_t krylov_steps, uint64_t seed, int32_t col_begin,
                               int32_t ncols, const vne_options *opt, double *psi, int32_t *pivots,
                               int32_t *rank);

/* ---- probing (Section 3.1, eqs. probing_vectors, trace_probing)
 * T_d = sum_l psi(v_l), v_l the indicator of colour class l.
 *   coloring   int32[n] colours 0..s-1 (host), or NULL to compute the greedy
 *              distance-`distance` colouring (Algorithm 1, nodes by
 *              descending degree, ties by ascending id) with
 *              vne_matrix_coloring.
 *   poles      as in vne_quadform_batch (NULL: polynomial Lanczos).
 *   num_colors output s (may be NULL). */
vne_status vne_entropy_probing(vne_matrix *mat, const int32_t *coloring, int32_t distance,
                               int32_t krylov_steps, const double *poles, int32_t num_poles,
                               const vne_options *opt, double *estimate, int32_t *num_colors);

/* ---- probing method with the choice of d (Section 5.1, Algorithm 2)
 * Target: |estimate - S| <~ eps S (a heuristic, not a guarantee).
 *   1. T_1, T_2, T_3: probing at d = 1, 2, 3 (colourings by
 *      vne_matrix_coloring).  T_1's quadratic forms stop when the Theorem
 *      4.4 estimate of each is <= eps/2 x psi_l; then eps_abs = eps/2 x T_1
 *      (T_1 <= S for a graph Laplacian) and every later quadratic form stops
 *      at <= eps_abs |V_l| / n (eq. algorithm-probing-quadform-error-
 *      requirement-abs), so the sum is within eps_abs of T_d.
 *   2. d from the fit of |S - T_d| ~ C q^d / d^k to |T_2 - T_1|, |T_3 - T_2|
 *      for k = 2 and 3, the larger of the two smallest d with a modelled
 *      error <= eps_abs (eq. probing-heuristic-convergence).  Without a
 *      decaying fit: the smallest d with |T_{d+1} - T_d| <= eps_abs.  d is
 *      capped at d_max.
 *   3. estimate = T_d (reused when d <= 3).
 * The Lanczos quadratures use krylov_steps as the step limit and the
 * options' check_every / spectrum_min (quad_tol is ignored).  Polynomial
 * Lanczos only.  report may be NULL.  EINVAL: eps outside (0, 1),
 * krylov_steps outside [1, 128], d_max outside [1, 1024]. */
#define VNE_PROBING_RULE_FIT 0          /* d from the fitted error model */
#define VNE_PROBING_RULE_DIFFERENCES 1  /* d from consecutive differences */
#define VNE_PROBING_RULE_CAPPED 2       /* d = d_max before the target was met */
typedef struct vne_probing_report {
    double t[3];           /* T_1, T_2, T_3 */
    double eps_abs;        /* eps/2 x T_1 */
    int32_t distance;      /* d of the estimate */
    int32_t num_colors;    /* colours of the distance-d colouring */
    int32_t colors_d[3];   /* colours at d = 1, 2, 3 */
    int32_t steps_d[3];    /* Lanczos steps at d = 1, 2, 3 (largest over blocks) */
    int32_t steps_chosen;  /* Lanczos steps at the chosen d */
    int32_t rule;          /* VNE_PROBING_RULE_* */
    int32_t evaluated;     /* T_1..T_evaluated were computed in sequence */
    int32_t reserved;
} vne_probing_report;
/* Caller-supplied colouring for vne_entropy_probing_auto (for instance an
 * optimal colouring of a structured graph): fill colors (host int32[n],
 * caller numbering) with a distance-`distance` colouring and return the
 * number of colours s (colours in [0, s)), or a value < 1 on failure (the
 * call then returns EINVAL).  Called from the calling thread. */
typedef int32_t (*vne_coloring_fn)(void *user, int32_t distance, int64_t n, int32_t *colors);
vne_status vne_entropy_probing_auto(vne_matrix *mat, double eps, int32_t krylov_steps, int32_t d_max,
                                    vne_coloring_fn coloring_fn /* NULL: vne_matrix_coloring */, void *user,
                                    const vne_options *opt, double *estimate, vne_probing_report *report);

/* Greedy distance-d colouring of a symmetric CSR pattern (Algorithm 1) on
 * the host: colors int32[n] receives colours 0..s-1, *num_colors = s. */
vne_status vne_greedy_coloring(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                               int32_t distance, int32_t *colors, int32_t *num_colors);

/* Greedy distance-d colouring (Algorithm 1, Section 3.1) of the matrix's
 * graph on the device: the colouring Algorithm 1 computes (nodes by
 * descending degree, ties by ascending caller id, each node the smallest
 * colour not used by an earlier node within distance `distance`), node for
 * node.  Nodes are coloured in rounds, each node as soon as every node of
 * higher priority in its distance-d ball has its colour.  For distance >= 3
 * the nodes within distance d - 1 are de-duplicated in a warp's shared
 * memory (about 1,500 nodes) or, for larger balls, by a whole CTA in global
 * memory (about 196,000 nodes); a larger ball gives EUNSUPPORTED (the
 * sequential sweep would need n x 196,000 steps or more).
 *   colors         host int32[n] (may be NULL): colours in the caller's
 *                  numbering (the numbering of vne_create_density_matrix's
 *                  input, whatever the relabelling).
 *   num_colors     s (may be NULL).
 *   device_rounds  rounds run on the device (may be NULL).
 * EINVAL for distance < 1. */
vne_status vne_matrix_coloring(vne_matrix *mat, int32_t distance, int32_t *colors, int32_t *num_colors,
                               int32_t *device_rounds);

/* ---- kernel-level entry points (device pointers; used by the tests) ---
 * Y = A X for a block of k columns, X and Y device arrays [n][k] row-major
 * in the matrix's precision (float or double), rows in the caller's node
 * numbering.  A is the normalised density matrix rho = L / tr(L) (Section
 * 2). */
vne_status vne_spmm(vne_matrix *mat, const void *X, void *Y, int32_t k);

/* C = X^T Y (the Gram of the Hutch++ sketch, Section 3.2: Y^T Y for the
 * Cholesky-QR and Q^T G for the projection) on the tcgen05 tensor cores.
 * X, Y: device float blocks in panel-major layout [k / ks][n][ks] (ks = 8,
 * 16 or 32 columns per panel), kx, ky <= 128 columns, multiples of ks;
 * C: host double[kx][ky] row-major.  TF32 three-product split (FP32
 * accuracy), FP32 accumulation within a CTA, FP64 across CTAs.  EINVAL for
 * bad sizes or NULL buffers; ETIMEOUT if a bounded wait of the kernel ran
 * out. */
vne_status vne_block_gram(vne_ctx *ctx, const float *X, int32_t kx, const float *Y, int32_t ky, int32_t ks,
                          int64_t n, double *C);

/* Out = In2 + coef In M (the block products of the Hutch++ sketch, Section
 * 3.2: Q = Y R^{-1} and G - Q (Q^T G)) on the tcgen05 tensor cores.  In,
 * In2 (nullable: no addend), Out: device float blocks in panel-major layout
 * [k / ks][n][ks] with kin and kout columns (<= 128, multiples of ks = 8, 16
 * or 32); M: host double[kin][kout] row-major.  TF32 three-product split
 * (FP32 accuracy).  Out must not overlap In or In2.  EINVAL for bad sizes or
 * NULL buffers; ETIMEOUT if a bounded wait of the kernel ran out. */
vne_status vne_block_apply(vne_ctx *ctx, const float *In, int32_t kin, const double *M, int32_t kout,
                           const float *In2, float *Out, int32_t ks, int64_t n, double coef);

/* Gauss quadrature of given tridiagonals (Section 4): for each of `count`
 * columns, T = tridiag(beta[0..m-2], alpha[0..m-1]), psi = norm2 *
 * sum_j u_{1j}^2 f(scale * theta_j).  alpha, beta: double[count][m] host;
 * beta[m-1] is ignored; a zero beta_j truncates T after row j. */
vne_status vne_tridiag_quadrature(vne_ctx *ctx, const double *alpha, const double *beta,
                                  const double *norm2, double scale, int32_t count, int32_t m,
                                  double *psi);

/* A-posteriori bounds of Theorem 4.4 (polynomial Krylov case) for the
 * quadratures above after m Lanczos steps: beta[m-1] holds beta_m of the
 * decomposition A V_m = V_m T_m + beta_m v_{m+1} e_m^T (T, beta_m in the
 * units of A / scale).  With g_m the function of eq. error-bound--gm-definition
 * and f(x) = -x log x, lower = norm2 * min |g_m|, upper = norm2 * max |g_m|
 * over [lam_min, lam_max] (0 < lam_min < lam_max, a spectral interval of A),
 * estimate = norm2 * sqrt(min max) (eq. error-bound-a-posteriori--estimate).
 * The extrema are taken over `grid` geometrically and `grid` linearly spaced
 * points plus the Ritz values inside the interval.  A block that broke down
 * (a zero beta_j, j < m) or beta_m = 0 gives 0.  Host arrays as for
 * vne_tridiag_quadrature; outputs double[count].  EINVAL for a bad interval,
 * grid < 1 or m outside [1, 128]. */
vne_status vne_quadrature_bounds(vne_ctx *ctx, const double *alpha, const double *beta, const double *norm2,
                                 double scale, int32_t count, int32_t m, double lam_min, double lam_max,
                                 int32_t grid, double *lower, double *upper, double *estimate);

/* The probe vectors of the trace estimators (Section 3.2; Rademacher
 * entries, E[x x^T] = I): fill a device array [n][k] (row-major, float or
 * double per `fp64`) with columns col_begin..col_begin+k-1 for node ids
 * 0..n-1.  EINVAL for bad sizes or a NULL buffer. */
vne_status vne_rademacher(vne_ctx *ctx, uint64_t seed, int64_t n, int32_t col_begin, int32_t k,
                          int32_t fp64, void *out_device);
/* The Gaussian probes of Section 3.2 on the same counters
 * (vne_options.gaussian_probes):
 * with h1 = h(j, i) the Rademacher hash of column j and node i and
 * h2 = mix64(h1 + 0x9E3779B97F4A7C15), u1 = ((h1 >> 11) + 1/2) 2^-53,
 * u2 = (h2 >> 11) 2^-53, x = sqrt(-2 log u1) cos(2 pi u2) (Box-Muller), FP64.
 * out_device: device double[n][k] row-major, columns col_begin.. .  EINVAL
 * for bad sizes or a NULL buffer. */
vne_status vne_gaussian_probes(vne_ctx *ctx, uint64_t seed, int64_t n, int32_t col_begin, int32_t k,
                               double *out_device);

/* ---- schedule autotuner --------------------------------------------------
 * Time the Lanczos step and update kernels of `mat` on one block of k
 * Rademacher columns for `steps` Lanczos steps under every candidate schedule
 * (panel width, nonzeros per warp work item, step-kernel variant, per-panel
 * interleaving); keep the fastest as the matrix's default for options left at
 * "auto" (panel = 0, item_nnz = 0, step_variant = -1, interleave = -1) and
 * report it in *chosen and its time per Lanczos step in *ms_per_step.
 * The choice is also cached in the context for matrices created later with
 * the same n, nnz, maximum degree, precision and kind. */
vne_status vne_autotune(vne_matrix *mat, int32_t k, int32_t steps, vne_options *chosen, double *ms_per_step);

/* ---- batched uneven graphs (one launch per step over all graphs) ------
 * Packs `count` matrices (same precision) block-diagonally and runs
 * Hutchinson's estimator (Section 3.2) with N Rademacher vectors and m
 * Lanczos steps (Section 4) on each, all graphs advancing together.  estimates double[count]; std_errors may be
 * NULL.  Each graph's result is independent of the others. */
vne_status vne_batch_hutchinson(vne_matrix *const *mats, int32_t count, int32_t num_vectors,
                                int32_t krylov_steps, uint64_t seed, const vne_options *opt,
                                double *estimates, double *std_errors);

/* ---- serving: continuous batching of entropy queries -------------------
 * A query asks for S(rho) of one graph to a relative accuracy eps.  It is
 * answered by Hutch++ (Section 3.2, eq. Hutch++_formula) in an adaptive
 * form, the stated proxy for the adaptive Hutch++ of Section 5.2 (whose
 * steps the paper does not print): at admission a sketch of N_r = 4 columns
 * (probe columns 0..3 of the query's seed) gives Q = orth(f(A) Omega) and
 * psi(q_i) for the query alone; then blocks of `block_vectors` deflated
 * probes g' = (I - Q Q^T) g (probe columns 4, 5, ... in block order) run
 * `krylov_steps` Lanczos steps each, until 2.576 * stderr(psi(g')) <=
 * (eps / 2) * |sum psi(q_i) + mean psi(g')| after at least two blocks, or
 * max_vectors probes.  The estimate is sum psi(q_i) + mean psi(g').
 * With opt->quad_tol != 0 at creation the Lanczos runs of a block stop
 * together at the first multiple of opt->check_every (default 5) below
 * krylov_steps at which every column's Theorem 4.4 estimate is at most
 * tau |psi| (lam_min half the column's smallest positive Ritz value, lam_max
 * the Gershgorin bound of A, |g_m| over 256 geometric and 256 linear points
 * and the Ritz values in between); tau = quad_tol, or for quad_tol < 0 half the
 * query's rel_eps, the Krylov share of the error budget of Section 5.2.
 * quad_tol = 0: every block runs krylov_steps steps.  The sketch columns
 * always run krylov_steps steps.
 *
 * Device memory: on the first submission the server takes an arena sized
 * from `hbm_budget_bytes` (the server's scalars, then rows and nonzeros,
 * up to 12 nonzeros per row); a query keeps its packed CSR (copied once, at
 * admission), its block's two Lanczos slots and u, and its Q at a row range
 * of the arena from admission to completion.  A query counts (n + 1) rows
 * of (8 + (3 K + 4) * element size) bytes plus 4 bytes per nonzero against
 * the budget; queries are admitted FIFO while that fits and a slot of the
 * `max_active` is free.  All queries of a server share one precision (that
 * of the first one); FP32 and FP64 graph patterns are accepted.
 *
 * Each vne_server_step is one tick: admission, then ONE Lanczos step of
 * every active query, each at its own step j of its own block (one step
 * kernel and one update kernel over all active queries, with per-query step
 * counters; queries whose block starts get their deflated start vectors
 * first, queries whose block ends get their Gauss quadratures and update
 * their statistics after).  A query's numbers depend only on its graph,
 * seed and the server's block_vectors and krylov_steps, so its result is
 * bit-identical alone and in any mix.  Matrices must be graph patterns of
 * the server's context and stay alive until their queries are done. */
typedef struct vne_server vne_server;
vne_status vne_server_create(vne_ctx *ctx, uint64_t hbm_budget_bytes, int32_t max_active, int32_t krylov_steps,
                             int32_t block_vectors, const vne_options *opt, vne_server **out);
vne_status vne_server_destroy(vne_server *srv);
/* Queue a query: relative accuracy rel_eps, probe seed, cap on probe vectors.
 * ENOMEM if the query alone exceeds the budget. */
vne_status vne_server_submit(vne_server *srv, vne_matrix *mat, double rel_eps, uint64_t seed, int32_t max_vectors,
                             int32_t *ticket);
/* One tick (admission + one Lanczos step of every active query); completed =
 * queries retired in it, active = queries that ran in it. */
vne_status vne_server_step(vne_server *srv, int32_t *completed, int32_t *active);
/* state 0 queued / 1 active / 2 done; ticks[3] = {submit, admit, done} tick. */
vne_status vne_server_result(const vne_server *srv, int32_t ticket, int32_t *state, double *estimate,
                             double *std_error, int64_t *vectors_used, int64_t *ticks);
vne_status vne_server_info(const vne_server *srv, int32_t *queued, int32_t *active, uint64_t *used_bytes);

/* ---- failure injection (test hooks) -----------------------------------
 * Host-side fault injection for the library's own error paths; nothing here
 * touches a kernel.  Every device and pinned host buffer the library
 * allocates goes through one pair of counted wrappers.
 * vne_debug_fail_allocation(k): the k-th allocation from now on (k >= 1)
 * fails as if the memory were exhausted, so the call that makes it returns
 * VNE_ENOMEM; k = 0 switches the injection off.  Process-wide, not thread
 * safe with concurrent calls.  EINVAL for k < 0.
 * vne_debug_live_allocations: the number of device buffers and of pinned
 * host buffers the library currently holds (across all contexts and
 * matrices), to check that a failed call leaks nothing. */
vne_status vne_debug_fail_allocation(int64_t k);
vne_status vne_debug_live_allocations(int64_t *device_buffers, int64_t *pinned_buffers);
/* Poll limit of the main-loop mbarrier waits of the tcgen05 sketch kernels
 * (vne_block_gram, vne_block_apply and the Hutch++ orthonormalisation):
 * polls >= 0 makes those waits give up after that many polls (0: at once),
 * so that the kernels take their time-out path -- set the error flag, wait
 * with the full limit for the MMAs already issued, free the tensor memory
 * and return -- and the call reports VNE_ETIMEOUT; polls < 0 restores the
 * built-in limit (2^20 polls).  Process-wide. */
vne_status vne_debug_tensor_wait_limit(int64_t polls);

/* ---- allocation-free quadratic forms ---------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need the result (code bound
 * to another framework's memory pool, allocator-free real-time loops,
 * embedding hosts that hand over only the buffers they own).
 *
 * Same quantity as vne_quadform_batch in the FP64 path with a plain
 * three-term recurrence (reorth = 0): psi[j] ~ b_j^T f(rho) b_j for the graph
 * Laplacian density rho = L / tr(L) of a CSR pattern, with implicit
 * desingularisation.  Everything is caller-owned device memory:
 *   row_ptr  int32[n+1], nondecreasing, row_ptr[n] = nnz > 0
 *   col_idx  int32[nnz] with 0 <= col < n -- a symmetric pattern without
 *            self-loops
 *   vectors  double[n][k] row-major
 *   psi      double[k] output
 * Work goes on `stream` (a cudaStream_t, NULL for the legacy stream) on the
 * current device; the call returns without synchronising.  The kernels check
 * the CSR as they read it: a negative or decreasing row offset, nnz = 0 or a
 * column outside [0, n) is never dereferenced and makes every psi NaN (the
 * call cannot report it, since it does not wait for the GPU).  Symmetry is
 * not checked.  If the calling thread already has a pending CUDA error, the
 * call launches nothing, leaves that error in place and returns
 * VNE_EDEVICE; a failing launch of its own also gives VNE_EDEVICE.
 *
 * Nothing is allocated: all intermediates live in one static device array of
 * VNE_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  It needs about 24 n ceil(k/8)*8 bytes plus small
 * terms; larger problems fail with VNE_EINVAL.  All calls share the array,
 * which keeps the previous call's contents (each call clears what must
 * start at zero), so calls that overlap on a GPU race: serialise them.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Not thread safe. */
#define VNE_NOALLOC_SCRATCH_BYTES (32u << 20)
vne_status vne_quadform_noalloc(void *stream, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                const double *vectors, int32_t k, int32_t krylov_steps, double *psi);

#ifdef __cplusplus
}
#endif
#endif /* VNE_H */
