// Hutch++ (Section 3.2, eq. Hutch++_formula): the sketch f(A) Omega by the
// Lanczos matvec approximation (eq. rational-krylov-approximation-matvec),
// Q by pivoted Cholesky-QR on the tcgen05 Grams, the projected Hutchinson
// vectors and one Lanczos block for all quadratic forms.
//
// The estimate is built from two stages that the C ABI also exposes, so that
// one estimate can be split over several GPUs (the quadratic forms are
// independent; remark after eq. rational-krylov-approximation-matvec):
//   sketch   columns [c0, c0 + k) of Y = f(A) Omega; every column is its own
//            Lanczos recurrence, so a column's value does not depend on which
//            other columns share its block;
//   project  from the whole Y: Q = orth(Y), G' = (I - Q Q^T) G and the
//            quadratic forms of any range of the columns [Q | G'].
// orth(Y) is the column-pivoted QR factor of Y: a pivoted Cholesky of Y^T Y
// (at every step the column with the largest remaining norm) gives Q1 =
// Y P R^{-1}, and a second, unpivoted Cholesky-QR pass on Q1 restores
// orthogonality to rounding level without reordering the columns.
#include "engine.h"

namespace {

__global__ void k_gamma(const double* norm2, const double* sigma, const double* zvec, int m, int K, double* gamma) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * K) return;
    int c = idx % K;
    gamma[idx] = sqrt(norm2[c]) * sigma[idx] * zvec[idx];
}

struct HppPlan {
    Problem* P;
    Sched sc;
    int ks, n, m;
    uint64_t seed_mixed;
    bool gaussian;
    int reorth;  // 0 none, 1 full, 2 partial
};

template <typename T>
HppPlan hpp_plan(vne_matrix* M, const vne_options* o, int m, uint64_t seed) {
    HppPlan h;
    h.P = matrix_problem(M, o);
    h.sc = resolve_sched(M, o);
    h.ks = h.sc.ks;
    check_ks<T>(M->ctx, h.ks);
    h.n = (int)M->n;
    h.m = m;
    h.seed_mixed = seed_mix(seed);
    h.gaussian = o && o->gaussian_probes != 0;
    h.reorth = want_reorth(M, o);
    return h;
}

// Sketch columns [c0, c0 + k) of Y = f(A) Omega into a panel-major block of
// Kp = round_up(k, ks) columns (workspace `ytag`; padding columns zero).
template <typename T>
T* sketch_block(vne_matrix* M, const HppPlan& h, int c0, int k, const std::string& ytag, int* Kp_out) {
    vne_ctx* ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    Problem& P = *h.P;
    StartSource s{};
    s.kind = SRC_RADEMACHER;
    s.gaussian = h.gaussian;
    s.seed_mixed = h.seed_mixed;
    s.col_begin = c0;
    s.ncols = k;
    BlockOut sk;
    // the sketch block only feeds f(A) Omega: its quadratures are not needed
    run_block<T>(ctx, P, s, nullptr, k, h.ks, h.m, h.reorth, true, M->desing, "sketch", sk, h.sc.variant,
                 h.sc.interleave, h.sc.graph, false);
    const int Kp = sk.Kp, m = h.m;
    double* zvec = ws_get_t<double>(ctx, "zvec", (size_t)m * Kp);
    VNE_TRY_CUDA(ctx, launch_tridiag_fvec(sk.alpha, sk.beta, sk.scale, Kp, m, Kp, zvec, st));
    double* gamma = ws_get_t<double>(ctx, "gamma", (size_t)m * Kp);
    k_gamma<<<(m * Kp + 255) / 256, 256, 0, st>>>(sk.norm2, sk.sigma, zvec, m, Kp, gamma);
    VNE_TRY_CUDA(ctx, cudaGetLastError());
    T* Y = ws_get_t<T>(ctx, ytag, (size_t)Kp * h.n);
    RecoverParams<T> rp{};
    rp.basis = (const T*)sk.basis;
    rp.slot_stride = sk.slot_stride;
    rp.y = Y;
    rp.gamma = gamma;
    rp.m = m;
    rp.K = Kp;
    rp.n_total = h.n;
    rp.tiles_per_panel = P.tiles_per_panel();
    rp.tiles = P.d_tiles;
    VNE_TRY_CUDA(ctx, launch_recover<T>(rp, h.ks, sk.panels, st));
    ctx->launches += 3;  // fvec, gamma, recover
    *Kp_out = Kp;
    return Y;
}

struct ProjectOut {
    std::vector<double> psi;  // the selected columns' quadratic forms
    std::vector<int> piv;     // [Nr]: sketch column of q_i, -1 beyond the rank
    int rank = 0;
};

// From the sketch Y (panel-major, Kp >= Nr columns, the first Nr real):
// Q = orth(Y), G' = G - Q (Q^T G), and the quadratic forms of the columns
// [c0, c0 + k) of [q_1 .. q_Nr | g'_1 .. g'_NH] (all of them for k < 0).
template <typename T>
void project_block(vne_matrix* M, const HppPlan& h, const T* Y, int Kp, int Nr, int NH, int c0, int k,
                   ProjectOut& out, const Adaptive* ad = nullptr) {
    vne_ctx* ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    Problem& P = *h.P;
    const int n = h.n, ks = h.ks, m = h.m;
    const size_t blk = (size_t)Kp * n;
    // Q = orthonormal basis of range(Y): pivoted Cholesky-QR, then an
    // unpivoted second pass
    const int nch = std::max(1, std::min(4 * ctx->sm_count, (n + 63) / 64));
    double* gpart = ws_get_t<double>(ctx, "gram.part", (size_t)nch * Kp * std::max(Kp, 128));
    double* G1 = ws_get_t<double>(ctx, "G1", (size_t)Kp * Kp);
    double* Minv = ws_get_t<double>(ctx, "Minv", (size_t)Kp * Kp);
    int* drank = ws_get_t<int>(ctx, "rank", 3);  // two ranks + the tensor-core kernels' wait flag
    int* gerr = drank + 2;
    double* cwork = ws_get_t<double>(ctx, "chol.work", (size_t)Kp * Kp + Kp);
    int* cpiv = ws_get_t<int>(ctx, "chol.piv", 2 * (size_t)Kp);
    VNE_TRY_CUDA(ctx, cudaMemsetAsync(gerr, 0, sizeof(int), st));
    T* Q1 = ws_get_t<T>(ctx, "Q1", blk);
    // Q and (I - Q Q^T) G share one buffer: Q in block columns [0, Kp), the
    // projected Hutchinson vectors in [Kp, Kp + Kg)
    const int Kg = NH > 0 ? ((NH + ks - 1) / ks) * ks : 0;
    VNE_REQUIRE(ctx, Kg <= 128, VNE_EUNSUPPORTED, "N_H > 128 not supported in one projection block");
    T* QG = ws_get_t<T>(ctx, "QG", (size_t)(Kp + Kg) * n);
    T* Q = QG;
    const double tol = M->fp64 ? 1e-13 : 1e-5;
    VNE_TRY_CUDA(ctx, launch_gram<T>(Y, Kp, Y, Kp, ks, n, gpart, nch, G1, gerr, st));
    VNE_TRY_CUDA(ctx, launch_chol_qr_factor(G1, Kp, tol, Minv, drank, cwork, cpiv, st, true));
    VNE_TRY_CUDA(ctx, launch_apply<T>(Y, Kp, Minv, Kp, nullptr, Q1, ks, n, 1.0, gerr, st));
    VNE_TRY_CUDA(ctx, launch_gram<T>(Q1, Kp, Q1, Kp, ks, n, gpart, nch, G1, gerr, st));
    VNE_TRY_CUDA(ctx, launch_chol_qr_factor(G1, Kp, tol, Minv, drank + 1, cwork, cpiv + Kp, st, false));
    VNE_TRY_CUDA(ctx, launch_apply<T>(Q1, Kp, Minv, Kp, nullptr, Q, ks, n, 1.0, gerr, st));
    ctx->launches += 12;  // 2 x (gram + reduce + symmetrise + factor + inverse + apply)
    if (Kg > 0) {
        // G (probe columns N_r..N_r+N_H-1), then G' = G - Q (Q^T G)
        const size_t gblk = (size_t)Kg * n;
        T* Gr = ws_get_t<T>(ctx, "Graw", gblk);
        T* Gp = QG + (size_t)Kp * n;
        StartSource sg{};
        sg.kind = SRC_RADEMACHER;
        sg.gaussian = h.gaussian;
        sg.seed_mixed = h.seed_mixed;
        sg.col_begin = Nr;
        sg.ncols = NH;
        StartParams<T> spp{};
        spp.src = sg;
        spp.node_id = P.node_id;
        spp.seg = P.d_segs;
        spp.nseg = 1;
        spp.K = Kg;
        spp.n_total = n;
        spp.tiles_per_panel = P.tiles_per_panel();
        spp.tiles = P.d_tiles;
        spp.desing = 0;
        spp.w1 = Gr;
        spp.mean = ws_get_t<double>(ctx, "mean", Kg);
        spp.norm2 = ws_get_t<double>(ctx, "g.norm2", Kg);
        spp.sig1 = ws_get_t<double>(ctx, "g.sig", Kg);
        spp.part = ws_get_t<double>(ctx, "part", (size_t)(Kg / ks) * P.tiles_per_panel() * ks);
        spp.counter = ws_get_t<uint32_t>(ctx, "counter", (size_t)(Kg / ks), true);
        VNE_TRY_CUDA(ctx, launch_start<T>(spp, ks, Kg / ks, st));
        double* C = ws_get_t<double>(ctx, "QtG", (size_t)Kp * Kg);
        double* gpart2 = ws_get_t<double>(ctx, "gram.part2", (size_t)nch * Kp * Kg);
        VNE_TRY_CUDA(ctx, launch_gram<T>(Q, Kp, Gr, Kg, ks, n, gpart2, nch, C, gerr, st));
        VNE_TRY_CUDA(ctx, launch_apply<T>(Q, Kp, C, Kg, Gr, Gp, ks, n, -1.0, gerr, st));
        ctx->launches += 4;
    }
    int hr[3] = {0, 0, 0};
    std::vector<int> hp(Kp);
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hr, drank, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaMemcpyAsync(hp.data(), cpiv, Kp * sizeof(int), cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    VNE_REQUIRE(ctx, hr[2] == 0, VNE_ETIMEOUT, "tensor-core sketch kernel: a bounded wait ran out");
    const int r = std::min(hr[0], hr[1]);
    out.rank = r;
    out.piv.assign(Nr, -1);
    for (int i = 0; i < std::min(r, Nr); i++) out.piv[i] = hp[i];
    // the quadratic forms: the whole [Q | G'] block, or a column range of it
    // gathered into its own block (a column's Lanczos recurrence and
    // quadrature do not depend on the other columns of its block)
    const int total = Nr + NH;
    const bool all = k < 0;
    if (all) {
        c0 = 0;
        k = total;
    }
    VNE_REQUIRE(ctx, c0 >= 0 && k >= 0 && c0 + k <= total, VNE_EINVAL, "column range outside [0, N_r + N_H)");
    out.psi.assign(k, 0.0);
    if (k == 0) return;
    StartSource sq{};
    sq.kind = SRC_PANEL;
    BlockOut qo;
    if (all) {
        sq.ncols = Kp + Kg;
        run_block<T>(ctx, P, sq, QG, Kp + Kg, ks, m, h.reorth, false, M->desing, "q", qo, h.sc.variant,
                     h.sc.interleave, h.sc.graph, true, ad);
        std::vector<double> hq = download(ctx, qo.psi, Kp + Kg);
        for (int c = 0; c < Nr; c++) out.psi[c] = c < r ? hq[c] : 0.0;
        for (int j = 0; j < NH; j++) out.psi[Nr + j] = hq[Kp + j];
    } else {
        std::vector<int32_t> src(k);
        for (int c = 0; c < k; c++) {
            const int i = c0 + c;
            src[c] = i < Nr ? i : Kp + (i - Nr);
        }
        const int Ks = ((k + ks - 1) / ks) * ks;
        int32_t* dsrc = upload(ctx, "hpp.sel", src);
        T* sel = ws_get_t<T>(ctx, "hpp.selblk", (size_t)Ks * n);
        VNE_TRY_CUDA(ctx, launch_select_columns<T>(QG, n, ks, dsrc, k, Ks, sel, st));
        ctx->launches += 1;
        sq.ncols = k;
        run_block<T>(ctx, P, sq, sel, k, ks, m, h.reorth, false, M->desing, "q", qo, h.sc.variant, h.sc.interleave,
                     h.sc.graph);
        std::vector<double> hq = download(ctx, qo.psi, k);
        for (int c = 0; c < k; c++) out.psi[c] = (c0 + c < Nr && c0 + c >= r) ? 0.0 : hq[c];
    }
}

template <typename T>
void hutchpp_impl(vne_matrix* M, const vne_options* o, int Nr, int NH, int m, uint64_t seed, double* estimate,
                  double* parts) {
    vne_ctx* ctx = M->ctx;
    VNE_REQUIRE(ctx, Nr >= 1 && Nr <= 128 && NH >= 0 && NH <= 4096, VNE_EINVAL, "need 1 <= N_r <= 128, 0 <= N_H");
    HppPlan h = hpp_plan<T>(M, o, m, seed);
    ctx->last_steps = 0;
    int Kp = 0;
    T* Y = sketch_block<T>(M, h, 0, Nr, "Y", &Kp);
    ProjectOut po;
    project_block<T>(M, h, Y, Kp, Nr, NH, 0, -1, po);
    double low = 0.0, resid = 0.0;
    for (int c = 0; c < po.rank; c++) low += po.psi[c];
    for (int j = 0; j < NH; j++) resid += po.psi[Nr + j];
    if (NH > 0) resid /= NH;
    *estimate = low + resid;
    if (parts) {
        parts[0] = low;
        parts[1] = resid;
        parts[2] = (double)po.rank;
    }
}

template <typename T>
void hutchpp_sketch_impl(vne_matrix* M, const vne_options* o, int c0, int k, int m, uint64_t seed, uint32_t flags,
                         void* Yout) {
    vne_ctx* ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    HppPlan h = hpp_plan<T>(M, o, m, seed);
    ctx->last_steps = 0;
    int Kp = 0;
    T* Y = sketch_block<T>(M, h, c0, k, "Y", &Kp);
    const size_t bytes = (size_t)h.n * k * sizeof(T);
    T* rows = (flags & VNE_VECTORS_DEVICE) ? (T*)Yout : ws_get_t<T>(ctx, "hpp.rows", (size_t)h.n * k);
    VNE_TRY_CUDA(ctx, launch_panel_to_rows<T>(Y, h.n, h.ks, 0, k, h.P->node_id, rows, st));
    ctx->launches += 1;
    if (!(flags & VNE_VECTORS_DEVICE))
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(Yout, rows, bytes, cudaMemcpyDeviceToHost, st));
    VNE_TRY_CUDA(ctx, cudaStreamSynchronize(st));
}

template <typename T>
void hutchpp_project_impl(vne_matrix* M, const vne_options* o, const void* Yin, uint32_t flags, int Nr, int NH, int m,
                          uint64_t seed, int c0, int k, double* psi, int32_t* pivots, int32_t* rank) {
    vne_ctx* ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    HppPlan h = hpp_plan<T>(M, o, m, seed);
    ctx->last_steps = 0;
    const int Kp = ((Nr + h.ks - 1) / h.ks) * h.ks;
    const T* rows = (const T*)Yin;
    if (!(flags & VNE_VECTORS_DEVICE)) {
        T* d = ws_get_t<T>(ctx, "hpp.rows", (size_t)h.n * Nr);
        VNE_TRY_CUDA(ctx, cudaMemcpyAsync(d, Yin, (size_t)h.n * Nr * sizeof(T), cudaMemcpyHostToDevice, st));
        rows = d;
    }
    T* Y = ws_get_t<T>(ctx, "Y", (size_t)Kp * h.n);
    VNE_TRY_CUDA(ctx, launch_rows_to_panel<T>(rows, h.n, h.ks, Nr, Kp, h.P->node_id, Y, st));
    ctx->launches += 1;
    ProjectOut po;
    project_block<T>(M, h, Y, Kp, Nr, NH, c0, k, po);
    std::copy(po.psi.begin(), po.psi.end(), psi);
    if (pivots) std::copy(po.piv.begin(), po.piv.end(), pivots);
    if (rank) *rank = po.rank;
}

}  // namespace

namespace vne_engine {

template <typename T>
void hutchpp_deflation(vne_matrix* M, const vne_options* o, int Nr, int m, int sketch_steps, uint64_t seed,
                       T* q_rows, std::vector<double>& psi_q, int& rank, const Adaptive* ad) {
    vne_ctx* ctx = M->ctx;
    HppPlan h = hpp_plan<T>(M, o, m, seed);
    HppPlan hs = h;  // the sketch f(A) Omega with its own step count
    hs.m = sketch_steps;
    int Kp = 0;
    T* Y = sketch_block<T>(M, hs, 0, Nr, "Y", &Kp);
    ProjectOut po;
    project_block<T>(M, h, Y, Kp, Nr, 0, 0, -1, po, ad);
    T* QG = ws_get_t<T>(ctx, "QG", (size_t)Kp * h.n);  // Q in its first Kp columns, zero beyond the rank
    VNE_TRY_CUDA(ctx, launch_panel_to_rows<T>(QG, h.n, h.ks, 0, Nr, nullptr, q_rows, ctx->stream));
    ctx->launches += 1;
    psi_q = po.psi;
    rank = po.rank;
}

template void hutchpp_deflation<float>(vne_matrix*, const vne_options*, int, int, int, uint64_t, float*,
                                       std::vector<double>&, int&, const Adaptive*);
template void hutchpp_deflation<double>(vne_matrix*, const vne_options*, int, int, int, uint64_t, double*,
                                        std::vector<double>&, int&, const Adaptive*);

}  // namespace vne_engine

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

extern "C" vne_status vne_hutchpp_sketch(vne_matrix* M, int32_t col_begin, int32_t ncols, int32_t krylov_steps,
                                         uint64_t seed, const vne_options* opt, uint32_t flags, void* Y) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, Y && col_begin >= 0 && ncols >= 1 && ncols <= 256, VNE_EINVAL,
                "need Y, col_begin >= 0 and 1 <= ncols <= 256");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    if (M->fp64) hutchpp_sketch_impl<double>(M, &o, col_begin, ncols, krylov_steps, seed, flags, Y);
    else hutchpp_sketch_impl<float>(M, &o, col_begin, ncols, krylov_steps, seed, flags, Y);
    VNE_API_END(ctx)
}

extern "C" vne_status vne_hutchpp_project(vne_matrix* M, const void* Y, uint32_t flags, int32_t sketch_cols,
                                          int32_t hutch_vectors, int32_t krylov_steps, uint64_t seed,
                                          int32_t col_begin, int32_t ncols, const vne_options* opt, double* psi,
                                          int32_t* pivots, int32_t* rank) {
    if (!M) return VNE_EINVAL;
    vne_ctx* ctx = M->ctx;
    VNE_API_BEGIN
    cudaSetDevice(ctx->device);
    vne_options o = opt ? *opt : defaults();
    VNE_REQUIRE(ctx, Y && (psi || ncols == 0), VNE_EINVAL, "need Y and psi");
    VNE_REQUIRE(ctx, sketch_cols >= 1 && sketch_cols <= 128 && hutch_vectors >= 0 && hutch_vectors <= 128,
                VNE_EINVAL, "need 1 <= N_r <= 128 and 0 <= N_H <= 128");
    VNE_REQUIRE(ctx, col_begin >= 0 && ncols >= 0 && col_begin + ncols <= sketch_cols + hutch_vectors, VNE_EINVAL,
                "column range outside [0, N_r + N_H)");
    VNE_REQUIRE(ctx, krylov_steps >= 1 && krylov_steps <= 128, VNE_EINVAL, "krylov_steps must be in [1, 128]");
    if (M->fp64)
        hutchpp_project_impl<double>(M, &o, Y, flags, sketch_cols, hutch_vectors, krylov_steps, seed, col_begin,
                                     ncols, psi, pivots, rank);
    else
        hutchpp_project_impl<float>(M, &o, Y, flags, sketch_cols, hutch_vectors, krylov_steps, seed, col_begin,
                                    ncols, psi, pivots, rank);
    VNE_API_END(ctx)
}
