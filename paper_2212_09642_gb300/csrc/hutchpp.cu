// Hutch++ (Section 3.2, eq. Hutch++_formula): the sketch f(A) Omega by the
// Lanczos matvec approximation (eq. rational-krylov-approximation-matvec),
// Q by pivoted Cholesky-QR on the tcgen05 Grams, the projected Hutchinson
// vectors and one Lanczos block for all quadratic forms.
#include "engine.h"

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
