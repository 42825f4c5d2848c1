// Host driver of the rational Krylov quadratures (Sections 4, 4.2, 5.3):
// multi-shift CG over a block of start vectors, the polynomial part (powers
// of A or, with the switching rule of Section 5.3, the seed CG residuals),
// the basis Gram matrices and the two Cholesky-QR passes of rational.cu.
#include "engine.h"

namespace {

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
    // the FP64 path orthonormalises W itself and applies A to the orthonormal
    // basis afterwards, so it needs no A W
    const bool need_aw = sizeof(T) != 8;
    if (mixed) {
        for (int j = 1; j < kpoly; j++) W[j] = rh + (size_t)(j - 1) * blk;
        for (int j = 0; j < kpoly && need_aw; j++) {
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
    for (int i = 0; i < nshift && need_aw; i++)  // A x_s into the (now free) direction buffers
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
    double* gram2 = ws_get_t<double>(ctx, "rat.gram2", gsz);
    double* dpsi = ws_get_t<double>(ctx, "rat.psi", Kp);
    int* drank = ws_get_t<int>(ctx, "rat.rank", Kp);
    if (sizeof(T) == 8) {
        // FP64: classical Gram-Schmidt applied twice to the vectors, in basis
        // order, each column on its own.  A direction is dropped only when its
        // remainder is at the rounding level of its norm (drop), which a
        // factorisation of the Gram matrix could not resolve; then A V by the
        // SpMM and the projection from the Gram matrices of (V, A V), whose
        // first matrix is the identity up to rounding.
        T* V = ws_get_t<T>(ctx, "rat.V", blk * nb);
        T* AV = ws_get_t<T>(ctx, "rat.AV", blk * nb);
        double* ones = upload(ctx, "rat.cgs.ones", std::vector<double>((size_t)nb * Kp, 1.0));
        double* coef = ws_get_t<double>(ctx, "rat.cgs.coef", (size_t)nb * Kp);
        double* cpart = ws_get_t<double>(ctx, "rat.cgs.part", (size_t)panels * nb * tiles * ks);
        double* orig2 = ws_get_t<double>(ctx, "rat.cgs.orig2", Kp);
        double* rem2 = ws_get_t<double>(ctx, "rat.cgs.rem2", Kp);
        ReorthParams<T> rp{};
        rp.basis = V;
        rp.slot_stride = blk;
        rp.K = Kp;
        rp.n_total = n;
        rp.panels = panels;
        rp.tiles_per_panel = tiles;
        rp.tiles = P.d_tiles;
        rp.part = cpart;
        rp.coef = coef;
        ReorthCoefParams cp{};
        cp.part = cpart;
        cp.sig = ones;
        cp.coef = coef;
        cp.K = Kp;
        cp.panels = panels;
        cp.tiles_per_panel = tiles;
        auto col_norm2 = [&](T* v, double* out) {  // out[col] = ||v[:, col]||^2
            ReorthParams<T> q = rp;
            q.basis = v;
            q.w = v;
            q.j = 1;
            ReorthCoefParams qc = cp;
            qc.j = 1;
            qc.coef = out;
            VNE_TRY_CUDA(ctx, launch_col_dots<T>(q, qc, ks, st));
        };
        for (int a = 0; a < nb; a++) {
            T* va = V + (size_t)a * blk;
            VNE_TRY_CUDA(ctx, cudaMemcpyAsync(va, W[a], blk * sizeof(T), cudaMemcpyDeviceToDevice, st));
            col_norm2(va, orig2);
            if (a > 0) {
                rp.w = va;
                rp.j = a;
                cp.j = a;
                for (int pass = 0; pass < 2; pass++) VNE_TRY_CUDA(ctx, launch_reorth<T>(rp, cp, ks, st));
            }
            col_norm2(va, rem2);
            VNE_TRY_CUDA(ctx, launch_cgs_scale<T>(va, orig2, rem2, drop, n, Kp, ks, tiles, P.d_tiles, st));
            ctx->launches += 5 + (a > 0 ? 6 : 0);
        }
        std::vector<const T*> Vv(nb), AVv(nb);
        for (int a = 0; a < nb; a++) {
            apply_operator<T>(ctx, P, ks, Kp, V + (size_t)a * blk, AV + (size_t)a * blk, 0.0, dq, variant, "rat.op0");
            Vv[a] = V + (size_t)a * blk;
            AVv[a] = AV + (size_t)a * blk;
        }
        gram_pairs(Vv, AVv, gram2);
        // ||c||^2 of every column from the start pass
        VNE_TRY_CUDA(ctx, launch_rational_pass2(gram2, gram2 + (size_t)nb * nb * Kp, norm2, nb, Kp, drop2, dpsi, drank,
                                                st));
        ctx->launches += 1;
    } else {
        double* gram = ws_get_t<double>(ctx, "rat.gram", gsz);
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
        // ||c||^2 is the (0,0) entry of the first Gram matrix
        VNE_TRY_CUDA(ctx, launch_rational_pass2(gram2, gram2 + (size_t)nb * nb * Kp, gram, nb, Kp, drop2, dpsi, drank,
                                                st));
        ctx->launches += 4;
    }
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

}  // namespace

namespace vne_engine {

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
    // a direction whose remainder after orthogonalising against the earlier
    // ones is below the threshold is treated as dependent.  Exact rational
    // Arnoldi drops nothing.  FP64 orthonormalises the vectors themselves and
    // drops only at the rounding level (remainder 1e-12 of the norm).  FP32
    // orthonormalises through the Gram matrices (Cholesky-QR2), which cannot
    // resolve remainders below the square root of the rounding unit, and drops
    // below a remainder of 1e-3 of the norm, because a kept direction's
    // A-image carries the vectors' rounding amplified by 1 / remainder.
    // FP64: relative remainder (Gram-Schmidt on the vectors); FP32: squared
    // relative remainder (pivot of the Cholesky factor of the Gram matrix)
    const double drop = M->fp64 ? 1e-12 : 1e-6;
    const double drop2 = M->fp64 ? 1e-12 : drop;
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

template void rational_quadforms<float>(vne_matrix*, const vne_options*, StartSource, int, const double*, int,
                                        std::vector<double>&, std::vector<int>&, std::vector<double>&);
template void rational_quadforms<double>(vne_matrix*, const vne_options*, StartSource, int, const double*, int,
                                         std::vector<double>&, std::vector<int>&, std::vector<double>&);

}  // namespace vne_engine

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

