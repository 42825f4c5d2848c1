// Batched Hutchinson estimates of uneven graphs packed block-diagonally.
#include "engine.h"

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
        P->owned.push_back(drp);
        int32_t* dci = dev_copy(ctx, ci);
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

