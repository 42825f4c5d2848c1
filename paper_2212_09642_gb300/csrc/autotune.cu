// Schedule autotuner of the SpMM step kernel.
#include "engine.h"

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
    const int ipws[3] = {1, 2, 4};
    const int nvar = M->fp64 ? 1 : kStepVariants;
    double best = 1e300;
    int bk = 0, bi = 0, bv = 0, bil = 0, bw = 1;
    const bool was_tuned = M->tuned;
    M->tuned = false;
    // the step loop of a k-column block under one schedule, best of two runs
    auto time_config = [&](int panel, int item, int v, int il, int ipw) {
        vne_options o;
        vne_options_default(&o);
        o.panel = panel;
        o.item_nnz = item;
        o.step_variant = v;
        o.interleave = il;
        o.items_per_warp = ipw;
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
            if (M->fp64) run_block<double>(ctx, *P, s, nullptr, k, panel, steps, false, false, M->desing, "tune", out, v, il, false);
            else run_block<float>(ctx, *P, s, nullptr, k, panel, steps, false, false, M->desing, "tune", out, v, il, false);
            ctx->time_steps = false;
            download(ctx, out.psi, 1);
            float ms = 0.f;
            VNE_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->loop_ev[0], ctx->loop_ev[1]));
            ms_min = std::min(ms_min, (double)ms);
        }
        if (ms_min < best) {
            best = ms_min;
            bk = panel;
            bi = item;
            bv = v;
            bil = il;
            bw = ipw;
        }
    };
    // phase 1: panel width, item size and kernel variant (one launch per
    // kernel and step, one item per warp); phase 2: for the winning panel
    // width and variant, item size x items per warp (together they set the
    // rows per CTA); phase 3: interleaved per-panel launches for the winner
    for (int pi = 0; pi < 3; pi++)
        for (int ii = 0; ii < 4; ii++)
            for (int v = 0; v < nvar; v++) time_config(M->fp64 ? panels_d[pi] : panels_f[pi], items[ii], v, 0, 1);
    const int p1k = bk, p1v = bv;
    for (int ii = 0; ii < 4; ii++)
        for (int wi = 1; wi < 3; wi++) time_config(p1k, items[ii], p1v, 0, ipws[wi]);
    time_config(bk, bi, bv, 1, bw);
    // release the tuning block's workspace
    for (auto it = ctx->ws.begin(); it != ctx->ws.end();) {
        if (it->first.compare(0, 5, "tune.") == 0) {
            dev_free(it->second.ptr);
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
    M->tuned_ipw = bw;
    ctx->tune_cache[vne_ctx::TuneKey{M->n, M->nnz, M->maxdeg, (int)M->fp64, (int)M->pattern}] = {bk, bi, bv, bil, bw};
    if (chosen) {
        vne_options_default(chosen);
        chosen->panel = bk;
        chosen->item_nnz = bi;
        chosen->step_variant = bv;
        chosen->interleave = bil;
        chosen->items_per_warp = bw;
    }
    if (ms_per_step) *ms_per_step = best / steps;
    VNE_API_END(ctx)
}

