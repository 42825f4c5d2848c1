// Probing (Section 3.1): device colourings (Algorithm 1), T_d by polynomial
// or rational quadratures, and the probing method with the choice of d
// (Section 5.1, Algorithm 2).
#include "engine.h"

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
    if (!ctx->pinned_ctr) VNE_TRY_CUDA(ctx, pinned_malloc((void**)&ctx->pinned_ctr, 8 * 8 * sizeof(int32_t)));
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

