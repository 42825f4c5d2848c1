// libvne C ABI: options, contexts, density-matrix assembly, quadratic forms,
// Hutchinson estimates, the kernel-level entry points used by the tests and
// the measurement calls.
//
// Probe generator (identical to the oracle's, written independently):
//   mix64 = SplitMix64 output mixer (Steele, Lea, Flood 2014),
//   s = mix64(seed + 0x9E3779B97F4A7C15),
//   h(j, i) = mix64((((j << 32) | i) ^ s) + 0x9E3779B97F4A7C15),
//   entry = +1 if the top bit of h is 0 else -1,
// j the global probe column, i the node id in the caller's numbering.
#include "engine.h"

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
    for (auto& kv : ctx->ws) dev_free(kv.second.ptr);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->loop_ev)
        if (e) cudaEventDestroy(e);
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaStream_t sx : ctx->color_streams) cudaStreamDestroy(sx);
    for (cudaEvent_t e : ctx->color_events) cudaEventDestroy(e);
    pinned_free(ctx->pinned_ctr);
    for (auto& kv : ctx->pinned) pinned_free(kv.second.first);
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
    VNE_TRY_CUDA(ctx, dev_malloc((void**)&M->d_rowptr, (n + 1) * sizeof(int32_t)));
    VNE_TRY_CUDA(ctx, dev_malloc((void**)&M->d_col, std::max<int64_t>(nnz, 1) * sizeof(int32_t)));
    if (vals) VNE_TRY_CUDA(ctx, dev_malloc(&M->d_vals, std::max<int64_t>(nnz, 1) * es));
    if (by_degree) {
        // degree order built above; inverse permutation and the moved
        // nonzeros on the device
        int32_t* d_inv = ws_get_t<int32_t>(ctx, "asm.inv", n);
        VNE_TRY_CUDA(ctx, dev_malloc((void**)&M->d_node_id, n * sizeof(int32_t)));
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
        VNE_TRY_CUDA(ctx, dev_malloc((void**)&M->d_node_id, n * sizeof(int32_t)));
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
            M->tuned_ipw = it->second[4];
        }
    }
    *out = M.release();
    VNE_API_END(ctx)
}

extern "C" vne_status vne_matrix_destroy(vne_matrix* M) {
    if (!M) return VNE_EINVAL;
    cudaSetDevice(M->ctx->device);
    if (M->ctx->stream) cudaStreamSynchronize(M->ctx->stream);
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
    const int reorth = want_reorth(M, &o);
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
    VNE_REQUIRE(ctx, herr == 0, VNE_ETIMEOUT, "tensor-core Gram: a bounded wait ran out");
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
    VNE_REQUIRE(ctx, herr == 0, VNE_ETIMEOUT, "tensor-core block product: a bounded wait ran out");
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

extern "C" vne_status vne_debug_fail_allocation(int64_t k) {
    if (k < 0) return VNE_EINVAL;
    fail_allocation_after(k);
    return VNE_OK;
}

extern "C" vne_status vne_debug_live_allocations(int64_t* device_buffers, int64_t* pinned_buffers) {
    if (device_buffers) *device_buffers = live_device_buffers();
    if (pinned_buffers) *pinned_buffers = live_pinned_buffers();
    return VNE_OK;
}

extern "C" vne_status vne_debug_tensor_wait_limit(int64_t polls) {
    set_tensor_wait_polls(polls);
    return VNE_OK;
}
