// Offline greedy (Alg. 1 / Alg. 4), basis file and basis read-back.
// Included at the end of rb_api.cu (same translation unit).

namespace {

__global__ void k_scale_into(long long N, double s, const double* v, double* dst) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        dst[i] = s * v[i];
}

__global__ void k_gather_rowmajor(long long N, int n, const double* W64c, double* Wrow, long long r0, long long rows) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n;
        const int k = (int)(idx % n);
        Wrow[idx] = W64c[(size_t)k * N + r0 + i];
    }
}

struct BuildBufs {
    double* snap = nullptr;     // [N]
    double* vecs = nullptr;     // [max(Q, R)][N]
    double* coef = nullptr;     // [max(Q,R)][MAX_N]
    double* mue = nullptr;      // [Q][n_mu]
    double* mutrain = nullptr;  // [ntrain][n_mu]
    double* score = nullptr;
    int* bad = nullptr;
    int* lparam = nullptr;
    double* Rsnap = nullptr;    // [MAX_N][MAX_N]
};

// order == nullptr: Alg. 1 (the next parameter is the argmax of the scores).  Otherwise the
// parameters are taken in the given order (the sample selected on a coarse grid) and no scores
// are computed.
rb_status build_greedy(rb_ctx* ctx, int n_max, int n_train, const double* mu_train, const rb_build_opts& b,
                       const rb_opts& so, const std::vector<int>* order = nullptr) {
    const long long N = ctx->N;
    const int Q = ctx->P, R = ctx->R, n_mu = ctx->n_mu;
    BuildBufs bb;
    const int nv = std::max(Q, R);
    TRY(dalloc(ctx, &bb.snap, N));
    TRY(dalloc(ctx, &bb.vecs, (size_t)nv * N));
    TRY(dalloc(ctx, &bb.coef, (size_t)nv * MAX_N));
    TRY(dalloc(ctx, &bb.mue, (size_t)Q * n_mu));
    TRY(dalloc(ctx, &bb.mutrain, (size_t)n_train * n_mu));
    TRY(dalloc(ctx, &bb.score, n_train));
    TRY(dalloc(ctx, &bb.bad, n_train));
    TRY(dalloc(ctx, &bb.lparam, R));
    TRY(dalloc(ctx, &bb.Rsnap, MAX_N * MAX_N));
    {
        std::vector<double> e((size_t)Q * n_mu, 0.0);
        for (int q = 0; q < Q; ++q) e[(size_t)q * n_mu + q] = 1.0;
        CK(cudaMemcpy(bb.mue, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(bb.mutrain, mu_train, (size_t)n_train * n_mu * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(bb.lparam, ctx->load_param, R * sizeof(int), cudaMemcpyHostToDevice));
    }
    for (size_t i = 0; i < (size_t)n_train * n_mu; ++i)
        if (!std::isfinite(mu_train[i])) { ctx->err = "training parameters hold a non-finite value"; return RB_EINVAL; }

    cudaStream_t s = ctx->own_stream;
    rb_opts o = so;
    o.tol = b.truth_tol;
    o.max_iter = b.truth_max_iter;
    // snapshots in the precision the caller asks for: FP64, or FP32 inner RBCG with FP64
    // residual refinement (the snapshot still reaches the FP64 relative residual truth_tol)
    const Mode snap_mode{false, so.precision == RB_PREC_MIXED};
    o.x0_mode = RB_X0_ZERO;
    o.stream = nullptr;
    o.max_outer = std::max(o.max_outer, 40);

    ctx->n = 0;
    ctx->h_ANq.clear();
    ctx->h_fNr.clear();
    ctx->h_Rsnap.clear();
    ctx->selected.clear();
    std::vector<char> excluded(n_train, 0);
    std::vector<double> last_scores;
    size_t next_in_order = 0;
    if (order && order->empty()) { ctx->err = "empty parameter sample"; return RB_EINVAL; }
    int cand = order ? (*order)[next_in_order++] : 0;
    std::vector<double> c1(MAX_N), c2(MAX_N);
    while (ctx->n < n_max) {
        const int n = ctx->n;
        // step 3: snapshot, RBCG with W_{n} (no basis when n = 0)
        rb_stats st;
        rb_status ws = run_wave(ctx, 1, mu_train + (size_t)cand * n_mu, bb.snap, false, o, snap_mode, &st, nullptr);
        // a snapshot that stalled at the FP64 residual floor within 10x the target is kept
        if (ws == RB_ENOCONV && st.rel_res < 10.0 * b.truth_tol) ws = RB_OK;
        if (ws != RB_OK) {
            if (ws == RB_ECUDA || ws == RB_ETIMEOUT || ws == RB_EINVAL) return ws;
            char buf[160];
            std::snprintf(buf, sizeof(buf), " (rel. residual %.3e after %d iterations, %d residual checks)",
                          st.rel_res, st.iters, st.outer);
            ctx->err = "snapshot solve for training parameter " + std::to_string(cand) + " failed: " +
                       rb_status_string(ws) + buf;
            return ws;
        }
        excluded[cand] = 1;
        // step 4: Gram-Schmidt against W_n, twice
        const double xnorm = launch_norm(ctx->geo, bb.snap, ctx->d_scratch, s);
        if (n > 0) {
            launch_project_cols(ctx->geo, n, ctx->d_W64c, 1, bb.snap, bb.coef, ctx->d_scratch, s);
            CK(cudaMemcpyAsync(c1.data(), bb.coef, n * sizeof(double), cudaMemcpyDeviceToHost, s));
            launch_sub_cols(ctx->geo, n, ctx->d_W64c, bb.coef, bb.snap, s);
            launch_project_cols(ctx->geo, n, ctx->d_W64c, 1, bb.snap, bb.coef, ctx->d_scratch, s);
            CK(cudaMemcpyAsync(c2.data(), bb.coef, n * sizeof(double), cudaMemcpyDeviceToHost, s));
            launch_sub_cols(ctx->geo, n, ctx->d_W64c, bb.coef, bb.snap, s);
            CK(cudaStreamSynchronize(s));
        }
        const double nrm = launch_norm(ctx->geo, bb.snap, ctx->d_scratch, s);
        if (!(nrm >= b.drop_tol * xnorm) || !(nrm > 0.0)) {
            // numerically inside span W: take the next candidate of the sample, or the next best
            // candidate of the last scores
            if (order) {
                if (next_in_order >= order->size()) break;
                cand = (*order)[next_in_order++];
                continue;
            }
            if (last_scores.empty()) { ctx->err = "first snapshot is zero"; return RB_EBREAKDOWN; }
            int best = -1;
            for (int t = 0; t < n_train; ++t)
                if (!excluded[t] && (best < 0 || last_scores[t] > last_scores[best])) best = t;
            if (best < 0) break;
            cand = best;
            continue;
        }
        k_scale_into<<<1024, 256, 0, s>>>(N, 1.0 / nrm, bb.snap, ctx->d_W64c + (size_t)n * N);
        CK(cudaGetLastError());
        // eq. 12c: new row and column of A_{N,q}, new entry of f_{N,r}
        for (int q = 0; q < Q; ++q)
            launch_apply(ctx->geo, 1, n_mu, bb.mue + (size_t)q * n_mu, ctx->d_W64c + (size_t)n * N,
                         bb.vecs + (size_t)q * N, s);
        launch_project_cols(ctx->geo, n + 1, ctx->d_W64c, Q, bb.vecs, bb.coef, ctx->d_scratch, s);
        std::vector<double> cols((size_t)Q * (n + 1)), fcol((size_t)R * (n + 1));
        CK(cudaMemcpyAsync(cols.data(), bb.coef, cols.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        launch_project_cols(ctx->geo, n + 1, ctx->d_W64c, R, ctx->d_fr, bb.coef, ctx->d_scratch, s);
        CK(cudaMemcpyAsync(fcol.data(), bb.coef, fcol.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int n1 = n + 1;
        std::vector<double> A((size_t)Q * n1 * n1, 0.0), F((size_t)R * n1, 0.0), Rs((size_t)n1 * n1, 0.0);
        for (int q = 0; q < Q; ++q) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) A[((size_t)q * n1 + i) * n1 + j] = ctx->h_ANq[((size_t)q * n + i) * n + j];
            for (int i = 0; i < n1; ++i) {
                const double v = cols[(size_t)q * n1 + i];
                A[((size_t)q * n1 + i) * n1 + n] = v;
                A[((size_t)q * n1 + n) * n1 + i] = v;
            }
        }
        for (int r = 0; r < R; ++r) {
            for (int i = 0; i < n; ++i) F[(size_t)r * n1 + i] = ctx->h_fNr[(size_t)r * n + i];
            F[(size_t)r * n1 + n] = fcol[(size_t)r * n1 + n];
        }
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) Rs[(size_t)i * n1 + j] = ctx->h_Rsnap[(size_t)i * n + j];
            Rs[(size_t)i * n1 + n] = c1[i] + c2[i];
        }
        Rs[(size_t)n * n1 + n] = nrm;
        ctx->h_ANq.swap(A);
        ctx->h_fNr.swap(F);
        ctx->h_Rsnap.swap(Rs);
        ctx->selected.push_back(cand);
        ctx->n = n1;
        TRY(ctx_refresh_basis(ctx));
        if (ctx->n == n_max) break;
        if (order) {
            if (next_in_order >= order->size()) break;
            cand = (*order)[next_in_order++];
            continue;
        }
        // steps 5-6: score every training parameter
        CK(cudaMemcpy(bb.Rsnap, ctx->h_Rsnap.data(), (size_t)n1 * n1 * sizeof(double), cudaMemcpyHostToDevice));
        launch_scores(ctx->geo, Q, R, bb.lparam, n_mu, n1, ctx->nbp, ctx->d_ANq, ctx->d_fNr, bb.Rsnap, n_train,
                      bb.mutrain, b.score, bb.score, bb.bad, s);
        CK(cudaGetLastError());
        last_scores.assign(n_train, 0.0);
        std::vector<int> bad(n_train);
        CK(cudaMemcpyAsync(last_scores.data(), bb.score, n_train * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(bad.data(), bb.bad, n_train * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        int best = -1;
        for (int t = 0; t < n_train; ++t) {
            if (excluded[t] || bad[t]) continue;
            if (best < 0 || last_scores[t] > last_scores[best]) best = t;
        }
        if (best < 0) break;
        cand = best;
    }
    return RB_OK;
}

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

rb_status read_basis_host(const rb_ctx* ctx, std::vector<double>& Wrow) {
    rb_ctx* c = const_cast<rb_ctx*>(ctx);
    const long long N = ctx->N;
    const int n = ctx->n;
    Wrow.assign((size_t)N * n, 0.0);
    if (n == 0) return RB_OK;
    const long long rows_per = std::max<long long>(1, (long long)(ctx->scratch_bytes / sizeof(double)) / n);
    for (long long r0 = 0; r0 < N; r0 += rows_per) {
        const long long rows = std::min(rows_per, N - r0);
        k_gather_rowmajor<<<1024, 256>>>(N, n, ctx->d_W64c, ctx->d_scratch, r0, rows);
        cudaError_t e = cudaMemcpy(Wrow.data() + (size_t)r0 * n, ctx->d_scratch, (size_t)rows * n * sizeof(double),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return RB_ECUDA; }
    }
    return RB_OK;
}

const char RBB_MAGIC[4] = {'R', 'B', 'B', '1'};

}  // namespace

extern "C" {

rb_status rb_offline_build(rb_ctx** out, const rb_problem* prob, int n_max, int n_train, const double* mu_train,
                           const rb_build_opts* bopts, const rb_opts* solve_opts, int max_batch) {
    if (!out) { g_create_error = "out is NULL"; return RB_EINVAL; }
    *out = nullptr;
    std::string why;
    rb_status v = validate_problem(prob, why);
    if (v != RB_OK) { g_create_error = why; return v; }
    if (n_max < 1 || n_max > MAX_N || n_train < 1 || !mu_train || max_batch < 1) {
        g_create_error = "need 1 <= n_max <= 128, n_train >= 1, mu_train and max_batch >= 1";
        return RB_EINVAL;
    }
    rb_build_opts b;
    rb_default_build_opts(&b);
    if (bopts) b = *bopts;
    rb_opts so;
    rb_default_opts(&so);
    if (solve_opts) so = *solve_opts;
    rb_ctx* ctx = new rb_ctx();
    rb_status s = ctx_init(ctx, prob, n_max, max_batch);
    if (s == RB_OK) s = validate_opts(ctx, so);
    if (s == RB_OK) s = build_greedy(ctx, n_max, n_train, mu_train, b, so);
    if (s != RB_OK) {
        g_create_error = ctx->err;
        ctx_destroy(ctx);
        return s;
    }
    *out = ctx;
    return RB_OK;
}

rb_status rb_offline_build_mf(rb_ctx** out, const rb_problem* fine, const rb_problem* coarse, int n_max, int n_train,
                              const double* mu_train, const rb_build_opts* bopts, const rb_opts* solve_opts,
                              int max_batch) {
    if (!out) { g_create_error = "out is NULL"; return RB_EINVAL; }
    *out = nullptr;
    std::string why;
    if (validate_problem(fine, why) != RB_OK || validate_problem(coarse, why) != RB_OK) {
        g_create_error = why;
        return RB_EINVAL;
    }
    bool same = fine->dim == coarse->dim && fine->n_loads == coarse->n_loads && fine->n_mu == coarse->n_mu;
    for (int d = 0; d < 3 && same; ++d) same = fine->nb[d] == coarse->nb[d];
    for (int r = 0; r < fine->n_loads && same; ++r) {
        const rb_load &a = fine->loads[r], &c = coarse->loads[r];
        same = a.kind == c.kind && a.param == c.param && a.sigma == c.sigma && a.center[0] == c.center[0] &&
               a.center[1] == c.center[1] && a.center[2] == c.center[2];
    }
    if (!same) {
        g_create_error = "the coarse problem must have the fine one's blocks, loads and parameters";
        return RB_EINVAL;
    }
    // the parameter sample S_N: the greedy on the coarse grid
    rb_ctx* cctx = nullptr;
    rb_status s = rb_offline_build(&cctx, coarse, n_max, n_train, mu_train, bopts, solve_opts, 1);
    if (s != RB_OK) return s;
    const std::vector<int> order = cctx->selected;
    ctx_destroy(cctx);
    // the fine snapshots of S_N, in the selection order
    rb_build_opts b;
    rb_default_build_opts(&b);
    if (bopts) b = *bopts;
    rb_opts so;
    rb_default_opts(&so);
    if (solve_opts) so = *solve_opts;
    rb_ctx* ctx = new rb_ctx();
    s = ctx_init(ctx, fine, (int)order.size(), max_batch);
    if (s == RB_OK) s = validate_opts(ctx, so);
    if (s == RB_OK) s = build_greedy(ctx, (int)order.size(), n_train, mu_train, b, so, &order);
    if (s != RB_OK) {
        g_create_error = ctx->err;
        ctx_destroy(ctx);
        return s;
    }
    *out = ctx;
    return RB_OK;
}

rb_status rb_get_basis(const rb_ctx* ctx, double* W, double* ANq, double* fNr, double* Rsnap, int* selected) {
    if (!ctx) return RB_EINVAL;
    const int n = ctx->n;
    if (W) {
        std::vector<double> Wrow;
        rb_status s = read_basis_host(ctx, Wrow);
        if (s != RB_OK) return s;
        std::memcpy(W, Wrow.data(), Wrow.size() * sizeof(double));
    }
    if (ANq && !ctx->h_ANq.empty()) std::memcpy(ANq, ctx->h_ANq.data(), ctx->h_ANq.size() * sizeof(double));
    if (fNr && !ctx->h_fNr.empty()) std::memcpy(fNr, ctx->h_fNr.data(), ctx->h_fNr.size() * sizeof(double));
    if (Rsnap) {
        for (size_t i = 0; i < (size_t)n * n; ++i) Rsnap[i] = i < ctx->h_Rsnap.size() ? ctx->h_Rsnap[i] : 0.0;
    }
    if (selected) {
        for (int i = 0; i < n; ++i) selected[i] = i < (int)ctx->selected.size() ? ctx->selected[i] : -1;
    }
    return RB_OK;
}

rb_status rb_save(const rb_ctx* ctx, const char* path) {
    if (!ctx || !path) return RB_EINVAL;
    rb_ctx* c = const_cast<rb_ctx*>(ctx);
    std::vector<double> Wrow;
    rb_status s = read_basis_host(ctx, Wrow);
    if (s != RB_OK) return s;
    std::vector<unsigned char> buf;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        buf.insert(buf.end(), b, b + n);
    };
    const int n = ctx->n;
    int32_t hdr[12] = {1, ctx->dim, ctx->m[0], ctx->m[1], ctx->m[2], ctx->nbk[0], ctx->nbk[1], ctx->nbk[2],
                       ctx->R, ctx->n_mu, n, ctx->n_fields};
    put(RBB_MAGIC, 4);
    put(hdr, sizeof(hdr));
    for (const rb_load& l : ctx->loads) {
        int32_t kp[2] = {l.kind, l.param};
        put(kp, sizeof(kp));
        put(l.center, sizeof(l.center));
        put(&l.sigma, sizeof(double));
    }
    // array and boundary loads: field index, value count, values; then the coefficient fields
    for (int r = 0; r < ctx->R; ++r) {
        if (ctx->loads[r].kind < RB_LOAD_ARRAY) continue;
        const int64_t cnt = (int64_t)ctx->load_vals[r].size();
        const int32_t fld = ctx->loads[r].field;
        put(&fld, sizeof(fld));
        put(&cnt, sizeof(cnt));
        put(ctx->load_vals[r].data(), (size_t)cnt * sizeof(double));
    }
    put(ctx->h_fields.data(), ctx->h_fields.size() * sizeof(double));
    put(Wrow.data(), Wrow.size() * sizeof(double));
    put(ctx->h_ANq.data(), ctx->h_ANq.size() * sizeof(double));
    put(ctx->h_fNr.data(), ctx->h_fNr.size() * sizeof(double));
    std::vector<double> Rs((size_t)n * n, 0.0);
    for (size_t i = 0; i < Rs.size() && i < ctx->h_Rsnap.size(); ++i) Rs[i] = ctx->h_Rsnap[i];
    put(Rs.data(), Rs.size() * sizeof(double));
    std::vector<int32_t> sel(n, -1);
    for (int i = 0; i < n && i < (int)ctx->selected.size(); ++i) sel[i] = ctx->selected[i];
    put(sel.data(), sel.size() * sizeof(int32_t));
    const uint64_t h = fnv1a(buf.data(), buf.size(), 1469598103934665603ULL);
    put(&h, sizeof(h));
    FILE* f = std::fopen(path, "wb");
    if (!f) { c->err = std::string("cannot open ") + path + " for writing"; return RB_EIO; }
    const size_t wr = std::fwrite(buf.data(), 1, buf.size(), f);
    const int cl = std::fclose(f);
    if (wr != buf.size() || cl != 0) { c->err = std::string("short write to ") + path; return RB_EIO; }
    return RB_OK;
}

rb_status rb_offline_load(rb_ctx** out, const char* path, int max_batch) {
    if (!out || !path) { g_create_error = "NULL argument"; return RB_EINVAL; }
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) { g_create_error = std::string("cannot open ") + path; return RB_EIO; }
    std::vector<unsigned char> buf;
    unsigned char tmp[1 << 16];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    const bool rd_err = std::ferror(f) != 0;
    std::fclose(f);
    if (rd_err) { g_create_error = std::string("read error on ") + path; return RB_EIO; }
    size_t off = 0;
    auto take = [&](void* dst, size_t n) -> bool {
        if (off + n > buf.size()) return false;
        std::memcpy(dst, buf.data() + off, n);
        off += n;
        return true;
    };
    char magic[4];
    int32_t hdr[12];
    if (!take(magic, 4) || std::memcmp(magic, RBB_MAGIC, 4) != 0 || !take(hdr, sizeof(hdr)) || hdr[0] != 1) {
        g_create_error = "not a version-1 .rbb basis file";
        return RB_EFORMAT;
    }
    rb_problem prob{};
    prob.dim = hdr[1];
    for (int d = 0; d < 3; ++d) { prob.m[d] = hdr[2 + d]; prob.nb[d] = hdr[5 + d]; }
    prob.n_loads = hdr[8];
    prob.n_mu = hdr[9];
    const int n = hdr[10];
    if (prob.n_loads < 1 || prob.n_loads > MAX_LOADS || n < 0 || n > MAX_N) {
        g_create_error = "basis file header out of range";
        return RB_EFORMAT;
    }
    std::vector<rb_load> loads(prob.n_loads);
    for (auto& l : loads) {
        int32_t kp[2];
        if (!take(kp, sizeof(kp)) || !take(l.center, sizeof(l.center)) || !take(&l.sigma, sizeof(double))) {
            g_create_error = "truncated basis file";
            return RB_EFORMAT;
        }
        l.kind = kp[0];
        l.param = kp[1];
        l.field = 0;
        l.values = nullptr;
    }
    const long long N = (long long)prob.m[0] * prob.m[1] * prob.m[2];
    if (prob.m[0] < 1 || prob.m[1] < 1 || prob.m[2] < 1 || N >= (1LL << 31) || hdr[11] < 0 || hdr[11] > MAX_P) {
        g_create_error = "basis file header out of range";
        return RB_EFORMAT;
    }
    std::vector<std::vector<double>> lvals(prob.n_loads);
    for (int r = 0; r < prob.n_loads; ++r) {
        if (loads[r].kind < RB_LOAD_ARRAY || loads[r].kind > RB_LOAD_BOUNDARY) continue;
        int32_t fld;
        int64_t cnt;
        const long long ext = (long long)(prob.m[0] + 2) * (prob.m[1] + 2) * (prob.dim == 3 ? prob.m[2] + 2 : 1);
        if (!take(&fld, sizeof(fld)) || !take(&cnt, sizeof(cnt)) ||
            cnt != (loads[r].kind == RB_LOAD_ARRAY ? N : ext)) {
            g_create_error = "truncated or inconsistent load values in basis file";
            return RB_EFORMAT;
        }
        lvals[r].resize((size_t)cnt);
        if (!take(lvals[r].data(), (size_t)cnt * sizeof(double))) {
            g_create_error = "truncated basis file";
            return RB_EFORMAT;
        }
        loads[r].field = fld;
        loads[r].values = lvals[r].data();
    }
    prob.n_fields = hdr[11];
    std::vector<double> fields((size_t)prob.n_fields * N);
    if (prob.n_fields > 0) {
        if (!take(fields.data(), fields.size() * sizeof(double))) {
            g_create_error = "truncated basis file";
            return RB_EFORMAT;
        }
        prob.fields = fields.data();
    }
    prob.loads = loads.data();
    std::string why;
    if (validate_problem(&prob, why) != RB_OK) { g_create_error = "basis file problem: " + why; return RB_EFORMAT; }
    const int Q = prob.n_fields > 0 ? prob.n_fields : prob.nb[0] * prob.nb[1] * prob.nb[2];
    const size_t need = ((size_t)N * n + (size_t)Q * n * n + (size_t)prob.n_loads * n + (size_t)n * n) * 8 +
                        (size_t)n * 4 + 8;
    if (buf.size() - off != need) { g_create_error = "basis file size does not match its header"; return RB_EFORMAT; }
    uint64_t h_stored;
    std::memcpy(&h_stored, buf.data() + buf.size() - 8, 8);
    if (fnv1a(buf.data(), buf.size() - 8, 1469598103934665603ULL) != h_stored) {
        g_create_error = "basis file checksum mismatch";
        return RB_EFORMAT;
    }
    std::vector<double> W((size_t)N * n), A((size_t)Q * n * n), F((size_t)prob.n_loads * n), Rs((size_t)n * n);
    std::vector<int32_t> sel(n);
    take(W.data(), W.size() * 8);
    take(A.data(), A.size() * 8);
    take(F.data(), F.size() * 8);
    take(Rs.data(), Rs.size() * 8);
    take(sel.data(), sel.size() * 4);
    rb_status s = rb_offline_load_arrays(out, &prob, n, W.data(), A.data(), F.data(), max_batch);
    if (s != RB_OK) return s;
    (*out)->h_Rsnap = Rs;
    (*out)->selected.assign(sel.begin(), sel.end());
    return RB_OK;
}

}  // extern "C"
