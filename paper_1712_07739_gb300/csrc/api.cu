// C ABI of the library: context life cycle, tree build and evaluation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.cuh"

int fmm_kernel_attrs(gbfmm_ctx *ctx);  // fmm.cu
void mlp_free(gbfmm_ctx *ctx);         // mlp.cu
int mixed_alloc(gbfmm_ctx *ctx);       // fmm.cu
int near_alloc(gbfmm_ctx *ctx, int64_t n_targets);  // near.cu
int near_sym_alloc(gbfmm_ctx *ctx);                 // near.cu
int mixed_pass(gbfmm_ctx *ctx, bool free_targets, int64_t n_t);

int set_err(gbfmm_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

template <typename T>
static void release(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

static void free_tree(gbfmm_ctx *ctx) {
    release(ctx->d_y);
    release(ctx->d_q);
    release(ctx->d_sid);
    release(ctx->d_slen);
    release(ctx->d_pos);
    release(ctx->d_pleaf);
    release(ctx->d_sig);
    release(ctx->d_P);
    release(ctx->d_Pf);
    release(ctx->d_y0);
    release(ctx->d_q0);
    release(ctx->d_leaf_of);
    release(ctx->d_perm);
    release(ctx->d_len0);
    release(ctx->d_W);
    release(ctx->d_S);
    release(ctx->d_Wf);
    release(ctx->d_Sf);
    release(ctx->d_tmp_i);
    release(ctx->d_leaf_start);
    release(ctx->d_t_start);
    release(ctx->d_cnt);
    release(ctx->d_cursor);
    release(ctx->d_tmp_d);
    release(ctx->d_part);
    release(ctx->d_bad);
    release(ctx->d_yrel);
    {
        auto &RF = ctx->rf;
        release(RF.child_of);
        release(RF.pfine);
        release(RF.ref_start);
        release(RF.ref_leaf);
        release(RF.child_start);
        release(RF.W7);
        release(RF.S7);
        release(RF.Wc7);
        release(RF.Sc7);
        RF.cap_N = RF.cap_leaves = RF.cap_ref = RF.cap_cells = 0;
    }
    ctx->mx_cap_N = ctx->mx_cap_cells = 0;
    ctx->cap_N = ctx->cap_segs = ctx->cap_cells = ctx->cap_leaves = 0;
    ctx->built = false;
}

// (Re)allocate the tree buffers only when a size exceeds its capacity, so a
// repeated build of a same-size network allocates nothing.
static int ensure_tree_buffers(gbfmm_ctx *ctx) {
    const int64_t N = ctx->N, ns = ctx->n_segs, nc = ctx->n_cells, nl = ctx->n_leaves;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p;
    const bool fp64 = ctx->opt.precision == GBFMM_FP64;
    const bool w64 = ctx->opt.precision != GBFMM_MIXED;  // FP64 multipole and local values
    {
        GrowBuf b[12] = {{(void **)&ctx->d_y, N * 3 * sizeof(double)},  {(void **)&ctx->d_q, N * 9 * sizeof(double)},
                         {(void **)&ctx->d_sid, N * sizeof(int64_t)},   {(void **)&ctx->d_slen, N * sizeof(double)},
                         {(void **)&ctx->d_pos, N * sizeof(int)},       {(void **)&ctx->d_pleaf, N * sizeof(int)},
                         {(void **)&ctx->d_sig, N * 6 * sizeof(double)}, {(void **)&ctx->d_y0, N * 3 * sizeof(double)},
                         {(void **)&ctx->d_q0, N * 9 * sizeof(double)}, {(void **)&ctx->d_leaf_of, N * sizeof(int)},
                         {(void **)&ctx->d_perm, N * sizeof(int)},      {(void **)&ctx->d_P, N * 108 * sizeof(double)}};
        if (int rc = grow_dev(ctx, ctx->cap_N, N, b, fp64 ? 12 : 11, "points")) return rc;
    }
    if (int rc = grow_dev(ctx, ctx->cap_segs, ns, {{(void **)&ctx->d_len0, ns * sizeof(double)}}, "segments"))
        return rc;
    {
        // occupancy scratch: sources and targets per cell (with the adaptive tree, one more
        // level for the children of split leaves, which fmm_work_counts counts)
        const int64_t n_occ = 2 * (ctx->rf.on ? cell_base(ctx->L + 1) : nc);
        GrowBuf b[3] = {{(void **)&ctx->d_tmp_i, n_occ * sizeof(int)},
                        {(void **)&ctx->d_W, nc * P3 * 9 * sizeof(double)},
                        {(void **)&ctx->d_S, nc * P3 * 6 * sizeof(double)}};
        if (int rc = grow_dev(ctx, ctx->cap_cells, nc, b, w64 ? 3 : 1, "cells")) return rc;
    }
    if (int rc = grow_dev(ctx, ctx->cap_leaves, nl,
                          {{(void **)&ctx->d_leaf_start, (nl + 1) * sizeof(int)},
                           {(void **)&ctx->d_t_start, (nl + 1) * sizeof(int)},
                           {(void **)&ctx->d_cnt, nl * sizeof(int)},
                           {(void **)&ctx->d_cursor, nl * sizeof(int)}},
                          "leaves"))
        return rc;
    if (!ctx->d_part) CK(cudaMalloc(&ctx->d_part, 512 * 6 * sizeof(double)));
    if (!ctx->d_bad) CK(cudaMalloc(&ctx->d_bad, sizeof(int)));
    if (ctx->rf.on) {
        // adaptive tree: split leaves hold more than refine_points points each, so there are
        // at most N / (refine_points + 1) of them
        auto &RF = ctx->rf;
        const int64_t cap_ref = N / (ctx->opt.refine_points + 1) + 1;
        if (int rc = grow_dev(ctx, RF.cap_N, N,
                              {{(void **)&RF.child_of, size_t(N)}, {(void **)&RF.pfine, N * sizeof(int)}},
                              "adaptive-tree points"))
            return rc;
        if (int rc = grow_dev(ctx, RF.cap_leaves, nl, {{(void **)&RF.ref_start, (nl + 1) * sizeof(int)}},
                              "adaptive-tree leaves"))
            return rc;
        if (int rc = grow_dev(ctx, RF.cap_ref, cap_ref,
                              {{(void **)&RF.ref_leaf, cap_ref * sizeof(int)},
                               {(void **)&RF.child_start, 9 * cap_ref * sizeof(int)}},
                              "adaptive-tree split leaves"))
            return rc;
    }
    return GBFMM_OK;
}

extern "C" void fmm_default_options(gbfmm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->p = 4;
    o->n_gauss = 4;
    o->levels = 0;
    o->precision = GBFMM_FP64;
    o->h_mode = GBFMM_H_ISO;
    o->circle_q = 0;
    o->leaf_segments = 0;
    o->near_fp64 = 0.0;
    o->m2l_split = GBFMM_M2L_FP16_SPLIT_ALL;
    o->m2l_fft = 1;
    o->m2l_chunks = 7;
    o->m2l_basis = 1;
    o->m2l_split_kblocks = 1;
}

extern "C" int fmm_create(gbfmm_ctx **out, const gbfmm_options *opt, void *stream) {
    if (!out || !opt) return GBFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (opt->p < 2 || opt->p > GB_MAXP || opt->n_gauss < 1 || opt->n_gauss > GB_MAXG ||
        (opt->levels != 0 && (opt->levels < 3 || opt->levels > 9)) ||
        (opt->precision < GBFMM_FP64 || opt->precision > GBFMM_MIXED_F64T) || opt->h_mode < 0 || opt->h_mode > 2 ||
        opt->circle_q < 0 || opt->leaf_segments < 0 || !(opt->near_fp64 >= 0.0) || opt->m2l_split < 0 ||
        opt->m2l_split > 6 || opt->m2l_fft < 0 || opt->m2l_fft > 1 || opt->m2l_chunks < 0 ||
        opt->m2l_chunks > 189 || opt->m2l_basis < 0 || opt->m2l_basis > 1 ||
        opt->m2l_split_kblocks < 0 || opt->m2l_kernel < 0 || opt->m2l_kernel > 1 || opt->nodes < 0 ||
        opt->nodes > 1 || !(opt->m2l_svd_tol >= 0.0) || opt->m2l_svd_tol >= 1.0)
        return GBFMM_ERR_INVALID_ARG;
    // the compressed M2L runs in the mixed pass only, and Chebyshev nodes need it (their
    // operators have no Toeplitz structure for the lattice table and the FFT M2L)
    if ((opt->m2l_svd_tol > 0.0 || opt->nodes == GBFMM_NODES_CHEBYSHEV) &&
        (opt->precision != GBFMM_MIXED || opt->m2l_svd_tol <= 0.0))
        return GBFMM_ERR_INVALID_ARG;
    // the adaptive tree runs its extra level through the compressed M2L and its near
    // field through the symmetric kernel of the unit-circle h
    if (opt->refine_points < 0 ||
        (opt->refine_points > 0 && (opt->m2l_svd_tol <= 0.0 || opt->h_mode != GBFMM_H_CIRCLE ||
                                    opt->m2l_split < GBFMM_M2L_FP16)))
        return GBFMM_ERR_INVALID_ARG;
    // the symmetry-reduced operator table belongs to the FP64 M2L through transforms
    if (opt->m2l_symmetry < 0 || opt->m2l_symmetry > 1 ||
        (opt->m2l_symmetry == 1 && (opt->precision != GBFMM_FP64 || opt->m2l_fft != 1)))
        return GBFMM_ERR_INVALID_ARG;
    gbfmm_ctx *ctx = new gbfmm_ctx();
    ctx->opt = *opt;
    ctx->rf.on = opt->refine_points > 0 ? 1 : 0;
    if (ctx->opt.near_fp64 == 0.0) ctx->opt.near_fp64 = 2.0;
    if (ctx->opt.leaf_segments == 0) ctx->opt.leaf_segments = 32;
    ctx->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return GBFMM_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (cudaMalloc(&ctx->d_box, sizeof(TreeBox)) != cudaSuccess) {
        delete ctx;
        return GBFMM_ERR_CUDA;
    }
    if (fmm_kernel_attrs(ctx) != GBFMM_OK) {
        cudaFree(ctx->d_box);
        delete ctx;
        return GBFMM_ERR_CUDA;
    }
    *out = ctx;
    return GBFMM_OK;
}

extern "C" void fmm_destroy(gbfmm_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_tree(ctx);
    if (ctx->borrowed_material) {
        ctx->d_mat = nullptr;
        ctx->d_Asym = nullptr;
        ctx->d_Asym_f = nullptr;
        ctx->d_Klat = nullptr;
        ctx->tc.Thi = ctx->tc.Tlo = nullptr;
    }
    void *ps[] = {ctx->d_box, ctx->d_mat, ctx->d_Asym, ctx->d_Asym_f, ctx->d_Klat,
                  ctx->d_t_pos, ctx->d_t_x, ctx->d_t_sig, ctx->d_t_tmp};
    for (void *p : ps)
        if (p) cudaFree(p);
    m2l_tc_free(ctx);
    m2l_fft_free(ctx);
    mlp_free(ctx);
    {
        NearWork &W = ctx->nw;
        void *ps2[] = {W.items, W.sorted, W.keys, W.cnt, W.key_of, W.off, W.misc, W.pitems, W.psorted, W.pkeys,
                       W.pmisc, W.part};
        for (void *q : ps2)
            if (q) cudaFree(q);
    }
    if (ctx->timer.on)
        for (auto &e : ctx->timer.ev) cudaEventDestroy(e);
    delete ctx;
}

extern "C" const char *fmm_last_error(const gbfmm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static int choose_levels(const gbfmm_ctx *ctx, int64_t n_segs) {
    if (ctx->opt.levels) return ctx->opt.levels;
    double leaves = double(n_segs) / double(ctx->opt.leaf_segments);
    int lf = int(std::lround(std::log(std::max(leaves, 1.0)) / std::log(8.0)));
    lf = std::max(2, std::min(7, lf));
    return lf + 1;
}

extern "C" int fmm_build_tree(gbfmm_ctx *ctx, int64_t n_nodes, const double *node_xyz, int64_t n_segs,
                              const int64_t *seg_nodes, const double *burgers) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    if (n_segs < 1 || n_nodes < 2 || !node_xyz || !seg_nodes || !burgers)
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_build_tree: empty network or null pointer");
    const int64_t N = n_segs * ctx->opt.n_gauss;
    if (N >= (int64_t(1) << 31)) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_build_tree: too many points");
    if (ctx->rf.on && N >= (int64_t(1) << 28))
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_build_tree: adaptive tree limited to 2^28 points");
    ctx->built = false;
    ctx->n_nodes = n_nodes;
    ctx->n_segs = n_segs;
    ctx->N = N;
    ctx->node_xyz = node_xyz;
    ctx->seg_nodes = seg_nodes;
    ctx->burgers = burgers;
    ctx->L = choose_levels(ctx, n_segs);
    const int L = ctx->L;
    if (ctx->rf.on && L + 1 > GB_TC_MAXLEV)
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_build_tree: adaptive tree needs levels <= 7");
    ctx->n_leaves = int64_t(1) << (3 * (L - 1));
    ctx->n_cells = cell_base(L);
    int rc = ensure_tree_buffers(ctx);
    if (rc) return rc;
    rc = tree_build(ctx);
    if (rc) return rc;
    if (ctx->opt.precision != GBFMM_FP64) {
        rc = mixed_alloc(ctx);
        if (rc) return rc;
    } else {
        // work list and partial sums of the FP64 symmetric near field (unit-circle h)
        rc = near_alloc(ctx, ctx->N);
        if (!rc) rc = near_sym_alloc(ctx);
        if (rc) return rc;
    }
    ctx->built = true;
    return GBFMM_OK;
}

uint64_t layout_hash(const gbfmm_ctx *c) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a, 64 bit
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    auto v = [&mix](auto x) { mix(&x, sizeof(x)); };
    mix(&c->opt, sizeof(c->opt));
    v(c->L), v(c->N), v(c->n_segs), v(c->n_nodes), v(c->n_cells), v(c->n_leaves), v(c->t_cap);
    v(c->node_xyz), v(c->seg_nodes), v(c->burgers), v(c->stream);
    const void *ptrs[] = {c->d_mat, c->d_Asym, c->d_Asym_f, c->d_Klat, c->d_box, c->d_y, c->d_q, c->d_sid,
                          c->d_slen, c->d_pos, c->d_pleaf, c->d_leaf_start, c->d_tmp_i, c->d_tmp_d, c->d_P,
                          c->d_Pf, c->d_W, c->d_S, c->d_Wf, c->d_Sf, c->d_sig, c->d_yrel, c->d_t_pos, c->d_t_start,
                          c->d_t_x, c->d_t_sig, c->tc.Thi, c->tc.Tlo, c->tc.Whi, c->tc.Wlo, c->tc.d_status,
                          c->tc.d_flags, c->tc.d_pos, c->tc.d_list, c->tc.d_seg, c->tc.d_wmax, c->mlp.theta, c->mlp.theta_h,
                          c->mlp.scale, c->mlp.d_binmask, c->nw.items, c->nw.sorted, c->nw.keys, c->nw.cnt,
                          c->nw.key_of, c->nw.off, c->nw.misc, c->nw.pitems, c->nw.psorted,
                          c->nw.pkeys, c->nw.pmisc, c->nw.part, c->tc.Uh, c->tc.Ul, c->tc.Rh, c->tc.Rl,
                          c->tc.Xh, c->tc.Xl, c->tc.d_scal, c->tc.d_bits, c->tc.Wc, c->tc.Sc, c->tc.blas_ws,
                          c->rf.child_of, c->rf.ref_start, c->rf.ref_leaf, c->rf.child_start, c->rf.pfine,
                          c->rf.W7, c->rf.S7, c->rf.Wc7, c->rf.Sc7, c->tc.d_pcnt, c->tc.d_pairs, c->tc.Gh,
                          c->tc.Gl, c->tc.Yf};
    mix(ptrs, sizeof(ptrs));
    v(c->mat.mode), v(c->mat.Q), v(c->mat.cubic), v(c->tc.n_work), v(c->tc.split), v(c->tc.tf32);
    mix(c->tc.wofs, sizeof(c->tc.wofs));
    v(c->tc.n_slots), v(c->tc.n_seg), v(c->nw.cap), v(c->nw.cap_leaves), v(c->mlp.trained);
    v(c->tc.r1), v(c->tc.r2), v(c->rf.cap_ref), v(c->rf.n_ref_host), v(c->tc.blas);
    return h;
}

static int begin_eval(gbfmm_ctx *ctx) {
    if (!ctx->have_material) return set_err(ctx, GBFMM_ERR_NO_MATERIAL, "fmm_eval: call fmm_set_material first");
    if (!ctx->built) return set_err(ctx, GBFMM_ERR_NOT_BUILT, "fmm_eval: call fmm_build_tree first");
    ctx->timer.n = 0;
    return GBFMM_OK;
}

static int end_eval(gbfmm_ctx *ctx) {
    if (!ctx->timer.on) return GBFMM_OK;
    CK(cudaEventSynchronize(ctx->timer.ev[ctx->timer.n - 1]));
    for (int i = 0; i < 8; ++i) ctx->stage_ms[i] = 0.0;
    for (int i = 0; i + 1 < ctx->timer.n && i < 8; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->timer.ev[i], ctx->timer.ev[i + 1]);
        ctx->stage_ms[i] = ms;
    }
    return GBFMM_OK;
}

static int run_pass(gbfmm_ctx *ctx, bool free_targets, int64_t n_t) {
    if (ctx->opt.precision != GBFMM_FP64) return mixed_pass(ctx, free_targets, n_t);
    return fmm_pass(ctx, free_targets, n_t);
}

extern "C" int fmm_eval_stress(gbfmm_ctx *ctx, int64_t n_t, const double *x, double *sigma) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    int rc = begin_eval(ctx);
    if (rc) return rc;
    if (n_t < 0 || (n_t > 0 && (!x || !sigma)) || n_t >= (int64_t(1) << 31))
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_eval_stress: bad target array");
    if (n_t == 0) return GBFMM_OK;
    rc = targets_sort(ctx, n_t, x);
    if (rc) return rc;
    rc = run_pass(ctx, true, n_t);
    if (rc) return rc;
    rc = targets_scatter(ctx, n_t, sigma);
    if (rc) return rc;
    return end_eval(ctx);
}

extern "C" int fmm_eval_nodal_forces(gbfmm_ctx *ctx, double *f_nodes, double *f_seg, double *sigma_pts) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    int rc = begin_eval(ctx);
    if (rc) return rc;
    if (!f_nodes) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_eval_nodal_forces: null output");
    rc = run_pass(ctx, false, ctx->N);
    if (rc) return rc;
    rc = forces_from_stress(ctx, f_nodes, f_seg, sigma_pts);
    if (rc) return rc;
    return end_eval(ctx);
}

extern "C" int fmm_tree_info(const gbfmm_ctx *ctx, int *levels, int64_t *n_leaves, int64_t *n_points) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    if (levels) *levels = ctx->L;
    if (n_leaves) *n_leaves = ctx->n_leaves;
    if (n_points) *n_points = ctx->N;
    return GBFMM_OK;
}

extern "C" int fmm_m2l_ranks(const gbfmm_ctx *ctx, int *ranks, double *sigma) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    const TcPlan &T = ctx->tc;
    const bool on = T.svd && T.bases_ok;
    if (ranks) {
        ranks[0] = on ? T.r1 : 0;
        ranks[1] = on ? T.r2 : 0;
        ranks[2] = on ? T.r1_raw : 0;
        ranks[3] = on ? T.r2_raw : 0;
    }
    if (sigma)
        for (int i = 0; i < 4; ++i) sigma[i] = on ? T.svd_sigma[i] : 0.0;
    return GBFMM_OK;
}

extern "C" int fmm_set_timing(gbfmm_ctx *ctx, int enable) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    if (enable && !ctx->timer.on) {
        for (auto &e : ctx->timer.ev) CK(cudaEventCreate(&e));
        ctx->timer.on = true;
    } else if (!enable && ctx->timer.on) {
        for (auto &e : ctx->timer.ev) cudaEventDestroy(e);
        ctx->timer.on = false;
    }
    return GBFMM_OK;
}

extern "C" int fmm_stage_times(const gbfmm_ctx *ctx, double *t) {
    if (!ctx || !t) return GBFMM_ERR_INVALID_ARG;
    for (int i = 0; i < 8; ++i) t[i] = ctx->stage_ms[i];
    return GBFMM_OK;
}

extern "C" int fmm_launch_count(const gbfmm_ctx *ctx, int64_t *count) {
    if (!ctx || !count) return GBFMM_ERR_INVALID_ARG;
    *count = ctx->launches;
    return GBFMM_OK;
}

int work_counts(gbfmm_ctx *ctx, int64_t *out);  // fmm.cu

extern "C" int fmm_work_counts(gbfmm_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return GBFMM_ERR_INVALID_ARG;
    if (!ctx->built) return set_err(ctx, GBFMM_ERR_NOT_BUILT, "fmm_work_counts: call fmm_build_tree first");
    return work_counts(ctx, out);
}

extern "C" int fmm_device_status(gbfmm_ctx *ctx, int *status) {
    if (!ctx || !status) return GBFMM_ERR_INVALID_ARG;
    return m2l_tc_status(ctx, status);
}

extern "C" int fmm_inject_fault(gbfmm_ctx *ctx, int kind) {
    if (!ctx || kind != 1) return GBFMM_ERR_INVALID_ARG;
    ctx->tc.inject_drop = 1;
    return GBFMM_OK;
}
