// Batched evaluation of many independent segment networks of uneven size.
//
// One batch holds one context per network.  They share everything that
// depends only on the medium and the order p (the kernel lattice and the M2L
// operator tables, Sec. 4.1: the operators do not depend on the
// configuration), so the tables exist once.  Each network gets its own tree
// depth from an autotuner that settles the near/far balance of App. B by
// measurement: the candidates from N_s / leaf_segments down by one level and
// up while the time falls are each timed on the network, and the fastest is
// kept (a fixed cost per cell does not hold: the tensor-core M2L's tiles fill
// up with depth).  The evaluation of all networks, or every network's tree
// build and evaluation, is recorded once into a CUDA graph (fanned out over
// a few streams) and replayed; a rebuild invalidates it.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

int work_counts(gbfmm_ctx *ctx, int64_t *out);  // fmm.cu

struct gbfmm_batch {
    gbfmm_options opt{};
    cudaStream_t stream = nullptr;  // caller's (may be the legacy default stream)
    cudaStream_t cap = nullptr;     // stream the graph is recorded on and launched on
    cudaEvent_t in = nullptr, done = nullptr;  // caller -> cap and cap -> caller ordering
    std::vector<gbfmm_ctx *> ctx;
    std::vector<cudaStream_t> side;  // fan-out streams
    std::vector<cudaEvent_t> ev;     // fork + one join per side stream
    std::vector<double *> out;       // force outputs recorded in the graph
    std::vector<uint64_t> layout;    // layout_hash of each context when the graph was recorded
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // fmm_batch_step: every slot's tree build and evaluation recorded as one graph
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    std::vector<double *> step_out;
    std::vector<uint64_t> step_layout;
    int64_t eval_kernels = 0, step_kernels = 0;  // kernel nodes of the recorded graphs
    int64_t replayed = 0;  // kernels run by graph replays (the contexts count only direct launches)
    bool auto_kernel = false;  // the autotuner picks the M2L tile form (m2l_kernel = 2 at creation)
    double m2l_ms_form[2] = {-1.0, -1.0};  // M2L stage times of the two forms on the calibration network (ms)
    double c_near = 0.0, c_far = 0.0;  // seconds per near pair / per cell, first network at L0 (reported)
    std::vector<int> tuned_L;          // depth chosen per slot, reused while N_s stays within 10 %
    std::vector<int64_t> tuned_ns;
    std::string err;
    bool material = false;
};

static int berr(gbfmm_batch *b, int code, const std::string &m) {
    if (b) b->err = m;
    return code;
}

// kernel nodes of a recorded graph: the kernels one replay launches
static int64_t kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// a capture records launches without running them: put the contexts' counters back
static void restore_launches(gbfmm_batch *b, const std::vector<int64_t> &saved) {
    for (size_t k = 0; k < b->ctx.size(); ++k) b->ctx[k]->launches = saved[k];
}

static void drop_graph(gbfmm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->step_exec) cudaGraphExecDestroy(b->step_exec);
    if (b->step_graph) cudaGraphDestroy(b->step_graph);
    b->step_exec = nullptr;
    b->step_graph = nullptr;
}

extern "C" int fmm_batch_create(gbfmm_batch **out, const gbfmm_options *opt_in, int n, void *stream) {
    if (!out || !opt_in || n < 1) return GBFMM_ERR_INVALID_ARG;
    *out = nullptr;
    gbfmm_options o = *opt_in;
    const bool auto_kernel = o.m2l_kernel == 2;  // the autotuner picks the tile form
    if (auto_kernel) o.m2l_kernel = 0;
    const gbfmm_options *opt = &o;
    gbfmm_batch *b = new gbfmm_batch();
    b->opt = *opt;
    b->auto_kernel = auto_kernel;
    b->stream = (cudaStream_t)stream;
    const int ns = std::min(n, 8);
    b->side.resize(ns);
    b->ev.resize(ns + 1);
    for (int i = 0; i < ns; ++i)
        if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return GBFMM_ERR_CUDA;
        }
    for (auto &e : b->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            delete b;
            return GBFMM_ERR_CUDA;
        }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return GBFMM_ERR_CUDA;
    }
    for (int k = 0; k < n; ++k) {
        gbfmm_ctx *c = nullptr;
        int rc = fmm_create(&c, opt, b->side[k % ns]);
        if (rc) {
            for (auto *x : b->ctx) fmm_destroy(x);
            delete b;
            return rc;
        }
        b->ctx.push_back(c);
    }
    b->out.assign(n, nullptr);
    b->layout.assign(n, 0);
    b->step_out.assign(n, nullptr);
    b->step_layout.assign(n, 0);
    b->tuned_L.assign(n, 0);
    b->tuned_ns.assign(n, 0);
    *out = b;
    return GBFMM_OK;
}

extern "C" void fmm_batch_destroy(gbfmm_batch *b) {
    if (!b) return;
    drop_graph(b);
    // borrowed material tables belong to context 0: free the others first
    for (size_t k = b->ctx.size(); k-- > 0;) fmm_destroy(b->ctx[k]);
    for (auto s : b->side) cudaStreamDestroy(s);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->in) cudaEventDestroy(b->in);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

extern "C" const char *fmm_batch_last_error(const gbfmm_batch *b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int fmm_batch_set_material(gbfmm_batch *b, const double *C_voigt) {
    if (!b) return GBFMM_ERR_INVALID_ARG;
    gbfmm_ctx *c0 = b->ctx[0];
    int rc = fmm_set_material(c0, C_voigt);
    if (rc) return berr(b, rc, fmm_last_error(c0));
    // the operator tables exist once, built here by the first slot, before the others share them
    if (c0->opt.precision != GBFMM_FP64 && (rc = m2l_tc_setup(c0))) return berr(b, rc, fmm_last_error(c0));
    for (size_t k = 1; k < b->ctx.size(); ++k) {
        int r2 = share_material(b->ctx[k], c0);
        if (r2) return berr(b, r2, fmm_last_error(b->ctx[k]));
    }
    b->material = true;
    drop_graph(b);
    return GBFMM_OK;
}

// Switch every slot to M2L tile form `form`: the operator tables' row padding depends
// on the form, so the first slot rebuilds them and the others share them again; slots
// already built get their tile plan for the new form.
static int batch_set_form(gbfmm_batch *b, int form) {
    drop_graph(b);
    if (cudaDeviceSynchronize() != cudaSuccess) return berr(b, GBFMM_ERR_CUDA, "fmm_batch_build: synchronise");
    for (auto *c : b->ctx) c->opt.m2l_kernel = form;
    gbfmm_ctx *c0 = b->ctx[0];
    c0->tc.ready_ops = false;
    int rc = m2l_tc_setup(c0);
    if (rc) return berr(b, rc, fmm_last_error(c0));
    for (size_t k = 1; k < b->ctx.size(); ++k) {
        rc = share_material(b->ctx[k], c0);
        if (rc) return berr(b, rc, fmm_last_error(b->ctx[k]));
    }
    for (auto *c : b->ctx)
        if (c->built && (rc = m2l_tc_prepare(c))) return berr(b, rc, fmm_last_error(c));
    return GBFMM_OK;
}

// M2L stage time of one pass of slot context c at its current build (milliseconds)
static int time_m2l(gbfmm_batch *b, gbfmm_ctx *c, int64_t n_nodes, double *ms) {
    double *f = nullptr;
    if (cudaMalloc(&f, n_nodes * 3 * sizeof(double)) != cudaSuccess)
        return berr(b, GBFMM_ERR_CUDA, "fmm_batch_build: calibration buffer");
    fmm_set_timing(c, 1);
    int rc = fmm_eval_nodal_forces(c, f, nullptr, nullptr);  // warm-up
    if (!rc) rc = fmm_eval_nodal_forces(c, f, nullptr, nullptr);
    double t[8];
    fmm_stage_times(c, t);
    fmm_set_timing(c, 0);
    cudaFree(f);
    if (rc) return berr(b, rc, fmm_last_error(c));
    *ms = t[2];
    return GBFMM_OK;
}

// Tile form of the M2L GEMM (autotuner): ms0 is form 0's M2L time on slot context c at
// its current build; time form 1 on the same network and keep the faster.  The
// operator tables are rebuilt at each switch, once per batch.
template <class Build>
static int tune_form(gbfmm_batch *b, gbfmm_ctx *c, int64_t n_nodes, double ms0, Build build_at) {
    const int L = c->L;
    b->m2l_ms_form[0] = ms0;
    double ms1 = 0.0;
    int rc = batch_set_form(b, 1);
    if (rc) return rc;
    if ((rc = build_at(L))) return berr(b, rc, fmm_last_error(c));
    if ((rc = time_m2l(b, c, n_nodes, &ms1))) return rc;
    b->m2l_ms_form[1] = ms1;
    if (ms1 >= ms0 && (rc = batch_set_form(b, 0))) return rc;
    return GBFMM_OK;
}

// Elapsed time of one pass of slot context c at its current build (milliseconds)
static int time_pass(gbfmm_batch *b, gbfmm_ctx *c, int64_t n_nodes, double *ms) {
    double *f = nullptr;
    if (cudaMalloc(&f, n_nodes * 3 * sizeof(double)) != cudaSuccess)
        return berr(b, GBFMM_ERR_CUDA, "fmm_batch_build: calibration buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    int rc = fmm_eval_nodal_forces(c, f, nullptr, nullptr);
    cudaEventRecord(e1, c->stream);
    float t = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = GBFMM_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(f);
    if (rc) return berr(b, rc, rc == GBFMM_ERR_CUDA ? std::string("fmm_batch_build: timed pass") : fmm_last_error(c));
    *ms = double(t);
    return GBFMM_OK;
}

// cells of levels 2 .. L-1 (the M2L work of the dense tensor-core pass)
static double far_cells(int L) {
    double s = 0.0;
    for (int l = 2; l < L; ++l) s += std::ldexp(1.0, 3 * l);
    return s;
}

extern "C" int fmm_batch_build(gbfmm_batch *b, int k, int64_t n_nodes, const double *node_xyz, int64_t n_segs,
                               const int64_t *seg_nodes, const double *burgers) {
    if (!b || k < 0 || k >= int(b->ctx.size())) return GBFMM_ERR_INVALID_ARG;
    if (!b->material) return berr(b, GBFMM_ERR_NO_MATERIAL, "fmm_batch_build: set the material first");
    gbfmm_ctx *c = b->ctx[k];
    drop_graph(b);
    auto build_at = [&](int L) {
        c->opt.levels = L;
        return fmm_build_tree(c, n_nodes, node_xyz, n_segs, seg_nodes, burgers);
    };
    if (b->opt.levels != 0) {
        int rc = build_at(b->opt.levels);
        if (rc) return berr(b, rc, fmm_last_error(c));
        if (b->auto_kernel && b->m2l_ms_form[0] < 0.0) {
            double ms0 = 0.0;
            if ((rc = time_m2l(b, c, n_nodes, &ms0))) return rc;
            return tune_form(b, c, n_nodes, ms0, build_at);
        }
        return GBFMM_OK;
    }
    // a slot keeps its tuned depth while its size stays within 10 %
    if (b->tuned_L[k] && std::llabs(n_segs - b->tuned_ns[k]) * 10 <= b->tuned_ns[k]) {
        int rc = build_at(b->tuned_L[k]);
        return rc ? berr(b, rc, fmm_last_error(c)) : GBFMM_OK;
    }
    // autotuner: candidates around the leaf-size guess
    const int ls = b->opt.leaf_segments > 0 ? b->opt.leaf_segments : 32;
    const double leaves = std::max(1.0, double(n_segs) / ls);
    const int L0 = std::max(3, std::min(8, int(std::lround(std::log(leaves) / std::log(8.0))) + 1));
    if (b->c_near <= 0.0) {
        // calibrate the two cost constants once, on this network at L0, with one timed pass
        int rc = build_at(L0);
        if (rc) return berr(b, rc, fmm_last_error(c));
        double *f = nullptr;
        if (cudaMalloc(&f, n_nodes * 3 * sizeof(double)) != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, "fmm_batch_build: calibration buffer");
        fmm_set_timing(c, 1);
        rc = fmm_eval_nodal_forces(c, f, nullptr, nullptr);  // warm-up
        if (!rc) rc = fmm_eval_nodal_forces(c, f, nullptr, nullptr);
        double t[8];
        fmm_stage_times(c, t);
        fmm_set_timing(c, 0);
        cudaFree(f);
        if (rc) return berr(b, rc, fmm_last_error(c));
        int64_t w[4];
        rc = work_counts(c, w);
        if (rc) return berr(b, rc, fmm_last_error(c));
        b->c_near = std::max(1e-15, 1e-3 * t[4] / double(std::max<int64_t>(w[0], 1)));
        b->c_far = std::max(1e-12, 1e-3 * t[2] / std::max(1.0, far_cells(c->L)));
        if (b->auto_kernel && b->m2l_ms_form[0] < 0.0 && (rc = tune_form(b, c, n_nodes, t[2], build_at)))
            return rc;
    }
    // every candidate depth L0 - 1 .. L0 + 1 timed on this network (one pass each): the
    // near field and the M2L trade against each other, and the M2L's cost per cell falls
    // steeply with depth while its tiles fill up, which no per-cell constant captures.
    // The deepest candidate is tried only while the time is still falling; the buffers
    // keep the size of the deepest candidate built, which bounds a batch's memory.
    int best = L0;
    double best_t = 1e300;
    for (int L = std::max(3, L0 - 1); L <= std::min(8, L0 + 1); ++L) {
        int rc = build_at(L);
        if (rc) return berr(b, rc, fmm_last_error(c));
        double ms = 0.0;
        if ((rc = time_pass(b, c, n_nodes, &ms))) return rc;
        if (ms < best_t) {
            best_t = ms;
            best = L;
        } else if (L > L0) {
            break;
        }
    }
    if (c->L != best) {
        int rc = build_at(best);
        if (rc) return berr(b, rc, fmm_last_error(c));
    }
    b->tuned_L[k] = best;
    b->tuned_ns[k] = n_segs;
    return GBFMM_OK;
}

extern "C" int fmm_batch_eval_nodal_forces(gbfmm_batch *b, double *const *f_nodes) {
    if (!b || !f_nodes) return GBFMM_ERR_INVALID_ARG;
    const int n = int(b->ctx.size()), ns = int(b->side.size());
    for (int k = 0; k < n; ++k)
        if (!b->ctx[k]->built) return berr(b, GBFMM_ERR_NOT_BUILT, "fmm_batch_eval: config " + std::to_string(k) + " not built");
    // the recorded graph is reused while every output pointer and every
    // context's layout (sizes, depth, buffers) is what it was when recorded
    bool same = b->exec != nullptr;
    for (int k = 0; k < n && same; ++k) same = b->out[k] == f_nodes[k] && b->layout[k] == layout_hash(b->ctx[k]);
    if (!same) {
        drop_graph(b);
        // record on the batch's own stream: fork onto the side streams, every
        // network's pass on its side stream, join back
        const cudaError_t pre = cudaGetLastError();
        if (pre != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_eval: pending error ") + cudaGetErrorString(pre));
        const cudaError_t eb = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (eb != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_eval: cudaStreamBeginCapture: ") + cudaGetErrorString(eb));
        std::vector<int64_t> saved(n);
        for (int k = 0; k < n; ++k) saved[k] = b->ctx[k]->launches;
        cudaEventRecord(b->ev[ns], b->cap);
        for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(b->side[i], b->ev[ns], 0);
        int rc = GBFMM_OK;
        for (int k = 0; k < n && !rc; ++k) rc = fmm_eval_nodal_forces(b->ctx[k], f_nodes[k], nullptr, nullptr);
        restore_launches(b, saved);
        for (int i = 0; i < ns; ++i) {
            cudaEventRecord(b->ev[i], b->side[i]);
            cudaStreamWaitEvent(b->cap, b->ev[i], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return berr(b, rc, "fmm_batch_eval: " + std::string(fmm_last_error(b->ctx[0])));
        }
        if (e != cudaSuccess) return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_eval: capture: ") + cudaGetErrorString(e));
        b->graph = g;
        b->eval_kernels = kernel_nodes(g);
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, "fmm_batch_eval: cudaGraphInstantiate");
        for (int k = 0; k < n; ++k) {
            b->out[k] = f_nodes[k];
            b->layout[k] = layout_hash(b->ctx[k]);
        }
    }
    // order the replay after the caller's prior work and the caller's later work after it
    if (cudaEventRecord(b->in, b->stream) != cudaSuccess || cudaStreamWaitEvent(b->cap, b->in, 0) != cudaSuccess ||
        cudaGraphLaunch(b->exec, b->cap) != cudaSuccess || cudaEventRecord(b->done, b->cap) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->done, 0) != cudaSuccess)
        return berr(b, GBFMM_ERR_CUDA, "fmm_batch_eval: graph launch");
    b->replayed += b->eval_kernels;
    return GBFMM_OK;
}

// Every slot's tree build (from the arrays of its last fmm_batch_build, without the
// host-side checks) and nodal-force evaluation, recorded once as one CUDA graph over the
// side streams and replayed while no slot's layout changes.
extern "C" int fmm_batch_step(gbfmm_batch *b, double *const *f_nodes) {
    if (!b || !f_nodes) return GBFMM_ERR_INVALID_ARG;
    const int n = int(b->ctx.size()), ns = int(b->side.size());
    for (int k = 0; k < n; ++k)
        if (!b->ctx[k]->built) return berr(b, GBFMM_ERR_NOT_BUILT, "fmm_batch_step: config " + std::to_string(k) + " not built");
    bool same = b->step_exec != nullptr;
    for (int k = 0; k < n && same; ++k)
        same = b->step_out[k] == f_nodes[k] && b->step_layout[k] == layout_hash(b->ctx[k]);
    if (!same) {
        if (b->step_exec) cudaGraphExecDestroy(b->step_exec);
        if (b->step_graph) cudaGraphDestroy(b->step_graph);
        b->step_exec = nullptr;
        b->step_graph = nullptr;
        for (auto *c : b->ctx)
            if (c->timer.on) fmm_set_timing(c, 0);  // no event synchronisation inside a capture
        const cudaError_t pre = cudaGetLastError();
        if (pre != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_step: pending error ") + cudaGetErrorString(pre));
        const cudaError_t eb = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (eb != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_step: cudaStreamBeginCapture: ") + cudaGetErrorString(eb));
        std::vector<int64_t> saved(n);
        for (int k = 0; k < n; ++k) saved[k] = b->ctx[k]->launches;
        cudaEventRecord(b->ev[ns], b->cap);
        for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(b->side[i], b->ev[ns], 0);
        int rc = GBFMM_OK;
        for (int k = 0; k < n && !rc; ++k) {
            rc = tree_build(b->ctx[k], false);
            if (!rc) rc = fmm_eval_nodal_forces(b->ctx[k], f_nodes[k], nullptr, nullptr);
        }
        restore_launches(b, saved);
        for (int i = 0; i < ns; ++i) {
            cudaEventRecord(b->ev[i], b->side[i]);
            cudaStreamWaitEvent(b->cap, b->ev[i], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return berr(b, rc, "fmm_batch_step: " + std::string(fmm_last_error(b->ctx[0])));
        }
        if (e != cudaSuccess) return berr(b, GBFMM_ERR_CUDA, std::string("fmm_batch_step: capture: ") + cudaGetErrorString(e));
        b->step_graph = g;
        b->step_kernels = kernel_nodes(g);
        if (cudaGraphInstantiate(&b->step_exec, g, 0) != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, "fmm_batch_step: cudaGraphInstantiate");
        for (int k = 0; k < n; ++k) {
            b->step_out[k] = f_nodes[k];
            b->step_layout[k] = layout_hash(b->ctx[k]);
        }
    }
    if (cudaEventRecord(b->in, b->stream) != cudaSuccess || cudaStreamWaitEvent(b->cap, b->in, 0) != cudaSuccess ||
        cudaGraphLaunch(b->step_exec, b->cap) != cudaSuccess || cudaEventRecord(b->done, b->cap) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->done, 0) != cudaSuccess)
        return berr(b, GBFMM_ERR_CUDA, "fmm_batch_step: graph launch");
    b->replayed += b->step_kernels;
    return GBFMM_OK;
}

// Checks the graph-recorded builds skip: zero-length or non-finite segments (device flag
// of each build), a non-finite root box, and the bounded-wait status of the M2L.
extern "C" int fmm_batch_status(gbfmm_batch *b, int *slot, int *status) {
    if (!b || !slot || !status) return GBFMM_ERR_INVALID_ARG;
    *slot = -1;
    *status = GBFMM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return berr(b, GBFMM_ERR_CUDA, "fmm_batch_status: synchronise");
    for (int k = 0; k < int(b->ctx.size()); ++k) {
        gbfmm_ctx *c = b->ctx[k];
        if (!c->built) continue;
        int bad = 0, m2l = 0;
        TreeBox hb{};
        if (cudaMemcpy(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&hb, c->d_box, sizeof(TreeBox), cudaMemcpyDeviceToHost) != cudaSuccess)
            return berr(b, GBFMM_ERR_CUDA, "fmm_batch_status: read back");
        if (m2l_tc_status(c, &m2l)) return berr(b, GBFMM_ERR_CUDA, fmm_last_error(c));
        const int st = bad ? GBFMM_ERR_DEGENERATE : (!std::isfinite(hb.H) ? GBFMM_ERR_INVALID_ARG : m2l);
        if (st != GBFMM_OK && *slot < 0) {
            *slot = k;
            *status = st;
        }
    }
    return GBFMM_OK;
}

extern "C" int fmm_batch_tuning(const gbfmm_batch *b, int *m2l_kernel, double *m2l_ms) {
    if (!b) return GBFMM_ERR_INVALID_ARG;
    if (m2l_kernel) *m2l_kernel = b->ctx[0]->opt.m2l_kernel;
    if (m2l_ms) {
        m2l_ms[0] = b->m2l_ms_form[0];
        m2l_ms[1] = b->m2l_ms_form[1];
    }
    return GBFMM_OK;
}

extern "C" int fmm_batch_info(const gbfmm_batch *b, int k, int *levels, int64_t *launches, double *c_near,
                              double *c_far) {
    if (!b || k < 0 || k >= int(b->ctx.size())) return GBFMM_ERR_INVALID_ARG;
    if (levels) *levels = b->ctx[k]->L;
    if (launches) {
        int64_t s = 0;
        for (auto *c : b->ctx) s += c->launches;
        *launches = s + b->replayed;
    }
    if (c_near) *c_near = b->c_near;
    if (c_far) *c_far = b->c_far;
    return GBFMM_OK;
}
