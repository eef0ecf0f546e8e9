// Batched evaluation of many independent segment networks of uneven size.
//
// One batch holds one context per network.  They share everything that
// depends only on the medium and the order p (the kernel lattice and the M2L
// operator tables, Sec. 4.1: the operators do not depend on the
// configuration), so the tables exist once.  Each network gets its own tree
// depth from an autotuner that follows the cost model of App. B with
// constants measured on this GPU: a pass costs c_near x (near point pairs) +
// c_far x (cells of levels >= 2), and the depth that minimises it is taken
// among the candidates around N_s / leaf_segments.  The evaluation of all
// networks is recorded once into a CUDA graph (fanned out over a few
// streams) and replayed; a rebuild invalidates it.
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
    double c_near = 0.0, c_far = 0.0;  // seconds per near pair / per cell (autotuner)
    std::vector<int> tuned_L;          // depth chosen per slot, reused while N_s stays within 10 %
    std::vector<int64_t> tuned_ns;
    std::string err;
    bool material = false;
};

static int berr(gbfmm_batch *b, int code, const std::string &m) {
    if (b) b->err = m;
    return code;
}

static void drop_graph(gbfmm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

extern "C" int fmm_batch_create(gbfmm_batch **out, const gbfmm_options *opt, int n, void *stream) {
    if (!out || !opt || n < 1) return GBFMM_ERR_INVALID_ARG;
    *out = nullptr;
    gbfmm_batch *b = new gbfmm_batch();
    b->opt = *opt;
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
    for (size_t k = 1; k < b->ctx.size(); ++k) {
        int r2 = share_material(b->ctx[k], c0);
        if (r2) return berr(b, r2, fmm_last_error(b->ctx[k]));
    }
    b->material = true;
    drop_graph(b);
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
        return rc ? berr(b, rc, fmm_last_error(c)) : GBFMM_OK;
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
    }
    int best = L0;
    double best_t = 1e300;
    for (int L = std::max(3, L0 - 1); L <= std::min(8, L0 + 1); ++L) {
        int rc = build_at(L);
        if (rc) return berr(b, rc, fmm_last_error(c));
        int64_t w[4];
        rc = work_counts(c, w);
        if (rc) return berr(b, rc, fmm_last_error(c));
        const double pred = b->c_near * double(w[0]) + b->c_far * far_cells(L);
        if (pred < best_t) {
            best_t = pred;
            best = L;
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
        cudaEventRecord(b->ev[ns], b->cap);
        for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(b->side[i], b->ev[ns], 0);
        int rc = GBFMM_OK;
        for (int k = 0; k < n && !rc; ++k) rc = fmm_eval_nodal_forces(b->ctx[k], f_nodes[k], nullptr, nullptr);
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
    return GBFMM_OK;
}

extern "C" int fmm_batch_info(const gbfmm_batch *b, int k, int *levels, int64_t *launches, double *c_near,
                              double *c_far) {
    if (!b || k < 0 || k >= int(b->ctx.size())) return GBFMM_ERR_INVALID_ARG;
    if (levels) *levels = b->ctx[k]->L;
    if (launches) {
        int64_t s = 0;
        for (auto *c : b->ctx) s += c->launches;
        *launches = s;
    }
    if (c_near) *c_near = b->c_near;
    if (c_far) *c_far = b->c_far;
    return GBFMM_OK;
}
