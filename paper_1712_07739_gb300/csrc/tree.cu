// Gauss points, root cube and leaf binning (the tree of Algorithm 2).
//
// Points are the n_g Gauss points of each segment (Sec. 2, Eq.
// "stress_discrete"): y = (x1 + x2)/2 + xi_k S/2 with S = x2 - x1 and
// strength q_wr = 1/2 b_w omega_k S_r.  The root is a cube of edge
// H = s (1 + 2^-10) centred on the bounding box of the points (s its largest
// extent); a point goes to the leaf floor((y - origin) * (2^(L-1) / H)),
// clamped.  Points are counting-sorted by leaf, and within a leaf by their
// original index, so that the order (and every sum over it) is
// deterministic.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace {

struct GaussParams {
    double xi[GB_MAXG];
    double w[GB_MAXG];
    int n;
};

__global__ void k_gauss_points(int64_t n_segs, const double *__restrict__ nodes, const int64_t *__restrict__ segs,
                               const double *__restrict__ b, GaussParams gp, double *__restrict__ y0,
                               double *__restrict__ q0, double *__restrict__ len0, int *__restrict__ bad) {
    int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (s >= n_segs) return;
    int64_t n0 = segs[2 * s], n1 = segs[2 * s + 1];
    double x1[3], S[3], bb[3];
    for (int i = 0; i < 3; ++i) {
        x1[i] = nodes[3 * n0 + i];
        S[i] = nodes[3 * n1 + i] - x1[i];
        bb[i] = b[3 * s + i];
    }
    double len = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    if (!(len > 0.0) || !isfinite(len)) atomicExch(bad, 1);
    len0[s] = len;
    for (int g = 0; g < gp.n; ++g) {
        int64_t k = s * gp.n + g;
        double f = 0.5 * (1.0 + gp.xi[g]);
        for (int i = 0; i < 3; ++i) y0[3 * k + i] = x1[i] + f * S[i];
        for (int w = 0; w < 3; ++w)
            for (int r = 0; r < 3; ++r) q0[9 * k + 3 * w + r] = 0.5 * bb[w] * gp.w[g] * S[r];
    }
}

// per-block min/max, then one block folds the partials and writes the box
__global__ void k_bbox_partial(int64_t n, const double *__restrict__ y, double *__restrict__ part) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double v = y[3 * i + d];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    __shared__ double sm[6][256];
    for (int d = 0; d < 3; ++d) {
        sm[d][threadIdx.x] = lo[d];
        sm[3 + d][threadIdx.x] = hi[d];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                sm[d][threadIdx.x] = fmin(sm[d][threadIdx.x], sm[d][threadIdx.x + s]);
                sm[3 + d][threadIdx.x] = fmax(sm[3 + d][threadIdx.x], sm[3 + d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 6; ++d) part[blockIdx.x * 6 + d] = sm[d][0];
}

__global__ void k_bbox_final(int nparts, const double *__restrict__ part, TreeBox *box) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nparts; ++b)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[b * 6 + d]);
            hi[d] = fmax(hi[d], part[b * 6 + 3 + d]);
        }
    double s = fmax(hi[0] - lo[0], fmax(hi[1] - lo[1], hi[2] - lo[2]));
    if (s == 0.0) s = 1.0;
    double H = s * (1.0 + 0.0009765625);
    for (int d = 0; d < 3; ++d) {
        box->lo[d] = lo[d];
        box->hi[d] = hi[d];
        box->origin[d] = 0.5 * (lo[d] + hi[d]) - 0.5 * H;
    }
    box->H = H;
}

__device__ __forceinline__ int leaf_coord(double v, double o, double f, int n) {
    double c = floor((v - o) * f);
    int i = c < 0.0 ? 0 : (c > double(n - 1) ? n - 1 : int(c));
    return i;
}

__global__ void k_leaf_count(int64_t n, const double *__restrict__ y, const TreeBox *__restrict__ box, int L,
                             int *__restrict__ leaf_of, int *__restrict__ cnt, unsigned char *__restrict__ child_of) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    int nl = 1 << (L - 1);
    double f = double(nl) / box->H;
    int cx = leaf_coord(y[3 * i], box->origin[0], f, nl);
    int cy = leaf_coord(y[3 * i + 1], box->origin[1], f, nl);
    int cz = leaf_coord(y[3 * i + 2], box->origin[2], f, nl);
    int leaf = (cz * nl + cy) * nl + cx;
    leaf_of[i] = leaf;
    if (child_of) {
        // the point's cell one level below the leaves, as a child (bit d: upper half along axis d)
        const int fx = leaf_coord(y[3 * i], box->origin[0], 2.0 * f, 2 * nl);
        const int fy = leaf_coord(y[3 * i + 1], box->origin[1], 2.0 * f, 2 * nl);
        const int fz = leaf_coord(y[3 * i + 2], box->origin[2], 2.0 * f, 2 * nl);
        child_of[i] = (unsigned char)((fx & 1) | ((fy & 1) << 1) | ((fz & 1) << 2));
    }
    atomicAdd(&cnt[leaf], 1);
}

// exclusive scan of cnt[0..n) into start[0..n], one block of 1024 threads
__global__ void k_scan(int64_t n, const int *__restrict__ cnt, int *__restrict__ start) {
    __shared__ int part[1024];
    int64_t per = (n + blockDim.x - 1) / blockDim.x;
    int64_t b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < int(blockDim.x); ++t) {
            int v = part[t];
            part[t] = run;
            run += v;
        }
        start[n] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        start[i] = run;
        run += cnt[i];
    }
}

__global__ void k_scatter(int64_t n, const int *__restrict__ leaf_of, const int *__restrict__ start,
                          int *__restrict__ cursor, int *__restrict__ perm) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    int leaf = leaf_of[i];
    int slot = start[leaf] + atomicAdd(&cursor[leaf], 1);
    perm[slot] = int(i);
}

// restore original order inside each leaf: one block per leaf, bitonic
// sort in shared memory (leaves above 8192 points: one-thread insertion sort).
// With child_of (adaptive tree) the points of a leaf holding more than refine points
// are ordered by child first (key child * 2^28 + original index; N < 2^28).
__global__ void k_leaf_sort(int64_t n_leaves, const int *__restrict__ start, int *__restrict__ perm,
                            const unsigned char *__restrict__ child_of, int refine) {
    constexpr int CAP = 8192;
    constexpr int MASK = (1 << 28) - 1;
    __shared__ int v[CAP];
    const int64_t l = blockIdx.x;
    const int b = start[l], e = start[l + 1], n = e - b;
    if (n <= 1) return;
    const bool by_child = child_of && n > refine;
    auto key = [&](int x) { return by_child ? (int(child_of[x]) << 28) | x : x; };
    if (n > CAP) {
        if (threadIdx.x == 0) {
            for (int i = b; i < e; ++i) perm[i] = key(perm[i]);
            for (int i = b + 1; i < e; ++i) {
                const int x = perm[i];
                int j = i - 1;
                while (j >= b && perm[j] > x) {
                    perm[j + 1] = perm[j];
                    --j;
                }
                perm[j + 1] = x;
            }
            if (by_child)
                for (int i = b; i < e; ++i) perm[i] &= MASK;
        }
        return;
    }
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = i < n ? key(perm[b + i]) : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int a = v[i], c = v[ixj];
                    if ((a > c) == up) {
                        v[i] = c;
                        v[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[b + i] = by_child ? (v[i] & MASK) : v[i];
}

// adaptive tree: split flag of every leaf (more than refine points)
__global__ void k_ref_flags(int64_t nl, const int *__restrict__ start, int refine, int *__restrict__ flags) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l < nl) flags[l] = (start[l + 1] - start[l]) > refine ? 1 : 0;
}

// adaptive tree: for every split leaf (index r from the scan of the flags) its leaf
// and the sorted-point ranges of its 8 children (the points are ordered by child)
__global__ void k_ref_children(int64_t nl, const int *__restrict__ start, const int *__restrict__ ref_start,
                               const int *__restrict__ perm, const unsigned char *__restrict__ child_of,
                               int *__restrict__ ref_leaf, int *__restrict__ child_start) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l >= nl || ref_start[l + 1] == ref_start[l]) return;
    const int r = ref_start[l];
    ref_leaf[r] = int(l);
    const int b = start[l], e = start[l + 1];
    int i = b;
    for (int c = 0; c < 8; ++c) {
        child_start[9 * r + c] = i;
        while (i < e && int(child_of[perm[i]]) == c) ++i;
    }
    child_start[9 * r + 8] = e;
}

__global__ void k_gather_points(int64_t n, int n_g, const int *__restrict__ perm, const double *__restrict__ y0,
                                const double *__restrict__ q0, const double *__restrict__ len0,
                                const int *__restrict__ leaf_of, double *__restrict__ y, double *__restrict__ q,
                                int64_t *__restrict__ sid, double *__restrict__ slen, int *__restrict__ pos,
                                int *__restrict__ pleaf, const unsigned char *__restrict__ child_of,
                                const int *__restrict__ ref_start, int *__restrict__ pfine) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    int k = perm[i];
    pleaf[i] = leaf_of[k];
    if (pfine) {
        const int lf = leaf_of[k];
        pfine[i] = ref_start[lf + 1] > ref_start[lf] ? 8 * ref_start[lf] + int(child_of[k]) : -1;
    }
    for (int d = 0; d < 3; ++d) y[3 * i + d] = y0[3 * int64_t(k) + d];
    for (int d = 0; d < 9; ++d) q[9 * i + d] = q0[9 * int64_t(k) + d];
    sid[i] = k / n_g;
    slen[i] = len0[k / n_g];
    pos[k] = int(i);
}

__global__ void k_gather_targets(int64_t n, const int *__restrict__ perm, const double *__restrict__ x0,
                                 double *__restrict__ x, int *__restrict__ pos) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    int k = perm[i];
    for (int d = 0; d < 3; ++d) x[3 * i + d] = x0[3 * int64_t(k) + d];
    pos[k] = int(i);
}

// Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method from the
// guess cos(pi (i + 3/4) / (n + 1/2)), weights 2 / ((1 - x^2) P_n'(x)^2),
// with P_n from the three-term recurrence k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}.
void legendre_pair(int n, double z, double *pn, double *pm) {
    double a = 1.0, b = z;  // P_0, P_1
    for (int k = 2; k <= n; ++k) {
        double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / k;
        a = b;
        b = c;
    }
    *pn = b;
    *pm = a;
}

void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn, pm, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, z, &pn, &pm);
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre_pair(n, z, &pn, &pm);
        dp = n * (z * pn - pm) / (z * z - 1.0);
        x[n - 1 - i] = z;  // ascending
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

}  // namespace

int tree_build(gbfmm_ctx *ctx, bool validate) {
    cudaStream_t st = ctx->stream;
    const int ng = ctx->opt.n_gauss;
    const int64_t N = ctx->N;
    GaussParams gp{};
    gp.n = ng;
    gauss_legendre(ng, gp.xi, gp.w);
    for (int i = 0; i < ng; ++i) {
        ctx->gauss_xi[i] = gp.xi[i];
        ctx->gauss_w[i] = gp.w[i];
    }
    const int64_t nl = ctx->n_leaves;
    double *y0 = ctx->d_y0, *q0 = ctx->d_q0, *len0 = ctx->d_len0, *part = ctx->d_part;
    int *leaf_of = ctx->d_leaf_of, *cnt = ctx->d_cnt, *cursor = ctx->d_cursor, *perm = ctx->d_perm;
    int *bad = ctx->d_bad;
    const int nparts = 512;
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    ++ctx->launches;
    k_gauss_points<<<nblk(ctx->n_segs, 128), 128, 0, st>>>(ctx->n_segs, ctx->node_xyz, ctx->seg_nodes, ctx->burgers,
                                                           gp, y0, q0, len0, bad);
    ++ctx->launches;
    k_bbox_partial<<<nparts, 256, 0, st>>>(N, y0, part);
    ++ctx->launches;
    k_bbox_final<<<1, 32, 0, st>>>(nparts, part, ctx->d_box);
    CK(cudaMemsetAsync(cnt, 0, nl * sizeof(int), st));
    CK(cudaMemsetAsync(cursor, 0, nl * sizeof(int), st));
    ++ctx->launches;
    auto &RF = ctx->rf;
    const bool refine = RF.on != 0;
    k_leaf_count<<<nblk(N, 256), 256, 0, st>>>(N, y0, ctx->d_box, ctx->L, leaf_of, cnt, refine ? RF.child_of : nullptr);
    ++ctx->launches;
    k_scan<<<1, 1024, 0, st>>>(nl, cnt, ctx->d_leaf_start);
    ++ctx->launches;
    k_scatter<<<nblk(N, 256), 256, 0, st>>>(N, leaf_of, ctx->d_leaf_start, cursor, perm);
    ++ctx->launches;
    k_leaf_sort<<<unsigned(nl), 128, 0, st>>>(nl, ctx->d_leaf_start, perm, refine ? RF.child_of : nullptr,
                                               ctx->opt.refine_points);
    RF.n_ref_host = -1;
    if (refine) {
        // split leaves: flags, their scan (leaf -> split index), each split leaf's child ranges
        ctx->launches += 3;
        k_ref_flags<<<nblk(nl, 256), 256, 0, st>>>(nl, ctx->d_leaf_start, ctx->opt.refine_points, cursor);
        k_scan<<<1, 1024, 0, st>>>(nl, cursor, RF.ref_start);
        k_ref_children<<<nblk(nl, 128), 128, 0, st>>>(nl, ctx->d_leaf_start, RF.ref_start, perm, RF.child_of,
                                                      RF.ref_leaf, RF.child_start);
    }
    ++ctx->launches;
    k_gather_points<<<nblk(N, 256), 256, 0, st>>>(N, ng, perm, y0, q0, len0, leaf_of, ctx->d_y, ctx->d_q,
                                                  ctx->d_sid, ctx->d_slen, ctx->d_pos, ctx->d_pleaf,
                                                  refine ? RF.child_of : nullptr, RF.ref_start,
                                                  refine ? RF.pfine : nullptr);
    CK(cudaGetLastError());
    // without validation (a build recorded into a graph) the flag stays on the device:
    // fmm_batch_status reads it with the root box
    if (!validate) return GBFMM_OK;
    int hbad = 0, href = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TreeBox hb{};
    CK(cudaMemcpyAsync(&hb, ctx->d_box, sizeof(TreeBox), cudaMemcpyDeviceToHost, st));
    if (refine) CK(cudaMemcpyAsync(&href, RF.ref_start + nl, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (refine) RF.n_ref_host = href;
    if (hbad) return set_err(ctx, GBFMM_ERR_DEGENERATE, "fmm_build_tree: zero-length or non-finite segment");
    if (!std::isfinite(hb.H)) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_build_tree: non-finite node coordinates");
    return GBFMM_OK;
}

// Free targets: bin into leaves of the built tree and sort.
int targets_sort(gbfmm_ctx *ctx, int64_t n_t, const double *x) {
    cudaStream_t st = ctx->stream;
    const int64_t nl = ctx->n_leaves;
    // the scratch holds per-target and per-leaf arrays: regrow for more targets or more leaves
    if (nl > ctx->t_cap_leaves) ctx->t_cap = 0;
    const int64_t t0 = ctx->t_cap;
    if (int rc = grow_dev(ctx, ctx->t_cap, n_t,
                          {{(void **)&ctx->d_t_pos, n_t * sizeof(int)}, {(void **)&ctx->d_t_x, n_t * 3 * sizeof(double)},
                           {(void **)&ctx->d_t_sig, n_t * 6 * sizeof(double)},
                           {(void **)&ctx->d_t_tmp, (2 * n_t + 2 * nl) * sizeof(int)}},
                          "targets")) {
        ctx->t_cap_leaves = 0;
        return rc;
    }
    if (ctx->t_cap != t0) ctx->t_cap_leaves = nl;
    int *leaf_of = ctx->d_t_tmp, *perm = leaf_of + n_t, *cnt = perm + n_t, *cursor = cnt + nl;
    CK(cudaMemsetAsync(cnt, 0, nl * sizeof(int), st));
    CK(cudaMemsetAsync(cursor, 0, nl * sizeof(int), st));
    ++ctx->launches;
    k_leaf_count<<<nblk(n_t, 256), 256, 0, st>>>(n_t, x, ctx->d_box, ctx->L, leaf_of, cnt, nullptr);
    ++ctx->launches;
    k_scan<<<1, 1024, 0, st>>>(nl, cnt, ctx->d_t_start);
    ++ctx->launches;
    k_scatter<<<nblk(n_t, 256), 256, 0, st>>>(n_t, leaf_of, ctx->d_t_start, cursor, perm);
    ++ctx->launches;
    k_leaf_sort<<<unsigned(nl), 128, 0, st>>>(nl, ctx->d_t_start, perm, nullptr, 0);
    ++ctx->launches;
    k_gather_targets<<<nblk(n_t, 256), 256, 0, st>>>(n_t, perm, x, ctx->d_t_x, ctx->d_t_pos);
    CK(cudaGetLastError());
    return GBFMM_OK;
}
