// Internal declarations of the gbfmm CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gbfmm.h"
#include "m2l_fft.cuh"
#include "m2l_tc.cuh"

#define GB_MAXP 8
#define GB_MAXG 16

// Stress components in Voigt order: (a, b) index pairs.
// h_vpq is symmetric in (v, p); the 6 pairs below use the same order, so a
// symmetric-pair index k = 3 * pair + q covers the 18 distinct components.
__host__ __device__ inline int voigt_a(int i) { return i < 3 ? i : (i == 3 ? 1 : 0); }
__host__ __device__ inline int voigt_b(int i) { return i < 3 ? i : (i == 5 ? 1 : 2); }

// Material as the device kernels see it (copied by value into kernel args
// through a device buffer).
struct DevMaterial {
    int mode;     // GBFMM_H_ISO / GBFMM_H_CIRCLE / GBFMM_H_MLP
    int Q;        // half-circle trapezoid points
    double hc;    // iso: 1 / (16 pi mu (1 - nu))
    double ha;    // iso: 3 - 4 nu
    double C[81]; // C_ijkl
    int cubic;    // 1: cubic with axes along x, y, z (c12, c44, cd below are set)
    double c12, c44, cd;  // C12, C44, C11 - C12 - 2 C44
};

// Geometry of the tree as kernels see it; the root box lives on the device
// (written by the bounding-box kernel), everything else is host-known.
struct TreeBox {
    double origin[3];
    double H;      // root cube edge
    double lo[3], hi[3];
};

// learned angular factor (mlp.cu)
struct MlpState {
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;  // FP32 masters, gradient, Adam moments
    __nv_bfloat16 *theta_h = nullptr;  // BF16 copy used by the kernels
    float *scale = nullptr;            // per-output scale [32]
    float *loss = nullptr;
    void *bufs = nullptr;              // batch activations
    uint32_t *d_binmask = nullptr;     // [48] angular bins where the plain evaluator is used
    double fallback_frac = 1.0;        // fraction of bins flagged by the last calibration
    bool trained = false;
    int64_t step = 0;
};

// work list of the near kernels (near.cu)
struct NearWork {
    int2 *items = nullptr, *sorted = nullptr;
    int *keys = nullptr, *cnt = nullptr, *key_of = nullptr, *off = nullptr, *misc = nullptr;
    int64_t cap = 0, cap_leaves = 0;
    // symmetric near field (nodal forces, unit-circle h): leaf-pair items and
    // per-direction partial stresses [28][N][6]
    int2 *pitems = nullptr, *psorted = nullptr;
    int *pkeys = nullptr, *pmisc = nullptr;
    double *part = nullptr;
    int64_t pcap = 0, part_cap = 0;
};

struct Timer {
    cudaEvent_t ev[16];
    bool on = false;
    int n = 0;
};

struct gbfmm_ctx {
    gbfmm_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    int sm_count = 0;

    // material
    bool have_material = false;
    DevMaterial mat{};
    DevMaterial *d_mat = nullptr;
    double Asym[6 * 9 * 18];   // A contracted over the (v,p) symmetry: [ab][wr][k]
    double *d_Asym = nullptr;
    float *d_Asym_f = nullptr;
    int lat_n = 0;             // lattice points per dimension, 8 (p-1) + 1
    double *d_Klat = nullptr;  // [lat_n^3][54] kernel at unit-cell lattice differences

    // mixed-precision M2L on tensor cores
    TcPlan tc;
    // FP64 M2L through transforms (gbfmm_options.m2l_fft)
    FftPlan fft;
    // learned h
    MlpState mlp;
    NearWork nw;
    bool borrowed_material = false;  // medium tables belong to another context (a batch)

    // tree
    bool built = false;
    int L = 0;                 // levels; leaves at level L-1
    int64_t n_nodes = 0, n_segs = 0, N = 0;
    int64_t n_cells = 0;       // all levels
    int64_t n_leaves = 0;
    TreeBox *d_box = nullptr;
    double gauss_xi[GB_MAXG], gauss_w[GB_MAXG];
    double *d_y = nullptr;     // [N][3] sorted by leaf
    double *d_q = nullptr;     // [N][9]
    int64_t *d_sid = nullptr;  // [N] segment of each sorted point
    double *d_slen = nullptr;  // [N] length of that segment
    int *d_pos = nullptr;      // [N] original point index -> sorted position
    int *d_pleaf = nullptr;    // [N] leaf of each sorted point
    int *d_leaf_start = nullptr;  // [n_leaves + 1]
    int *d_tmp_i = nullptr;       // scratch ints, N + n_leaves + 1
    double *d_tmp_d = nullptr;    // scratch doubles
    // build scratch
    double *d_y0 = nullptr, *d_q0 = nullptr, *d_len0 = nullptr, *d_part = nullptr;
    int *d_leaf_of = nullptr, *d_cnt = nullptr, *d_cursor = nullptr, *d_perm = nullptr, *d_bad = nullptr;
    // capacities (elements) of the buffers sized by N, segments, cells, leaves
    int64_t cap_N = 0, cap_segs = 0, cap_cells = 0, cap_leaves = 0;
    const int64_t *seg_nodes = nullptr;  // caller's arrays (kept for forces)
    const double *burgers = nullptr;
    const double *node_xyz = nullptr;

    // adaptive tree (gbfmm_options.refine_points > 0): every leaf holding more points is
    // split once more; sizes are bounded by N / (refine_points + 1) split leaves, so the
    // build needs no host read-back
    struct Refine {
        int on = 0;
        int64_t cap_ref = 0;                   // split leaves the buffers hold
        int64_t n_ref_host = -1;               // split leaves of the last validated build (-1: not read)
        int64_t cap_N = 0, cap_leaves = 0, cap_cells = 0;
        unsigned char *child_of = nullptr;     // [N] original order: child (0..7) of the point's leaf
        int *ref_start = nullptr;              // [n_leaves + 1] scan of the split flags: leaf -> split index
        int *ref_leaf = nullptr;               // [cap_ref] split index -> leaf
        int *child_start = nullptr;            // [cap_ref][9] sorted-point ranges of the children
        int *pfine = nullptr;                  // [N] sorted point -> child cell 8 r + c, or -1
        float *W7 = nullptr;                   // [8 cap_ref][9 p^3] children's multipole values
        float *S7 = nullptr;                   // [8 cap_ref][6 p^3] children's local values
        float *Wc7 = nullptr;                  // [8 cap_ref][r2] compressed multipole values
        float *Sc7 = nullptr;                  // [8 cap_ref][r1] compressed local values
        // child cells the fine-level launches cover: the split leaves a validated build read
        // back, else the capacity (kernels skip the rows past the device count)
        int64_t fine_rows() const { return 8 * (n_ref_host >= 0 ? n_ref_host : cap_ref); }
    } rf;

    // per-eval buffers
    double *d_P = nullptr;     // [N][108] precontracted source tensors (FP64)
    float *d_Pf = nullptr;     // [N][108] FP32 copy for the mixed path
    double *d_W = nullptr;     // [n_cells][p^3][9] multipole weights
    double *d_S = nullptr;     // [n_cells][p^3][6] local values
    float *d_Wf = nullptr;
    float *d_Sf = nullptr;
    double *d_sig = nullptr;   // [N][6] stress at sorted points
    float4 *d_yrel = nullptr;  // [N] mixed: leaf-relative FP32 position, segment length
    int64_t mx_cap_N = 0, mx_cap_cells = 0;

    // free-target evaluation
    int64_t t_cap = 0;                 // targets the buffers below hold (0 after a failed allocation)
    int64_t t_cap_leaves = 0;          // leaves the target scratch was sized for
    int *d_t_pos = nullptr;     // target -> sorted slot
    int *d_t_start = nullptr;   // [n_leaves + 1]
    double *d_t_x = nullptr;    // sorted targets
    double *d_t_sig = nullptr;  // sorted results
    int *d_t_tmp = nullptr;

    int64_t launches = 0;      // kernels launched by this context so far
    Timer timer;
    double stage_ms[8] = {0};
};

// error helpers
int set_err(gbfmm_ctx *c, int code, const std::string &msg);

// Hash of everything an evaluation's launches depend on besides the contents
// of device memory: sizes, depth, options and every device pointer.  A graph
// recorded from an evaluation stays valid while this value is unchanged.
uint64_t layout_hash(const gbfmm_ctx *ctx);  // api.cu
#include "grow.h"

// grow_set on device memory (cudaMalloc / cudaFree); a failed allocation sets
// the context's error and returns GBFMM_ERR_CUDA
inline int grow_dev(gbfmm_ctx *ctx, int64_t &cap, int64_t need, const GrowBuf *bufs, int n, const char *what) {
    const int rc = grow_set(
        cap, need, bufs, n, [](void **p, size_t b) { return cudaMalloc(p, b) == cudaSuccess ? 0 : -1; },
        [](void *p) { cudaFree(p); });
    if (rc == 0) return GBFMM_OK;
    const cudaError_t e = cudaGetLastError();  // clears the (non-sticky) allocation error
    return set_err(ctx, GBFMM_ERR_CUDA, std::string("cudaMalloc (") + what + "): " + cudaGetErrorString(e));
}
inline int grow_dev(gbfmm_ctx *ctx, int64_t &cap, int64_t need, std::initializer_list<GrowBuf> bufs,
                    const char *what) {
    return grow_dev(ctx, cap, need, bufs.begin(), int(bufs.size()), what);
}
#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return set_err(ctx, GBFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// cell indexing: level l occupies [cell_base(l), cell_base(l) + 8^l),
// linear index (z * n + y) * n + x with n = 2^l.
inline int64_t cell_base(int l) { return ((int64_t(1) << (3 * l)) - 1) / 7; }
__host__ __device__ inline int64_t cell_base_d(int l) { return ((int64_t(1) << (3 * l)) - 1) / 7; }

// stages (implemented in the .cu files)
int material_setup(gbfmm_ctx *ctx);                 // material.cu
int tree_build(gbfmm_ctx *ctx, bool validate = true);  // tree.cu; validate: read back the checks (synchronises)
int fmm_pass(gbfmm_ctx *ctx, bool free_targets, int64_t n_t);  // fmm.cu
int forces_from_stress(gbfmm_ctx *ctx, double *f_nodes, double *f_seg, double *sigma_pts);
int targets_sort(gbfmm_ctx *ctx, int64_t n_t, const double *x);
int targets_scatter(gbfmm_ctx *ctx, int64_t n_t, double *sigma);
void timer_mark(gbfmm_ctx *ctx);
void compute_occ(gbfmm_ctx *ctx, const int *start, int *occ);
int share_material(gbfmm_ctx *dst, const gbfmm_ctx *src);  // material.cu
