/*
 * gbfmm -- Lagrange fast multipole method for the stress field and
 * Peach-Koehler forces of straight dislocation segments, on one GPU.
 *
 * Method: Chen, Aubry, Oppelstrup, Arsenlis, Darve, "Fast algorithms for
 * evaluating the stress field of dislocation lines in anisotropic elastic
 * media" (arXiv:1712.07739).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer argument marked "device" is a CUDA device pointer owned by
 *   the caller; the library never frees it and never copies it to the host.
 *   Pointers marked "host" are read during the call only.
 * - All device work is issued, in order, on the CUDA stream given to
 *   fmm_create (the legacy default stream if NULL).  Entry points return as
 *   soon as the work is queued, except where a comment says they
 *   synchronise.  Results are valid once that stream reaches the call.
 * - Return value: GBFMM_OK (0) or a negative GBFMM_ERR_* code; the context
 *   keeps a message for the last error (fmm_last_error).  On an error the
 *   outputs of that call are undefined and the context stays usable.
 * - Stress is stored in Voigt order xx, yy, zz, yz, xz, xy (6 doubles per
 *   point); vectors are xyz triples; all arrays are row-major and densely
 *   packed.
 * - The library owns its workspaces (tree, multipole and local values, the
 *   M2L operator tables), allocated by fmm_set_material and fmm_build_tree
 *   and released by fmm_destroy.  fmm_eval_nodal_forces allocates nothing;
 *   fmm_eval_stress grows a target buffer when n_t exceeds every earlier
 *   call's.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define GBFMM_OK 0
#define GBFMM_ERR_INVALID_ARG -1   /* a size, pointer or option is out of range */
#define GBFMM_ERR_NOT_BUILT -2     /* fmm_eval_* before fmm_build_tree */
#define GBFMM_ERR_NO_MATERIAL -3   /* fmm_build_tree / fmm_eval_* before fmm_set_material */
#define GBFMM_ERR_CUDA -4          /* a CUDA runtime call failed (message has the name) */
#define GBFMM_ERR_TIMEOUT -5       /* a bounded device wait gave up */
#define GBFMM_ERR_DEGENERATE -6    /* zero-length segment or non-positive-definite medium */

/* precision of the pass */
#define GBFMM_FP64 0   /* every stage in FP64 */
#define GBFMM_MIXED 1  /* FP32 P2M/M2M/L2L/L2P and near field (FP64 for close pairs),
                          M2L on tcgen05 tensor cores (operand precision: m2l_split) */
#define GBFMM_MIXED_F64T 2  /* as GBFMM_MIXED with P2M, M2M, L2L and L2P in FP64, which removes the
                               rounding of those interpolations (the Lebesgue constants of
                               equispaced nodes amplify it at high orders) */

/* how the Green's-function factor h_vpq(T) = R^2 dG_vp/dx_q is evaluated */
#define GBFMM_H_ISO 0     /* closed form of the isotropic Green's function (Sec. 2, Eq. "k_iso") */
#define GBFMM_H_CIRCLE 1  /* trapezoid rule of the unit-circle integral (any medium) */
#define GBFMM_H_MLP 2     /* trained network (fmm_mlp_train), plain evaluator where flagged */

/* operand precision of the tensor-core M2L (gbfmm_options.m2l_split, MIXED only) */
#define GBFMM_M2L_BF16_SPLIT 0      /* BF16, residual passes on the offsets with max |o_i| = 2 */
#define GBFMM_M2L_BF16 1            /* BF16 only */
#define GBFMM_M2L_BF16_SPLIT_ALL 2  /* BF16, residual passes on all 316 offsets */
#define GBFMM_M2L_TF32 3            /* FP32 operands, kind::tf32 */
#define GBFMM_M2L_FP16 4            /* FP16, multipole values scaled per level */
#define GBFMM_M2L_FP16_SPLIT 5      /* FP16 scaled, residual passes on the offsets with max |o_i| = 2 */
#define GBFMM_M2L_FP16_SPLIT_ALL 6  /* FP16 scaled, residual passes on all 316 offsets (fmm_default_options,
                                       over the leading K block: m2l_split_kblocks = 1) */

/* interpolation nodes per axis of a cell (gbfmm_options.nodes) */
#define GBFMM_NODES_EQUISPACED 0  /* t_a = a / (p - 1), faces included (Sec. 4.1) */
#define GBFMM_NODES_CHEBYSHEV 1   /* zeros of T_p mapped to [0, 1] (the Chebyshev FMM, Sec. 3) */

typedef struct {
    int p;                 /* Lagrange nodes per dimension, 2..8 (Sec. 4.1) */
    int n_gauss;           /* Gauss points per segment, 1..16 (Sec. 2, Eq. "stress_discrete") */
    int levels;            /* octree levels L >= 3, leaves at level L-1; 0 = choose from N_s */
    int precision;         /* GBFMM_FP64, GBFMM_MIXED or GBFMM_MIXED_F64T */
    int h_mode;            /* GBFMM_H_ISO, GBFMM_H_CIRCLE or GBFMM_H_MLP */
    int circle_q;          /* trapezoid points on the half circle for GBFMM_H_CIRCLE; 0 = 64 */
    int leaf_segments;     /* with levels == 0: target mean segments per occupied leaf; 0 = 32 */
    double near_fp64;      /* MIXED: near pairs closer than near_fp64 x (source segment length)
                              are evaluated in FP64; 0 = 2.0 */
    int m2l_split;         /* MIXED: operand precision of the tensor-core M2L, GBFMM_M2L_*:
                              0 = BF16 with residual (split) passes on the offsets with
                              max |o_i| = 2, 1 = BF16 only, 2 = BF16 with residual passes on
                              all 316 offsets, 3 = TF32 (FP32 operands), 4 = FP16 with
                              per-level scaling of the multipole values (a power of two from
                              each level's largest |W|) and one power-of-two scale for the
                              operators, 5 = as 4 plus residual passes
                              on the offsets with max |o_i| = 2, 6 = as 4 plus residual
                              passes on all 316 offsets (fmm_default_options) */
    double mlp_min_dist;   /* GBFMM_H_MLP: near pairs closer than this many source segment
                              lengths use the plain evaluator; 0 = 8 */
    int m2l_fft;           /* FP64: 1 = M2L through the Toeplitz structure of the operators
                              (Sec. 4.1, Theorem 1): each offset's node-to-node map applied as
                              a convolution, by products of discrete Fourier transforms of size
                              (2p)^3 (54 (2p)^2 (p+1) complex multiply-adds per cell pair
                              instead of 54 p^6; fmm_default_options); 0 = dense node-pair
                              sums.  The transform form reads each level's count of occupied
                              cells back to the host, so an FP64 evaluation synchronises the
                              stream once per level; it falls back to the dense form while the
                              stream is being captured into a graph. */
    int m2l_chunks;        /* MIXED: the tensor-core M2L sums each class's 189 offsets in this
                              many consecutive runs, each accumulated in tensor memory from
                              zero and added to the local values in FP32 (FP64 with
                              GBFMM_MIXED_F64T); shorter accumulation chains, one launch per
                              run.  0 = 1; fmm_default_options: 7. */
    int m2l_basis;         /* MIXED: operands of the tensor-core M2L.  0 = the node values of
                              Eq. "m2l" (multipole values at the source cell's nodes); 1 = the
                              Legendre moments of each source cell, sum_j P_k(y_j) q_j with
                              Legendre polynomials of degree < p per axis, against operators
                              T V^-1 precomputed in FP64 -- the same product in exact
                              arithmetic, without the oscillating node values whose
                              cancellation inside each GEMM costs precision
                              (fmm_default_options). */
    int m2l_split_levels;  /* MIXED, m2l_split 0, 2, 5 or 6: the residual passes apply only at
                              the tree levels whose bit is set (bit l = level l); 0 = all. */
    int m2l_split_kblocks; /* MIXED, with residual passes: they cover only this many leading
                              K blocks of 64 operand columns (0 = all).  With m2l_basis = 1
                              the columns are ordered by the moments' total degree, so the
                              leading blocks hold the low-order moments, which carry most of
                              every product and hence most of its rounding error
                              (fmm_default_options: 1). */
    int m2l_kernel;        /* MIXED: form of the tile GEMM of the tensor-core M2L.  0 = three
                              tiles of 128 target cells per CTA as the M operands, one block of
                              operator rows shared as N; 1 = two 128-row blocks of operator
                              rows as the M operands, the CTA's 256 target cells shared as
                              N = 256 (half the gathered bytes per product). */
    int nodes;             /* GBFMM_NODES_EQUISPACED (fmm_default_options) or
                              GBFMM_NODES_CHEBYSHEV; Chebyshev nodes need the compressed M2L
                              (m2l_svd_tol > 0, MIXED): their operators have no Toeplitz
                              structure. */
    double m2l_svd_tol;    /* MIXED: > 0 compresses the M2L by the singular value decomposition
                              (the Chebyshev FMM's compression, Sec. 3, Eq. "mem_cheb"): the
                              316 unit-cell operators T_o [6 p^3 x 9 p^3] side by side give a
                              target basis U (left singular vectors), stacked a source basis R
                              (right singular vectors); a vector is kept while its singular
                              value exceeds m2l_svd_tol times the largest, the kept counts
                              rounded up to the tile granularity (r1 to 16, r2 to 64).  Each
                              pass then transforms every cell's multipole values W -> R^T W
                              (r2 values), runs the tensor-core M2L on the r1 x r2 operators
                              U^T T_o R, and expands the local values S = U S'.  The bases and
                              operators are built in FP64 at fmm_set_material; m2l_basis is
                              ignored.  0 = off (fmm_default_options). */
    int refine_points;     /* MIXED with the compressed M2L on FP16 operands (m2l_split 4, 5
                              or 6) and the unit-circle h: > 0 makes
                              the tree adaptive -- every leaf holding more than this many Gauss
                              points is split once more (one level below the leaves).  Two
                              adjacent split leaves interact through their children: adjacent
                              children directly, the others by an M2L one level down; all
                              other adjacent leaves directly; points of split leaves take their
                              child's local values.  The children's M2L runs one GEMM per
                              offset over the occupied pairs (cuBLAS) and reads the pair counts
                              back, so the pass synchronises once.  Nodal forces only
                              (fmm_eval_stress keeps the uniform tree).  0 = off
                              (fmm_default_options). */
    int m2l_symmetry;      /* FP64 with m2l_fft = 1: 1 = keep the transformed operators of 16
                              offsets only (Sec. 6: the cube's symmetries of space and kernel
                              map every one of the 316 operators to a signed permutation of
                              rows and columns of one of 16; the table shrinks 316/16 times) and
                              apply each offset's from its representative's at permuted
                              frequencies.  Needs a medium with those symmetries (isotropic, or
                              cubic with axes along x, y, z): fmm_eval_* returns INVALID_ARG
                              for any other.  0 = off (fmm_default_options). */
} gbfmm_options;

typedef struct gbfmm_ctx gbfmm_ctx;

/* Fill *opt with defaults (p=4, n_gauss=4, levels=0, FP64, H_ISO, m2l_fft = 1; for the mixed
   pass: m2l_split = GBFMM_M2L_FP16_SPLIT_ALL with m2l_split_kblocks = 1, m2l_basis = 1,
   m2l_chunks = 7 -- FP16 Legendre-moment operands, residual passes on the leading block of
   low-order moments, offsets summed in 7 runs). */
void fmm_default_options(gbfmm_options *opt);

/* Create a context.  opt: host, copied.  cuda_stream: a cudaStream_t or NULL.
 * The current CUDA device at this call is the one the context uses. */
int fmm_create(gbfmm_ctx **out, const gbfmm_options *opt, void *cuda_stream);

/* Destroy a context and free its device memory (synchronises its stream). */
void fmm_destroy(gbfmm_ctx *ctx);

/* Message of the last error on this context ("" if none). */
const char *fmm_last_error(const gbfmm_ctx *ctx);

/* Set the elastic medium and precompute the M2L operators.
 *
 * C_voigt: host, 36 doubles, the 6x6 stiffness in Voigt order
 * (11, 22, 33, 23, 13, 12), row-major; must be symmetric positive definite.
 * With GBFMM_H_ISO the medium must be isotropic (C11 - C12 = 2 C44, cubic
 * form); mu = C44 and nu = C12 / (2 (C12 + C44)) are taken from it.
 *
 * Builds, on the device, the kernel K_abwr = A_{ab,wr,vpq} h_vpq / R^2 of
 * Sec. 2, Eq. "kernel" at every node difference of every M2L offset (the
 * operators T_{A->B} of Sec. 4.1, Eq. "m2l"; they depend only on the medium
 * and p, Sec. 4.1) for cells of unit size; level l scales them by
 * (2^l / H)^2 (homogeneity of degree -2, Sec. 4.1 footnote).
 * Synchronises the stream.  Errors: INVALID_ARG, DEGENERATE, CUDA. */
int fmm_set_material(gbfmm_ctx *ctx, const double *C_voigt);

/* Build the octree of a segment network.
 *
 * node_xyz:  device, [n_nodes][3] double, node positions.
 * seg_nodes: device, [n_segs][2] int64, node indices (line sense n0 -> n1).
 * burgers:   device, [n_segs][3] double, Burgers vector per segment.
 *
 * Computes the Gauss points y and strengths q_wr = 1/2 b_w omega S_r of
 * Sec. 2, Eq. "stress_discrete", the root cube (edge H = s (1 + 2^-10), s the
 * largest extent of the Gauss points, centred on their bounding box), bins
 * every point into its leaf and sorts points by leaf.  The context keeps
 * the three pointers: fmm_eval_nodal_forces reads them again, so they must
 * stay valid and unchanged until the next fmm_build_tree or fmm_destroy.
 * Synchronises the stream (reads back the bounding box).
 * Errors: INVALID_ARG (n_segs < 1, n_nodes < 2, null pointer), CUDA. */
int fmm_build_tree(gbfmm_ctx *ctx, int64_t n_nodes, const double *node_xyz,
                   int64_t n_segs, const int64_t *seg_nodes, const double *burgers);

/* Stress at arbitrary points (Sec. 2, Eq. "stress3" by Algorithm 2).
 *
 * x:     device, [n_t][3] double target positions.  Targets outside the root
 *        cube are assigned to the nearest boundary leaf.
 * sigma: device, [n_t][6] double, output (Voigt).
 * Every source point contributes (no self exclusion: targets are free
 * points).  Errors: NOT_BUILT, NO_MATERIAL, INVALID_ARG, CUDA. */
int fmm_eval_stress(gbfmm_ctx *ctx, int64_t n_t, const double *x, double *sigma);

/* Peach-Koehler nodal forces of the built network (Sec. 2 and Sec. 1).
 *
 * The stress is evaluated at every Gauss point, leaving out the point's own
 * segment; the force per unit length (sigma . b) x xi is integrated against
 * the linear shape functions of the segment ends with the same Gauss rule:
 *   f1 = sum_k (omega_k/2) (1 - xi_k)/2 (sigma_k b) x S,
 *   f2 = sum_k (omega_k/2) (1 + xi_k)/2 (sigma_k b) x S.
 * f_nodes: device, [n_nodes][3] double, output: sum of the end forces of
 *          the segments incident to each node (overwritten).
 * f_seg:   device, [n_segs][2][3] double (f1, f2 per segment) or NULL.
 * sigma_pts: device, [n_segs * n_gauss][6] double (stress at each Gauss point,
 *          segment-major) or NULL.
 * Errors: NOT_BUILT, NO_MATERIAL, CUDA. */
int fmm_eval_nodal_forces(gbfmm_ctx *ctx, double *f_nodes, double *f_seg, double *sigma_pts);

/* Level count, leaf count and number of Gauss points of the built tree
 * (host outputs; any may be NULL). */
int fmm_tree_info(const gbfmm_ctx *ctx, int *levels, int64_t *n_leaves, int64_t *n_points);

/* The compressed M2L of a context (m2l_svd_tol > 0; set up by its first
 * build): ranks[0..3] = target and source coefficients per cell as run (r1,
 * r2, rounded up to the tiles) and the counts above the tolerance;
 * sigma[0..3] = largest and smallest kept singular value, target side then
 * source side.  All zero when the M2L is not compressed or not set up.
 * ranks: host, 4 ints; sigma: host, 4 doubles; either may be NULL. */
int fmm_m2l_ranks(const gbfmm_ctx *ctx, int *ranks, double *sigma);

/* Device time in milliseconds of each stage of the last fmm_eval_* call,
 * measured with CUDA events on the context stream: [0] precompute
 * source tensors, [1] P2M+M2M, [2] M2L, [3] L2L, [4] L2P+P2P, [5] forces.
 * Only filled when timing was enabled with fmm_set_timing(ctx, 1); the
 * call then synchronises the stream.  times: host, 8 doubles. */
int fmm_set_timing(gbfmm_ctx *ctx, int enable);
int fmm_stage_times(const gbfmm_ctx *ctx, double *times);

/* Number of CUDA kernels this context has launched since fmm_create
 * (host output). */
int fmm_launch_count(const gbfmm_ctx *ctx, int64_t *count);

/* Work of one pass over the built tree, for roofline accounting
 * (host output, 4 int64): [0] near-field point pairs evaluated by the
 * self-evaluation of fmm_eval_nodal_forces (target x source point pairs in
 * neighbouring leaves, own-segment pairs excluded; with refine_points > 0,
 * pairs between non-adjacent children of two split leaves excluded too),
 * [1] M2L cell pairs (target cell, interaction-list cell) with both
 * non-empty, the split leaves' children included, [2] occupied leaves,
 * [3] Gauss points.  Launches a few small kernels and synchronises.
 * Errors: NOT_BUILT, CUDA. */
int fmm_work_counts(gbfmm_ctx *ctx, int64_t *counts);

/* Status word of the device kernels that wait on barriers (the tensor-core
 * M2L): GBFMM_OK, or GBFMM_ERR_TIMEOUT when a bounded wait gave up during an
 * earlier pass (that pass's outputs are then invalid).  Synchronises the
 * stream, reads the word into *status (host) and clears it. */
int fmm_device_status(gbfmm_ctx *ctx, int *status);

/* ------------------------------------------------------------------------
 * Testing only: failure injection (not part of the method; no production
 * caller needs it).
 * ------------------------------------------------------------------------ */

/* Failure-detection test hook.  kind = 1: the next tensor-core M2L
 * (GBFMM_MIXED) arms its first pipeline stage without loading it, so the
 * consumer's bounded wait runs out (about 10 s); the pass then reports
 * GBFMM_ERR_TIMEOUT through fmm_device_status and its outputs are invalid.
 * Nothing faults and the context stays usable.  Errors: INVALID_ARG. */
int fmm_inject_fault(gbfmm_ctx *ctx, int kind);

/* ------------------------------------------------------------------------
 * Measurement (not part of the method): the device's fused multiply-add
 * throughput, the denominator of the near-field and FP64-pass rooflines.
 * ------------------------------------------------------------------------ */

/* Measured peak rate in TFLOP/s (2 per multiply-add) on the current device:
 * kind 0 = FP32 scalar FMA, 1 = FP32 packed pairs (two multiply-adds per
 * instruction), 2 = FP64 FMA.  Every thread of 8 blocks per SM runs 8
 * independent chains x <- x/2 + 1 (CUDA events, on cuda_stream, which may be
 * NULL); the launch grows until it lasts ~150 ms and the best of three such
 * launches is reported.  Each chain must end exactly at its fixed point 2
 * (self-check).  Synchronises.  Allocates 4 bytes of device memory.
 * Errors: INVALID_ARG, CUDA, DEGENERATE (a chain missed its fixed point). */
int fmm_probe_fma(int kind, void *cuda_stream, double *tflops);

/* ------------------------------------------------------------------------
 * Batches of independent segment networks.
 *
 * A batch holds one network per slot; all slots share the medium's tables
 * (kernel lattice and M2L operators, which do not depend on the network).
 * With opt.levels == 0 each slot's tree depth is chosen by an autotuner
 * (the near/far cost balance of App. B): one pass of the network is timed at
 * each candidate depth L0 - 1 .. L0 + 1 (L0 from N_s / leaf_segments; the
 * deepest only while the time is still falling) and the fastest is kept; the slot keeps
 * it for later builds while its N_s stays within 10 %.  The first network
 * built also gives two informational constants (c_near, c_far: seconds per
 * near pair and per cell of levels >= 2 at L0).  Created with m2l_kernel = 2,
 * that first network also times both tile forms of the tensor-core M2L
 * (gbfmm_options.m2l_kernel) and the faster is kept for every slot.
 * fmm_batch_eval_nodal_forces records the passes of
 * all slots into one CUDA graph (spread over up to 8 internal streams and
 * joined back onto the batch's stream) on its first call after a build, and
 * replays it afterwards.
 * ------------------------------------------------------------------------ */
typedef struct gbfmm_batch gbfmm_batch;

/* n_configs >= 1 slots, options as for fmm_create; cuda_stream: the
 * stream the batch's evaluation is ordered on. */
int fmm_batch_create(gbfmm_batch **out, const gbfmm_options *opt, int n_configs, void *cuda_stream);
void fmm_batch_destroy(gbfmm_batch *batch);
const char *fmm_batch_last_error(const gbfmm_batch *batch);
/* Medium for every slot (host, 36 doubles, as fmm_set_material).  Synchronises. */
int fmm_batch_set_material(gbfmm_batch *batch, const double *C_voigt);
/* Build slot k's tree (arguments as fmm_build_tree; the same lifetime rule
 * for the three arrays).  Runs the autotuner when the batch's options have
 * levels == 0.  Synchronises.  Errors: INVALID_ARG, NO_MATERIAL, CUDA. */
int fmm_batch_build(gbfmm_batch *batch, int k, int64_t n_nodes, const double *node_xyz, int64_t n_segs,
                    const int64_t *seg_nodes, const double *burgers);
/* Nodal forces of every slot: f_nodes is a host array of n_configs device
 * pointers ([n_nodes_k][3] double each, overwritten).  Asynchronous on the
 * batch's stream.  Errors: NOT_BUILT, CUDA. */
int fmm_batch_eval_nodal_forces(gbfmm_batch *batch, double *const *f_nodes);
/* One step of every slot as one CUDA graph: each slot's tree is rebuilt from
 * the arrays given at its last fmm_batch_build (the caller may have changed
 * their contents, e.g. moved the nodes, but not their sizes or addresses) and
 * its nodal forces evaluated into f_nodes[k] (host array of n_configs device
 * pointers).  The graph is recorded on the first call (and again after a
 * build that changes a slot's depth, sizes or buffers) and replayed after;
 * nothing synchronises the host.  The recorded builds skip the host-side
 * checks of fmm_batch_build: fmm_batch_status reports what they found.
 * Every slot must have been built once with fmm_batch_build.
 * Errors: NOT_BUILT, CUDA. */
int fmm_batch_step(gbfmm_batch *batch, double *const *f_nodes);

/* Checks of the last builds and passes of every slot (synchronises): *status
 * is GBFMM_OK, or for the first slot *slot with a problem GBFMM_ERR_DEGENERATE
 * (a zero-length or non-finite segment), GBFMM_ERR_INVALID_ARG (non-finite
 * node coordinates) or GBFMM_ERR_TIMEOUT (a bounded wait of the M2L gave up;
 * cleared by the read).  slot, status: host. */
int fmm_batch_status(gbfmm_batch *batch, int *slot, int *status);

/* Tile form of the tensor-core M2L the slots use, and when the autotuner chose
 * it (batch created with m2l_kernel = 2) the M2L stage time of each form on
 * the calibration network in milliseconds (-1 when not measured).  Any output
 * may be NULL; m2l_ms: host, 2 doubles. */
int fmm_batch_tuning(const gbfmm_batch *batch, int *m2l_kernel, double *m2l_ms);

/* Slot k's tree depth, the total kernel launches of all slots (direct
 * launches plus the kernel nodes of every graph replay), and the cost
 * constants measured on the first network (seconds per near pair, per cell);
 * any output may be NULL. */
int fmm_batch_info(const gbfmm_batch *batch, int k, int *levels, int64_t *launches, double *c_near, double *c_far);

/* ------------------------------------------------------------------------
 * Learned angular factor (a stand-in for the plain evaluator of h).
 *
 * A network 3 -> 128 -> 128 -> 128 -> 27 (SiLU; BF16 weight matrices, FP32
 * biases and accumulation) maps a unit direction T to h_vpq(T) (27
 * components, index (v*3 + p)*3 + q); h is odd, so the network sees T folded
 * into the upper half-space and the sign is restored.  Parameters: 37,664
 * floats, order W1 [128x3], b1 [128], W2 [128x128], b2, W3 [128x128], b3,
 * W4 [32x128] (rows 27..31 zero), b4 [32]; plus 27 output scales.
 * Directions are device float [n][3] (unit length not required).
 * ------------------------------------------------------------------------ */

/* h by the plain evaluator of the context's medium (FP64 unit-circle rule,
 * or the isotropic closed form), as float y [n][27] (device).
 * Errors: NO_MATERIAL, INVALID_ARG, CUDA. */
int fmm_mlp_labels(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *y);

/* Train the network on the plain evaluator's h at the given directions
 * (device, [n][3]; the caller draws them): Adam, mini-batches of `batch`,
 * `epochs` passes, cosine-decayed learning rate from `lr`, initial weights
 * and shuffling from `seed`.  final_loss (host, may be NULL): last batch's
 * mean squared error in scaled units.  Synchronises the stream.
 * Errors: NO_MATERIAL, INVALID_ARG, CUDA. */
int fmm_mlp_train(gbfmm_ctx *ctx, int64_t n, const float *dirs, int epochs, int batch, double lr,
                  uint64_t seed, float *final_loss);

/* Assess the network against the plain evaluator per angular bin (5 x 256
 * bins of direction, 64 sample directions each) and record which bins the
 * near field of GBFMM_H_MLP must evaluate with the plain rule: those whose
 * largest component error exceeds bin_tol x (RMS of h).  fallback_frac
 * (host, may be NULL): fraction of bins flagged.  Required before a
 * GBFMM_H_MLP evaluation.  Synchronises the stream.
 * Errors: INVALID_ARG (network not set), NO_MATERIAL, CUDA. */
int fmm_mlp_calibrate(gbfmm_ctx *ctx, double bin_tol, double *fallback_frac);

/* Copy the parameters (host, 37,664 floats) and output scales (host, 27). */
int fmm_mlp_get(gbfmm_ctx *ctx, float *theta, float *scale);
int fmm_mlp_set(gbfmm_ctx *ctx, const float *theta, const float *scale);

/* Network h at n directions: h (device, float [n][27]). */
int fmm_mlp_eval(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *h);

/* Loss and gradient of one batch for the current parameters: y (device,
 * [n][27] target h), grad (device, 37,664 floats), loss (host, may be NULL;
 * synchronises when given). */
int fmm_mlp_grad(gbfmm_ctx *ctx, int n, const float *dirs, const float *y, float *grad, float *loss);

/* Network h at n directions without allocating device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate during the call -- a dislocation-dynamics code that
 * evaluates h from inside its own fixed memory pool or a time step it
 * replays, or one that runs under a device-memory budget it manages itself.
 * Results equal those of fmm_mlp_eval.  Instead of per-context buffers it
 * uses one statically allocated device array of 4.5 MiB (activations of
 * 4,096 directions; larger n is processed 4,096 at a time), which every
 * GPU that loads this library holds until the process exits.
 *
 * dirs: device, float [n][3]; h: device, float [n][27]; n <= 2^24, larger
 * n returns GBFMM_ERR_INVALID_ARG with a message.  Call it with the
 * context's device current.  The first call on a device looks up the
 * array's device address (no allocation); make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other
 * contexts on the same device, other host threads) race and must be
 * serialised by the caller.  Errors: INVALID_ARG (sizes, pointers, network
 * not set), CUDA. */
int fmm_mlp_eval_noalloc(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *h);

#ifdef __cplusplus
}
#endif
#endif
