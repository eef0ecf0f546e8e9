// Tensor-core M2L plan (see m2l_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#define GB_TC_MAXLEV 8

struct gbfmm_ctx;

struct TcPlan {
    bool ready_ops = false;
    int Kp = 0, Np = 0;        // padded K (9 p^3 -> multiple of 64) and N (6 p^3 -> groups x 3 nsub)
    int Kp_lo = 0;             // K columns of the residual operators (the leading blocks the residual passes read)
    int nsub = 0, ncta = 0, groups = 0, tmem_cols = 0;
    int swap = 0;              // operators as the A operand (gbfmm_options.m2l_kernel = 1)
    int tpc = 3;               // tiles of 128 target cells per CTA
    int nblk = 0;              // operators as A: 128-row operator blocks
    int n_off = 0, n_lo = 0;   // operators and residual operators
    int split = 1;             // residual passes on offsets with max |o_i| = 2
    int tf32 = 0;              // operands in FP32 storage, MMA kind::tf32 (no residual passes)
    int fp16 = 0;              // FP16 operands: operators x op_scale, multipole values x a power of
                               // two per level chosen from the level's largest |W|
    double op_scale = 1.0;     // power of two applied to the FP16 operators
    int modal = 0;             // operands are the source cells' Legendre moments (gbfmm_options.m2l_basis)
    double basisV[64] = {0}, basisCt[64] = {0};  // V1[n][a] = P_n(2 t_a - 1) and (V1^-1)^T
    unsigned *d_wmax = nullptr;  // per level: bits of max |W| over occupied cells (FP16 mode)
    int esz = 2;               // operand element size in bytes
    void *Thi = nullptr, *Tlo = nullptr;  // operators [n_off][Np][Kp] (bf16, or fp32 when tf32)
    void *Whi = nullptr, *Wlo = nullptr;  // packed multipole weights
    int64_t wofs[GB_TC_MAXLEV] = {0};
    int64_t w_cap = 0;
    int n_work = 0;            // blocks launched: tile bound x groups (surplus blocks return)
    int *d_status = nullptr;
    int inject_drop = 0;       // set by fmm_inject_fault: the next run leaves one stage unfilled
    int *d_flags = nullptr, *d_pos = nullptr, *d_list = nullptr;  // target cells of levels >= 2
    int4 *d_seg = nullptr;     // per (level, class): first list entry, count, first tile
    int64_t slot_cap = 0, n_slots = 0;
    int n_seg = 0;
    // SVD-compressed M2L (gbfmm_options.m2l_svd_tol > 0, m2l_svd.cu): the GEMM runs on
    // r2 source and r1 target coefficients per cell
    int svd = 0;
    int r1 = 0, r2 = 0;        // kept target / source singular vectors (rounded up to 16 / 64)
    int r1_raw = 0, r2_raw = 0;  // counts above the tolerance
    float *Uf = nullptr;       // target basis [6 p^3][r1], column-major (ld 6 p^3), shared in a batch
    float *Rf = nullptr;       // source basis [9 p^3][r2], column-major (ld 9 p^3), shared in a batch
    double *U64 = nullptr, *R64 = nullptr;  // the bases in FP64 (operator construction)
    void *Uh = nullptr, *Ul = nullptr;  // U split into FP16 hi + lo (x sU), [6 p^3 padded to 8][r1], shared
    void *Rh = nullptr, *Rl = nullptr;  // R split likewise, [9 p^3 padded to 8][r2], shared
    float sU = 1.f, sR = 1.f;  // the bases' power-of-two scales
    int bases_ok = 0;          // U, R belong to the current medium and options
    void *Xh = nullptr, *Xl = nullptr;  // per tree: one level's transform input split into FP16 hi + lo
    int64_t x_cap = 0;
    float *d_scal = nullptr;   // per tree: 0, 1 and the per-level GEMM scale factors (device scalars)
    unsigned *d_bits = nullptr;  // per tree: per-level largest |value| bits of the transform inputs
    double svd_sigma[4] = {0}; // largest and smallest kept singular values: target, source
    float *Wc = nullptr;       // per tree: [n_cells][r2] compressed multipole values
    float *Sc = nullptr;       // per tree: [n_cells][r1] compressed local values
    int64_t c_cap = 0;
    void *blas = nullptr;      // cuBLAS handle of this context (its own workspace: contexts of a
    void *blas_ws = nullptr;   // batch run concurrently)
    size_t blas_ws_bytes = 0;
    short lo_host[320] = {0};  // per operator (offset order of the table): its residual operator or -1
    // adaptive tree: the children's M2L over the occupied (target, source) pairs, one GEMM per
    // offset (m2l_svd.cu, fine_m2l)
    int *d_pcnt = nullptr;     // [343 offset slot -> operator][316 counts][317 firsts][316 cursors]
    int2 *d_pairs = nullptr;   // (target child, source child), grouped by operator
    int64_t pair_cap = 0;
    void *Gh = nullptr, *Gl = nullptr;  // gathered source rows of a run of offsets, FP16 hi / lo
    float *Yf = nullptr;       // their products [pairs][Np]
    int64_t g_cap = 0;
    int h_pcnt[316] = {0}, h_pfirst[317] = {0};  // host copies of the counts and their scan
};

int m2l_tc_setup(gbfmm_ctx *ctx);    // operators (per medium and p)
int m2l_tc_prepare(gbfmm_ctx *ctx);  // per tree
// W64 / S64 non-null: FP64 multipole values in, FP64 local values out (GBFMM_MIXED_F64T);
// fine: the adaptive tree's children take part (compressed M2L: transforms of their values,
// fine_m2l over their pairs, expansion into their local values)
int m2l_tc_run(gbfmm_ctx *ctx, const float *Wf, const double *W64, const int *occ, const int *tocc, float *Sf,
               double *S64, bool fine = false);
void m2l_tc_free(gbfmm_ctx *ctx);
int m2l_tc_status(gbfmm_ctx *ctx, int *out);

// SVD compression (m2l_svd.cu).  svd_bases: the two bases and the kept ranks (before the
// operator tables are sized); svd_operators: the compressed operators U^T T_o R of the
// n_off offsets (xyz in d_off) into T.Thi / T.Tlo with the FP16 scale; svd_prepare: per-tree
// buffers; svd_transform_w / svd_expand_s: R^T W per cell of levels 2..L-1 before the
// M2L and S = U S' after it; svd_free: this context's handle and buffers (and the bases
// unless borrowed).
int svd_bases(gbfmm_ctx *ctx);
int svd_operators(gbfmm_ctx *ctx, const int *d_off, const int *d_lo, int n_off);
int svd_prepare(gbfmm_ctx *ctx);
int fine_m2l(gbfmm_ctx *ctx);  // adaptive tree: children's M2L into their compressed local values
int svd_transform_w(gbfmm_ctx *ctx, const float *Wf, bool fine);
int svd_expand_s(gbfmm_ctx *ctx, float *Sf, bool fine);
void svd_free(gbfmm_ctx *ctx, bool borrowed);
