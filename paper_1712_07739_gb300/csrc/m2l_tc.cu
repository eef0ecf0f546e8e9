// M2L on the tcgen05 tensor cores: offset-grouped dense GEMMs (Sec. 4.1,
// Eq. "m2l"; the M2L stage of Algorithm 2) with FP32 accumulation in TMEM.
//
// Formulation.  At level l the cells form a 2^l grid.  Split it into the 8
// parity classes c = (x & 1, y & 1, z & 1); each class is an m^3 sub-grid,
// m = 2^(l-1).  For a target cell B = 2P + c and an offset o in its
// interaction list, the source A = B - o lies in class c' = (c - o) mod 2 at
// sub-grid position P + s, s = floor((c - o) / 2) in [-1, 1]^3.  The 189
// offsets of class c are therefore, each, a constant shift between two
// sub-grids.
//
// Tiles.  The cells of a (level, class) that hold targets are listed in
// Morton order of their sub-grid position; 128 consecutive ones form a tile,
// and a CTA takes TPC = 3 consecutive tiles and one group of nsub operator
// rows.  The M2L of a tile is
//     S[cell, n] = (2^l / H)^2  sum_o  sum_k  W_c'[cell + s_o, k] T_o[n, k]
// with k = (node m, component wr) and n = (node l, stress component ab):
// per tile one GEMM of M = 128 cells, N = nsub and K = (active offsets) x
// 9 p^3, accumulated in tensor memory (TPC accumulators of nsub columns).
// Each pipeline stage holds the three tiles' multipole rows (gathered by
// cp.async, one row per thread and tile, into the swizzled layout the MMA
// reads; sources outside the sub-grid or without segments read as zeros)
// and one block of operator rows (TMA) that all three tiles use: a stage
// moves 66 KB for 7.1 MFLOP, mostly rows of the level's multipole table,
// which stay in L2 far better than the 1.6 GB of operators.  Offsets whose
// sources are all empty are skipped.
//
// Precision: BF16 operands (hi); for the offsets nearest to the target
// (max |o_i| = 2, the largest far-field terms) the residuals W_lo = W - hi(W)
// and T_lo = T - hi(T) add two more passes, hi*hi + lo*hi + hi*lo.  Other
// modes: TF32 operands; FP16 operands with a power-of-two scale per level for
// W and one for the operators (FP16 carries 3 more mantissa bits than BF16).
//
// Warp roles (192 threads): warp 0 loads the operator rows by TMA, warp 1
// owns TMEM and issues the MMAs, warps 2-5 gather the multipole rows (each
// thread waits for its copies, fences them to the async proxy and arrives on
// the stage's barrier) and then read the accumulator out (warp w reads TMEM
// lanes 32 (w % 4) .. 32 (w % 4) + 31).  Every mbarrier wait is bounded; on
// time-out a device status word gets GBFMM_ERR_TIMEOUT and the block winds
// down, freeing its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "m2l_tc.cuh"

namespace {

struct OffsetEntry {
    short top;      // operator index 0..315
    short lo;       // index in the residual table, -1 when the offset has no split pass
    signed char cls;  // source parity class
    signed char sx, sy, sz;
};

__constant__ OffsetEntry c_offs[8][189];

struct M2LParams {
    const uint8_t *Whi, *Wlo;         // packed W (hi, residual), level l at byte wofs[l]
    int64_t wofs[GB_TC_MAXLEV];
    int row_bytes;                    // K_pad x element size
    CUtensorMap tmT;                  // T hi: (Kp, Np, 316)
    CUtensorMap tmTlo;                // T residual: (Kp, Np, n_lo)
    int kb;         // K blocks of 64
    int kb_res;     // K blocks the residual passes cover (the leading ones)
    int nsub;       // N per MMA (multiple of 16, <= 256)
    int ncta;       // operator rows per CTA (= nsub)
    int nvalid;     // 6 p^3
    int tmem_cols;  // power of two >= ncta
    int split;      // residual passes on the near offsets, at the levels whose bit is set in split_levels
    int split_levels;
    int drop_first; // failure-detection test: arm the first stage but issue no load into it
    int kstep;      // operand elements per 128-byte row: 64 (bf16, fp16) or 32 (tf32)
    uint32_t idesc; // tcgen05 instruction descriptor
    const unsigned *wmax;  // FP16 mode: per-level max |W| bits (the W scale), else null
    float inv_op_scale;    // FP16 mode: 1 / operator scale, else 1
    int nblk;              // operators as A: 128-row blocks of operator rows (a CTA takes two)
    int o_lo, o_hi;        // this launch takes the entries o_lo .. o_hi - 1 of each class's offset list
    int accumulate;        // 0: the epilogue writes the local values, 1: it adds to them
};

// FP16 mode: power of two that brings a level's largest |W| into [2^12, 2^13)
// (FP16 is normal from 2^-14 to 65504, so 26 binades below the largest value
// keep full relative precision); 1 for a level without values
__device__ __forceinline__ float wscale_of(unsigned bits) {
    const float mx = __uint_as_float(bits);
    if (!(mx > 0.f)) return 1.f;
    int e;
    frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, 13 - e);
}

// Two forms of the tile GEMM (gbfmm_options.m2l_kernel):
//  cells as A (SWAP = false): three tiles of 128 target cells per CTA are the M = 128
//    operands of three MMAs that share one block of nsub operator rows (B, N = nsub);
//  operators as A (SWAP = true): two 128-row blocks of operator rows are the M = 128
//    operands (TMA) of two MMAs that share the CTA's two tiles of target cells as one
//    N = 256 operand, so a gathered row feeds 256 instead of nsub output columns and a
//    stage gathers 32 instead of 48 KB for about the same tensor work.
constexpr int kTileA = 128 * 128;  // one tile's multipole rows per stage: 16 KB
template <bool SWAP> constexpr int tpc_of() { return SWAP ? 2 : 3; }  // tiles of 128 cells per CTA

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: gives up after ~10 s of device time (a healthy wait lasts microseconds)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > 10000000000ull) {
            atomicExch(status, GBFMM_ERR_TIMEOUT);
            return false;
        }
    }
}

// 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n groups of this thread are pending (n is 0..5)
__device__ __forceinline__ void cp_async_wait(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    }
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// UMMA shared-memory descriptor, K-major, 128-byte swizzle: start address,
// leading offset 16 B (unused inside one swizzle atom), stride offset 1024 B
// between 8-row groups, descriptor version 1, layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFF);
    d |= uint64_t(1) << 16;
    d |= uint64_t(1024 >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}

// instruction descriptor: D f32 (bits 4-5 = 1), A and B format (bits 7-9,
// 10-12: 1 = bf16 for kind::f16, 2 = tf32 for kind::tf32), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
inline uint32_t idesc_of(int M, int N, bool tf32, bool fp16) {
    // operand formats: kind::tf32 -> 2 (TF32); kind::f16 -> 0 (F16) or 1 (BF16); D in F32
    const uint32_t f = tf32 ? 2u : (fp16 ? 0u : 1u);
    return (1u << 4) | (f << 7) | (f << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Target lists.  Every cell of levels 2 .. L-1 has one slot: level l starts
// at cell_base(l) - cell_base(2), then class c (m^3 slots each), then the
// Morton code of the cell's sub-grid position.  The cells holding targets are
// listed in slot order; 128 consecutive ones of a (level, class) make a tile.
__host__ __device__ inline int64_t slot_base(int l) { return cell_base_d(l) - cell_base_d(2); }

__device__ __forceinline__ uint32_t morton_part(uint32_t v) {  // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t morton_compact(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}

// Segments: one per (level, class), index (l - 2) * 8 + c.  seg[s] = {first
// list entry, cells, first tile}; seg[n_seg].z = total tiles.
constexpr int kMaxSeg = 8 * GB_TC_MAXLEV;

// number of K-block iterations of one work item (same count on every warp);
// split: the residual passes apply at this level
__device__ __forceinline__ int passes_of(const OffsetEntry &e, int split) { return (split && e.lo >= 0) ? 3 : 1; }

template <bool TF32, bool SWAP>
__global__ void __launch_bounds__(192, 1)
    k_m2l_tc(const __grid_constant__ M2LParams P, const int4 *__restrict__ seg, int n_seg,
             const int *__restrict__ list, const int *__restrict__ occ, const int *__restrict__ tocc,
             const TreeBox *__restrict__ box, float *__restrict__ S, double *__restrict__ S64,
             int *__restrict__ status, int stages, int groups) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int TPC = tpc_of<SWAP>();
    constexpr int kStageA = TPC * kTileA;  // the tiles' gathered multipole rows
    // operator rows per stage: nsub rows (cells as A) or two 128-row blocks (operators as A)
    const int stageB = SWAP ? 2 * kTileA : P.ncta * 128;
    const int stage_bytes = kStageA + stageB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + stages * stage_bytes);
    // bars[0..stages): full, [stages..2 stages): empty, [2 stages]: accumulator ready
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 1);

    __shared__ int s_level, s_cls, s_rows, s_nrow, s_stop;  // s_rows, s_nrow: first list entry, cells of the CTA
    __shared__ short s_tgt[TPC][128][3];  // sub-grid positions of the tiles' target cells
    __shared__ uint32_t s_active[6];   // offsets with at least one occupied source cell
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int tile = blockIdx.x / groups, group = blockIdx.x % groups;
    if (threadIdx.x == 0) {
        s_level = -1;
        s_stop = *reinterpret_cast<volatile int *>(status) != 0;
        if (tile < seg[n_seg].z)
            for (int si = 0; si < n_seg; ++si) {
                const int4 sg = seg[si];
                const int nt = ((sg.y + 127) / 128 + TPC - 1) / TPC;
                if (tile >= sg.z && tile < sg.z + nt) {
                    s_level = si / 8 + 2;
                    s_cls = si % 8;
                    s_rows = sg.x + 128 * TPC * (tile - sg.z);  // first list entry of the CTA's tiles
                    s_nrow = min(128 * TPC, sg.y - 128 * TPC * (tile - sg.z));
                    break;
                }
            }
    }
    if (threadIdx.x < 6) s_active[threadIdx.x] = 0u;
    __syncthreads();
    if (s_level < 0 || s_stop) return;  // surplus block, or an earlier block timed out
    const int level = s_level, cls = s_cls, nrow = s_nrow;
    const int split = P.split && ((P.split_levels >> level) & 1);
    const int mbc = SWAP ? min(2, P.nblk - 2 * group) : 1;  // operator blocks of this CTA (operators as A)
    const int m = 1 << (level - 1), n = 1 << level;
    const int64_t cbase = cell_base_d(level);
    for (int r = threadIdx.x; r < 128 * TPC; r += blockDim.x) {
        int sx = -1024, sy = -1024, sz = -1024;  // rows past the CTA's cells: far outside the sub-grid
        if (r < nrow) {
            const uint32_t code = uint32_t(list[s_rows + r]);
            sx = int(morton_compact(code)), sy = int(morton_compact(code >> 1)), sz = int(morton_compact(code >> 2));
        }
        s_tgt[r / 128][r % 128][0] = short(sx), s_tgt[r / 128][r % 128][1] = short(sy);
        s_tgt[r / 128][r % 128][2] = short(sz);
    }
    __syncthreads();

    // active offsets: lane r of warp w checks rows 4r .. 4r + 3 of every tile
    for (int oi = P.o_lo + warp; oi < P.o_hi; oi += 6) {
        const OffsetEntry e = c_offs[cls][oi];
        const int ccx = e.cls & 1, ccy = (e.cls >> 1) & 1, ccz = e.cls >> 2;
        bool hit = false;
        for (int q = 0; q < 4 * TPC; ++q) {
            const int t = q / 4, row = 4 * lane + q % 4;
            const int px = s_tgt[t][row][0] + e.sx, py = s_tgt[t][row][1] + e.sy, pz = s_tgt[t][row][2] + e.sz;
            if (px >= 0 && py >= 0 && pz >= 0 && px < m && py < m && pz < m) {
                const int64_t g = cbase + (int64_t(2 * pz + ccz) * n + (2 * py + ccy)) * n + (2 * px + ccx);
                hit |= occ[g] > 0;
            }
        }
        if (__any_sync(0xffffffffu, hit) && lane == 0) atomicOr(&s_active[oi / 32], 1u << (oi % 32));
    }

    if (threadIdx.x == 0) {
        // full: the operator-load thread (expect_tx) + 128 gathering threads; empty: the MMA commit
        for (int s = 0; s < stages; ++s) mbar_init(smem_u32(&bars[s]), 129);
        for (int s = stages; s < 2 * stages + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[stages]), accb = smem_u32(&bars[2 * stages]);
    const uint32_t smem0 = smem_u32(smem);

    if (warp == 0 && lane == 0) {
        // ---------------- operator rows (B) by TMA
        int it = 0;
        bool ok = true;
        for (int oi = 0; oi < 189 && ok; ++oi) {
            if (!((s_active[oi / 32] >> (oi % 32)) & 1u)) continue;
            const OffsetEntry e = c_offs[cls][oi];
            const int np = passes_of(e, split);
            for (int pass = 0; pass < np && ok; ++pass) {
                const CUtensorMap *tb = (pass == 2) ? &P.tmTlo : &P.tmT;
                const int tidx = (pass == 2) ? e.lo : e.top;
                for (int kb = 0; kb < (pass == 0 ? P.kb : P.kb_res); ++kb, ++it) {
                    const int s = it % stages;
                    const uint32_t ph = (it / stages) & 1;
                    if (!mbar_wait(empty0 + 8 * s, ph ^ 1, status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * s;
                    mbar_expect_tx(fb, uint32_t(SWAP ? mbc * kTileA : stageB));
                    if (P.drop_first && it == 0) continue;  // the MMA warp's wait on this stage runs out
                    if (SWAP)
                        for (int mb = 0; mb < mbc; ++mb)
                            tma_load_3d(smem0 + s * stage_bytes + kStageA + mb * kTileA, tb, kb * P.kstep,
                                        group * 256 + mb * 128, tidx, fb);
                    else
                        tma_load_3d(smem0 + s * stage_bytes + kStageA, tb, kb * P.kstep, group * P.ncta, tidx, fb);
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = P.idesc;
        int it = 0;
        bool ok = true;
        for (int oi = 0; oi < 189 && ok; ++oi) {
            if (!((s_active[oi / 32] >> (oi % 32)) & 1u)) continue;
            const OffsetEntry e = c_offs[cls][oi];
            const int np = passes_of(e, split);
            for (int pass = 0; pass < np && ok; ++pass) {
                for (int kb = 0; kb < (pass == 0 ? P.kb : P.kb_res); ++kb, ++it) {
                    const int s = it % stages;
                    const uint32_t ph = (it / stages) & 1;
                    if (!mbar_wait(full0 + 8 * s, ph, status)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a = smem0 + s * stage_bytes;
                    for (int kk = 0; kk < 4; ++kk) {
                        if (SWAP) {
                            // the two tiles' 256 rows (contiguous, 1024 B per 8 rows) are the N operand
                            const uint64_t bd = sw128_desc(a + kk * 32);
                            for (int mb = 0; mb < mbc; ++mb) {
                                const uint64_t ad = sw128_desc(a + kStageA + mb * kTileA + kk * 32);
                                mma_issue<TF32>(tmem + mb * 256, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                            }
                        } else {
                            const uint64_t bd = sw128_desc(a + kStageA + kk * 32);
                            for (int t = 0; t < TPC; ++t) {
                                const uint64_t ad = sw128_desc(a + t * kTileA + kk * 32);
                                mma_issue<TF32>(tmem + t * P.nsub, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                    }
                    mma_commit(empty0 + 8 * s);
                }
            }
        }
        // fires when every MMA issued above has completed (no MMA, no wait: see the epilogue)
        if (s_active[0] | s_active[1] | s_active[2] | s_active[3] | s_active[4] | s_active[5]) mma_commit(accb);
    } else if (warp >= 2) {
        const int row = threadIdx.x - 64;  // 0..127: this thread's tile row
        {
            // ---------------- multipole rows (A): gathered by cp.async into the 128-byte
            // swizzled K-major layout (16-byte piece c of row r at (c ^ (r & 7)) * 16);
            // sources outside the sub-grid, or empty, read as zeros.  Each thread finds
            // the source of its own row; the copies go by 8 lanes per row (lane l moves
            // piece l % 8 of rows 4 i + l / 8 of its warp's 32), so a warp instruction
            // reads four whole 128-byte row pieces.  A thread signals stage j full once it
            // has issued stage j + 1: issuing stage j + lag waits for the MMAs of stage
            // j + lag - stages, so with lag = stages - 1 the MMAs of stage j could not be
            // issued before those of stage j - 1 had finished; with lag = 1 they wait only
            // for stage j - 2, and two stages of copies stay in flight.
            const int lag = 1;
            int it = 0, done = 0;
            bool ok = true;
            const int c = lane & 7, wrow0 = row - lane;  // this warp's first tile row
            for (int oi = 0; oi < 189 && ok; ++oi) {
                if (!((s_active[oi / 32] >> (oi % 32)) & 1u)) continue;
                const OffsetEntry e = c_offs[cls][oi];
                int64_t own[TPC];
                uint32_t own_nb = 0;
#pragma unroll
                for (int t = 0; t < TPC; ++t) {
                    const int px = s_tgt[t][row][0] + e.sx, py = s_tgt[t][row][1] + e.sy,
                              pz = s_tgt[t][row][2] + e.sz;
                    bool have = px >= 0 && py >= 0 && pz >= 0 && px < m && py < m && pz < m;
                    own[t] = 0;
                    if (have) {
                        const int ccx = e.cls & 1, ccy = (e.cls >> 1) & 1, ccz = e.cls >> 2;
                        have = occ[cbase + (int64_t(2 * pz + ccz) * n + (2 * py + ccy)) * n + (2 * px + ccx)] > 0;
                        own[t] = (((int64_t(e.cls) * m + pz) * m + py) * m + px) * P.row_bytes;
                    }
                    own_nb |= have ? (1u << t) : 0u;
                }
                int64_t srcoff[8][TPC];
                uint32_t nbm = 0;  // bit 8 t + i: row 4 i + lane / 8 of tile t has a source
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int from = 4 * i + (lane >> 3);
                    const uint32_t f = __shfl_sync(0xffffffffu, own_nb, from);
#pragma unroll
                    for (int t = 0; t < TPC; ++t) {
                        srcoff[i][t] = __shfl_sync(0xffffffffu, own[t], from);
                        nbm |= ((f >> t) & 1u) << (8 * t + i);
                    }
                }
                const int np = passes_of(e, split);
                for (int pass = 0; pass < np && ok; ++pass) {
                    const uint8_t *wb = ((pass == 1) ? P.Wlo : P.Whi) + P.wofs[level];
                    for (int kb = 0; kb < (pass == 0 ? P.kb : P.kb_res); ++kb, ++it) {
                        const int s = it % stages;
                        const uint32_t ph = (it / stages) & 1;
                        if (!mbar_wait(empty0 + 8 * s, ph ^ 1, status)) {
                            ok = false;
                            break;
                        }
                        const uint32_t sbase = smem0 + s * stage_bytes;
                        const uint8_t *wk = wb + kb * 128 + 16 * c;
#pragma unroll
                        for (int t = 0; t < TPC; ++t)
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int r = wrow0 + 4 * i + (lane >> 3);
                                cp_async16(sbase + t * kTileA + r * 128 + ((c ^ (r & 7)) << 4), wk + srcoff[i][t],
                                           ((nbm >> (8 * t + i)) & 1u) ? 16u : 0u);
                            }
                        cp_async_commit();
                        if (it - done >= lag) {
                            // the copies of stage `done` are complete: make them visible to the
                            // tensor cores, then count this thread in that stage's full barrier
                            cp_async_wait(lag);
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            mbar_arrive(full0 + 8 * (done % stages));
                            ++done;
                        }
                    }
                }
            }
            cp_async_wait(0);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (; done < it; ++done) mbar_arrive(full0 + 8 * (done % stages));
        }
        // ---------------- epilogue: TMEM -> scaled FP32 local values of the tile's target cells
        bool any_src = false;
        for (int i = 0; i < 6; ++i) any_src |= s_active[i] != 0u;
        const bool ok = any_src ? mbar_wait(accb, 0, status) : true;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int q = warp % 4;
        const int trow = q * 32 + lane;  // TMEM lane = tile row
        float sc = float(double(n) / box->H) * float(double(n) / box->H);
        if (P.wmax) sc *= P.inv_op_scale / wscale_of(P.wmax[level]);
        const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;
        if (SWAP) {
            // TMEM lane = operator row (of block mb), column = target cell (tile col / 128)
            for (int mb = 0; mb < mbc; ++mb) {
                const int nr = group * 256 + mb * 128 + trow;  // this thread's operator row
                const bool rv = nr < P.nvalid;
                for (int c0 = 0; c0 < 256; c0 += 16) {
                    float v[16];
                    if (ok && any_src) tmem_ld16(tmem + (uint32_t(q * 32) << 16) + uint32_t(mb * 256 + c0), v);
                    for (int i = 0; i < 16; ++i) {
                        const int cell = c0 + i, t = cell >> 7, r = cell & 127;
                        if (!ok || !rv || cell >= nrow) continue;
                        const int64_t g = cbase +
                                          (int64_t(2 * s_tgt[t][r][2] + cz) * n + (2 * s_tgt[t][r][1] + cy)) * n +
                                          (2 * s_tgt[t][r][0] + cx);
                        const int64_t e = g * int64_t(P.nvalid) + nr;
                        if (!any_src) {
                            if (!P.accumulate) {
                                if (S64) S64[e] = 0.0;
                                else S[e] = 0.f;
                            }
                        } else if (P.accumulate) {
                            if (S64) S64[e] += double(v[i]) * double(sc);
                            else S[e] += v[i] * sc;
                        } else {
                            if (S64) S64[e] = double(v[i]) * double(sc);
                            else S[e] = v[i] * sc;
                        }
                    }
                }
            }
        }
        for (int t = 0; t < (SWAP ? 0 : TPC); ++t) {
            const bool valid = ok && t * 128 + trow < nrow;
            int64_t g = 0;
            if (valid)
                g = cbase + (int64_t(2 * s_tgt[t][trow][2] + cz) * n + (2 * s_tgt[t][trow][1] + cy)) * n +
                    (2 * s_tgt[t][trow][0] + cx);
            float *dst = S + g * int64_t(P.nvalid);
            double *dst64 = S64 ? S64 + g * int64_t(P.nvalid) : nullptr;  // FP64 local values, when kept
            if (ok && !any_src) {
                // no occupied source among this launch's offsets: zero local values (or nothing to add)
                if (valid && !P.accumulate)
                    for (int col = group * P.ncta; col < min(P.nvalid, (group + 1) * P.ncta); ++col) {
                        if (dst64) dst64[col] = 0.0;
                        else dst[col] = 0.f;
                    }
            } else if (ok) {
                for (int c0 = 0; c0 < P.nsub; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + (uint32_t(q * 32) << 16) + uint32_t(t * P.nsub + c0), v);
                    const int col = group * P.ncta + c0;
                    if (valid)
                        for (int i = 0; i < 16; ++i)
                            if (col + i < P.nvalid) {
                                if (P.accumulate) {
                                    if (dst64) dst64[col + i] += double(v[i]) * double(sc);
                                    else dst[col + i] += v[i] * sc;
                                } else {
                                    if (dst64) dst64[col + i] = double(v[i]) * double(sc);
                                    else dst[col + i] = v[i] * sc;
                                }
                            }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols));
    }
}

// ---------------------------------------------------------------- operators
// T_o[n = l*6 + ab][k = m*9 + wr] = Klat[o (p-1) + l - m][ab][wr] (unit cell);
// hi = bf16(T), lo = bf16(T - hi) (residual table only for split offsets).
template <typename E>
__device__ __forceinline__ E to_elem(double v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ float to_elem<float>(double v) {
    return float(v);
}
template <>
__device__ __forceinline__ __half to_elem<__half>(double v) {
    return __double2half(v);
}
__device__ __forceinline__ double elem_value(__half x) { return double(__half2float(x)); }
__device__ __forceinline__ double elem_value(__nv_bfloat16 x) { return double(__bfloat162float(x)); }
__device__ __forceinline__ double elem_value(float x) { return double(x); }

template <typename E>
__global__ void k_build_ops(int p, int lat_n, int Np, int Kp, int Kp_lo, const double *__restrict__ Klat,
                            const int *__restrict__ off_xyz, const int *__restrict__ lo_of, int n_off,
                            double scale, E *__restrict__ Thi, E *__restrict__ Tlo) {
    const int64_t total = int64_t(n_off) * Np * Kp;
    const int P3 = p * p * p;
    const int R0 = (lat_n - 1) / 2;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(idx % Kp);
        const int nn = int((idx / Kp) % Np);
        const int o = int(idx / (int64_t(Kp) * Np));
        double v = 0.0;
        if (nn < 6 * P3 && k < 9 * P3) {
            const int l = nn / 6, ab = nn % 6, mm = k / 9, wr = k % 9;
            const int ox = off_xyz[3 * o], oy = off_xyz[3 * o + 1], oz = off_xyz[3 * o + 2];
            const int Dx = ox * (p - 1) + (l % p) - (mm % p) + R0;
            const int Dy = oy * (p - 1) + ((l / p) % p) - ((mm / p) % p) + R0;
            const int Dz = oz * (p - 1) + (l / (p * p)) - (mm / (p * p)) + R0;
            v = scale * Klat[((int64_t(Dz) * lat_n + Dy) * lat_n + Dx) * 54 + ab * 9 + wr];
        }
        const E hi = to_elem<E>(v);
        Thi[idx] = hi;
        const int li = lo_of[o];
        if (li >= 0 && Tlo && k < Kp_lo) Tlo[(int64_t(li) * Np + nn) * Kp_lo + k] = to_elem<E>(v - elem_value(hi));
    }
}

// ---------------------------------------------------------------- Legendre-moment operands
// With gbfmm_options.m2l_basis = 1 the GEMM runs on the Legendre moments of
// each source cell instead of its node values: W'_k = sum_m P_k(ybar_m) W_m
// with P_k(t) = P_k1(2 t_1 - 1) P_k2(2 t_2 - 1) P_k3(2 t_3 - 1) (degrees
// k_i < p), which, since the node values come from Lagrange interpolation
// of degree p - 1, equals sum_j P_k(y_j) q_j over the cell's sources, and
// the operators become T' = T V^-1 (V = V1 x V1 x V1, V1[n][a] = P_n(2 t_a - 1)),
// so T' W' = T W exactly.  The moments are bounded by sum |q| and the rows of
// T' decay with the degree (Legendre coefficients of a smooth kernel), so the
// products summed in one GEMM do not cancel the way the oscillating node
// values of equispaced interpolation do, and 16-bit operands and FP32
// accumulation lose far less.  Every transform is separable: three passes
// of a p x p matrix along the node axes.
// Basis matrices, passed by value (they depend on p, which differs between contexts)
struct BasisMats {
    double V[GB_MAXP * GB_MAXP];   // V1[n][a]
    double Ct[GB_MAXP * GB_MAXP];  // (V1^-1)^T[n][a]
    float Vf[GB_MAXP * GB_MAXP];   // V1 in FP32 (moments of the FP32 pass)
    short pos[GB_MAXP * GB_MAXP * GB_MAXP];  // K position of moment (kz p + ky) p + kx: by total degree
};

// out[.., n, ..] = sum_a M[n][a] in[.., a, ..] along one node axis of a [p^3][9] block,
// summed in the precision R of the values
template <typename R, typename MT>
__device__ __forceinline__ void axis_pass(int p, int axis, const MT *M, const R *__restrict__ in, R *__restrict__ out) {
    const int P3 = p * p * p, stride = axis == 0 ? 1 : (axis == 1 ? p : p * p);
    for (int e = threadIdx.x; e < 9 * P3; e += blockDim.x) {
        const int m = e / 9, wr = e - 9 * m;
        const int n = (m / stride) % p, base = m - n * stride;
        R acc = R(0);
        for (int a = 0; a < p; ++a) acc += R(M[n * p + a]) * in[(base + a * stride) * 9 + wr];
        out[e] = acc;
    }
}

// Modal operator rows T'[o][n][k'] (FP64 arithmetic).  mode 0: largest |T'| into
// *absmax (the FP16 scale); mode 1: write hi (and lo for split offsets).
template <typename E>
__global__ void k_build_ops_modal(int p, int lat_n, int Np, int Kp, int Kp_lo, const double *__restrict__ Klat,
                                  const int *__restrict__ off_xyz, const int *__restrict__ lo_of, double scale,
                                  const __grid_constant__ BasisMats B, int mode, unsigned long long *__restrict__ absmax,
                                  E *__restrict__ Thi, E *__restrict__ Tlo) {
    extern __shared__ double sm_modal[];
    const int P3 = p * p * p, R0 = (lat_n - 1) / 2;
    const int o = blockIdx.x / Np, nn = blockIdx.x % Np;
    double *a = sm_modal, *b = sm_modal + 9 * P3;
    const int64_t row = (int64_t(o) * Np + nn) * Kp;
    const int li = lo_of[o];
    if (nn >= 6 * P3) {  // padding rows
        if (mode == 1)
            for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
                Thi[row + k] = to_elem<E>(0.0);
                if (li >= 0 && Tlo && k < Kp_lo) Tlo[(int64_t(li) * Np + nn) * Kp_lo + k] = to_elem<E>(0.0);
            }
        return;
    }
    const int l = nn / 6, ab = nn % 6;
    const int ox = off_xyz[3 * o], oy = off_xyz[3 * o + 1], oz = off_xyz[3 * o + 2];
    for (int e = threadIdx.x; e < 9 * P3; e += blockDim.x) {
        const int mm = e / 9, wr = e % 9;
        const int Dx = ox * (p - 1) + (l % p) - (mm % p) + R0;
        const int Dy = oy * (p - 1) + ((l / p) % p) - ((mm / p) % p) + R0;
        const int Dz = oz * (p - 1) + (l / (p * p)) - (mm / (p * p)) + R0;
        a[e] = Klat[((int64_t(Dz) * lat_n + Dy) * lat_n + Dx) * 54 + ab * 9 + wr];
    }
    __syncthreads();
    axis_pass<double, double>(p, 0, B.Ct, a, b);
    __syncthreads();
    axis_pass<double, double>(p, 1, B.Ct, b, a);
    __syncthreads();
    axis_pass<double, double>(p, 2, B.Ct, a, b);
    __syncthreads();
    if (mode == 0) {
        double mx = 0.0;
        for (int e = threadIdx.x; e < 9 * P3; e += blockDim.x) mx = fmax(mx, fabs(b[e]));
        for (int s = 16; s > 0; s >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, s));
        if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(absmax, (unsigned long long)__double_as_longlong(mx));
        return;
    }
    // column of moment kk, component wr: 9 pos[kk] + wr (moments ordered by total degree)
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        const int e = k < 9 * P3 ? 9 * B.pos[k / 9] + k % 9 : k;
        const double v = k < 9 * P3 ? scale * b[k] : 0.0;
        const E hi = to_elem<E>(v);
        Thi[row + e] = hi;
        if (li >= 0 && Tlo && e < Kp_lo) Tlo[(int64_t(li) * Np + nn) * Kp_lo + e] = to_elem<E>(v - elem_value(hi));
    }
}

// Node values -> Legendre moments, in place, for the occupied cells of one level
template <typename TW>
__global__ void k_w_modal(int level, int p, const __grid_constant__ BasisMats B, TW *__restrict__ W,
                          const int *__restrict__ occ) {
    extern __shared__ __align__(16) unsigned char sm_wm[];
    const int P3 = p * p * p;
    TW *a = reinterpret_cast<TW *>(sm_wm), *b = a + 9 * P3;
    const int64_t cells = int64_t(1) << (3 * level), base = cell_base_d(level);
    for (int64_t lin = blockIdx.x; lin < cells; lin += gridDim.x) {
        if (occ[base + lin] <= 0) continue;
        TW *w = W + (base + lin) * int64_t(9 * P3);
        __syncthreads();
        for (int e = threadIdx.x; e < 9 * P3; e += blockDim.x) a[e] = w[e];
        __syncthreads();
        if constexpr (sizeof(TW) == 8) {
            axis_pass<TW, double>(p, 0, B.V, a, b);
            __syncthreads();
            axis_pass<TW, double>(p, 1, B.V, b, a);
            __syncthreads();
            axis_pass<TW, double>(p, 2, B.V, a, b);
        } else {
            axis_pass<TW, float>(p, 0, B.Vf, a, b);
            __syncthreads();
            axis_pass<TW, float>(p, 1, B.Vf, b, a);
            __syncthreads();
            axis_pass<TW, float>(p, 2, B.Vf, a, b);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 9 * P3; e += blockDim.x) w[9 * B.pos[e / 9] + e % 9] = b[e];
    }
}

// W (FP32, [cell][kv]: kv = 9 p^3 node values or moments, or r2 compressed values) ->
// parity-split hi / lo, [class][mz][my][mx][Kp] per level, one block per cell at a time.
// Rows of cells without segments are not written: the gather never reads them (their
// copies are zero fills).
template <typename E, typename TW>
__global__ void k_pack_w(int level, int kv, int Kp, const TW *__restrict__ W, const int *__restrict__ occ,
                         const unsigned *__restrict__ wmax, E *__restrict__ hi, E *__restrict__ lo) {
    const int n = 1 << level, m = n / 2;
    const double s = wmax ? double(wscale_of(wmax[level])) : 1.0;
    const int64_t cells = int64_t(n) * n * n;
    for (int64_t lin = blockIdx.x; lin < cells; lin += gridDim.x) {
        const int64_t g = cell_base_d(level) + lin;
        if (occ[g] <= 0) continue;
        const int x = int(lin % n), y = int((lin / n) % n), z = int(lin / (int64_t(n) * n));
        const int cls = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        const int64_t row = (((int64_t(cls) * m + z / 2) * m + y / 2) * m + x / 2) * Kp;
        for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
            const double v = k < kv ? double(W[g * kv + k]) : 0.0;
            const double vs = s * v;
            const E h = to_elem<E>(vs);
            hi[row + k] = h;
            if (lo) lo[row + k] = to_elem<E>(vs - elem_value(h));
        }
    }
}

// largest |W| over the occupied cells of one level (non-negative floats order
// like their bit patterns), one block per cell at a time
template <typename TW>
__global__ void k_wmax(int level, int kv, const TW *__restrict__ W, const int *__restrict__ occ,
                       unsigned *__restrict__ wmax) {
    const int64_t cells = int64_t(1) << (3 * level), base = cell_base_d(level);
    float mx = 0.f;
    for (int64_t lin = blockIdx.x; lin < cells; lin += gridDim.x) {
        if (occ[base + lin] <= 0) continue;
        const TW *w = W + (base + lin) * int64_t(kv);
        for (int k = threadIdx.x; k < kv; k += blockDim.x) mx = fmaxf(mx, fabsf(float(w[k])));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(wmax + level, __float_as_uint(mx));
}

// largest |K| over the kernel lattice, skipping the singular origin
__global__ void k_lattice_absmax(int64_t n_pts, int64_t origin, const double *__restrict__ Klat,
                                 unsigned long long *__restrict__ out) {
    double mx = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_pts * 54;
         i += int64_t(gridDim.x) * blockDim.x)
        if (i / 54 != origin && isfinite(Klat[i])) mx = fmax(mx, fabs(Klat[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Target flags of one level: the slot of every cell that holds targets
__global__ void k_mb_flags(int level, const int *__restrict__ tocc, int *__restrict__ flags) {
    const int n = 1 << level, m = n / 2;
    const int64_t cells = int64_t(n) * n * n, m3 = int64_t(m) * m * m;
    for (int64_t lin = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; lin < cells;
         lin += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(lin % n), y = int((lin / n) % n), z = int(lin / (int64_t(n) * n));
        const int cls = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        const uint32_t code = morton_part(uint32_t(x >> 1)) | (morton_part(uint32_t(y >> 1)) << 1) |
                              (morton_part(uint32_t(z >> 1)) << 2);
        flags[slot_base(level) + cls * m3 + code] = tocc[cell_base_d(level) + lin] > 0 ? 1 : 0;
    }
}

// exclusive scan of n flags into pos[0..n] (one block)
__global__ void k_scan_flags(int n, const int *__restrict__ flags, int *__restrict__ pos) {
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024 * 8) {
        int v[8], sum = 0;
        for (int i = 0; i < 8; ++i) {
            const int k = base + threadIdx.x * 8 + i;
            v[i] = k < n ? flags[k] : 0;
            sum += v[i];
        }
        part[threadIdx.x] = sum;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        int run = carry + part[threadIdx.x] - sum;
        for (int i = 0; i < 8; ++i) {
            const int k = base + threadIdx.x * 8 + i;
            if (k < n) pos[k] = run;
            run += v[i];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) pos[n] = carry;
}

// compact list of the flagged slots (Morton code of the cell within its class)
__global__ void k_mb_list(int n, int L, const int *__restrict__ flags, const int *__restrict__ pos,
                          int *__restrict__ list) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (!flags[k]) continue;
        int l = 2;
        while (l + 1 < L && k >= slot_base(l + 1)) ++l;
        const int64_t m3 = int64_t(1) << (3 * (l - 1));
        list[pos[k]] = int((k - slot_base(l)) % m3);
    }
}

// segment table: {first list entry, cells, first CTA}; seg[n_seg].z = CTAs (per operator group)
__global__ void k_seg_table(int L, int tpc, const int *__restrict__ pos, int4 *__restrict__ seg) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int tiles = 0, si = 0;
    for (int l = 2; l < L; ++l) {
        const int64_t m3 = int64_t(1) << (3 * (l - 1));
        for (int c = 0; c < 8; ++c, ++si) {
            const int64_t s0 = slot_base(l) + c * m3;
            const int first = pos[s0], cnt = pos[s0 + m3] - first;
            seg[si] = make_int4(first, cnt, tiles, 0);
            tiles += ((cnt + 127) / 128 + tpc - 1) / tpc;  // CTAs: tpc tiles each
        }
    }
    seg[si] = make_int4(0, 0, tiles, 0);
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

inline unsigned nblk(int64_t n, int b) { return unsigned(std::min<int64_t>((n + b - 1) / b, 1 << 20)); }

}  // namespace

// V1[n][a] = P_n(2 t_a - 1) on the p equispaced nodes t_a = a / (p - 1), and the
// transpose of its inverse (Gauss-Jordan with partial pivoting, FP64)
static bool basis_matrices(int p, double *V, double *Ct) {
    for (int a = 0; a < p; ++a) {
        const double x = 2.0 * a / (p - 1) - 1.0;
        double pm = 1.0, pc = x;
        for (int n = 0; n < p; ++n) {
            const double v = n == 0 ? 1.0 : (n == 1 ? x : 0.0);
            if (n <= 1) {
                V[n * p + a] = v;
                continue;
            }
            const double nx = ((2.0 * n - 1.0) * x * pc - (n - 1.0) * pm) / n;
            pm = pc;
            pc = nx;
            V[n * p + a] = nx;
        }
    }
    double A[GB_MAXP][2 * GB_MAXP];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < 2 * p; ++j) A[i][j] = j < p ? V[i * p + j] : (j - p == i ? 1.0 : 0.0);
    for (int c = 0; c < p; ++c) {
        int piv = c;
        for (int r = c + 1; r < p; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (std::fabs(A[piv][c]) < 1e-300) return false;
        for (int j = 0; j < 2 * p; ++j) std::swap(A[c][j], A[piv][j]);
        const double d = A[c][c];
        for (int j = 0; j < 2 * p; ++j) A[c][j] /= d;
        for (int r = 0; r < p; ++r)
            if (r != c) {
                const double f = A[r][c];
                for (int j = 0; j < 2 * p; ++j) A[r][j] -= f * A[c][j];
            }
    }
    for (int n = 0; n < p; ++n)
        for (int a = 0; a < p; ++a) Ct[n * p + a] = A[a][p + n];  // (V1^-1)[a][n]
    return true;
}

static BasisMats basis_of(const TcPlan &T, int p) {
    BasisMats B;
    std::memset(&B, 0, sizeof(B));
    for (int i = 0; i < p * p; ++i) {
        B.V[i] = T.basisV[i];
        B.Ct[i] = T.basisCt[i];
        B.Vf[i] = float(T.basisV[i]);
    }
    // moments ordered by total degree kx + ky + kz (then by index): the leading K
    // blocks hold the low-order moments, which carry most of each product
    int next = 0;
    for (int deg = 0; deg <= 3 * (p - 1); ++deg)
        for (int kk = 0; kk < p * p * p; ++kk)
            if (kk % p + (kk / p) % p + kk / (p * p) == deg) B.pos[kk] = short(next++);
    return B;
}

// Offsets, their parity-class lists and the operator tables.
int m2l_tc_setup(gbfmm_ctx *ctx) {
    const int p = ctx->opt.p, P3 = p * p * p;
    TcPlan &T = ctx->tc;
    T.tf32 = ctx->opt.m2l_split == 3 ? 1 : 0;
    T.fp16 = (ctx->opt.m2l_split >= 4) ? 1 : 0;
    T.esz = T.tf32 ? 4 : 2;
    // compressed M2L: the GEMM's K and N are the kept source and target ranks
    T.svd = ctx->opt.m2l_svd_tol > 0.0 ? 1 : 0;
    if (T.svd)
        if (int rc = svd_bases(ctx)) return rc;
    T.Kp = ((((T.svd ? T.r2 : 9 * P3)) + 63) / 64) * 64;
    const int nv = T.svd ? T.r1 : 6 * P3;
    T.swap = ctx->opt.m2l_kernel == 1 ? 1 : 0;
    T.tpc = T.swap ? 2 : 3;
    if (T.swap) {
        // operators as A: blocks of 128 operator rows, two per CTA; N = 256 cells per MMA;
        // two accumulators of 256 columns
        T.nblk = (nv + 127) / 128;
        T.Np = T.nblk * 128;
        T.groups = (T.nblk + 1) / 2;
        T.nsub = 256;
        T.ncta = 256;
        T.tmem_cols = 512;
    } else {
        // N per MMA (= operator rows per CTA): multiple of 16, one accumulator per
        // tile, 3 x nsub <= 512 TMEM columns
        int best = 0, best_waste = 1 << 30;
        for (int ns = 16; ns * 3 <= 512 && ns <= 256; ns += 16) {
            const int g = (nv + ns - 1) / ns;
            const int waste = g * ns - nv + g * 32;  // padding plus a per-group cost (the tiles' rows are re-read)
            if (waste < best_waste) {
                best_waste = waste;
                best = ns;
            }
        }
        T.nsub = best;
        T.ncta = best;
        T.groups = (nv + T.ncta - 1) / T.ncta;
        T.Np = T.groups * T.ncta;
        T.nblk = 0;
        T.tmem_cols = 32;
        while (T.tmem_cols < 3 * T.nsub) T.tmem_cols *= 2;
    }
    // the 316 offsets, and which of them get the residual passes
    std::vector<int> off;
    std::vector<int> lo_of;
    int n_lo = 0;
    for (int oz = -3; oz <= 3; ++oz)
        for (int oy = -3; oy <= 3; ++oy)
            for (int ox = -3; ox <= 3; ++ox) {
                const int mx = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz)));
                if (mx < 2) continue;
                off.push_back(ox);
                off.push_back(oy);
                off.push_back(oz);
                const int sm = ctx->opt.m2l_split;
                const bool split = !T.tf32 && (sm == 2 || sm == 6 || ((sm == 0 || sm == 5) && mx == 2));
                lo_of.push_back(split ? n_lo++ : -1);
            }
    T.n_off = int(off.size() / 3);
    T.n_lo = n_lo;
    for (int i = 0; i < T.n_off && i < 320; ++i) T.lo_host[i] = short(lo_of[i]);
    OffsetEntry ent[8][189];
    for (int c = 0; c < 8; ++c) {
        const int cc[3] = {c & 1, (c >> 1) & 1, c >> 2};
        int cnt = 0;
        for (int i = 0; i < T.n_off; ++i) {
            const int o[3] = {off[3 * i], off[3 * i + 1], off[3 * i + 2]};
            bool in = true;
            for (int d = 0; d < 3; ++d)
                if (o[d] < -3 + cc[d] || o[d] > 2 + cc[d]) in = false;
            if (!in) continue;
            OffsetEntry &e = ent[c][cnt++];
            e.top = short(i);
            e.lo = short(lo_of[i]);
            int sc = 0;
            signed char sh[3];
            for (int d = 0; d < 3; ++d) {
                const int t = cc[d] - o[d];  // in [-2, 3]
                const int fl = (t >= 0) ? t / 2 : -((-t + 1) / 2);
                sh[d] = (signed char)fl;
                sc |= (t - 2 * fl) << d;
            }
            e.cls = (signed char)sc;
            e.sx = sh[0];
            e.sy = sh[1];
            e.sz = sh[2];
        }
        if (cnt != 189) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "m2l setup: class offset count != 189");
    }
    CK(cudaMemcpyToSymbol(c_offs, ent, sizeof(ent)));
    int *d_off = nullptr, *d_lo = nullptr;
    CK(cudaMalloc(&d_off, off.size() * sizeof(int)));
    CK(cudaMalloc(&d_lo, lo_of.size() * sizeof(int)));
    CK(cudaMemcpy(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_lo, lo_of.data(), lo_of.size() * sizeof(int), cudaMemcpyHostToDevice));
    // the residual passes read the leading m2l_split_kblocks blocks of K only
    const int kstep = 128 / T.esz;
    T.Kp_lo = ctx->opt.m2l_split_kblocks > 0 ? std::min(T.Kp, ctx->opt.m2l_split_kblocks * kstep) : T.Kp;
    const size_t hi_elems = size_t(T.n_off) * T.Np * T.Kp, lo_elems = size_t(T.n_lo) * T.Np * T.Kp_lo;
    if (T.Thi) cudaFree(T.Thi);
    if (T.Tlo) cudaFree(T.Tlo);
    T.Thi = T.Tlo = nullptr;
    CK(cudaMalloc(&T.Thi, hi_elems * T.esz));
    CK(cudaMalloc(&T.Tlo, std::max<size_t>(lo_elems, 1) * T.esz));
    T.split = n_lo > 0 ? 1 : 0;
    T.op_scale = 1.0;
    T.modal = (ctx->opt.m2l_basis == 1 && !T.svd) ? 1 : 0;
    if (T.modal && !basis_matrices(p, T.basisV, T.basisCt))
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "m2l setup: singular Legendre basis matrix");
    const size_t sm_modal = size_t(2) * 9 * P3 * sizeof(double);
    if (T.modal) {
        CK(cudaFuncSetAttribute(k_build_ops_modal<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_modal)));
        CK(cudaFuncSetAttribute(k_build_ops_modal<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_modal)));
        CK(cudaFuncSetAttribute(k_build_ops_modal<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(sm_modal)));
        CK(cudaFuncSetAttribute(k_w_modal<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_modal)));
        CK(cudaFuncSetAttribute(k_w_modal<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_modal / 2)));
    }
    const BasisMats B = basis_of(T, p);
    if (T.svd) {
        // U^T T_o R for every offset (FP64), with the FP16 scale from their largest entry
        if (int rc = svd_operators(ctx, d_off, d_lo, T.n_off)) {
            cudaFree(d_off);
            cudaFree(d_lo);
            return rc;
        }
        if (T.fp16 && !T.d_wmax) CK(cudaMalloc(&T.d_wmax, GB_TC_MAXLEV * sizeof(unsigned)));
    } else if (T.fp16 && T.modal) {
        // one power of two for all operators from the largest modal entry
        unsigned long long *d_mx = nullptr, mx_bits = 0;
        CK(cudaMalloc(&d_mx, sizeof(unsigned long long)));
        CK(cudaMemsetAsync(d_mx, 0, sizeof(unsigned long long), ctx->stream));
        ++ctx->launches;
        k_build_ops_modal<__half><<<unsigned(T.n_off * T.Np), 256, sm_modal, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off, d_lo, 1.0, B, 0, d_mx, (__half *)nullptr, (__half *)nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&mx_bits, d_mx, sizeof(mx_bits), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(d_mx);
        double mx = 0.0;
        std::memcpy(&mx, &mx_bits, sizeof(mx));
        if (mx > 0.0) {
            int e = 0;
            std::frexp(mx, &e);
            T.op_scale = std::ldexp(1.0, 14 - e);
        }
        if (!T.d_wmax) CK(cudaMalloc(&T.d_wmax, GB_TC_MAXLEV * sizeof(unsigned)));
    } else if (T.fp16) {
        // one power of two for all operators: the largest lattice value maps below 2^14
        unsigned long long *d_mx = nullptr, mx_bits = 0;
        CK(cudaMalloc(&d_mx, sizeof(unsigned long long)));
        CK(cudaMemsetAsync(d_mx, 0, sizeof(unsigned long long), ctx->stream));
        const int64_t n_pts = int64_t(ctx->lat_n) * ctx->lat_n * ctx->lat_n;
        const int64_t origin = n_pts / 2;  // lattice centre, D = 0
        ++ctx->launches;
        k_lattice_absmax<<<1024, 256, 0, ctx->stream>>>(n_pts, origin, ctx->d_Klat, d_mx);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&mx_bits, d_mx, sizeof(mx_bits), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(d_mx);
        double mx = 0.0;
        std::memcpy(&mx, &mx_bits, sizeof(mx));
        if (mx > 0.0) {
            int e = 0;
            std::frexp(mx, &e);
            T.op_scale = std::ldexp(1.0, 14 - e);
        }
        if (!T.d_wmax) CK(cudaMalloc(&T.d_wmax, GB_TC_MAXLEV * sizeof(unsigned)));
    }
    if (!T.svd) ++ctx->launches;
    if (T.svd) {
        // written by svd_operators
    } else if (T.modal) {
        const unsigned g = unsigned(T.n_off * T.Np);
        if (T.tf32)
            k_build_ops_modal<float><<<g, 256, sm_modal, ctx->stream>>>(p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off,
                                                                        d_lo, 1.0, B, 1, nullptr, (float *)T.Thi,
                                                                        (float *)nullptr);
        else if (T.fp16)
            k_build_ops_modal<__half><<<g, 256, sm_modal, ctx->stream>>>(p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off,
                                                                         d_lo, T.op_scale, B, 1, nullptr,
                                                                         (__half *)T.Thi, (__half *)T.Tlo);
        else
            k_build_ops_modal<__nv_bfloat16><<<g, 256, sm_modal, ctx->stream>>>(
                p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off, d_lo, 1.0, B, 1, nullptr, (__nv_bfloat16 *)T.Thi,
                (__nv_bfloat16 *)T.Tlo);
    } else if (T.tf32)
        k_build_ops<float><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off, d_lo, T.n_off, 1.0, (float *)T.Thi, (float *)nullptr);
    else if (T.fp16)
        k_build_ops<__half><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off, d_lo, T.n_off, T.op_scale, (__half *)T.Thi,
            (__half *)T.Tlo);
    else
        k_build_ops<__nv_bfloat16><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, T.Kp_lo, ctx->d_Klat, d_off, d_lo, T.n_off, 1.0, (__nv_bfloat16 *)T.Thi,
            (__nv_bfloat16 *)T.Tlo);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(d_off);
    cudaFree(d_lo);
    if (!T.d_status) CK(cudaMalloc(&T.d_status, sizeof(int)));
    CK(cudaMemset(T.d_status, 0, sizeof(int)));
    T.ready_ops = true;
    return GBFMM_OK;
}

static int encode(gbfmm_ctx *ctx, CUtensorMap *tm, void *base, int rank, const cuuint64_t *dims,
                  const cuuint64_t *strides, const cuuint32_t *boxd, const TcPlan &T) {
    EncodeTiled enc = get_encoder();
    if (!enc) return set_err(ctx, GBFMM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUtensorMapDataType dt = T.tf32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : T.fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(tm, dt, cuuint32_t(rank),
                     base, dims, strides, boxd, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, GBFMM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(r));
    return GBFMM_OK;
}

// Per-tree buffers: packed W (hi / lo), tensor maps, work list.
int m2l_tc_prepare(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    const int L = ctx->L;
    if (L - 1 >= GB_TC_MAXLEV) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "tensor-core M2L: too many levels");
    int64_t tot = 0;
    for (int l = 2; l < L; ++l) {
        T.wofs[l] = tot;
        tot += (int64_t(1) << (3 * l)) * T.Kp;
    }
    if (int rc = grow_dev(ctx, T.w_cap, tot, {{&T.Whi, size_t(tot) * T.esz}, {&T.Wlo, size_t(tot) * T.esz}},
                          "packed multipole values"))
        return rc;
    // cell slots, target list and segment table (filled on the device per pass)
    const int64_t slots = slot_base(L);
    int64_t tiles = 0;  // CTAs per operator group, upper bound: every cell holds targets
    for (int l = 2; l < L; ++l) tiles += 8 * ((((int64_t(1) << (3 * (l - 1))) + 127) / 128 + T.tpc - 1) / T.tpc);
    if (int rc = grow_dev(ctx, T.slot_cap, slots,
                          {{(void **)&T.d_flags, slots * sizeof(int)}, {(void **)&T.d_pos, (slots + 1) * sizeof(int)},
                           {(void **)&T.d_list, slots * sizeof(int)}},
                          "M2L target lists"))
        return rc;
    if (!T.d_seg) CK(cudaMalloc(&T.d_seg, (kMaxSeg + 1) * sizeof(int4)));
    T.n_slots = slots;
    T.n_seg = 8 * (L - 2);
    T.n_work = int(tiles * T.groups);
    if (T.svd) return svd_prepare(ctx);
    return GBFMM_OK;
}

int m2l_tc_run(gbfmm_ctx *ctx, const float *Wf, const double *W64, const int *occ, const int *tocc, float *Sf,
               double *S64, bool fine) {
    TcPlan &T = ctx->tc;
    // fine: the adaptive tree's children (level ctx->L) take part through fine_m2l, after the
    // tensor-core M2L of levels 2 .. L-1
    const int L = ctx->L, p = ctx->opt.p, P3 = p * p * p;
    M2LParams prm;  // copied by value into the launch (kernel parameter space)
    std::memset(&prm, 0, sizeof(prm));
    if (T.fp16) CK(cudaMemsetAsync(T.d_wmax, 0, GB_TC_MAXLEV * sizeof(unsigned), ctx->stream));
    const BasisMats B = basis_of(T, p);
    const int split_levels = ctx->opt.m2l_split_levels ? ctx->opt.m2l_split_levels : ~0;
    // compressed M2L: every cell's multipole values -> r2 coefficients R^T W first
    if (T.svd)
        if (int rc = svd_transform_w(ctx, Wf, fine)) return rc;
    const float *Wsrc = T.svd ? T.Wc : Wf;
    const int kv = T.svd ? T.r2 : 9 * P3;  // valid values per cell row
    for (int l = 2; l < L; ++l) {
        const bool split_l = T.split && ((split_levels >> l) & 1);  // residual W only where it is read
        const int64_t cells_l = int64_t(1) << (3 * l);
        void *whi = (char *)T.Whi + T.wofs[l] * T.esz, *wlo = (char *)T.Wlo + T.wofs[l] * T.esz;
        const unsigned gb = unsigned(std::min<int64_t>(cells_l, 8 * 152));  // blocks stride over the cells
        if (T.modal && !T.svd) {
            // node values -> Legendre moments (in place: nothing reads these W after the M2L)
            ++ctx->launches;
            if (W64)
                k_w_modal<double><<<gb, 256, size_t(2) * 9 * P3 * sizeof(double), ctx->stream>>>(
                    l, p, B, const_cast<double *>(W64), occ);
            else
                k_w_modal<float><<<gb, 256, size_t(2) * 9 * P3 * sizeof(float), ctx->stream>>>(
                    l, p, B, const_cast<float *>(Wf), occ);
        }
        if (T.tf32) {
            ++ctx->launches;
            if (W64)
                k_pack_w<float><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, W64, occ, nullptr, (float *)whi, (float *)nullptr);
            else
                k_pack_w<float><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, Wsrc, occ, nullptr, (float *)whi, (float *)nullptr);
        } else if (T.fp16) {
            const unsigned gm = gb;
            __half *lo = split_l ? (__half *)wlo : nullptr;
            ctx->launches += 2;
            if (W64) {
                k_wmax<<<gm, 256, 0, ctx->stream>>>(l, kv, W64, occ, T.d_wmax);
                k_pack_w<__half><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, W64, occ, T.d_wmax, (__half *)whi, lo);
            } else {
                k_wmax<<<gm, 256, 0, ctx->stream>>>(l, kv, Wsrc, occ, T.d_wmax);
                k_pack_w<__half><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, Wsrc, occ, T.d_wmax, (__half *)whi, lo);
            }
        } else {
            __nv_bfloat16 *lo = split_l ? (__nv_bfloat16 *)wlo : nullptr;
            ++ctx->launches;
            if (W64)
                k_pack_w<__nv_bfloat16><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, W64, occ, nullptr,
                                                                     (__nv_bfloat16 *)whi, lo);
            else
                k_pack_w<__nv_bfloat16><<<gb, 256, 0, ctx->stream>>>(l, kv, T.Kp, Wsrc, occ, nullptr,
                                                                     (__nv_bfloat16 *)whi, lo);
        }
        prm.wofs[l] = T.wofs[l] * T.esz;
    }
    prm.Whi = static_cast<const uint8_t *>(T.Whi);
    prm.Wlo = static_cast<const uint8_t *>(T.Wlo);
    prm.row_bytes = T.Kp * T.esz;
    for (int l = 2; l < L; ++l) {
        ++ctx->launches;
        k_mb_flags<<<nblk(int64_t(1) << (3 * l), 256), 256, 0, ctx->stream>>>(l, tocc, T.d_flags);
    }
    ctx->launches += 3;
    k_scan_flags<<<1, 1024, 0, ctx->stream>>>(int(T.n_slots), T.d_flags, T.d_pos);
    k_mb_list<<<nblk(T.n_slots, 256), 256, 0, ctx->stream>>>(int(T.n_slots), L, T.d_flags, T.d_pos, T.d_list);
    k_seg_table<<<1, 32, 0, ctx->stream>>>(L, T.tpc, T.d_pos, T.d_seg);
    {
        const cuuint64_t dims[3] = {cuuint64_t(T.Kp), cuuint64_t(T.Np), cuuint64_t(T.n_off)};
        const cuuint64_t strides[2] = {cuuint64_t(T.Kp) * T.esz, cuuint64_t(T.Kp) * T.esz * T.Np};
        // box: one K block of operator rows: nsub rows (cells as A) or a 128-row block (operators as A)
        const cuuint32_t boxd[3] = {cuuint32_t(128 / T.esz), cuuint32_t(T.swap ? 128 : T.nsub), 1};
        int rc = encode(ctx, &prm.tmT, T.Thi, 3, dims, strides, boxd, T);
        if (rc) return rc;
        const cuuint64_t dl[3] = {cuuint64_t(T.Kp_lo), cuuint64_t(T.Np), cuuint64_t(std::max(T.n_lo, 1))};
        const cuuint64_t sl[2] = {cuuint64_t(T.Kp_lo) * T.esz, cuuint64_t(T.Kp_lo) * T.esz * T.Np};
        rc = encode(ctx, &prm.tmTlo, T.Tlo, 3, dl, sl, boxd, T);
        if (rc) return rc;
    }
    prm.kstep = 128 / T.esz;
    prm.kb = T.Kp / prm.kstep;
    prm.kb_res = ctx->opt.m2l_split_kblocks > 0 ? std::min(prm.kb, ctx->opt.m2l_split_kblocks) : prm.kb;
    prm.idesc = idesc_of(128, T.nsub, T.tf32, T.fp16);  // M = 128; N = nsub, or 256 cells (operators as A)
    prm.nblk = T.nblk;
    prm.wmax = T.fp16 ? T.d_wmax : nullptr;
    prm.inv_op_scale = float(1.0 / T.op_scale);
    prm.nsub = T.nsub;
    prm.ncta = T.ncta;
    prm.nvalid = T.svd ? T.r1 : 6 * P3;
    prm.tmem_cols = T.tmem_cols;
    prm.split = T.split;
    prm.split_levels = split_levels;
    prm.drop_first = T.inject_drop;
    T.inject_drop = 0;
    const int stage_bytes = T.tpc * kTileA + (T.swap ? 2 * kTileA : T.ncta * 128);
    // as many stages as fit in the shared memory a block may opt into, next to the
    // kernel's static arrays, the 1 KB alignment pad and the barriers
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto kern = T.tf32 ? (T.swap ? k_m2l_tc<true, true> : k_m2l_tc<true, false>)
                       : (T.swap ? k_m2l_tc<false, true> : k_m2l_tc<false, false>);
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, kern));
    const int64_t room = int64_t(optin) - int64_t(fa.sharedSizeBytes) - 1024 - (2 * 6 + 2) * 8 - 64;
    const int stages = int(std::min<int64_t>(6, room / stage_bytes));
    if (stages < 2) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "tensor-core M2L: operator block too large");
    const size_t smem = size_t(stages) * stage_bytes + 1024 + (2 * stages + 2) * 8 + 64;
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    // offset chunks: each launch accumulates a run of consecutive offsets of every class's list
    // in tensor memory; the chunks' sums are added outside the tensor cores, in the local values
    const int chunks = std::max(1, std::min(189, ctx->opt.m2l_chunks));
    float *Sout = T.svd ? T.Sc : Sf;  // compressed: the r1 coefficients of every target cell
    if (T.svd) CK(cudaMemsetAsync(T.Sc, 0, size_t(ctx->n_cells) * T.r1 * sizeof(float), ctx->stream));
    for (int c = 0; c < chunks; ++c) {
        prm.o_lo = (189 * c) / chunks;
        prm.o_hi = (189 * (c + 1)) / chunks;
        prm.accumulate = c > 0 ? 1 : 0;
        if (c > 0) prm.drop_first = 0;
        ++ctx->launches;
        kern<<<T.n_work, 192, smem, ctx->stream>>>(prm, T.d_seg, 8 * (L - 2), T.d_list, occ, tocc, ctx->d_box, Sout,
                                                   S64, T.d_status, stages, T.groups);
        CK(cudaGetLastError());
    }
    if (T.svd) {
        if (fine)
            if (int rc = fine_m2l(ctx)) return rc;
        return svd_expand_s(ctx, Sf, fine);  // S = U S'
    }
    return GBFMM_OK;
}

// read and clear the device status word of the tensor-core M2L
int m2l_tc_status(gbfmm_ctx *ctx, int *out) {
    *out = 0;
    if (!ctx->tc.d_status) return GBFMM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(out, ctx->tc.d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->tc.d_status, 0, sizeof(int)));
    return GBFMM_OK;
}

void m2l_tc_free(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    svd_free(ctx, ctx->borrowed_material);
    void *ps[] = {T.Thi, T.Tlo, T.Whi, T.Wlo, T.d_status, T.d_flags, T.d_pos, T.d_list, T.d_seg, T.d_wmax};
    for (void *q : ps)
        if (q) cudaFree(q);
    T = TcPlan{};
}
