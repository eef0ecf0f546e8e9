// M2L on the tcgen05 tensor cores: offset-grouped dense GEMMs (Sec. 4.1,
// Eq. "m2l"; Algorithm 2 step 2) in BF16 with FP32 accumulation in TMEM.
//
// Formulation.  At level l the cells form a 2^l grid.  Split it into the 8
// parity classes c = (x & 1, y & 1, z & 1); each class is an m^3 sub-grid,
// m = 2^(l-1).  For a target cell B = 2P + c and an offset o in its
// interaction list, the source A = B - o lies in class c' = (c - o) mod 2 at
// sub-grid position P + s, s = floor((c - o) / 2) in [-1, 1]^3.  The 189
// offsets of class c are therefore, each, a constant shift between two
// sub-grids, and the M2L of a brick of 128 target cells (8 x 4 x 4 in the
// sub-grid) is
//     S[brick, n] = (2^l / H)^2  sum_o  sum_k  W_c'[brick + s_o, k] T_o[n, k]
// with k = (node m, component wr) and n = (node l, stress component ab):
// one GEMM of M = 128 cells, N = 6 p^3 and K = 189 x 9 p^3, accumulated in
// tensor memory.  The A tile (shifted brick of multipole weights) and the
// B tile (rows of the operator T_o) are both plain TMA box loads; boxes that
// stick out of the sub-grid are zero-filled by the TMA unit.
//
// Precision: W and T_o are rounded to BF16 (hi).  For the offsets nearest
// to the target (max |o_i| = 2, the largest far-field terms) the residuals
// W_lo = W - hi(W) and T_lo = T - hi(T) add two more passes,
// hi*hi + lo*hi + hi*lo, which restores ~FP32 accuracy where it matters.
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and
// issues the MMAs, warps 2-5 read the accumulator out (warp w reads TMEM
// lanes 32 (w % 4) .. 32 (w % 4) + 31).  Every mbarrier wait is bounded;
// on time-out a device status word gets GBFMM_ERR_TIMEOUT and the block
// winds down, freeing its tensor memory.
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
    CUtensorMap tmW[GB_TC_MAXLEV];    // W hi per level: (Kp, m, m, m, 8) bf16
    CUtensorMap tmWlo[GB_TC_MAXLEV];  // W residual per level
    CUtensorMap tmT;                  // T hi: (Kp, Np, 316)
    CUtensorMap tmTlo;                // T residual: (Kp, Np, n_lo)
    int kb;         // K blocks of 64
    int nsub;       // N per MMA (multiple of 16, <= 256)
    int ncta;       // 3 * nsub
    int nvalid;     // 6 p^3
    int tmem_cols;  // power of two >= ncta
    int split;      // residual passes on the near offsets
    int drop_first; // failure-detection test: arm the first stage but issue no load into it
    int kstep;      // operand elements per 128-byte row: 64 (bf16, fp16) or 32 (tf32)
    uint32_t idesc; // tcgen05 instruction descriptor
    const unsigned *wmax;  // FP16 mode: per-level max |W| bits (the W scale), else null
    float inv_op_scale;    // FP16 mode: 1 / operator scale, else 1
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

constexpr int kStageA = 128 * 64 * 2;  // 16 KB

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

// Is any cell of the shifted source box occupied?  Brick flags are per level,
// class and aligned 8 x 4 x 4 brick of the sub-grid; the box of a shift in
// [-1, 1]^3 overlaps at most 2 x 2 x 2 aligned bricks.
__device__ __forceinline__ bool source_occupied(const unsigned char *__restrict__ bocc, int m, int bx0, int by0,
                                                int bz0, const OffsetEntry &e) {
    const int nbx = (m + 7) / 8, nby = (m + 3) / 4, nbz = (m + 3) / 4;
    const int x0 = bx0 + e.sx, y0 = by0 + e.sy, z0 = bz0 + e.sz;
    const int ax0 = max(x0, 0) / 8, ax1 = min(x0 + 7, m - 1) / 8;
    const int ay0 = max(y0, 0) / 4, ay1 = min(y0 + 3, m - 1) / 4;
    const int az0 = max(z0, 0) / 4, az1 = min(z0 + 3, m - 1) / 4;
    if (x0 + 7 < 0 || y0 + 3 < 0 || z0 + 3 < 0 || x0 >= m || y0 >= m || z0 >= m) return false;
    for (int bz = az0; bz <= az1; ++bz)
        for (int by = ay0; by <= ay1; ++by)
            for (int bx = ax0; bx <= ax1; ++bx)
                if (bocc[((int64_t(e.cls) * nbz + bz) * nby + by) * nbx + bx]) return true;
    return false;
}

// number of K-block iterations of one work item (same count on every warp)
__device__ __forceinline__ int passes_of(const OffsetEntry &e, int split) { return (split && e.lo >= 0) ? 3 : 1; }

template <bool TF32>
__global__ void __launch_bounds__(192, 1)
    k_m2l_tc(const __grid_constant__ M2LParams P, const int4 *__restrict__ work, const int *__restrict__ tocc,
             const unsigned char *__restrict__ bocc_all, const int64_t *__restrict__ bocc_ofs,
             const TreeBox *__restrict__ box, float *__restrict__ S, int *__restrict__ status, int stages) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int stageB = P.ncta * 128;
    const int stage_bytes = kStageA + stageB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + stages * stage_bytes);
    // bars[0..stages): full, [stages..2 stages): empty, [2 stages]: accumulator ready
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 1);

    const int4 w = work[blockIdx.x];
    const int level = w.x, cls = w.y, brick = w.z, group = w.w;
    const int m = 1 << (level - 1), n = 1 << level;
    const int nbx = (m + 7) / 8, nby = (m + 3) / 4;
    const int bx0 = (brick % nbx) * 8, by0 = ((brick / nbx) % nby) * 4, bz0 = (brick / (nbx * nby)) * 4;
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;
    const unsigned char *bocc = bocc_all + bocc_ofs[level];

    // skip bricks without targets, and do no work once an earlier block's
    // time-out is flagged (both decided once for the whole block)
    {
        __shared__ int any, stop;
        if (threadIdx.x == 0) {
            any = 0;
            stop = *reinterpret_cast<volatile int *>(status) != 0;
        }
        __syncthreads();
        if (threadIdx.x < 128) {
            const int rx = threadIdx.x % 8, ry = (threadIdx.x / 8) % 4, rz = threadIdx.x / 32;
            const int px = bx0 + rx, py = by0 + ry, pz = bz0 + rz;
            if (px < m && py < m && pz < m) {
                const int64_t g = cell_base_d(level) + (int64_t(2 * pz + cz) * n + (2 * py + cy)) * n + (2 * px + cx);
                if (tocc[g] > 0) any = 1;
            }
        }
        __syncthreads();
        if (!any || stop) return;
    }

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * stages + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
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
        // ---------------- TMA producer
        int it = 0;
        bool ok = true;
        for (int oi = 0; oi < 189 && ok; ++oi) {
            const OffsetEntry e = c_offs[cls][oi];
            if (!source_occupied(bocc, m, bx0, by0, bz0, e)) continue;
            const int np = passes_of(e, P.split);
            for (int pass = 0; pass < np && ok; ++pass) {
                const CUtensorMap *ta = (pass == 1) ? &P.tmWlo[level] : &P.tmW[level];
                const CUtensorMap *tb = (pass == 2) ? &P.tmTlo : &P.tmT;
                const int tidx = (pass == 2) ? e.lo : e.top;
                for (int kb = 0; kb < P.kb; ++kb, ++it) {
                    const int s = it % stages;
                    const uint32_t ph = (it / stages) & 1;
                    if (!mbar_wait(empty0 + 8 * s, ph ^ 1, status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * s;
                    mbar_expect_tx(fb, kStageA + stageB);
                    if (P.drop_first && it == 0) continue;  // the MMA warp's wait on this stage runs out
                    const uint32_t a = smem0 + s * stage_bytes;
                    tma_load_5d(a, ta, kb * P.kstep, bx0 + e.sx, by0 + e.sy, bz0 + e.sz, e.cls, fb);
                    for (int j = 0; j < 3; ++j)
                        tma_load_3d(a + kStageA + j * P.nsub * 128, tb, kb * P.kstep, group * P.ncta + j * P.nsub,
                                    tidx, fb);
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = P.idesc;
        int it = 0;
        bool ok = true;
        for (int oi = 0; oi < 189 && ok; ++oi) {
            const OffsetEntry e = c_offs[cls][oi];
            if (!source_occupied(bocc, m, bx0, by0, bz0, e)) continue;
            const int np = passes_of(e, P.split);
            for (int pass = 0; pass < np && ok; ++pass) {
                for (int kb = 0; kb < P.kb; ++kb, ++it) {
                    const int s = it % stages;
                    const uint32_t ph = (it / stages) & 1;
                    if (!mbar_wait(full0 + 8 * s, ph, status)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a = smem0 + s * stage_bytes;
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = sw128_desc(a + kk * 32);
                        for (int j = 0; j < 3; ++j) {
                            const uint64_t bd = sw128_desc(a + kStageA + j * P.nsub * 128 + kk * 32);
                            mma_issue<TF32>(tmem + j * P.nsub, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(empty0 + 8 * s);
                }
            }
        }
        mma_commit(accb);  // fires when every MMA issued above has completed
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> scaled FP32 local values
        bool any_src = false;
        for (int oi = 0; oi < 189 && !any_src; ++oi) any_src = source_occupied(bocc, m, bx0, by0, bz0, c_offs[cls][oi]);
        const bool ok = mbar_wait(accb, 0, status);
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int q = warp % 4;
        const int row = q * 32 + lane;
        const int rx = row % 8, ry = (row / 8) % 4, rz = row / 32;
        const int px = bx0 + rx, py = by0 + ry, pz = bz0 + rz;
        const bool valid = ok && px < m && py < m && pz < m;
        const int64_t g = cell_base_d(level) + (int64_t(2 * pz + cz) * n + (2 * py + cy)) * n + (2 * px + cx);
        float sc = float(double(n) / box->H) * float(double(n) / box->H);
        if (P.wmax) sc *= P.inv_op_scale / wscale_of(P.wmax[level]);
        float *dst = S + g * int64_t(P.nvalid);
        if (ok && !any_src) {
            // no occupied source anywhere in the interaction list: zero local values
            if (valid)
                for (int col = group * P.ncta; col < min(P.nvalid, (group + 1) * P.ncta); ++col) dst[col] = 0.f;
        } else if (ok) {
            for (int j = 0; j < 3; ++j)
                for (int c0 = 0; c0 < P.nsub; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + (uint32_t(q * 32) << 16) + uint32_t(j * P.nsub + c0), v);
                    const int col = group * P.ncta + j * P.nsub + c0;
                    if (valid)
                        for (int i = 0; i < 16; ++i)
                            if (col + i < P.nvalid) dst[col + i] = v[i] * sc;
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
__global__ void k_build_ops(int p, int lat_n, int Np, int Kp, const double *__restrict__ Klat,
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
        if (li >= 0 && Tlo) Tlo[(int64_t(li) * Np + nn) * Kp + k] = to_elem<E>(v - elem_value(hi));
    }
}

// W (FP32, [cell][p^3 * 9]) -> parity-split BF16 hi / lo, [class][mz][my][mx][Kp] per level
template <typename E>
__global__ void k_pack_w(int level, int P3, int Kp, const float *__restrict__ W, const int *__restrict__ occ,
                         const unsigned *__restrict__ wmax, E *__restrict__ hi, E *__restrict__ lo) {
    const int n = 1 << level, m = n / 2;
    const double s = wmax ? double(wscale_of(wmax[level])) : 1.0;
    const int64_t cells = int64_t(n) * n * n;
    const int64_t total = cells * Kp;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(idx % Kp);
        const int64_t lin = idx / Kp;
        const int x = int(lin % n), y = int((lin / n) % n), z = int(lin / (int64_t(n) * n));
        const int cls = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        const int64_t dst = ((((int64_t(cls) * m + z / 2) * m + y / 2) * m + x / 2) * Kp) + k;
        const int64_t g = cell_base_d(level) + lin;
        float v = 0.f;
        if (k < 9 * P3 && occ[g] > 0) v = W[g * 9 * P3 + k];
        const double vs = s * double(v);
        const E h = to_elem<E>(vs);
        hi[dst] = h;
        if (lo) lo[dst] = to_elem<E>(vs - elem_value(h));
    }
}

// largest |W| over the occupied cells of one level (non-negative floats order
// like their bit patterns)
__global__ void k_wmax(int level, int P3, const float *__restrict__ W, const int *__restrict__ occ,
                       unsigned *__restrict__ wmax) {
    const int64_t cells = int64_t(1) << (3 * level), base = cell_base_d(level);
    const int64_t total = cells * 9 * P3;
    float mx = 0.f;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = base + idx / (9 * P3);
        if (occ[g] > 0) mx = fmaxf(mx, fabsf(W[base * 9 * P3 + idx]));
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

// brick flags: one byte per (class, aligned 8 x 4 x 4 brick) of a level
__global__ void k_brick_occ(int level, const int *__restrict__ occ, unsigned char *__restrict__ bocc) {
    const int n = 1 << level, m = n / 2;
    const int nbx = (m + 7) / 8, nby = (m + 3) / 4, nbz = (m + 3) / 4;
    const int64_t cells = int64_t(n) * n * n;
    for (int64_t lin = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; lin < cells;
         lin += int64_t(gridDim.x) * blockDim.x) {
        if (occ[cell_base_d(level) + lin] == 0) continue;
        const int x = int(lin % n), y = int((lin / n) % n), z = int(lin / (int64_t(n) * n));
        const int cls = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        bocc[((int64_t(cls) * nbz + (z / 2) / 4) * nby + (y / 2) / 4) * nbx + (x / 2) / 8] = 1;
    }
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

// Offsets, their parity-class lists and the operator tables.
int m2l_tc_setup(gbfmm_ctx *ctx) {
    const int p = ctx->opt.p, P3 = p * p * p;
    TcPlan &T = ctx->tc;
    T.tf32 = ctx->opt.m2l_split == 3 ? 1 : 0;
    T.fp16 = (ctx->opt.m2l_split == 4 || ctx->opt.m2l_split == 5) ? 1 : 0;
    T.esz = T.tf32 ? 4 : 2;
    T.Kp = ((9 * P3 + 63) / 64) * 64;
    // N per MMA: multiple of 16, three of them per block, 3 nsub <= 512 TMEM columns
    const int nv = 6 * P3;
    int best = 0, best_waste = 1 << 30;
    for (int ns = 16; ns <= 160; ns += 16) {
        const int g = (nv + 3 * ns - 1) / (3 * ns);
        const int waste = g * 3 * ns - nv + g * 64;  // padding plus a per-group cost
        if (waste < best_waste) {
            best_waste = waste;
            best = ns;
        }
    }
    T.nsub = best;
    T.ncta = 3 * best;
    T.groups = (nv + T.ncta - 1) / T.ncta;
    T.Np = T.groups * T.ncta;
    T.tmem_cols = 32;
    while (T.tmem_cols < T.ncta) T.tmem_cols *= 2;
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
                const bool split = !T.tf32 && (sm == 2 || ((sm == 0 || sm == 5) && mx == 2));
                lo_of.push_back(split ? n_lo++ : -1);
            }
    T.n_off = int(off.size() / 3);
    T.n_lo = n_lo;
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
    const size_t hi_elems = size_t(T.n_off) * T.Np * T.Kp, lo_elems = size_t(T.n_lo) * T.Np * T.Kp;
    if (T.Thi) cudaFree(T.Thi);
    if (T.Tlo) cudaFree(T.Tlo);
    T.Thi = T.Tlo = nullptr;
    CK(cudaMalloc(&T.Thi, hi_elems * T.esz));
    CK(cudaMalloc(&T.Tlo, std::max<size_t>(lo_elems, 1) * T.esz));
    T.split = n_lo > 0 ? 1 : 0;
    T.op_scale = 1.0;
    if (T.fp16) {
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
    ++ctx->launches;
    if (T.tf32)
        k_build_ops<float><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, ctx->d_Klat, d_off, d_lo, T.n_off, 1.0, (float *)T.Thi, (float *)nullptr);
    else if (T.fp16)
        k_build_ops<__half><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, ctx->d_Klat, d_off, d_lo, T.n_off, T.op_scale, (__half *)T.Thi,
            (__half *)T.Tlo);
    else
        k_build_ops<__nv_bfloat16><<<nblk(int64_t(hi_elems), 256), 256, 0, ctx->stream>>>(
            p, ctx->lat_n, T.Np, T.Kp, ctx->d_Klat, d_off, d_lo, T.n_off, 1.0, (__nv_bfloat16 *)T.Thi,
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
    if (tot > T.w_cap) {
        if (T.Whi) cudaFree(T.Whi);
        if (T.Wlo) cudaFree(T.Wlo);
        T.Whi = T.Wlo = nullptr;
        CK(cudaMalloc(&T.Whi, tot * T.esz));
        CK(cudaMalloc(&T.Wlo, tot * T.esz));
        T.w_cap = tot;
    }
    int64_t bocc_tot = 0;
    std::vector<int64_t> bofs(GB_TC_MAXLEV, 0);
    for (int l = 2; l < L; ++l) {
        const int m = 1 << (l - 1);
        bofs[l] = bocc_tot;
        bocc_tot += int64_t(8) * ((m + 7) / 8) * ((m + 3) / 4) * ((m + 3) / 4);
    }
    if (bocc_tot > T.bocc_cap) {
        if (T.d_bocc) cudaFree(T.d_bocc);
        T.d_bocc = nullptr;
        CK(cudaMalloc(&T.d_bocc, bocc_tot));
        T.bocc_cap = bocc_tot;
    }
    T.bocc_tot = bocc_tot;
    for (int l = 0; l < GB_TC_MAXLEV; ++l) T.bocc_h[l] = bofs[l];
    if (!T.d_bocc_ofs) CK(cudaMalloc(&T.d_bocc_ofs, GB_TC_MAXLEV * sizeof(int64_t)));
    CK(cudaMemcpy(T.d_bocc_ofs, bofs.data(), GB_TC_MAXLEV * sizeof(int64_t), cudaMemcpyHostToDevice));
    std::vector<int4> wl;
    for (int l = 2; l < L; ++l) {
        const int m = 1 << (l - 1);
        const int nb = ((m + 7) / 8) * ((m + 3) / 4) * ((m + 3) / 4);
        for (int c = 0; c < 8; ++c)
            for (int b = 0; b < nb; ++b)
                for (int g = 0; g < T.groups; ++g) wl.push_back(make_int4(l, c, b, g));
    }
    T.n_work = int(wl.size());
    if (T.n_work > T.work_cap) {
        if (T.d_work) cudaFree(T.d_work);
        T.d_work = nullptr;
        CK(cudaMalloc(&T.d_work, wl.size() * sizeof(int4)));
        T.work_cap = T.n_work;
    }
    CK(cudaMemcpy(T.d_work, wl.data(), wl.size() * sizeof(int4), cudaMemcpyHostToDevice));
    return GBFMM_OK;
}

int m2l_tc_run(gbfmm_ctx *ctx, const float *Wf, const int *occ, const int *tocc, float *Sf) {
    TcPlan &T = ctx->tc;
    const int L = ctx->L, p = ctx->opt.p, P3 = p * p * p;
    static M2LParams prm;  // large: build on the heap-like static, copied by value at launch
    std::memset(&prm, 0, sizeof(prm));
    if (T.fp16) CK(cudaMemsetAsync(T.d_wmax, 0, GB_TC_MAXLEV * sizeof(unsigned), ctx->stream));
    for (int l = 2; l < L; ++l) {
        const int m = 1 << (l - 1);
        const int64_t el = (int64_t(1) << (3 * l)) * T.Kp;
        void *whi = (char *)T.Whi + T.wofs[l] * T.esz, *wlo = (char *)T.Wlo + T.wofs[l] * T.esz;
        if (T.tf32) {
            ++ctx->launches;
            k_pack_w<float><<<nblk(el, 256), 256, 0, ctx->stream>>>(l, P3, T.Kp, Wf, occ, nullptr, (float *)whi,
                                                                    (float *)nullptr);
        } else if (T.fp16) {
            const int64_t vals = (int64_t(1) << (3 * l)) * 9 * P3;
            ctx->launches += 2;
            k_wmax<<<unsigned(std::min<int64_t>(nblk(vals, 256), 4 * 152)), 256, 0, ctx->stream>>>(l, P3, Wf, occ,
                                                                                                   T.d_wmax);
            k_pack_w<__half><<<nblk(el, 256), 256, 0, ctx->stream>>>(l, P3, T.Kp, Wf, occ, T.d_wmax, (__half *)whi,
                                                                     (__half *)wlo);
        } else {
            ++ctx->launches;
            k_pack_w<__nv_bfloat16><<<nblk(el, 256), 256, 0, ctx->stream>>>(l, P3, T.Kp, Wf, occ, nullptr,
                                                                             (__nv_bfloat16 *)whi, (__nv_bfloat16 *)wlo);
        }
        const cuuint64_t dims[5] = {cuuint64_t(T.Kp), cuuint64_t(m), cuuint64_t(m), cuuint64_t(m), 8};
        const cuuint64_t row = cuuint64_t(T.Kp) * T.esz;
        const cuuint64_t strides[4] = {row, row * m, row * m * m, row * m * m * m};
        const cuuint32_t boxd[5] = {cuuint32_t(128 / T.esz), 8, 4, 4, 1};
        int rc = encode(ctx, &prm.tmW[l], whi, 5, dims, strides, boxd, T);
        if (rc) return rc;
        rc = encode(ctx, &prm.tmWlo[l], wlo, 5, dims, strides, boxd, T);
        if (rc) return rc;
    }
    CK(cudaMemsetAsync(T.d_bocc, 0, T.bocc_tot, ctx->stream));
    for (int l = 2; l < L; ++l) {
        ++ctx->launches;
        k_brick_occ<<<nblk(int64_t(1) << (3 * l), 256), 256, 0, ctx->stream>>>(l, occ, T.d_bocc + T.bocc_h[l]);
    }
    {
        const cuuint64_t dims[3] = {cuuint64_t(T.Kp), cuuint64_t(T.Np), cuuint64_t(T.n_off)};
        const cuuint64_t strides[2] = {cuuint64_t(T.Kp) * T.esz, cuuint64_t(T.Kp) * T.esz * T.Np};
        const cuuint32_t boxd[3] = {cuuint32_t(128 / T.esz), cuuint32_t(T.nsub), 1};
        int rc = encode(ctx, &prm.tmT, T.Thi, 3, dims, strides, boxd, T);
        if (rc) return rc;
        const cuuint64_t dl[3] = {cuuint64_t(T.Kp), cuuint64_t(T.Np), cuuint64_t(std::max(T.n_lo, 1))};
        rc = encode(ctx, &prm.tmTlo, T.Tlo, 3, dl, strides, boxd, T);
        if (rc) return rc;
    }
    prm.kstep = 128 / T.esz;
    prm.kb = T.Kp / prm.kstep;
    prm.idesc = idesc_of(128, T.nsub, T.tf32, T.fp16);
    prm.wmax = T.fp16 ? T.d_wmax : nullptr;
    prm.inv_op_scale = float(1.0 / T.op_scale);
    prm.nsub = T.nsub;
    prm.ncta = T.ncta;
    prm.nvalid = 6 * P3;
    prm.tmem_cols = T.tmem_cols;
    prm.split = T.split;
    prm.drop_first = T.inject_drop;
    T.inject_drop = 0;
    const int stage_bytes = 128 * 64 * 2 + T.ncta * 128;
    int stages = std::max(2, std::min(6, (200 * 1024) / stage_bytes));
    const size_t smem = size_t(stages) * stage_bytes + 1024 + (2 * stages + 2) * 8 + 64;
    ++ctx->launches;
    if (T.tf32) {
        CK(cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_m2l_tc<true><<<T.n_work, 192, smem, ctx->stream>>>(prm, T.d_work, tocc, T.d_bocc, T.d_bocc_ofs, ctx->d_box,
                                                             Sf, T.d_status, stages);
    } else {
        CK(cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_m2l_tc<false><<<T.n_work, 192, smem, ctx->stream>>>(prm, T.d_work, tocc, T.d_bocc, T.d_bocc_ofs, ctx->d_box,
                                                              Sf, T.d_status, stages);
    }
    CK(cudaGetLastError());
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
    void *ps[] = {T.Thi, T.Tlo, T.Whi, T.Wlo, T.d_work, T.d_status, T.d_bocc, T.d_bocc_ofs, T.d_wmax};
    for (void *q : ps)
        if (q) cudaFree(q);
    T = TcPlan{};
}
