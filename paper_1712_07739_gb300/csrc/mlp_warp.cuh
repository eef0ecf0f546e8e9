// Warp-level evaluation of the angular network inside the near-field loop.
//
// Sixteen queued pair directions form the rows of one m16n8k16 tile; the
// layers run as warp MMAs (BF16 in, FP32 accumulate) with weights in shared
// memory and activations kept in registers: the FP32 accumulator fragment of
// one layer, passed through SiLU and packed to BF16 pairs, is exactly the A
// fragment of the next layer for the same lane.  Layout of the parameter
// vector as in mlp.cu (W1 [128x3], b1, W2 [128x128], b2, W3, b3, W4 [32x128], b4).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace mlpw {

constexpr int OFF_W1 = 0, OFF_B1 = 384, OFF_W2 = 512, OFF_B2 = 16896, OFF_W3 = 17024, OFF_B3 = 33408,
              OFF_W4 = 33536, OFF_B4 = 37632;
constexpr int LD = 136;  // padded row (bf16) of the weight matrices: conflict-free fragment loads

struct Weights {
    __nv_bfloat16 W2[128 * LD];
    __nv_bfloat16 W3[128 * LD];
    __nv_bfloat16 W4[32 * LD];
    float W1[128 * 3];
    float b1[128], b2[128], b3[128], b4[32], scale[32];
};

// cooperative copy of the parameters into shared memory (whole block)
__device__ inline void load(Weights &w, const __nv_bfloat16 *__restrict__ th, const float *__restrict__ th32,
                            const float *__restrict__ scale) {
    for (int i = threadIdx.x; i < 128 * 128; i += blockDim.x) {
        const int r = i / 128, c = i % 128;
        w.W2[r * LD + c] = th[OFF_W2 + i];
        w.W3[r * LD + c] = th[OFF_W3 + i];
    }
    for (int i = threadIdx.x; i < 32 * 128; i += blockDim.x) w.W4[(i / 128) * LD + (i % 128)] = th[OFF_W4 + i];
    for (int i = threadIdx.x; i < 384; i += blockDim.x) w.W1[i] = __bfloat162float(th[OFF_W1 + i]);
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        w.b1[i] = th32[OFF_B1 + i];
        w.b2[i] = th32[OFF_B2 + i];
        w.b3[i] = th32[OFF_B3 + i];
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        w.b4[i] = th32[OFF_B4 + i];
        w.scale[i] = i < 27 ? scale[i] : 0.f;
    }
}

// SiLU through the hardware tanh: silu(z) = z sigmoid(z) = z (1 + tanh(z/2)) / 2
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu_t(float z) { return 0.5f * z * (1.f + tanh_approx(0.5f * z)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// one hidden 128 -> 128 layer: a (A fragments, 8 k-steps) -> next A fragments
__device__ __forceinline__ void hidden(const __nv_bfloat16 *__restrict__ W, const float *__restrict__ b,
                                       uint32_t a[8][4], int g, int t) {
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const float b0 = b[nt * 8 + 2 * t], b1 = b[nt * 8 + 2 * t + 1];
        acc[nt][0] = b0;
        acc[nt][1] = b1;
        acc[nt][2] = b0;
        acc[nt][3] = b1;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const __nv_bfloat16 *row = W + (nt * 8 + g) * LD + kk * 16 + 2 * t;
            mma16816(acc[nt], a[kk], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        a[kk][0] = pack2(silu_t(acc[2 * kk][0]), silu_t(acc[2 * kk][1]));
        a[kk][1] = pack2(silu_t(acc[2 * kk][2]), silu_t(acc[2 * kk][3]));
        a[kk][2] = pack2(silu_t(acc[2 * kk + 1][0]), silu_t(acc[2 * kk + 1][1]));
        a[kk][3] = pack2(silu_t(acc[2 * kk + 1][2]), silu_t(acc[2 * kk + 1][3]));
    }
}

// sign of the half-space fold (h is odd)
__device__ __forceinline__ float fold_sign(float x, float y, float z) {
    return (z > 0.f || (z == 0.f && (y > 0.f || (y == 0.f && x >= 0.f)))) ? 1.f : -1.f;
}

// Network outputs for rows g and g + 8 of a 16-direction tile.  dlo, dhi:
// the two directions this lane's rows hold (already folded, |T| = 1).
// out[e]: for e = 0..7, column 8 (e / 2) + 2 t + (e & 1), row g (lo) / g + 8 (hi).
__device__ __forceinline__ void eval16(const Weights &w, const float dlo[3], const float dhi[3], int g, int t,
                                       float olo[8], float ohi[8]) {
    uint32_t a[8][4];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        float z[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = kk * 16 + 2 * t + (e & 1) + (e >> 1) * 8;
            const float w0 = w.W1[3 * c], w1 = w.W1[3 * c + 1], w2 = w.W1[3 * c + 2], bb = w.b1[c];
            z[2 * e] = silu_t(fmaf(w0, dlo[0], fmaf(w1, dlo[1], fmaf(w2, dlo[2], bb))));
            z[2 * e + 1] = silu_t(fmaf(w0, dhi[0], fmaf(w1, dhi[1], fmaf(w2, dhi[2], bb))));
        }
        // e = 0: col 2t (lo, hi); e = 1: col 2t+1; e = 2: col 2t+8; e = 3: col 2t+9
        a[kk][0] = pack2(z[0], z[2]);
        a[kk][1] = pack2(z[1], z[3]);
        a[kk][2] = pack2(z[4], z[6]);
        a[kk][3] = pack2(z[5], z[7]);
    }
    hidden(w.W2, w.b2, a, g, t);
    hidden(w.W3, w.b3, a, g, t);
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float b0 = w.b4[nt * 8 + 2 * t], b1 = w.b4[nt * 8 + 2 * t + 1];
        acc[nt][0] = b0;
        acc[nt][1] = b1;
        acc[nt][2] = b0;
        acc[nt][3] = b1;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const __nv_bfloat16 *row = w.W4 + (nt * 8 + g) * LD + kk * 16 + 2 * t;
            mma16816(acc[nt], a[kk], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        olo[2 * nt] = acc[nt][0];
        olo[2 * nt + 1] = acc[nt][1];
        ohi[2 * nt] = acc[nt][2];
        ohi[2 * nt + 1] = acc[nt][3];
    }
}

}  // namespace mlpw
