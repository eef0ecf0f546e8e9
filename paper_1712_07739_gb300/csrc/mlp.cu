// Learned angular factor: a small network T -> h_vpq(T) (the 27 components
// of R^2 dG_vp/dx_q, Sec. 2), trained on the GPU against the plain
// unit-circle evaluator and used in place of it where its error is small.
//
// Network (BF16 weights, FP32 accumulation): x = s T with s = +-1 putting T in
// the upper half-space (h is odd, so h(T) = s h(x) holds exactly), then
// 3 -> 128 -> 128 -> 128 -> 27 with SiLU activations; the output is in units
// of a per-component scale (RMS of the training labels).  Parameters are one
// flat FP32 master vector (W1 [128x3], b1, W2 [128x128], b2, W3, b3,
// W4 [32x128] (rows 27..31 stay zero), b4 [32]) with a BF16 copy for compute.
//
// Training: Adam on the mean-squared error in scaled units.  Every matrix
// product of the forward and backward passes runs in k_gemm_bf16 (warp
// mma.m16n8k16, BF16 in, FP32 accumulate); the first layer (3 inputs) and
// the element-wise steps are plain kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.cuh"
#include "kernel_math.cuh"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int OFF_W1 = 0, OFF_B1 = 384, OFF_W2 = 512, OFF_B2 = 16896, OFF_W3 = 17024, OFF_B3 = 33408,
              OFF_W4 = 33536, OFF_B4 = 37632, NPAR = 37664;

inline unsigned nblk(int64_t n, int b) { return unsigned(std::min<int64_t>((n + b - 1) / b, 1 << 22)); }

// SiLU through the hardware tanh (the same form the near-field kernel uses):
// sigmoid(z) = (1 + tanh(z/2)) / 2, silu = z sigmoid(z), silu' = s (1 + z (1 - s))
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu(float z) { return 0.5f * z * (1.f + tanh_hw(0.5f * z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 0.5f * (1.f + tanh_hw(0.5f * z));
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ float half_space_sign(float x, float y, float z) {
    return (z > 0.f || (z == 0.f && (y > 0.f || (y == 0.f && x >= 0.f)))) ? 1.f : -1.f;
}

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]); A(m,k) = A[m sam + k sak],
// B(k,n) = B[k sbk + n sbn], BF16 in, FP32 out.  64 x 64 block tile, 4 warps,
// each warp 16 rows x 64 columns as 8 mma.m16n8k16 per 16-wide K step.
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const bf16 *__restrict__ A, int64_t sam,
                                                   int64_t sak, const bf16 *__restrict__ B, int64_t sbk, int64_t sbn,
                                                   const float *__restrict__ bias, float *__restrict__ C, int64_t ldc) {
    __shared__ __align__(16) bf16 As[64][24];
    __shared__ __align__(16) bf16 Bs[64][24];
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[8][4];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = tid; i < 64 * 16; i += 128) {
            const int r = i / 16, c = i % 16, m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? A[m * sam + k * sak] : zero;
            const int n = n0 + r;
            Bs[r][c] = (n < N && k < K) ? B[k * sbk + n * sbn] : zero;
        }
        __syncthreads();
        const int r0 = warp * 16;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t *>(&As[r0 + g][2 * t]);
        a[1] = *reinterpret_cast<const uint32_t *>(&As[r0 + g + 8][2 * t]);
        a[2] = *reinterpret_cast<const uint32_t *>(&As[r0 + g][2 * t + 8]);
        a[3] = *reinterpret_cast<const uint32_t *>(&As[r0 + g + 8][2 * t + 8]);
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Bs[nt * 8 + g][2 * t]);
            uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Bs[nt * 8 + g][2 * t + 8]);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};"
                : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
        }
        __syncthreads();
    }
    const int r0 = m0 + warp * 16;
    for (int nt = 0; nt < 8; ++nt)
        for (int j = 0; j < 4; ++j) {
            const int m = r0 + g + (j >= 2 ? 8 : 0), n = n0 + nt * 8 + 2 * t + (j & 1);
            if (m < M && n < N) C[m * ldc + n] = acc[nt][j] + (bias ? bias[n] : 0.f);
        }
}

void gemm(cudaStream_t st, int M, int N, int K, const bf16 *A, int64_t sam, int64_t sak, const bf16 *B, int64_t sbk,
          int64_t sbn, const float *bias, float *C, int64_t ldc) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, C, ldc);
}

// first layer on canonical inputs: z1 = W1 x + b1, a1 = silu(z1)
__global__ void k_layer1(int n, const float *__restrict__ dirs, const bf16 *__restrict__ th,
                         const float *__restrict__ th32, float *__restrict__ x, float *__restrict__ z1,
                         bf16 *__restrict__ a1) {
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (idx >= int64_t(n) * 128) return;
    const int b = int(idx / 128), o = int(idx % 128);
    const float tx = dirs[3 * b], ty = dirs[3 * b + 1], tz = dirs[3 * b + 2];
    const float s = half_space_sign(tx, ty, tz);
    const float xx = s * tx, xy = s * ty, xz = s * tz;
    if (o == 0 && x) {
        x[3 * b] = xx;
        x[3 * b + 1] = xy;
        x[3 * b + 2] = xz;
    }
    const float z = __bfloat162float(th[OFF_W1 + 3 * o]) * xx + __bfloat162float(th[OFF_W1 + 3 * o + 1]) * xy +
                    __bfloat162float(th[OFF_W1 + 3 * o + 2]) * xz + th32[OFF_B1 + o];
    if (z1) z1[idx] = z;
    a1[idx] = __float2bfloat16(silu(z));
}

__global__ void k_silu(int64_t n, const float *__restrict__ z, bf16 *__restrict__ a) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) a[i] = __float2bfloat16(silu(z[i]));
}

// scaled output -> h (sign of the half-space restored)
__global__ void k_output(int n, const float *__restrict__ dirs, const float *__restrict__ o32,
                         const float *__restrict__ scale, float *__restrict__ h) {
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (idx >= int64_t(n) * 27) return;
    const int b = int(idx / 27), c = int(idx % 27);
    const float s = half_space_sign(dirs[3 * b], dirs[3 * b + 1], dirs[3 * b + 2]);
    h[idx] = s * scale[c] * o32[int64_t(b) * 32 + c];
}

// d loss / d o for loss = mean_{b,c} (o - s y / scale)^2
__global__ void k_loss_grad(int n, const float *__restrict__ dirs, const float *__restrict__ o32,
                            const float *__restrict__ y, const float *__restrict__ scale, bf16 *__restrict__ go,
                            float *__restrict__ loss) {
    const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    float l = 0.f;
    if (idx < int64_t(n) * 32) {
        const int b = int(idx / 32), c = int(idx % 32);
        float gval = 0.f;
        if (c < 27) {
            const float s = half_space_sign(dirs[3 * b], dirs[3 * b + 1], dirs[3 * b + 2]);
            const float r = o32[idx] - s * y[int64_t(b) * 27 + c] / scale[c];
            gval = 2.f * r / (float(n) * 27.f);
            l = r * r / (float(n) * 27.f);
        }
        go[idx] = __float2bfloat16(gval);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

__global__ void k_dsilu_mul(int64_t n, const float *__restrict__ da, const float *__restrict__ z,
                            bf16 *__restrict__ g, float *__restrict__ g32) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const float v = da[i] * dsilu(z[i]);
    g[i] = __float2bfloat16(v);
    if (g32) g32[i] = v;
}

// db[c] = sum_b g[b][c]  (g given as BF16 rows of width ld)
__global__ void k_colsum(int n, int cols, int ld, const bf16 *__restrict__ g, float *__restrict__ db) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += __bfloat162float(g[int64_t(b) * ld + c]);
    __shared__ float sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && c < cols) db[c] = sm[0];
}

// dW1[o][i] = sum_b g1[b][o] x[b][i]
__global__ void k_dw1(int n, const float *__restrict__ g1, const float *__restrict__ x, float *__restrict__ dW1) {
    const int o = blockIdx.x / 3, i = blockIdx.x % 3;
    float s = 0.f;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += g1[int64_t(b) * 128 + o] * x[3 * b + i];
    __shared__ float sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) dW1[3 * o + i] = sm[0];
}

__global__ void k_adam(int n, float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float c1, float c2, bf16 *__restrict__ thh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the padding rows of W4 and b4 (outputs 27..31) stay zero
    const bool pad = (i >= OFF_W4 + 27 * 128 && i < OFF_B4) || i >= OFF_B4 + 27;
    if (!pad) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
    thh[i] = __float2bfloat16(th[i]);
}

__global__ void k_to_bf16(int n, const float *__restrict__ a, bf16 *__restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// plain-evaluator labels (FP64 unit-circle rule), all 27 components
__global__ void k_labels(int64_t n, const DevMaterial *__restrict__ mat, const float *__restrict__ dirs,
                         float *__restrict__ y) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (b >= n) return;
    double T[3] = {dirs[3 * b], dirs[3 * b + 1], dirs[3 * b + 2]};
    const double r = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
    for (int i = 0; i < 3; ++i) T[i] /= r;
    double hs[18];
    if (mat->mode == GBFMM_H_ISO)
        h_iso_sym<double>(mat->hc, mat->ha, T, hs);
    else if (mat->cubic)
        h_circle_cubic<double>(mat->c12, mat->c44, mat->cd, mat->Q, T, hs);
    else
        h_circle_sym<double, double>(mat->C, mat->Q, T, hs);
    constexpr int PI_[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};  // (v,p) -> symmetric pair index
    for (int v = 0; v < 3; ++v)
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) y[b * 27 + (v * 3 + p) * 3 + q] = float(hs[3 * PI_[v][p] + q]);
}

__global__ void k_sumsq(int64_t n, const float *__restrict__ y, double *__restrict__ acc) {
    const int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (b >= n) return;
    for (int c = 0; c < 27; ++c) atomicAdd(&acc[c], double(y[b * 27 + c]) * double(y[b * 27 + c]));
}

__global__ void k_gather_rows(int n, int w, const int *__restrict__ idx, const float *__restrict__ src,
                              float *__restrict__ dst) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= int64_t(n) * w) return;
    dst[i] = src[int64_t(idx[i / w]) * w + (i % w)];
}

}  // namespace

// ---------------------------------------------------------------- host side
struct MlpBuffers {
    int cap = 0;
    float *x = nullptr, *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *o = nullptr, *da = nullptr, *g32 = nullptr;
    bf16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *go = nullptr, *g = nullptr;
};

static MlpBuffers &bufs(gbfmm_ctx *ctx) { return *reinterpret_cast<MlpBuffers *>(ctx->mlp.bufs); }

static int mlp_alloc_state(gbfmm_ctx *ctx) {
    MlpState &M = ctx->mlp;
    if (M.theta) return GBFMM_OK;
    CK(cudaMalloc(&M.theta, NPAR * sizeof(float)));
    CK(cudaMalloc(&M.grad, NPAR * sizeof(float)));
    CK(cudaMalloc(&M.m, NPAR * sizeof(float)));
    CK(cudaMalloc(&M.v, NPAR * sizeof(float)));
    CK(cudaMalloc(&M.theta_h, NPAR * sizeof(bf16)));
    CK(cudaMalloc(&M.scale, 32 * sizeof(float)));
    CK(cudaMalloc(&M.loss, sizeof(float)));
    M.bufs = new MlpBuffers();
    return GBFMM_OK;
}

static int mlp_alloc_batch(gbfmm_ctx *ctx, int n) {
    MlpBuffers &B = bufs(ctx);
    if (n <= B.cap) return GBFMM_OK;
    void *ps[] = {B.x, B.z1, B.z2, B.z3, B.o, B.da, B.g32, B.a1, B.a2, B.a3, B.go, B.g};
    for (void *p : ps)
        if (p) cudaFree(p);
    const int64_t n128 = int64_t(n) * 128;
    CK(cudaMalloc(&B.x, int64_t(n) * 3 * sizeof(float)));
    CK(cudaMalloc(&B.z1, n128 * sizeof(float)));
    CK(cudaMalloc(&B.z2, n128 * sizeof(float)));
    CK(cudaMalloc(&B.z3, n128 * sizeof(float)));
    CK(cudaMalloc(&B.o, int64_t(n) * 32 * sizeof(float)));
    CK(cudaMalloc(&B.da, n128 * sizeof(float)));
    CK(cudaMalloc(&B.g32, n128 * sizeof(float)));
    CK(cudaMalloc(&B.a1, n128 * sizeof(bf16)));
    CK(cudaMalloc(&B.a2, n128 * sizeof(bf16)));
    CK(cudaMalloc(&B.a3, n128 * sizeof(bf16)));
    CK(cudaMalloc(&B.go, int64_t(n) * 32 * sizeof(bf16)));
    CK(cudaMalloc(&B.g, n128 * sizeof(bf16)));
    B.cap = n;
    return GBFMM_OK;
}

// forward of n directions (batch buffers hold the activations): BF16
// weight matrices, FP32 biases, FP32 accumulation
static int mlp_forward(gbfmm_ctx *ctx, int n, const float *dirs) {
    MlpState &M = ctx->mlp;
    MlpBuffers &B = bufs(ctx);
    cudaStream_t st = ctx->stream;
    const bf16 *th = M.theta_h;
    const float *b = M.theta;
    ctx->launches += 6;
    k_layer1<<<nblk(int64_t(n) * 128, 256), 256, 0, st>>>(n, dirs, th, b, B.x, B.z1, B.a1);
    gemm(st, n, 128, 128, B.a1, 128, 1, th + OFF_W2, 1, 128, b + OFF_B2, B.z2, 128);
    k_silu<<<nblk(int64_t(n) * 128, 256), 256, 0, st>>>(int64_t(n) * 128, B.z2, B.a2);
    gemm(st, n, 128, 128, B.a2, 128, 1, th + OFF_W3, 1, 128, b + OFF_B3, B.z3, 128);
    k_silu<<<nblk(int64_t(n) * 128, 256), 256, 0, st>>>(int64_t(n) * 128, B.z3, B.a3);
    gemm(st, n, 32, 128, B.a3, 128, 1, th + OFF_W4, 1, 128, b + OFF_B4, B.o, 32);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

// gradient of the loss on one batch into M.grad; loss (scaled units) into M.loss
static int mlp_backward(gbfmm_ctx *ctx, int n, const float *dirs, const float *y) {
    MlpState &M = ctx->mlp;
    MlpBuffers &B = bufs(ctx);
    cudaStream_t st = ctx->stream;
    const bf16 *th = M.theta_h;
    const int64_t n128 = int64_t(n) * 128;
    CK(cudaMemsetAsync(M.loss, 0, sizeof(float), st));
    ctx->launches += 16;
    k_loss_grad<<<nblk(int64_t(n) * 32, 256), 256, 0, st>>>(n, dirs, B.o, y, M.scale, B.go, M.loss);
    // layer 4
    gemm(st, 32, 128, n, B.go, 1, 32, B.a3, 128, 1, nullptr, M.grad + OFF_W4, 128);
    k_colsum<<<32, 256, 0, st>>>(n, 32, 32, B.go, M.grad + OFF_B4);
    gemm(st, n, 128, 32, B.go, 32, 1, th + OFF_W4, 128, 1, nullptr, B.da, 128);
    k_dsilu_mul<<<nblk(n128, 256), 256, 0, st>>>(n128, B.da, B.z3, B.g, nullptr);
    // layer 3
    gemm(st, 128, 128, n, B.g, 1, 128, B.a2, 128, 1, nullptr, M.grad + OFF_W3, 128);
    k_colsum<<<128, 256, 0, st>>>(n, 128, 128, B.g, M.grad + OFF_B3);
    gemm(st, n, 128, 128, B.g, 128, 1, th + OFF_W3, 128, 1, nullptr, B.da, 128);
    k_dsilu_mul<<<nblk(n128, 256), 256, 0, st>>>(n128, B.da, B.z2, B.g, nullptr);
    // layer 2
    gemm(st, 128, 128, n, B.g, 1, 128, B.a1, 128, 1, nullptr, M.grad + OFF_W2, 128);
    k_colsum<<<128, 256, 0, st>>>(n, 128, 128, B.g, M.grad + OFF_B2);
    gemm(st, n, 128, 128, B.g, 128, 1, th + OFF_W2, 128, 1, nullptr, B.da, 128);
    k_dsilu_mul<<<nblk(n128, 256), 256, 0, st>>>(n128, B.da, B.z1, B.g, B.g32);
    // layer 1 (3 inputs)
    k_dw1<<<384, 256, 0, st>>>(n, B.g32, B.x, M.grad + OFF_W1);
    k_colsum<<<128, 256, 0, st>>>(n, 128, 128, B.g, M.grad + OFF_B1);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

// BF16 copy of the master parameters
static void sync_params(gbfmm_ctx *ctx) {
    ++ctx->launches;
    k_to_bf16<<<nblk(NPAR, 256), 256, 0, ctx->stream>>>(NPAR, ctx->mlp.theta, ctx->mlp.theta_h);
}

int mlp_eval_device(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *h) {
    MlpState &M = ctx->mlp;
    if (!M.trained) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_eval: network not trained or set");
    const int chunk = 1 << 18;
    int rc = mlp_alloc_batch(ctx, int(std::min<int64_t>(n, chunk)));
    if (rc) return rc;
    for (int64_t b0 = 0; b0 < n; b0 += chunk) {
        const int nb = int(std::min<int64_t>(chunk, n - b0));
        rc = mlp_forward(ctx, nb, dirs + 3 * b0);
        if (rc) return rc;
        ++ctx->launches;
        k_output<<<nblk(int64_t(nb) * 27, 256), 256, 0, ctx->stream>>>(nb, dirs + 3 * b0, bufs(ctx).o, M.scale,
                                                                         h + 27 * b0);
    }
    CK(cudaGetLastError());
    return GBFMM_OK;
}

extern "C" int fmm_mlp_set(gbfmm_ctx *ctx, const float *theta, const float *scale) {
    if (!ctx || !theta || !scale) return GBFMM_ERR_INVALID_ARG;
    int rc = mlp_alloc_state(ctx);
    if (rc) return rc;
    std::vector<float> th(theta, theta + NPAR);
    for (int i = OFF_W4 + 27 * 128; i < OFF_B4; ++i) th[i] = 0.f;
    for (int i = OFF_B4 + 27; i < NPAR; ++i) th[i] = 0.f;
    float sc[32] = {0};
    for (int i = 0; i < 27; ++i) sc[i] = scale[i];
    CK(cudaMemcpy(ctx->mlp.theta, th.data(), NPAR * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->mlp.scale, sc, sizeof(sc), cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->mlp.m, 0, NPAR * sizeof(float)));
    CK(cudaMemset(ctx->mlp.v, 0, NPAR * sizeof(float)));
    rc = mlp_alloc_batch(ctx, 1024);
    if (rc) return rc;
    sync_params(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp.trained = true;
    ctx->mlp.step = 0;
    return GBFMM_OK;
}

extern "C" int fmm_mlp_get(gbfmm_ctx *ctx, float *theta, float *scale) {
    if (!ctx || !theta || !scale) return GBFMM_ERR_INVALID_ARG;
    if (!ctx->mlp.theta) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_get: no network");
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(theta, ctx->mlp.theta, NPAR * sizeof(float), cudaMemcpyDeviceToHost));
    float sc[32];
    CK(cudaMemcpy(sc, ctx->mlp.scale, sizeof(sc), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 27; ++i) scale[i] = sc[i];
    return GBFMM_OK;
}

extern "C" int fmm_mlp_eval(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *h) {
    if (!ctx || n < 0 || (n > 0 && (!dirs || !h))) return GBFMM_ERR_INVALID_ARG;
    if (n == 0) return GBFMM_OK;
    return mlp_eval_device(ctx, n, dirs, h);
}

extern "C" int fmm_mlp_grad(gbfmm_ctx *ctx, int n, const float *dirs, const float *y, float *grad, float *loss) {
    if (!ctx || n < 1 || !dirs || !y || !grad) return GBFMM_ERR_INVALID_ARG;
    if (!ctx->mlp.trained) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_grad: set parameters first");
    int rc = mlp_alloc_batch(ctx, n);
    if (rc) return rc;
    rc = mlp_forward(ctx, n, dirs);
    if (rc) return rc;
    rc = mlp_backward(ctx, n, dirs, y);
    if (rc) return rc;
    CK(cudaMemcpyAsync(grad, ctx->mlp.grad, NPAR * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    if (loss) {
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(loss, ctx->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return GBFMM_OK;
}

extern "C" int fmm_mlp_labels(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *y) {
    if (!ctx || n < 0 || (n > 0 && (!dirs || !y))) return GBFMM_ERR_INVALID_ARG;
    if (!ctx->have_material) return set_err(ctx, GBFMM_ERR_NO_MATERIAL, "fmm_mlp_labels: set the material first");
    if (n == 0) return GBFMM_OK;
    ++ctx->launches;
    k_labels<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, ctx->d_mat, dirs, y);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

extern "C" int fmm_mlp_train(gbfmm_ctx *ctx, int64_t n, const float *dirs, int epochs, int batch, double lr,
                             uint64_t seed, float *final_loss) {
    if (!ctx || n < batch || batch < 64 || epochs < 1 || !dirs || !(lr > 0.0))
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_train: bad arguments");
    if (!ctx->have_material) return set_err(ctx, GBFMM_ERR_NO_MATERIAL, "fmm_mlp_train: set the material first");
    cudaStream_t st = ctx->stream;
    int rc = mlp_alloc_state(ctx);
    if (rc) return rc;
    rc = mlp_alloc_batch(ctx, batch);
    if (rc) return rc;
    MlpState &M = ctx->mlp;
    // labels by the plain evaluator and their per-component RMS
    float *y = nullptr, *bd = nullptr, *by = nullptr;
    int *perm = nullptr;
    double *acc = nullptr;
    CK(cudaMalloc(&y, n * 27 * sizeof(float)));
    CK(cudaMalloc(&bd, int64_t(batch) * 3 * sizeof(float)));
    CK(cudaMalloc(&by, int64_t(batch) * 27 * sizeof(float)));
    CK(cudaMalloc(&perm, n * sizeof(int)));
    CK(cudaMalloc(&acc, 27 * sizeof(double)));
    rc = fmm_mlp_labels(ctx, n, dirs, y);
    if (rc) return rc;
    CK(cudaMemsetAsync(acc, 0, 27 * sizeof(double), st));
    ++ctx->launches;
    k_sumsq<<<nblk(n, 256), 256, 0, st>>>(n, y, acc);
    double h_acc[27];
    CK(cudaMemcpyAsync(h_acc, acc, sizeof(h_acc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float sc[32] = {0};
    double smax = 0.0;
    for (int c = 0; c < 27; ++c) smax = std::max(smax, std::sqrt(h_acc[c] / double(n)));
    for (int c = 0; c < 27; ++c) sc[c] = float(std::max(std::sqrt(h_acc[c] / double(n)), 1e-3 * smax));
    // He-style initialisation from a seeded generator
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    std::vector<float> th(NPAR, 0.f);
    auto fill = [&](int off, int rows, int cols, int fan_in) {
        const float sd = std::sqrt(2.f / float(fan_in));
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) th[off + r * cols + c] = sd * nd(rng);
    };
    fill(OFF_W1, 128, 3, 3);
    fill(OFF_W2, 128, 128, 128);
    fill(OFF_W3, 128, 128, 128);
    fill(OFF_W4, 27, 128, 128);
    rc = fmm_mlp_set(ctx, th.data(), sc);
    if (rc) return rc;
    // Adam with cosine decay of the learning rate
    const int steps_per_epoch = int(n / batch);
    const int64_t total = int64_t(steps_per_epoch) * epochs;
    std::vector<int> hp(n);
    float last = 0.f;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t i = 0; i < n; ++i) hp[i] = int(i);
        std::shuffle(hp.begin(), hp.end(), rng);
        CK(cudaMemcpyAsync(perm, hp.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        for (int s = 0; s < steps_per_epoch; ++s) {
            ctx->launches += 2;
            k_gather_rows<<<nblk(int64_t(batch) * 3, 256), 256, 0, st>>>(batch, 3, perm + int64_t(s) * batch, dirs, bd);
            k_gather_rows<<<nblk(int64_t(batch) * 27, 256), 256, 0, st>>>(batch, 27, perm + int64_t(s) * batch, y, by);
            rc = mlp_forward(ctx, batch, bd);
            if (rc) return rc;
            rc = mlp_backward(ctx, batch, bd, by);
            if (rc) return rc;
            ++M.step;
            const double frac = double(M.step) / double(total);
            const float lr_t = float(lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(M_PI * std::min(1.0, frac)))));
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, float(M.step)), c2 = 1.f - std::pow(b2, float(M.step));
            ++ctx->launches;
            k_adam<<<nblk(NPAR, 256), 256, 0, st>>>(NPAR, M.theta, M.grad, M.m, M.v, lr_t, b1, b2, c1, c2,
                                                      M.theta_h);
        }
        CK(cudaMemcpyAsync(&last, M.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    cudaFree(y);
    cudaFree(bd);
    cudaFree(by);
    cudaFree(perm);
    cudaFree(acc);
    M.trained = true;
    if (final_loss) *final_loss = last;
    return GBFMM_OK;
}

// Assess the network per angular bin against the plain evaluator: 64 directions
// per bin of the near-field kernel's binning (dominant axis face +z, +x, -x,
// +y, -y and a 16 x 16 grid of the other two components); a bin whose largest
// component error exceeds bin_tol x (RMS of h over all samples) is flagged
// and its pairs take the plain evaluator.
extern "C" int fmm_mlp_calibrate(gbfmm_ctx *ctx, double bin_tol, double *fallback_frac) {
    if (!ctx || !(bin_tol > 0.0)) return GBFMM_ERR_INVALID_ARG;
    if (!ctx->mlp.trained) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_calibrate: train or set the network first");
    const int nb = 5 * 256, per = 64;
    std::vector<float> dirs(size_t(nb) * per * 3);
    for (int b = 0; b < nb; ++b) {
        const int f = b / 256, bu = (b / 16) % 16, bv = b % 16;
        for (int i = 0; i < per; ++i) {
            const float u = -1.f + 2.f * (bu + (i % 8 + 0.5f) / 8.f) / 16.f;
            const float v = -1.f + 2.f * (bv + (i / 8 + 0.5f) / 8.f) / 16.f;
            float d[3];
            if (f == 0) { d[0] = u; d[1] = v; d[2] = 1.f; }
            else if (f <= 2) { d[0] = f == 1 ? 1.f : -1.f; d[1] = u; d[2] = v; }
            else { d[0] = u; d[1] = f == 3 ? 1.f : -1.f; d[2] = v; }
            const float n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int c = 0; c < 3; ++c) dirs[(size_t(b) * per + i) * 3 + c] = d[c] / n;
        }
    }
    const int64_t n = int64_t(nb) * per;
    float *dd = nullptr, *y = nullptr, *hm = nullptr;
    CK(cudaMalloc(&dd, n * 3 * sizeof(float)));
    CK(cudaMalloc(&y, n * 27 * sizeof(float)));
    CK(cudaMalloc(&hm, n * 27 * sizeof(float)));
    CK(cudaMemcpy(dd, dirs.data(), n * 3 * sizeof(float), cudaMemcpyHostToDevice));
    int rc = fmm_mlp_labels(ctx, n, dd, y);
    if (rc) return rc;
    rc = mlp_eval_device(ctx, n, dd, hm);
    if (rc) return rc;
    std::vector<float> hy(n * 27), hh(n * 27);
    CK(cudaMemcpyAsync(hy.data(), y, n * 27 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hh.data(), hm, n * 27 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(dd);
    cudaFree(y);
    cudaFree(hm);
    double ss = 0.0;
    for (float v : hy) ss += double(v) * v;
    const double rms = std::sqrt(ss / double(hy.size()));
    uint32_t mask[48] = {0};
    int flagged = 0;
    for (int b = 0; b < nb; ++b) {
        double e = 0.0;
        for (int i = 0; i < per * 27; ++i) {
            const size_t k = size_t(b) * per * 27 + i;
            e = std::max(e, std::fabs(double(hh[k]) - double(hy[k])));
        }
        if (e > bin_tol * rms) {
            mask[b >> 5] |= 1u << (b & 31);
            ++flagged;
        }
    }
    if (!ctx->mlp.d_binmask) CK(cudaMalloc(&ctx->mlp.d_binmask, sizeof(mask)));
    CK(cudaMemcpy(ctx->mlp.d_binmask, mask, sizeof(mask), cudaMemcpyHostToDevice));
    ctx->mlp.fallback_frac = double(flagged) / double(nb);
    if (fallback_frac) *fallback_frac = ctx->mlp.fallback_frac;
    return GBFMM_OK;
}

void mlp_free(gbfmm_ctx *ctx) {
    MlpState &M = ctx->mlp;
    void *ps[] = {M.theta, M.grad, M.m, M.v, M.theta_h, M.scale, M.loss, M.d_binmask};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (M.bufs) {
        MlpBuffers &B = bufs(ctx);
        void *qs[] = {B.x, B.z1, B.z2, B.z3, B.o, B.da, B.g32, B.a1, B.a2, B.a3, B.go, B.g};
        for (void *p : qs)
            if (p) cudaFree(p);
        delete &B;
    }
    M = MlpState{};
}

// ---------------------------------------------------------------- no-allocation evaluation
// fmm_mlp_eval_noalloc: the network evaluation of fmm_mlp_eval for callers
// that must not allocate device memory during the call (see gbfmm.h).  The
// activations live in one file-scope device array; its device address is
// looked up once per device.
#define GB_NOALLOC_CHUNK 4096                      // directions per pass over the scratch
#define GB_NOALLOC_MAX (int64_t(1) << 24)          // largest n accepted per call
static constexpr size_t kNoallocZ = size_t(GB_NOALLOC_CHUNK) * 128 * sizeof(float);   // pre-activations
static constexpr size_t kNoallocA = size_t(GB_NOALLOC_CHUNK) * 128 * sizeof(bf16);    // one activation buffer
static constexpr size_t kNoallocO = size_t(GB_NOALLOC_CHUNK) * 32 * sizeof(float);    // outputs
static constexpr size_t kNoallocBytes = kNoallocZ + 2 * kNoallocA + kNoallocO;         // 4.5 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static unsigned char *noalloc_base(gbfmm_ctx *ctx) {
    // one lookup per device, made with that device current (the context's)
    static unsigned char *base[64] = {nullptr};
    const int dev = ctx->device;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != dev || dev < 0 || dev >= 64) return nullptr;
    if (!base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        base[dev] = static_cast<unsigned char *>(p);
    }
    return base[dev];
}

extern "C" int fmm_mlp_eval_noalloc(gbfmm_ctx *ctx, int64_t n, const float *dirs, float *h) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!dirs || !h)))
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_eval_noalloc: bad arguments");
    if (n > GB_NOALLOC_MAX)
        return set_err(ctx, GBFMM_ERR_INVALID_ARG,
                       "fmm_mlp_eval_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
                           std::to_string(GB_NOALLOC_MAX) + " directions per call");
    if (!ctx->mlp.trained) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_mlp_eval_noalloc: network not set");
    if (n == 0) return GBFMM_OK;
    unsigned char *base = noalloc_base(ctx);
    if (!base)
        return set_err(ctx, GBFMM_ERR_CUDA,
                       "fmm_mlp_eval_noalloc: scratch address lookup failed (is the context's device current?)");
    float *z = reinterpret_cast<float *>(base);
    bf16 *a = reinterpret_cast<bf16 *>(base + kNoallocZ);
    bf16 *b = reinterpret_cast<bf16 *>(base + kNoallocZ + kNoallocA);
    float *o = reinterpret_cast<float *>(base + kNoallocZ + 2 * kNoallocA);
    cudaStream_t st = ctx->stream;
    const MlpState &M = ctx->mlp;
    const bf16 *th = M.theta_h;
    const float *bias = M.theta;
    for (int64_t b0 = 0; b0 < n; b0 += GB_NOALLOC_CHUNK) {
        const int nb = int(std::min<int64_t>(GB_NOALLOC_CHUNK, n - b0));
        const int64_t e = int64_t(nb) * 128;
        const float *d = dirs + 3 * b0;
        ctx->launches += 7;
        k_layer1<<<nblk(e, 256), 256, 0, st>>>(nb, d, th, bias, nullptr, nullptr, a);
        gemm(st, nb, 128, 128, a, 128, 1, th + OFF_W2, 1, 128, bias + OFF_B2, z, 128);
        k_silu<<<nblk(e, 256), 256, 0, st>>>(e, z, b);
        gemm(st, nb, 128, 128, b, 128, 1, th + OFF_W3, 1, 128, bias + OFF_B3, z, 128);
        k_silu<<<nblk(e, 256), 256, 0, st>>>(e, z, a);
        gemm(st, nb, 32, 128, a, 128, 1, th + OFF_W4, 1, 128, bias + OFF_B4, o, 32);
        k_output<<<nblk(int64_t(nb) * 27, 256), 256, 0, st>>>(nb, d, o, M.scale, h + 27 * b0);
    }
    CK(cudaGetLastError());
    return GBFMM_OK;
}
