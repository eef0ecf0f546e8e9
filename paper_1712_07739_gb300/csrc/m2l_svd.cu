// SVD-compressed M2L: the compression of the Chebyshev FMM the paper compares
// against (Sec. 3, Eq. "mem_cheb"), on equispaced or Chebyshev nodes.
//
// The 316 node-to-node operators T_o of a unit cell (Eq. "m2l"; rows n =
// (target node l, stress component ab), columns k = (source node m, strength
// component wr)) are built in FP64.  Side by side, their left singular
// vectors give a target basis U; stacked, their right singular vectors give a
// source basis R.  These are the eigenvectors of sum_o T_o T_o^T and
// sum_o T_o^T T_o, whose eigenvalues are the squared singular values.  A
// vector is kept while its singular value exceeds m2l_svd_tol times the
// largest; the counts are rounded up to the tile granularity of the
// tensor-core GEMM (16 target, 64 source coefficients) by keeping the next
// vectors.  Each offset's operator becomes C_o = U^T T_o R (r1 x r2), and
// the M2L of a cell pair U C_o R^T W: every cell's multipole values are
// transformed once, W' = R^T W, the tensor-core GEMMs of m2l_tc.cu run on W'
// and the C_o, and every cell's compressed local values are expanded once,
// S = U S'.  The kernel's homogeneity (degree -2) makes the bases the same at
// every level.
//
// The setup is FP64 dense linear algebra done by library routines (cuBLAS
// DSYRK and DGEMM, cuSOLVER's symmetric eigensolver).  The per-pass
// transforms are plain dense GEMMs with FP32 results, run by cuBLAS on the
// tensor cores as three FP16 products of hi + lo splits of both factors
// (hi*hi + hi*lo + lo*hi, FP32 accumulation; each level's operand scaled by
// its own power of two).
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "kernel_math.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

#define BL(call)                                                                                 \
    do {                                                                                         \
        const cublasStatus_t s_ = (call);                                                        \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                                         \
            return set_err(ctx, GBFMM_ERR_CUDA, std::string("cuBLAS ") + #call + ": " + std::to_string(int(s_))); \
    } while (0)

#define SL(call)                                                                                 \
    do {                                                                                         \
        const cusolverStatus_t s_ = (call);                                                      \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                       \
            return set_err(ctx, GBFMM_ERR_CUDA, std::string("cuSOLVER ") + #call + ": " + std::to_string(int(s_))); \
    } while (0)

// T_o for the nc offsets from o0 (xyz in off), FP64, unit cell, row-major [o][n][k]:
// n = 6 l + ab, k = 9 m + wr.  Equispaced nodes read the kernel lattice (the same
// values as the dense operators of m2l_tc.cu); Chebyshev nodes evaluate the kernel
// at the node differences o + t_l - t_m.  One thread per (offset, l, m): 54 entries.
__global__ void k_node_ops(int p, int nodes, int o0, int nc, const int *__restrict__ off,
                           const DevMaterial *__restrict__ mat, const double *__restrict__ Asym, int lat_n,
                           const double *__restrict__ Klat, double *__restrict__ T) {
    const int P3 = p * p * p, nt = 6 * P3, ns = 9 * P3;
    const int64_t total = int64_t(nc) * P3 * P3;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int mm = int(idx % P3), l = int((idx / P3) % P3), oc = int(idx / (int64_t(P3) * P3));
        const int o = o0 + oc;
        const int ox = off[3 * o], oy = off[3 * o + 1], oz = off[3 * o + 2];
        const int lx = l % p, ly = (l / p) % p, lz = l / (p * p);
        const int mx = mm % p, my = (mm / p) % p, mz = mm / (p * p);
        double K[54];
        if (nodes == GBFMM_NODES_CHEBYSHEV) {
            const double d[3] = {ox + cheb_node<double>(lx, p) - cheb_node<double>(mx, p),
                                 oy + cheb_node<double>(ly, p) - cheb_node<double>(my, p),
                                 oz + cheb_node<double>(lz, p) - cheb_node<double>(mz, p)};
            kernel_at(mat, Asym, d, K);
        } else {
            const int R0 = (lat_n - 1) / 2;
            const int Dx = ox * (p - 1) + lx - mx + R0, Dy = oy * (p - 1) + ly - my + R0,
                      Dz = oz * (p - 1) + lz - mz + R0;
            const double *src = Klat + ((int64_t(Dz) * lat_n + Dy) * lat_n + Dx) * 54;
            for (int i = 0; i < 54; ++i) K[i] = src[i];
        }
        double *dst = T + (int64_t(oc) * nt + 6 * l) * ns + 9 * mm;
        for (int ab = 0; ab < 6; ++ab)
            for (int wr = 0; wr < 9; ++wr) dst[int64_t(ab) * ns + wr] = K[ab * 9 + wr];
    }
}

// out[:, j] = G[:, n - 1 - j] for j < r: the eigenvectors of the r largest
// eigenvalues (the solver returns them in increasing order), FP64 and FP32
__global__ void k_take_cols(int n, int r, const double *__restrict__ G, double *__restrict__ out,
                            float *__restrict__ outf) {
    const int64_t total = int64_t(n) * r;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(idx % n), j = int(idx / n);
        const double v = G[int64_t(n - 1 - j) * n + i];
        out[idx] = v;
        outf[idx] = float(v);
    }
}

__global__ void k_absmax(int64_t n, const double *__restrict__ x, unsigned long long *__restrict__ out) {
    double mx = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        mx = fmax(mx, fabs(x[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

template <typename E>
__device__ __forceinline__ E from_f64(double v);
template <>
__device__ __forceinline__ __half from_f64<__half>(double v) {
    return __double2half(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ float from_f64<float>(double v) {
    return float(v);
}
__device__ __forceinline__ double as_f64(__half x) { return double(__half2float(x)); }
__device__ __forceinline__ double as_f64(__nv_bfloat16 x) { return double(__bfloat162float(x)); }
__device__ __forceinline__ double as_f64(float x) { return double(x); }

// compressed operators [o][Np][Kp] (FP64, zero padded) -> operand tables: hi = E(scale C),
// residual lo = E(scale C - hi) on the leading Kp_lo columns of the offsets with a residual table
template <typename E>
__global__ void k_ops_convert(int64_t total, int Np, int Kp, int Kp_lo, const double *__restrict__ C,
                              const int *__restrict__ lo_of, double scale, E *__restrict__ Thi, E *__restrict__ Tlo) {
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(idx % Kp);
        const int nn = int((idx / Kp) % Np);
        const int o = int(idx / (int64_t(Kp) * Np));
        const double v = scale * C[idx];
        const E hi = from_f64<E>(v);
        Thi[idx] = hi;
        const int li = lo_of[o];
        if (li >= 0 && Tlo && k < Kp_lo) Tlo[(int64_t(li) * Np + nn) * Kp_lo + k] = from_f64<E>(v - as_f64(hi));
    }
}

inline int pad8(int n) { return (n + 7) / 8 * 8; }

// largest |x| over n values into *bits (non-negative floats order like their bit patterns)
__global__ void k_absmax_f32(int64_t n, const float *__restrict__ x, unsigned *__restrict__ bits) {
    float mx = 0.f;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        mx = fmaxf(mx, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(bits, __float_as_uint(mx));
}

// rows vectors of n FP32 values (contiguous) -> FP16 hi + lo, stride ldx (zero padded), all
// scaled by the power of two s that maps the largest |value| just below 2^14:
// hi = fp16(s x), lo = fp16(s x - hi).  *alpha (if given) = 1 / (s sbasis), the factor that
// undoes both scales of a product with a basis split the same way.
__global__ void k_split_f16(int64_t rows, int n, int ldx, const float *__restrict__ src,
                            const unsigned *__restrict__ bits, float sbasis, __half *__restrict__ hi,
                            __half *__restrict__ lo, float *__restrict__ alpha) {
    const float mx = __uint_as_float(*bits);
    int e = 0;
    frexpf(mx, &e);
    const float s = mx > 0.f ? ldexpf(1.f, 14 - e) : 1.f;
    if (alpha && blockIdx.x == 0 && threadIdx.x == 0) *alpha = 1.f / (s * sbasis);
    const int64_t total = rows * ldx;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = idx / ldx;
        const int k = int(idx - r * ldx);
        const float v = k < n ? src[r * n + k] * s : 0.f;
        const __half h = __float2half_rn(v);
        hi[idx] = h;
        lo[idx] = __float2half_rn(v - __half2float(h));
    }
}

// the 316 offsets o in [-3, 3]^3 with max |o_i| >= 2
std::vector<int> all_offsets() {
    std::vector<int> off;
    for (int oz = -3; oz <= 3; ++oz)
        for (int oy = -3; oy <= 3; ++oy)
            for (int ox = -3; ox <= 3; ++ox)
                if (std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) >= 2) {
                    off.push_back(ox);
                    off.push_back(oy);
                    off.push_back(oz);
                }
    return off;
}

// offsets per chunk of dense FP64 operators: at most ~1 GiB of them at a time
int chunk_offsets(int p) {
    const int64_t P3 = int64_t(p) * p * p;
    const int64_t per = 54 * P3 * P3 * int64_t(sizeof(double));
    return int(std::max<int64_t>(1, std::min<int64_t>(316, (int64_t(1) << 30) / per)));
}

int ensure_blas(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    if (!T.blas) {
        cublasHandle_t h = nullptr;
        BL(cublasCreate(&h));
        T.blas = h;
        T.blas_ws_bytes = size_t(64) << 20;
        CK(cudaMalloc(&T.blas_ws, T.blas_ws_bytes));
        BL(cublasSetWorkspace(h, T.blas_ws, T.blas_ws_bytes));
    }
    BL(cublasSetStream((cublasHandle_t)T.blas, ctx->stream));
    // host scalars unless a caller switches to device scalars for its own calls (and back),
    // also after a call that returned early
    BL(cublasSetPointerMode((cublasHandle_t)T.blas, CUBLAS_POINTER_MODE_HOST));
    return GBFMM_OK;
}

}  // namespace

int svd_bases(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    if (T.bases_ok && T.Uf && T.Rf) return GBFMM_OK;  // a switch of the tile form keeps them
    const int p = ctx->opt.p, P3 = p * p * p, nt = 6 * P3, ns = 9 * P3;
    const double tol = ctx->opt.m2l_svd_tol;
    cudaStream_t st = ctx->stream;
    if (int rc = ensure_blas(ctx)) return rc;
    cublasHandle_t h = (cublasHandle_t)T.blas;
    const std::vector<int> off = all_offsets();
    const int n_off = int(off.size() / 3), nc = chunk_offsets(p);
    int *d_off = nullptr;
    double *Tb = nullptr, *Gt = nullptr, *Gs = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_off);
        cudaFree(Tb);
        cudaFree(Gt);
        cudaFree(Gs);
    };
    if (cudaMalloc(&d_off, off.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&Tb, size_t(nc) * nt * ns * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Gt, size_t(nt) * nt * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Gs, size_t(ns) * ns * sizeof(double)) != cudaSuccess) {
        cleanup();
        return set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: out of device memory");
    }
    int rc = GBFMM_OK;
    auto run = [&]() -> int {
        CK(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(Gt, 0, size_t(nt) * nt * sizeof(double), st));
        CK(cudaMemsetAsync(Gs, 0, size_t(ns) * ns * sizeof(double), st));
        const double one = 1.0;
        for (int o0 = 0; o0 < n_off; o0 += nc) {
            const int m = std::min(nc, n_off - o0);
            ++ctx->launches;
            k_node_ops<<<nblk(int64_t(m) * P3 * P3, 128), 128, 0, st>>>(p, ctx->opt.nodes, o0, m, d_off, ctx->d_mat,
                                                                         ctx->d_Asym, ctx->lat_n, ctx->d_Klat, Tb);
            CK(cudaGetLastError());
            // sum_o T_o^T T_o: the chunk read column-major is [T_1^T ... T_m^T] (ns x m nt)
            BL(cublasDsyrk(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, ns, m * nt, &one, Tb, ns, &one, Gs, ns));
            // sum_o T_o T_o^T: each T_o read column-major is T_o^T (ns x nt)
            for (int i = 0; i < m; ++i)
                BL(cublasDsyrk(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, nt, ns, &one, Tb + size_t(i) * nt * ns, ns,
                               &one, Gt, nt));
        }
        // eigenvectors of the two Gram matrices (in place), eigenvalues increasing
        std::vector<double> wt(nt), ws(ns);
        cusolverDnHandle_t sh = nullptr;
        SL(cusolverDnCreate(&sh));
        auto eig = [&](double *G, int n, std::vector<double> &w_host) -> int {
            double *w = nullptr, *work = nullptr;
            int *info = nullptr, lwork = 0, hinfo = 0;
            int r = GBFMM_OK;
            if (cusolverDnSetStream(sh, st) != CUSOLVER_STATUS_SUCCESS ||
                cusolverDnDsyevd_bufferSize(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, G, n, w, &lwork) !=
                    CUSOLVER_STATUS_SUCCESS)
                return set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: cuSOLVER workspace query");
            if (cudaMalloc(&w, size_t(n) * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&work, size_t(lwork) * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&info, sizeof(int)) != cudaSuccess)
                r = set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: out of device memory (eigensolver)");
            else if (cusolverDnDsyevd(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, G, n, w, work, lwork,
                                      info) != CUSOLVER_STATUS_SUCCESS)
                r = set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: cusolverDnDsyevd");
            else if (cudaMemcpyAsync(w_host.data(), w, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                         cudaSuccess ||
                     cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess)
                r = set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: eigenvalue read-back");
            else if (hinfo != 0)
                r = set_err(ctx, GBFMM_ERR_CUDA, "SVD setup: eigensolver did not converge (" + std::to_string(hinfo) + ")");
            cudaFree(w);
            cudaFree(work);
            cudaFree(info);
            return r;
        };
        int r = eig(Gt, nt, wt);
        if (!r) r = eig(Gs, ns, ws);
        cusolverDnDestroy(sh);
        if (r) return r;
        // singular values, decreasing; ranks above the tolerance, rounded up to the tiles
        auto sig = [](const std::vector<double> &w, int i) { return std::sqrt(std::max(w[w.size() - 1 - i], 0.0)); };
        int r1 = 0, r2 = 0;
        while (r1 < nt && sig(wt, r1) > tol * sig(wt, 0)) ++r1;
        while (r2 < ns && sig(ws, r2) > tol * sig(ws, 0)) ++r2;
        T.r1_raw = r1;
        T.r2_raw = r2;
        T.r1 = std::min(nt, std::max(16, (r1 + 15) / 16 * 16));
        T.r2 = std::min(ns, std::max(64, (r2 + 63) / 64 * 64));
        T.svd_sigma[0] = sig(wt, 0);
        T.svd_sigma[1] = sig(wt, T.r1 - 1);
        T.svd_sigma[2] = sig(ws, 0);
        T.svd_sigma[3] = sig(ws, T.r2 - 1);
        // the kept vectors, FP64 for the operators and FP32 for the per-pass transforms
        void *old[4] = {T.U64, T.R64, T.Uf, T.Rf};
        for (void *q : old)
            if (q) cudaFree(q);
        T.U64 = T.R64 = nullptr;
        T.Uf = T.Rf = nullptr;
        CK(cudaMalloc(&T.U64, size_t(nt) * T.r1 * sizeof(double)));
        CK(cudaMalloc(&T.R64, size_t(ns) * T.r2 * sizeof(double)));
        CK(cudaMalloc(&T.Uf, size_t(nt) * T.r1 * sizeof(float)));
        CK(cudaMalloc(&T.Rf, size_t(ns) * T.r2 * sizeof(float)));
        ctx->launches += 2;
        k_take_cols<<<nblk(int64_t(nt) * T.r1, 256), 256, 0, st>>>(nt, T.r1, Gt, T.U64, T.Uf);
        k_take_cols<<<nblk(int64_t(ns) * T.r2, 256), 256, 0, st>>>(ns, T.r2, Gs, T.R64, T.Rf);
        CK(cudaGetLastError());
        // FP16 hi + lo of both bases for the per-pass transforms, columns padded to 8 rows
        void *olds[4] = {T.Uh, T.Ul, T.Rh, T.Rl};
        for (void *q : olds)
            if (q) cudaFree(q);
        T.Uh = T.Ul = T.Rh = T.Rl = nullptr;
        const size_t nu = size_t(pad8(nt)) * T.r1, nr = size_t(pad8(ns)) * T.r2;
        CK(cudaMalloc(&T.Uh, nu * sizeof(__half)));
        CK(cudaMalloc(&T.Ul, nu * sizeof(__half)));
        CK(cudaMalloc(&T.Rh, nr * sizeof(__half)));
        CK(cudaMalloc(&T.Rl, nr * sizeof(__half)));
        unsigned *d_b = nullptr;
        CK(cudaMalloc(&d_b, 2 * sizeof(unsigned)));
        CK(cudaMemsetAsync(d_b, 0, 2 * sizeof(unsigned), st));
        ctx->launches += 4;
        k_absmax_f32<<<256, 256, 0, st>>>(int64_t(nt) * T.r1, T.Uf, d_b);
        k_absmax_f32<<<256, 256, 0, st>>>(int64_t(ns) * T.r2, T.Rf, d_b + 1);
        k_split_f16<<<nblk(int64_t(nu), 256), 256, 0, st>>>(T.r1, nt, pad8(nt), T.Uf, d_b, 1.f, (__half *)T.Uh,
                                                             (__half *)T.Ul, nullptr);
        k_split_f16<<<nblk(int64_t(nr), 256), 256, 0, st>>>(T.r2, ns, pad8(ns), T.Rf, d_b + 1, 1.f, (__half *)T.Rh,
                                                             (__half *)T.Rl, nullptr);
        CK(cudaGetLastError());
        unsigned hb[2] = {0, 0};
        CK(cudaMemcpyAsync(hb, d_b, sizeof(hb), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cudaFree(d_b);
        auto scale_of = [](unsigned b) {
            float mx;
            std::memcpy(&mx, &b, sizeof(mx));
            int e = 0;
            std::frexp(mx, &e);
            return mx > 0.f ? std::ldexp(1.f, 14 - e) : 1.f;
        };
        T.sU = scale_of(hb[0]);
        T.sR = scale_of(hb[1]);
        return GBFMM_OK;
    };
    rc = run();
    cleanup();
    if (rc) return rc;
    T.bases_ok = 1;
    return GBFMM_OK;
}

int svd_operators(gbfmm_ctx *ctx, const int *d_off, const int *d_lo, int n_off) {
    TcPlan &T = ctx->tc;
    const int p = ctx->opt.p, P3 = p * p * p, nt = 6 * P3, ns = 9 * P3;
    const int r1 = T.r1, r2 = T.r2, Np = T.Np, Kp = T.Kp, nc = chunk_offsets(p);
    cudaStream_t st = ctx->stream;
    if (int rc = ensure_blas(ctx)) return rc;
    cublasHandle_t h = (cublasHandle_t)T.blas;
    const size_t n_c = size_t(n_off) * Np * Kp;
    double *Tb = nullptr, *Z = nullptr, *C = nullptr;
    unsigned long long *d_mx = nullptr;
    auto cleanup = [&]() {
        cudaFree(Tb);
        cudaFree(Z);
        cudaFree(C);
        cudaFree(d_mx);
    };
    if (cudaMalloc(&Tb, size_t(nc) * nt * ns * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Z, size_t(nc) * r2 * nt * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&C, n_c * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_mx, sizeof(unsigned long long)) != cudaSuccess) {
        cleanup();
        return set_err(ctx, GBFMM_ERR_CUDA, "SVD operators: out of device memory");
    }
    auto run = [&]() -> int {
        CK(cudaMemsetAsync(C, 0, n_c * sizeof(double), st));  // the padding rows and columns stay zero
        CK(cudaMemsetAsync(d_mx, 0, sizeof(unsigned long long), st));
        const double one = 1.0, zero = 0.0;
        for (int o0 = 0; o0 < n_off; o0 += nc) {
            const int m = std::min(nc, n_off - o0);
            ++ctx->launches;
            k_node_ops<<<nblk(int64_t(m) * P3 * P3, 128), 128, 0, st>>>(p, ctx->opt.nodes, o0, m, d_off, ctx->d_mat,
                                                                         ctx->d_Asym, ctx->lat_n, ctx->d_Klat, Tb);
            CK(cudaGetLastError());
            // Z_o^T = R^T T_o^T (r2 x nt): T_o read column-major is T_o^T (ns x nt)
            BL(cublasDgemmStridedBatched(h, CUBLAS_OP_T, CUBLAS_OP_N, r2, nt, ns, &one, T.R64, ns, 0, Tb, ns,
                                         (long long)nt * ns, &zero, Z, r2, (long long)r2 * nt, m));
            // C_o^T = Z_o^T U (r2 x r1), column-major with leading dimension Kp: C_o row-major [Np][Kp]
            BL(cublasDgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, r2, r1, nt, &one, Z, r2, (long long)r2 * nt,
                                         T.U64, nt, 0, &zero, C + size_t(o0) * Np * Kp, Kp, (long long)Np * Kp, m));
        }
        T.op_scale = 1.0;
        if (T.fp16) {
            // one power of two for all operators: the largest entry maps below 2^14
            ++ctx->launches;
            k_absmax<<<1024, 256, 0, st>>>(int64_t(n_c), C, d_mx);
            unsigned long long bits = 0;
            CK(cudaMemcpyAsync(&bits, d_mx, sizeof(bits), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double mx = 0.0;
            std::memcpy(&mx, &bits, sizeof(mx));
            if (mx > 0.0) {
                int e = 0;
                std::frexp(mx, &e);
                T.op_scale = std::ldexp(1.0, 14 - e);
            }
        }
        ++ctx->launches;
        const unsigned g = nblk(int64_t(n_c), 256);
        if (T.tf32)
            k_ops_convert<float><<<g, 256, 0, st>>>(int64_t(n_c), Np, Kp, T.Kp_lo, C, d_lo, 1.0, (float *)T.Thi,
                                                    (float *)nullptr);
        else if (T.fp16)
            k_ops_convert<__half><<<g, 256, 0, st>>>(int64_t(n_c), Np, Kp, T.Kp_lo, C, d_lo, T.op_scale,
                                                     (__half *)T.Thi, (__half *)T.Tlo);
        else
            k_ops_convert<__nv_bfloat16><<<g, 256, 0, st>>>(int64_t(n_c), Np, Kp, T.Kp_lo, C, d_lo, 1.0,
                                                            (__nv_bfloat16 *)T.Thi, (__nv_bfloat16 *)T.Tlo);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        return GBFMM_OK;
    };
    const int rc = run();
    cleanup();
    return rc;
}

// per-tree scale slots: the W transforms of levels 0..MAXLEV-1, the S transforms of the same
// levels, and the children's compressed multipole values of the adaptive tree
constexpr int kFineSlot = 2 * GB_TC_MAXLEV;
constexpr int kScaleSlots = 2 * GB_TC_MAXLEV + 1;

static int split_level(gbfmm_ctx *ctx, const float *src, int64_t rows, int n, int ldx, int slot, float sbasis);

// adaptive tree: the (target child, source child) pairs of the children's M2L, grouped by
// operator.  The children of a split leaf meet the children of the split leaves around it
// that are not adjacent to them at the children's level (the interaction list one level
// below the leaves, restricted to children of split leaves; offset = target - source).
// pass 0 counts the pairs of every operator, pass 1 writes them from the scanned counts.
__global__ void k_fine_pairs(int pass, int64_t n_fine, int L, const int *__restrict__ n_ref,
                             const int *__restrict__ ref_leaf, const int *__restrict__ ref_start,
                             const int *__restrict__ child_start, const int *__restrict__ op_of,
                             int *__restrict__ cnt, const int *__restrict__ first, int *__restrict__ cur,
                             int2 *__restrict__ pairs) {
    const int64_t f = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (f >= n_fine) return;
    const int r = int(f >> 3), c = int(f & 7);
    if (r >= *n_ref || child_start[9 * r + c + 1] == child_start[9 * r + c]) return;
    const int nl = 1 << (L - 1);
    const int A = ref_leaf[r];
    const int ax = A % nl, ay = (A / nl) % nl, az = A / (nl * nl);
    const int tx = 2 * ax + (c & 1), ty = 2 * ay + ((c >> 1) & 1), tz = 2 * az + (c >> 2);
    for (int nb = 0; nb < 27; ++nb) {
        if (nb == 13) continue;  // siblings are adjacent to each other
        const int bx = ax + nb % 3 - 1, by = ay + (nb / 3) % 3 - 1, bz = az + nb / 9 - 1;
        if (bx < 0 || by < 0 || bz < 0 || bx >= nl || by >= nl || bz >= nl) continue;
        const int B = (bz * nl + by) * nl + bx;
        if (ref_start[B + 1] == ref_start[B]) continue;
        const int rB = ref_start[B];
        for (int c2 = 0; c2 < 8; ++c2) {
            if (child_start[9 * rB + c2 + 1] == child_start[9 * rB + c2]) continue;
            const int ox = tx - (2 * bx + (c2 & 1)), oy = ty - (2 * by + ((c2 >> 1) & 1)),
                      oz = tz - (2 * bz + (c2 >> 2));
            if (max(abs(ox), max(abs(oy), abs(oz))) < 2) continue;
            const int i = op_of[((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3)];
            if (pass == 0)
                atomicAdd(&cnt[i], 1);
            else
                pairs[first[i] + atomicAdd(&cur[i], 1)] = make_int2(int(f), 8 * rB + c2);
        }
    }
}

// the source rows of pairs [p0, p0 + n): FP16 hi (Kp values) and lo (the leading Kp_lo)
__global__ void k_fine_gather(int64_t n, const int2 *__restrict__ pairs, int Kp, int Kp_lo,
                              const __half *__restrict__ Xh, const __half *__restrict__ Xl, __half *__restrict__ Gh,
                              __half *__restrict__ Gl) {
    const int64_t total = n * (Kp + Kp_lo);
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = idx / (Kp + Kp_lo);
        const int k = int(idx - row * (Kp + Kp_lo));
        const int64_t src = pairs[row].y;
        if (k < Kp)
            Gh[row * Kp + k] = Xh[src * Kp + k];
        else
            Gl[row * Kp_lo + (k - Kp)] = Xl[src * Kp + (k - Kp)];
    }
}

// target children's compressed local values += the products of one operator's pairs, times
// the level factor (2^L / H)^2 of the children's cells (each target once per operator)
__global__ void k_fine_scatter(int64_t n, const int2 *__restrict__ pairs, const float *__restrict__ Y, int Np,
                               int r1, int L, const TreeBox *__restrict__ box, float *__restrict__ Sc7) {
    const double nh = double(1 << L) / box->H;
    const float lvl = float(nh * nh);
    const int64_t total = n * r1;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = idx / r1;
        const int k = int(idx - row * r1);
        Sc7[int64_t(pairs[row].x) * r1 + k] += Y[row * Np + k] * lvl;
    }
}

// The children's M2L of the adaptive tree (Algorithm 2's M2L one level below the leaves,
// between children of split leaves): their compressed multipole values split into FP16
// hi + lo with their own power of two, then per operator C_o the gathered source rows of its
// pairs as one GEMM (hi x hi over all of K, the residual products on the leading Kp_lo
// columns as in the tensor-core kernel), added to the target children's compressed local
// values operator by operator (a fixed order).  Reads the pair counts back to size the GEMMs.
int fine_m2l(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    auto &RF = ctx->rf;
    if (int rc = ensure_blas(ctx)) return rc;
    cudaStream_t st = ctx->stream;
    const int L = ctx->L, n_op = T.n_off;
    const int64_t n_fine = RF.fine_rows();
    if (!T.fp16 || n_op != 316)
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "adaptive tree: the children's M2L needs FP16 operands");
    if (n_fine == 0) return GBFMM_OK;
    const int *n_ref = RF.ref_start + ctx->n_leaves;
    if (!T.d_pcnt) {
        CK(cudaMalloc(&T.d_pcnt, (343 + 316 + 317 + 316) * sizeof(int)));
        int op_of[343];
        for (int oi = 0, i = 0; oi < 343; ++oi) {
            const int ox = oi % 7 - 3, oy = (oi / 7) % 7 - 3, oz = oi / 49 - 3;
            op_of[oi] = std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) >= 2 ? i++ : -1;
        }
        CK(cudaMemcpy(T.d_pcnt, op_of, sizeof(op_of), cudaMemcpyHostToDevice));
    }
    int *op_of = T.d_pcnt, *cnt = T.d_pcnt + 343, *first = cnt + 316, *cur = first + 317;
    CK(cudaMemsetAsync(cnt, 0, 316 * sizeof(int), st));
    CK(cudaMemsetAsync(cur, 0, 316 * sizeof(int), st));
    CK(cudaMemsetAsync(RF.Sc7, 0, size_t(n_fine) * T.r1 * sizeof(float), st));
    ++ctx->launches;
    k_fine_pairs<<<nblk(n_fine, 128), 128, 0, st>>>(0, n_fine, L, n_ref, RF.ref_leaf, RF.ref_start, RF.child_start,
                                                    op_of, cnt, nullptr, nullptr, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(T.h_pcnt, cnt, 316 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    T.h_pfirst[0] = 0;
    int64_t biggest = 0;
    for (int i = 0; i < 316; ++i) {
        T.h_pfirst[i + 1] = T.h_pfirst[i] + T.h_pcnt[i];
        biggest = std::max<int64_t>(biggest, T.h_pcnt[i]);
    }
    const int64_t total = T.h_pfirst[316];
    if (total == 0) return GBFMM_OK;
    if (int rc = grow_dev(ctx, T.pair_cap, total, {{(void **)&T.d_pairs, size_t(total) * sizeof(int2)}},
                          "adaptive-tree M2L pairs"))
        return rc;
    CK(cudaMemcpyAsync(first, T.h_pfirst, 317 * sizeof(int), cudaMemcpyHostToDevice, st));
    ++ctx->launches;
    k_fine_pairs<<<nblk(n_fine, 128), 128, 0, st>>>(1, n_fine, L, n_ref, RF.ref_leaf, RF.ref_start, RF.child_start,
                                                    op_of, nullptr, first, cur, T.d_pairs);
    CK(cudaGetLastError());
    // the children's values in FP16 (operator scale folded into alpha)
    const int Kp = T.Kp, Kp_lo = T.Kp_lo, Np = T.Np;
    if (int rc = split_level(ctx, RF.Wc7, n_fine, T.r2, Kp, kFineSlot, float(T.op_scale))) return rc;
    // runs of consecutive operators of at most `run` pairs (at least the largest operator's)
    const int64_t run = std::max<int64_t>(biggest, int64_t(1) << 19);
    if (int rc = grow_dev(ctx, T.g_cap, run,
                          {{&T.Gh, size_t(run) * Kp * sizeof(__half)},
                           {&T.Gl, size_t(run) * std::max(Kp_lo, 1) * sizeof(__half)},
                           {(void **)&T.Yf, size_t(run) * Np * sizeof(float)}},
                          "adaptive-tree M2L operands"))
        return rc;
    cublasHandle_t h = (cublasHandle_t)T.blas;
    const float *alpha = T.d_scal + 2 + kFineSlot, *zero = T.d_scal, *one = T.d_scal + 1;
    const __half *Thi = static_cast<const __half *>(T.Thi), *Tlo = static_cast<const __half *>(T.Tlo);
    __half *Gh = static_cast<__half *>(T.Gh), *Gl = static_cast<__half *>(T.Gl);
    BL(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_DEVICE));
    auto gemm = [&](int k, const __half *A, int lda, const __half *B, int ldb, const float *beta, float *C,
                    int n) -> int {
        const cublasStatus_t e = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, Np, n, k, alpha, A, CUDA_R_16F, lda, B,
                                              CUDA_R_16F, ldb, beta, C, CUDA_R_32F, Np, CUBLAS_COMPUTE_32F,
                                              CUBLAS_GEMM_DEFAULT);
        if (e == CUBLAS_STATUS_SUCCESS) return GBFMM_OK;
        cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST);
        return set_err(ctx, GBFMM_ERR_CUDA, "cuBLAS adaptive-tree M2L GEMM: " + std::to_string(int(e)));
    };
    for (int i0 = 0; i0 < 316;) {
        int i1 = i0;
        while (i1 < 316 && T.h_pfirst[i1 + 1] - T.h_pfirst[i0] <= run) ++i1;
        const int64_t p0 = T.h_pfirst[i0], np = T.h_pfirst[i1] - p0;
        if (np > 0) {
            ++ctx->launches;
            k_fine_gather<<<unsigned(std::min<int64_t>(nblk(np * (Kp + Kp_lo), 256), 16 * 152)), 256, 0, st>>>(
                np, T.d_pairs + p0, Kp, Kp_lo, static_cast<const __half *>(T.Xh), static_cast<const __half *>(T.Xl),
                Gh, Gl);
            CK(cudaGetLastError());
        }
        for (int i = i0; i < i1; ++i) {
            const int n = T.h_pcnt[i];
            if (n == 0) continue;
            const int64_t row = T.h_pfirst[i] - p0;
            float *Y = T.Yf + row * Np;
            // Y^T (Np x n) = C_o (Np x Kp, row-major) W'^T (Kp x n)
            if (int rc = gemm(Kp, Thi + size_t(i) * Np * Kp, Kp, Gh + row * Kp, Kp, zero, Y, n)) return rc;
            if (T.lo_host[i] >= 0 && Kp_lo > 0) {
                if (int rc = gemm(Kp_lo, Tlo + size_t(T.lo_host[i]) * Np * Kp_lo, Kp_lo, Gh + row * Kp, Kp, one, Y, n))
                    return rc;
                if (int rc = gemm(Kp_lo, Thi + size_t(i) * Np * Kp, Kp, Gl + row * Kp_lo, Kp_lo, one, Y, n))
                    return rc;
            }
            ++ctx->launches;
            k_fine_scatter<<<unsigned(std::min<int64_t>(nblk(int64_t(n) * T.r1, 256), 8 * 152)), 256, 0, st>>>(
                n, T.d_pairs + T.h_pfirst[i], Y, Np, T.r1, L, ctx->d_box, RF.Sc7);
            CK(cudaGetLastError());
        }
        i0 = i1;
    }
    BL(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
    return GBFMM_OK;
}

int svd_prepare(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    auto &RF = ctx->rf;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p;
    const int64_t per = std::max(T.r1, T.r2);
    // rows of every M2L level (the adaptive tree's children keep compact arrays)
    const int64_t rows = cell_base(ctx->L);
    if (int rc = grow_dev(ctx, T.c_cap, rows * per,
                          {{(void **)&T.Wc, size_t(rows) * per * sizeof(float)},
                           {(void **)&T.Sc, size_t(rows) * per * sizeof(float)}},
                          "compressed M2L values"))
        return rc;
    const int64_t n_fine = RF.on ? 8 * RF.cap_ref : 0;
    if (RF.on)
        if (int rc = grow_dev(ctx, RF.cap_cells, n_fine * (15 * P3 + T.r1 + T.r2),
                              {{(void **)&RF.W7, size_t(n_fine) * 9 * P3 * sizeof(float)},
                               {(void **)&RF.S7, size_t(n_fine) * 6 * P3 * sizeof(float)},
                               {(void **)&RF.Wc7, size_t(n_fine) * T.r2 * sizeof(float)},
                               {(void **)&RF.Sc7, size_t(n_fine) * T.r1 * sizeof(float)}},
                              "adaptive-tree children"))
            return rc;
    // one level's transform input split into FP16 hi + lo (the deepest level, or the children)
    const int64_t xrow = std::max<int64_t>(pad8(9 * P3), T.r1);
    const int64_t need = std::max<int64_t>(int64_t(1) << (3 * (ctx->L - 1)), n_fine) * xrow;
    if (int rc = grow_dev(ctx, T.x_cap, need,
                          {{&T.Xh, size_t(need) * sizeof(__half)}, {&T.Xl, size_t(need) * sizeof(__half)}},
                          "compressed M2L transform operands"))
        return rc;
    if (!T.d_scal) CK(cudaMalloc(&T.d_scal, (2 + kScaleSlots) * sizeof(float)));
    if (!T.d_bits) CK(cudaMalloc(&T.d_bits, kScaleSlots * sizeof(unsigned)));
    const float consts[2] = {0.f, 1.f};
    CK(cudaMemcpyAsync(T.d_scal, consts, sizeof(consts), cudaMemcpyHostToDevice, ctx->stream));
    return ensure_blas(ctx);
}

// Y (m x rows, ld ldy, FP32) = alpha (Ah^T|Ah) (Xh + Xl) + Al (Xh): the product of an FP16-split
// basis and an FP16-split operand on the tensor cores with FP32 accumulation, hi*hi + hi*lo + lo*hi
// (the lo*lo term is below FP32 rounding); alpha, 0 and 1 are device scalars
static int split_gemm(gbfmm_ctx *ctx, cublasOperation_t opA, int m, int64_t rows, int k, const void *Ah,
                      const void *Al, int lda, int ldx, const float *alpha, float *Y, int ldy) {
    TcPlan &T = ctx->tc;
    cublasHandle_t h = (cublasHandle_t)T.blas;
    const float *zero = T.d_scal, *one = T.d_scal + 1;
    const void *A[3] = {Ah, Ah, Al}, *X[3] = {T.Xh, T.Xl, T.Xh};
    BL(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_DEVICE));
    for (int t = 0; t < 3; ++t) {
        const cublasStatus_t st = cublasGemmEx(h, opA, CUBLAS_OP_N, m, int(rows), k, alpha, A[t], CUDA_R_16F, lda, X[t],
                                               CUDA_R_16F, ldx, t ? one : zero, Y, CUDA_R_32F, ldy, CUBLAS_COMPUTE_32F,
                                               CUBLAS_GEMM_DEFAULT);
        if (st != CUBLAS_STATUS_SUCCESS) {
            cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST);
            return set_err(ctx, GBFMM_ERR_CUDA, "cuBLAS FP16 transform GEMM: " + std::to_string(int(st)));
        }
    }
    BL(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
    return GBFMM_OK;
}

// One level's rows [rows][n] of src (FP32) into the FP16 split with its own power-of-two scale
static int split_level(gbfmm_ctx *ctx, const float *src, int64_t rows, int n, int ldx, int slot, float sbasis) {
    TcPlan &T = ctx->tc;
    cudaStream_t st = ctx->stream;
    const int64_t cnt = rows * n;
    const unsigned g = unsigned(std::min<int64_t>(nblk(cnt, 256), 8 * 152));
    CK(cudaMemsetAsync(T.d_bits + slot, 0, sizeof(unsigned), st));
    ctx->launches += 2;
    k_absmax_f32<<<g, 256, 0, st>>>(cnt, src, T.d_bits + slot);
    k_split_f16<<<unsigned(std::min<int64_t>(nblk(rows * ldx, 256), 16 * 152)), 256, 0, st>>>(
        rows, n, ldx, src, T.d_bits + slot, sbasis, (__half *)T.Xh, (__half *)T.Xl, T.d_scal + 2 + slot);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

int svd_transform_w(gbfmm_ctx *ctx, const float *Wf, bool fine) {
    TcPlan &T = ctx->tc;
    auto &RF = ctx->rf;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p, ns = 9 * P3, lds = pad8(ns);
    if (int rc = ensure_blas(ctx)) return rc;
    // W'^T (r2 x cells) = R^T (r2 x 9 p^3) W^T (9 p^3 x cells), level by level (each its own scale)
    for (int l = 2; l < ctx->L; ++l) {
        const int64_t row0 = cell_base(l), rows = int64_t(1) << (3 * l);
        if (int rc = split_level(ctx, Wf + row0 * ns, rows, ns, lds, l, T.sR)) return rc;
        if (int rc = split_gemm(ctx, CUBLAS_OP_T, T.r2, rows, lds, T.Rh, T.Rl, lds, lds, T.d_scal + 2 + l,
                                T.Wc + row0 * T.r2, T.r2))
            return rc;
    }
    if (fine) {
        // the children of split leaves, in their compact rows (fine_m2l reads them there)
        const int l = ctx->L;
        const int64_t n_fine = RF.fine_rows();
        if (int rc = split_level(ctx, RF.W7, n_fine, ns, lds, l, T.sR)) return rc;
        if (int rc = split_gemm(ctx, CUBLAS_OP_T, T.r2, n_fine, lds, T.Rh, T.Rl, lds, lds, T.d_scal + 2 + l, RF.Wc7,
                                T.r2))
            return rc;
    }
    return GBFMM_OK;
}

int svd_expand_s(gbfmm_ctx *ctx, float *Sf, bool fine) {
    TcPlan &T = ctx->tc;
    auto &RF = ctx->rf;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p, nt = 6 * P3;
    if (int rc = ensure_blas(ctx)) return rc;
    // S^T (6 p^3 x cells) = U (6 p^3 x r1) S'^T (r1 x cells), level by level
    for (int l = 2; l < ctx->L; ++l) {
        const int64_t row0 = cell_base(l), rows = int64_t(1) << (3 * l);
        if (int rc = split_level(ctx, T.Sc + row0 * T.r1, rows, T.r1, T.r1, GB_TC_MAXLEV + l, T.sU)) return rc;
        if (int rc = split_gemm(ctx, CUBLAS_OP_N, nt, rows, T.r1, T.Uh, T.Ul, pad8(nt), T.r1,
                                T.d_scal + 2 + GB_TC_MAXLEV + l, Sf + row0 * nt, nt))
            return rc;
    }
    if (fine) {
        // the children's compressed local values (fine_m2l), expanded into S7
        const int l = ctx->L;
        const int64_t n_fine = RF.fine_rows();
        if (int rc = split_level(ctx, RF.Sc7, n_fine, T.r1, T.r1, GB_TC_MAXLEV + l, T.sU)) return rc;
        if (int rc = split_gemm(ctx, CUBLAS_OP_N, nt, n_fine, T.r1, T.Uh, T.Ul, pad8(nt), T.r1,
                                T.d_scal + 2 + GB_TC_MAXLEV + l, RF.S7, nt))
            return rc;
    }
    return GBFMM_OK;
}

void svd_free(gbfmm_ctx *ctx, bool borrowed) {
    TcPlan &T = ctx->tc;
    if (T.blas) cublasDestroy((cublasHandle_t)T.blas);
    void *mine[] = {T.Wc, T.Sc, T.blas_ws, T.Xh, T.Xl, T.d_scal, T.d_bits, T.d_pcnt, T.d_pairs, T.Gh, T.Gl, T.Yf};
    for (void *q : mine)
        if (q) cudaFree(q);
    if (!borrowed) {
        void *tabs[] = {T.Uf, T.Rf, T.U64, T.R64, T.Uh, T.Ul, T.Rh, T.Rl};
        for (void *q : tabs)
            if (q) cudaFree(q);
    }
    T.blas = T.blas_ws = nullptr;
    T.Wc = T.Sc = nullptr;
    T.Xh = T.Xl = nullptr;
    T.d_scal = nullptr;
    T.d_bits = nullptr;
    T.Uf = T.Rf = nullptr;
    T.U64 = T.R64 = nullptr;
    T.Uh = T.Ul = T.Rh = T.Rl = nullptr;
    T.c_cap = 0;
    T.x_cap = 0;
    T.d_pcnt = nullptr;
    T.d_pairs = nullptr;
    T.Gh = T.Gl = nullptr;
    T.Yf = nullptr;
    T.pair_cap = T.g_cap = 0;
    T.bases_ok = 0;
}
