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
// DSYRK and DGEMM, cuSOLVER's symmetric eigensolver); the per-pass
// transforms are plain FP32 GEMMs (cuBLAS, FP32 accuracy from the BF16x9
// emulation on the tensor cores where available).
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
        // per-pass transforms: FP32 GEMMs emulated on the tensor cores where cuBLAS can
        BL(cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER));
    }
    BL(cublasSetStream((cublasHandle_t)T.blas, ctx->stream));
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
        CK(cudaStreamSynchronize(st));
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

int svd_prepare(gbfmm_ctx *ctx) {
    TcPlan &T = ctx->tc;
    const int64_t per = std::max(T.r1, T.r2);
    if (int rc = grow_dev(ctx, T.c_cap, ctx->n_cells * per,
                          {{(void **)&T.Wc, size_t(ctx->n_cells) * per * sizeof(float)},
                           {(void **)&T.Sc, size_t(ctx->n_cells) * per * sizeof(float)}},
                          "compressed M2L values"))
        return rc;
    if (int rc = ensure_blas(ctx)) return rc;
    if (!T.gemm_emulated) {
        // does this cuBLAS run FP32 GEMMs as BF16x9 emulation on this device?  A small
        // product on the (allocated) buffers settles it once, outside any graph capture
        const float one = 1.f, zero = 0.f;
        const cublasStatus_t s =
            cublasGemmEx((cublasHandle_t)T.blas, CUBLAS_OP_N, CUBLAS_OP_N, 16, 16, 16, &one, T.Wc, CUDA_R_32F, 16,
                         T.Wc, CUDA_R_32F, 16, &zero, T.Sc, CUDA_R_32F, 16, CUBLAS_COMPUTE_32F_EMULATED_16BFX9,
                         CUBLAS_GEMM_DEFAULT);
        T.gemm_emulated = s == CUBLAS_STATUS_SUCCESS ? 1 : -1;
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return GBFMM_OK;
}

static cublasComputeType_t f32_compute(const TcPlan &T) {
    return T.gemm_emulated > 0 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F;
}

int svd_transform_w(gbfmm_ctx *ctx, const float *Wf) {
    TcPlan &T = ctx->tc;
    const int L = ctx->L, P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p, ns = 9 * P3;
    const int64_t base = cell_base(2), rows = cell_base(L) - base;
    if (rows <= 0) return GBFMM_OK;
    if (int rc = ensure_blas(ctx)) return rc;
    const float one = 1.f, zero = 0.f;
    // W'^T (r2 x cells) = R^T (r2 x 9 p^3) W^T (9 p^3 x cells): every cell of levels 2 .. L-1
    BL(cublasGemmEx((cublasHandle_t)T.blas, CUBLAS_OP_T, CUBLAS_OP_N, T.r2, int(rows), ns, &one, T.Rf, CUDA_R_32F,
                    ns, Wf + base * ns, CUDA_R_32F, ns, &zero, T.Wc + base * T.r2, CUDA_R_32F, T.r2, f32_compute(T),
                    CUBLAS_GEMM_DEFAULT));
    return GBFMM_OK;
}

int svd_expand_s(gbfmm_ctx *ctx, float *Sf) {
    TcPlan &T = ctx->tc;
    const int L = ctx->L, P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p, nt = 6 * P3;
    const int64_t base = cell_base(2), rows = cell_base(L) - base;
    if (rows <= 0) return GBFMM_OK;
    if (int rc = ensure_blas(ctx)) return rc;
    const float one = 1.f, zero = 0.f;
    // S^T (6 p^3 x cells) = U (6 p^3 x r1) S'^T (r1 x cells)
    BL(cublasGemmEx((cublasHandle_t)T.blas, CUBLAS_OP_N, CUBLAS_OP_N, nt, int(rows), T.r1, &one, T.Uf, CUDA_R_32F,
                    nt, T.Sc + base * T.r1, CUDA_R_32F, T.r1, &zero, Sf + base * nt, CUDA_R_32F, nt, f32_compute(T),
                    CUBLAS_GEMM_DEFAULT));
    return GBFMM_OK;
}

void svd_free(gbfmm_ctx *ctx, bool borrowed) {
    TcPlan &T = ctx->tc;
    if (T.blas) cublasDestroy((cublasHandle_t)T.blas);
    void *mine[] = {T.Wc, T.Sc, T.blas_ws};
    for (void *q : mine)
        if (q) cudaFree(q);
    if (!borrowed) {
        void *tabs[] = {T.Uf, T.Rf, T.U64, T.R64};
        for (void *q : tabs)
            if (q) cudaFree(q);
    }
    T.blas = T.blas_ws = nullptr;
    T.Wc = T.Sc = nullptr;
    T.Uf = T.Rf = nullptr;
    T.U64 = T.R64 = nullptr;
    T.c_cap = 0;
    T.bases_ok = 0;
}
