// FP64 M2L through the Toeplitz structure of the operators (Sec. 4.1,
// Theorem 1; the M2L stage of Algorithm 2).
//
// For an offset o (target cell B = source cell A + o, in cell units of the
// level) the local value at node l of B is
//     S_B[l][ab] = (2^lev / H)^2 sum_m sum_wr K_o[l - m][ab][wr] W_A[m][wr],
// K_o[d] = Klat[o (p - 1) + d] on the unit-cell node-difference lattice,
// d in [-(p-1), p-1]^3: a linear convolution over the p^3 nodes.  Embedded
// in a periodic grid of N = 2p points per axis (d < 0 at N + d, index p
// unused) it becomes a circular convolution, diagonal in the discrete
// Fourier basis:
//     S^_B[f][ab] = sum_o sum_wr K^_o[f][ab][wr] W^_{B-o}[f][wr],
// and S_B = inverse transform of S^_B restricted to [0, p)^3.  The inputs are
// real, so only fx = 0 .. p is kept (N N (p + 1) frequencies, NF); the
// inverse weights fx = 1 .. p-1 twice.  Per cell pair that is 54 NF complex
// multiply-adds (54 x 1008 at p = 6) instead of 54 p^6 real ones.
//
// Kernels: k_fft_ops transforms the 54 kernel components of every offset
// once per medium; per level, k_fft_slots numbers the occupied cells,
// k_fft_w transforms their 9 multipole components, and k_m2l_fft (one block
// per target cell) accumulates S^ over the interaction list in a fixed order
// (three stress components per sweep, thread per frequency) and transforms
// it back.  Every transform is a separable pass per axis over a shared
// table of the N roots of unity.
//
// Symmetry reduction (gbfmm_options.m2l_symmetry; Sec. 6): in a medium
// invariant under a signed permutation g of the axes (g_{i pi(i)} = s_i) the
// kernel obeys K(g d) = det(g) rho(g) K(d), rho(g) acting on the stress pair
// ab and the strength pair wr as (rho K)[ab][wr] = s_a s_b s_w s_r
// K[pi(a) pi(b)][pi(w) pi(r)] (det(g): the permutation symbol of the kernel).
// Every offset o is g rep for one of 16 representatives (components sorted,
// non-negative), node differences map by g, so the transforms obey
//     K^_o[f] = det(g) rho(g) K^_rep[g^T f],   (g^T f)_j = s_i f_i, pi(i) = j,
// frequencies mod N; where (g^T f)_x > p the half spectrum holds the
// conjugate at -(g^T f).  The table keeps the 16 representatives (316/16 times
// smaller) and k_m2l_fft reads each offset's entries from its
// representative's at the permuted frequency, with permuted, signed components.
#include <algorithm>
#include <cmath>
#include <string>

#include "cube_sym.h"
#include "internal.cuh"
#include "m2l_fft.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return unsigned(std::min<int64_t>((n + b - 1) / b, int64_t(1) << 30)); }

__device__ __forceinline__ void cell_xyz_f(int64_t lin, int n, int &x, int &y, int &z) {
    x = int(lin % n);
    y = int((lin / n) % n);
    z = int(lin / (int64_t(n) * n));
}

// tw[k] = exp(-2 pi i k / N)
__device__ __forceinline__ void load_twiddles(int N, double2 *tw) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * double(k) / double(N), &s, &c);
        tw[k] = make_double2(c, -s);
    }
}

__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {  // acc += a b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void rmac(double2 &acc, double a, double2 b) {  // acc += a b, a real
    acc.x = fma(a, b.x, acc.x);
    acc.y = fma(a, b.y, acc.y);
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

// Forward transform of a real array a[z][y][x] (x, y, z < sup, row stride sup;
// zero elsewhere in [0, N)^3) to the half spectrum out[(fz N + fy) NH + fx].
// A1: sup sup NH, A2: sup N NH complex (shared).  Ends with the block synchronised.
__device__ void fwd3(int N, int NH, int sup, const double *a, double2 *A1, double2 *A2, const double2 *tw,
                     double2 *out) {
    for (int t = threadIdx.x; t < sup * sup * NH; t += blockDim.x) {
        const int fx = t % NH, zy = t / NH;
        double2 s = make_double2(0.0, 0.0);
        for (int x = 0; x < sup; ++x) rmac(s, a[zy * sup + x], tw[(fx * x) % N]);
        A1[t] = s;  // [z][y][fx]
    }
    __syncthreads();
    for (int t = threadIdx.x; t < sup * N * NH; t += blockDim.x) {
        const int fx = t % NH, fy = (t / NH) % N, z = t / (NH * N);
        double2 s = make_double2(0.0, 0.0);
        for (int y = 0; y < sup; ++y) cmac(s, A1[(z * sup + y) * NH + fx], tw[(fy * y) % N]);
        A2[t] = s;  // [z][fy][fx]
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N * N * NH; t += blockDim.x) {
        const int fx = t % NH, fy = (t / NH) % N, fz = t / (NH * N);
        double2 s = make_double2(0.0, 0.0);
        for (int z = 0; z < sup; ++z) cmac(s, A2[(z * N + fy) * NH + fx], tw[(fz * z) % N]);
        out[t] = s;  // [fz][fy][fx]
    }
    __syncthreads();
}

// Inverse of a half spectrum Sh[(fz N + fy) NH + fx] at the nodes [0, p)^3
// (without the 1 / N^3): s[(z p + y) p + x].  B1: p N NH, B2: p p NH complex.
__device__ void inv3(int N, int NH, int p, const double2 *Sh, double2 *B1, double2 *B2, const double2 *tw,
                     double *s_out) {
    for (int t = threadIdx.x; t < p * N * NH; t += blockDim.x) {
        const int fx = t % NH, fy = (t / NH) % N, z = t / (NH * N);
        double2 s = make_double2(0.0, 0.0);
        for (int fz = 0; fz < N; ++fz) cmac(s, Sh[(fz * N + fy) * NH + fx], conj2(tw[(fz * z) % N]));
        B1[t] = s;  // [z][fy][fx]
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p * p * NH; t += blockDim.x) {
        const int fx = t % NH, y = (t / NH) % p, z = t / (NH * p);
        double2 s = make_double2(0.0, 0.0);
        for (int fy = 0; fy < N; ++fy) cmac(s, B1[(z * N + fy) * NH + fx], conj2(tw[(fy * y) % N]));
        B2[t] = s;  // [z][y][fx]
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p * p * p; t += blockDim.x) {
        const int x = t % p, zy = t / p;
        double s = 0.0;
        for (int fx = 0; fx < NH; ++fx) {
            const double2 b = B2[zy * NH + fx], w = conj2(tw[(fx * x) % N]);
            const double re = b.x * w.x - b.y * w.y;
            s += (fx == 0 || fx == NH - 1) ? re : 2.0 * re;
        }
        s_out[t] = s;
    }
    __syncthreads();
}


// Transformed kernel components of every offset o with max |o_i| >= 2:
// block (table slot, comp); slot = oi = ((oz + 3) 7 + (oy + 3)) 7 + (ox + 3), or
// with reps the slot's representative.
__global__ void __launch_bounds__(256) k_fft_ops(int p, int lat_n, const double *__restrict__ Klat,
                                                 double2 *__restrict__ Khat, int use_reps, cube_sym::RepList reps) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int N = 2 * p, NH = p + 1, NF = N * N * NH;
    double2 *tw = reinterpret_cast<double2 *>(sm_raw);
    double2 *A1 = tw + N;
    double2 *A2 = A1 + N * N * NH;
    double *a = reinterpret_cast<double *>(A2 + N * N * NH);
    const int slot = blockIdx.x / 54, comp = blockIdx.x % 54;
    const int oi = use_reps ? reps.oi[slot] : slot;
    const int ox = oi % 7 - 3, oy = (oi / 7) % 7 - 3, oz = oi / 49 - 3;
    if (max(abs(ox), max(abs(oy), abs(oz))) < 2) return;
    const int R0 = (lat_n - 1) / 2;
    load_twiddles(N, tw);
    for (int t = threadIdx.x; t < N * N * N; t += blockDim.x) {
        const int ix = t % N, iy = (t / N) % N, iz = t / (N * N);
        double v = 0.0;
        if (ix != p && iy != p && iz != p) {
            const int dx = ix < p ? ix : ix - N, dy = iy < p ? iy : iy - N, dz = iz < p ? iz : iz - N;
            const int Dx = ox * (p - 1) + dx + R0, Dy = oy * (p - 1) + dy + R0, Dz = oz * (p - 1) + dz + R0;
            v = Klat[((int64_t(Dz) * lat_n + Dy) * lat_n + Dx) * 54 + comp];
        }
        a[t] = v;
    }
    __syncthreads();
    fwd3(N, NH, N, a, A1, A2, tw, Khat + (int64_t(slot) * 54 + comp) * NF);
}

// Slots of the occupied cells of one level
__global__ void k_fft_slots(int lev, const int *__restrict__ occ, int *__restrict__ slot, int *__restrict__ slot_cell,
                            int *__restrict__ count) {
    const int64_t cells = int64_t(1) << (3 * lev), base = cell_base_d(lev);
    for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < cells; c += int64_t(gridDim.x) * blockDim.x) {
        int s = -1;
        if (occ[base + c] > 0) {
            s = atomicAdd(count, 1);
            slot_cell[s] = int(c);
        }
        slot[c] = s;
    }
}

// Transformed multipole values W^[slot][wr][f] of the occupied cells of one level
__global__ void __launch_bounds__(256) k_fft_w(int p, int lev, const double *__restrict__ W,
                                               const int *__restrict__ slot_cell, double2 *__restrict__ What) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int N = 2 * p, NH = p + 1, NF = N * N * NH, P3 = p * p * p;
    double2 *tw = reinterpret_cast<double2 *>(sm_raw);
    double2 *A1 = tw + N;
    double2 *A2 = A1 + p * p * NH;
    double *a = reinterpret_cast<double *>(A2 + p * N * NH);
    const int s = blockIdx.x;
    const int64_t g = cell_base_d(lev) + slot_cell[s];
    load_twiddles(N, tw);
    for (int wr = 0; wr < 9; ++wr) {
        for (int m = threadIdx.x; m < P3; m += blockDim.x) a[m] = W[(g * P3 + m) * 9 + wr];
        __syncthreads();
        fwd3(N, NH, p, a, A1, A2, tw, What + (int64_t(s) * 9 + wr) * NF);
    }
}

// One block per cell of the level: S for the cells with targets (SYM: Khat holds the 16
// representatives, osym and gmap map each offset onto one)
template <bool SYM>
__global__ void __launch_bounds__(256) k_m2l_fft(int p, int lev, const TreeBox *__restrict__ box,
                                                 const int *__restrict__ tocc, const int *__restrict__ slot,
                                                 const double2 *__restrict__ Khat, const double2 *__restrict__ What,
                                                 double *__restrict__ S, const int *__restrict__ osym,
                                                 const unsigned char *__restrict__ gmap) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int N = 2 * p, NH = p + 1, NF = N * N * NH, P3 = p * p * p;
    double2 *tw = reinterpret_cast<double2 *>(sm_raw);
    double2 *Sh = tw + N;             // [3][NF]
    double2 *B1 = Sh + 3 * NF;        // [p][N][NH]
    double2 *B2 = B1 + p * N * NH;    // [p][p][NH]
    double *sout = reinterpret_cast<double *>(B2 + p * p * NH);  // [p^3]
    __shared__ int s_src[216], s_oi[216];
    __shared__ unsigned char s_gmap[SYM ? 48 * 60 : 4];
    const int n = 1 << lev;
    const int64_t g = cell_base_d(lev) + blockIdx.x;
    if (tocc[g] == 0) return;
    int bx, by, bz;
    cell_xyz_f(blockIdx.x, n, bx, by, bz);
    load_twiddles(N, tw);
    if (SYM)
        for (int t = threadIdx.x; t < 48 * 60; t += blockDim.x) s_gmap[t] = gmap[t];
    // interaction list in a fixed order: children of the parent's 27 neighbours
    // that are not neighbours of B and hold sources
    for (int c = threadIdx.x; c < 216; c += blockDim.x) {
        const int nb = c / 8, ch = c % 8;
        const int px = bx / 2 + nb % 3 - 1, py = by / 2 + (nb / 3) % 3 - 1, pz = bz / 2 + nb / 9 - 1;
        const int ax = 2 * px + (ch & 1), ay = 2 * py + ((ch >> 1) & 1), az = 2 * pz + (ch >> 2);
        int src = -1, oi = 0;
        if (ax >= 0 && ay >= 0 && az >= 0 && ax < n && ay < n && az < n) {
            const int ox = bx - ax, oy = by - ay, oz = bz - az;
            if (max(abs(ox), max(abs(oy), abs(oz))) >= 2) {
                src = slot[(int64_t(az) * n + ay) * n + ax];
                oi = ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3);
                if (SYM) oi = osym[oi];  // representative | map << 8
            }
        }
        s_src[c] = src;
        s_oi[c] = oi;
    }
    __syncthreads();
    const double sc = double(n) / box->H;
    const double scale = sc * sc / double(N * N * N);
    for (int grp = 0; grp < 2; ++grp) {  // stress components 3 grp .. 3 grp + 2
        for (int f = threadIdx.x; f < NF; f += blockDim.x) {
            double2 acc[3];
            for (int k = 0; k < 3; ++k) acc[k] = make_double2(0.0, 0.0);
            for (int c = 0; c < 216; ++c) {
                const int src = s_src[c];
                if (src < 0) continue;
                const double2 *wv = What + int64_t(src) * 9 * NF + f;
                double2 w[9];
#pragma unroll
                for (int wr = 0; wr < 9; ++wr) w[wr] = wv[int64_t(wr) * NF];
                if (SYM) {
                    // the representative's entries at g^T f, components permuted and signed
                    const int code = s_oi[c];
                    const unsigned char *gm = s_gmap + (code >> 8) * 60;
                    const int fv[3] = {f % NH, (f / NH) % N, f / (NH * N)};
                    int f2[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int a = gm[54 + j], v = fv[a & 3];
                        f2[j] = (a & 4) ? (v ? N - v : 0) : v;
                    }
                    const bool cj = f2[0] > p;  // stored as the conjugate at -(g^T f)
                    if (cj)
#pragma unroll
                        for (int j = 0; j < 3; ++j) f2[j] = f2[j] ? N - f2[j] : 0;
                    const double2 *kb = Khat + int64_t(code & 255) * 54 * NF + (f2[2] * N + f2[1]) * NH + f2[0];
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int wr = 0; wr < 9; ++wr) {
                            const int cc = gm[27 * grp + 9 * k + wr];
                            const double2 v = kb[int64_t(cc & 63) * NF];
                            const bool neg = (cc & 64) != 0;
                            cmac(acc[k], make_double2(neg ? -v.x : v.x, (neg != cj) ? -v.y : v.y), w[wr]);
                        }
                } else {
                    const double2 *kv = Khat + (int64_t(s_oi[c]) * 54 + 27 * grp) * NF + f;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int wr = 0; wr < 9; ++wr) cmac(acc[k], kv[int64_t(k * 9 + wr) * NF], w[wr]);
                }
            }
            for (int k = 0; k < 3; ++k) Sh[k * NF + f] = acc[k];
        }
        __syncthreads();
        for (int k = 0; k < 3; ++k) {
            inv3(N, NH, p, Sh + k * NF, B1, B2, tw, sout);
            for (int t = threadIdx.x; t < P3; t += blockDim.x) S[(g * P3 + t) * 6 + 3 * grp + k] = sout[t] * scale;
            __syncthreads();
        }
    }
}

}  // namespace

int m2l_fft_run(gbfmm_ctx *ctx, const int *occ, const int *tocc) {
    FftPlan &F = ctx->fft;
    const int p = ctx->opt.p, L = ctx->L;
    const int N = 2 * p, NH = p + 1, NF = N * N * NH, P3 = p * p * p;
    cudaStream_t st = ctx->stream;
    if (L < 3) return GBFMM_OK;
    const bool sym = ctx->opt.m2l_symmetry == 1;
    cube_sym::RepList reps{};
    if (!F.ready || F.p != p || F.sym != sym) {
        F.ready = false;
        if (F.Khat) cudaFree(F.Khat);
        F.Khat = nullptr;
        int n_tab = 343;
        if (sym) {
            if (!cube_sym::cube_invariant(ctx->mat.C))
                return set_err(ctx, GBFMM_ERR_INVALID_ARG,
                               "m2l_symmetry: the medium lacks the cube's symmetries (isotropic, or cubic with "
                               "axes along x, y, z)");
            int osym[343];
            unsigned char gmap[48 * 60];
            cube_sym::sym_tables(reps, osym, gmap);
            if (!F.d_osym) CK(cudaMalloc(&F.d_osym, sizeof(osym)));
            if (!F.d_gmap) CK(cudaMalloc(&F.d_gmap, sizeof(gmap)));
            CK(cudaMemcpyAsync(F.d_osym, osym, sizeof(osym), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(F.d_gmap, gmap, sizeof(gmap), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));  // the host tables are locals
            n_tab = 16;
        }
        CK(cudaMalloc(&F.Khat, size_t(n_tab) * 54 * NF * sizeof(double2)));
        const size_t sm = size_t(N) * sizeof(double2) + 2 * size_t(N) * N * NH * sizeof(double2) +
                          size_t(N) * N * N * sizeof(double);
        CK(cudaFuncSetAttribute(k_fft_ops, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        ++ctx->launches;
        k_fft_ops<<<unsigned(n_tab * 54), 256, sm, st>>>(p, ctx->lat_n, ctx->d_Klat, F.Khat, sym ? 1 : 0, reps);
        CK(cudaGetLastError());
        F.ready = true;
        F.p = p;
        F.sym = sym;
    }
    const int64_t max_cells = int64_t(1) << (3 * (L - 1));
    if (int rc = grow_dev(ctx, F.cell_cap, max_cells,
                          {{(void **)&F.slot, max_cells * sizeof(int)}, {(void **)&F.slot_cell, max_cells * sizeof(int)}},
                          "M2L transform slots"))
        return rc;
    if (!F.count) CK(cudaMalloc(&F.count, sizeof(int)));
    const size_t sm_w = size_t(N) * sizeof(double2) + size_t(p) * p * NH * sizeof(double2) +
                        size_t(p) * N * NH * sizeof(double2) + size_t(P3) * sizeof(double);
    const size_t sm_a = size_t(N) * sizeof(double2) + 3 * size_t(NF) * sizeof(double2) +
                        size_t(p) * N * NH * sizeof(double2) + size_t(p) * p * NH * sizeof(double2) +
                        size_t(P3) * sizeof(double);
    CK(cudaFuncSetAttribute(k_fft_w, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_w)));
    auto kern = sym ? k_m2l_fft<true> : k_m2l_fft<false>;
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm_a)));
    for (int lev = 2; lev < L; ++lev) {
        const int64_t cells = int64_t(1) << (3 * lev);
        CK(cudaMemsetAsync(F.count, 0, sizeof(int), st));
        ctx->launches += 1;
        k_fft_slots<<<nblk(cells, 256), 256, 0, st>>>(lev, occ, F.slot, F.slot_cell, F.count);
        CK(cudaGetLastError());
        int cnt = 0;
        CK(cudaMemcpyAsync(&cnt, F.count, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (int rc = grow_dev(ctx, F.what_cap, cnt, {{(void **)&F.What, size_t(cnt) * 9 * NF * sizeof(double2)}},
                              "transformed multipole values"))
            return rc;
        if (cnt > 0) {
            ++ctx->launches;
            k_fft_w<<<unsigned(cnt), 256, sm_w, st>>>(p, lev, ctx->d_W, F.slot_cell, F.What);
            CK(cudaGetLastError());
        }
        ++ctx->launches;
        kern<<<unsigned(cells), 256, sm_a, st>>>(p, lev, ctx->d_box, tocc, F.slot, F.Khat, F.What, ctx->d_S,
                                                 F.d_osym, F.d_gmap);
        CK(cudaGetLastError());
    }
    return GBFMM_OK;
}

void m2l_fft_free(gbfmm_ctx *ctx) {
    FftPlan &F = ctx->fft;
    void *ps[] = {F.Khat, F.What, F.slot, F.slot_cell, F.count, F.d_osym, F.d_gmap};
    for (void *q : ps)
        if (q) cudaFree(q);
    F = FftPlan{};
}
