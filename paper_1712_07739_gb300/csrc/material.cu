// Elastic medium, the contraction A of Sec. 2 Eq. "kernel", and the
// precomputed M2L node kernels of Sec. 4.1 Eq. "m2l".
//
// Theorem 1 says the node kernel of an offset o depends only on l - m; with
// the cell size factored out (homogeneity of degree -2, Sec. 4.1 footnote)
// every entry of every one of the 316 operators is K at one point of the
// integer lattice D = o (p-1) + (l - m), |D_i| <= 4 (p-1), scaled by
// 1/(p-1).  The table d_Klat holds K at all of those points for a unit
// cell; the FP64 M2L reads it directly and the tensor-core M2L expands it
// into dense per-offset operators.
#include <cmath>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "kernel_math.cuh"

namespace {

int levi(int i, int j, int k) { return ((i - j) * (j - k) * (k - i)) / 2; }

// C_ijkl from the 6x6 Voigt matrix (11, 22, 33, 23, 13, 12)
void voigt_to_full(const double *V, double *C) {
    auto vi = [](int i, int j) {
        if (i == j) return i;
        if ((i == 1 && j == 2) || (i == 2 && j == 1)) return 3;
        if ((i == 0 && j == 2) || (i == 2 && j == 0)) return 4;
        return 5;
    };
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) C[((i * 3 + j) * 3 + k) * 3 + l] = V[vi(i, j) * 6 + vi(k, l)];
}

// Positive definiteness of the strain-energy form: Cholesky of the Mandel
// matrix (Voigt with shear rows/columns scaled by sqrt 2).
bool positive_definite(const double *V) {
    double M[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            M[i * 6 + j] = V[i * 6 + j] * (i >= 3 ? std::sqrt(2.0) : 1.0) * (j >= 3 ? std::sqrt(2.0) : 1.0);
    for (int j = 0; j < 6; ++j) {
        double d = M[j * 6 + j];
        for (int k = 0; k < j; ++k) d -= M[j * 6 + k] * M[j * 6 + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        M[j * 6 + j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double s = M[i * 6 + j];
            for (int k = 0; k < j; ++k) s -= M[i * 6 + k] * M[j * 6 + k];
            M[i * 6 + j] = s / d;
        }
    }
    return true;
}

// K at every lattice point D (unit cell, node spacing 1/(p-1)):
// K[ab][wr] = sum_k Asym[ab][wr][k] h_k(D/|D|) / |D/(p-1)|^2
__global__ void k_lattice(const DevMaterial *mat, const double *Asym, int p, int lat_n, double *Klat) {
    int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    int64_t total = int64_t(lat_n) * lat_n * lat_n;
    if (idx >= total) return;
    int R0 = (lat_n - 1) / 2;
    int dx = int(idx % lat_n) - R0;
    int dy = int((idx / lat_n) % lat_n) - R0;
    int dz = int(idx / (int64_t(lat_n) * lat_n)) - R0;
    const double s = 1.0 / double(p - 1);
    const double d[3] = {dx * s, dy * s, dz * s};
    kernel_at(mat, Asym, d, Klat + idx * 54);
}

}  // namespace

int material_setup(gbfmm_ctx *ctx) {
    const int p = ctx->opt.p;
    // A_{ab,wr,vpq} = sum_{n,g} eps_ngr C_abvg C_pqwn, folded over (v,p) <-> (p,v)
    const double *C = ctx->mat.C;
    static const int PV[6] = {0, 1, 2, 1, 0, 0}, PP[6] = {0, 1, 2, 2, 2, 1};
    for (int ab = 0; ab < 6; ++ab) {
        int a = voigt_a(ab), b = voigt_b(ab);
        for (int w = 0; w < 3; ++w)
            for (int r = 0; r < 3; ++r)
                for (int pr = 0; pr < 6; ++pr)
                    for (int q = 0; q < 3; ++q) {
                        double tot = 0.0;
                        for (int sym = 0; sym < 2; ++sym) {
                            int v = sym ? PP[pr] : PV[pr];
                            int pp = sym ? PV[pr] : PP[pr];
                            if (sym && v == pp) break;
                            double s = 0.0;
                            for (int n = 0; n < 3; ++n)
                                for (int g = 0; g < 3; ++g) {
                                    int e = levi(n, g, r);
                                    if (!e) continue;
                                    s += e * C[((a * 3 + b) * 3 + v) * 3 + g] * C[((pp * 3 + q) * 3 + w) * 3 + n];
                                }
                            tot += s;
                        }
                        ctx->Asym[(ab * 9 + w * 3 + r) * 18 + pr * 3 + q] = tot;
                    }
    }
    float Af[6 * 9 * 18];
    for (int i = 0; i < 6 * 9 * 18; ++i) Af[i] = float(ctx->Asym[i]);
    if (!ctx->d_mat) CK(cudaMalloc(&ctx->d_mat, sizeof(DevMaterial)));
    if (!ctx->d_Asym) CK(cudaMalloc(&ctx->d_Asym, sizeof(ctx->Asym)));
    if (!ctx->d_Asym_f) CK(cudaMalloc(&ctx->d_Asym_f, sizeof(Af)));
    CK(cudaMemcpyAsync(ctx->d_mat, &ctx->mat, sizeof(DevMaterial), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_Asym, ctx->Asym, sizeof(ctx->Asym), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_Asym_f, Af, sizeof(Af), cudaMemcpyHostToDevice, ctx->stream));

    int lat_n = 8 * (p - 1) + 1;
    int64_t total = int64_t(lat_n) * lat_n * lat_n;
    if (ctx->lat_n != lat_n) {
        if (ctx->d_Klat) cudaFree(ctx->d_Klat);
        ctx->d_Klat = nullptr;
        CK(cudaMalloc(&ctx->d_Klat, total * 54 * sizeof(double)));
        ctx->lat_n = lat_n;
    }
    ++ctx->launches;
    k_lattice<<<unsigned((total + 127) / 128), 128, 0, ctx->stream>>>(ctx->d_mat, ctx->d_Asym, p, lat_n, ctx->d_Klat);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return GBFMM_OK;
}

// Use src's medium tables (kernel lattice, M2L operators) without copying:
// contexts of one batch share them.  dst must not outlive src.
int share_material(gbfmm_ctx *ctx, const gbfmm_ctx *src) {
    if (!src->have_material) return set_err(ctx, GBFMM_ERR_NO_MATERIAL, "share_material: source has no material");
    if (ctx->opt.p != src->opt.p || ctx->opt.precision != src->opt.precision || ctx->opt.h_mode != src->opt.h_mode ||
        ctx->opt.m2l_split != src->opt.m2l_split || ctx->opt.m2l_basis != src->opt.m2l_basis ||
        ctx->opt.m2l_split_kblocks != src->opt.m2l_split_kblocks || ctx->opt.m2l_kernel != src->opt.m2l_kernel ||
        ctx->opt.nodes != src->opt.nodes || ctx->opt.m2l_svd_tol != src->opt.m2l_svd_tol)
        return set_err(ctx, GBFMM_ERR_INVALID_ARG, "share_material: options differ");
    ctx->mat = src->mat;
    std::memcpy(ctx->Asym, src->Asym, sizeof(ctx->Asym));
    ctx->d_mat = src->d_mat;
    ctx->d_Asym = src->d_Asym;
    ctx->d_Asym_f = src->d_Asym_f;
    ctx->d_Klat = src->d_Klat;
    ctx->lat_n = src->lat_n;
    TcPlan &T = ctx->tc;
    const TcPlan &S = src->tc;
    T.ready_ops = S.ready_ops;
    T.Kp = S.Kp;
    T.Kp_lo = S.Kp_lo;
    T.Np = S.Np;
    T.nsub = S.nsub;
    T.ncta = S.ncta;
    T.groups = S.groups;
    T.swap = S.swap;
    T.tpc = S.tpc;
    T.nblk = S.nblk;
    T.tmem_cols = S.tmem_cols;
    T.n_off = S.n_off;
    T.n_lo = S.n_lo;
    T.split = S.split;
    T.tf32 = S.tf32;
    T.fp16 = S.fp16;
    T.op_scale = S.op_scale;
    std::memcpy(T.lo_host, S.lo_host, sizeof(T.lo_host));
    T.modal = S.modal;
    std::memcpy(T.basisV, S.basisV, sizeof(T.basisV));
    std::memcpy(T.basisCt, S.basisCt, sizeof(T.basisCt));
    T.esz = S.esz;
    T.Thi = S.Thi;
    T.Tlo = S.Tlo;
    // compressed M2L: the bases are shared, the per-tree buffers and the cuBLAS handle are not
    T.svd = S.svd;
    T.r1 = S.r1;
    T.r2 = S.r2;
    T.r1_raw = S.r1_raw;
    T.r2_raw = S.r2_raw;
    T.Uf = S.Uf;
    T.Rf = S.Rf;
    T.U64 = S.U64;
    T.R64 = S.R64;
    T.bases_ok = S.bases_ok;
    T.Uh = S.Uh;
    T.Ul = S.Ul;
    T.Rh = S.Rh;
    T.Rl = S.Rl;
    T.sU = S.sU;
    T.sR = S.sR;
    std::memcpy(T.svd_sigma, S.svd_sigma, sizeof(T.svd_sigma));
    if (!T.d_status) {
        CK(cudaMalloc(&T.d_status, sizeof(int)));
        CK(cudaMemset(T.d_status, 0, sizeof(int)));
    }
    if (T.fp16 && !T.d_wmax) CK(cudaMalloc(&T.d_wmax, GB_TC_MAXLEV * sizeof(unsigned)));
    ctx->borrowed_material = true;
    ctx->have_material = true;
    return GBFMM_OK;
}

extern "C" int fmm_set_material(gbfmm_ctx *ctx, const double *V) {
    if (!ctx) return GBFMM_ERR_INVALID_ARG;
    if (ctx->borrowed_material) {
        // stop sharing: this context builds its own tables from here on
        ctx->d_mat = nullptr;
        ctx->d_Asym = nullptr;
        ctx->d_Asym_f = nullptr;
        ctx->d_Klat = nullptr;
        ctx->lat_n = 0;
        ctx->tc.Thi = ctx->tc.Tlo = nullptr;
        ctx->tc.Uf = ctx->tc.Rf = nullptr;
        ctx->tc.U64 = ctx->tc.R64 = nullptr;
        ctx->tc.Uh = ctx->tc.Ul = ctx->tc.Rh = ctx->tc.Rl = nullptr;
        ctx->tc.ready_ops = false;
        ctx->fft.ready = false;
        ctx->borrowed_material = false;
    }
    if (!V) return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_set_material: null stiffness");
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            if (!std::isfinite(V[i * 6 + j]) || std::fabs(V[i * 6 + j] - V[j * 6 + i]) > 1e-12 * std::fabs(V[i * 6 + j]) + 1e-300)
                return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_set_material: stiffness not symmetric/finite");
    if (!positive_definite(V)) return set_err(ctx, GBFMM_ERR_DEGENERATE, "fmm_set_material: stiffness not positive definite");
    DevMaterial m{};
    voigt_to_full(V, m.C);
    {
        // cubic with axes along x, y, z: C11 = C22 = C33, C12 = C13 = C23, C44 = C55 = C66, rest 0
        const double c11 = V[0], c12 = V[1], c44 = V[21];
        const double sc = std::fabs(c11) + std::fabs(c12) + std::fabs(c44);
        bool cub = true;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double want = 0.0;
                if (i < 3 && j < 3) want = (i == j) ? c11 : c12;
                if (i >= 3 && i == j) want = c44;
                if (std::fabs(V[i * 6 + j] - want) > 1e-14 * sc) cub = false;
            }
        m.cubic = cub ? 1 : 0;
        m.c12 = c12;
        m.c44 = c44;
        m.cd = c11 - c12 - 2.0 * c44;
    }
    m.mode = ctx->opt.h_mode;
    m.Q = ctx->opt.circle_q > 0 ? ctx->opt.circle_q : 64;
    if (m.mode == GBFMM_H_ISO) {
        double c11 = V[0], c12 = V[1], c44 = V[21];
        double scale = std::fabs(c11) + std::fabs(c12) + std::fabs(c44);
        bool cubic = true;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 6; ++j) {
                double want = (j < 3) ? (i == j ? c11 : c12) : 0.0;
                if (std::fabs(V[i * 6 + j] - want) > 1e-12 * scale) cubic = false;
            }
        for (int i = 3; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double want = (i == j) ? c44 : 0.0;
                if (std::fabs(V[i * 6 + j] - want) > 1e-12 * scale) cubic = false;
            }
        if (!cubic || std::fabs(c11 - c12 - 2.0 * c44) > 1e-12 * scale)
            return set_err(ctx, GBFMM_ERR_INVALID_ARG, "fmm_set_material: GBFMM_H_ISO needs an isotropic stiffness");
        double mu = c44, nu = c12 / (2.0 * (c12 + c44));
        m.hc = 1.0 / (16.0 * M_PI * mu * (1.0 - nu));
        m.ha = 3.0 - 4.0 * nu;
    }
    ctx->mat = m;
    ctx->fft.ready = false;  // the transformed operators belong to the previous medium
    ctx->tc.ready_ops = false;
    ctx->tc.bases_ok = 0;
    int rc = material_setup(ctx);
    if (rc) return rc;
    ctx->have_material = true;
    return GBFMM_OK;
}
