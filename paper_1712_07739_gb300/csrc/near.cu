// Near field (the direct sum over neighbouring leaves in Algorithm 2) and L2P of the mixed-
// precision pass: one warp per target leaf.
//
// For a source point j the kernel contraction of Sec. 2 Eq. "stress3",
// s_ab += sum_wr K_abwr(x - y_j) q_j,wr, is folded once per source into
// P_j[ab][k] = sum_wr Asym[ab][wr][k] q_j,wr, so a pair costs
// s_ab += sum_k P_j[ab][k] h_k(T) / R^2 (k over the 18 distinct h
// components).  Since q_j = (omega_g / 2) b (x S), P_j is the segment's
// tensor scaled by the point's Gauss weight.
//
// Isotropic medium: h is the odd cubic polynomial of Sec. 2 Eq. "k_iso"
// differentiated, h_vpq = c [-a d_vp T_q + d_vq T_p + d_pq T_v - 3 T_v T_p T_q],
// so sum_k P[ab][k] h_k(T) / R^2 = (lin_ab . d) / R^3 + (cub_ab . d^(3)) / R^5
// with d = x - y, 3 linear and 10 cubic-monomial coefficients per ab
// (78 per source, an exact rewrite).  Other media keep the 108 entries of P
// and evaluate h by the unit-circle rule in FP32.
//
// Precision: positions enter as FP32 offsets from their own leaf centre, so
// a separation carries the rounding of leaf-sized numbers, not of the box
// size; pairs closer than near_fp64 x (source segment length) take their
// separation from the FP64 positions and are summed apart in extended
// precision (FP64 in the one-sided kernels, two-float in the symmetric one).
#include <cmath>

#include "internal.cuh"
#include "kernel_math.cuh"
#include "mlp_warp.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

__device__ __forceinline__ void cell_xyz3(int64_t lin, int n, int &x, int &y, int &z) {
    x = int(lin % n);
    y = int((lin / n) % n);
    z = int(lin / (int64_t(n) * n));
}

// cubic monomials d_i d_j d_k, i <= j <= k
__host__ __device__ constexpr int mono_index(int i, int j, int k) {
    // sorted triple -> 0..9 in the order 000 001 002 011 012 022 111 112 122 222
    return (i == 0) ? ((j == 0) ? k : (j == 1 ? 2 + k : 5)) : ((i == 1) ? (j == 1 ? 5 + k : 8) : 9);
}

template <typename R>
__device__ __forceinline__ void monomials(const R d[3], R m[10]) {
    const R a00 = d[0] * d[0], a01 = d[0] * d[1], a02 = d[0] * d[2];
    const R a11 = d[1] * d[1], a12 = d[1] * d[2], a22 = d[2] * d[2];
    m[0] = a00 * d[0];
    m[1] = a00 * d[1];
    m[2] = a00 * d[2];
    m[3] = a11 * d[0];
    m[4] = a01 * d[2];
    m[5] = a22 * d[0];
    m[6] = a11 * d[1];
    m[7] = a11 * d[2];
    m[8] = a22 * d[1];
    m[9] = a22 * d[2];
    (void)a02;
    (void)a12;
}

// Per-source coefficient tensors of the isotropic polynomial form, 80 per
// point (78 used, padded for 16-byte rows): 3 linear and 10 cubic-monomial
// coefficients per stress component, from P = sum_wr A q formed in FP32
// (nine terms per entry; the near field reads FP32 coefficients, and FP64
// arithmetic runs at a small fraction of the FP32 rate on this part).
__global__ void k_src_coef80(int64_t N, const double *__restrict__ q, const double *__restrict__ Asym, float hc,
                             float ha, float *__restrict__ c32) {
    __shared__ float As[6 * 9 * 18];
    for (int i = threadIdx.x; i < 6 * 9 * 18; i += blockDim.x) As[i] = float(Asym[i]);
    __syncthreads();
    const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (j >= N) return;
    float qq[9];
    for (int i = 0; i < 9; ++i) qq[i] = float(q[9 * j + i]);
    constexpr int PV[6] = {0, 1, 2, 1, 0, 0}, PP[6] = {0, 1, 2, 2, 2, 1};
    for (int ab = 0; ab < 6; ++ab) {
        float P[18];
        for (int k = 0; k < 18; ++k) {
            float s = 0.f;
            for (int wr = 0; wr < 9; ++wr) s = fmaf(As[(ab * 9 + wr) * 18 + k], qq[wr], s);
            P[k] = s;
        }
        float lin[3] = {0, 0, 0}, cub[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int pr = 0; pr < 6; ++pr) {
            const int v = PV[pr], p = PP[pr];
            for (int qd = 0; qd < 3; ++qd) {
                const float w = P[3 * pr + qd];
                if (v == p) lin[qd] += -ha * hc * w;
                if (v == qd) lin[p] += hc * w;
                if (p == qd) lin[v] += hc * w;
                int a = v, b = p, c = qd, t;
                if (a > b) { t = a; a = b; b = t; }
                if (b > c) { t = b; b = c; c = t; }
                if (a > b) { t = a; a = b; b = t; }
                cub[mono_index(a, b, c)] += -3.f * hc * w;
            }
        }
        for (int i = 0; i < 3; ++i) c32[j * 80 + ab * 13 + i] = lin[i];
        for (int i = 0; i < 10; ++i) c32[j * 80 + ab * 13 + 3 + i] = cub[i];
    }
    for (int i = 78; i < 80; ++i) c32[j * 80 + i] = 0.f;
}

// The 108-entry tensors P for 64 points per block: q staged in shared memory,
// consecutive threads compute and store consecutive entries (coalesced rows).
constexpr int kCoefPts = 64;
__global__ void __launch_bounds__(256) k_src_coef108(int64_t N, const double *__restrict__ q,
                                                     const double *__restrict__ Asym, float *__restrict__ c32) {
    __shared__ float As[6 * 9 * 18];
    __shared__ float sq[kCoefPts][9];
    for (int i = threadIdx.x; i < 6 * 9 * 18; i += blockDim.x) As[i] = float(Asym[i]);
    const int64_t j0 = blockIdx.x * int64_t(kCoefPts);
    const int np = int(min(int64_t(kCoefPts), N - j0));
    for (int i = threadIdx.x; i < np * 9; i += blockDim.x) (&sq[0][0])[i] = float(q[9 * j0 + i]);
    __syncthreads();
    for (int idx = threadIdx.x; idx < np * 108; idx += blockDim.x) {
        const int jl = idx / 108, e = idx - jl * 108, ab = e / 18, k = e - ab * 18;
        float acc = 0.f;
#pragma unroll
        for (int wr = 0; wr < 9; ++wr) acc = fmaf(As[(ab * 9 + wr) * 18 + k], sq[jl][wr], acc);
        c32[j0 * 108 + idx] = acc;
    }
}

template <typename R>
__device__ __forceinline__ void pair_iso(const R d[3], R ir, const R *c, R acc[6]) {
    const R ir2 = ir * ir, ir3 = ir * ir2, ir5 = ir3 * ir2;
    R m[10];
    monomials<R>(d, m);
#pragma unroll
    for (int ab = 0; ab < 6; ++ab) {
        const R *cc = c + ab * 13;
        const R l = cc[0] * d[0] + cc[1] * d[1] + cc[2] * d[2];
        R u = R(0);
#pragma unroll
        for (int i = 0; i < 10; ++i) u += cc[3 + i] * m[i];
        acc[ab] += ir3 * l + ir5 * u;
    }
}

// h models of the near kernel
constexpr int HM_ISO = 0, HM_CUBIC = 1, HM_GENERIC = 2;

template <int HM, typename R, typename CT>
__device__ __forceinline__ void pair_generic(const R d[3], R ir, const R *c, const CT *C, int Q, R c12, R c44, R cd,
                                             R acc[6], const float2 *tab = nullptr) {
    R T[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    R hs[18];
    if (HM == HM_CUBIC) {
        if constexpr (sizeof(R) == 4)
            h_cubic_f32(c12 + c44, c44, cd, Q, tab, T, hs);
        else
            h_circle_cubic<R>(c12, c44, cd, Q, T, hs);
    } else {
        h_circle_sym<R, CT>(C, Q, T, hs);
    }
    const R ir2 = ir * ir;
#pragma unroll
    for (int ab = 0; ab < 6; ++ab) {
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 18; ++k) s += c[ab * 18 + k] * hs[k];
        acc[ab] += s * ir2;
    }
}

constexpr int WARPS = 4;

// NCS: per-source coefficient stride (80 isotropic, 108 otherwise); SCH
// sources are staged per warp chunk (static shared memory stays < 48 KB)
template <int HM, int NCS, int SCH>
__global__ void __launch_bounds__(WARPS * 32) k_near_mixed(
    int p, int nodes, int L, int64_t nl, float near2, const TreeBox *__restrict__ box, const DevMaterial *__restrict__ mat,
    const int *__restrict__ tstart, const double *__restrict__ xt, const int64_t *__restrict__ tsid,
    const int *__restrict__ sstart, const float4 *__restrict__ yrel, const double *__restrict__ ys,
    const float *__restrict__ c32, const int64_t *__restrict__ ssid,
    const float *__restrict__ S, double *__restrict__ sig, const int2 *__restrict__ items,
    const int *__restrict__ n_items) {
    __shared__ __align__(16) float sP[WARPS][SCH * NCS];
    __shared__ float4 sy[WARPS][SCH];
    __shared__ int ssd[WARPS][SCH];
    __shared__ float sC[81];
    __shared__ float2 sTab[128];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (HM == HM_GENERIC)
        for (int i = threadIdx.x; i < 81; i += blockDim.x) sC[i] = float(mat->C[i]);
    if (HM == HM_CUBIC)
        for (int i = threadIdx.x; i < mat->Q && i < 128; i += blockDim.x) {
            float sn, cs;
            sincospif(float(i) / float(mat->Q), &sn, &cs);
            sTab[i] = make_float2(cs, sn);
        }
    __syncthreads();
    // one work item per warp: up to 32 targets of one leaf, heaviest first
    const int64_t item = blockIdx.x * int64_t(WARPS) + warp;
    if (item >= *n_items) return;
    const int2 wi = items[item];
    const int64_t leaf = wi.x;
    const int t0 = wi.y, t1 = min(wi.y + 32, tstart[leaf + 1]);
    const int P3 = p * p * p;
    const int nlv = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz3(leaf, nlv, cx, cy, cz);
    const bool far = L >= 3;
    const double h = box->H / nlv, ih = double(nlv) / box->H;
    const double c0[3] = {box->origin[0] + cx * h, box->origin[1] + cy * h, box->origin[2] + cz * h};
    const int Q = mat->Q;
    const float c12f = float(mat->c12), c44f = float(mat->c44), cdf = float(mat->cd);
    const float *Sl = S + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 6;
    float *wP = sP[warp];
    float4 *wy = sy[warp];
    int *wsd = ssd[warp];
    for (int r0 = t0; r0 < t1; r0 += 32) {
        // tg targets in this pass, 32 / tg lanes per target splitting the sources
        const int nrem = min(32, t1 - r0);
        int tg = 1;
        while (tg < nrem) tg <<= 1;
        const int ls = 32 / tg, tl = lane % tg, ph = lane / tg;
        const int t = r0 + tl;
        const bool valid = tl < nrem;
        double x[3] = {0, 0, 0};
        float xr[3] = {0.f, 0.f, 0.f};
        float acc[6] = {0, 0, 0, 0, 0, 0};
        double acc64[6] = {0, 0, 0, 0, 0, 0};
        int myseg = -1;
        if (valid) {
            for (int d = 0; d < 3; ++d) {
                x[d] = xt[3 * int64_t(t) + d];
                xr[d] = float(x[d] - (c0[d] + 0.5 * h));
            }
            myseg = tsid ? int(tsid[t]) : -1;
        }
        if (far && ph == 0) {
            float bx[GB_MAXP], by[GB_MAXP], bz[GB_MAXP];
            lagrange_1d<float>(p, float((x[0] - c0[0]) * ih), bx, nodes);
            lagrange_1d<float>(p, float((x[1] - c0[1]) * ih), by, nodes);
            lagrange_1d<float>(p, float((x[2] - c0[2]) * ih), bz, nodes);
            for (int lz = 0; lz < p; ++lz)
                for (int ly = 0; ly < p; ++ly) {
                    const float wyz = by[ly] * bz[lz];
                    for (int lx = 0; lx < p; ++lx) {
                        const float w = bx[lx] * wyz;
                        const float *s6 = Sl + ((lz * p + ly) * p + lx) * 6;
                        for (int ab = 0; ab < 6; ++ab) acc[ab] += w * __ldg(s6 + ab);
                    }
                }
        }
        for (int nb = 0; nb < 27; ++nb) {
            const int dxn = nb % 3 - 1, dyn = (nb / 3) % 3 - 1, dzn = nb / 9 - 1;
            const int ax = cx + dxn, ay = cy + dyn, az = cz + dzn;
            if (ax < 0 || ay < 0 || az < 0 || ax >= nlv || ay >= nlv || az >= nlv) continue;
            const int64_t A = (int64_t(az) * nlv + ay) * nlv + ax;
            const int s0 = sstart[A], s1 = sstart[A + 1];
            const float xs[3] = {xr[0] - float(dxn * h), xr[1] - float(dyn * h), xr[2] - float(dzn * h)};
            for (int j0 = s0; j0 < s1; j0 += SCH) {
                const int nj = min(SCH, s1 - j0);
                __syncwarp();
                if (lane < nj) {
                    wy[lane] = yrel[j0 + lane];
                    wsd[lane] = int(ssid[j0 + lane]);
                }
                {
                    const float4 *src = reinterpret_cast<const float4 *>(c32 + int64_t(NCS) * j0);
                    float4 *dst = reinterpret_cast<float4 *>(wP);
                    const int nv = nj * NCS / 4;
                    for (int i = lane; i < nv; i += 32) dst[i] = __ldg(src + i);
                }
                __syncwarp();
                if (!valid) continue;
                for (int j = ph; j < nj; j += ls) {
                    if (wsd[j] == myseg) continue;
                    const float4 yj = wy[j];
                    float d[3] = {xs[0] - yj.x, xs[1] - yj.y, xs[2] - yj.z};
                    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    // A close pair takes its separation from the FP64 positions (the
                    // FP32 difference would cancel) and goes to its own FP64
                    // accumulator; the kernel itself is evaluated in FP32 on that
                    // separation, whose relative error is then ~1e-7.
                    const bool close = r2 < near2 * yj.w * yj.w;
                    float ir;
                    if (close) {
                        const int64_t jj = j0 + j;
                        const double dd0 = x[0] - ys[3 * jj], dd1 = x[1] - ys[3 * jj + 1], dd2 = x[2] - ys[3 * jj + 2];
                        const double rr = dd0 * dd0 + dd1 * dd1 + dd2 * dd2;
                        if (rr == 0.0) continue;
                        d[0] = float(dd0);
                        d[1] = float(dd1);
                        d[2] = float(dd2);
                        ir = float(rsqrt(rr));
                    } else {
                        ir = rsqrtf(r2);
                    }
                    float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    if (HM == HM_ISO)
                        pair_iso<float>(d, ir, wP + 80 * j, part);
                    else
                        pair_generic<HM, float, float>(d, ir, wP + 108 * j, sC, Q, c12f, c44f, cdf, part, sTab);
                    if (close) {
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) acc64[ab] += double(part[ab]);
                    } else {
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) acc[ab] += part[ab];
                    }
                }
            }
        }
        // fold the lanes that shared a target (fixed order: deterministic)
        for (int off = tg; off < 32; off <<= 1)
            for (int ab = 0; ab < 6; ++ab) {
                acc[ab] += __shfl_xor_sync(0xffffffffu, acc[ab], off);
                acc64[ab] += __shfl_xor_sync(0xffffffffu, acc64[ab], off);
            }
        if (valid && ph == 0)
            for (int ab = 0; ab < 6; ++ab) sig[6 * int64_t(t) + ab] = double(acc[ab]) + acc64[ab];
    }
}

// ---------------------------------------------------------------- symmetric near field
// Nodal forces (targets = sources): h is odd, h(-T) = -h(T), so one
// evaluation of h for the point pair (i, j) serves both directions,
//     s_i += P_j h(T_ij) / R^2   and   s_j -= P_i h(T_ij) / R^2.
// Work items are leaf pairs (A, B) with B = A + o over the 14 offsets o of
// the upper half of the 3 x 3 x 3 neighbourhood (o = 0 included: pairs j > i
// of one leaf).  Contributions are written to partial slots, one per point
// and neighbour direction (27 directions + the reverse half of the own
// leaf), each written by exactly one warp in a fixed order; the combine kernel
// adds the far field (L2P) and the slots in a fixed order.  Close pairs
// (closer than near_fp64 x the longer of the two segments) take their
// separation from the FP64 positions, where the cancellation is, and are
// summed apart from the other pairs in two-float (hi + lo) sums.
// One warp per block (a block's shared-memory slice is freed as soon as its leaf pair is
// done) and 12 resident blocks per SM (152 registers): at 1M segments, Q = 16, the near
// field took 195 ms against 204 ms with four warps per block at the same 12 warps per SM
// (there the slowest warp of a block held the other three slices).
constexpr int SYM_WARPS = 1, SYM_SCH = 8, SYM_MINB = 12;
constexpr int kSlots = 28;

// Two-float sums for the close pairs: the value is hi + lo, and each addition
// keeps its exact rounding error (Knuth's two-sum, six FP32 operations), so
// the sum of FP32 terms carries ~48 mantissa bits without FP64 arithmetic
// (FP64 runs at a small fraction of the FP32 rate on this part).
__device__ __forceinline__ void tsum(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}
__device__ __forceinline__ void tsum2(float &hi, float &lo, float bhi, float blo) {
    const float s = hi + bhi;
    const float bb = s - hi;
    lo += ((hi - (s - bb)) + (bhi - bb)) + blo;
    hi = s;
}

template <int HM>
__global__ void __launch_bounds__(SYM_WARPS * 32, SYM_MINB) k_near_sym(
    int L, float near2, const TreeBox *__restrict__ box, const DevMaterial *__restrict__ mat,
    const int *__restrict__ sstart, const float4 *__restrict__ yrel, const double *__restrict__ ys,
    const float *__restrict__ c32, const int64_t *__restrict__ ssid, double *__restrict__ part, int64_t N,
    const int2 *__restrict__ items, const int *__restrict__ n_items, const int *__restrict__ ref_start,
    const int *__restrict__ child_start) {
    extern __shared__ __align__(16) float sm_sym[];
    float *wPA = sm_sym + (threadIdx.x / 32) * (32 * 108 + SYM_SCH * 108);  // [32][108]: lanes' own tensors
    float *wPB = wPA + 32 * 108;                                            // [SCH][108] staged sources
    __shared__ float4 syB[SYM_WARPS][SYM_SCH];
    __shared__ int sdB[SYM_WARPS][SYM_SCH];
    __shared__ float saccB[SYM_WARPS][SYM_SCH][6];
    __shared__ float2 saccCB[SYM_WARPS][SYM_SCH][6];  // close pairs: two-float (hi, lo)
    __shared__ double sxB[SYM_WARPS][SYM_SCH][3];      // FP64 positions of the staged sources
    __shared__ float sC[81];
    __shared__ __align__(16) float2 sTab[128];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (HM == HM_GENERIC)
        for (int i = threadIdx.x; i < 81; i += blockDim.x) sC[i] = float(mat->C[i]);
    if (HM == HM_CUBIC)
        for (int i = threadIdx.x; i < mat->Q && i < 128; i += blockDim.x) {
            float sn, cs;
            sincospif(float(i) / float(mat->Q), &sn, &cs);
            sTab[i] = make_float2(cs, sn);
        }
    __syncthreads();
    const bool packed = (mat->Q & 1) == 0;  // two circle points per packed step
    const int64_t item = blockIdx.x * int64_t(SYM_WARPS) + warp;
    if (item >= *n_items) return;
    const int2 wi = items[item];
    const int64_t Aleaf = wi.x;
    const int d = wi.y;  // 0..13: neighbour index 13 + d
    const int nlv = 1 << (L - 1);
    int ax, ay, az;
    cell_xyz3(Aleaf, nlv, ax, ay, az);
    const int nb = 13 + d;
    const int ox = nb % 3 - 1, oy = (nb / 3) % 3 - 1, oz = nb / 9 - 1;
    const int64_t Bleaf = (int64_t(az + oz) * nlv + (ay + oy)) * nlv + (ax + ox);
    const bool self = d == 0;
    const int sA0 = sstart[Aleaf], sA1 = sstart[Aleaf + 1];
    const int sB0 = sstart[Bleaf], sB1 = sstart[Bleaf + 1];
    const int slot_f = nb, slot_r = self ? 27 : 26 - nb;
    const double h = box->H / nlv;
    // B's leaf-relative positions, seen from A's leaf centre
    const float bsh[3] = {float(ox * h), float(oy * h), float(oz * h)};
    const int Q = mat->Q;
    const float c12f = float(mat->c12), c44f = float(mat->c44), cdf = float(mat->cd);
    bool first_chunk = true;
    // adaptive tree: two different split leaves interact through their adjacent children
    // only (the others through the M2L one level down): the targets go child by child and
    // each target child meets the children of B adjacent to it
    int rA = -1, rB = -1;
    if (ref_start && !self) {
        if (ref_start[Aleaf + 1] > ref_start[Aleaf]) rA = ref_start[Aleaf];
        if (ref_start[Bleaf + 1] > ref_start[Bleaf]) rB = ref_start[Bleaf];
    }
    const bool fine = rA >= 0 && rB >= 0;
    if (fine) {
        // B's reverse slots then collect several target children: they start from zero
        for (int k = lane; k < (sB1 - sB0) * 6; k += 32)
            part[(int64_t(slot_r) * N + sB0 + k / 6) * 6 + k % 6] = 0.0;
        __syncwarp();
    }
    for (int ts = 0; ts < (fine ? 8 : 1); ++ts) {
    const int tA0 = fine ? child_start[9 * rA + ts] : sA0, tA1 = fine ? child_start[9 * rA + ts + 1] : sA1;
    for (int r0 = tA0, nrem = 0; r0 < tA1; r0 += nrem) {
        // nrem targets in this chunk on tg lanes (a power of two), 32 / tg lanes per
        // target splitting the sources.  A chunk costs max(1, tg / 4) warp steps per
        // 8 sources, so the targets left are cut into power-of-two chunks where that
        // is cheaper than rounding them up (20 targets: 16 + 4, five steps instead
        // of eight; 30 targets: one chunk of 32)
        const int left = tA1 - r0;
        const int tg = left >= 29 ? 32 : left >= 13 ? 16 : left >= 5 ? 8 : left >= 3 ? 4 : left;
        nrem = min(tg, left);
        const int ls = 32 / tg, ti = lane % tg, tj = lane / tg;
        const int i = r0 + ti;
        const bool vi = i < tA1;
        // stage the lanes' own source tensors, one 432-byte row per target: the
        // 16-byte reads of 8 consecutive rows fall in 8 different bank quads
        __syncwarp();
        {
            const float4 *src = reinterpret_cast<const float4 *>(c32 + int64_t(108) * r0);
            float4 *dst = reinterpret_cast<float4 *>(wPA);
            for (int k = lane; k < nrem * 27; k += 32) dst[k] = __ldg(src + k);
        }
        __syncwarp();
        float4 yi = make_float4(0.f, 0.f, 0.f, 0.f);
        double xi[3] = {0.0, 0.0, 0.0};
        int segi = -2;
        if (vi) {
            yi = yrel[i];
            xi[0] = ys[3 * int64_t(i)], xi[1] = ys[3 * int64_t(i) + 1], xi[2] = ys[3 * int64_t(i) + 2];
            segi = int(ssid[i]);
        }
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float accC[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, accCl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // close pairs
        const float4 *Pi4 = reinterpret_cast<const float4 *>(wPA + 108 * ti);
        for (int ss = 0; ss < (fine ? 8 : 1); ++ss) {
        int jb0 = self ? r0 : sB0, jb1 = sB1;  // own leaf: pairs j > i only
        if (fine) {
            // B's child ss against A's child ts: adjacent at the children's level?
            const int dx = 2 * ox + (ss & 1) - (ts & 1), dy = 2 * oy + ((ss >> 1) & 1) - ((ts >> 1) & 1),
                      dz = 2 * oz + (ss >> 2) - (ts >> 2);
            if (abs(dx) > 1 || abs(dy) > 1 || abs(dz) > 1) continue;
            jb0 = child_start[9 * rB + ss];
            jb1 = child_start[9 * rB + ss + 1];
        }
        for (int j0 = jb0; j0 < jb1; j0 += SYM_SCH) {
            const int nj = min(SYM_SCH, jb1 - j0);
            __syncwarp();
            if (lane < nj) {
                syB[warp][lane] = yrel[j0 + lane];
                sdB[warp][lane] = int(ssid[j0 + lane]);
            }
            for (int k = lane; k < nj * 3; k += 32) (&sxB[warp][0][0])[k] = ys[3 * int64_t(j0) + k];
            for (int k = lane; k < SYM_SCH * 6; k += 32) {
                (&saccB[warp][0][0])[k] = 0.f;
                (&saccCB[warp][0][0])[k] = make_float2(0.f, 0.f);
            }
            {
                const float4 *src = reinterpret_cast<const float4 *>(c32 + int64_t(108) * j0);
                float4 *dst = reinterpret_cast<float4 *>(wPB);
                for (int k = lane; k < nj * 27; k += 32) dst[k] = __ldg(src + k);
            }
            __syncwarp();
            for (int jj = 0; jj < nj; jj += ls) {
                const int jl = jj + tj;  // this lane's source within the chunk
                const int j = j0 + jl;
                bool on = vi && jl < nj && (!self || j > i);
                float4 yj = make_float4(0.f, 0.f, 0.f, 1.f);
                if (on) {
                    yj = syB[warp][jl];
                    on = sdB[warp][jl] != segi;
                }
                float d3[3] = {yi.x - (yj.x + bsh[0]), yi.y - (yj.y + bsh[1]), yi.z - (yj.z + bsh[2])};
                const float r2 = d3[0] * d3[0] + d3[1] * d3[1] + d3[2] * d3[2];
                const float lmax = fmaxf(yi.w, yj.w);
                const bool close = on && r2 < near2 * lmax * lmax;
                float ir = 1.f;
                if (close) {
                    // the separation from the FP64 positions (no cancellation in the
                    // leaf-relative FP32 coordinates); its length in FP32
                    d3[0] = float(xi[0] - sxB[warp][jl][0]);
                    d3[1] = float(xi[1] - sxB[warp][jl][1]);
                    d3[2] = float(xi[2] - sxB[warp][jl][2]);
                    const float rr = d3[0] * d3[0] + d3[1] * d3[1] + d3[2] * d3[2];
                    if (rr == 0.f) on = false;
                    ir = rr > 0.f ? rsqrtf(rr) : 1.f;
                } else if (on) {
                    ir = rsqrtf(r2);
                }
                float fw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, rv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (on) {
                    float T[3] = {d3[0] * ir, d3[1] * ir, d3[2] * ir};
                    float hs[18];
                    if (HM == HM_CUBIC) {
                        if (packed)
                            h_cubic_f32x2(c12f + c44f, c44f, cdf, Q, reinterpret_cast<const float4 *>(sTab), T, hs);
                        else
                            h_cubic_f32(c12f + c44f, c44f, cdf, Q, sTab, T, hs);
                    } else {
                        h_circle_sym<float, float>(sC, Q, T, hs);
                    }
                    const float ir2 = ir * ir;
                    const float4 *Pj4 = reinterpret_cast<const float4 *>(wPB + 108 * jl);
                    // both contractions over the 108 entries in 16-byte pieces (entry c = 18 ab + k)
#pragma unroll
                    for (int c4 = 0; c4 < 27; ++c4) {
                        const float4 pj = Pj4[c4], pi = Pi4[c4];
                        const float vj[4] = {pj.x, pj.y, pj.z, pj.w}, vi4[4] = {pi.x, pi.y, pi.z, pi.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = 4 * c4 + e;
                            fw[c / 18] = fmaf(vj[e], hs[c % 18], fw[c / 18]);
                            rv[c / 18] = fmaf(vi4[e], hs[c % 18], rv[c / 18]);
                        }
                    }
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) {
                        fw[ab] *= ir2;
                        rv[ab] *= -ir2;
                    }
                    if (close) {
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) tsum(accC[ab], accCl[ab], fw[ab]);
                    } else {
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) acc[ab] += fw[ab];
                    }
                }
                // reverse: sum over the tg lanes that share source jl (fixed order); close
                // pairs go through two-float sums, only when the warp has one
                if (__any_sync(0xffffffffu, close)) {
                    float ch[6], cl[6];
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) {
                        ch[ab] = close ? rv[ab] : 0.f;
                        cl[ab] = 0.f;
                        if (close) rv[ab] = 0.f;
                    }
                    for (int off = 1; off < tg; off <<= 1)
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) {
                            const float oh = __shfl_xor_sync(0xffffffffu, ch[ab], off);
                            const float ol = __shfl_xor_sync(0xffffffffu, cl[ab], off);
                            tsum2(ch[ab], cl[ab], oh, ol);
                        }
                    if (ti == 0 && jl < nj)
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) {
                            float2 &a = saccCB[warp][jl][ab];
                            tsum2(a.x, a.y, ch[ab], cl[ab]);
                        }
                }
                for (int off = 1; off < tg; off <<= 1)
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) rv[ab] += __shfl_xor_sync(0xffffffffu, rv[ab], off);
                if (ti == 0 && jl < nj) {
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) saccB[warp][jl][ab] += rv[ab];
                }
            }
            __syncwarp();
            // reverse partials of this chunk's sources: this warp is their only writer; the
            // first target chunk stores, later ones add (in the own leaf the first chunk
            // visits every source, later chunks only j >= r0)
            for (int k = lane; k < nj * 6; k += 32) {
                const int jl = k / 6, ab = k % 6;
                double *dst = part + (int64_t(slot_r) * N + (j0 + jl)) * 6 + ab;
                const float2 cc = saccCB[warp][jl][ab];
                const double v = double(saccB[warp][jl][ab]) + (double(cc.x) + double(cc.y));
                *dst = (first_chunk && !fine) ? v : *dst + v;
            }
        }
        }
        first_chunk = false;
        // forward: sum over the lanes that share target i (fixed order)
        for (int off = tg; off < 32; off <<= 1)
#pragma unroll
            for (int ab = 0; ab < 6; ++ab) {
                acc[ab] += __shfl_xor_sync(0xffffffffu, acc[ab], off);
                const float oh = __shfl_xor_sync(0xffffffffu, accC[ab], off);
                const float ol = __shfl_xor_sync(0xffffffffu, accCl[ab], off);
                tsum2(accC[ab], accCl[ab], oh, ol);
            }
        if (vi && tj == 0)
#pragma unroll
            for (int ab = 0; ab < 6; ++ab)
                part[(int64_t(slot_f) * N + i) * 6 + ab] = double(acc[ab]) + (double(accC[ab]) + double(accCl[ab]));
    }
    }
}

// FP64 form of the symmetric near field for the FP64 pass: the same leaf-pair
// work items, target chunks and partial slots as k_near_sym, with FP64
// positions, source tensors (P of k_precontract<double>), h and sums.  The
// cubic rule takes its circle points from a shared table; the general
// medium uses h_circle_sym.  FP64 arithmetic is the bound, so two warps per
// block and the full 108-entry tensors staged as doubles suffice.
constexpr int S64_WARPS = 2, S64_SCH = 8;

template <int HM>
__global__ void __launch_bounds__(S64_WARPS * 32) k_near_sym64(
    int L, const TreeBox *__restrict__ box, const DevMaterial *__restrict__ mat, const int *__restrict__ sstart,
    const double *__restrict__ ys, const double *__restrict__ P64, const int64_t *__restrict__ ssid,
    double *__restrict__ part, int64_t N, const int2 *__restrict__ items, const int *__restrict__ n_items) {
    extern __shared__ __align__(16) double sm_s64[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double *wPA = sm_s64 + warp * (32 * 108 + S64_SCH * 108);  // [32][108]: the chunk's target tensors
    double *wPB = wPA + 32 * 108;                               // [SCH][108]: staged sources
    __shared__ double sxB[S64_WARPS][S64_SCH][3];
    __shared__ int64_t sdB[S64_WARPS][S64_SCH];
    __shared__ double saccB[S64_WARPS][S64_SCH][6];
    __shared__ double sC[81];
    __shared__ double sTc[256], sTs[256];
    if (HM == HM_GENERIC)
        for (int i = threadIdx.x; i < 81; i += blockDim.x) sC[i] = mat->C[i];
    if (HM == HM_CUBIC)
        for (int i = threadIdx.x; i < mat->Q && i < 256; i += blockDim.x) sincospi(double(i) / double(mat->Q), &sTs[i], &sTc[i]);
    __syncthreads();
    const int64_t item = blockIdx.x * int64_t(S64_WARPS) + warp;
    if (item >= *n_items) return;
    const int2 wi = items[item];
    const int64_t Aleaf = wi.x;
    const int d = wi.y;
    const int nlv = 1 << (L - 1);
    int ax, ay, az;
    cell_xyz3(Aleaf, nlv, ax, ay, az);
    const int nb = 13 + d;
    const int ox = nb % 3 - 1, oy = (nb / 3) % 3 - 1, oz = nb / 9 - 1;
    const int64_t Bleaf = (int64_t(az + oz) * nlv + (ay + oy)) * nlv + (ax + ox);
    const bool self = d == 0;
    const int sA0 = sstart[Aleaf], sA1 = sstart[Aleaf + 1];
    const int sB0 = sstart[Bleaf], sB1 = sstart[Bleaf + 1];
    const int slot_f = nb, slot_r = self ? 27 : 26 - nb;
    const int Q = mat->Q;
    const double cp = mat->c12 + mat->c44, c44 = mat->c44, cd = mat->cd;
    bool first_chunk = true;
    for (int r0 = sA0, nrem = 0; r0 < sA1; r0 += nrem) {
        const int left = sA1 - r0;
        const int tg = left >= 29 ? 32 : left >= 13 ? 16 : left >= 5 ? 8 : left >= 3 ? 4 : left;
        nrem = min(tg, left);
        const int ls = 32 / tg, ti = lane % tg, tj = lane / tg;
        const int i = r0 + ti;
        const bool vi = i < sA1;
        __syncwarp();
        {
            const double2 *src = reinterpret_cast<const double2 *>(P64 + int64_t(108) * r0);
            double2 *dst = reinterpret_cast<double2 *>(wPA);
            for (int k = lane; k < nrem * 54; k += 32) dst[k] = __ldg(src + k);
        }
        __syncwarp();
        double xi[3] = {0.0, 0.0, 0.0};
        int64_t segi = -2;
        if (vi) {
            xi[0] = ys[3 * int64_t(i)], xi[1] = ys[3 * int64_t(i) + 1], xi[2] = ys[3 * int64_t(i) + 2];
            segi = ssid[i];
        }
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const double *Pi = wPA + 108 * ti;
        const int jb0 = self ? r0 : sB0;
        for (int j0 = jb0; j0 < sB1; j0 += S64_SCH) {
            const int nj = min(S64_SCH, sB1 - j0);
            __syncwarp();
            if (lane < nj) sdB[warp][lane] = ssid[j0 + lane];
            for (int k = lane; k < nj * 3; k += 32) (&sxB[warp][0][0])[k] = ys[3 * int64_t(j0) + k];
            for (int k = lane; k < S64_SCH * 6; k += 32) (&saccB[warp][0][0])[k] = 0.0;
            {
                const double2 *src = reinterpret_cast<const double2 *>(P64 + int64_t(108) * j0);
                double2 *dst = reinterpret_cast<double2 *>(wPB);
                for (int k = lane; k < nj * 54; k += 32) dst[k] = __ldg(src + k);
            }
            __syncwarp();
            for (int jj = 0; jj < nj; jj += ls) {
                const int jl = jj + tj;
                const int j = j0 + jl;
                const bool on = vi && jl < nj && (!self || j > i) && sdB[warp][jl] != segi;
                double fw[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, rv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                if (on) {
                    const double d3[3] = {xi[0] - sxB[warp][jl][0], xi[1] - sxB[warp][jl][1], xi[2] - sxB[warp][jl][2]};
                    const double r2 = d3[0] * d3[0] + d3[1] * d3[1] + d3[2] * d3[2];
                    if (r2 > 0.0) {
                        const double ir = rsqrt(r2);
                        const double T[3] = {d3[0] * ir, d3[1] * ir, d3[2] * ir};
                        double hs[18];
                        if (HM == HM_CUBIC)
                            h_cubic_tab<double>(cp, c44, cd, Q, sTc, sTs, T, hs);
                        else
                            h_circle_sym<double, double>(sC, Q, T, hs);
                        const double *Pj = wPB + 108 * jl;
#pragma unroll
                        for (int c = 0; c < 108; ++c) {
                            fw[c / 18] = fma(Pj[c], hs[c % 18], fw[c / 18]);
                            rv[c / 18] = fma(Pi[c], hs[c % 18], rv[c / 18]);
                        }
                        const double ir2 = ir * ir;
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) {
                            acc[ab] += fw[ab] * ir2;
                            rv[ab] *= -ir2;
                        }
                    }
                }
                for (int off = 1; off < tg; off <<= 1)
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) rv[ab] += __shfl_xor_sync(0xffffffffu, rv[ab], off);
                if (ti == 0 && jl < nj)
#pragma unroll
                    for (int ab = 0; ab < 6; ++ab) saccB[warp][jl][ab] += rv[ab];
            }
            __syncwarp();
            for (int k = lane; k < nj * 6; k += 32) {
                const int jl = k / 6, ab = k % 6;
                double *dst = part + (int64_t(slot_r) * N + (j0 + jl)) * 6 + ab;
                const double v = saccB[warp][jl][ab];
                *dst = first_chunk ? v : *dst + v;
            }
        }
        first_chunk = false;
        for (int off = tg; off < 32; off <<= 1)
#pragma unroll
            for (int ab = 0; ab < 6; ++ab) acc[ab] += __shfl_xor_sync(0xffffffffu, acc[ab], off);
        if (vi && tj == 0)
#pragma unroll
            for (int ab = 0; ab < 6; ++ab) part[(int64_t(slot_f) * N + i) * 6 + ab] = acc[ab];
    }
}

// far field (L2P) plus the partial slots, in a fixed order
__global__ void k_near_combine(int p, int nodes, int L, int64_t N, const TreeBox *__restrict__ box,
                               const int *__restrict__ sstart, const int *__restrict__ pleaf,
                               const double *__restrict__ xt, const float *__restrict__ S,
                               const double *__restrict__ S64, const double *__restrict__ part,
                               double *__restrict__ sig, const int *__restrict__ pfine,
                               const float *__restrict__ S7) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (t >= N) return;
    const int nlv = 1 << (L - 1);
    const int64_t leaf = pleaf[t];
    int cx, cy, cz;
    cell_xyz3(leaf, nlv, cx, cy, cz);
    double out[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (L >= 3 && S64) {
        // FP64 local values (GBFMM_MIXED_F64T): interpolate in FP64
        const int P3 = p * p * p;
        const double h = box->H / nlv, ih = double(nlv) / box->H;
        double bx[GB_MAXP], by[GB_MAXP], bz[GB_MAXP];
        lagrange_1d<double>(p, (xt[3 * t] - (box->origin[0] + cx * h)) * ih, bx, nodes);
        lagrange_1d<double>(p, (xt[3 * t + 1] - (box->origin[1] + cy * h)) * ih, by, nodes);
        lagrange_1d<double>(p, (xt[3 * t + 2] - (box->origin[2] + cz * h)) * ih, bz, nodes);
        const double *Sl = S64 + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 6;
        for (int lz = 0; lz < p; ++lz)
            for (int ly = 0; ly < p; ++ly) {
                const double wyz = by[ly] * bz[lz];
                for (int lx = 0; lx < p; ++lx) {
                    const double w = bx[lx] * wyz;
                    const double *s6 = Sl + ((lz * p + ly) * p + lx) * 6;
                    for (int ab = 0; ab < 6; ++ab) out[ab] += w * s6[ab];
                }
            }
    } else if (L >= 3) {
        const int P3 = p * p * p;
        double h = box->H / nlv, ih = double(nlv) / box->H;
        double c0[3] = {box->origin[0] + cx * h, box->origin[1] + cy * h, box->origin[2] + cz * h};
        const float *Sl = S + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 6;
        const int f = pfine ? pfine[t] : -1;
        if (f >= 0) {
            // a point of a split leaf: its child's local values and cell (adaptive tree)
            h *= 0.5;
            ih *= 2.0;
            c0[0] += (f & 1) * h;
            c0[1] += ((f >> 1) & 1) * h;
            c0[2] += ((f >> 2) & 1) * h;
            Sl = S7 + int64_t(f) * P3 * 6;
        }
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float bx[GB_MAXP], by[GB_MAXP], bz[GB_MAXP];
        lagrange_1d<float>(p, float((xt[3 * t] - c0[0]) * ih), bx, nodes);
        lagrange_1d<float>(p, float((xt[3 * t + 1] - c0[1]) * ih), by, nodes);
        lagrange_1d<float>(p, float((xt[3 * t + 2] - c0[2]) * ih), bz, nodes);
        for (int lz = 0; lz < p; ++lz)
            for (int ly = 0; ly < p; ++ly) {
                const float wyz = by[ly] * bz[lz];
                for (int lx = 0; lx < p; ++lx) {
                    const float w = bx[lx] * wyz;
                    const float *s6 = Sl + ((lz * p + ly) * p + lx) * 6;
                    for (int ab = 0; ab < 6; ++ab) acc[ab] += w * __ldg(s6 + ab);
                }
            }
        for (int ab = 0; ab < 6; ++ab) out[ab] = double(acc[ab]);
    }
    for (int s = 0; s < kSlots; ++s) {
        const int nb = s == 27 ? 13 : s;
        const int bx = cx + nb % 3 - 1, by = cy + (nb / 3) % 3 - 1, bz = cz + nb / 9 - 1;
        if (bx < 0 || by < 0 || bz < 0 || bx >= nlv || by >= nlv || bz >= nlv) continue;
        const int64_t B = (int64_t(bz) * nlv + by) * nlv + bx;
        if (sstart[B + 1] == sstart[B]) continue;
        const double *ps = part + (int64_t(s) * N + t) * 6;
        for (int ab = 0; ab < 6; ++ab) out[ab] += ps[ab];
    }
    for (int ab = 0; ab < 6; ++ab) sig[6 * t + ab] = out[ab];
}

// leaf-pair work items (A, d), heaviest first (log2 of |A| |B| buckets)
__global__ void k_pairs_count(int64_t nl, int L, const int *__restrict__ sstart, int *__restrict__ cnt) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l >= nl) return;
    const int nA = sstart[l + 1] - sstart[l];
    int c = 0;
    if (nA > 0) {
        const int nlv = 1 << (L - 1);
        int x, y, z;
        cell_xyz3(l, nlv, x, y, z);
        for (int d = 0; d < 14; ++d) {
            const int nb = 13 + d;
            const int bx = x + nb % 3 - 1, by = y + (nb / 3) % 3 - 1, bz = z + nb / 9 - 1;
            if (bx < 0 || by < 0 || bz < 0 || bx >= nlv || by >= nlv || bz >= nlv) continue;
            const int64_t B = (int64_t(bz) * nlv + by) * nlv + bx;
            if (sstart[B + 1] > sstart[B]) ++c;
        }
    }
    cnt[l] = c;
}

__global__ void k_pairs_fill(int64_t nl, int L, const int *__restrict__ sstart, const int *__restrict__ off,
                             int2 *__restrict__ items, int *__restrict__ keys, int *__restrict__ hist) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l >= nl) return;
    const int nA = sstart[l + 1] - sstart[l];
    if (nA == 0) return;
    const int nlv = 1 << (L - 1);
    int x, y, z;
    cell_xyz3(l, nlv, x, y, z);
    int o = off[l];
    for (int d = 0; d < 14; ++d) {
        const int nb = 13 + d;
        const int bx = x + nb % 3 - 1, by = y + (nb / 3) % 3 - 1, bz = z + nb / 9 - 1;
        if (bx < 0 || by < 0 || bz < 0 || bx >= nlv || by >= nlv || bz >= nlv) continue;
        const int64_t B = (int64_t(bz) * nlv + by) * nlv + bx;
        const int nB = sstart[B + 1] - sstart[B];
        if (nB == 0) continue;
        const int64_t cost = d == 0 ? int64_t(nA) * nA / 2 + 1 : int64_t(nA) * nB;
        const int key = 63 - (63 - __clzll(cost));
        items[o] = make_int2(int(l), d);
        keys[o] = key;
        atomicAdd(&hist[key], 1);
        ++o;
    }
}

// ---------------------------------------------------------------- near field with the learned h
// Angular bin of a folded direction (upper half-space): dominant axis face
// (+z, +x, -x, +y, -y) and a 16 x 16 grid of the two other components.
__device__ __forceinline__ int dir_bin(float x, float y, float z) {
    const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    int f;
    float u, v, m;
    if (az >= ax && az >= ay) {
        f = 0, u = x, v = y, m = az;
    } else if (ax >= ay) {
        f = x > 0.f ? 1 : 2, u = y, v = z, m = ax;
    } else {
        f = y > 0.f ? 3 : 4, u = x, v = z, m = ay;
    }
    const int bu = min(15, max(0, int((u / m + 1.f) * 8.f)));
    const int bv = min(15, max(0, int((v / m + 1.f) * 8.f)));
    return f * 256 + bu * 16 + bv;
}

constexpr int MSCH = 16;  // sources staged per warp chunk in the network kernel

// Pairs at distance >= rmin x (source segment length) whose direction lies in
// an angular bin the plain evaluator accepted use the network; the rest take
// the plain path of k_near_mixed (FP32 cubic or generic rule, FP64
// separation for close pairs).  Network pairs are queued per warp and
// evaluated sixteen at a time by warp MMAs; every queued contribution is
// added by the lane that queued it, in queue order (deterministic).
template <bool CUBIC>
__global__ void __launch_bounds__(WARPS * 32) k_near_mlp(
    int p, int nodes, int L, int64_t nl, float near2, float rmin2, const TreeBox *__restrict__ box,
    const DevMaterial *__restrict__ mat, const int *__restrict__ tstart, const double *__restrict__ xt,
    const int64_t *__restrict__ tsid, const int *__restrict__ sstart, const float4 *__restrict__ yrel,
    const double *__restrict__ ys, const float *__restrict__ c32, const int64_t *__restrict__ ssid,
    const float *__restrict__ S, double *__restrict__ sig, const __nv_bfloat16 *__restrict__ th,
    const float *__restrict__ th32, const float *__restrict__ hscale, const uint32_t *__restrict__ binmask,
    const int2 *__restrict__ items, const int *__restrict__ n_items) {
    extern __shared__ __align__(16) unsigned char dsm[];
    mlpw::Weights &Wt = *reinterpret_cast<mlpw::Weights *>(dsm);
    __shared__ __align__(16) float sP[WARPS][MSCH * 108];
    __shared__ float4 sy[WARPS][MSCH];
    __shared__ int ssd[WARPS][MSCH];
    __shared__ float4 qd[WARPS][48];
    __shared__ int qj[WARPS][48], ql[WARPS][48];
    __shared__ float qc[WARPS][16][6];
    __shared__ float sC[81];
    __shared__ float2 sTab[128];
    __shared__ uint32_t sBin[48];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int g = lane >> 2, tq = lane & 3;
    mlpw::load(Wt, th, th32, hscale);
    for (int i = threadIdx.x; i < 81; i += blockDim.x) sC[i] = float(mat->C[i]);
    for (int i = threadIdx.x; i < mat->Q && i < 128; i += blockDim.x) {
        float sn, cs;
        sincospif(float(i) / float(mat->Q), &sn, &cs);
        sTab[i] = make_float2(cs, sn);
    }
    for (int i = threadIdx.x; i < 48; i += blockDim.x) sBin[i] = binmask[i];
    __syncthreads();
    // one work item per warp: up to 32 targets of one leaf, heaviest first
    const int64_t item = blockIdx.x * int64_t(WARPS) + warp;
    if (item >= *n_items) return;
    const int2 wi = items[item];
    const int64_t leaf = wi.x;
    const int t0 = wi.y, t1 = min(wi.y + 32, tstart[leaf + 1]);
    const int P3 = p * p * p;
    const int nlv = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz3(leaf, nlv, cx, cy, cz);
    const bool far = L >= 3;
    const double h = box->H / nlv, ih = double(nlv) / box->H;
    const double c0[3] = {box->origin[0] + cx * h, box->origin[1] + cy * h, box->origin[2] + cz * h};
    const int Q = mat->Q;
    const float c12f = float(mat->c12), c44f = float(mat->c44), cdf = float(mat->cd);
    const float *Sl = S + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 6;
    float *wP = sP[warp];
    float4 *wy = sy[warp];
    int *wsd = ssd[warp];
    float4 *wq = qd[warp];
    int *wj = qj[warp], *wl = ql[warp];
    float(*wc)[6] = qc[warp];
    for (int r0 = t0; r0 < t1; r0 += 32) {
        const int nrem = min(32, t1 - r0);
        int tg = 1;
        while (tg < nrem) tg <<= 1;
        const int ls = 32 / tg, tl = lane % tg, ph = lane / tg;
        const int t = r0 + tl;
        const bool valid = tl < nrem;
        double x[3] = {0, 0, 0};
        float xr[3] = {0.f, 0.f, 0.f};
        float acc[6] = {0, 0, 0, 0, 0, 0};
        double acc64[6] = {0, 0, 0, 0, 0, 0};
        int myseg = -1;
        if (valid) {
            for (int d = 0; d < 3; ++d) {
                x[d] = xt[3 * int64_t(t) + d];
                xr[d] = float(x[d] - (c0[d] + 0.5 * h));
            }
            myseg = tsid ? int(tsid[t]) : -1;
        }
        if (far && ph == 0) {
            float bx[GB_MAXP], by[GB_MAXP], bz[GB_MAXP];
            lagrange_1d<float>(p, float((x[0] - c0[0]) * ih), bx, nodes);
            lagrange_1d<float>(p, float((x[1] - c0[1]) * ih), by, nodes);
            lagrange_1d<float>(p, float((x[2] - c0[2]) * ih), bz, nodes);
            for (int lz = 0; lz < p; ++lz)
                for (int ly = 0; ly < p; ++ly) {
                    const float wyz = by[ly] * bz[lz];
                    for (int lx = 0; lx < p; ++lx) {
                        const float w = bx[lx] * wyz;
                        const float *s6 = Sl + ((lz * p + ly) * p + lx) * 6;
                        for (int ab = 0; ab < 6; ++ab) acc[ab] += w * __ldg(s6 + ab);
                    }
                }
        }
        int qn = 0;  // queued network pairs (warp-uniform)
        for (int nb = 0; nb < 27; ++nb) {
            const int dxn = nb % 3 - 1, dyn = (nb / 3) % 3 - 1, dzn = nb / 9 - 1;
            const int ax = cx + dxn, ay = cy + dyn, az = cz + dzn;
            if (ax < 0 || ay < 0 || az < 0 || ax >= nlv || ay >= nlv || az >= nlv) continue;
            const int64_t A = (int64_t(az) * nlv + ay) * nlv + ax;
            const int s0 = sstart[A], s1 = sstart[A + 1];
            const float xs[3] = {xr[0] - float(dxn * h), xr[1] - float(dyn * h), xr[2] - float(dzn * h)};
            for (int j0 = s0; j0 < s1; j0 += MSCH) {
                const int nj = min(MSCH, s1 - j0);
                __syncwarp();
                if (lane < nj) {
                    wy[lane] = yrel[j0 + lane];
                    wsd[lane] = int(ssid[j0 + lane]);
                }
                {
                    const float4 *src = reinterpret_cast<const float4 *>(c32 + int64_t(108) * j0);
                    float4 *dst = reinterpret_cast<float4 *>(wP);
                    for (int i = lane; i < nj * 27; i += 32) dst[i] = __ldg(src + i);
                }
                __syncwarp();
                const int nit = (nj + ls - 1) / ls;
                for (int it = 0; it < nit; ++it) {
                    const int j = ph + it * ls;
                    bool eligible = false;
                    float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid && j < nj && wsd[j] != myseg) {
                        const float4 yj = wy[j];
                        float d[3] = {xs[0] - yj.x, xs[1] - yj.y, xs[2] - yj.z};
                        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        const bool close = r2 < near2 * yj.w * yj.w;
                        bool ok = true;
                        float ir;
                        if (close) {
                            const int64_t jj = j0 + j;
                            const double dd0 = x[0] - ys[3 * jj], dd1 = x[1] - ys[3 * jj + 1], dd2 = x[2] - ys[3 * jj + 2];
                            const double rr = dd0 * dd0 + dd1 * dd1 + dd2 * dd2;
                            ok = rr != 0.0;
                            d[0] = float(dd0);
                            d[1] = float(dd1);
                            d[2] = float(dd2);
                            ir = ok ? float(rsqrt(rr)) : 0.f;
                        } else {
                            ir = rsqrtf(r2);
                        }
                        if (ok) {
                            const float T0 = d[0] * ir, T1 = d[1] * ir, T2 = d[2] * ir;
                            const float sg = mlpw::fold_sign(T0, T1, T2);
                            const int bin = dir_bin(sg * T0, sg * T1, sg * T2);
                            const bool net = !close && r2 >= rmin2 * yj.w * yj.w && !((sBin[bin >> 5] >> (bin & 31)) & 1u);
                            if (net) {
                                eligible = true;
                                qv = make_float4(T0, T1, T2, ir * ir);
                            } else {
                                float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                                if (CUBIC)
                                    pair_generic<HM_CUBIC, float, float>(d, ir, wP + 108 * j, sC, Q, c12f, c44f, cdf,
                                                                         part, sTab);
                                else
                                    pair_generic<HM_GENERIC, float, float>(d, ir, wP + 108 * j, sC, Q, c12f, c44f,
                                                                           cdf, part, sTab);
                                if (close) {
                                    for (int ab = 0; ab < 6; ++ab) acc64[ab] += double(part[ab]);
                                } else {
                                    for (int ab = 0; ab < 6; ++ab) acc[ab] += part[ab];
                                }
                            }
                        }
                    }
                    // enqueue this iteration's network pairs in lane order
                    const unsigned m = __ballot_sync(0xffffffffu, eligible);
                    if (eligible) {
                        const int pos = qn + __popc(m & ((1u << lane) - 1u));
                        wq[pos] = qv;
                        wj[pos] = j;
                        wl[pos] = lane;
                    }
                    qn += __popc(m);
                    __syncwarp();
                    // evaluate full tiles of 16 (and the remainder at the chunk's end)
                    while (qn >= 16 || (qn > 0 && it == nit - 1)) {
                        const int nrow = min(16, qn);
                        const bool vlo = g < nrow, vhi = g + 8 < nrow;
                        const float4 ql4 = vlo ? wq[g] : make_float4(0.f, 0.f, 1.f, 0.f);
                        const float4 qh4 = vhi ? wq[g + 8] : make_float4(0.f, 0.f, 1.f, 0.f);
                        const float slo = mlpw::fold_sign(ql4.x, ql4.y, ql4.z);
                        const float shi = mlpw::fold_sign(qh4.x, qh4.y, qh4.z);
                        const float dlo[3] = {slo * ql4.x, slo * ql4.y, slo * ql4.z};
                        const float dhi[3] = {shi * qh4.x, shi * qh4.y, shi * qh4.z};
                        float olo[8], ohi[8];
                        mlpw::eval16(Wt, dlo, dhi, g, tq, olo, ohi);
                        float plo[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, phi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        const float *Plo = wP + 108 * (vlo ? wj[g] : 0), *Phi = wP + 108 * (vhi ? wj[g + 8] : 0);
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int col = 8 * (e >> 1) + 2 * tq + (e & 1);
                            if (col >= 27) continue;
                            const int v = col / 9, pp = (col / 3) % 3, q = col % 3;
                            constexpr int PIX[9] = {0, 5, 4, 5, 1, 3, 4, 3, 2};
                            const int k = 3 * PIX[v * 3 + pp] + q;
                            const float wgt = (v == pp ? 1.f : 0.5f) * Wt.scale[col];
                            const float hl = olo[e] * wgt * slo, hh = ohi[e] * wgt * shi;
#pragma unroll
                            for (int ab = 0; ab < 6; ++ab) {
                                plo[ab] += Plo[ab * 18 + k] * hl;
                                phi[ab] += Phi[ab * 18 + k] * hh;
                            }
                        }
#pragma unroll
                        for (int ab = 0; ab < 6; ++ab) {
                            plo[ab] += __shfl_xor_sync(0xffffffffu, plo[ab], 1);
                            plo[ab] += __shfl_xor_sync(0xffffffffu, plo[ab], 2);
                            phi[ab] += __shfl_xor_sync(0xffffffffu, phi[ab], 1);
                            phi[ab] += __shfl_xor_sync(0xffffffffu, phi[ab], 2);
                        }
                        if (tq == 0 && vlo)
                            for (int ab = 0; ab < 6; ++ab) wc[g][ab] = plo[ab] * ql4.w;
                        if (tq == 1 && vhi)
                            for (int ab = 0; ab < 6; ++ab) wc[g + 8][ab] = phi[ab] * qh4.w;
                        __syncwarp();
                        for (int r = 0; r < nrow; ++r)
                            if (wl[r] == lane)
                                for (int ab = 0; ab < 6; ++ab) acc[ab] += wc[r][ab];
                        __syncwarp();
                        // drop the evaluated rows
                        const int rest = qn - nrow;
                        float4 mv = make_float4(0.f, 0.f, 0.f, 0.f);
                        int mj = 0, ml = 0;
                        if (lane < rest) {
                            mv = wq[nrow + lane];
                            mj = wj[nrow + lane];
                            ml = wl[nrow + lane];
                        }
                        __syncwarp();
                        if (lane < rest) {
                            wq[lane] = mv;
                            wj[lane] = mj;
                            wl[lane] = ml;
                        }
                        qn = rest;
                        __syncwarp();
                    }
                }
            }
        }
        for (int off = tg; off < 32; off <<= 1)
            for (int ab = 0; ab < 6; ++ab) {
                acc[ab] += __shfl_xor_sync(0xffffffffu, acc[ab], off);
                acc64[ab] += __shfl_xor_sync(0xffffffffu, acc64[ab], off);
            }
        if (valid && ph == 0)
            for (int ab = 0; ab < 6; ++ab) sig[6 * int64_t(t) + ab] = double(acc[ab]) + acc64[ab];
    }
}

// ---------------------------------------------------------------- work list
// Items are (leaf, first target) for every 32 targets of a leaf; the cost of
// an item is ~ (its targets) x (sources in the 27 neighbour leaves).  Items
// are ordered by decreasing cost class (floor log2) so that the heaviest
// start first and the uneven leaf populations of clustered networks do not
// leave a long tail.
__global__ void k_items_count(int64_t nl, int L, const int *__restrict__ tstart, const int *__restrict__ sstart,
                              int *__restrict__ cnt, int *__restrict__ key_cnt) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l >= nl) return;
    const int nt = tstart[l + 1] - tstart[l];
    cnt[l] = (nt + 31) / 32;
    if (nt == 0) return;
    const int nlv = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz3(l, nlv, cx, cy, cz);
    int64_t ns = 0;
    for (int nb = 0; nb < 27; ++nb) {
        const int ax = cx + nb % 3 - 1, ay = cy + (nb / 3) % 3 - 1, az = cz + nb / 9 - 1;
        if (ax < 0 || ay < 0 || az < 0 || ax >= nlv || ay >= nlv || az >= nlv) continue;
        const int64_t A = (int64_t(az) * nlv + ay) * nlv + ax;
        ns += sstart[A + 1] - sstart[A];
    }
    const int64_t cost = int64_t(min(nt, 32)) * ns;
    const int key = cost > 0 ? 63 - __clzll(cost) : 0;  // floor log2
    key_cnt[l] = key;
}

__global__ void k_items_fill(int64_t nl, const int *__restrict__ tstart, const int *__restrict__ off,
                             const int *__restrict__ key_of, int2 *__restrict__ items, int *__restrict__ keys,
                             int *__restrict__ hist) {
    const int64_t l = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (l >= nl) return;
    const int t0 = tstart[l], t1 = tstart[l + 1];
    const int key = 63 - key_of[l];
    int o = off[l];
    for (int r0 = t0; r0 < t1; r0 += 32, ++o) {
        items[o] = make_int2(int(l), r0);
        keys[o] = key;
        atomicAdd(&hist[key], 1);
    }
}

__global__ void k_items_order(int n_total_cap, const int *__restrict__ total, const int2 *__restrict__ items,
                              const int *__restrict__ keys, const int *__restrict__ hist, int *__restrict__ cursor,
                              int2 *__restrict__ sorted, int *__restrict__ n_items) {
    __shared__ int base[64];
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < 64; ++k) {
            base[k] = run;
            run += hist[k];
        }
    }
    __syncthreads();
    const int n = *total;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_items = n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n && i < n_total_cap; i += gridDim.x * blockDim.x) {
        const int k = keys[i];
        sorted[base[k] + atomicAdd(&cursor[k], 1)] = items[i];
    }
}

__global__ void k_scan_small(int64_t n, const int *__restrict__ cnt, int *__restrict__ start) {
    // exclusive scan, one block of 1024 threads (cnt -> start[0..n])
    __shared__ int part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < int(blockDim.x); ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
        start[n] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        start[i] = run;
        run += cnt[i];
    }
}

}  // namespace

int near_coef_count(const gbfmm_ctx *ctx) { return ctx->mat.mode == GBFMM_H_ISO ? 80 : 108; }

int near_prepare(gbfmm_ctx *ctx) {
    const int64_t N = ctx->N;
    ++ctx->launches;
    if (near_coef_count(ctx) == 80)
        k_src_coef80<<<nblk(N, 128), 128, 0, ctx->stream>>>(N, ctx->d_q, ctx->d_Asym, float(ctx->mat.hc),
                                                              float(ctx->mat.ha), ctx->d_Pf);
    else
        k_src_coef108<<<nblk(N, kCoefPts), 256, 0, ctx->stream>>>(N, ctx->d_q, ctx->d_Asym, ctx->d_Pf);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

// capacity of the near-field work list for n_targets targets: called when
// the tree is built, so that an evaluation recorded into a CUDA graph
// allocates nothing
int near_alloc(gbfmm_ctx *ctx, int64_t n_targets) {
    const int64_t nl = ctx->n_leaves;
    const int64_t cap = nl + n_targets / 32 + 1;
    NearWork &W = ctx->nw;
    if (nl > W.cap_leaves) W.cap = 0;  // the per-leaf arrays grow with the item arrays
    const int64_t cap0 = W.cap;
    if (int rc = grow_dev(ctx, W.cap, cap,
                          {{(void **)&W.items, cap * sizeof(int2)}, {(void **)&W.sorted, cap * sizeof(int2)},
                           {(void **)&W.keys, cap * sizeof(int)}, {(void **)&W.cnt, nl * sizeof(int)},
                           {(void **)&W.key_of, nl * sizeof(int)}, {(void **)&W.off, (nl + 1) * sizeof(int)},
                           {(void **)&W.misc, 192 * sizeof(int)}},  // hist[64], cursor[64], n_items, total
                          "near-field work list")) {
        W.cap_leaves = 0;
        return rc;
    }
    if (W.cap != cap0) W.cap_leaves = nl;
    return GBFMM_OK;
}

// work list for the near kernels (no host synchronisation: the item count
// stays on the device and surplus warps return)
static int build_items(gbfmm_ctx *ctx, const int *tstart, int64_t n_targets, int *&n_items, int2 *&items,
                       int64_t &cap) {
    const int64_t nl = ctx->n_leaves;
    cap = nl + n_targets / 32 + 1;
    if (int rc = near_alloc(ctx, n_targets)) return rc;
    NearWork &W = ctx->nw;
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(W.misc, 0, 192 * sizeof(int), st));
    CK(cudaMemsetAsync(W.key_of, 0, nl * sizeof(int), st));
    ctx->launches += 4;
    k_items_count<<<nblk(nl, 256), 256, 0, st>>>(nl, ctx->L, tstart, ctx->d_leaf_start, W.cnt, W.key_of);
    k_scan_small<<<1, 1024, 0, st>>>(nl, W.cnt, W.off);
    k_items_fill<<<nblk(nl, 256), 256, 0, st>>>(nl, tstart, W.off, W.key_of, W.items, W.keys, W.misc);
    k_items_order<<<nblk(cap, 256) < 1024 ? nblk(cap, 256) : 1024, 256, 0, st>>>(
        int(cap), W.off + nl, W.items, W.keys, W.misc, W.misc + 64, W.sorted, W.misc + 128);
    CK(cudaGetLastError());
    n_items = W.misc + 128;
    items = W.sorted;
    return GBFMM_OK;
}

// the symmetric kernel applies to nodal forces with the unit-circle h
static bool near_symmetric(const gbfmm_ctx *ctx) { return ctx->mat.mode == GBFMM_H_CIRCLE; }

int near_sym_alloc(gbfmm_ctx *ctx) {
    if (!near_symmetric(ctx)) return GBFMM_OK;
    NearWork &W = ctx->nw;
    const int64_t pcap = 14 * ctx->n_leaves;
    if (int rc = grow_dev(ctx, W.pcap, pcap,
                          {{(void **)&W.pitems, pcap * sizeof(int2)}, {(void **)&W.psorted, pcap * sizeof(int2)},
                           {(void **)&W.pkeys, pcap * sizeof(int)}, {(void **)&W.pmisc, 192 * sizeof(int)}},
                          "near-field leaf pairs"))
        return rc;
    if (int rc = grow_dev(ctx, W.part_cap, ctx->N,
                          {{(void **)&W.part, size_t(kSlots) * ctx->N * 6 * sizeof(double)}}, "near-field partial sums"))
        return rc;
    return GBFMM_OK;
}

// leaf-pair work items of the symmetric near fields, heaviest first (count, scan, fill, order)
static int build_pair_items(gbfmm_ctx *ctx) {
    const int64_t nl = ctx->n_leaves, N = ctx->N;
    if (int rc = near_alloc(ctx, N)) return rc;
    if (int rc = near_sym_alloc(ctx)) return rc;
    NearWork &W = ctx->nw;
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(W.pmisc, 0, 192 * sizeof(int), st));
    ctx->launches += 4;
    k_pairs_count<<<nblk(nl, 256), 256, 0, st>>>(nl, ctx->L, ctx->d_leaf_start, W.cnt);
    k_scan_small<<<1, 1024, 0, st>>>(nl, W.cnt, W.off);
    k_pairs_fill<<<nblk(nl, 256), 256, 0, st>>>(nl, ctx->L, ctx->d_leaf_start, W.off, W.pitems, W.pkeys, W.pmisc);
    k_items_order<<<nblk(W.pcap, 256) < 1024 ? nblk(W.pcap, 256) : 1024, 256, 0, st>>>(
        int(W.pcap), W.off + nl, W.pitems, W.pkeys, W.pmisc, W.pmisc + 64, W.psorted, W.pmisc + 128);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

// FP64 pass, nodal forces with the unit-circle h: symmetric near field in FP64, then
// L2P from the FP64 local values and the partial slots (k_near_combine)
int near_run_sym64(gbfmm_ctx *ctx, double *sig) {
    if (int rc = build_pair_items(ctx)) return rc;
    const int64_t N = ctx->N;
    NearWork &W = ctx->nw;
    cudaStream_t st = ctx->stream;
    const size_t smem = size_t(S64_WARPS) * (32 + S64_SCH) * 108 * sizeof(double);
    const unsigned grid = nblk(W.pcap, S64_WARPS);
    ctx->launches += 2;
    if (ctx->mat.cubic) {
        CK(cudaFuncSetAttribute(k_near_sym64<HM_CUBIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_near_sym64<HM_CUBIC><<<grid, S64_WARPS * 32, smem, st>>>(ctx->L, ctx->d_box, ctx->d_mat, ctx->d_leaf_start,
                                                                   ctx->d_y, ctx->d_P, ctx->d_sid, W.part, N,
                                                                   W.psorted, W.pmisc + 128);
    } else {
        CK(cudaFuncSetAttribute(k_near_sym64<HM_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_near_sym64<HM_GENERIC><<<grid, S64_WARPS * 32, smem, st>>>(ctx->L, ctx->d_box, ctx->d_mat,
                                                                     ctx->d_leaf_start, ctx->d_y, ctx->d_P, ctx->d_sid,
                                                                     W.part, N, W.psorted, W.pmisc + 128);
    }
    k_near_combine<<<nblk(N, 256), 256, 0, st>>>(ctx->opt.p, ctx->opt.nodes, ctx->L, N, ctx->d_box, ctx->d_leaf_start, ctx->d_pleaf,
                                                 ctx->d_y, nullptr, ctx->d_S, W.part, sig, nullptr, nullptr);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

static int near_run_sym(gbfmm_ctx *ctx, double *sig) {
    if (int rc = build_pair_items(ctx)) return rc;
    // adaptive tree (nodal forces): split leaves, their children's ranges and local values
    const int *ref_start = ctx->rf.on && ctx->L >= 3 ? ctx->rf.ref_start : nullptr;
    const int64_t N = ctx->N;
    NearWork &W = ctx->nw;
    cudaStream_t st = ctx->stream;
    ctx->launches += 2;
    const float near2 = float(ctx->opt.near_fp64 * ctx->opt.near_fp64);
    const size_t smem = size_t(SYM_WARPS) * (32 + SYM_SCH) * 108 * sizeof(float);
    const unsigned grid = nblk(W.pcap, SYM_WARPS);
    if (ctx->mat.cubic) {
        CK(cudaFuncSetAttribute(k_near_sym<HM_CUBIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_near_sym<HM_CUBIC><<<grid, SYM_WARPS * 32, smem, st>>>(ctx->L, near2, ctx->d_box, ctx->d_mat,
                                                                 ctx->d_leaf_start, ctx->d_yrel, ctx->d_y, ctx->d_Pf,
                                                                 ctx->d_sid, W.part, N, W.psorted, W.pmisc + 128,
                                                                 ref_start, ctx->rf.child_start);
    } else {
        CK(cudaFuncSetAttribute(k_near_sym<HM_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        k_near_sym<HM_GENERIC><<<grid, SYM_WARPS * 32, smem, st>>>(ctx->L, near2, ctx->d_box, ctx->d_mat,
                                                                   ctx->d_leaf_start, ctx->d_yrel, ctx->d_y,
                                                                   ctx->d_Pf, ctx->d_sid, W.part, N, W.psorted,
                                                                   W.pmisc + 128, ref_start, ctx->rf.child_start);
    }
    const double *S64 = ctx->opt.precision == GBFMM_MIXED_F64T ? ctx->d_S : nullptr;
    k_near_combine<<<nblk(N, 256), 256, 0, st>>>(ctx->opt.p, ctx->opt.nodes, ctx->L, N, ctx->d_box, ctx->d_leaf_start, ctx->d_pleaf,
                                                 ctx->d_y, ctx->d_Sf, S64, W.part, sig,
                                                 ref_start ? ctx->rf.pfine : nullptr, ctx->rf.S7);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

int near_run(gbfmm_ctx *ctx, const int *tstart, const double *xt, const int64_t *tsid, double *sig) {
    if (tsid && near_symmetric(ctx)) return near_run_sym(ctx, sig);
    const int64_t nl = ctx->n_leaves;
    const float near2 = float(ctx->opt.near_fp64 * ctx->opt.near_fp64);
    int *n_items = nullptr;
    int2 *items = nullptr;
    int64_t cap = 0;
    const int64_t n_targets = tsid ? ctx->N : ctx->t_cap;
    if (int rc = build_items(ctx, tstart, n_targets, n_items, items, cap)) return rc;
    const unsigned grid = nblk(cap, WARPS);
    ++ctx->launches;
    if (ctx->mat.mode == GBFMM_H_MLP) {
        if (!ctx->mlp.trained || !ctx->mlp.d_binmask)
            return set_err(ctx, GBFMM_ERR_INVALID_ARG, "GBFMM_H_MLP: train (or set) and calibrate the network first");
        const float rmin = float(ctx->opt.mlp_min_dist > 0.0 ? ctx->opt.mlp_min_dist : 8.0);
        const size_t smem = sizeof(mlpw::Weights);
#define GB_MLP_ARGS                                                                                                  \
    ctx->opt.p, ctx->opt.nodes, ctx->L, nl, near2, rmin *rmin, ctx->d_box, ctx->d_mat, tstart, xt, tsid, ctx->d_leaf_start, ctx->d_yrel, \
        ctx->d_y, ctx->d_Pf, ctx->d_sid, ctx->d_Sf, sig, ctx->mlp.theta_h, ctx->mlp.theta, ctx->mlp.scale,        \
        ctx->mlp.d_binmask, items, n_items
        if (ctx->mat.cubic) {
            CK(cudaFuncSetAttribute(k_near_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_near_mlp<true><<<grid, WARPS * 32, smem, ctx->stream>>>(GB_MLP_ARGS);
        } else {
            CK(cudaFuncSetAttribute(k_near_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            k_near_mlp<false><<<grid, WARPS * 32, smem, ctx->stream>>>(GB_MLP_ARGS);
        }
#undef GB_MLP_ARGS
        CK(cudaGetLastError());
        return GBFMM_OK;
    }
#define GB_NEAR_ARGS                                                                                           \
    ctx->opt.p, ctx->opt.nodes, ctx->L, nl, near2, ctx->d_box, ctx->d_mat, tstart, xt, tsid, ctx->d_leaf_start, ctx->d_yrel, ctx->d_y, \
        ctx->d_Pf, ctx->d_sid, ctx->d_Sf, sig, items, n_items
    if (near_coef_count(ctx) == 80)
        k_near_mixed<HM_ISO, 80, 32><<<grid, WARPS * 32, 0, ctx->stream>>>(GB_NEAR_ARGS);
    else if (ctx->mat.cubic)
        k_near_mixed<HM_CUBIC, 108, 24><<<grid, WARPS * 32, 0, ctx->stream>>>(GB_NEAR_ARGS);
    else
        k_near_mixed<HM_GENERIC, 108, 24><<<grid, WARPS * 32, 0, ctx->stream>>>(GB_NEAR_ARGS);
#undef GB_NEAR_ARGS
    CK(cudaGetLastError());
    return GBFMM_OK;
}
