// The Lagrange FMM pass (Sec. 4, Algorithm 2), FP64 path:
//   precontract  P_j[ab][k] = sum_wr Asym[ab][wr][k] q_j[wr]   (per source)
//   P2M  W_m = sum_{y_j in leaf} L_p(ybar_m, y_j) q_j          (Eq. "far-field", source side)
//   M2M  W_m' = sum_children sum_m L_p(ybar_m', ybar_m) W_m    (parent basis at the child nodes)
//   M2L  s(xbar_l) = sum_{A in I(B)} sum_m K(xbar_l - ybar_m) W_m   (Eq. "m2l")
//   L2L  s(xbar_l') += sum_l L_p(xbar_l', xbar_l) s(xbar_l)    (parent local values at the child nodes)
//   L2P  s(x_i) = sum_l L_p(xbar_l, x_i) s(xbar_l) + near field over N(leaf)
// Nodes of a cell of edge h at corner c are c + h t_a, t_a = a/(p-1)
// (Sec. 4.1); node index m = (mz p + my) p + mx.
#include <cmath>
#include <string>

#include "internal.cuh"
#include "kernel_math.cuh"

namespace {

struct Transfer {
    double M[2][GB_MAXP][GB_MAXP];  // M[c][A'][a] = ell_A'((c + t_a) / 2)
};

inline unsigned nblk(int64_t n, int b) { return unsigned((n + b - 1) / b); }

__device__ __forceinline__ void cell_xyz(int64_t lin, int n, int &x, int &y, int &z) {
    x = int(lin % n);
    y = int((lin / n) % n);
    z = int(lin / (int64_t(n) * n));
}

// ---------------------------------------------------------------- precontract
template <typename R>
__global__ void k_precontract(int64_t N, const double *__restrict__ q, const double *__restrict__ Asym,
                              R *__restrict__ P) {
    __shared__ double As[6 * 9 * 18];
    for (int i = threadIdx.x; i < 6 * 9 * 18; i += blockDim.x) As[i] = Asym[i];
    __syncthreads();
    int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (j >= N) return;
    double qq[9];
    for (int i = 0; i < 9; ++i) qq[i] = q[9 * j + i];
    for (int ab = 0; ab < 6; ++ab)
        for (int k = 0; k < 18; ++k) {
            double s = 0.0;
            for (int wr = 0; wr < 9; ++wr) s += As[(ab * 9 + wr) * 18 + k] * qq[wr];
            P[108 * j + ab * 18 + k] = R(s);
        }
}

// ---------------------------------------------------------------- occupancy
__global__ void k_occ_leaves(int64_t nl, const int *__restrict__ start, int64_t base, int *__restrict__ occ) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= nl) return;
    occ[base + i] = start[i + 1] - start[i];
}

__global__ void k_occ_up(int level, int *__restrict__ occ) {
    int n = 1 << level;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= int64_t(n) * n * n) return;
    int x, y, z;
    cell_xyz(i, n, x, y, z);
    int nc = 2 * n;
    int64_t cb = cell_base_d(level + 1);
    int s = 0;
    for (int c = 0; c < 8; ++c) {
        int cx = 2 * x + (c & 1), cy = 2 * y + ((c >> 1) & 1), cz = 2 * z + (c >> 2);
        s += occ[cb + (int64_t(cz) * nc + cy) * nc + cx];
    }
    occ[cell_base_d(level) + i] = s;
}

// ---------------------------------------------------------------- P2M
// one block per leaf; thread m accumulates W[m][0..8].  The local
// coordinate of a point is formed in FP64; the basis and sums in R.
template <typename R>
__device__ void p2m_range(int p, int nodes, int b, int e, const double c0[3], double ih, const double *__restrict__ y,
                          const double *__restrict__ q, R *__restrict__ Wc);

template <typename R>
__global__ void k_p2m(int p, int nodes, int L, const TreeBox *__restrict__ box, const int *__restrict__ start,
                      const double *__restrict__ y, const double *__restrict__ q, R *__restrict__ W) {
    const int64_t leaf = blockIdx.x;
    const int nl = 1 << (L - 1);
    const int P3 = p * p * p;
    R *Wc = W + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 9;
    const int b = start[leaf], e = start[leaf + 1];
    if (b == e) {
        for (int i = threadIdx.x; i < P3 * 9; i += blockDim.x) Wc[i] = R(0);
        return;
    }
    int cx, cy, cz;
    cell_xyz(leaf, nl, cx, cy, cz);
    const double h = box->H / nl;
    const double ih = double(nl) / box->H;
    const double c0[3] = {box->origin[0] + cx * h, box->origin[1] + cy * h, box->origin[2] + cz * h};
    p2m_range<R>(p, nodes, b, e, c0, ih, y, q, Wc);
}

// adaptive tree: P2M of the children of split leaves, one block per child cell 8 r + c
// (compact rows; empty and absent children get zeros)
template <typename R>
__global__ void k_p2m_fine(int p, int nodes, int L, const TreeBox *__restrict__ box, const int *__restrict__ n_ref,
                           const int *__restrict__ ref_leaf, const int *__restrict__ child_start,
                           const double *__restrict__ y, const double *__restrict__ q, R *__restrict__ W7) {
    const int64_t f = blockIdx.x;
    const int r = int(f >> 3), c = int(f & 7);
    const int P3 = p * p * p;
    R *Wc = W7 + f * int64_t(P3) * 9;
    int b = 0, e = 0;
    if (r < *n_ref) {
        b = child_start[9 * r + c];
        e = child_start[9 * r + c + 1];
    }
    if (b == e) {
        for (int i = threadIdx.x; i < P3 * 9; i += blockDim.x) Wc[i] = R(0);
        return;
    }
    const int nl = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz(ref_leaf[r], nl, cx, cy, cz);
    const double h = box->H / (2 * nl);
    const double ih = double(2 * nl) / box->H;
    const double c0[3] = {box->origin[0] + (2 * cx + (c & 1)) * h, box->origin[1] + (2 * cy + ((c >> 1) & 1)) * h,
                          box->origin[2] + (2 * cz + (c >> 2)) * h};
    p2m_range<R>(p, nodes, b, e, c0, ih, y, q, Wc);
}

// W[m][wr] = sum over the points b..e of L_m(local position) q_wr (Sec. 4.3, P2M)
template <typename R>
__device__ void p2m_range(int p, int nodes, int b, int e, const double c0[3], double ih, const double *__restrict__ y,
                          const double *__restrict__ q, R *__restrict__ Wc) {
    const int P3 = p * p * p;
    constexpr int CH = 64;
    __shared__ R sb[CH][3][GB_MAXP];
    __shared__ R sq[CH][9];
    R acc[2][9];
    for (int u = 0; u < 2; ++u)
        for (int i = 0; i < 9; ++i) acc[u][i] = R(0);
    for (int j0 = b; j0 < e; j0 += CH) {
        const int nj = min(CH, e - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nj * 3; t += blockDim.x) {
            int j = t / 3, d = t % 3;
            R tt = R((y[3 * int64_t(j0 + j) + d] - c0[d]) * ih);
            R v[GB_MAXP];
            lagrange_1d<R>(p, tt, v, nodes);
            for (int a = 0; a < p; ++a) sb[j][d][a] = v[a];
        }
        for (int t = threadIdx.x; t < nj * 9; t += blockDim.x) sq[t / 9][t % 9] = R(q[9 * int64_t(j0) + t]);
        __syncthreads();
        for (int u = 0; u < 2; ++u) {
            int m = threadIdx.x + u * blockDim.x;
            if (m >= P3) break;
            int mx = m % p, my = (m / p) % p, mz = m / (p * p);
            for (int j = 0; j < nj; ++j) {
                R w = sb[j][0][mx] * sb[j][1][my] * sb[j][2][mz];
                for (int i = 0; i < 9; ++i) acc[u][i] += w * sq[j][i];
            }
        }
    }
    for (int u = 0; u < 2; ++u) {
        int m = threadIdx.x + u * blockDim.x;
        if (m >= P3) break;
        for (int i = 0; i < 9; ++i) Wc[m * 9 + i] = acc[u][i];
    }
}

// ---------------------------------------------------------------- M2M / L2L
// Separable tensor-product transfer on p x p x p x NC node values in shared
// memory: out[A',B',C'] = sum_{a,b,c} Mx[A'][a] My[B'][b] Mz[C'][c] in[a,b,c]
// (forward = true), or with each M transposed (forward = false).
template <int NC, typename R>
__device__ void transfer3(int p, const double (*Mx)[GB_MAXP], const double (*My)[GB_MAXP],
                          const double (*Mz)[GB_MAXP], bool fwd, R *in, R *t1) {
    const int P3 = p * p * p;
    auto m = [&](const double (*M)[GB_MAXP], int o, int i) { return R(fwd ? M[o][i] : M[i][o]); };
    // x pass: t1[z][y][X] = sum_x m(X, x) in[z][y][x]
    for (int t = threadIdx.x; t < P3 * NC; t += blockDim.x) {
        int c = t % NC, node = t / NC;
        int X = node % p, yz = node / p;
        R s = R(0);
        for (int x = 0; x < p; ++x) s += m(Mx, X, x) * in[(yz * p + x) * NC + c];
        t1[t] = s;
    }
    __syncthreads();
    // y pass: in[z][Y][X] = sum_y m(Y, y) t1[z][y][X]
    for (int t = threadIdx.x; t < P3 * NC; t += blockDim.x) {
        int c = t % NC, node = t / NC;
        int X = node % p, Y = (node / p) % p, z = node / (p * p);
        R s = R(0);
        for (int yy = 0; yy < p; ++yy) s += m(My, Y, yy) * t1[((z * p + yy) * p + X) * NC + c];
        in[t] = s;
    }
    __syncthreads();
    // z pass: t1[Z][Y][X] = sum_z m(Z, z) in[z][Y][X]
    for (int t = threadIdx.x; t < P3 * NC; t += blockDim.x) {
        int c = t % NC, node = t / NC;
        int XY = node % (p * p), Z = node / (p * p);
        R s = R(0);
        for (int zz = 0; zz < p; ++zz) s += m(Mz, Z, zz) * in[(zz * p * p + XY) * NC + c];
        t1[t] = s;
    }
    __syncthreads();
}

// parent weights at `level` from its 8 children at level + 1
template <typename R>
__global__ void k_m2m(int p, int level, Transfer tr, const int *__restrict__ occ, R *__restrict__ W) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int P3 = p * p * p;
    const int n = 1 << level;
    const int64_t cell = blockIdx.x;
    R *Wp = W + (cell_base_d(level) + cell) * int64_t(P3) * 9;
    R *in = sm, *t1 = sm + P3 * 9;
    if (occ[cell_base_d(level) + cell] == 0) {
        for (int i = threadIdx.x; i < P3 * 9; i += blockDim.x) Wp[i] = R(0);
        return;
    }
    int x, y, z;
    cell_xyz(cell, n, x, y, z);
    R acc[18];
    for (int i = 0; i < 18; ++i) acc[i] = R(0);
    const int nc = 2 * n;
    for (int c = 0; c < 8; ++c) {
        const int ox = c & 1, oy = (c >> 1) & 1, oz = c >> 2;
        const int64_t ch = cell_base_d(level + 1) + (int64_t(2 * z + oz) * nc + (2 * y + oy)) * nc + (2 * x + ox);
        if (occ[ch] == 0) continue;
        const R *Wc = W + ch * int64_t(P3) * 9;
        __syncthreads();
        for (int i = threadIdx.x; i < P3 * 9; i += blockDim.x) in[i] = Wc[i];
        __syncthreads();
        transfer3<9, R>(p, tr.M[ox], tr.M[oy], tr.M[oz], true, in, t1);
        for (int u = 0; u < 18; ++u) {
            int i = threadIdx.x + u * blockDim.x;
            if (i >= P3 * 9) break;
            acc[u] += t1[i];
        }
    }
    for (int u = 0; u < 18; ++u) {
        int i = threadIdx.x + u * blockDim.x;
        if (i >= P3 * 9) break;
        Wp[i] = acc[u];
    }
}

// child locals at `level` += parent's, interpolated
template <typename R>
__global__ void k_l2l(int p, int level, Transfer tr, const int *__restrict__ tocc, R *__restrict__ S) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int P3 = p * p * p;
    const int n = 1 << level;
    const int64_t cell = blockIdx.x;
    if (tocc[cell_base_d(level) + cell] == 0) return;
    int x, y, z;
    cell_xyz(cell, n, x, y, z);
    const int np = n / 2;
    const int64_t par = cell_base_d(level - 1) + (int64_t(z / 2) * np + y / 2) * np + x / 2;
    R *in = sm, *t1 = sm + P3 * 6;
    for (int i = threadIdx.x; i < P3 * 6; i += blockDim.x) in[i] = S[par * P3 * 6 + i];
    __syncthreads();
    transfer3<6, R>(p, tr.M[x & 1], tr.M[y & 1], tr.M[z & 1], false, in, t1);
    R *Sc = S + (cell_base_d(level) + cell) * int64_t(P3) * 6;
    for (int i = threadIdx.x; i < P3 * 6; i += blockDim.x) Sc[i] += t1[i];
}

// adaptive tree: occupancy of the children of split leaves at level L (one below the
// leaves), into occL (the level's part of the occupancy array, zeroed before); the work
// counts read it to count the children's M2L pairs
__global__ void k_fine_occ(int64_t n_fine, int L, const int *__restrict__ n_ref, const int *__restrict__ ref_leaf,
                           const int *__restrict__ child_start, int *__restrict__ occL) {
    const int64_t f = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (f >= n_fine) return;
    const int r = int(f >> 3), c = int(f & 7);
    if (r >= *n_ref) return;
    const int cnt = child_start[9 * r + c + 1] - child_start[9 * r + c];
    if (cnt == 0) return;
    const int nl = 1 << (L - 1), nf = 2 * nl;
    int x, y, z;
    cell_xyz(ref_leaf[r], nl, x, y, z);
    const int64_t lin = (int64_t(2 * z + (c >> 2)) * nf + (2 * y + ((c >> 1) & 1))) * nf + (2 * x + (c & 1));
    occL[lin] = cnt;
}

// adaptive tree: children's local values += their split parent's, interpolated (L2L),
// one block per child cell 8 r + c that holds points
template <typename R>
__global__ void k_l2l_fine(int p, int L, Transfer tr, const int *__restrict__ n_ref, const int *__restrict__ ref_leaf,
                           const int *__restrict__ child_start, const R *__restrict__ S, R *__restrict__ S7) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *in = reinterpret_cast<R *>(sm_raw);
    const int64_t f = blockIdx.x;
    const int r = int(f >> 3), c = int(f & 7);
    if (r >= *n_ref || child_start[9 * r + c + 1] == child_start[9 * r + c]) return;
    const int P3 = p * p * p;
    R *t1 = in + P3 * 6;
    const R *Sp = S + (cell_base_d(L - 1) + ref_leaf[r]) * int64_t(P3) * 6;
    for (int i = threadIdx.x; i < P3 * 6; i += blockDim.x) in[i] = Sp[i];
    __syncthreads();
    transfer3<6, R>(p, tr.M[c & 1], tr.M[(c >> 1) & 1], tr.M[c >> 2], false, in, t1);
    R *out = S7 + f * int64_t(P3) * 6;
    for (int i = threadIdx.x; i < P3 * 6; i += blockDim.x) out[i] += t1[i];
}

// Parent weights at `level` from its 8 children at level + 1 (Sec. 3.2,
// M2M), with the children merged one axis at a time: for each child row
// (oy, oz) the x transfer sums over both x children (2p terms), then the y
// transfer over both y halves, then the z transfer over both z halves --
// 14 p multiply-adds per parent value instead of 24 p for eight separate
// tensor-product transfers, and two barriers per parent instead of 24.
// Shared memory: 4 x 9 p^3 values (x-merged rows of one z half, x- and
// y-merged halves).
template <typename R>
__global__ void __launch_bounds__(256) k_m2m_merge(int p, int level, Transfer tr, const int *__restrict__ occ,
                                                   R *__restrict__ W) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *tx = reinterpret_cast<R *>(sm_raw);
    __shared__ R Ms[2][GB_MAXP][GB_MAXP];
    __shared__ int64_t s_ch[8];
    const int P3 = p * p * p, NV = P3 * 9;
    R *u = tx + 2 * NV;
    const int n = 1 << level, nc = 2 * n;
    const int64_t cell = blockIdx.x;
    R *Wp = W + (cell_base_d(level) + cell) * int64_t(NV);
    if (occ[cell_base_d(level) + cell] == 0) {
        for (int i = threadIdx.x; i < NV; i += blockDim.x) Wp[i] = R(0);
        return;
    }
    int x, y, z;
    cell_xyz(cell, n, x, y, z);
    for (int i = threadIdx.x; i < 2 * GB_MAXP * GB_MAXP; i += blockDim.x) {
        const int c = i / (GB_MAXP * GB_MAXP), o = (i / GB_MAXP) % GB_MAXP, a = i % GB_MAXP;
        Ms[c][o][a] = R(tr.M[c][o][a]);
    }
    if (threadIdx.x < 8) {
        const int ox = threadIdx.x & 1, oy = (threadIdx.x >> 1) & 1, oz = threadIdx.x >> 2;
        const int64_t ch = cell_base_d(level + 1) + (int64_t(2 * z + oz) * nc + (2 * y + oy)) * nc + (2 * x + ox);
        s_ch[threadIdx.x] = occ[ch] > 0 ? ch * int64_t(NV) : int64_t(-1);
    }
    __syncthreads();
    for (int oz = 0; oz < 2; ++oz) {
        // x: tx[oy][((c p + b) p + A) 9 + k] = sum_ox sum_a M[ox][A][a] W_(ox,oy,oz)[((c p + b) p + a) 9 + k]
        for (int t = threadIdx.x; t < 2 * NV; t += blockDim.x) {
            const int oy = t / NV, r = t - oy * NV;
            const int k = r % 9, node = r / 9, A = node % p, bc = node / p;
            R s = R(0);
            for (int ox = 0; ox < 2; ++ox) {
                const int64_t base = s_ch[ox + 2 * oy + 4 * oz];
                if (base < 0) continue;
                const R *Wc = W + base + int64_t(bc) * p * 9 + k;
                for (int a = 0; a < p; ++a) s += Ms[ox][A][a] * Wc[9 * a];
            }
            tx[t] = s;
        }
        __syncthreads();
        // y: u[oz][((c p + B) p + A) 9 + k] = sum_oy sum_b M[oy][B][b] tx[oy][((c p + b) p + A) 9 + k]
        for (int r = threadIdx.x; r < NV; r += blockDim.x) {
            const int k = r % 9, node = r / 9, A = node % p, B = (node / p) % p, c = node / (p * p);
            R s = R(0);
            for (int oy = 0; oy < 2; ++oy)
                for (int b = 0; b < p; ++b) s += Ms[oy][B][b] * tx[oy * NV + ((c * p + b) * p + A) * 9 + k];
            u[oz * NV + r] = s;
        }
        __syncthreads();
    }
    // z: W[((C p + B) p + A) 9 + k] = sum_oz sum_c M[oz][C][c] u[oz][((c p + B) p + A) 9 + k]
    for (int r = threadIdx.x; r < NV; r += blockDim.x) {
        const int k = r % 9, node = r / 9, AB = node % (p * p), C = node / (p * p);
        R s = R(0);
        for (int oz = 0; oz < 2; ++oz)
            for (int c = 0; c < p; ++c) s += Ms[oz][C][c] * u[oz * NV + (c * p * p + AB) * 9 + k];
        Wp[r] = s;
    }
}

// Child locals at `level` += their parent's, interpolated (Sec. 3.2, L2L),
// one block per parent at level - 1 producing all eight children axis by
// axis: the parent's values are read once, the x transfer gives both x
// halves, the y transfer the four (ox, oy) quarters, the z transfer the
// eight children -- 14 p multiply-adds per child value on average instead
// of 24 p.  Shared memory: 7 x 6 p^3 values.
template <typename R>
__global__ void __launch_bounds__(256) k_l2l_split(int p, int level, Transfer tr, const int *__restrict__ tocc,
                                                   R *__restrict__ S) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *in = reinterpret_cast<R *>(sm_raw);
    __shared__ R Ms[2][GB_MAXP][GB_MAXP];
    __shared__ int64_t s_ch[8];
    const int P3 = p * p * p, NV = P3 * 6;
    R *tx = in + NV, *ty = tx + 2 * NV;
    const int np = 1 << (level - 1), n = 2 * np;
    const int64_t par = blockIdx.x;
    int x, y, z;
    cell_xyz(par, np, x, y, z);
    if (threadIdx.x < 8) {
        const int ox = threadIdx.x & 1, oy = (threadIdx.x >> 1) & 1, oz = threadIdx.x >> 2;
        const int64_t ch = cell_base_d(level) + (int64_t(2 * z + oz) * n + (2 * y + oy)) * n + (2 * x + ox);
        s_ch[threadIdx.x] = tocc[ch] > 0 ? ch * int64_t(NV) : int64_t(-1);
    }
    for (int i = threadIdx.x; i < 2 * GB_MAXP * GB_MAXP; i += blockDim.x) {
        const int c = i / (GB_MAXP * GB_MAXP), o = (i / GB_MAXP) % GB_MAXP, a = i % GB_MAXP;
        Ms[c][o][a] = R(tr.M[c][o][a]);
    }
    __syncthreads();
    bool any = false;
    for (int c = 0; c < 8; ++c) any |= s_ch[c] >= 0;
    if (!any) return;
    const R *Sp = S + (cell_base_d(level - 1) + par) * int64_t(NV);
    for (int i = threadIdx.x; i < NV; i += blockDim.x) in[i] = Sp[i];
    __syncthreads();
    // x: tx[ox][((c p + b) p + A) 6 + k] = sum_a M[ox][a][A] in[((c p + b) p + a) 6 + k]
    for (int t = threadIdx.x; t < 2 * NV; t += blockDim.x) {
        const int ox = t / NV, r = t - ox * NV;
        const int k = r % 6, node = r / 6, A = node % p, bc = node / p;
        R s = R(0);
        for (int a = 0; a < p; ++a) s += Ms[ox][a][A] * in[(bc * p + a) * 6 + k];
        tx[t] = s;
    }
    __syncthreads();
    // y: ty[ox + 2 oy][((c p + B) p + A) 6 + k] = sum_b M[oy][b][B] tx[ox][((c p + b) p + A) 6 + k]
    for (int t = threadIdx.x; t < 4 * NV; t += blockDim.x) {
        const int q = t / NV, r = t - q * NV, ox = q & 1, oy = q >> 1;
        const int k = r % 6, node = r / 6, A = node % p, B = (node / p) % p, c = node / (p * p);
        R s = R(0);
        for (int b = 0; b < p; ++b) s += Ms[oy][b][B] * tx[ox * NV + ((c * p + b) * p + A) * 6 + k];
        ty[t] = s;
    }
    __syncthreads();
    // z: child (ox, oy, oz) += sum_c M[oz][c][C] ty[ox + 2 oy][((c p + B) p + A) 6 + k]
    for (int t = threadIdx.x; t < 8 * NV; t += blockDim.x) {
        const int ci = t / NV, r = t - ci * NV, oz = ci >> 2;
        const int64_t base = s_ch[ci];
        if (base < 0) continue;
        const int k = r % 6, node = r / 6, AB = node % (p * p), C = node / (p * p);
        const R *tq = ty + (ci & 3) * NV;
        R s = R(0);
        for (int c = 0; c < p; ++c) s += Ms[oz][c][C] * tq[(c * p * p + AB) * 6 + k];
        S[base + r] += s;
    }
}

// ---------------------------------------------------------------- M2L (FP64)
// One block per target cell of levels 2..L-1; thread l owns node l's 6
// components.  Sources: the interaction list I(B) = children of the
// parent's neighbours that are not neighbours of B.  Node kernels come
// from the lattice table: K(xbar_l - ybar_m) at level `lev` is
// Klat[o (p-1) + l - m] * (2^lev / H)^2.
__global__ void k_m2l_f64(int p, int L, int lat_n, const TreeBox *__restrict__ box, const double *__restrict__ Klat,
                          const int *__restrict__ occ, const int *__restrict__ tocc, const double *__restrict__ W,
                          double *__restrict__ S) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double *sW = reinterpret_cast<double *>(sm_raw);
    const int P3 = p * p * p;
    int64_t g = cell_base_d(2) + blockIdx.x;
    int lev = 2;
    while (lev + 1 < L && g >= cell_base_d(lev + 1)) ++lev;
    const int64_t cell = g - cell_base_d(lev);
    if (tocc[g] == 0) return;
    const int n = 1 << lev;
    int bx, by, bz;
    cell_xyz(cell, n, bx, by, bz);
    const int l = threadIdx.x;
    const bool own = l < P3;
    const int lx = l % p, ly = (l / p) % p, lz = l / (p * p);
    const int R0 = (lat_n - 1) / 2;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int nb = 0; nb < 27; ++nb) {
        const int px = bx / 2 + nb % 3 - 1, py = by / 2 + (nb / 3) % 3 - 1, pz = bz / 2 + nb / 9 - 1;
        for (int c = 0; c < 8; ++c) {
            const int ax = 2 * px + (c & 1), ay = 2 * py + ((c >> 1) & 1), az = 2 * pz + (c >> 2);
            if (ax < 0 || ay < 0 || az < 0 || ax >= n || ay >= n || az >= n) continue;
            const int ox = bx - ax, oy = by - ay, oz = bz - az;
            if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
            const int64_t A = cell_base_d(lev) + (int64_t(az) * n + ay) * n + ax;
            if (occ[A] == 0) continue;
            __syncthreads();
            for (int i = threadIdx.x; i < P3 * 9; i += blockDim.x) sW[i] = W[A * P3 * 9 + i];
            __syncthreads();
            if (!own) continue;
            const int Dx0 = ox * (p - 1) + lx + R0, Dy0 = oy * (p - 1) + ly + R0, Dz0 = oz * (p - 1) + lz + R0;
            for (int m = 0; m < P3; ++m) {
                const int mx = m % p, my = (m / p) % p, mz = m / (p * p);
                const double *K = Klat + ((int64_t(Dz0 - mz) * lat_n + (Dy0 - my)) * lat_n + (Dx0 - mx)) * 54;
                const double *w = sW + m * 9;
                for (int ab = 0; ab < 6; ++ab) {
                    double s = 0.0;
                    for (int wr = 0; wr < 9; ++wr) s += K[ab * 9 + wr] * w[wr];
                    acc[ab] += s;
                }
            }
        }
    }
    if (own) {
        const double sc = double(n) / box->H;
        double *Sc = S + g * int64_t(P3) * 6 + l * 6;
        for (int ab = 0; ab < 6; ++ab) Sc[ab] = acc[ab] * sc * sc;
    }
}

// ---------------------------------------------------------------- L2P + P2P (FP64)
// One block per leaf holding targets.  Far part: interpolate the leaf's
// local values at the target; near part: direct sum over the source points
// of the 27 neighbouring leaves (Eq. "stress3"), skipping the target's own
// segment.
template <int MODE>
__global__ void k_leaf_eval_f64(int p, int nodes, int L, const TreeBox *__restrict__ box, const DevMaterial *__restrict__ mat,
                                const int *__restrict__ tstart, const double *__restrict__ xt,
                                const int64_t *__restrict__ tsid, const int *__restrict__ sstart,
                                const double *__restrict__ ys, const double *__restrict__ P,
                                const int64_t *__restrict__ ssid, const double *__restrict__ S,
                                double *__restrict__ sig) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double *sm = reinterpret_cast<double *>(sm_raw);
    constexpr int CH = 64;
    const int P3 = p * p * p;
    const int64_t leaf = blockIdx.x;
    const int t0 = tstart[leaf], t1 = tstart[leaf + 1];
    if (t0 == t1) return;
    const int nl = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz(leaf, nl, cx, cy, cz);
    const bool far = L >= 3;
    double *sS = sm;                     // [P3][6]
    double *sy = sm + P3 * 6;            // [CH][3]
    double *sP = sy + CH * 3;            // [CH][108]
    int64_t *ssd = (int64_t *)(sP + CH * 108);  // [CH]
    if (far) {
        const double *Sl = S + (cell_base_d(L - 1) + leaf) * int64_t(P3) * 6;
        for (int i = threadIdx.x; i < P3 * 6; i += blockDim.x) sS[i] = Sl[i];
    }
    const double h = box->H / nl, ih = double(nl) / box->H;
    const double c0[3] = {box->origin[0] + cx * h, box->origin[1] + cy * h, box->origin[2] + cz * h};
    DevMaterial m = *mat;
    for (int r0 = t0; r0 < t1; r0 += blockDim.x) {
        const int t = r0 + threadIdx.x;
        const bool valid = t < t1;
        double x[3] = {0, 0, 0}, acc[6] = {0, 0, 0, 0, 0, 0};
        int64_t myseg = -1;
        __syncthreads();
        if (valid) {
            for (int d = 0; d < 3; ++d) x[d] = xt[3 * int64_t(t) + d];
            myseg = tsid ? tsid[t] : -1;
            if (far) {
                double bx[GB_MAXP], by[GB_MAXP], bz[GB_MAXP];
                lagrange_1d<double>(p, (x[0] - c0[0]) * ih, bx, nodes);
                lagrange_1d<double>(p, (x[1] - c0[1]) * ih, by, nodes);
                lagrange_1d<double>(p, (x[2] - c0[2]) * ih, bz, nodes);
                for (int l = 0; l < P3; ++l) {
                    double w = bx[l % p] * by[(l / p) % p] * bz[l / (p * p)];
                    for (int ab = 0; ab < 6; ++ab) acc[ab] += w * sS[l * 6 + ab];
                }
            }
        }
        for (int nb = 0; nb < 27; ++nb) {
            const int ax = cx + nb % 3 - 1, ay = cy + (nb / 3) % 3 - 1, az = cz + nb / 9 - 1;
            if (ax < 0 || ay < 0 || az < 0 || ax >= nl || ay >= nl || az >= nl) continue;
            const int64_t A = (int64_t(az) * nl + ay) * nl + ax;
            const int s0 = sstart[A], s1 = sstart[A + 1];
            for (int j0 = s0; j0 < s1; j0 += CH) {
                const int nj = min(CH, s1 - j0);
                __syncthreads();
                for (int i = threadIdx.x; i < nj * 3; i += blockDim.x) sy[i] = ys[3 * int64_t(j0) + i];
                for (int i = threadIdx.x; i < nj * 108; i += blockDim.x) sP[i] = P[108 * int64_t(j0) + i];
                for (int i = threadIdx.x; i < nj; i += blockDim.x) ssd[i] = ssid[j0 + i];
                __syncthreads();
                if (!valid) continue;
                for (int j = 0; j < nj; ++j) {
                    if (ssd[j] == myseg) continue;
                    double d[3] = {x[0] - sy[3 * j], x[1] - sy[3 * j + 1], x[2] - sy[3 * j + 2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0) continue;
                    double ir = rsqrt(r2);
                    double T[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
                    double hs[18];
                    if (MODE == GBFMM_H_ISO)
                        h_iso_sym<double>(m.hc, m.ha, T, hs);
                    else if (m.cubic)
                        h_circle_cubic<double>(m.c12, m.c44, m.cd, m.Q, T, hs);
                    else
                        h_circle_sym<double, double>(mat->C, m.Q, T, hs);
                    const double ir2 = ir * ir;
                    const double *Pj = sP + 108 * j;
                    for (int ab = 0; ab < 6; ++ab) {
                        double s = 0.0;
                        for (int k = 0; k < 18; ++k) s += Pj[ab * 18 + k] * hs[k];
                        acc[ab] += s * ir2;
                    }
                }
            }
        }
        if (valid)
            for (int ab = 0; ab < 6; ++ab) sig[6 * int64_t(t) + ab] = acc[ab];
    }
}

// ---------------------------------------------------------------- mixed-precision leaf pass
// Source points relative to their leaf centre, in FP32, plus the length of
// their segment: yrel[i] = (y_i - c_leaf(i), |S|).
__global__ void k_prep_mixed(int64_t N, int L, const TreeBox *__restrict__ box, const double *__restrict__ y,
                             const int *__restrict__ pleaf, const double *__restrict__ slen,
                             float4 *__restrict__ yrel) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= N) return;
    const int nl = 1 << (L - 1);
    int cx, cy, cz;
    cell_xyz(pleaf[i], nl, cx, cy, cz);
    const double h = box->H / nl;
    yrel[i] = make_float4(float(y[3 * i] - (box->origin[0] + (cx + 0.5) * h)),
                          float(y[3 * i + 1] - (box->origin[1] + (cy + 0.5) * h)),
                          float(y[3 * i + 2] - (box->origin[2] + (cz + 0.5) * h)), float(slen[i]));
}

// ---------------------------------------------------------------- forces
struct ForceParams {
    double xi[GB_MAXG], w[GB_MAXG];
    int n;
};

__global__ void k_forces(int64_t n_segs, ForceParams fp, const double *__restrict__ nodes,
                         const int64_t *__restrict__ segs, const double *__restrict__ b, const int *__restrict__ pos,
                         const double *__restrict__ sig, double *__restrict__ f_nodes, double *__restrict__ f_seg,
                         double *__restrict__ sig_out) {
    int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (s >= n_segs) return;
    const int64_t n0 = segs[2 * s], n1 = segs[2 * s + 1];
    double S[3], bb[3];
    for (int i = 0; i < 3; ++i) {
        S[i] = nodes[3 * n1 + i] - nodes[3 * n0 + i];
        bb[i] = b[3 * s + i];
    }
    double f1[3] = {0, 0, 0}, f2[3] = {0, 0, 0};
    for (int g = 0; g < fp.n; ++g) {
        const int i = pos[s * fp.n + g];
        const double *sg = sig + 6 * int64_t(i);
        if (sig_out)
            for (int a = 0; a < 6; ++a) sig_out[6 * (s * fp.n + g) + a] = sg[a];
        // (sigma b)_i with sigma in Voigt order xx yy zz yz xz xy
        const double sb[3] = {sg[0] * bb[0] + sg[5] * bb[1] + sg[4] * bb[2],
                              sg[5] * bb[0] + sg[1] * bb[1] + sg[3] * bb[2],
                              sg[4] * bb[0] + sg[3] * bb[1] + sg[2] * bb[2]};
        const double pk[3] = {sb[1] * S[2] - sb[2] * S[1], sb[2] * S[0] - sb[0] * S[2], sb[0] * S[1] - sb[1] * S[0]};
        const double w1 = 0.5 * fp.w[g] * 0.5 * (1.0 - fp.xi[g]);
        const double w2 = 0.5 * fp.w[g] * 0.5 * (1.0 + fp.xi[g]);
        for (int d = 0; d < 3; ++d) {
            f1[d] += w1 * pk[d];
            f2[d] += w2 * pk[d];
        }
    }
    for (int d = 0; d < 3; ++d) {
        atomicAdd(&f_nodes[3 * n0 + d], f1[d]);
        atomicAdd(&f_nodes[3 * n1 + d], f2[d]);
    }
    if (f_seg)
        for (int d = 0; d < 3; ++d) {
            f_seg[6 * s + d] = f1[d];
            f_seg[6 * s + 3 + d] = f2[d];
        }
}

__global__ void k_scatter_targets(int64_t n, const int *__restrict__ pos, const double *__restrict__ src,
                                  double *__restrict__ dst) {
    int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (k >= n) return;
    const double *s = src + 6 * int64_t(pos[k]);
    for (int a = 0; a < 6; ++a) dst[6 * k + a] = s[a];
}

// M[c][A][a] = ell_A((c + t_a) / 2): the parent's basis function A at node a of child c
// (equispaced nodes as before; Chebyshev nodes, the zeros of T_p on [0, 1])
Transfer make_transfer(int p, int nodes) {
    Transfer t{};
    if (nodes == GBFMM_NODES_CHEBYSHEV) {
        double tn[GB_MAXP];
        for (int b = 0; b < p; ++b) tn[b] = 0.5 * (1.0 - std::cos(M_PI * double(2 * b + 1) / double(2 * p)));
        for (int c = 0; c < 2; ++c)
            for (int A = 0; A < p; ++A)
                for (int a = 0; a < p; ++a) {
                    const double x = (c + tn[a]) / 2.0;
                    double v = 1.0;
                    for (int b = 0; b < p; ++b)
                        if (b != A) v *= (x - tn[b]) / (tn[A] - tn[b]);
                    t.M[c][A][a] = v;
                }
        return t;
    }
    for (int c = 0; c < 2; ++c)
        for (int A = 0; A < p; ++A)
            for (int a = 0; a < p; ++a) {
                double x = (c + double(a) / (p - 1)) / 2.0;
                double v = 1.0;
                for (int b = 0; b < p; ++b)
                    if (b != A) v *= (x - double(b) / (p - 1)) / (double(A - b) / (p - 1));
                t.M[c][A][a] = v;
            }
    return t;
}

}  // namespace

// points per cell at every level, from the leaf ranges
void compute_occ(gbfmm_ctx *ctx, const int *start, int *occ) {
    const int L = ctx->L;
    const int64_t nl = ctx->n_leaves;
    ++ctx->launches;
    k_occ_leaves<<<nblk(nl, 256), 256, 0, ctx->stream>>>(nl, start, cell_base(L - 1), occ);
    for (int lev = L - 2; lev >= 0; --lev) {
        ++ctx->launches;
        k_occ_up<<<nblk(int64_t(1) << (3 * lev), 256), 256, 0, ctx->stream>>>(lev, occ);
    }
}

namespace {
// near pairs per target point: sources in the 27 neighbour leaves minus the
// points of its own segment that lie there
// (adaptive tree: a point of a split leaf meets, in another split leaf, the points of the
// children adjacent to its own child only)
__device__ inline bool fine_adjacent(int ox, int oy, int oz, int ca, int cb) {
    return abs(2 * ox + (cb & 1) - (ca & 1)) <= 1 && abs(2 * oy + ((cb >> 1) & 1) - ((ca >> 1) & 1)) <= 1 &&
           abs(2 * oz + (cb >> 2) - (ca >> 2)) <= 1;
}
__global__ void k_count_near(int64_t N, int L, int n_g, const int *__restrict__ start, const int *__restrict__ pleaf,
                             const int64_t *__restrict__ sid, const int *__restrict__ pos,
                             const int *__restrict__ ref_start, const int *__restrict__ child_start,
                             const int *__restrict__ pfine, unsigned long long *__restrict__ out) {
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    unsigned long long c = 0;
    if (i < N) {
        const int nl = 1 << (L - 1);
        int bx, by, bz;
        const int Bl = pleaf[i];
        cell_xyz(Bl, nl, bx, by, bz);
        const int fi = pfine ? pfine[i] : -1;
        for (int nb = 0; nb < 27; ++nb) {
            int ax = bx + nb % 3 - 1, ay = by + (nb / 3) % 3 - 1, az = bz + nb / 9 - 1;
            if (ax < 0 || ay < 0 || az < 0 || ax >= nl || ay >= nl || az >= nl) continue;
            int64_t A = (int64_t(az) * nl + ay) * nl + ax;
            if (fi >= 0 && A != Bl && ref_start[A + 1] > ref_start[A]) {
                const int rA = ref_start[A];
                for (int cb = 0; cb < 8; ++cb)
                    if (fine_adjacent(ax - bx, ay - by, az - bz, fi & 7, cb))
                        c += child_start[9 * rA + cb + 1] - child_start[9 * rA + cb];
            } else {
                c += start[A + 1] - start[A];
            }
        }
        const int64_t s = sid[i];
        for (int g = 0; g < n_g; ++g) {
            const int j = pos[s * n_g + g];
            int ox, oy, oz;
            cell_xyz(pleaf[j], nl, ox, oy, oz);
            if (abs(ox - bx) > 1 || abs(oy - by) > 1 || abs(oz - bz) > 1) continue;
            const int fj = pfine ? pfine[j] : -1;
            if (fi >= 0 && fj >= 0 && pleaf[j] != Bl && !fine_adjacent(ox - bx, oy - by, oz - bz, fi & 7, fj & 7))
                continue;  // not a near pair of the adaptive tree
            --c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// levels 2 .. Lm - 1 (Lm = L + 1 adds the adaptive tree's children)
__global__ void k_count_m2l(int L, int Lm, const int *__restrict__ occ, unsigned long long *__restrict__ out) {
    int64_t g = cell_base_d(2) + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    unsigned long long c = 0, leaves = 0;
    if (g < cell_base_d(Lm)) {
        int lev = 2;
        while (lev + 1 < Lm && g >= cell_base_d(lev + 1)) ++lev;
        const int n = 1 << lev;
        int bx, by, bz;
        cell_xyz(g - cell_base_d(lev), n, bx, by, bz);
        if (occ[g] > 0) {
            if (lev == L - 1) leaves = 1;
            for (int nb = 0; nb < 27; ++nb) {
                const int px = bx / 2 + nb % 3 - 1, py = by / 2 + (nb / 3) % 3 - 1, pz = bz / 2 + nb / 9 - 1;
                for (int ch = 0; ch < 8; ++ch) {
                    const int ax = 2 * px + (ch & 1), ay = 2 * py + ((ch >> 1) & 1), az = 2 * pz + (ch >> 2);
                    if (ax < 0 || ay < 0 || az < 0 || ax >= n || ay >= n || az >= n) continue;
                    if (abs(bx - ax) <= 1 && abs(by - ay) <= 1 && abs(bz - az) <= 1) continue;
                    if (occ[cell_base_d(lev) + (int64_t(az) * n + ay) * n + ax] > 0) ++c;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        leaves += __shfl_down_sync(0xffffffffu, leaves, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(out + 1, c);
        if (leaves) atomicAdd(out + 2, leaves);
    }
}
}  // namespace

int work_counts(gbfmm_ctx *ctx, int64_t *res) {
    cudaStream_t st = ctx->stream;
    unsigned long long *d = nullptr;
    CK(cudaMallocAsync(&d, 4 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), st));
    int *occ = ctx->d_tmp_i;
    const int L = ctx->L;
    compute_occ(ctx, ctx->d_leaf_start, occ);
    const auto &RF = ctx->rf;
    const bool fine = RF.on && L >= 3 && RF.fine_rows() > 0;
    if (fine) {  // the children of split leaves at level L
        const int64_t n_fine = RF.fine_rows();
        CK(cudaMemsetAsync(occ + cell_base(L), 0, (cell_base(L + 1) - cell_base(L)) * sizeof(int), st));
        ++ctx->launches;
        k_fine_occ<<<nblk(n_fine, 256), 256, 0, st>>>(n_fine, L, RF.ref_start + ctx->n_leaves, RF.ref_leaf,
                                                      RF.child_start, occ + cell_base(L));
    }
    ++ctx->launches;
    k_count_near<<<nblk(ctx->N, 256), 256, 0, st>>>(ctx->N, L, ctx->opt.n_gauss, ctx->d_leaf_start, ctx->d_pleaf,
                                                     ctx->d_sid, ctx->d_pos, fine ? RF.ref_start : nullptr,
                                                     RF.child_start, fine ? RF.pfine : nullptr, d);
    ++ctx->launches;
    const int Lm = fine ? L + 1 : L;
    k_count_m2l<<<nblk(cell_base(Lm) - cell_base(2), 256), 256, 0, st>>>(L, Lm, occ, d);
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(d, st));
    CK(cudaStreamSynchronize(st));
    res[0] = int64_t(h[0]);
    res[1] = int64_t(h[1]);
    res[2] = int64_t(h[2]);
    res[3] = ctx->N;
    return GBFMM_OK;
}

void timer_mark(gbfmm_ctx *ctx) {
    if (!ctx->timer.on || ctx->timer.n >= 16) return;
    cudaEventRecord(ctx->timer.ev[ctx->timer.n++], ctx->stream);
}

int near_run_sym64(gbfmm_ctx *ctx, double *sig);  // near.cu

// Runs the pass.  free_targets: targets are the sorted free points of
// targets_sort (no segment exclusion), else the sorted Gauss points.
int fmm_pass(gbfmm_ctx *ctx, bool free_targets, int64_t n_t) {
    cudaStream_t st = ctx->stream;
    const int p = ctx->opt.p, L = ctx->L, P3 = p * p * p;
    const int64_t N = ctx->N, nl = ctx->n_leaves;
    int *occ = ctx->d_tmp_i;                 // [n_cells] sources per cell
    int *tocc = free_targets ? occ + ctx->n_cells : occ;
    const int *tstart = free_targets ? ctx->d_t_start : ctx->d_leaf_start;
    Transfer tr = make_transfer(p, ctx->opt.nodes);

    timer_mark(ctx);
    ++ctx->launches;
    k_precontract<double><<<nblk(N, 128), 128, 0, st>>>(N, ctx->d_q, ctx->d_Asym, ctx->d_P);
    compute_occ(ctx, ctx->d_leaf_start, occ);
    if (free_targets) compute_occ(ctx, ctx->d_t_start, tocc);
    CK(cudaGetLastError());
    timer_mark(ctx);
    if (L >= 3) {
        ++ctx->launches;
        k_p2m<double><<<unsigned(nl), 256, 0, st>>>(p, ctx->opt.nodes, L, ctx->d_box, ctx->d_leaf_start, ctx->d_y, ctx->d_q, ctx->d_W);
        const size_t sm9 = size_t(2) * P3 * 9 * sizeof(double);
        for (int lev = L - 2; lev >= 2; --lev)
            { ++ctx->launches; k_m2m<double><<<unsigned(int64_t(1) << (3 * lev)), 256, sm9, st>>>(p, lev, tr, occ, ctx->d_W); }
        CK(cudaGetLastError());
    }
    timer_mark(ctx);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (L >= 3 && ctx->opt.m2l_fft && cap == cudaStreamCaptureStatusNone) {
        if (int rc = m2l_fft_run(ctx, occ, tocc)) return rc;
    } else if (L >= 3) {
        const int64_t ncell = ctx->n_cells - cell_base(2);
        const int bd = ((P3 + 31) / 32) * 32;
        ++ctx->launches;
        k_m2l_f64<<<unsigned(ncell), bd, P3 * 9 * sizeof(double), st>>>(p, L, ctx->lat_n, ctx->d_box, ctx->d_Klat,
                                                                         occ, tocc, ctx->d_W, ctx->d_S);
        CK(cudaGetLastError());
    }
    timer_mark(ctx);
    if (L >= 4) {
        const size_t sm6 = size_t(2) * P3 * 6 * sizeof(double);
        for (int lev = 3; lev <= L - 1; ++lev)
            { ++ctx->launches; k_l2l<double><<<unsigned(int64_t(1) << (3 * lev)), 256, sm6, st>>>(p, lev, tr, tocc, ctx->d_S); }
        CK(cudaGetLastError());
    }
    timer_mark(ctx);
    if (!free_targets && ctx->mat.mode == GBFMM_H_CIRCLE) {
        // nodal forces with the unit-circle h: one h per unordered point pair (h is odd)
        if (int rc = near_run_sym64(ctx, ctx->d_sig)) return rc;
    } else {
        const size_t smem = (size_t(P3) * 6 + 64 * 3 + 64 * 108) * sizeof(double) + 64 * sizeof(int64_t);
        const double *xt = free_targets ? ctx->d_t_x : ctx->d_y;
        const int64_t *tsid = free_targets ? nullptr : ctx->d_sid;
        double *sig = free_targets ? ctx->d_t_sig : ctx->d_sig;
        ++ctx->launches;
        if (ctx->mat.mode == GBFMM_H_ISO)
            k_leaf_eval_f64<GBFMM_H_ISO><<<unsigned(nl), 128, smem, st>>>(
                p, ctx->opt.nodes, L, ctx->d_box, ctx->d_mat, tstart, xt, tsid, ctx->d_leaf_start, ctx->d_y, ctx->d_P, ctx->d_sid,
                ctx->d_S, sig);
        else
            k_leaf_eval_f64<GBFMM_H_CIRCLE><<<unsigned(nl), 128, smem, st>>>(
                p, ctx->opt.nodes, L, ctx->d_box, ctx->d_mat, tstart, xt, tsid, ctx->d_leaf_start, ctx->d_y, ctx->d_P, ctx->d_sid,
                ctx->d_S, sig);
        CK(cudaGetLastError());
    }
    timer_mark(ctx);
    (void)n_t;
    return GBFMM_OK;
}

int forces_from_stress(gbfmm_ctx *ctx, double *f_nodes, double *f_seg, double *sigma_pts) {
    ForceParams fp{};
    fp.n = ctx->opt.n_gauss;
    for (int i = 0; i < fp.n; ++i) {
        fp.xi[i] = ctx->gauss_xi[i];
        fp.w[i] = ctx->gauss_w[i];
    }
    CK(cudaMemsetAsync(f_nodes, 0, ctx->n_nodes * 3 * sizeof(double), ctx->stream));
    ++ctx->launches;
    k_forces<<<nblk(ctx->n_segs, 128), 128, 0, ctx->stream>>>(ctx->n_segs, fp, ctx->node_xyz, ctx->seg_nodes,
                                                               ctx->burgers, ctx->d_pos, ctx->d_sig, f_nodes, f_seg,
                                                               sigma_pts);
    CK(cudaGetLastError());
    timer_mark(ctx);
    return GBFMM_OK;
}

int targets_scatter(gbfmm_ctx *ctx, int64_t n_t, double *sigma) {
    ++ctx->launches;
    k_scatter_targets<<<nblk(n_t, 256), 256, 0, ctx->stream>>>(n_t, ctx->d_t_pos, ctx->d_t_sig, sigma);
    CK(cudaGetLastError());
    return GBFMM_OK;
}

int mixed_kernel_attrs(gbfmm_ctx *ctx);

int fmm_kernel_attrs(gbfmm_ctx *ctx) {
    if (int rc = mixed_kernel_attrs(ctx)) return rc;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p;
    const size_t smem = (size_t(P3) * 6 + 64 * 3 + 64 * 108) * sizeof(double) + 64 * sizeof(int64_t);
    CK(cudaFuncSetAttribute(k_leaf_eval_f64<GBFMM_H_ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    CK(cudaFuncSetAttribute(k_leaf_eval_f64<GBFMM_H_CIRCLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    CK(cudaFuncSetAttribute(k_m2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(2 * P3 * 9 * sizeof(double))));
    CK(cudaFuncSetAttribute(k_l2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(2 * P3 * 6 * sizeof(double))));
    CK(cudaFuncSetAttribute(k_m2l_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, int(P3 * 9 * sizeof(double))));
    return GBFMM_OK;
}

int near_prepare(gbfmm_ctx *ctx);  // near.cu
int near_alloc(gbfmm_ctx *ctx, int64_t n_targets);  // near.cu
int near_sym_alloc(gbfmm_ctx *ctx);                 // near.cu
int near_run(gbfmm_ctx *ctx, const int *tstart, const double *xt, const int64_t *tsid, double *sig);

int mixed_alloc(gbfmm_ctx *ctx) {
    const int64_t N = ctx->N, nc = ctx->n_cells;
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p;
    if (int rc = grow_dev(ctx, ctx->mx_cap_N, N,
                          {{(void **)&ctx->d_Pf, N * 108 * sizeof(float)}, {(void **)&ctx->d_yrel, N * sizeof(float4)}},
                          "mixed-pass points"))
        return rc;
    if (int rc = grow_dev(ctx, ctx->mx_cap_cells, nc,
                          {{(void **)&ctx->d_Wf, nc * P3 * 9 * sizeof(float)},
                           {(void **)&ctx->d_Sf, nc * P3 * 6 * sizeof(float)}},
                          "mixed-pass cells"))
        return rc;
    if (int rc = near_alloc(ctx, N)) return rc;
    if (int rc = near_sym_alloc(ctx)) return rc;
    if (!ctx->tc.ready_ops) {
        int rc = m2l_tc_setup(ctx);
        if (rc) return rc;
    }
    return m2l_tc_prepare(ctx);
}

// leaf-level local values FP64 -> FP32 (GBFMM_MIXED_F64T, for the near kernels that read FP32)
__global__ void k_leaf_s_to_f32(int64_t n, const double *__restrict__ S, float *__restrict__ Sf) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        Sf[i] = float(S[i]);
}

int mixed_pass(gbfmm_ctx *ctx, bool free_targets, int64_t n_t) {
    if (!ctx->tc.ready_ops) {  // the medium changed after the build
        if (int rc = m2l_tc_setup(ctx)) return rc;
        if (int rc = m2l_tc_prepare(ctx)) return rc;
    }
    cudaStream_t st = ctx->stream;
    const bool t64 = ctx->opt.precision == GBFMM_MIXED_F64T;  // FP64 P2M, M2M, L2L, L2P
    const int p = ctx->opt.p, L = ctx->L, P3 = p * p * p;
    const int64_t N = ctx->N, nl = ctx->n_leaves;
    int *occ = ctx->d_tmp_i;
    int *tocc = free_targets ? occ + ctx->n_cells : occ;
    const int *tstart = free_targets ? ctx->d_t_start : ctx->d_leaf_start;
    Transfer tr = make_transfer(p, ctx->opt.nodes);
    // adaptive tree: the children of split leaves take part in nodal-force passes (free
    // targets keep the uniform tree, whose near field covers whole leaves)
    auto &RF = ctx->rf;
    const int64_t n_fine = RF.fine_rows();
    const bool fine = RF.on && !free_targets && L >= 3 && n_fine > 0;
    const int *n_ref = RF.ref_start ? RF.ref_start + nl : nullptr;
    timer_mark(ctx);
    if (int rc = near_prepare(ctx)) return rc;
    ++ctx->launches;
    k_prep_mixed<<<nblk(N, 256), 256, 0, st>>>(N, L, ctx->d_box, ctx->d_y, ctx->d_pleaf, ctx->d_slen, ctx->d_yrel);
    compute_occ(ctx, ctx->d_leaf_start, occ);
    if (free_targets) compute_occ(ctx, ctx->d_t_start, tocc);
    CK(cudaGetLastError());
    timer_mark(ctx);
    if (L >= 3) {
        ++ctx->launches;
        if (t64)
            k_p2m<double><<<unsigned(nl), 256, 0, st>>>(p, ctx->opt.nodes, L, ctx->d_box, ctx->d_leaf_start, ctx->d_y, ctx->d_q,
                                                        ctx->d_W);
        else
            k_p2m<float><<<unsigned(nl), 256, 0, st>>>(p, ctx->opt.nodes, L, ctx->d_box, ctx->d_leaf_start, ctx->d_y, ctx->d_q,
                                                       ctx->d_Wf);
        for (int lev = L - 2; lev >= 2; --lev) {
            ++ctx->launches;
            const unsigned g = unsigned(int64_t(1) << (3 * lev));
            if (t64)
                k_m2m<double><<<g, 256, size_t(2) * P3 * 9 * sizeof(double), st>>>(p, lev, tr, occ, ctx->d_W);
            else
                k_m2m_merge<float><<<g, 256, size_t(4) * P3 * 9 * sizeof(float), st>>>(p, lev, tr, occ, ctx->d_Wf);
        }
        if (fine) {
            // the children of split leaves: their multipole values
            ++ctx->launches;
            k_p2m_fine<float><<<unsigned(n_fine), 256, 0, st>>>(p, ctx->opt.nodes, L, ctx->d_box, n_ref, RF.ref_leaf,
                                                                RF.child_start, ctx->d_y, ctx->d_q, RF.W7);
        }
        CK(cudaGetLastError());
    }
    timer_mark(ctx);
    if (L >= 3) {
        int rc = m2l_tc_run(ctx, ctx->d_Wf, t64 ? ctx->d_W : nullptr, occ, tocc, ctx->d_Sf, t64 ? ctx->d_S : nullptr,
                            fine);
        if (rc) return rc;
    }
    timer_mark(ctx);
    if (L >= 4) {
        for (int lev = 3; lev <= L - 1; ++lev) {
            ++ctx->launches;
            const unsigned g = unsigned(int64_t(1) << (3 * lev));
            if (t64)
                k_l2l<double><<<g, 256, size_t(2) * P3 * 6 * sizeof(double), st>>>(p, lev, tr, tocc, ctx->d_S);
            else  // one block per parent
                k_l2l_split<float><<<g / 8, 256, size_t(7) * P3 * 6 * sizeof(float), st>>>(p, lev, tr, tocc,
                                                                                          ctx->d_Sf);
        }
        CK(cudaGetLastError());
    }
    if (fine) {
        // the children's local values (the level-L M2L, written by m2l_tc_run) += the parent's
        ++ctx->launches;
        k_l2l_fine<float><<<unsigned(n_fine), 256, size_t(2) * P3 * 6 * sizeof(float), st>>>(
            p, L, tr, n_ref, RF.ref_leaf, RF.child_start, ctx->d_Sf, RF.S7);
        CK(cudaGetLastError());
    }
    if (t64 && L >= 3) {
        // FP32 copy of the leaf level for the near kernels that read FP32 local values
        const int64_t n = nl * P3 * 6;
        ++ctx->launches;
        k_leaf_s_to_f32<<<unsigned(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, st>>>(
            n, ctx->d_S + cell_base(L - 1) * P3 * 6, ctx->d_Sf + cell_base(L - 1) * P3 * 6);
    }
    timer_mark(ctx);
    {
        const double *xt = free_targets ? ctx->d_t_x : ctx->d_y;
        const int64_t *tsid = free_targets ? nullptr : ctx->d_sid;
        double *sig = free_targets ? ctx->d_t_sig : ctx->d_sig;
        if (int rc = near_run(ctx, tstart, xt, tsid, sig)) return rc;
    }
    timer_mark(ctx);
    (void)n_t;
    return GBFMM_OK;
}

int mixed_kernel_attrs(gbfmm_ctx *ctx) {
    const int P3 = ctx->opt.p * ctx->opt.p * ctx->opt.p;
    CK(cudaFuncSetAttribute(k_m2m_merge<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(4 * P3 * 9 * sizeof(float))));
    CK(cudaFuncSetAttribute(k_l2l_split<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(7 * P3 * 6 * sizeof(float))));
    CK(cudaFuncSetAttribute(k_l2l_fine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(2 * P3 * 6 * sizeof(float))));
    return GBFMM_OK;
}
