/*
 * FP64 CPU oracle for the dislocation stress / Peach-Koehler force path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * calls it, and it shares no code with the CUDA sources.
 *
 * What it computes (arXiv:1712.07739):
 *   - Mura's stress formula (Section 2, Eq. "stress"): for a closed loop,
 *       sigma_ab(x) = b_w  oint  eps_ngr C_abvg C_pqwn dG_vp/dx_q (x - y) dy_r
 *   - the DD kernel (Section 2, Eq. "kernel"):
 *       K_abwr(x - y) = eps_ngr C_abvg C_pqwn dG_vp/dx_q (x - y)
 *     written here as K_abwr = A[ab][wr][vpq] h_vpq(T) / R^2 with
 *     A_{ab,wr,vpq} = sum_{n,g} eps_ngr C_abvg C_pqwn and
 *     dG_vp/dx_q = h_vpq(T)/R^2, T = (x - y)/R.
 *   - h for an isotropic medium from the Green's function of Section 2,
 *     Eq. "k_iso" (Kelvin's solution), differentiated in closed form:
 *       G_vp = [(3 - 4 nu) delta_vp + T_v T_p] / (16 pi mu (1 - nu) R)
 *       h_vpq = [-(3-4nu) delta_vp T_q + delta_vq T_p + delta_pq T_v
 *                - 3 T_v T_p T_q] / (16 pi mu (1 - nu))
 *   - h for a general anisotropic medium by the unit-circle integral of the
 *     Green's function (the paper evaluates the same derivative by a series,
 *     Section 2, Eq. "k_aniso"; this oracle uses the line integral over the
 *     unit circle z . T = 0, which has a plain definition):
 *       G(x)      = 1/(8 pi^2 R) oint (zz)^-1 dphi
 *       h_vpq(T)  = 1/(8 pi^2)  oint [ -T_q (zz)^-1_vp + z_q F_vp ] dphi
 *       F = (zz)^-1 [(zT) + (Tz)] (zz)^-1,  (ab)_jk = a_i C_ijkl b_l
 *     The integrand has period pi in phi (z -> -z leaves it unchanged), so
 *     the integral is twice a Q-point trapezoid sum over [0, pi).
 *   - the discrete N-body sum (Section 2, Eq. "stress3"):
 *       s(x_i) = sum_j K(x_i - y_j) q_j,  points of the target's own segment
 *       excluded (the kernel is singular there, Section 4.3).
 *
 * Index conventions: C is C[i][j][k][l] row-major (81 doubles); h is
 * h[v][p][q] (27); K is K[ab][w][r] with ab in Voigt order
 * xx, yy, zz, yz, xz, xy (6 x 9 = 54); q is q[w][r] (9); stress is Voigt (6).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

static const int VA[6] = {0, 1, 2, 1, 0, 0};
static const int VB[6] = {0, 1, 2, 2, 2, 1};

static double eps3(int i, int j, int k) {
    return (double)((i - j) * (j - k) * (k - i)) / 2.0;
}

/* A_{ab,wr,vpq} = sum_{n,g} eps_ngr C_{a b v g} C_{p q w n}  (Eq. "kernel") */
void orc_A_tensor(const double *C, double *A) {
    for (int ab = 0; ab < 6; ++ab) {
        int a = VA[ab], b = VB[ab];
        for (int w = 0; w < 3; ++w)
            for (int r = 0; r < 3; ++r)
                for (int v = 0; v < 3; ++v)
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) {
                            double s = 0.0;
                            for (int n = 0; n < 3; ++n)
                                for (int g = 0; g < 3; ++g) {
                                    double e = eps3(n, g, r);
                                    if (e == 0.0) continue;
                                    s += e * C[((a * 3 + b) * 3 + v) * 3 + g] *
                                         C[((p * 3 + q) * 3 + w) * 3 + n];
                                }
                            A[(ab * 9 + w * 3 + r) * 27 + v * 9 + p * 3 + q] = s;
                        }
    }
}

void orc_h_iso(double mu, double nu, const double *T, double *h) {
    double c = 1.0 / (16.0 * PI * mu * (1.0 - nu));
    double a = 3.0 - 4.0 * nu;
    for (int v = 0; v < 3; ++v)
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                double s = -3.0 * T[v] * T[p] * T[q];
                if (v == p) s -= a * T[q];
                if (v == q) s += T[p];
                if (p == q) s += T[v];
                h[v * 9 + p * 3 + q] = c * s;
            }
}

/* (ab)_jk = a_i C_ijkl b_l */
static void cmat(const double *C, const double *a, const double *b, double *M) {
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int l = 0; l < 3; ++l)
                    s += a[i] * C[((i * 3 + j) * 3 + k) * 3 + l] * b[l];
            M[j * 3 + k] = s;
        }
}

static void inv3(const double *M, double *R) {
    double c00 = M[4] * M[8] - M[5] * M[7];
    double c01 = M[5] * M[6] - M[3] * M[8];
    double c02 = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    double id = 1.0 / det;
    R[0] = c00 * id;
    R[1] = (M[2] * M[7] - M[1] * M[8]) * id;
    R[2] = (M[1] * M[5] - M[2] * M[4]) * id;
    R[3] = c01 * id;
    R[4] = (M[0] * M[8] - M[2] * M[6]) * id;
    R[5] = (M[2] * M[3] - M[0] * M[5]) * id;
    R[6] = c02 * id;
    R[7] = (M[1] * M[6] - M[0] * M[7]) * id;
    R[8] = (M[0] * M[4] - M[1] * M[3]) * id;
}

static void mm3(const double *A, const double *B, double *R) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}

/* Orthonormal pair (e1, e2) spanning the plane normal to unit T.
 * rot rotates the pair in that plane by the given angle (used by the pins
 * that check independence of the circle parametrisation). */
static void circle_basis(const double *T, double rot, double *e1, double *e2) {
    double a[3] = {0, 0, 0};
    int k = 0;
    if (fabs(T[1]) < fabs(T[k])) k = 1;
    if (fabs(T[2]) < fabs(T[k])) k = 2;
    a[k] = 1.0;
    double d = a[0] * T[0] + a[1] * T[1] + a[2] * T[2];
    double u[3] = {a[0] - d * T[0], a[1] - d * T[1], a[2] - d * T[2]};
    double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int i = 0; i < 3; ++i) u[i] /= n;
    double w[3] = {T[1] * u[2] - T[2] * u[1], T[2] * u[0] - T[0] * u[2], T[0] * u[1] - T[1] * u[0]};
    double c = cos(rot), s = sin(rot);
    for (int i = 0; i < 3; ++i) {
        e1[i] = c * u[i] + s * w[i];
        e2[i] = -s * u[i] + c * w[i];
    }
}

void orc_G_circle_rot(const double *C, const double *x, int Q, double rot, double *G) {
    double R = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double T[3] = {x[0] / R, x[1] / R, x[2] / R};
    double e1[3], e2[3];
    circle_basis(T, rot, e1, e2);
    double acc[9] = {0};
    for (int k = 0; k < Q; ++k) {
        double ph = PI * (double)k / (double)Q;
        double z[3];
        for (int i = 0; i < 3; ++i) z[i] = cos(ph) * e1[i] + sin(ph) * e2[i];
        double M[9], Mi[9];
        cmat(C, z, z, M);
        inv3(M, Mi);
        for (int i = 0; i < 9; ++i) acc[i] += Mi[i];
    }
    /* oint dphi over [0, 2 pi) = 2 * (pi / Q) * sum over [0, pi) */
    double f = 2.0 * (PI / Q) / (8.0 * PI * PI * R);
    for (int i = 0; i < 9; ++i) G[i] = f * acc[i];
}

void orc_G_circle(const double *C, const double *x, int Q, double *G) {
    orc_G_circle_rot(C, x, Q, 0.0, G);
}

void orc_h_circle_rot(const double *C, const double *Tin, int Q, double rot, double *h) {
    double n = sqrt(Tin[0] * Tin[0] + Tin[1] * Tin[1] + Tin[2] * Tin[2]);
    double T[3] = {Tin[0] / n, Tin[1] / n, Tin[2] / n};
    double e1[3], e2[3];
    circle_basis(T, rot, e1, e2);
    double acc[27] = {0};
    for (int k = 0; k < Q; ++k) {
        double ph = PI * (double)k / (double)Q;
        double z[3];
        for (int i = 0; i < 3; ++i) z[i] = cos(ph) * e1[i] + sin(ph) * e2[i];
        double M[9], Mi[9], ZT[9], TZ[9], S[9], tmp[9], F[9];
        cmat(C, z, z, M);
        inv3(M, Mi);
        cmat(C, z, T, ZT);
        cmat(C, T, z, TZ);
        for (int i = 0; i < 9; ++i) S[i] = ZT[i] + TZ[i];
        mm3(Mi, S, tmp);
        mm3(tmp, Mi, F);
        for (int v = 0; v < 3; ++v)
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                    acc[v * 9 + p * 3 + q] += -T[q] * Mi[v * 3 + p] + z[q] * F[v * 3 + p];
    }
    double f = 2.0 * (PI / Q) / (8.0 * PI * PI);
    for (int i = 0; i < 27; ++i) h[i] = f * acc[i];
}

void orc_h_circle(const double *C, const double *T, int Q, double *h) {
    orc_h_circle_rot(C, T, Q, 0.0, h);
}

/* Material descriptor for the kernel evaluation.
 * mode 0: isotropic closed form (mu, nu); mode 1: unit-circle integral (C, Q). */
typedef struct {
    int mode;
    int Q;
    double mu, nu;
    const double *C;
    const double *A; /* [54][27] */
} orc_mat;

static void eval_h(const orc_mat *m, const double *T, double *h) {
    if (m->mode == 0)
        orc_h_iso(m->mu, m->nu, T, h);
    else
        orc_h_circle(m->C, T, m->Q, h);
}

/* K_abwr(d) = A_{ab,wr,vpq} h_vpq(d/|d|) / |d|^2 */
static void eval_K(const orc_mat *m, const double *d, double *K) {
    double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double R = sqrt(R2);
    double T[3] = {d[0] / R, d[1] / R, d[2] / R};
    double h[27];
    eval_h(m, T, h);
    for (int i = 0; i < 54; ++i) {
        double s = 0.0;
        for (int c = 0; c < 27; ++c) s += m->A[i * 27 + c] * h[c];
        K[i] = s / R2;
    }
}

void orc_kernel_batch(int mode, double mu, double nu, const double *C, int Q, const double *A,
                      int64_t n, const double *d, double *K, int nthreads) {
    orc_mat m = {mode, Q, mu, nu, C, A};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) eval_K(&m, d + 3 * i, K + 54 * i);
}

/* Direct sum of Eq. "stress3" at n_t targets:
 *   sigma(x_i) = sum_{j : sseg[j] != tseg[i]} K(x_i - y_j) q_j
 * xt [n_t][3], tseg [n_t], ys [n_s][3], qs [n_s][9], sseg [n_s]; out [n_t][6].
 * Returns the number of OpenMP threads used. */
int orc_direct_stress(int mode, double mu, double nu, const double *C, int Q, const double *A,
                      int64_t n_t, const double *xt, const int64_t *tseg,
                      int64_t n_s, const double *ys, const double *qs, const int64_t *sseg,
                      double *out, int nthreads) {
    orc_mat m = {mode, Q, mu, nu, C, A};
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t i = 0; i < n_t; ++i) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n_s; ++j) {
            if (sseg[j] == tseg[i]) continue;
            double d[3] = {xt[3 * i] - ys[3 * j], xt[3 * i + 1] - ys[3 * j + 1],
                           xt[3 * i + 2] - ys[3 * j + 2]};
            double K[54];
            eval_K(&m, d, K);
            for (int ab = 0; ab < 6; ++ab) {
                double t = 0.0;
                for (int c = 0; c < 9; ++c) t += K[ab * 9 + c] * qs[9 * j + c];
                s[ab] += t;
            }
        }
        for (int ab = 0; ab < 6; ++ab) out[6 * i + ab] = s[ab];
    }
    return used;
}
