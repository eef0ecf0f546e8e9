// Device arithmetic of the dislocation kernel, shared by the setup and the
// near-field kernels of this library.
//
// The kernel of Sec. 2, Eq. "kernel" is K_abwr = A_{ab,wr,vpq} dG_vp/dx_q
// with dG_vp/dx_q = h_vpq(T) / R^2.  h is symmetric in (v, p), so only 18
// components are kept, in the order k = 3 * pair + q with pairs
// (0,0) (1,1) (2,2) (1,2) (0,2) (0,1).
#pragma once
#include "internal.cuh"

// Isotropic medium: derivative of the Kelvin Green's function
// G_vp = [(3 - 4 nu) delta_vp + T_v T_p] / (16 pi mu (1 - nu) R), which is
// Sec. 2, Eq. "k_iso" with R,ii = 2/R and R,vp = (delta_vp - T_v T_p)/R:
// h_vpq = hc [ -ha delta_vp T_q + delta_vq T_p + delta_pq T_v - 3 T_v T_p T_q ].
template <typename R>
__device__ __forceinline__ void h_iso_sym(R hc, R ha, const R T[3], R hs[18]) {
    constexpr int PV[6] = {0, 1, 2, 1, 0, 0};
    constexpr int PP[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
        const int v = PV[pr], p = PP[pr];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            R s = R(-3) * T[v] * T[p] * T[q];
            if (v == p) s -= ha * T[q];
            if (v == q) s += T[p];
            if (p == q) s += T[v];
            hs[3 * pr + q] = hc * s;
        }
    }
}

// sin and cos of pi k / Q in the precision of the caller (no FP64 on the FP32 path)
template <typename R>
__device__ __forceinline__ void circle_point(int k, int Q, R *s, R *c);
template <>
__device__ __forceinline__ void circle_point<double>(int k, int Q, double *s, double *c) {
    sincospi(double(k) / double(Q), s, c);
}
template <>
__device__ __forceinline__ void circle_point<float>(int k, int Q, float *s, float *c) {
    sincospif(float(k) / float(Q), s, c);
}

// (a b)_jk = a_i C_ijkl b_l
template <typename R, typename CT>
__device__ __forceinline__ void cmat(const CT *C, const R a[3], const R b[3], R M[9]) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R s = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int l = 0; l < 3; ++l) s += a[i] * R(C[((i * 3 + j) * 3 + k) * 3 + l]) * b[l];
            M[j * 3 + k] = s;
        }
}

// Any medium: h_vpq(T) = 1/(8 pi^2) oint [ -T_q (zz)^-1_vp + z_q F_vp ] dphi
// over the unit circle z . T = 0, F = (zz)^-1 [(zT) + (Tz)] (zz)^-1.
// The integrand has period pi, so the loop is the Q-point trapezoid rule on
// [0, pi) doubled.  C is read through the generic 81-entry tensor.
template <typename R, typename CT>
__device__ __forceinline__ void h_circle_sym(const CT *C, int Q, const R Tin[3], R hs[18]) {
    R T[3] = {Tin[0], Tin[1], Tin[2]};
    // e1: T with its smallest component replaced, orthogonalised; e2 = T x e1
    int k0 = 0;
    if (fabs(T[1]) < fabs(T[k0])) k0 = 1;
    if (fabs(T[2]) < fabs(T[k0])) k0 = 2;
    R e1[3] = {R(0), R(0), R(0)};
    e1[k0] = R(1);
    R d = e1[0] * T[0] + e1[1] * T[1] + e1[2] * T[2];
    for (int i = 0; i < 3; ++i) e1[i] -= d * T[i];
    R n = R(1) / sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] *= n;
    R e2[3] = {T[1] * e1[2] - T[2] * e1[1], T[2] * e1[0] - T[0] * e1[2], T[0] * e1[1] - T[1] * e1[0]};
    R acc[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) acc[i] = 0;
    for (int k = 0; k < Q; ++k) {
        R s, c;
        circle_point<R>(k, Q, &s, &c);
        R z[3];
        for (int i = 0; i < 3; ++i) z[i] = c * e1[i] + s * e2[i];
        R M[9], ZT[9];
        cmat<R, CT>(C, z, z, M);
        cmat<R, CT>(C, z, T, ZT);
        // inverse of the symmetric positive-definite M (adjugate / determinant)
        R i00 = M[4] * M[8] - M[5] * M[7];
        R i01 = M[2] * M[7] - M[1] * M[8];
        R i02 = M[1] * M[5] - M[2] * M[4];
        R i11 = M[0] * M[8] - M[2] * M[6];
        R i12 = M[2] * M[3] - M[0] * M[5];
        R i22 = M[0] * M[4] - M[1] * M[3];
        R idet = R(1) / (M[0] * i00 + M[1] * (M[5] * M[6] - M[3] * M[8]) + M[2] * (M[3] * M[7] - M[4] * M[6]));
        R Mi[9] = {i00 * idet, i01 * idet, i02 * idet, i01 * idet, i11 * idet,
                   i12 * idet, i02 * idet, i12 * idet, i22 * idet};
        R S[9];
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) S[j * 3 + l] = ZT[j * 3 + l] + ZT[l * 3 + j];
        R tmp[9], F[9];
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l)
                tmp[j * 3 + l] = Mi[j * 3] * S[l] + Mi[j * 3 + 1] * S[3 + l] + Mi[j * 3 + 2] * S[6 + l];
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l)
                F[j * 3 + l] = tmp[j * 3] * Mi[l] + tmp[j * 3 + 1] * Mi[3 + l] + tmp[j * 3 + 2] * Mi[6 + l];
        constexpr int PV[6] = {0, 1, 2, 1, 0, 0};
        constexpr int PP[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            const int v = PV[pr], p = PP[pr];
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[3 * pr + q] += -T[q] * Mi[v * 3 + p] + z[q] * F[v * 3 + p];
        }
    }
    // 2 (pi / Q) / (8 pi^2) = 1 / (4 pi Q)
    const R f = R(1.0 / (4.0 * 3.14159265358979323846 * double(Q)));
#pragma unroll
    for (int i = 0; i < 18; ++i) hs[i] = acc[i] * f;
}

// Cubic medium with crystal axes along x, y, z:
// C_ijkl = C12 d_ij d_kl + C44 (d_ik d_jl + d_il d_jk) + D d_ijkl, D = C11 - C12 - 2 C44,
// so (zz)_jk = (C12 + C44) z_j z_k + (C44 |z|^2 + D z_j^2) d_jk and, for z . T = 0,
// (zT) + (Tz) = (C12 + C44) (z_j T_k + z_k T_j) + 2 D z_j T_j d_jk.
// Same integral as h_circle_sym, about a third of the arithmetic.
template <typename R>
__device__ __forceinline__ void h_circle_cubic(R c12, R c44, R D, int Q, const R Tin[3], R hs[18]) {
    R T[3] = {Tin[0], Tin[1], Tin[2]};
    int k0 = 0;
    if (fabs(T[1]) < fabs(T[k0])) k0 = 1;
    if (fabs(T[2]) < fabs(T[k0])) k0 = 2;
    R e1[3] = {R(0), R(0), R(0)};
    e1[k0] = R(1);
    R dd = e1[0] * T[0] + e1[1] * T[1] + e1[2] * T[2];
    for (int i = 0; i < 3; ++i) e1[i] -= dd * T[i];
    R nrm = R(1) / sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] *= nrm;
    R e2[3] = {T[1] * e1[2] - T[2] * e1[1], T[2] * e1[0] - T[0] * e1[2], T[0] * e1[1] - T[1] * e1[0]};
    const R cp = c12 + c44;
    R acc[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) acc[i] = 0;
    for (int k = 0; k < Q; ++k) {
        R sn, cs;
        circle_point<R>(k, Q, &sn, &cs);
        R z[3];
        for (int i = 0; i < 3; ++i) z[i] = cs * e1[i] + sn * e2[i];
        // M = (zz) (symmetric; |z| = 1)
        const R m00 = cp * z[0] * z[0] + c44 + D * z[0] * z[0];
        const R m11 = cp * z[1] * z[1] + c44 + D * z[1] * z[1];
        const R m22 = cp * z[2] * z[2] + c44 + D * z[2] * z[2];
        const R m01 = cp * z[0] * z[1], m02 = cp * z[0] * z[2], m12 = cp * z[1] * z[2];
        // inverse by cofactors
        const R i00 = m11 * m22 - m12 * m12, i01 = m02 * m12 - m01 * m22, i02 = m01 * m12 - m02 * m11;
        const R i11 = m00 * m22 - m02 * m02, i12 = m01 * m02 - m00 * m12, i22 = m00 * m11 - m01 * m01;
        const R idet = R(1) / (m00 * i00 + m01 * i01 + m02 * i02);
        const R Mi[9] = {i00 * idet, i01 * idet, i02 * idet, i01 * idet, i11 * idet,
                         i12 * idet, i02 * idet, i12 * idet, i22 * idet};
        // S = (zT) + (Tz)
        R S[9];
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) S[j * 3 + l] = cp * (z[j] * T[l] + z[l] * T[j]);
        for (int j = 0; j < 3; ++j) S[j * 3 + j] += R(2) * D * z[j] * T[j];
        R tmp[9], F[9];
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l)
                tmp[j * 3 + l] = Mi[j * 3] * S[l] + Mi[j * 3 + 1] * S[3 + l] + Mi[j * 3 + 2] * S[6 + l];
        for (int j = 0; j < 3; ++j)
            for (int l = j; l < 3; ++l)
                F[j * 3 + l] = tmp[j * 3] * Mi[l] + tmp[j * 3 + 1] * Mi[3 + l] + tmp[j * 3 + 2] * Mi[6 + l];
        constexpr int PV[6] = {0, 1, 2, 1, 0, 0};
        constexpr int PP[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            const int v = PV[pr], p = PP[pr];
            const int vl = v < p ? v : p, ph = v < p ? p : v;
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[3 * pr + q] += -T[q] * Mi[v * 3 + p] + z[q] * F[vl * 3 + ph];
        }
    }
    const R f = R(1.0 / (4.0 * 3.14159265358979323846 * double(Q)));
#pragma unroll
    for (int i = 0; i < 18; ++i) hs[i] = acc[i] * f;
}

// FP32 form of h_circle_cubic for the near-field loop: scalar registers only,
// the points (cos, sin)(pi k / Q) of the half circle from a table.
__device__ __forceinline__ void h_cubic_f32(float cp, float c44, float D, int Q, const float2 *__restrict__ tab,
                                            const float T[3], float hs[18]) {
    const float T0 = T[0], T1 = T[1], T2 = T[2];
    int k0 = 0;
    if (fabsf(T1) < fabsf(T0)) k0 = 1;
    if (fabsf(T2) < fabsf(k0 == 0 ? T0 : T1)) k0 = 2;
    float a0 = k0 == 0 ? 1.f : 0.f, a1 = k0 == 1 ? 1.f : 0.f, a2 = k0 == 2 ? 1.f : 0.f;
    const float dd = a0 * T0 + a1 * T1 + a2 * T2;
    a0 -= dd * T0;
    a1 -= dd * T1;
    a2 -= dd * T2;
    const float nr = rsqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    const float e10 = a0 * nr, e11 = a1 * nr, e12 = a2 * nr;
    const float e20 = T1 * e12 - T2 * e11, e21 = T2 * e10 - T0 * e12, e22 = T0 * e11 - T1 * e10;
    const float cpD = cp + D, cpD2 = 2.f * (cp + D);
    // With C = adj(zz), (zz)^-1 = C / det and F = C S C / det^2, so the point's
    // factors fold into z (z / det^2) and the (zz)^-1 sum (C / det); the
    // T-term of the integrand is summed over the points first,
    // sum_k T_q (zz)^-1_vp = T_q sum_k (zz)^-1_vp.
    float acc[18], msum[6];
#pragma unroll
    for (int i = 0; i < 18; ++i) acc[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) msum[i] = 0.f;
    for (int k = 0; k < Q; ++k) {
        const float2 t = tab[k];
        const float z0 = t.x * e10 + t.y * e20, z1 = t.x * e11 + t.y * e21, z2 = t.x * e12 + t.y * e22;
        const float m00 = fmaf(cpD, z0 * z0, c44), m11 = fmaf(cpD, z1 * z1, c44), m22 = fmaf(cpD, z2 * z2, c44);
        const float m01 = cp * z0 * z1, m02 = cp * z0 * z2, m12 = cp * z1 * z2;
        const float i00 = m11 * m22 - m12 * m12, i01 = m02 * m12 - m01 * m22, i02 = m01 * m12 - m02 * m11;
        const float i11 = m00 * m22 - m02 * m02, i12 = m01 * m02 - m00 * m12, i22 = m00 * m11 - m01 * m01;
        float idet;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet) : "f"(m00 * i00 + m01 * i01 + m02 * i02));
        const float s00 = cpD2 * z0 * T0, s11 = cpD2 * z1 * T1, s22 = cpD2 * z2 * T2;
        const float s01 = cp * (z0 * T1 + z1 * T0), s02 = cp * (z0 * T2 + z2 * T0), s12 = cp * (z1 * T2 + z2 * T1);
        // U = C S, F = U C (symmetric), both without the 1 / det factors
        const float u00 = i00 * s00 + i01 * s01 + i02 * s02, u01 = i00 * s01 + i01 * s11 + i02 * s12,
                    u02 = i00 * s02 + i01 * s12 + i02 * s22;
        const float u10 = i01 * s00 + i11 * s01 + i12 * s02, u11 = i01 * s01 + i11 * s11 + i12 * s12,
                    u12 = i01 * s02 + i11 * s12 + i12 * s22;
        const float u20 = i02 * s00 + i12 * s01 + i22 * s02, u21 = i02 * s01 + i12 * s11 + i22 * s12,
                    u22 = i02 * s02 + i12 * s12 + i22 * s22;
        const float F00 = u00 * i00 + u01 * i01 + u02 * i02, F01 = u00 * i01 + u01 * i11 + u02 * i12,
                    F02 = u00 * i02 + u01 * i12 + u02 * i22;
        const float F11 = u10 * i01 + u11 * i11 + u12 * i12, F12 = u10 * i02 + u11 * i12 + u12 * i22,
                    F22 = u20 * i02 + u21 * i12 + u22 * i22;
        const float w = idet * idet;
        const float y0 = z0 * w, y1 = z1 * w, y2 = z2 * w;
        // pairs (00) (11) (22) (12) (02) (01), each with q = 0, 1, 2
        const float Mp[6] = {i00, i11, i22, i12, i02, i01};
        const float Fp[6] = {F00, F11, F22, F12, F02, F01};
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            acc[3 * pr + 0] = fmaf(y0, Fp[pr], acc[3 * pr + 0]);
            acc[3 * pr + 1] = fmaf(y1, Fp[pr], acc[3 * pr + 1]);
            acc[3 * pr + 2] = fmaf(y2, Fp[pr], acc[3 * pr + 2]);
            msum[pr] = fmaf(Mp[pr], idet, msum[pr]);
        }
    }
    const float f = 1.f / (4.f * 3.14159265358979f * float(Q));
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
        hs[3 * pr + 0] = (acc[3 * pr + 0] - T0 * msum[pr]) * f;
        hs[3 * pr + 1] = (acc[3 * pr + 1] - T1 * msum[pr]) * f;
        hs[3 * pr + 2] = (acc[3 * pr + 2] - T2 * msum[pr]) * f;
    }
}

// Same rule with two circle points per step in packed FP32x2 arithmetic
// (one instruction for the two points' products); Q even.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// a b - c d
__device__ __forceinline__ float2 fms2(float2 a, float2 b, float2 c, float2 d) { return fma2(a, b, mul2(neg2(c), d)); }

__device__ __forceinline__ void h_cubic_f32x2(float cp, float c44, float D, int Q, const float4 *__restrict__ tab2,
                                              const float T[3], float hs[18]) {
    const float T0 = T[0], T1 = T[1], T2 = T[2];
    int k0 = 0;
    if (fabsf(T1) < fabsf(T0)) k0 = 1;
    if (fabsf(T2) < fabsf(k0 == 0 ? T0 : T1)) k0 = 2;
    float a0 = k0 == 0 ? 1.f : 0.f, a1 = k0 == 1 ? 1.f : 0.f, a2 = k0 == 2 ? 1.f : 0.f;
    const float dd = a0 * T0 + a1 * T1 + a2 * T2;
    a0 -= dd * T0;
    a1 -= dd * T1;
    a2 -= dd * T2;
    const float nr = rsqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    const float e10 = a0 * nr, e11 = a1 * nr, e12 = a2 * nr;
    const float e20 = T1 * e12 - T2 * e11, e21 = T2 * e10 - T0 * e12, e22 = T0 * e11 - T1 * e10;
    const float2 cpD = f2(cp + D), cp2 = f2(cp), c442 = f2(c44);
    // zT products folded with their constants: s_ii = z_i (2 (cp + D) T_i), s_ij = z_i (cp T_j) + z_j (cp T_i)
    const float2 dT0 = f2(2.f * (cp + D) * T0), dT1 = f2(2.f * (cp + D) * T1), dT2 = f2(2.f * (cp + D) * T2);
    const float2 cT0 = f2(cp * T0), cT1 = f2(cp * T1), cT2 = f2(cp * T2);
    float2 acc[18], msum[6];
#pragma unroll
    for (int i = 0; i < 18; ++i) acc[i] = f2(0.f);
#pragma unroll
    for (int i = 0; i < 6; ++i) msum[i] = f2(0.f);
    for (int k = 0; k < Q / 2; ++k) {
        const float4 t = tab2[k];  // (cos, sin) of points 2k and 2k + 1
        const float2 c = make_float2(t.x, t.z), sn = make_float2(t.y, t.w);
        const float2 z0 = fma2(c, f2(e10), mul2(sn, f2(e20)));
        const float2 z1 = fma2(c, f2(e11), mul2(sn, f2(e21)));
        const float2 z2 = fma2(c, f2(e12), mul2(sn, f2(e22)));
        const float2 m00 = fma2(cpD, mul2(z0, z0), c442), m11 = fma2(cpD, mul2(z1, z1), c442),
                     m22 = fma2(cpD, mul2(z2, z2), c442);
        const float2 cz0 = mul2(cp2, z0), cz1 = mul2(cp2, z1);
        const float2 m01 = mul2(cz0, z1), m02 = mul2(cz0, z2), m12 = mul2(cz1, z2);
        const float2 i00 = fms2(m11, m22, m12, m12), i01 = fms2(m02, m12, m01, m22), i02 = fms2(m01, m12, m02, m11);
        const float2 i11 = fms2(m00, m22, m02, m02), i12 = fms2(m01, m02, m00, m12), i22 = fms2(m00, m11, m01, m01);
        const float2 det = fma2(m00, i00, fma2(m01, i01, mul2(m02, i02)));
        float2 idet;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet.x) : "f"(det.x));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet.y) : "f"(det.y));
        const float2 s00 = mul2(z0, dT0), s11 = mul2(z1, dT1), s22 = mul2(z2, dT2);
        const float2 s01 = fma2(z0, cT1, mul2(z1, cT0)), s02 = fma2(z0, cT2, mul2(z2, cT0)),
                     s12 = fma2(z1, cT2, mul2(z2, cT1));
        // U = C S, F = U C (symmetric), without the 1 / det factors
        const float2 u00 = fma2(i00, s00, fma2(i01, s01, mul2(i02, s02)));
        const float2 u01 = fma2(i00, s01, fma2(i01, s11, mul2(i02, s12)));
        const float2 u02 = fma2(i00, s02, fma2(i01, s12, mul2(i02, s22)));
        const float2 u10 = fma2(i01, s00, fma2(i11, s01, mul2(i12, s02)));
        const float2 u11 = fma2(i01, s01, fma2(i11, s11, mul2(i12, s12)));
        const float2 u12 = fma2(i01, s02, fma2(i11, s12, mul2(i12, s22)));
        const float2 u20 = fma2(i02, s00, fma2(i12, s01, mul2(i22, s02)));
        const float2 u21 = fma2(i02, s01, fma2(i12, s11, mul2(i22, s12)));
        const float2 u22 = fma2(i02, s02, fma2(i12, s12, mul2(i22, s22)));
        const float2 F00 = fma2(u00, i00, fma2(u01, i01, mul2(u02, i02)));
        const float2 F01 = fma2(u00, i01, fma2(u01, i11, mul2(u02, i12)));
        const float2 F02 = fma2(u00, i02, fma2(u01, i12, mul2(u02, i22)));
        const float2 F11 = fma2(u10, i01, fma2(u11, i11, mul2(u12, i12)));
        const float2 F12 = fma2(u10, i02, fma2(u11, i12, mul2(u12, i22)));
        const float2 F22 = fma2(u20, i02, fma2(u21, i12, mul2(u22, i22)));
        const float2 w = mul2(idet, idet);
        const float2 y0 = mul2(z0, w), y1 = mul2(z1, w), y2 = mul2(z2, w);
        const float2 Mp[6] = {i00, i11, i22, i12, i02, i01};
        const float2 Fp[6] = {F00, F11, F22, F12, F02, F01};
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            acc[3 * pr + 0] = fma2(y0, Fp[pr], acc[3 * pr + 0]);
            acc[3 * pr + 1] = fma2(y1, Fp[pr], acc[3 * pr + 1]);
            acc[3 * pr + 2] = fma2(y2, Fp[pr], acc[3 * pr + 2]);
            msum[pr] = fma2(Mp[pr], idet, msum[pr]);
        }
    }
    const float f = 1.f / (4.f * 3.14159265358979f * float(Q));
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
        const float ms = msum[pr].x + msum[pr].y;
        hs[3 * pr + 0] = (acc[3 * pr + 0].x + acc[3 * pr + 0].y - T0 * ms) * f;
        hs[3 * pr + 1] = (acc[3 * pr + 1].x + acc[3 * pr + 1].y - T1 * ms) * f;
        hs[3 * pr + 2] = (acc[3 * pr + 2].x + acc[3 * pr + 2].y - T2 * ms) * f;
    }
}

// The cubic rule of h_cubic_f32 in any precision (the FP64 pass's symmetric
// near field): points from a table, the adjugate C of (zz) with
// (zz)^-1 = C / det and F = C S C / det^2, so each point costs one reciprocal.
template <typename R>
__device__ __forceinline__ void h_cubic_tab(R cp, R c44, R D, int Q, const R *__restrict__ tab_c,
                                            const R *__restrict__ tab_s, const R T[3], R hs[18]) {
    const R T0 = T[0], T1 = T[1], T2 = T[2];
    int k0 = 0;
    if (fabs(T1) < fabs(T0)) k0 = 1;
    if (fabs(T2) < fabs(k0 == 0 ? T0 : T1)) k0 = 2;
    R a0 = k0 == 0 ? R(1) : R(0), a1 = k0 == 1 ? R(1) : R(0), a2 = k0 == 2 ? R(1) : R(0);
    const R dd = a0 * T0 + a1 * T1 + a2 * T2;
    a0 -= dd * T0;
    a1 -= dd * T1;
    a2 -= dd * T2;
    const R nr = R(1) / sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    const R e10 = a0 * nr, e11 = a1 * nr, e12 = a2 * nr;
    const R e20 = T1 * e12 - T2 * e11, e21 = T2 * e10 - T0 * e12, e22 = T0 * e11 - T1 * e10;
    const R cpD = cp + D, cpD2 = R(2) * (cp + D);
    R acc[18], msum[6];
#pragma unroll
    for (int i = 0; i < 18; ++i) acc[i] = R(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) msum[i] = R(0);
    for (int k = 0; k < Q; ++k) {
        const R c = tab_c[k], sn = tab_s[k];
        const R z0 = c * e10 + sn * e20, z1 = c * e11 + sn * e21, z2 = c * e12 + sn * e22;
        const R m00 = cpD * z0 * z0 + c44, m11 = cpD * z1 * z1 + c44, m22 = cpD * z2 * z2 + c44;
        const R m01 = cp * z0 * z1, m02 = cp * z0 * z2, m12 = cp * z1 * z2;
        const R i00 = m11 * m22 - m12 * m12, i01 = m02 * m12 - m01 * m22, i02 = m01 * m12 - m02 * m11;
        const R i11 = m00 * m22 - m02 * m02, i12 = m01 * m02 - m00 * m12, i22 = m00 * m11 - m01 * m01;
        const R idet = R(1) / (m00 * i00 + m01 * i01 + m02 * i02);
        const R s00 = cpD2 * z0 * T0, s11 = cpD2 * z1 * T1, s22 = cpD2 * z2 * T2;
        const R s01 = cp * (z0 * T1 + z1 * T0), s02 = cp * (z0 * T2 + z2 * T0), s12 = cp * (z1 * T2 + z2 * T1);
        const R u00 = i00 * s00 + i01 * s01 + i02 * s02, u01 = i00 * s01 + i01 * s11 + i02 * s12,
                u02 = i00 * s02 + i01 * s12 + i02 * s22;
        const R u10 = i01 * s00 + i11 * s01 + i12 * s02, u11 = i01 * s01 + i11 * s11 + i12 * s12,
                u12 = i01 * s02 + i11 * s12 + i12 * s22;
        const R u20 = i02 * s00 + i12 * s01 + i22 * s02, u21 = i02 * s01 + i12 * s11 + i22 * s12,
                u22 = i02 * s02 + i12 * s12 + i22 * s22;
        const R F00 = u00 * i00 + u01 * i01 + u02 * i02, F01 = u00 * i01 + u01 * i11 + u02 * i12,
                F02 = u00 * i02 + u01 * i12 + u02 * i22;
        const R F11 = u10 * i01 + u11 * i11 + u12 * i12, F12 = u10 * i02 + u11 * i12 + u12 * i22,
                F22 = u20 * i02 + u21 * i12 + u22 * i22;
        const R w = idet * idet;
        const R y0 = z0 * w, y1 = z1 * w, y2 = z2 * w;
        const R Mp[6] = {i00, i11, i22, i12, i02, i01};
        const R Fp[6] = {F00, F11, F22, F12, F02, F01};
#pragma unroll
        for (int pr = 0; pr < 6; ++pr) {
            acc[3 * pr + 0] += y0 * Fp[pr];
            acc[3 * pr + 1] += y1 * Fp[pr];
            acc[3 * pr + 2] += y2 * Fp[pr];
            msum[pr] += Mp[pr] * idet;
        }
    }
    const R f = R(1.0 / (4.0 * 3.14159265358979323846 * double(Q)));
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
        hs[3 * pr + 0] = (acc[3 * pr + 0] - T0 * msum[pr]) * f;
        hs[3 * pr + 1] = (acc[3 * pr + 1] - T1 * msum[pr]) * f;
        hs[3 * pr + 2] = (acc[3 * pr + 2] - T2 * msum[pr]) * f;
    }
}

// Lagrange basis ell_a(t) = prod_{b != a} (t - t_b) / (t_a - t_b) on the p
// nodes of [0, 1]: nodes = GBFMM_NODES_EQUISPACED, t_a = a / (p - 1) (Sec. 4.1
// footnote); nodes = GBFMM_NODES_CHEBYSHEV, the zeros of the Chebyshev
// polynomial T_p mapped to [0, 1], t_a = (1 - cos((2a + 1) pi / (2p))) / 2
// (the nodes of the Chebyshev FMM, Sec. 3).
template <typename R>
__device__ __forceinline__ R cheb_node(int a, int p) {
    if constexpr (sizeof(R) == 8)
        return 0.5 * (1.0 - cospi(double(2 * a + 1) / double(2 * p)));
    else
        return 0.5f * (1.0f - cospif(float(2 * a + 1) / float(2 * p)));
}

template <typename R>
__device__ __forceinline__ void lagrange_1d(int p, R t, R *out, int nodes) {
    if (nodes == GBFMM_NODES_CHEBYSHEV) {
        // node positions recomputed in the loops: a local table of them, inlined into
        // the near-field kernels next to the three output arrays, gave wrong basis values
        // there (measured: the y-axis values equalled the z-axis ones)
        for (int a = 0; a < p; ++a) {
            const R ta = cheb_node<R>(a, p);
            R v = R(1);
            for (int b = 0; b < p; ++b)
                if (b != a) {
                    const R tb = cheb_node<R>(b, p);
                    v *= (t - tb) / (ta - tb);
                }
            out[a] = v;
        }
        return;
    }
    const R inv = R(1) / R(p - 1);
    for (int a = 0; a < p; ++a) {
        R v = R(1);
        for (int b = 0; b < p; ++b)
            if (b != a) v *= (t - R(b) * inv) / (R(a - b) * inv);
        out[a] = v;
    }
}

// The kernel of Sec. 2, Eq. "kernel" at separation d (FP64, 54 values
// K[ab][wr]): K = sum_k Asym[ab wr][k] h_k(d / |d|) / |d|^2, zero at d = 0.
__device__ __forceinline__ void kernel_at(const DevMaterial *mat, const double *Asym, const double d[3],
                                          double out[54]) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        for (int i = 0; i < 54; ++i) out[i] = 0.0;
        return;
    }
    const double ir = 1.0 / sqrt(r2);
    const double T[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    double hs[18];
    if (mat->mode == GBFMM_H_ISO)
        h_iso_sym<double>(mat->hc, mat->ha, T, hs);
    else if (mat->cubic)
        h_circle_cubic<double>(mat->c12, mat->c44, mat->cd, mat->Q, T, hs);
    else
        h_circle_sym<double, double>(mat->C, mat->Q, T, hs);
    const double ir2 = 1.0 / r2;
    for (int i = 0; i < 54; ++i) {
        double acc = 0.0;
        for (int k = 0; k < 18; ++k) acc += Asym[i * 18 + k] * hs[k];
        out[i] = acc * ir2;
    }
}
