// Host tables of the cube's symmetries for the symmetry-reduced M2L through transforms
// (Sec. 6: 16 of the 316 operators).  Plain host code with no CUDA dependency, so the CPU
// tests compile it on its own and check it against an independent construction.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace cube_sym {

// the 16 representatives' offset indices, oi = ((oz + 3) 7 + (oy + 3)) 7 + (ox + 3)
struct RepList {
    int oi[16];
};

// The cube's 48 signed axis permutations, map gi = 8 (permutation index) + sign bits
// (bit i: s_i = -1), permutations in lexicographic order; g_{i pi(i)} = s_i.
struct CubeMap {
    int pi[3], s[3], det;
};
inline CubeMap cube_map(int gi) {
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    static const int parity[6] = {1, -1, -1, 1, 1, -1};
    CubeMap m{};
    const int pk = gi / 8, sb = gi % 8;
    m.det = parity[pk];
    for (int i = 0; i < 3; ++i) {
        m.pi[i] = perms[pk][i];
        m.s[i] = (sb >> i) & 1 ? -1 : 1;
        m.det *= m.s[i];
    }
    return m;
}

inline int voigt_of(int a, int b) {
    if (a == b) return a;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 1 ? 3 : (hi == 2 ? 4 : 5);  // (1,2) yz, (0,2) xz, (0,1) xy
}

// C_ijkl (index ((i 3 + j) 3 + k) 3 + l) unchanged by all 48 maps?
inline bool cube_invariant(const double *C) {
    double mx = 0.0;
    for (int i = 0; i < 81; ++i) mx = std::max(mx, std::fabs(C[i]));
    for (int gi = 0; gi < 48; ++gi) {
        const CubeMap m = cube_map(gi);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        const double c = m.s[i] * m.s[j] * m.s[k] * m.s[l] *
                                         C[((m.pi[i] * 3 + m.pi[j]) * 3 + m.pi[k]) * 3 + m.pi[l]];
                        if (std::fabs(c - C[((i * 3 + j) * 3 + k) * 3 + l]) > 1e-12 * mx) return false;
                    }
    }
    return true;
}

// Representatives (r0 >= r1 >= r2 >= 0, r0 in {2, 3}) in a fixed order, each offset's
// representative and map (o = g rep), and per map its component and frequency-axis tables
inline void sym_tables(RepList &reps, int osym[343], unsigned char gmap[48 * 60]) {
    int rep_key[16], nr = 0;
    for (int r0 = 2; r0 <= 3; ++r0)
        for (int r1 = 0; r1 <= r0; ++r1)
            for (int r2 = 0; r2 <= r1; ++r2) {
                rep_key[nr] = (r0 * 4 + r1) * 4 + r2;
                reps.oi[nr++] = ((r2 + 3) * 7 + (r1 + 3)) * 7 + (r0 + 3);  // (x, y, z) = (r0, r1, r2)
            }
    for (int oi = 0; oi < 343; ++oi) {
        const int o[3] = {oi % 7 - 3, (oi / 7) % 7 - 3, oi / 49 - 3};
        int a[3] = {std::abs(o[0]), std::abs(o[1]), std::abs(o[2])};
        std::sort(a, a + 3);
        osym[oi] = -1;
        if (a[2] < 2) continue;
        const int r[3] = {a[2], a[1], a[0]}, key = (r[0] * 4 + r[1]) * 4 + r[2];
        const int ri = int(std::find(rep_key, rep_key + 16, key) - rep_key);
        for (int gi = 0; gi < 48 && osym[oi] < 0; ++gi) {
            const CubeMap m = cube_map(gi);
            bool ok = true;
            for (int i = 0; i < 3; ++i) ok = ok && o[i] == m.s[i] * r[m.pi[i]];
            if (ok) osym[oi] = ri | (gi << 8);
        }
    }
    static const int va[6] = {0, 1, 2, 1, 0, 0}, vb[6] = {0, 1, 2, 2, 2, 1};
    for (int gi = 0; gi < 48; ++gi) {
        const CubeMap m = cube_map(gi);
        unsigned char *gm = gmap + gi * 60;
        for (int ab = 0; ab < 6; ++ab)
            for (int w = 0; w < 3; ++w)
                for (int r = 0; r < 3; ++r) {
                    const int a = va[ab], b = vb[ab];
                    const int src = voigt_of(m.pi[a], m.pi[b]) * 9 + m.pi[w] * 3 + m.pi[r];
                    const int sg = m.det * m.s[a] * m.s[b] * m.s[w] * m.s[r];
                    gm[ab * 9 + w * 3 + r] = (unsigned char)(src | (sg < 0 ? 64 : 0));
                }
        // frequency axis j of the representative's frame: (g^T f)_j = s_i f_i with pi(i) = j
        for (int i = 0; i < 3; ++i) gm[54 + m.pi[i]] = (unsigned char)(i | (m.s[i] < 0 ? 4 : 0));
        for (int t = 57; t < 60; ++t) gm[t] = 0;
    }
}

}  // namespace cube_sym
