// Prints the host tables of paper_1712_07739_gb300/csrc/cube_sym.h for the CPU test
// (tests/test_host_cube_sym.py), which checks them against an independent construction.
//   cube_sym_dump tables         -> maps, representatives, per-offset (rep, map), per-map tables
//   cube_sym_dump invariant      -> reads 81 C_ijkl values on stdin, prints 1 or 0
#include <cstdio>
#include <cstring>

#include "../paper_1712_07739_gb300/csrc/cube_sym.h"

int main(int argc, char **argv) {
    if (argc > 1 && std::strcmp(argv[1], "invariant") == 0) {
        double C[81];
        for (double &c : C)
            if (std::scanf("%lf", &c) != 1) return 2;
        std::printf("%d\n", cube_sym::cube_invariant(C) ? 1 : 0);
        return 0;
    }
    for (int gi = 0; gi < 48; ++gi) {
        const cube_sym::CubeMap m = cube_sym::cube_map(gi);
        std::printf("map %d %d %d %d %d %d %d %d\n", gi, m.pi[0], m.pi[1], m.pi[2], m.s[0], m.s[1], m.s[2], m.det);
    }
    cube_sym::RepList reps{};
    int osym[343];
    unsigned char gmap[48 * 60];
    cube_sym::sym_tables(reps, osym, gmap);
    for (int r = 0; r < 16; ++r) std::printf("rep %d %d\n", r, reps.oi[r]);
    for (int oi = 0; oi < 343; ++oi) std::printf("off %d %d\n", oi, osym[oi]);
    for (int gi = 0; gi < 48; ++gi) {
        std::printf("gmap %d", gi);
        for (int t = 0; t < 60; ++t) std::printf(" %d", int(gmap[gi * 60 + t]));
        std::printf("\n");
    }
    return 0;
}
