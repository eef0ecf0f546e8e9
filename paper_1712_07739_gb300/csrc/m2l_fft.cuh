// FP64 M2L through the Toeplitz structure of the operators (Sec. 4.1,
// Theorem 1): per offset the node-to-node map is a 3-D discrete convolution,
// applied as a product of transforms of size (2p)^3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct gbfmm_ctx;

struct FftPlan {
    bool ready = false;            // Khat holds the transformed operators of the current medium and p
    int p = 0;
    bool sym = false;              // Khat holds the 16 representatives of the cube's symmetry orbits
    double2 *Khat = nullptr;       // [343 offsets][54][NF]: offsets with max |o_i| >= 2 filled;
                                   // with sym [16 representatives][54][NF]
    int *d_osym = nullptr;         // sym: [343] representative | map << 8 of each offset
    unsigned char *d_gmap = nullptr;  // sym: [48][60] per map: 54 source components (bit 6: negate),
                                      // then per frequency axis its source axis and sign (bit 2)
    double2 *What = nullptr;       // [slots][9][NF]: transformed multipole values of one level
    int64_t what_cap = 0;          // slots
    int *slot = nullptr;           // [cells of one level]: slot of each occupied cell, else -1
    int *slot_cell = nullptr;      // [cells of one level]: cell of each slot
    int *count = nullptr;          // occupied cells of the level (device)
    int64_t cell_cap = 0;
};

// S at levels 2 .. L-1 from W (FP64), for every cell with targets (tocc > 0)
int m2l_fft_run(gbfmm_ctx *ctx, const int *occ, const int *tocc);
void m2l_fft_free(gbfmm_ctx *ctx);
