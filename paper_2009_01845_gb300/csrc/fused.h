// Fused 5-qubit tensor-core blocks: kernel parameters and the fusion planner.
#pragma once

#include <vector>

#include "device.cuh"
#include "internal.h"

namespace qsim {

struct FusedP {
    float2 u[1024];          // the block's 32 x 32 complex matrix, row-major
    uint64_t chunk_mask;     // the 11 index bits a chunk spans (block bits + 6 column bits)
    InsertBits cins;         // sorted positions of the chunk bits (chunk number -> index)
    int chunk_shift;         // log2(chunks per member) = n - 11
    int ms;                  // member shift
    uint64_t total_chunks;
    // element i = t + 256 h of a chunk (t: thread, h = 0..7) sits at address
    // offset dep(t) | dhi[h], row rlo(t) | rhi[h], column clo(t) | chi[h]: the
    // chunk bits split between the block (row) and the columns
    uint64_t dhi[8];
    uint8_t rhi[8], chi[8];
    uint8_t lmap[256];       // row of thread t's bits (h = 0)
    uint8_t cmap[256];       // column of thread t's bits (h = 0)
};

// Apply a 32 x 32 complex matrix U (row-major, local index MSB = bits[0]) to the
// index bits bits[0..4] of every member (complex64 states, n >= 11).
qs_status k_fused5(qs_state *s, const std::vector<cd> &U, const int *bits);

// Fused execution of a gate queue: gates are grouped into blocks of at most
// `width` (<= 5) qubits (a gate joins the latest block holding all of its
// qubits' latest gates, when the union stays within the width), each block's
// matrix is the product of its gates' matrices, and every block is one
// tensor-core pass. Gates on more qubits, and everything on complex128 or
// small states, fall back to the tiled planner.
qs_status run_fused(qs_state *s, const std::vector<LGate> &gates, int width, const double *params, int n_params);

}  // namespace qsim
