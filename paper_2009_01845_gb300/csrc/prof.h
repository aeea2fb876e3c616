// Launch accounting: when enabled, every kernel launch of the library is
// bracketed by CUDA events on its stream, per kernel class.
#pragma once

#include <cuda_runtime.h>

namespace qsim {

enum KClass {
    KC_INIT = 0,
    KC_DENSE,
    KC_PHASE,
    KC_DIAG,
    KC_SWAP,
    KC_PARAM,
    KC_TILED,
    KC_FUSED_TC,
    KC_REDUCE,
    KC_TROTTER_DIAG,
    KC_ADJOINT,
    KC_HPSI,     // lambda = H psi of the adjoint (Pauli-sum application)
    KC_EVOLVE,   // exact time-evolution solvers: H psi and linear combinations
    KC_HOSTCOPY, // host-memory states: chunk copies between host and device
    KC_COUNT
};

bool prof_enabled();
// suspend launch accounting on this thread (while a CUDA graph is captured)
void prof_suspend(bool on);
// record the start/end of one launch of class c on stream st
void prof_begin(cudaStream_t st, int c);
void prof_end(cudaStream_t st, int c);
// add the algorithmic bytes (HBM reads + writes the operation needs) and
// flops of the launches of class c
void prof_add_work(int c, double bytes, double flops);

struct ProfScope {
    cudaStream_t st;
    int c;
    bool on;
    ProfScope(cudaStream_t s, int cls, double bytes = 0.0, double flops = 0.0)
        : st(s), c(cls), on(prof_enabled()) {
        if (on) {
            prof_begin(st, c);
            prof_add_work(c, bytes, flops);
        }
    }
    ~ProfScope() {
        if (on) prof_end(st, c);
    }
};

}  // namespace qsim
