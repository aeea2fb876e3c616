// Adjoint gradient: shared declarations of its kernels and driver.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace qsim {

// A (possibly strided) batch of n-qubit states: member b starts at amplitude b << ms.
struct StateView {
    void *data;
    int n;
    int ms;
    int batch;
    qs_dtype dtype;
};

constexpr int kPAMaxTerms = 384;
constexpr int kPAMaxGroups = 64;

template <typename R> struct PauliApplyP {
    R cre[kPAMaxTerms];
    R cim[kPAMaxTerms];
    uint64_t zb[kPAMaxTerms];
    uint64_t gx[kPAMaxGroups];
    int gbeg[kPAMaxGroups + 1];
    // groups whose terms have no Z bits: their coefficient sum, a constant
    R gcre[kPAMaxGroups];
    R gcim[kPAMaxGroups];
    uint8_t gconst[kPAMaxGroups];
    // groups 0 .. run0 - 1 are constant groups with one coefficient (run0 = 0:
    // none); with no earlier partial sum (accumulate = 0) the tile kernel adds
    // their partner amplitudes and multiplies by the coefficient once
    int run0;
    // the group of Z-only terms (X mask 0), or -1; for the shared-memory tile
    // kernel its terms sorted by the bits 8 .. 8 + log2(tile / 256) - 1 their Z
    // masks include (the bits that tell a thread's outputs apart): dord[dmb[m]
    // .. dmb[m+1]) are the ones with mask m
    int gdiag;
    uint16_t dord[kPAMaxTerms];
    int dmb[17];
    // The Z-only group's terms of weight 0, 1 and 2 (an Ising energy) are not
    // in dord: the tile kernel evaluates E(y) = qc0 + sum_i qh[i] z_i +
    // sum_{i<j} qJ[i][j] z_i z_j (z_i = 1 - 2 y_i, index bits, qJ symmetric
    // with a zero diagonal) by its split over the outside bits (per tile), the
    // thread bits (per thread) and the chunk bits (per output); qecc[c] is the
    // chunk bits' pair energy for chunk value c. quad = 0: no such term.
    int quad;
    R qc0;
    R qh[32];
    R qJ[32][32];
    R qecc[16];
    int ng;
    int n;
    int ms;
    int accumulate;
    uint64_t total;
};

static_assert(sizeof(PauliApplyP<double>) <= 32764, "Pauli-sum kernel parameters exceed the parameter space");

constexpr int kGRMaxRows = 1024;   // parameters per reduction launch
constexpr int kGRMaxSlots = 2048;  // gradient slots per reduction launch

struct GradReduceP {
    int beg[kGRMaxRows + 1];   // slot list of parameter row i: slot[beg[i] .. beg[i+1])
    int slot[kGRMaxSlots];
    float coef[kGRMaxSlots];   // 1 for rotations (Im<l|P|phi>), -2 for phase gates
    uint64_t total_tiles;
    uint64_t tiles_per_member;
    int n_params;
    int param0;                // first parameter row of this launch
};

qs_status k_pauli_apply(const StateView &src, const StateView &dst, const qs_pauli_term *terms, size_t count,
                        cudaStream_t st);
qs_status k_dot(const StateView &a, const StateView &b, double *scratch, size_t scratch_doubles, double *out,
                cudaStream_t st);
// gradient op on a small (phi, lambda) state: out[b] for every member b
qs_status k_grad_small(qs_state *w, const LGate &g, double *out);
qs_status k_grad_reduce(const double *part, const GradReduceP &p, int n_param_rows, int batch, double *grad,
                        cudaStream_t st);

}  // namespace qsim
