// Internal declarations of the qsim CUDA library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "qsim.h"

struct qs_state {
    int n = 0;              // qubits per batch member
    int batch = 1;          // number of members
    int ms = 0;             // member b starts at amplitude b << ms (ms = n for a
                            // contiguous batch; ms > n for internal strided views)
    qs_dtype dtype = QS_C64;
    void *data = nullptr;   // batch * 2^n amplitudes
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    // device scratch for reductions, owned by the handle
    double *scratch = nullptr;
    size_t scratch_doubles = 0;
    // pinned host buffer for read-outs
    double *host_pinned = nullptr;
    size_t host_pinned_doubles = 0;
    // device table of per-member gate matrices (batched parameters)
    void *gtab = nullptr;
    size_t gtab_bytes = 0;
    // per-member matrices of all batched-parameter gates of one tiled run
    void *ptab = nullptr;
    size_t ptab_bytes = 0;
    int ptab_dd = 0;  // the table holds double-float pairs (complex128 passes in double-float)
    // Ising coefficients of the Trotter diagonal (see tiled.h); stride 0 = shared
    double *itab = nullptr;
    size_t itab_bytes = 0;
    uint32_t ising_stride = 0;
    // per-pass tables of the Ising op's tile-independent parts (see tiled.h)
    double *ithr = nullptr;
    size_t ithr_bytes = 0;
    // density matrix of dm qubits (n = 2 dm: entry (r, c) at index r 2^dm + c);
    // 0 for a state vector
    int dm = 0;
    // host-memory state (partition.cpp): the amplitudes in pinned host memory
    // (data stays null), two device buffers of 2^pm amplitudes, chunks of 2^pl
    void *host = nullptr;
    int pm = 0;
    int pl = 0;
    void *pbuf[2] = {nullptr, nullptr};
};

namespace qsim {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();
qs_status cuda_status(cudaError_t e, const char *what);

#define QS_CUDA_TRY(expr)                                                  \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return ::qsim::cuda_status(_e, #expr);      \
    } while (0)

#define QS_TRY(expr)                                                       \
    do {                                                                   \
        qs_status _s = (expr);                                             \
        if (_s != QS_OK) return _s;                                        \
    } while (0)

inline uint64_t qbit(int n, int q) { return 1ull << (n - 1 - q); }

// ------------------------------------------------------------------ gates (host)
// A gate lowered to index-bit form: targets as bit positions, controls as a
// bit mask, matrix in double precision (row-major, local index MSB = target 0).
struct LGate {
    int k = 0;                 // number of targets
    int tbit[QS_MAX_TARGETS];  // bit position of target j (= n-1-qubit)
    uint64_t cmask = 0;        // control bits (index-bit mask)
    std::vector<cd> m;         // 2^k x 2^k
    bool diagonal = false;     // m is diagonal
    bool phase_only = false;   // diagonal with all entries 1 but the last
    bool is_swap = false;      // the SWAP permutation
    int param_index = -1;      // batched parameter column, or -1
    int kind = -1;             // QS_GATE_* of the source gate, or kKindGrad
    // tiled pass: if the gate is a real rotation (no diagonal factors), apply
    // it as three in-place shears, which need no diagonal block after it (set
    // where no other diagonal sits between a qubit's rotations: Trotter layers)
    bool paeth = false;
    // adjoint sweep only (kind == kKindGrad): generator (GEN_X/Y/Z/PROJ) and
    // the gradient slot the op accumulates into
    int grad_gen = -1;
    int grad_slot = -1;
};

// internal pseudo-kinds: an adjoint-sweep gradient op; an Ising phase
// exp(-i tau E(x)) (tau in m[0].real(), coefficients in the state's ising table)
constexpr int kKindGrad = 1000;
constexpr int kKindIsing = 1001;

// number of targets and parameters of a kind, or -1 if unknown
int kind_targets(int kind);
int kind_params(int kind);
// matrix of a named kind (not UNITARY) with angles p
std::vector<cd> kind_matrix(int kind, const double *p);
// validate one gate against n qubits and lower it (qubit -> bit form)
qs_status lower_gate(int n, const qs_gate &g, LGate *out);
// diagonal / phase_only flags of a lowered matrix
void set_matrix_flags(LGate *g);

// host-memory states (partition.cpp)
qs_status host_state_buffers(qs_state *s);
qs_status host_init(qs_state *s, bool plus, uint64_t x);
qs_status host_apply(qs_state *s, const std::vector<LGate> &G, int mode, const qs_opts *opts);
qs_status host_norm2(qs_state *s, double *out);
qs_status host_probabilities(qs_state *s, double *out);
qs_status host_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double *re, double *im);

// ------------------------------------------------------------------ kernels (host launchers)
qs_status k_init_basis(qs_state *s, uint64_t x);
qs_status k_init_plus(qs_state *s);
qs_status k_apply_unfused(qs_state *s, const LGate &g);
// this thread's complex128 passes in FP64 (true) or in double-float on the
// FP32 pipes (false, the default: one-gate passes of dense 1- and 2-qubit
// gates, and tiled passes without per-member matrices or gradients)
void set_c128_fp64(bool on);
bool c128_fp64();
qs_status k_probabilities(qs_state *s, double *out_dev);
// reductions: results land in the state's scratch; *out_dev points at them
qs_status k_norm2(qs_state *s, double **out_dev);        // batch doubles
qs_status k_expectation(qs_state *s, const qs_pauli_term *terms, size_t count,
                        double **out_dev);               // 2 * batch doubles (re, im)
qs_status ensure_scratch(qs_state *s, size_t doubles);
qs_status ensure_gtab(qs_state *s, size_t bytes);
// measurements (kernels_measure.cu): marginal probabilities of the qubits at
// index bits bitpos[0..m) per member into out_dev (batch * 2^m doubles);
// samples of member `member` for the uniforms u_dev into out_dev
constexpr int kMarginalMaxQubits = QS_MARGINAL_MAX_QUBITS;
qs_status k_marginal(qs_state *s, const int *bitpos, int m, double *out_dev);
qs_status k_sample(qs_state *s, int member, const double *u_dev, uint64_t shots, uint64_t *out_dev);
// Per-member matrices of batched-parameter gates, 4 entries per slot: RX/RY the
// row-major 2x2, RZ its diagonal (d0, d1), U1/CU1 the phase of the all-ones
// block in entry 0. slot j uses column pidx[j] of the parameter
// table, gate kind kind[j], angle sign * theta. Fills s->ptab as
// [member][slot][4] in the state's precision; *stride = entries per member.
// (dd_table: a complex128 table as double-float pairs, for double-float passes;
// s->ptab_dd records the format)
qs_status k_param_table(qs_state *s, const std::vector<int> &pidx, const std::vector<int> &kind,
                        const double *params_dev, int n_params, double sign, uint32_t *stride,
                        bool dd_table = false);
// batched-parameter rotation (RX RY RZ U1 CU1) of one gate
qs_status k_apply_param_gate(qs_state *s, const LGate &g, const double *params_dev, int n_params,
                             double sign = 1.0);
qs_status ensure_host_pinned(qs_state *s, size_t doubles);

// density matrices (kernels_density.cu): rho = |psi><psi| from psi_dev (batch x
// 2^dm amplitudes); the diagonal into out_dev (batch x 2^dm doubles); traces and
// Tr(rho H) into the scratch (batch doubles; batch (re, im) pairs)
qs_status k_dm_init_pure(qs_state *s, const void *psi_dev);
qs_status k_dm_probabilities(qs_state *s, double *out_dev);
qs_status k_dm_trace(qs_state *s, double **out_dev);
qs_status k_dm_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double **out_dev);

// Trotter factors
qs_status k_diagonal_evolution(qs_state *s, const std::vector<double> &coeff,
                               const std::vector<uint64_t> &zbits, double tau);

}  // namespace qsim
