// Execution planning: turns a lowered gate queue into kernel passes.
#pragma once

#include "internal.h"

namespace qsim {

// Apply a lowered gate queue with the requested strategy. params_dev/n_params
// drive gates with param_index >= 0 (batched parameters), else nullptr/0.
qs_status run_gates(qs_state *s, std::vector<LGate> &gates, int mode, const qs_opts *opts,
                    const double *params_dev, int n_params);

// Trotter evolution (Sec. 2.6). With steps == 1 and s_fixed >= 0: one step at
// s = s_fixed. With s_fixed < 0: `steps` steps of the linear schedule over
// total time T, step k at s = (k + 1/2) dt / T, adjacent half diagonals merged.
qs_status run_trotter(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                      size_t n_h1, double s_fixed, double dt, double T, int steps);

// How the tiled planner chooses its passes (the autotuner times the
// variants). select 0: the pass that takes the most gates among the greedy
// choice of high bits and every window of consecutive high bits; 1: the greedy
// choice only; 2: the windows only (the greedy choice where no window takes a
// gate). max_gates > 0 caps the gates of a pass.
struct TileSchedule {
    int select = 0;
    int max_gates = 0;
};
TileSchedule tile_schedule();  // the calling thread's (default: {0, 0})
void set_tile_schedule(TileSchedule s);

// Tiled multi-gate passes (falls back to one pass per gate for gates a tile
// cannot express and for states smaller than a tile).
// force_bit >= 0 (adjoint sweep): that index bit is kept in every tile and
// every stage's register set (it is the top register bit); gradient ops write
// per-tile partials to gpart; batched-parameter gates use angle * param_sign.
qs_status run_tiled(qs_state *s, const std::vector<LGate> &gates, const double *params_dev, int n_params,
                    int force_bit = -1, double *gpart = nullptr, double param_sign = 1.0);

// The gate queue of a second-order Trotter evolution on the tiled path: per
// step k an Ising phase exp(-i taus[k] E) (the merged half steps; none where
// `ising` is false or the angle is 0), then RX(2 dt a_q(s_k)) on every qubit
// with a_q(s) = (1 - s) a0[q] + s a1[q]; a last Ising phase taus[steps]. It is
// written in the frame of S = diag(1, i) on every qubit: S X S^dag = Y, so
// RX(t) = S^dag RY(t) S, and S commutes with the diagonal Ising phases; the
// queue is S on every qubit, the steps with RY for RX, then S^dag on every
// qubit. The RY layers are real rotations with no diagonal factors, applied as
// three in-place shears: no diagonal block between the layers.
qs_status trotter_queue(int n, const std::vector<double> &a0, const std::vector<double> &a1,
                        const std::vector<double> &taus, const std::vector<double> &svals, double dt, bool ising,
                        std::vector<LGate> *G);

// Adiabatic evolution of a batch whose members have their own H1 (terms
// h1[off[b] .. off[b+1]) for member b).
qs_status run_adiabatic_batch(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                              const size_t *off, double dt, double T, int steps);

// Adiabatic evolution of instances of several widths, one handle per width
// (h0 terms of handle i: h0[h0_off[i] .. h0_off[i+1]); H1 of member j, counted
// over all handles in order: h1[h1_off[j] .. h1_off[j+1])), the handles on
// streams of their own run side by side; `chunk` steps are enqueued per handle
// in turn.
qs_status run_adiabatic_multi(qs_state *const *states, int n_states, const qs_pauli_term *h0,
                              const size_t *h0_off, const qs_pauli_term *h1, const size_t *h1_off, double dt,
                              double T, int steps, int chunk);

// Exact time evolution (evolve.cpp): `steps` steps of dt of H(t) = (1 - s) H0
// + s H1, s = t / T, with the solver QS_SOLVER_*; and the schedule gradient of
// the Trotterised evolution with schedule values svals[0 .. K).
qs_status run_evolve(qs_state *s, const qs_pauli_term *h0, size_t n0, const qs_pauli_term *h1, size_t n1, double T,
                     double dt, int steps, int solver);
qs_status run_schedule_gradient(qs_state *s, const qs_pauli_term *h0, size_t n0, const qs_pauli_term *h1, size_t n1,
                                const double *svals, int K, double dt, double *energy, double *dE_ds, double *dE_ddt);

// Free anything cached per state.
void plan_cache_release(qs_state *s);

}  // namespace qsim
