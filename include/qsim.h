/*
 * qsim.h -- C-ABI of the GB300 (sm_103a) state-vector simulator core.
 *
 * The operations follow the Qibo paper (arXiv:2009.01845):
 *   - state allocation and initialisation: Sec. 2.3 (dense 2^n complex state,
 *     updated in place, 2^n complex numbers of memory);
 *   - gate application: Eq. (1) of Sec. 2.3, controls as in Sec. 2.4
 *     ("Controlled gates"), fused blocks as in Sec. 2.4 ("Gate fusion");
 *   - probabilities, outcome probabilities of qubit groups and measurement
 *     samples: Sec. 2.4 ("Measurements"), Sec. 3.3;
 *   - Pauli-sum expectation values: Sec. 2.4 ("Callbacks", Energy);
 *   - Trotter steps of H(s) = (1-s) H0 + s H1: Sec. 2.6, Eqs. (4)-(6);
 *   - adjoint gradients and batched execution have no counterpart in the
 *     paper (which differentiates through its TensorFlow backends only,
 *     Sec. 2.3); their definitions are stated at each declaration.
 *
 * Conventions used by every call:
 *   - qubit q is bit (n-1-q) of a basis index: qubit 0 is the most
 *     significant bit (Sec. 2.5, global qubits split the state in contiguous
 *     halves);
 *   - amplitudes are interleaved (re, im): complex64 = 2 x float,
 *     complex128 = 2 x double; a batch of B states of n qubits is B contiguous
 *     blocks of 2^n amplitudes;
 *   - a k-target gate matrix is row-major 2^k x 2^k with local index
 *     sum_j bit(target_j) 2^(k-1-j) (the first target is the local MSB);
 *   - rotation conventions: R_P(t) = exp(-i t P/2); U1(l) = diag(1, e^{il});
 *     CU1(t) = diag(1,1,1,e^{it}); U3 is OpenQASM 2's
 *     [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]];
 *     U2(p,l) = U3(pi/2,p,l);
 *   - Pauli masks: bit q of x_mask/z_mask refers to qubit q; X = x only,
 *     Z = z only, Y = both (Y = i X Z).
 *
 * Errors: every call returns a qs_status and never throws or aborts. On a
 * non-zero status nothing was launched unless the status is QS_ERR_CUDA, in
 * which case the device state is unspecified. qs_last_error() returns a
 * thread-local message for the last failure on the calling thread.
 *
 * Streams: every call is ordered on the state's stream (set at create/wrap;
 * NULL = the legacy default stream). Calls that return values to host memory
 * synchronise that stream before returning; all others are asynchronous.
 * Host pointers need not be pinned.
 *
 * Threads: a qs_state may be used by one host thread at a time.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qs_status;
#define QS_OK 0
#define QS_ERR_ARG 1          /* invalid argument: qubit range, arity, null pointer, size */
#define QS_ERR_OOM 2          /* device allocation failed */
#define QS_ERR_CUDA 3         /* a CUDA runtime call or kernel launch failed */
#define QS_ERR_UNSUPPORTED 4  /* valid request outside what the library implements */
#define QS_ERR_TIMEOUT 5      /* a bounded device-side wait ran out */

typedef int32_t qs_dtype;
#define QS_C64 0              /* complex64 state: float re, float im */
#define QS_C128 1             /* complex128 state: double re, double im */

/* Gate kinds. Arity (targets, parameters) in parentheses. */
#define QS_GATE_H 0           /* (1,0) Hadamard */
#define QS_GATE_X 1           /* (1,0) */
#define QS_GATE_Y 2           /* (1,0) */
#define QS_GATE_Z 3           /* (1,0) */
#define QS_GATE_S 4           /* (1,0) diag(1, i) */
#define QS_GATE_SDG 5         /* (1,0) diag(1, -i) */
#define QS_GATE_T 6           /* (1,0) diag(1, e^{i pi/4}) */
#define QS_GATE_TDG 7         /* (1,0) diag(1, e^{-i pi/4}) */
#define QS_GATE_RX 8          /* (1,1) */
#define QS_GATE_RY 9          /* (1,1) */
#define QS_GATE_RZ 10         /* (1,1) */
#define QS_GATE_U1 11         /* (1,1) */
#define QS_GATE_U2 12         /* (1,2) */
#define QS_GATE_U3 13         /* (1,3) */
#define QS_GATE_CZ 14         /* (2,0) diag(1,1,1,-1) */
#define QS_GATE_CU1 15        /* (2,1) diag(1,1,1,e^{it}); CZPow(t) = CU1(pi t) */
#define QS_GATE_SWAP 16       /* (2,0) */
#define QS_GATE_UNITARY 17    /* (k,0), 1 <= k <= 5, matrix given */
#define QS_GATE_KIND_COUNT 18

#define QS_MAX_TARGETS 5
#define QS_MAX_QUBITS 40
/* Largest batch of one handle: the per-member reductions put the member on the
   second grid dimension, whose extent CUDA limits to 65535. */
#define QS_MAX_BATCH 65535

/* One gate of a queue (Eq. (1); a circuit is an ordered queue, Sec. 2.3). */
typedef struct qs_gate {
    int32_t kind;                     /* QS_GATE_* */
    int32_t n_targets;                /* must equal the kind's arity; 1..5 for UNITARY */
    int32_t targets[QS_MAX_TARGETS];  /* qubit indices, distinct, in [0, n) */
    int32_t param_index;              /* batched calls: column of the parameter
                                         table driving params[0], or -1 */
    uint64_t control_mask;            /* bit q set: qubit q is a control (all must be 1) */
    double params[3];                 /* angles, used by RX RY RZ U1 U2 U3 CU1 */
    const double *matrix;             /* UNITARY only: host pointer to 2^k x 2^k
                                         complex128 (interleaved, row-major); read
                                         during the call only */
} qs_gate;

/* One term c * P of a Pauli-sum Hamiltonian. */
typedef struct qs_pauli_term {
    double coeff;
    uint64_t x_mask;
    uint64_t z_mask;
} qs_pauli_term;

/* Execution strategy for qs_apply_gates. */
#define QS_MODE_AUTO 0        /* planner's choice (tiled passes) */
#define QS_MODE_UNFUSED 1     /* one kernel pass per gate (the plain simulator) */
#define QS_MODE_TILED 2       /* shared-memory/register tiles, many gates per pass */
#define QS_MODE_FUSED_TC 3    /* gates fused into <=5-qubit dense blocks on tensor cores */

typedef struct qs_opts {
    int32_t mode;             /* QS_MODE_* */
    int32_t tile_qubits;      /* tiled mode: tile width k; 0 or the kernels' own
                                 width (13 complex64, 12 complex128), else
                                 QS_ERR_UNSUPPORTED */
    int32_t fuse_qubits;      /* fused mode: block width (0 = 5) */
    int32_t flags;            /* QS_OPT_* bits, or 0 */
} qs_opts;

/* complex128 arithmetic. By default complex128 gates run in double-float
   arithmetic on the FP32 pipes: each double is split into two floats (47
   significant bits), products are exact FMA products and sums exact two-sums,
   and the result is joined back into a double; the error per gate is a few
   2^-47 of the amplitudes' magnitude (~1e-14). This covers one-gate passes of
   dense 1- and 2-qubit gates and tiled passes, per-member angles and the
   adjoint sweep's gradient ops included (GB300's FP64 rate would bind them at
   a third of the HBM bandwidth or less). QS_OPT_C128_FP64 in qs_opts.flags
   runs every complex128 gate of the call in FP64 instead (the calls that take
   qs_opts: gate application, batched application, channels and plans; the
   Trotter, adiabatic, evolution and gradient calls always use the default).
   Either way, one-gate passes of diagonal gates and of dense gates on 3 to 5
   qubits are FP64 (swaps move amplitudes exactly), and read-outs and gradient
   partials accumulate in FP64. The double-float range is that of a float
   pair: amplitudes of magnitude 2^128 or more, and non-finite ones, are not
   represented (below 2^-126 they become 0); use the FP64 flag for such
   states. */
#define QS_OPT_C128_FP64 1

typedef struct qs_state qs_state;

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *qs_last_error(void);
/* Library version string. */
const char *qs_version(void);

/* ---------------------------------------------------------------- states */
/* Allocate a batch of `batch` states of n qubits (batch * 2^n amplitudes) on the
   current CUDA device; the library owns and frees the memory. Contents are
   undefined until initialised. 1 <= batch <= QS_MAX_BATCH and
   batch * 2^n <= 2^46, else QS_ERR_ARG; QS_ERR_OOM if the allocation fails. */
qs_status qs_state_create(int n, int batch, qs_dtype dtype, void *cuda_stream, qs_state **out);
/* Wrap caller-owned device memory of batch * 2^n amplitudes (16-byte aligned);
   the handle never frees it and it must outlive the handle. */
qs_status qs_state_wrap(int n, int batch, qs_dtype dtype, void *dev_ptr, void *cuda_stream,
                        qs_state **out);
/* Release the handle (and the memory if the library allocated it). NULL is a no-op. */
qs_status qs_state_destroy(qs_state *s);
/* Device pointer of the amplitudes. */
qs_status qs_state_data(const qs_state *s, void **dev_ptr);
/* Change the stream later calls are ordered on. */
qs_status qs_state_set_stream(qs_state *s, void *cuda_stream);

/* |x> in every batch member (x < 2^n). */
qs_status qs_state_init_basis(qs_state *s, uint64_t x);
/* |+>^n in every batch member: every amplitude 2^{-n/2}. */
qs_status qs_state_init_plus(qs_state *s);
/* Copy batch * 2^n amplitudes in (from host when on_device = 0, else device). */
qs_status qs_state_set(qs_state *s, const void *src, int on_device);
/* Copy batch * 2^n amplitudes out (to host when on_device = 0, else device). */
qs_status qs_state_get(const qs_state *s, void *dst, int on_device);

/* ---------------------------------------------------------------- gates */
/* Apply a gate queue in order to every batch member (Eq. (1), Sec. 2.3-2.4).
   opts may be NULL (= QS_MODE_AUTO). Qubits are validated: in range, targets
   distinct, controls disjoint from targets, arity matching the kind, else
   QS_ERR_ARG and nothing is applied. */
qs_status qs_apply_gates(qs_state *s, const qs_gate *gates, size_t count, const qs_opts *opts);

/* Batched parameters: like qs_apply_gates, but a gate whose param_index p >= 0
   takes its angle params[0] from params[b * n_params + p] for batch member b.
   `params` is a device pointer to batch * n_params doubles (row-major), read
   in stream order. Supported for RX RY RZ U1 CU1 gates. */
qs_status qs_apply_gates_batched(qs_state *s, const qs_gate *gates, size_t count,
                                 const double *params_dev, int n_params, const qs_opts *opts);

/* ---------------------------------------------------------------- plans (CUDA graphs) */
/* A gate queue prepared for repeated execution on one state (no counterpart in
   the paper, which dispatches every gate on every execution). The gates are
   validated and lowered once; the strategy is opts->mode, or, with opts NULL
   or QS_MODE_AUTO and autotune = 1, the fastest of the tiled passes, fused
   tensor-core blocks (width 5 and 4; complex64, n >= 11) and the one-gate-
   per-pass kernels, timed once on a scratch copy of the state (skipped, with
   the tiled passes chosen, when no copy fits) and remembered per circuit
   shape for the process. The tuner first times the tiled planner's pass
   schedules (qs_plan_schedule) and uses the fastest for the tiled passes.
   The kernel sequence is captured in a CUDA graph.
   params_dev/n_params as in qs_apply_gates_batched (the pointer is captured:
   execute reads the table's current contents). */
typedef struct qs_plan qs_plan;
qs_status qs_plan_create(qs_state *s, const qs_gate *gates, size_t count, const double *params_dev, int n_params,
                         const qs_opts *opts, int autotune, qs_plan **out);
/* Replay the captured graph on the state's stream (asynchronous). */
qs_status qs_plan_execute(qs_plan *p);
/* Chosen mode and fusion width, the autotuner's best time in ms (-1 if not
   tuned) and the number of graph nodes; NULL outputs are skipped. */
qs_status qs_plan_info(const qs_plan *p, int *mode, int *fuse_qubits, double *tuned_ms, size_t *graph_nodes);
/* The tiled planner's pass schedule in the plan: select 0 = per pass, the
   most gates among the greedy choice of tile bits and every window of
   consecutive bits (the default); 1 = the greedy choice only; 2 = the windows
   only; max_gates > 0 caps the gates of a pass (0: no cap). The autotuner
   chooses among {0, 0}, {1, 0}, {2, 0} and {0, 32}; untuned plans use {0, 0}. */
qs_status qs_plan_schedule(const qs_plan *p, int *select, int *max_gates);
/* Release the plan (the state is not touched). NULL is a no-op. */
qs_status qs_plan_destroy(qs_plan *p);

/* ---------------------------------------------------------------- read-out */
/* |psi_x|^2 for every batch member, FP64, index = b * 2^n + x (qubit 0 = MSB of x).
   out: host (on_device = 0) or device pointer to batch * 2^n doubles. */
qs_status qs_probabilities(qs_state *s, double *out, int on_device);
/* sum_x |psi_x|^2 per batch member (FP64 accumulation); out: host, batch doubles. */
qs_status qs_norm2(qs_state *s, double *out);

/* Outcome probabilities of a group of qubits, traced over the others (Sec. 2.4,
   Measurements: the qubits of one register are measured together and the
   probability is summed over the unmeasured ones), per batch member:
   out[b * 2^m + y] = sum of |psi_b[x]|^2 over the x whose qubits[j] equals bit
   (m-1-j) of y (qubits[0] is the most significant bit of y, as qubit 0 is of
   the basis index). FP64 accumulation over per-block partial sums in a fixed
   order (the order inside a block is not fixed: results may differ between
   runs in the last bits). 1 <= m <= QS_MARGINAL_MAX_QUBITS, qubits distinct and
   in [0, n), else QS_ERR_ARG. out: host (on_device = 0; the call synchronises)
   or device pointer to batch * 2^m doubles. */
#define QS_MARGINAL_MAX_QUBITS 12
qs_status qs_marginal_probabilities(qs_state *s, const int *qubits, int m, double *out, int on_device);

/* Samples of the measurement of every qubit of batch member `member` (Sec. 2.4,
   "Measurements": sampling the final state vector; Sec. 3.3): for each uniform
   u in [0, 1), the smallest basis index x with cdf(x) > u * cdf(2^n - 1), where
   cdf(x) = sum_{x' <= x} |psi[x']|^2 (prefix sums in FP64 over blocks of 4096
   amplitudes). The caller draws the uniforms, so equal uniforms give equal
   samples (away from ties at a block boundary, where the prefix sum's
   rounding decides). uniforms and out: `shots` values each, both in host
   memory (on_device = 0; the call synchronises) or both in device memory.
   member outside [0, batch), a NULL pointer with shots > 0, or (host
   uniforms) a uniform that is not in [0, 1): QS_ERR_ARG. Device uniforms are
   not checked: one below 0 is taken as 0 and one of 1 or above, or NaN, as 1,
   so every sample is an outcome of nonzero probability (for a nonzero state). */
qs_status qs_sample(qs_state *s, int member, const double *uniforms, size_t shots, uint64_t *out,
                    int on_device);
/* <psi|H|psi> per batch member for H = sum_t coeff_t P_t (FP64 accumulation).
   out_re/out_im: host arrays of batch doubles (out_im may be NULL). */
qs_status qs_expectation(qs_state *s, const qs_pauli_term *terms, size_t count,
                         double *out_re, double *out_im);

/* Allocation-free variant of qs_expectation, for callers that cannot allocate
   device memory: code running while a CUDA graph is being captured, an
   allocator callback or an out-of-memory handler, a host that hands out only
   memory it owns. The paper has no counterpart; it is a deployment aid.
   psi_dev: device pointer to batch * 2^n amplitudes of `dtype` (read only);
   out_dev: device pointer to 2 * batch doubles, written as (re, im) per member
   in stream order on `cuda_stream` (NULL = legacy default stream). The call
   needs no handle and calls no cudaMalloc/cudaFree or other allocator: its
   partial sums live in one fixed device array of QS_NOALLOC_MAX_PARTIALS
   (65536) double2 entries (1 MiB) that every GPU loading this library holds
   until the process exits; batch must be <= QS_MAX_BATCH (65535, the grid
   limit every batched read-out shares; larger: QS_ERR_ARG). The first call on a device looks up that array's
   device address (a runtime query, not an allocation); make that first call
   before any stream capture. Every call shares the array and leaves its
   partial sums in it (each call overwrites the slots it uses before summing
   into them), so calls whose kernels overlap on the GPU -- e.g. on two
   streams without ordering -- race and give wrong results. Asynchronous:
   read out_dev after synchronising the stream. */
#define QS_NOALLOC_MAX_PARTIALS 65536
qs_status qs_expectation_noalloc(const void *psi_dev, int n, int batch, qs_dtype dtype,
                                 const qs_pauli_term *terms, size_t count, double *out_dev,
                                 void *cuda_stream);

/* ---------------------------------------------------------------- adjoint gradient */
/* Energies E_b(theta) = Re <psi_b|H|psi_b>, psi_b = U_N(theta_b) .. U_1(theta_b) psi0,
   and their gradients dE_b/dtheta for a batch of parameter sets, by the adjoint
   method: one forward pass, lambda = H psi, then one reverse sweep that undoes
   each gate on (psi, lambda) with its inverse and reads the gradient of every
   parametrised gate from <lambda|dU|psi>. The paper has no adjoint method (it
   differentiates through its TensorFlow backends only, Sec. 2.3); the circuit
   and H follow Sec. 2.3-2.4 and the variational ansatz of Sec. 3.2.
   work: a handle of batch members of n + 1 qubits (batch * 2^(n+1) amplitudes)
     for an n-qubit circuit; member b holds psi_b in its first 2^n amplitudes
     and lambda_b in the next 2^n. Gate qubits refer to the n-qubit circuit.
   gates: as in qs_apply_gates_batched; a gate with param_index p >= 0 (RX RY RZ
     U1 CU1) takes its angle from params_dev[b * n_params + p] and receives a
     gradient; other gates are fixed.
   init_zero: 1 = psi0 = |0...0>, 0 = psi0 is what the first half holds.
   energy_dev: batch doubles (device); grad_dev: batch * n_params doubles
     (device, row-major), parameters used by no gate get 0; tied parameters
     (several gates, one column) get the sum.
   mode: QS_GRAD_FULL (forward, energy, sweep), QS_GRAD_FORWARD (forward and
     energy only; psi and lambda stay in `work`), QS_GRAD_SWEEP (the sweep only,
     continuing a QS_GRAD_FORWARD call on the same work buffer; needs
     ckpt_every = 0).
   ckpt_every > 0 (QS_GRAD_FULL): psi is checkpointed every ckpt_every gates in
     the forward pass and restored at those boundaries of the sweep, bounding
     the drift of uncomputing psi by inverse gates (extra memory: one psi copy
     per checkpoint); 0 = pure uncompute.
   Gradients are accumulated per tile and reduced in FP64 in a fixed order. */
#define QS_GRAD_FULL 0
#define QS_GRAD_FORWARD 1
#define QS_GRAD_SWEEP 2
qs_status qs_energy_gradient(qs_state *work, const qs_gate *gates, size_t count, const double *params_dev,
                             int n_params, const qs_pauli_term *terms, size_t n_terms, int init_zero,
                             double *energy_dev, double *grad_dev, int ckpt_every, int mode);

/* ---------------------------------------------------------------- Trotter (Sec. 2.6) */
/* One second-order Trotter step of H(s) = (1-s) H0 + s H1 on every batch member:
     psi <- exp(-i dt/2 D(s)) exp(-i dt X(s)) exp(-i dt/2 D(s)) psi
   where D(s) collects the Z-string terms (x_mask = 0) and X(s) the
   single-qubit X terms (z_mask = 0, one x bit) of H(s). Phase angles are
   evaluated in FP64. Any other term: QS_ERR_UNSUPPORTED. */
qs_status qs_trotter_step(qs_state *s, const qs_pauli_term *h0, size_t n_h0,
                          const qs_pauli_term *h1, size_t n_h1, double s_val, double dt);
/* Adiabatic evolution with the linear schedule s = t/T (Sec. 2.6): K = round(T/dt)
   second-order steps, step k taking s = (k + 1/2) dt / T; `steps` >= 0 stops after
   that many steps (-1 = all K). Adjacent half-step diagonals of consecutive steps
   are merged (they commute), which changes only rounding. */
qs_status qs_adiabatic_evolve(qs_state *s, const qs_pauli_term *h0, size_t n_h0,
                              const qs_pauli_term *h1, size_t n_h1, double T, double dt,
                              int steps);

/* ---------------------------------------------------------------- launch accounting */
/* Tracing aid (no counterpart in the paper). While enabled, every kernel launch
   of the library is bracketed by CUDA events on the launching stream, grouped
   by kernel class (dense, phase, diag, swap, param, tiled, fused_tc, reduce,
   trotter_diag, adjoint, hpsi = the adjoint's lambda = H psi, evolve = the exact
   time-evolution solvers, host_copy = chunk copies of host-memory states,
   init).
   Process-wide. */
qs_status qs_profile_enable(int on);
/* Wait for the recorded launches, write per-class total milliseconds, launch
   counts, algorithmic bytes (the HBM reads + writes each operation needs) and
   algorithmic flops into arrays of n_classes entries, and reset the record. */
qs_status qs_profile_collect(double *total_ms, long long *launches, double *bytes, double *flops,
                             int n_classes);
/* Name of kernel class c ("" if out of range) and the number of classes. */
const char *qs_profile_class_name(int c);
int qs_profile_class_count(void);

/* Adiabatic evolution of instances of different widths in one call (Sec. 2.6,
   Eq. (4)): handle i holds states[i]->batch instances of its own width, all
   handles of one dtype on one device, none sharing memory. Handle i's members
   share H0 = the h0_counts[i] terms of h0 that follow handle i-1's; member j,
   counted over all handles in order, has its own H1 = the h1_counts[j] terms
   of h1 that follow member j-1's. Schedule, splitting, step count and the
   restrictions on the terms are those of qs_adiabatic_evolve_batch, per
   handle. The handles evolve side by side on streams of their own, forked
   from states[0]'s stream (after each handle's own earlier work) and joined
   back into states[0]'s stream and each handle's own; steps are enqueued in
   chunks of 10 per handle in turn, so every width has work on the GPU from
   the start. Chunks close and reopen their half-step diagonals (the GPU merges
   them only inside a chunk), which changes only rounding. Asynchronous. */
qs_status qs_adiabatic_run_batch(qs_state *const *states, int n_states, const qs_pauli_term *h0,
                                 const size_t *h0_counts, const qs_pauli_term *h1, const size_t *h1_counts,
                                 double T, double dt, int steps);

/* ---------------------------------------------------------------- exact evolution (Sec. 2.6) */
/* Time evolution i d/dt psi = H(t) psi, H(t) = (1 - s) H0 + s H1 with s = t/T
   (any Pauli terms; H0 = H1 gives a constant H), by the solvers the paper
   names besides Trotter: QS_SOLVER_EXP applies exp(-i dt H(s_mid)) per step,
   s_mid at the step's midpoint, as the Taylor series of the exponential on the
   state (the step cut into pieces tau with sum|c| tau <= 1, each summed to
   the order whose remainder bound falls below the precision's unit
   roundoff); QS_SOLVER_RK4 the classical fourth-order Runge-Kutta step;
   QS_SOLVER_RK45 the fifth-order solution of the Dormand-Prince 5(4) pair with
   the fixed step dt. Each step applies H to whole states (no matrix is
   built), so any n fits; the call allocates 2 (exp), 3 (rk4) or 7 (rk45)
   scratch states with the stream-ordered allocator. K = round(T/dt) steps,
   or `steps` >= 0 of them; every batch member. Asynchronous. */
#define QS_SOLVER_EXP 0
#define QS_SOLVER_RK4 1
#define QS_SOLVER_RK45 2
qs_status qs_evolve(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1, size_t n_h1,
                    double T, double dt, int steps, int solver);

/* Schedule gradient of the Trotterised adiabatic evolution (Sec. 4: the
   schedule s(t) and the total time are optimised for the final energy). From
   the handle's state psi_0 (per member) the call applies K second-order
   Trotter steps of H(s_k) = (1 - s_k) H0 + s_k H1, step k with svals[k] and
   the step dt (the splitting of qs_trotter_step: H0, H1 must have Z-string and
   single-qubit X terms only, else QS_ERR_UNSUPPORTED), leaves psi_K in the
   handle, and returns E = Re <psi_K|H1|psi_K> (energy: batch doubles, host,
   may be NULL) with its derivatives by one adjoint sweep: dE_ds[b K + k] =
   dE/ds_k and dE_ddt[b] = dE/d(dt) for dt shared by all steps (host arrays).
   A schedule s(t; theta) and total time T = K dt follow by the chain rule
   (dE/dtheta = sum_k dE/ds_k ds_k/dtheta). The sweep undoes each step's
   factors on psi and lambda = H1 psi and reads <lambda|G|psi> for the
   generators G (the diagonal and X parts of H0 and H1) the factors'
   derivatives insert. Scratch: 3 states and K small buffers from the
   stream-ordered allocator. Synchronises. */
qs_status qs_schedule_gradient(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                               size_t n_h1, const double *svals, int K, double dt, double *energy, double *dE_ds,
                               double *dE_ddt);

/* ---------------------------------------------------------------- host-memory states (Sec. 2.5) */
/* A state of n qubits (one member) whose 2^n amplitudes live in pinned host
   memory, for states larger than the GPU's memory (Sec. 2.5: one device
   reused for the pieces of a state; Sec. 3.1 reaches 34 qubits on a 32 GB GPU
   this way). The handle uses at most device_bytes of device memory (0 = a
   quarter of the free memory): two buffers of 2^m amplitudes. Gates run in
   segments: a run of gates whose dense targets lie in the low chunk bits and
   a few high bits S (at most 6) is applied to groups of 2^|S| chunks copied
   into a buffer, every gate rewritten for the group (controls and diagonal
   factors on the other high bits resolved), on the ordinary gate kernels;
   groups alternate between the buffers on two streams, so copies of one
   overlap kernels of the other. Supported on such a handle:
   qs_state_init_basis / init_plus / set / get (the host copy; the call
   synchronises), qs_apply_gates (any mode; a gate with more dense targets
   above the chunk bits than a group holds: QS_ERR_UNSUPPORTED), qs_norm2,
   qs_probabilities (host output) and qs_expectation (terms whose X bits act
   on qubits n-m .. n-1; others QS_ERR_UNSUPPORTED); every other call returns
   QS_ERR_UNSUPPORTED. cudaHostAlloc failing: QS_ERR_CUDA. */
qs_status qs_state_create_host(int n, qs_dtype dtype, size_t device_bytes, void *cuda_stream, qs_state **out);

/* ---------------------------------------------------------------- density matrices */
/* Density matrices and noise channels (Sec. 2.4, "Density matrices and
   noise"). A density matrix rho of n qubits (1 <= n <= 20) is a handle of
   2n qubits holding the 4^n entries of rho row-major: entry (r, c) at index
   r 2^n + c (per batch member, 4^n entries each), r and c basis integers with
   qubit 0 the most significant bit. qs_state_get/qs_state_set move those
   entries. On a density handle:
     - qs_state_init_basis(x) sets |x><x| (x < 2^n); qs_state_init_plus sets
       |+><+| (every entry 2^-n);
     - qs_apply_gates applies rho -> U rho U^dag for every gate U (qubits in
       [0, n)): U on the row qubits and its complex conjugate on the column
       qubits, on the ordinary gate kernels (any mode);
     - qs_probabilities returns the diagonal (batch * 2^n doubles), and
       qs_expectation Tr(rho H) (FP64 accumulation; Im ~ 0 for Hermitian rho);
     - qs_norm2 returns sum |rho_rc|^2 = Tr(rho^2), the purity;
     - batched parameters, measurements (marginals, samples), Trotter
       evolution, gradients and plans are not supported (QS_ERR_UNSUPPORTED). */
qs_status qs_density_create(int n, int batch, qs_dtype dtype, void *cuda_stream, qs_state **out);
/* Wrap caller-owned device memory of batch * 4^n amplitudes (16-byte aligned). */
qs_status qs_density_wrap(int n, int batch, qs_dtype dtype, void *dev_ptr, void *cuda_stream, qs_state **out);
/* rho_b = |psi_b><psi_b| from batch * 2^n amplitudes of the handle's dtype,
   host (on_device = 0; the call synchronises) or device memory. */
qs_status qs_density_init_pure(qs_state *s, const void *psi, int on_device);
/* Tr(rho_b) per member (FP64); out: host, batch doubles. */
qs_status qs_density_trace(qs_state *s, double *out);

/* A quantum channel in Kraus form on one or two qubits: rho -> sum_i K_i rho
   K_i^dag. kraus: host pointer to n_kraus matrices of 2^k x 2^k complex128
   (interleaved, row-major, local index as for gates: targets[0] the most
   significant bit), read during the call; sum_i K_i^dag K_i must equal the
   identity within 1e-8 (trace preserving), else QS_ERR_ARG. */
typedef struct qs_channel {
    int32_t n_targets;     /* 1 or 2 */
    int32_t targets[2];    /* distinct qubits in [0, n) */
    int32_t n_kraus;       /* 1 .. 4^n_targets */
    const double *kraus;
} qs_channel;
/* Apply channels in order to every member of a density handle (anything
   else: QS_ERR_ARG). Each channel runs as one superoperator sum_i K_i (x)
   conj(K_i) on the row and column copies of its targets (a 4 x 4 or 16 x 16
   matrix on the 2n-qubit vector), on the ordinary gate kernels. opts as in
   qs_apply_gates. */
qs_status qs_apply_channels(qs_state *s, const qs_channel *channels, size_t count, const qs_opts *opts);

/* ---------------------------------------------------------------- pass specialisation */
/* Run-time specialisation of the tiled passes (no counterpart in the paper).
   A tiled pass is first run by a generic kernel that decodes its ops at run
   time; a kernel specialised for the pass's structure (its ops, bits and
   stage maps compiled in with NVRTC for the device; its angles and matrix
   entries passed as parameters) computes the same result with far fewer
   instructions. Kernels are cached per pass structure for the process, so
   passes that differ only in their values share one (e.g. the steps of a
   Trotter evolution). The policy says when a structure gets a kernel:
   QS_JIT_OFF never; QS_JIT_TIERED (default) in the background once it is
   launched a second time; QS_JIT_EAGER in the background at its first
   launch; QS_JIT_SYNC before its first launch (the launching call waits for
   the compile). Until a kernel is ready the generic kernel runs the pass, so
   results never wait on a compile except under QS_JIT_SYNC. qs_plan_create
   with autotuning specialises the passes in its timing runs, before it
   captures them (unless the policy is QS_JIT_OFF); a plan captures whichever
   kernels are ready. With QS_JIT_FOLD or-ed into the policy, a pass launched
   a second time with the same values also gets a kernel with its values
   compiled in (a few percent faster, e.g. for a circuit run many times with
   fixed angles; queued in the background; one kernel per set of values). The
   environment variable QSIM_JIT = off, tiered, eager or sync (with "+fold"
   appended for QS_JIT_FOLD) sets the initial policy. Process-wide.
   Diagnostics on stderr: QSIM_JIT_VERBOSE (set) prints each compile's time and
   log; QSIM_PLAN_STATS (set) prints each tiled pass's op and stage counts. */
#define QS_JIT_OFF 0
#define QS_JIT_TIERED 1
#define QS_JIT_EAGER 2
#define QS_JIT_SYNC 3
#define QS_JIT_FOLD 8
qs_status qs_jit_set_policy(int policy);
/* Block until every queued background compile has finished. */
qs_status qs_jit_wait(void);
/* Drop the queued compiles that have not started (their passes stay on the
   generic kernel until queued again) and wait for the ones in progress. A
   program that exits while a compile runs should call this (or qs_jit_wait)
   first; the library also waits for them at exit. */
qs_status qs_jit_cancel(void);
/* Counters since the process started: tiled passes launched on specialised
   and on generic kernels, kernels compiled, compiles (or loads) that failed
   (their passes stay on the generic kernel), and seconds spent compiling
   (summed over threads). NULL outputs are skipped. */
qs_status qs_jit_stats(long long *specialised_launches, long long *generic_launches, long long *compiled,
                       long long *failed, double *compile_seconds);

/* Batched adiabatic evolution (Sec. 2.6, Eq. (4)) of a batch whose members have
   their own H1: member b uses the h1_counts[b] terms that follow member b-1's in
   `h1`; H0 is shared. Same schedule, splitting and step count as
   qs_adiabatic_evolve. This fast form needs: no Z terms in H0, H1's Z terms
   on at most two qubits (Ising form), the same X terms in every member's H1,
   and n >= 13 (complex64) or 12 (complex128); otherwise QS_ERR_UNSUPPORTED.
   Batch members of different widths are separate handles. */
qs_status qs_adiabatic_evolve_batch(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                                    const size_t *h1_counts, double T, double dt, int steps);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
