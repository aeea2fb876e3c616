// Gate-queue execution strategies and the Trotter driver.
#include <cmath>
#include <cstring>

#include "fused.h"
#include "plan.h"
#include "tiled.h"

#include <algorithm>

namespace qsim {

void plan_cache_release(qs_state *) {}

static qs_status run_unfused(qs_state *s, const std::vector<LGate> &gates, const double *params, int n_params) {
    for (const LGate &g : gates) {
        if (g.param_index >= 0)
            QS_TRY(k_apply_param_gate(s, g, params, n_params));
        else
            QS_TRY(k_apply_unfused(s, g));
    }
    return QS_OK;
}

qs_status run_gates(qs_state *s, std::vector<LGate> &gates, int mode, const qs_opts *opts,
                    const double *params_dev, int n_params) {
    // complex128 arithmetic of the one-gate passes for this call
    struct Fp64Scope {
        explicit Fp64Scope(bool on) { set_c128_fp64(on); }
        ~Fp64Scope() { set_c128_fp64(false); }
    } fp64(opts && (opts->flags & QS_OPT_C128_FP64));
    switch (mode) {
    case QS_MODE_UNFUSED:
        return run_unfused(s, gates, params_dev, n_params);
    case QS_MODE_FUSED_TC:
        return run_fused(s, gates, opts ? opts->fuse_qubits : 5, params_dev, n_params);
    case QS_MODE_AUTO:
    case QS_MODE_TILED:
    default:
        return run_tiled(s, gates, params_dev, n_params);
    }
}

// ------------------------------------------------------------------ Trotter
// H(s) = (1-s) H0 + s H1 split into D(s) (Z strings) and X(s) = sum_q a_q(s) X_q.
struct TrotterTerms {
    std::vector<double> d0, d1;   // diagonal coefficients of H0 / H1 terms
    std::vector<uint64_t> z0, z1; // their Z masks in index bits
    std::vector<double> a0, a1;   // per-qubit X coefficient of H0 / H1
};

static qs_status split_terms(int n, const qs_pauli_term *t, size_t count, std::vector<double> *d,
                             std::vector<uint64_t> *z, std::vector<double> *a) {
    a->assign(n, 0.0);
    for (size_t i = 0; i < count; ++i) {
        if (t[i].x_mask == 0) {
            uint64_t zb = 0;
            for (int q = 0; q < n; ++q)
                if ((t[i].z_mask >> q) & 1ull) zb |= qbit(n, q);
            d->push_back(t[i].coeff);
            z->push_back(zb);
        } else if (t[i].z_mask == 0 && __builtin_popcountll(t[i].x_mask) == 1) {
            (*a)[__builtin_ctzll(t[i].x_mask)] += t[i].coeff;
        } else {
            set_error("Trotter terms must be Z strings or single-qubit X terms (term %zu)", i);
            return QS_ERR_UNSUPPORTED;
        }
    }
    return QS_OK;
}

// exp(-i tau [w0 D0 + w1 D1])
static qs_status diag_factor(qs_state *s, const TrotterTerms &tt, double w0, double w1, double tau) {
    std::vector<double> c;
    std::vector<uint64_t> z;
    for (size_t i = 0; i < tt.d0.size(); ++i) {
        c.push_back(w0 * tt.d0[i]);
        z.push_back(tt.z0[i]);
    }
    for (size_t i = 0; i < tt.d1.size(); ++i) {
        c.push_back(w1 * tt.d1[i]);
        z.push_back(tt.z1[i]);
    }
    if (c.empty()) return QS_OK;
    return k_diagonal_evolution(s, c, z, tau);
}

// exp(-i dt X(s)) = prod_q RX(2 dt a_q(s)), RX(th) = exp(-i th X / 2)
static qs_status x_layer(qs_state *s, const TrotterTerms &tt, double sv, double dt) {
    const int n = s->n;
    for (int q = 0; q < n; ++q) {
        const double a = (1.0 - sv) * tt.a0[q] + sv * tt.a1[q];
        if (a == 0.0) continue;
        qs_gate g;
        std::memset(&g, 0, sizeof(g));
        g.kind = QS_GATE_RX;
        g.n_targets = 1;
        g.targets[0] = q;
        g.param_index = -1;
        g.params[0] = 2.0 * dt * a;
        LGate lg;
        QS_TRY(lower_gate(n, g, &lg));
        QS_TRY(k_apply_unfused(s, lg));
    }
    return QS_OK;
}

// Ising table of a diagonal Pauli sum (terms of at most two Z bits), in index
// bits: J[a * n + b] (symmetric), h[n], constant. False if a term has more bits.
static bool ising_table(int n, const std::vector<double> &d, const std::vector<uint64_t> &z, double *out) {
    std::fill(out, out + (size_t)n * n + n + 1, 0.0);
    for (size_t i = 0; i < d.size(); ++i) {
        const int pc = __builtin_popcountll(z[i]);
        if (pc == 0) {
            out[(size_t)n * n + n] += d[i];
        } else if (pc == 1) {
            out[(size_t)n * n + __builtin_ctzll(z[i])] += d[i];
        } else if (pc == 2) {
            const int a = __builtin_ctzll(z[i]), b = 63 - __builtin_clzll(z[i]);
            out[(size_t)a * n + b] += d[i];
            out[(size_t)b * n + a] += d[i];
        } else {
            return false;
        }
    }
    return true;
}

qs_status ensure_itab(qs_state *s, size_t doubles) {
    if (s->itab_bytes >= doubles * sizeof(double)) return QS_OK;
    if (s->itab) {
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        cudaFree(s->itab);
        s->itab = nullptr;
        s->itab_bytes = 0;
    }
    QS_CUDA_TRY(cudaMalloc(&s->itab, doubles * sizeof(double)));
    s->itab_bytes = doubles * sizeof(double);
    return QS_OK;
}

// The Trotter queue of tiled passes: Ising phases exp(-i tau E1(x)) and RX
// layers. `taus[k]` precedes layer k; layer k rotates qubit q by 2 dt a_q(s_k).
static qs_status trotter_tiled(qs_state *s, const TrotterTerms &tt, const std::vector<double> &taus,
                               const std::vector<double> &svals, double dt) {
    std::vector<LGate> G;
    QS_TRY(trotter_queue(s->n, tt.a0, tt.a1, taus, svals, dt, !tt.d1.empty(), &G));
    return run_tiled(s, G, nullptr, 0);
}

qs_status run_trotter(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1, size_t n_h1,
                      double s_fixed, double dt, double T, int steps) {
    TrotterTerms tt;
    QS_TRY(split_terms(s->n, h0, n_h0, &tt.d0, &tt.z0, &tt.a0));
    QS_TRY(split_terms(s->n, h1, n_h1, &tt.d1, &tt.z1, &tt.a1));
    // tiled path: the state spans a tile, H0 has no diagonal part and H1's is Ising-form
    std::vector<double> table((size_t)s->n * s->n + s->n + 1);
    if (s->n >= tile_bits(s->dtype) && tt.d0.empty() && ising_table(s->n, tt.d1, tt.z1, table.data())) {
        QS_TRY(ensure_itab(s, table.size()));
        s->ising_stride = 0;
        QS_CUDA_TRY(cudaMemcpyAsync(s->itab, table.data(), table.size() * sizeof(double), cudaMemcpyHostToDevice,
                                    s->stream));
        std::vector<double> taus, svals;
        if (s_fixed >= 0.0) {
            svals = {s_fixed};
            taus = {0.5 * dt * s_fixed, 0.5 * dt * s_fixed};
        } else {
            for (int k = 0; k < steps; ++k) svals.push_back((k + 0.5) * dt / T);
            taus.push_back(0.5 * dt * svals[0]);
            for (int k = 0; k + 1 < steps; ++k) taus.push_back(0.5 * dt * (svals[k] + svals[k + 1]));
            taus.push_back(0.5 * dt * svals[steps - 1]);
        }
        return trotter_tiled(s, tt, taus, svals, dt);
    }
    if (s_fixed >= 0.0) {
        const double sv = s_fixed;
        QS_TRY(diag_factor(s, tt, 1.0 - sv, sv, 0.5 * dt));
        QS_TRY(x_layer(s, tt, sv, dt));
        QS_TRY(diag_factor(s, tt, 1.0 - sv, sv, 0.5 * dt));
        return QS_OK;
    }
    // linear schedule, midpoint s; the closing half diagonal of step k and the
    // opening one of step k+1 commute and merge into one pass
    for (int k = 0; k < steps; ++k) {
        const double sk = (k + 0.5) * dt / T;
        if (k == 0) QS_TRY(diag_factor(s, tt, 1.0 - sk, sk, 0.5 * dt));
        QS_TRY(x_layer(s, tt, sk, dt));
        if (k + 1 < steps) {
            const double sn = (k + 1.5) * dt / T;
            QS_TRY(diag_factor(s, tt, (1.0 - sk) + (1.0 - sn), sk + sn, 0.5 * dt));
        } else {
            QS_TRY(diag_factor(s, tt, 1.0 - sk, sk, 0.5 * dt));
        }
    }
    return QS_OK;
}

// Batched adiabatic evolution: member b evolves under its own H1 (terms
// h1[off[b] .. off[b+1])). Every member's X terms must agree (one RX layer for
// the batch); the Ising diagonals are per member. Prepare validates the terms
// and uploads the per-member Ising tables on the state's stream.
static qs_status adiabatic_batch_prepare(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                                         const size_t *off, TrotterTerms *tt) {
    const int n = s->n;
    const size_t stride = (size_t)n * n + n + 1;
    QS_TRY(split_terms(n, h0, n_h0, &tt->d0, &tt->z0, &tt->a0));
    if (!tt->d0.empty()) {
        set_error("batched evolution needs an H0 without Z terms");
        return QS_ERR_UNSUPPORTED;
    }
    if (n < tile_bits(s->dtype)) {
        set_error("batched evolution needs n >= %d", tile_bits(s->dtype));
        return QS_ERR_UNSUPPORTED;
    }
    std::vector<double> tables(stride * s->batch);
    for (int b = 0; b < s->batch; ++b) {
        std::vector<double> d;
        std::vector<uint64_t> z;
        std::vector<double> a;
        QS_TRY(split_terms(n, h1 + off[b], off[b + 1] - off[b], &d, &z, &a));
        if (b == 0) {
            tt->a1 = a;
            tt->d1 = d;  // only its emptiness is used below
        } else if (a != tt->a1) {
            set_error("member %d: X terms of H1 differ from member 0", b);
            return QS_ERR_UNSUPPORTED;
        }
        if (!d.empty()) tt->d1.assign(1, 1.0);
        if (!ising_table(n, d, z, tables.data() + stride * b)) {
            set_error("member %d: H1 has a Z term on more than two qubits", b);
            return QS_ERR_UNSUPPORTED;
        }
    }
    QS_TRY(ensure_itab(s, tables.size()));
    s->ising_stride = (uint32_t)stride;
    // (a copy from pageable host memory has read the table when it returns)
    QS_CUDA_TRY(cudaMemcpyAsync(s->itab, tables.data(), tables.size() * sizeof(double), cudaMemcpyHostToDevice,
                                s->stream));
    return QS_OK;
}

// Steps k0 .. k1-1 of the K-step linear schedule (step k at s_k = (k + 1/2)
// dt / T): inside the range adjacent half diagonals are merged; the range opens
// with its first half step and closes with its last, so consecutive ranges
// compose to the whole evolution (up to rounding).
static qs_status adiabatic_batch_steps(qs_state *s, const TrotterTerms &tt, double dt, double T, int k0, int k1) {
    std::vector<double> taus, svals;
    for (int k = k0; k < k1; ++k) svals.push_back((k + 0.5) * dt / T);
    const int m = (int)svals.size();
    taus.push_back(0.5 * dt * svals[0]);
    for (int k = 0; k + 1 < m; ++k) taus.push_back(0.5 * dt * (svals[k] + svals[k + 1]));
    taus.push_back(0.5 * dt * svals[m - 1]);
    return trotter_tiled(s, tt, taus, svals, dt);
}

qs_status run_adiabatic_batch(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                              const size_t *off, double dt, double T, int steps) {
    TrotterTerms tt;
    QS_TRY(adiabatic_batch_prepare(s, h0, n_h0, h1, off, &tt));
    return adiabatic_batch_steps(s, tt, dt, T, 0, steps);
}

// Instances of several widths: one handle per width, each evolved on a stream
// of its own, forked from states[0]'s stream and joined back into it (and into
// each handle's own stream). The steps are enqueued in chunks, round robin over
// the handles, so every stream has work queued early and the GPU runs the
// widths side by side (no stream's queue grows long enough to block the host).
qs_status run_adiabatic_multi(qs_state *const *states, int n_states, const qs_pauli_term *h0,
                              const size_t *h0_off, const qs_pauli_term *h1, const size_t *h1_off, double dt,
                              double T, int steps, int chunk) {
    std::vector<cudaStream_t> own(n_states), work(n_states, nullptr);
    std::vector<cudaEvent_t> done(n_states, nullptr);
    cudaEvent_t fork = nullptr;
    for (int i = 0; i < n_states; ++i) own[i] = states[i]->stream;
    auto cleanup = [&]() {
        for (int i = 0; i < n_states; ++i) {
            states[i]->stream = own[i];
            if (work[i]) cudaStreamDestroy(work[i]);  // released once its work completes
            if (done[i]) cudaEventDestroy(done[i]);
        }
        if (fork) cudaEventDestroy(fork);
    };
    qs_status st = QS_OK;
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == QS_OK) st = cuda_status(e, what);
        return st == QS_OK;
    };
    if (!cuda(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event") ||
        !cuda(cudaEventRecord(fork, own[0]), "fork")) {
        cleanup();
        return st;
    }
    for (int i = 0; i < n_states && st == QS_OK; ++i) {
        if (!cuda(cudaStreamCreateWithFlags(&work[i], cudaStreamNonBlocking), "stream") ||
            !cuda(cudaStreamWaitEvent(work[i], fork, 0), "fork wait"))
            break;
        // the handle's own earlier work comes first too
        cudaEvent_t e = nullptr;
        if (own[i] != own[0]) {
            if (!cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event")) break;
            cuda(cudaEventRecord(e, own[i]), "record");
            cuda(cudaStreamWaitEvent(work[i], e, 0), "wait");
            cudaEventDestroy(e);
        }
        states[i]->stream = work[i];
    }
    std::vector<TrotterTerms> tt(n_states);
    size_t m0 = 0;  // first member of handle i among all members
    for (int i = 0; i < n_states && st == QS_OK; ++i) {
        std::vector<size_t> off(states[i]->batch + 1);
        for (int b = 0; b <= states[i]->batch; ++b) off[b] = h1_off[m0 + b] - h1_off[m0];
        st = adiabatic_batch_prepare(states[i], h0 + h0_off[i], h0_off[i + 1] - h0_off[i], h1 + h1_off[m0],
                                     off.data(), &tt[i]);
        m0 += states[i]->batch;
    }
    for (int k0 = 0; k0 < steps && st == QS_OK; k0 += chunk)
        for (int i = 0; i < n_states && st == QS_OK; ++i)
            st = adiabatic_batch_steps(states[i], tt[i], dt, T, k0, std::min(steps, k0 + chunk));
    for (int i = 0; i < n_states && work[i]; ++i) {
        if (!cuda(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming), "event") ||
            !cuda(cudaEventRecord(done[i], work[i]), "join"))
            break;
        cuda(cudaStreamWaitEvent(own[0], done[i], 0), "join wait");
        if (own[i] != own[0]) cuda(cudaStreamWaitEvent(own[i], done[i], 0), "join wait");
    }
    cleanup();
    return st;
}

}  // namespace qsim
