// Gate-queue execution strategies and the Trotter driver.
#include <cmath>
#include <cstring>

#include "plan.h"

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
    (void)opts;
    switch (mode) {
    case QS_MODE_UNFUSED:
        return run_unfused(s, gates, params_dev, n_params);
    case QS_MODE_AUTO:
    case QS_MODE_TILED:
    case QS_MODE_FUSED_TC:
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

qs_status run_trotter(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1, size_t n_h1,
                      double s_fixed, double dt, double T, int steps) {
    TrotterTerms tt;
    QS_TRY(split_terms(s->n, h0, n_h0, &tt.d0, &tt.z0, &tt.a0));
    QS_TRY(split_terms(s->n, h1, n_h1, &tt.d1, &tt.z1, &tt.a1));
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

}  // namespace qsim
