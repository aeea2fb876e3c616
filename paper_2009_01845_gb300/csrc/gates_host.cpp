// Host-side gate definitions: validation and lowering of qs_gate records to
// index-bit form with a double-precision matrix (Eq. (1), Sec. 2.3-2.4).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace qsim {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }
const char *last_error() { return g_err; }

qs_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("%s: out of device memory", what);
        return QS_ERR_OOM;
    }
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QS_ERR_CUDA;
}

int kind_targets(int kind) {
    switch (kind) {
    case QS_GATE_H: case QS_GATE_X: case QS_GATE_Y: case QS_GATE_Z:
    case QS_GATE_S: case QS_GATE_SDG: case QS_GATE_T: case QS_GATE_TDG:
    case QS_GATE_RX: case QS_GATE_RY: case QS_GATE_RZ: case QS_GATE_U1:
    case QS_GATE_U2: case QS_GATE_U3:
        return 1;
    case QS_GATE_CZ: case QS_GATE_CU1: case QS_GATE_SWAP:
        return 2;
    case QS_GATE_UNITARY:
        return 0;  // given by n_targets
    default:
        return -1;
    }
}

int kind_params(int kind) {
    switch (kind) {
    case QS_GATE_RX: case QS_GATE_RY: case QS_GATE_RZ: case QS_GATE_U1: case QS_GATE_CU1:
        return 1;
    case QS_GATE_U2:
        return 2;
    case QS_GATE_U3:
        return 3;
    default:
        return 0;
    }
}

// Matrices written from the gate definitions in qsim.h.
std::vector<cd> kind_matrix(int kind, const double *p) {
    const cd I(0.0, 1.0);
    const double r2 = 1.0 / std::sqrt(2.0);
    auto u3 = [&](double th, double ph, double la) {
        const double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
        return std::vector<cd>{cd(c, 0), -std::exp(I * la) * s, std::exp(I * ph) * s,
                               std::exp(I * (ph + la)) * c};
    };
    switch (kind) {
    case QS_GATE_H: return {r2, r2, r2, -r2};
    case QS_GATE_X: return {0.0, 1.0, 1.0, 0.0};
    case QS_GATE_Y: return {0.0, -I, I, 0.0};
    case QS_GATE_Z: return {1.0, 0.0, 0.0, -1.0};
    case QS_GATE_S: return {1.0, 0.0, 0.0, I};
    case QS_GATE_SDG: return {1.0, 0.0, 0.0, -I};
    case QS_GATE_T: return {1.0, 0.0, 0.0, std::exp(I * (M_PI / 4))};
    case QS_GATE_TDG: return {1.0, 0.0, 0.0, std::exp(-I * (M_PI / 4))};
    case QS_GATE_RX: {
        const double c = std::cos(0.5 * p[0]), s = std::sin(0.5 * p[0]);
        return {c, -I * s, -I * s, c};
    }
    case QS_GATE_RY: {
        const double c = std::cos(0.5 * p[0]), s = std::sin(0.5 * p[0]);
        return {c, -s, s, c};
    }
    case QS_GATE_RZ: return {std::exp(-0.5 * I * p[0]), 0.0, 0.0, std::exp(0.5 * I * p[0])};
    case QS_GATE_U1: return {1.0, 0.0, 0.0, std::exp(I * p[0])};
    case QS_GATE_U2: return u3(M_PI / 2, p[0], p[1]);
    case QS_GATE_U3: return u3(p[0], p[1], p[2]);
    case QS_GATE_CZ: {
        std::vector<cd> m(16, 0.0);
        m[0] = m[5] = m[10] = 1.0;
        m[15] = -1.0;
        return m;
    }
    case QS_GATE_CU1: {
        std::vector<cd> m(16, 0.0);
        m[0] = m[5] = m[10] = 1.0;
        m[15] = std::exp(I * p[0]);
        return m;
    }
    case QS_GATE_SWAP: {
        std::vector<cd> m(16, 0.0);
        m[0] = m[15] = 1.0;
        m[1 * 4 + 2] = m[2 * 4 + 1] = 1.0;
        return m;
    }
    default:
        return {};
    }
}

qs_status lower_gate(int n, const qs_gate &g, LGate *out) {
    const int kt = kind_targets(g.kind);
    if (kt < 0) {
        set_error("unknown gate kind %d", g.kind);
        return QS_ERR_ARG;
    }
    const int k = (g.kind == QS_GATE_UNITARY) ? g.n_targets : kt;
    if (g.n_targets != k || k < 1 || k > QS_MAX_TARGETS) {
        set_error("gate kind %d: n_targets %d does not match its arity", g.kind, g.n_targets);
        return QS_ERR_ARG;
    }
    if (k > n) {
        set_error("gate has %d targets on a %d-qubit state", k, n);
        return QS_ERR_ARG;
    }
    uint64_t tq = 0;
    for (int j = 0; j < k; ++j) {
        const int q = g.targets[j];
        if (q < 0 || q >= n) {
            set_error("target qubit %d out of range [0, %d)", q, n);
            return QS_ERR_ARG;
        }
        if (tq & (1ull << q)) {
            set_error("target qubit %d repeated", q);
            return QS_ERR_ARG;
        }
        tq |= 1ull << q;
    }
    if (n < 64 && (g.control_mask >> n) != 0) {
        set_error("control mask names a qubit >= n = %d", n);
        return QS_ERR_ARG;
    }
    if (g.control_mask & tq) {
        set_error("a qubit is both target and control");
        return QS_ERR_ARG;
    }
    out->k = k;
    out->kind = g.kind;
    out->param_index = g.param_index;
    for (int j = 0; j < k; ++j) out->tbit[j] = n - 1 - g.targets[j];
    out->cmask = 0;
    for (int q = 0; q < n; ++q)
        if ((g.control_mask >> q) & 1ull) out->cmask |= qbit(n, q);
    const int K = 1 << k;
    if (g.kind == QS_GATE_UNITARY) {
        if (!g.matrix) {
            set_error("UNITARY gate without a matrix");
            return QS_ERR_ARG;
        }
        out->m.resize(K * K);
        for (int i = 0; i < K * K; ++i) {
            out->m[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
            if (!std::isfinite(g.matrix[2 * i]) || !std::isfinite(g.matrix[2 * i + 1])) {
                set_error("UNITARY matrix has a non-finite entry");
                return QS_ERR_ARG;
            }
        }
    } else {
        for (int i = 0; i < kind_params(g.kind); ++i)
            if (!std::isfinite(g.params[i])) {
                set_error("non-finite gate angle");
                return QS_ERR_ARG;
            }
        out->m = kind_matrix(g.kind, g.params);
    }
    set_matrix_flags(out);
    out->is_swap = (g.kind == QS_GATE_SWAP);
    return QS_OK;
}

void set_matrix_flags(LGate *g) {
    const int K = 1 << g->k;
    bool diag = true, phase = true;
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) {
            const cd v = g->m[r * K + c];
            if (r != c && v != cd(0.0)) diag = false;
            if (r == c && r != K - 1 && v != cd(1.0)) phase = false;
        }
    g->diagonal = diag;
    g->phase_only = diag && phase;
}

}  // namespace qsim
