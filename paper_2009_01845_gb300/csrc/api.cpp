// The C-ABI entry points declared in include/qsim.h: argument validation,
// state handles, and dispatch to the planners and kernels. No exception or
// abort crosses this boundary; every failure becomes a qs_status plus a
// thread-local message.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "tiled.h"

namespace qsim {
qs_status energy_gradient(qs_state *w, const std::vector<LGate> &G, const double *params, int n_params,
                          const qs_pauli_term *terms, size_t n_terms, int init_zero, double *energy,
                          double *grad, int ckpt_every, int mode);
}

namespace qsim {
const char *last_error();
}

using namespace qsim;

#define QS_GUARD_BEGIN try {
#define QS_GUARD_END                                                     \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        set_error("host allocation failed");                             \
        return QS_ERR_OOM;                                               \
    }                                                                    \
    catch (...) {                                                        \
        set_error("internal error");                                     \
        return QS_ERR_CUDA;                                              \
    }

static qs_status check_state(const qs_state *s) {
    if (!s) {
        set_error("null state handle");
        return QS_ERR_ARG;
    }
    return QS_OK;
}

static qs_status check_shape(int n, int batch, qs_dtype dtype) {
    if (n < 1 || n > QS_MAX_QUBITS) {
        set_error("n = %d outside [1, %d]", n, QS_MAX_QUBITS);
        return QS_ERR_ARG;
    }
    if (batch < 1 || batch > QS_MAX_BATCH) {
        set_error("batch = %d outside [1, %d] (members are a grid dimension of at most 65535)", batch,
                  QS_MAX_BATCH);
        return QS_ERR_ARG;
    }
    if (dtype != QS_C64 && dtype != QS_C128) {
        set_error("unknown dtype %d", dtype);
        return QS_ERR_ARG;
    }
    // total amplitudes must stay below 2^46 (64-bit index arithmetic with headroom)
    if ((uint64_t)batch > (1ull << (46 - n))) {
        set_error("batch * 2^n too large");
        return QS_ERR_ARG;
    }
    return QS_OK;
}

static size_t state_bytes(const qs_state *s) {
    return ((size_t)s->batch << s->n) * (s->dtype == QS_C64 ? 8 : 16);
}

extern "C" {

const char *qs_last_error(void) { return qsim::last_error(); }
const char *qs_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

qs_status qs_state_create(int n, int batch, qs_dtype dtype, void *stream, qs_state **out) {
    QS_GUARD_BEGIN
    clear_error();
    if (!out) {
        set_error("null output pointer");
        return QS_ERR_ARG;
    }
    *out = nullptr;
    QS_TRY(check_shape(n, batch, dtype));
    qs_state *s = new qs_state();
    s->n = n;
    s->ms = n;
    s->batch = batch;
    s->dtype = dtype;
    s->stream = (cudaStream_t)stream;
    s->owns = true;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->data, state_bytes(s));
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e, "cudaMalloc(state)");
    }
    *out = s;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_state_wrap(int n, int batch, qs_dtype dtype, void *dev_ptr, void *stream, qs_state **out) {
    QS_GUARD_BEGIN
    clear_error();
    if (!out) {
        set_error("null output pointer");
        return QS_ERR_ARG;
    }
    *out = nullptr;
    QS_TRY(check_shape(n, batch, dtype));
    if (!dev_ptr || ((uintptr_t)dev_ptr & 15u)) {
        set_error("device pointer must be non-null and 16-byte aligned");
        return QS_ERR_ARG;
    }
    qs_state *s = new qs_state();
    s->n = n;
    s->ms = n;
    s->batch = batch;
    s->dtype = dtype;
    s->stream = (cudaStream_t)stream;
    s->data = dev_ptr;
    s->owns = false;
    cudaGetDevice(&s->device);
    *out = s;
    return QS_OK;
    QS_GUARD_END
}

static qs_status check_density_n(int n) {
    if (n < 1 || 2 * n > QS_MAX_QUBITS) {
        set_error("density matrix of n = %d qubits: 1 <= n <= %d", n, QS_MAX_QUBITS / 2);
        return QS_ERR_ARG;
    }
    return QS_OK;
}

qs_status qs_density_create(int n, int batch, qs_dtype dtype, void *stream, qs_state **out) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_density_n(n));
    QS_TRY(qs_state_create(2 * n, batch, dtype, stream, out));
    (*out)->dm = n;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_density_wrap(int n, int batch, qs_dtype dtype, void *dev_ptr, void *stream, qs_state **out) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_density_n(n));
    QS_TRY(qs_state_wrap(2 * n, batch, dtype, dev_ptr, stream, out));
    (*out)->dm = n;
    return QS_OK;
    QS_GUARD_END
}

static qs_status not_for_density(const qs_state *s, const char *what) {
    if (s && s->dm) {
        set_error("%s is not supported on a density matrix", what);
        return QS_ERR_UNSUPPORTED;
    }
    if (s && s->host) {
        set_error("%s is not supported on a host-memory state", what);
        return QS_ERR_UNSUPPORTED;
    }
    return QS_OK;
}

static qs_status not_for_host(const qs_state *s, const char *what) {
    if (s && s->host) {
        set_error("%s is not supported on a host-memory state", what);
        return QS_ERR_UNSUPPORTED;
    }
    return QS_OK;
}

qs_status qs_state_create_host(int n, qs_dtype dtype, size_t device_bytes, void *stream, qs_state **out) {
    QS_GUARD_BEGIN
    clear_error();
    if (!out) {
        set_error("null output pointer");
        return QS_ERR_ARG;
    }
    *out = nullptr;
    QS_TRY(check_shape(n, 1, dtype));
    int dev = 0;
    QS_CUDA_TRY(cudaGetDevice(&dev));
    const size_t b = dtype == QS_C64 ? 8 : 16;
    if (device_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        QS_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        device_bytes = free_b / 4;
    }
    int m = 0;
    while (m < n && ((size_t)2 << (m + 1)) * b <= device_bytes) ++m;  // two buffers of 2^m amplitudes
    if (m < 1) {
        set_error("a device budget of %zu bytes holds no buffer", device_bytes);
        return QS_ERR_ARG;
    }
    qs_state *s = new qs_state();
    s->n = n;
    s->ms = n;
    s->batch = 1;
    s->dtype = dtype;
    s->stream = (cudaStream_t)stream;
    s->device = dev;
    s->owns = true;
    s->pm = m;
    // high bits a group brings into a buffer: up to 6, keeping chunks of at
    // least 2^16 amplitudes where the buffer allows (copies stay large), and at
    // least 2 (or m - 1 for a tiny buffer) so a two-qubit gate always fits
    s->pm = std::min(m, n);
    const int sg = std::min(std::min(6, std::max(2, m - 16)), std::max(0, m - 1));
    s->pl = m - sg;
    const cudaError_t e = cudaHostAlloc(&s->host, ((size_t)1 << n) * b, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e, "cudaHostAlloc(state)");
    }
    *out = s;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_state_destroy(qs_state *s) {
    QS_GUARD_BEGIN
    if (!s) return QS_OK;
    if (s->owns || s->scratch || s->host_pinned || s->gtab || s->ptab || s->itab || s->ithr)
        cudaStreamSynchronize(s->stream);
    if (s->owns && s->data) cudaFree(s->data);
    if (s->host) {
        cudaStreamSynchronize(s->stream);
        cudaFreeHost(s->host);
    }
    for (void *pb : s->pbuf)
        if (pb) cudaFree(pb);
    if (s->scratch) cudaFree(s->scratch);
    if (s->host_pinned) cudaFreeHost(s->host_pinned);
    if (s->gtab) cudaFree(s->gtab);
    if (s->ptab) cudaFree(s->ptab);
    if (s->itab) cudaFree(s->itab);
    if (s->ithr) cudaFree(s->ithr);
    plan_cache_release(s);
    delete s;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_state_data(const qs_state *s, void **dev_ptr) {
    QS_TRY(check_state(s));
    if (!dev_ptr) {
        set_error("null output pointer");
        return QS_ERR_ARG;
    }
    if (s->host) {
        set_error("a host-memory state has no device array");
        return QS_ERR_UNSUPPORTED;
    }
    *dev_ptr = s->data;
    return QS_OK;
}

qs_status qs_state_set_stream(qs_state *s, void *stream) {
    QS_TRY(check_state(s));
    s->stream = (cudaStream_t)stream;
    return QS_OK;
}

qs_status qs_state_init_basis(qs_state *s, uint64_t x) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (s->dm) {  // |x><x|: entry (x, x)
        if ((x >> s->dm) != 0) {
            set_error("basis index %llu >= 2^%d", (unsigned long long)x, s->dm);
            return QS_ERR_ARG;
        }
        return k_init_basis(s, x * ((1ull << s->dm) + 1ull));
    }
    if (s->n < 64 && (x >> s->n) != 0) {
        set_error("basis index %llu >= 2^%d", (unsigned long long)x, s->n);
        return QS_ERR_ARG;
    }
    if (s->host) return host_init(s, false, x);
    return k_init_basis(s, x);
    QS_GUARD_END
}

qs_status qs_state_init_plus(qs_state *s) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (s->host) return host_init(s, true, 0);
    return k_init_plus(s);
    QS_GUARD_END
}

qs_status qs_state_set(qs_state *s, const void *src, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!src) {
        set_error("null source");
        return QS_ERR_ARG;
    }
    if (s->host) {
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        QS_CUDA_TRY(cudaMemcpy(s->host, src, state_bytes(s), on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
        return QS_OK;
    }
    QS_CUDA_TRY(cudaMemcpyAsync(s->data, src, state_bytes(s),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
    if (!on_device) QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_state_get(const qs_state *s, void *dst, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!dst) {
        set_error("null destination");
        return QS_ERR_ARG;
    }
    if (s->host) {
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        QS_CUDA_TRY(cudaMemcpy(dst, s->host, state_bytes(s), on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
        return QS_OK;
    }
    QS_CUDA_TRY(cudaMemcpyAsync(dst, s->data, state_bytes(s),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    if (!on_device) QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
    QS_GUARD_END
}

// On a density matrix of dm qubits (a 2 dm-qubit vector, row qubit q = vector
// qubit q, column qubit q = vector qubit dm + q), U rho U^dag is U on the row
// bits (index bits dm .. 2 dm - 1) and conj(U) on the column bits.
static void density_pair(int dm, const LGate &g, LGate *row, LGate *col) {
    *row = g;
    for (int j = 0; j < g.k; ++j) row->tbit[j] = g.tbit[j] + dm;
    row->cmask = g.cmask << dm;
    *col = g;
    for (auto &v : col->m) v = std::conj(v);
    col->kind = QS_GATE_UNITARY;
    set_matrix_flags(col);
}

static qs_status lower_all(const qs_state *s, const qs_gate *gates, size_t count, std::vector<LGate> *out) {
    if (count && !gates) {
        set_error("null gate array");
        return QS_ERR_ARG;
    }
    const int n = s->dm ? s->dm : s->n;
    out->resize(count);
    for (size_t i = 0; i < count; ++i) {
        qs_status st = lower_gate(n, gates[i], &(*out)[i]);
        if (st != QS_OK) {
            char buf[512];
            std::snprintf(buf, sizeof(buf), "gate %zu: %s", i, qs_last_error());
            set_error("%s", buf);
            return st;
        }
    }
    if (s->dm) {
        std::vector<LGate> both(2 * count);
        for (size_t i = 0; i < count; ++i) density_pair(s->dm, (*out)[i], &both[2 * i], &both[2 * i + 1]);
        out->swap(both);
    }
    return QS_OK;
}

static qs_status check_opts(const qs_state *s, const qs_opts *o, int *mode) {
    *mode = o ? o->mode : QS_MODE_AUTO;
    if (*mode < QS_MODE_AUTO || *mode > QS_MODE_FUSED_TC) {
        set_error("unknown mode %d", *mode);
        return QS_ERR_ARG;
    }
    // the tile width is the kernel's own (its register, lane and warp bits)
    if (o && o->tile_qubits != 0 && o->tile_qubits != tile_bits(s->dtype)) {
        set_error("tile width %d: the tiled kernels take %d bits for this precision", o->tile_qubits,
                  tile_bits(s->dtype));
        return QS_ERR_UNSUPPORTED;
    }
    if (o && (o->flags & ~QS_OPT_C128_FP64) != 0) {
        set_error("unknown opts.flags bits 0x%x", o->flags & ~QS_OPT_C128_FP64);
        return QS_ERR_ARG;
    }
    return QS_OK;
}

qs_status qs_apply_gates(qs_state *s, const qs_gate *gates, size_t count, const qs_opts *opts) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    int mode;
    QS_TRY(check_opts(s, opts, &mode));
    std::vector<LGate> lg;
    QS_TRY(lower_all(s, gates, count, &lg));
    for (auto &g : lg)
        if (g.param_index >= 0) g.param_index = -1;  // unbatched call: angles come from params
    if (s->host) return host_apply(s, lg, mode, opts);
    return run_gates(s, lg, mode, opts, nullptr, 0);
    QS_GUARD_END
}

qs_status qs_apply_gates_batched(qs_state *s, const qs_gate *gates, size_t count, const double *params_dev,
                                 int n_params, const qs_opts *opts) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "batched parameters"));
    int mode;
    QS_TRY(check_opts(s, opts, &mode));
    std::vector<LGate> lg;
    QS_TRY(lower_all(s, gates, count, &lg));
    for (size_t i = 0; i < lg.size(); ++i) {
        const int p = lg[i].param_index;
        if (p < 0) continue;
        if (p >= n_params || !params_dev) {
            set_error("gate %zu: param_index %d outside [0, %d)", i, p, n_params);
            return QS_ERR_ARG;
        }
        const int kd = lg[i].kind;
        if (kd != QS_GATE_RX && kd != QS_GATE_RY && kd != QS_GATE_RZ && kd != QS_GATE_U1 && kd != QS_GATE_CU1) {
            set_error("gate %zu: batched parameters apply to RX RY RZ U1 CU1 only", i);
            return QS_ERR_ARG;
        }
    }
    return run_gates(s, lg, mode, opts, params_dev, n_params);
    QS_GUARD_END
}

static qs_status read_back(qs_state *s, const double *dev, double *host, size_t count) {
    QS_CUDA_TRY(cudaMemcpyAsync(host, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
}

qs_status qs_probabilities(qs_state *s, double *out, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!out) {
        set_error("null output");
        return QS_ERR_ARG;
    }
    auto probs = [&](double *dst) { return s->dm ? k_dm_probabilities(s, dst) : k_probabilities(s, dst); };
    if (s->host) {
        if (on_device) {
            set_error("probabilities of a host-memory state go to host memory");
            return QS_ERR_UNSUPPORTED;
        }
        return host_probabilities(s, out);
    }
    if (on_device) return probs(out);
    const size_t total = (size_t)s->batch << (s->dm ? s->dm : s->n);
    double *tmp = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&tmp, total * sizeof(double), s->stream));
    qs_status st = probs(tmp);
    if (st == QS_OK) st = read_back(s, tmp, out, total);
    cudaFreeAsync(tmp, s->stream);
    return st;
    QS_GUARD_END
}

qs_status qs_marginal_probabilities(qs_state *s, const int *qubits, int m, double *out, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "marginal probabilities"));
    if (!out || !qubits) {
        set_error("null argument");
        return QS_ERR_ARG;
    }
    if (m < 1 || m > QS_MARGINAL_MAX_QUBITS || m > s->n) {
        set_error("group of %d qubits: 1 to %d and at most n", m, QS_MARGINAL_MAX_QUBITS);
        return QS_ERR_ARG;
    }
    int bitpos[QS_MARGINAL_MAX_QUBITS];
    uint64_t seen = 0;
    for (int j = 0; j < m; ++j) {
        const int q = qubits[j];
        if (q < 0 || q >= s->n || ((seen >> q) & 1ull)) {
            set_error("qubit %d out of range or repeated", q);
            return QS_ERR_ARG;
        }
        seen |= 1ull << q;
        bitpos[j] = s->n - 1 - q;
    }
    const size_t total = (size_t)s->batch << m;
    if (on_device) return k_marginal(s, bitpos, m, out);
    double *tmp = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&tmp, total * sizeof(double), s->stream));
    qs_status st = k_marginal(s, bitpos, m, tmp);
    if (st == QS_OK) st = read_back(s, tmp, out, total);
    cudaFreeAsync(tmp, s->stream);
    return st;
    QS_GUARD_END
}

qs_status qs_sample(qs_state *s, int member, const double *uniforms, size_t shots, uint64_t *out, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "sampling"));
    if (member < 0 || member >= s->batch) {
        set_error("member %d outside the batch of %d", member, s->batch);
        return QS_ERR_ARG;
    }
    if (shots == 0) return QS_OK;
    if (!uniforms || !out) {
        set_error("null argument");
        return QS_ERR_ARG;
    }
    if (on_device) return k_sample(s, member, uniforms, shots, out);
    for (size_t i = 0; i < shots; ++i)
        if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) {
            set_error("uniform %zu = %g is not in [0, 1)", i, uniforms[i]);
            return QS_ERR_ARG;
        }
    auto ok = [](cudaError_t e, const char *what) { return e == cudaSuccess ? QS_OK : cuda_status(e, what); };
    double *ud = nullptr;
    uint64_t *od = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&ud, shots * sizeof(double), s->stream));
    qs_status st = ok(cudaMallocAsync(&od, shots * sizeof(uint64_t), s->stream), "sample buffer");
    if (st == QS_OK)
        st = ok(cudaMemcpyAsync(ud, uniforms, shots * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                "uniforms copy");
    if (st == QS_OK) st = k_sample(s, member, ud, shots, od);
    if (st == QS_OK)
        st = ok(cudaMemcpyAsync(out, od, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream),
                "samples copy");
    if (st == QS_OK) st = ok(cudaStreamSynchronize(s->stream), "sample sync");
    cudaFreeAsync(ud, s->stream);
    if (od) cudaFreeAsync(od, s->stream);
    return st;
    QS_GUARD_END
}

qs_status qs_norm2(qs_state *s, double *out) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!out) {
        set_error("null output");
        return QS_ERR_ARG;
    }
    if (s->host) return host_norm2(s, out);
    QS_TRY(ensure_host_pinned(s, (size_t)s->batch));
    double *dev = nullptr;
    QS_TRY(k_norm2(s, &dev));
    QS_TRY(read_back(s, dev, s->host_pinned, s->batch));
    std::memcpy(out, s->host_pinned, sizeof(double) * s->batch);
    return QS_OK;
    QS_GUARD_END
}

static qs_status check_terms(const qs_state *s, const qs_pauli_term *t, size_t count) {
    if (count && !t) {
        set_error("null term array");
        return QS_ERR_ARG;
    }
    const int n = s->dm ? s->dm : s->n;
    for (size_t i = 0; i < count; ++i) {
        if (n < 64 && ((t[i].x_mask | t[i].z_mask) >> n) != 0) {
            set_error("term %zu names a qubit >= n", i);
            return QS_ERR_ARG;
        }
        if (!std::isfinite(t[i].coeff)) {
            set_error("term %zu has a non-finite coefficient", i);
            return QS_ERR_ARG;
        }
    }
    return QS_OK;
}

qs_status qs_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double *out_re, double *out_im) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!out_re) {
        set_error("null output");
        return QS_ERR_ARG;
    }
    QS_TRY(check_terms(s, terms, count));
    if (s->host) return host_expectation(s, terms, count, out_re, out_im);
    QS_TRY(ensure_host_pinned(s, (size_t)2 * s->batch));
    double *dev = nullptr;
    if (s->dm)
        QS_TRY(k_dm_expectation(s, terms, count, &dev));
    else
        QS_TRY(k_expectation(s, terms, count, &dev));
    QS_TRY(read_back(s, dev, s->host_pinned, 2 * (size_t)s->batch));
    for (int b = 0; b < s->batch; ++b) {
        out_re[b] = s->host_pinned[2 * b];
        if (out_im) out_im[b] = s->host_pinned[2 * b + 1];
    }
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_energy_gradient(qs_state *w, const qs_gate *gates, size_t count, const double *params_dev,
                             int n_params, const qs_pauli_term *terms, size_t n_terms, int init_zero,
                             double *energy_dev, double *grad_dev, int ckpt_every, int mode) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(w));
    QS_TRY(not_for_density(w, "the adjoint gradient"));
    if (w->n < 2) {
        set_error("the work handle needs n + 1 >= 2 qubits");
        return QS_ERR_ARG;
    }
    if (mode != QS_GRAD_FULL && mode != QS_GRAD_FORWARD && mode != QS_GRAD_SWEEP) {
        set_error("unknown mode %d", mode);
        return QS_ERR_ARG;
    }
    if (mode != QS_GRAD_SWEEP && !energy_dev) {
        set_error("null energy output");
        return QS_ERR_ARG;
    }
    if (mode != QS_GRAD_FORWARD && !grad_dev) {
        set_error("null gradient output");
        return QS_ERR_ARG;
    }
    if (mode == QS_GRAD_SWEEP && ckpt_every != 0) {
        set_error("checkpoints need the forward pass in the same call (mode QS_GRAD_FULL)");
        return QS_ERR_ARG;
    }
    if (ckpt_every < 0 || n_params < 0) {
        set_error("negative ckpt_every or n_params");
        return QS_ERR_ARG;
    }
    qs_state circ = *w;   // lowering view: n-qubit circuit
    circ.n = w->n - 1;
    QS_TRY(check_terms(&circ, terms, n_terms));
    std::vector<LGate> lg;
    QS_TRY(lower_all(&circ, gates, count, &lg));
    for (size_t i = 0; i < lg.size(); ++i) {
        const int p = lg[i].param_index;
        if (p < 0) continue;
        if (p >= n_params || !params_dev) {
            set_error("gate %zu: param_index %d outside [0, %d)", i, p, n_params);
            return QS_ERR_ARG;
        }
        const int kd = lg[i].kind;
        if (kd != QS_GATE_RX && kd != QS_GATE_RY && kd != QS_GATE_RZ && kd != QS_GATE_U1 && kd != QS_GATE_CU1) {
            set_error("gate %zu: parametrised gates must be RX RY RZ U1 CU1", i);
            return QS_ERR_ARG;
        }
    }
    return energy_gradient(w, lg, params_dev, n_params, terms, n_terms, init_zero, energy_dev, grad_dev,
                           ckpt_every, mode);
    QS_GUARD_END
}

qs_status qs_trotter_step(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                          size_t n_h1, double s_val, double dt) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "Trotter evolution"));
    QS_TRY(check_terms(s, h0, n_h0));
    QS_TRY(check_terms(s, h1, n_h1));
    if (!std::isfinite(s_val) || !std::isfinite(dt)) {
        set_error("non-finite s or dt");
        return QS_ERR_ARG;
    }
    return run_trotter(s, h0, n_h0, h1, n_h1, s_val, dt, 0.0, 1);
    QS_GUARD_END
}

qs_status qs_adiabatic_evolve(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                              size_t n_h1, double T, double dt, int steps) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "Trotter evolution"));
    QS_TRY(check_terms(s, h0, n_h0));
    QS_TRY(check_terms(s, h1, n_h1));
    if (!(T > 0) || !(dt > 0) || !std::isfinite(T) || !std::isfinite(dt)) {
        set_error("T and dt must be positive and finite");
        return QS_ERR_ARG;
    }
    const long K = std::lround(T / dt);
    if (K < 1 || K > (1l << 30)) {
        set_error("T/dt gives %ld steps", K);
        return QS_ERR_ARG;
    }
    const long run = steps < 0 ? K : std::min<long>(K, steps);
    if (run == 0) return QS_OK;
    return run_trotter(s, h0, n_h0, h1, n_h1, -1.0, dt, T, (int)run);
    QS_GUARD_END
}

qs_status qs_adiabatic_evolve_batch(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                                    const size_t *h1_counts, double T, double dt, int steps) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "Trotter evolution"));
    if (!h1_counts) {
        set_error("null h1_counts");
        return QS_ERR_ARG;
    }
    std::vector<size_t> off(s->batch + 1, 0);
    for (int b = 0; b < s->batch; ++b) off[b + 1] = off[b] + h1_counts[b];
    QS_TRY(check_terms(s, h0, n_h0));
    QS_TRY(check_terms(s, h1, off[s->batch]));
    if (!(T > 0) || !(dt > 0) || !std::isfinite(T) || !std::isfinite(dt)) {
        set_error("T and dt must be positive and finite");
        return QS_ERR_ARG;
    }
    const long K = std::lround(T / dt);
    if (K < 1 || K > (1l << 30)) {
        set_error("T/dt gives %ld steps", K);
        return QS_ERR_ARG;
    }
    const long run = steps < 0 ? K : std::min<long>(K, steps);
    if (run == 0) return QS_OK;
    return run_adiabatic_batch(s, h0, n_h0, h1, off.data(), dt, T, (int)run);
    QS_GUARD_END
}


qs_status qs_adiabatic_run_batch(qs_state *const *states, int n_states, const qs_pauli_term *h0,
                                 const size_t *h0_counts, const qs_pauli_term *h1, const size_t *h1_counts, double T,
                                 double dt, int steps) {
    QS_GUARD_BEGIN
    clear_error();
    if (n_states < 1 || !states || !h0_counts || !h1_counts) {
        set_error("need at least one state handle and the term counts");
        return QS_ERR_ARG;
    }
    std::vector<size_t> h0_off(n_states + 1, 0);
    std::vector<size_t> h1_off(1, 0);
    for (int i = 0; i < n_states; ++i) {
        qs_state *s = states[i];
        QS_TRY(check_state(s));
        QS_TRY(not_for_density(s, "Trotter evolution"));
        if (s->dtype != states[0]->dtype || s->device != states[0]->device) {
            set_error("handle %d: every handle needs the dtype and device of handle 0", i);
            return QS_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (states[j] == s || states[j]->data == s->data) {
                set_error("handles %d and %d share their amplitudes", j, i);
                return QS_ERR_ARG;
            }
        h0_off[i + 1] = h0_off[i] + h0_counts[i];
        QS_TRY(check_terms(s, h0 + h0_off[i], h0_counts[i]));
        for (int b = 0; b < s->batch; ++b) {
            const size_t m = h1_off.size() - 1;
            h1_off.push_back(h1_off[m] + h1_counts[m]);
            QS_TRY(check_terms(s, h1 + h1_off[m], h1_counts[m]));
        }
    }
    if ((h0_off[n_states] && !h0) || (h1_off.back() && !h1)) {
        set_error("null term array");
        return QS_ERR_ARG;
    }
    if (!(T > 0) || !(dt > 0) || !std::isfinite(T) || !std::isfinite(dt)) {
        set_error("T and dt must be positive and finite");
        return QS_ERR_ARG;
    }
    const long K = std::lround(T / dt);
    if (K < 1 || K > (1l << 30)) {
        set_error("T/dt gives %ld steps", K);
        return QS_ERR_ARG;
    }
    const long run = steps < 0 ? K : std::min<long>(K, steps);
    if (run == 0) return QS_OK;
    return run_adiabatic_multi(states, n_states, h0, h0_off.data(), h1, h1_off.data(), dt, T, (int)run, 10);
    QS_GUARD_END
}

qs_status qs_evolve(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1, size_t n_h1,
                    double T, double dt, int steps, int solver) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "time evolution"));
    QS_TRY(check_terms(s, h0, n_h0));
    QS_TRY(check_terms(s, h1, n_h1));
    if (solver != QS_SOLVER_EXP && solver != QS_SOLVER_RK4 && solver != QS_SOLVER_RK45) {
        set_error("unknown solver %d", solver);
        return QS_ERR_ARG;
    }
    if (!(T > 0) || !(dt > 0) || !std::isfinite(T) || !std::isfinite(dt)) {
        set_error("T and dt must be positive and finite");
        return QS_ERR_ARG;
    }
    const long K = std::lround(T / dt);
    if (K < 1 || K > (1l << 30)) {
        set_error("T/dt gives %ld steps", K);
        return QS_ERR_ARG;
    }
    const long run = steps < 0 ? K : std::min<long>(K, steps);
    if (run == 0) return QS_OK;
    return run_evolve(s, h0, n_h0, h1, n_h1, T, dt, (int)run, solver);
    QS_GUARD_END
}

qs_status qs_schedule_gradient(qs_state *s, const qs_pauli_term *h0, size_t n_h0, const qs_pauli_term *h1,
                               size_t n_h1, const double *svals, int K, double dt, double *energy, double *dE_ds,
                               double *dE_ddt) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    QS_TRY(not_for_density(s, "the schedule gradient"));
    QS_TRY(check_terms(s, h0, n_h0));
    QS_TRY(check_terms(s, h1, n_h1));
    if (K < 1 || !svals || !dE_ds || !dE_ddt) {
        set_error("need K >= 1 schedule values and the gradient outputs");
        return QS_ERR_ARG;
    }
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(svals[k])) {
            set_error("schedule value %d is not finite", k);
            return QS_ERR_ARG;
        }
    if (!(dt > 0) || !std::isfinite(dt)) {
        set_error("dt must be positive and finite");
        return QS_ERR_ARG;
    }
    return run_schedule_gradient(s, h0, n_h0, h1, n_h1, svals, K, dt, energy, dE_ds, dE_ddt);
    QS_GUARD_END
}

qs_status qs_density_init_pure(qs_state *s, const void *psi, int on_device) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!s->dm) {
        set_error("not a density matrix");
        return QS_ERR_ARG;
    }
    if (!psi) {
        set_error("null state");
        return QS_ERR_ARG;
    }
    if (on_device) return k_dm_init_pure(s, psi);
    const size_t bytes = ((size_t)s->batch << s->dm) * (s->dtype == QS_C64 ? 8 : 16);
    void *tmp = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&tmp, bytes, s->stream));
    qs_status st = QS_OK;
    const cudaError_t e = cudaMemcpyAsync(tmp, psi, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) st = cuda_status(e, "state copy");
    if (st == QS_OK) st = k_dm_init_pure(s, tmp);
    cudaFreeAsync(tmp, s->stream);
    if (st == QS_OK) QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return st;
    QS_GUARD_END
}

qs_status qs_density_trace(qs_state *s, double *out) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!s->dm || !out) {
        set_error(!out ? "null output" : "not a density matrix");
        return QS_ERR_ARG;
    }
    QS_TRY(ensure_host_pinned(s, (size_t)s->batch));
    double *dev = nullptr;
    QS_TRY(k_dm_trace(s, &dev));
    QS_TRY(read_back(s, dev, s->host_pinned, s->batch));
    std::memcpy(out, s->host_pinned, sizeof(double) * s->batch);
    return QS_OK;
    QS_GUARD_END
}

// The superoperator of a channel on the vector of rho: targets first on the
// row bits, then on the column bits; S[(r1, c1), (r2, c2)] = sum_i
// K_i[r1, r2] conj(K_i[c1, c2]).
static qs_status lower_channel(const qs_state *s, const qs_channel &ch, LGate *out) {
    const int dm = s->dm, k = ch.n_targets;
    if (k < 1 || k > 2) {
        set_error("a channel acts on 1 or 2 qubits (got %d)", k);
        return QS_ERR_ARG;
    }
    const int K = 1 << k;
    if (ch.n_kraus < 1 || ch.n_kraus > K * K || !ch.kraus) {
        set_error("a channel needs 1 to %d Kraus operators", K * K);
        return QS_ERR_ARG;
    }
    for (int j = 0; j < k; ++j)
        if (ch.targets[j] < 0 || ch.targets[j] >= dm || (j == 1 && ch.targets[1] == ch.targets[0])) {
            set_error("channel target %d out of range or repeated", ch.targets[j]);
            return QS_ERR_ARG;
        }
    std::vector<cd> kr((size_t)ch.n_kraus * K * K);
    for (size_t i = 0; i < kr.size(); ++i) {
        if (!std::isfinite(ch.kraus[2 * i]) || !std::isfinite(ch.kraus[2 * i + 1])) {
            set_error("non-finite Kraus entry");
            return QS_ERR_ARG;
        }
        kr[i] = cd(ch.kraus[2 * i], ch.kraus[2 * i + 1]);
    }
    for (int a = 0; a < K; ++a)  // sum_i K_i^dag K_i = I
        for (int b = 0; b < K; ++b) {
            cd acc = 0.0;
            for (int i = 0; i < ch.n_kraus; ++i)
                for (int r = 0; r < K; ++r)
                    acc += std::conj(kr[((size_t)i * K + r) * K + a]) * kr[((size_t)i * K + r) * K + b];
            if (std::abs(acc - cd(a == b ? 1.0 : 0.0)) > 1e-8) {
                set_error("Kraus operators are not trace preserving (sum K^dag K differs from I by %g)",
                          std::abs(acc - cd(a == b ? 1.0 : 0.0)));
                return QS_ERR_ARG;
            }
        }
    const int K2 = K * K;
    out->k = 2 * k;
    for (int j = 0; j < k; ++j) {
        out->tbit[j] = dm - 1 - ch.targets[j] + dm;  // row copy
        out->tbit[k + j] = dm - 1 - ch.targets[j];    // column copy
    }
    out->cmask = 0;
    out->kind = QS_GATE_UNITARY;
    out->param_index = -1;
    out->m.assign((size_t)K2 * K2, cd(0.0));
    for (int i = 0; i < ch.n_kraus; ++i) {
        const cd *Ki = &kr[(size_t)i * K * K];
        for (int r1 = 0; r1 < K; ++r1)
            for (int c1 = 0; c1 < K; ++c1)
                for (int r2 = 0; r2 < K; ++r2)
                    for (int c2 = 0; c2 < K; ++c2)
                        out->m[(size_t)(r1 * K + c1) * K2 + (r2 * K + c2)] += Ki[r1 * K + r2] * std::conj(Ki[c1 * K + c2]);
    }
    set_matrix_flags(out);
    out->is_swap = false;
    return QS_OK;
}

qs_status qs_apply_channels(qs_state *s, const qs_channel *channels, size_t count, const qs_opts *opts) {
    QS_GUARD_BEGIN
    clear_error();
    QS_TRY(check_state(s));
    if (!s->dm) {
        set_error("channels act on density matrices (qs_density_create)");
        return QS_ERR_ARG;
    }
    if (count && !channels) {
        set_error("null channel array");
        return QS_ERR_ARG;
    }
    int mode;
    QS_TRY(check_opts(s, opts, &mode));
    std::vector<LGate> lg(count);
    for (size_t i = 0; i < count; ++i) {
        const qs_status st = lower_channel(s, channels[i], &lg[i]);
        if (st != QS_OK) {
            char buf[512];
            std::snprintf(buf, sizeof(buf), "channel %zu: %s", i, qs_last_error());
            set_error("%s", buf);
            return st;
        }
    }
    return run_gates(s, lg, mode, opts, nullptr, 0);
    QS_GUARD_END
}

}  // extern "C"
