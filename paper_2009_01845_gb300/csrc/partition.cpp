// States larger than the GPU's memory: the amplitudes live in pinned host
// memory and pass through the device in groups (Sec. 2.5: a single device is
// reused for the pieces of a state that does not fit it; the paper's 33/34
// qubits on one 32 GB GPU with host memory, Sec. 3.1).
//
// The device holds two buffers of M = 2^m amplitudes (within the handle's
// device budget). The index bits split into L low "chunk" bits (chunks of 2^L
// contiguous amplitudes) and n - L high bits. A segment is a run of gates (in
// queue order) whose dense targets lie in the chunk bits and a set S of at most
// m - L high bits; its groups fix the other high bits F to one value each, and
// a group is the 2^|S| chunks that differ in the S bits, copied into a buffer
// (one copy per chunk) where S becomes buffer bits L .. L + |S| - 1. Every gate
// is rewritten for the group: controls on F bits are resolved (the gate is
// dropped or the control removed), diagonal factors on F bits are fixed
// (the diagonal restricted to the group's values, a scalar where nothing
// remains), and the group runs on the ordinary gate kernels (tiled or
// unfused) as a state of L + |S| qubits. Groups alternate between the two
// buffers, each on a stream of its own, so one group's copies overlap the
// other's kernels; consecutive segments are ordered by events. Read-outs
// (squared norm, probabilities, Pauli sums whose X bits lie in the low m bits)
// stream blocks of M contiguous amplitudes the same way.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "prof.h"

namespace qsim {

namespace {

size_t abytes(qs_dtype d) { return d == QS_C64 ? 8 : 16; }

// fill [0, count) amplitudes of host memory with (re, 0) or a single basis
// amplitude, on several threads
void host_fill(qs_state *s, double re, uint64_t one) {
    const uint64_t total = 1ull << s->n;
    const size_t b = abytes(s->dtype);
    const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([=]() {
            const uint64_t lo = total * t / nt, hi = total * (t + 1) / nt;
            char *base = (char *)s->host;
            if (s->dtype == QS_C64) {
                float2 *p = (float2 *)base;
                for (uint64_t i = lo; i < hi; ++i) p[i] = make_float2((float)re, 0.f);
            } else {
                double2 *p = (double2 *)base;
                for (uint64_t i = lo; i < hi; ++i) p[i] = make_double2(re, 0.0);
            }
            (void)b;
        });
    for (auto &x : th) x.join();
    if (one != ~0ull) {
        if (s->dtype == QS_C64)
            ((float2 *)s->host)[one] = make_float2(1.f, 0.f);
        else
            ((double2 *)s->host)[one] = make_double2(1.0, 0.0);
    }
}

// A view handle on device buffer `data` of nv qubits that shares nothing with s
// but its dtype and stream.
qs_state view_of(const qs_state *s, void *data, int nv, cudaStream_t st) {
    qs_state v;
    v.n = nv;
    v.ms = nv;
    v.batch = 1;
    v.dtype = s->dtype;
    v.data = data;
    v.owns = false;
    v.stream = st;
    v.device = s->device;
    return v;
}

void release_view(qs_state *v) {
    if (v->scratch) cudaFree(v->scratch);
    if (v->host_pinned) cudaFreeHost(v->host_pinned);
    if (v->gtab) cudaFree(v->gtab);
    if (v->ptab) cudaFree(v->ptab);
    if (v->itab) cudaFree(v->itab);
    if (v->ithr) cudaFree(v->ithr);
    v->scratch = nullptr;
    v->host_pinned = nullptr;
    v->gtab = v->ptab = nullptr;
    v->itab = v->ithr = nullptr;
}

// the gate rewritten for one group: bit b of the full index maps to
// vbit[b] >= 0 in the buffer, or to the fixed value (fixed >> b) & 1 when
// vbit[b] < 0. Returns false when the gate does nothing on this group.
bool specialise(const LGate &g, const int *vbit, uint64_t fixed, LGate *out) {
    *out = g;
    out->cmask = 0;
    for (int b = 0; b < 64; ++b) {
        if (!((g.cmask >> b) & 1ull)) continue;
        if (vbit[b] < 0) {
            if (!((fixed >> b) & 1ull)) return false;  // a control is 0 on this group
        } else {
            out->cmask |= 1ull << vbit[b];
        }
    }
    int keep[QS_MAX_TARGETS], nk = 0, fixed_local = 0;
    for (int j = 0; j < g.k; ++j) {
        const int t = g.tbit[j];
        if (vbit[t] >= 0) {
            keep[nk++] = j;
        } else if ((fixed >> t) & 1ull) {
            fixed_local |= 1 << (g.k - 1 - j);
        }
    }
    if (nk == g.k) {
        for (int j = 0; j < g.k; ++j) out->tbit[j] = vbit[g.tbit[j]];
        return true;
    }
    // a diagonal with targets on fixed bits (the planner keeps dense targets
    // resident): its entries on the group's values
    const int K = 1 << g.k, Kn = 1 << nk;
    std::vector<cd> m((size_t)std::max(Kn, 2) * std::max(Kn, 2), cd(0.0));
    for (int l = 0; l < Kn; ++l) {
        int full = fixed_local;
        for (int i = 0; i < nk; ++i)
            if ((l >> (nk - 1 - i)) & 1) full |= 1 << (g.k - 1 - keep[i]);
        m[(size_t)l * Kn + l] = g.m[(size_t)full * K + full];
    }
    if (nk == 0) {  // a scalar on the whole group: diag(d, d) on buffer bit 0
        const cd d = m[0];
        if (d == cd(1.0)) return false;
        out->k = 1;
        out->tbit[0] = 0;
        out->m = {d, cd(0.0), cd(0.0), d};
    } else {
        out->k = nk;
        for (int i = 0; i < nk; ++i) out->tbit[i] = vbit[g.tbit[keep[i]]];
        out->m = m;
    }
    out->kind = QS_GATE_UNITARY;
    set_matrix_flags(out);
    out->is_swap = false;
    return true;
}

uint64_t dense_bits(const LGate &g) {
    if (g.diagonal) return 0;
    uint64_t m = 0;
    for (int j = 0; j < g.k; ++j) m |= 1ull << g.tbit[j];
    return m;
}

struct Pipe {
    qs_state *s;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    void *buf[2] = {nullptr, nullptr};
    ~Pipe() {
        for (int i = 0; i < 2; ++i) {
            if (st[i]) cudaStreamDestroy(st[i]);
            if (ev[i]) cudaEventDestroy(ev[i]);
        }
    }
    qs_status init() {
        for (int i = 0; i < 2; ++i) {
            QS_CUDA_TRY(cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking));
            QS_CUDA_TRY(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
            buf[i] = s->pbuf[i];
        }
        // after the handle's earlier work on its own stream
        QS_CUDA_TRY(cudaEventRecord(ev[0], s->stream));
        for (int i = 0; i < 2; ++i) QS_CUDA_TRY(cudaStreamWaitEvent(st[i], ev[0], 0));
        return QS_OK;
    }
    // both streams wait for each other (a segment boundary)
    qs_status barrier() {
        for (int i = 0; i < 2; ++i) QS_CUDA_TRY(cudaEventRecord(ev[i], st[i]));
        QS_CUDA_TRY(cudaStreamWaitEvent(st[0], ev[1], 0));
        QS_CUDA_TRY(cudaStreamWaitEvent(st[1], ev[0], 0));
        return QS_OK;
    }
    // the handle's stream waits for both (the call's end)
    qs_status join() {
        for (int i = 0; i < 2; ++i) {
            QS_CUDA_TRY(cudaEventRecord(ev[i], st[i]));
            QS_CUDA_TRY(cudaStreamWaitEvent(s->stream, ev[i], 0));
        }
        return QS_OK;
    }
};

}  // namespace

qs_status host_state_buffers(qs_state *s) {
    if (s->pbuf[0]) return QS_OK;
    const size_t bytes = ((size_t)1 << s->pm) * abytes(s->dtype);
    for (int i = 0; i < 2; ++i) QS_CUDA_TRY(cudaMalloc(&s->pbuf[i], bytes));
    return QS_OK;
}

qs_status host_init(qs_state *s, bool plus, uint64_t x) {
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));  // earlier copies of the state have finished
    if (plus)
        host_fill(s, std::pow(2.0, -0.5 * s->n), ~0ull);
    else
        host_fill(s, 0.0, x);
    return QS_OK;
}

qs_status host_apply(qs_state *s, const std::vector<LGate> &G, int mode, const qs_opts *opts) {
    QS_TRY(host_state_buffers(s));
    const int n = s->n, m = s->pm;
    const int L = s->pl;            // chunk bits
    const int smax = std::min(m - L, n - L);
    const size_t b = abytes(s->dtype);
    Pipe p;
    p.s = s;
    QS_TRY(p.init());
    qs_state views[2] = {view_of(s, p.buf[0], L + smax, p.st[0]), view_of(s, p.buf[1], L + smax, p.st[1])};
    qs_status st = QS_OK;
    size_t pos = 0;
    while (pos < G.size() && st == QS_OK) {
        // the segment: gates in order while their dense high bits fit S
        uint64_t S = 0;
        size_t end = pos;
        for (; end < G.size(); ++end) {
            const uint64_t need = dense_bits(G[end]) & ~((1ull << L) - 1ull);
            if (__builtin_popcountll(S | need) > smax) break;
            S |= need;
        }
        if (end == pos) {
            set_error("gate %zu has more dense targets above the chunk bits than a group holds (%d)", pos, smax);
            st = QS_ERR_UNSUPPORTED;
            break;
        }
        for (int bit = L; bit < n && __builtin_popcountll(S) < smax; ++bit) S |= 1ull << bit;
        int sb[64], ns = 0, fb[64], nf = 0;
        for (int bit = L; bit < n; ++bit) {
            if ((S >> bit) & 1ull) sb[ns++] = bit;
            else fb[nf++] = bit;
        }
        int vbit[64];
        for (int bit = 0; bit < 64; ++bit) vbit[bit] = -1;
        for (int bit = 0; bit < L; ++bit) vbit[bit] = bit;
        for (int j = 0; j < ns; ++j) vbit[sb[j]] = L + j;
        const uint64_t groups = 1ull << nf;
        const size_t chunk_bytes = ((size_t)1 << L) * b;
        for (uint64_t gi = 0; gi < groups && st == QS_OK; ++gi) {
            const int w = (int)(gi & 1);
            qs_state &v = views[w];
            uint64_t fixed = 0;
            for (int j = 0; j < nf; ++j)
                if ((gi >> j) & 1ull) fixed |= 1ull << fb[j];
            std::vector<LGate> spec;
            for (size_t i = pos; i < end; ++i) {
                LGate o;
                if (specialise(G[i], vbit, fixed, &o)) spec.push_back(std::move(o));
            }
            auto chunk_base = [&](uint64_t c) {
                uint64_t base = fixed;
                for (int j = 0; j < ns; ++j)
                    if ((c >> j) & 1ull) base |= 1ull << sb[j];
                return base;
            };
            {
                ProfScope _ps(p.st[w], KC_HOSTCOPY, (double)chunk_bytes * (1ull << ns));
                for (uint64_t c = 0; c < (1ull << ns) && st == QS_OK; ++c) {
                    const cudaError_t e = cudaMemcpyAsync((char *)p.buf[w] + c * chunk_bytes,
                                                          (char *)s->host + chunk_base(c) * b, chunk_bytes,
                                                          cudaMemcpyHostToDevice, p.st[w]);
                    if (e != cudaSuccess) st = cuda_status(e, "chunk upload");
                }
            }
            if (st == QS_OK && !spec.empty()) st = run_gates(&v, spec, mode, opts, nullptr, 0);
            {
                ProfScope _ps(p.st[w], KC_HOSTCOPY, (double)chunk_bytes * (1ull << ns));
                for (uint64_t c = 0; c < (1ull << ns) && st == QS_OK; ++c) {
                    const cudaError_t e = cudaMemcpyAsync((char *)s->host + chunk_base(c) * b,
                                                          (char *)p.buf[w] + c * chunk_bytes, chunk_bytes,
                                                          cudaMemcpyDeviceToHost, p.st[w]);
                    if (e != cudaSuccess) st = cuda_status(e, "chunk download");
                }
            }
        }
        if (st == QS_OK) st = p.barrier();
        pos = end;
    }
    if (st == QS_OK) st = p.join();
    // the views' scratch buffers are freed after their streams' work
    for (auto &v : views) {
        cudaStreamSynchronize(v.stream);
        release_view(&v);
    }
    return st;
}

// Blocks of M contiguous amplitudes through the device, one reduction each;
// `per_block` launches on the view and returns a device pointer to `outn`
// doubles that are copied to host_out + block * outn.
template <typename F>
static qs_status stream_blocks(qs_state *s, size_t outn, double *host_out, F per_block) {
    QS_TRY(host_state_buffers(s));
    const int n = s->n, m = std::min(s->pm, s->n);
    const size_t b = abytes(s->dtype);
    const uint64_t blocks = 1ull << (n - m);
    const size_t block_bytes = ((size_t)1 << m) * b;
    Pipe p;
    p.s = s;
    QS_TRY(p.init());
    qs_state views[2] = {view_of(s, p.buf[0], m, p.st[0]), view_of(s, p.buf[1], m, p.st[1])};
    qs_status st = QS_OK;
    for (uint64_t blk = 0; blk < blocks && st == QS_OK; ++blk) {
        const int w = (int)(blk & 1);
        cudaError_t e = cudaMemcpyAsync(p.buf[w], (char *)s->host + blk * block_bytes, block_bytes,
                                        cudaMemcpyHostToDevice, p.st[w]);
        if (e != cudaSuccess) {
            st = cuda_status(e, "block upload");
            break;
        }
        const double *dev = nullptr;
        st = per_block(&views[w], blk, &dev);
        if (st != QS_OK) break;
        e = cudaMemcpyAsync(host_out + blk * outn, dev, outn * sizeof(double), cudaMemcpyDeviceToHost, p.st[w]);
        if (e != cudaSuccess) st = cuda_status(e, "block result");
        // the next use of this view's scratch must wait for the copy: same stream
    }
    if (st == QS_OK) st = p.join();
    for (auto &v : views) {
        cudaStreamSynchronize(v.stream);
        release_view(&v);
    }
    if (st == QS_OK) QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return st;
}

qs_status host_norm2(qs_state *s, double *out) {
    const uint64_t blocks = 1ull << (s->n - std::min(s->pm, s->n));
    double *part = nullptr;
    QS_CUDA_TRY(cudaMallocHost(&part, blocks * sizeof(double)));
    const qs_status st = stream_blocks(s, 1, part, [&](qs_state *v, uint64_t, const double **dev) {
        double *d = nullptr;
        QS_TRY(k_norm2(v, &d));
        *dev = d;
        return QS_OK;
    });
    double sum = 0.0;
    for (uint64_t i = 0; i < blocks && st == QS_OK; ++i) sum += part[i];
    cudaFreeHost(part);
    if (st == QS_OK) *out = sum;
    return st;
}

qs_status host_probabilities(qs_state *s, double *out) {
    const int m = std::min(s->pm, s->n);
    double *dp = nullptr;
    QS_CUDA_TRY(cudaMalloc(&dp, 2 * ((size_t)1 << m) * sizeof(double)));
    const qs_status st = stream_blocks(s, (size_t)1 << m, out, [&](qs_state *v, uint64_t blk, const double **dev) {
        double *d = dp + (blk & 1) * ((size_t)1 << m);
        QS_TRY(k_probabilities(v, d));
        *dev = d;
        return QS_OK;
    });
    cudaFree(dp);
    return st;
}

qs_status host_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double *re, double *im) {
    const int n = s->n, m = std::min(s->pm, s->n);
    const uint64_t blocks = 1ull << (n - m);
    // terms in the block's qubits (the low m index bits are qubits n-m .. n-1);
    // Z bits above them are a sign per block
    std::vector<qs_pauli_term> low(count);
    std::vector<uint64_t> zhigh(count);
    for (size_t i = 0; i < count; ++i) {
        uint64_t xh = 0;
        zhigh[i] = 0;
        for (int q = 0; q < n - m; ++q) {
            if ((terms[i].x_mask >> q) & 1ull) xh |= 1ull << q;
            if ((terms[i].z_mask >> q) & 1ull) zhigh[i] |= 1ull << (n - 1 - q);
        }
        if (xh) {
            set_error("term %zu flips a qubit above the device block (qubits 0..%d): not supported on a "
                      "host-memory state", i, n - m - 1);
            return QS_ERR_UNSUPPORTED;
        }
        low[i].coeff = terms[i].coeff;
        low[i].x_mask = terms[i].x_mask >> (n - m);
        low[i].z_mask = terms[i].z_mask >> (n - m);
    }
    double *part = nullptr;
    QS_CUDA_TRY(cudaMallocHost(&part, 2 * blocks * sizeof(double)));
    std::vector<qs_pauli_term> t(count);
    const qs_status st = stream_blocks(s, 2, part, [&](qs_state *v, uint64_t blk, const double **dev) {
        const uint64_t hi = blk << m;  // the block's high index bits
        for (size_t i = 0; i < count; ++i) {
            t[i] = low[i];
            if (__builtin_popcountll(hi & zhigh[i]) & 1) t[i].coeff = -t[i].coeff;
        }
        double *d = nullptr;
        QS_TRY(k_expectation(v, t.data(), t.size(), &d));
        *dev = d;
        return QS_OK;
    });
    double sr = 0.0, si = 0.0;
    for (uint64_t i = 0; i < blocks && st == QS_OK; ++i) {
        sr += part[2 * i];
        si += part[2 * i + 1];
    }
    cudaFreeHost(part);
    if (st == QS_OK) {
        *re = sr;
        if (im) *im = si;
    }
    return st;
}

}  // namespace qsim
