// Test infrastructure: a host emulator of the tiled-pass descriptors.
//
// It links the library's planner (plan_tiled.cpp) and gate lowering
// (gates_host.cpp) and replaces every device launch they make with a host
// routine: a tiled pass is interpreted op by op on each tile of a host state,
// with the kernel's semantics (tiled.h, kernels_tiled.cu) written out on the
// tile's local indices; gates the planner sends to unfused passes are applied
// as dense matrices. The test-suite compares the results with the oracle, so
// planner logic (pass selection, stages, factor placement, commutation rules,
// the adjoint sweep's gradient ops, the register frame) is checked without a
// GPU. Nothing here is part of the library. Each stage's registers are held per
// thread as the kernel holds them: filled from the tile's local indices when
// the stage opens, changed by the ops in place, and written back (through the
// stage's register frame) when it ends; shared-memory positions and swizzles
// are not emulated.
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "tiled.h"

using namespace qsim;

// ------------------------------------------------------------------ CUDA runtime stand-ins
// (the planner only allocates its small tables and waits on the stream)
extern "C" {
cudaError_t cudaMalloc(void **p, size_t bytes) {
    *p = std::malloc(bytes ? bytes : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p) {
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char *cudaGetErrorString(cudaError_t) { return "emulated"; }
}

namespace qsim {
bool prof_enabled() { return false; }
void prof_add_work(int, double, double) {}
const char *last_error();
}  // namespace qsim

using cdd = std::complex<double>;

static std::vector<double> *g_gpart = nullptr;  // gradient partials of the adjoint sweep

// a dense 2^k x 2^k gate with controls on a host state (batch members of size 2^ms)
static void apply_dense(cdd *psi, int n, int ms, int batch, const LGate &g) {
    const int K = 1 << g.k;
    std::vector<cdd> in(K), out(K);
    for (int b = 0; b < batch; ++b)
        for (uint64_t x = 0; x < (1ull << n); ++x) {
            bool base = (x & g.cmask) == g.cmask;
            for (int j = 0; j < g.k && base; ++j) base = !((x >> g.tbit[j]) & 1ull);
            if (!base) continue;
            auto idx = [&](int l) {
                uint64_t y = x;
                for (int j = 0; j < g.k; ++j)
                    if ((l >> (g.k - 1 - j)) & 1) y |= 1ull << g.tbit[j];
                return ((uint64_t)b << ms) | y;
            };
            for (int c = 0; c < K; ++c) in[c] = psi[idx(c)];
            for (int r = 0; r < K; ++r) {
                cdd acc = 0.0;
                for (int c = 0; c < K; ++c) acc += g.m[r * K + c] * in[c];
                out[r] = acc;
            }
            for (int r = 0; r < K; ++r) psi[idx(r)] = out[r];
        }
}

namespace qsim {
qs_status k_apply_unfused(qs_state *s, const LGate &g) {
    apply_dense((cdd *)s->data, s->n, s->ms, s->batch, g);
    return QS_OK;
}
qs_status k_apply_param_gate(qs_state *, const LGate &, const double *, int, double) {
    set_error("batched parameters are not emulated");
    return QS_ERR_UNSUPPORTED;
}
qs_status k_param_table(qs_state *, const std::vector<int> &, const std::vector<int> &, const double *, int, double,
                        uint32_t *, bool) {
    set_error("batched parameters are not emulated");
    return QS_ERR_UNSUPPORTED;
}
bool c128_fp64() { return false; }
qs_status k_ising_table(qs_state *, const IsingTabP &) { return QS_OK; }
}  // namespace qsim

template <typename R> static cdd C(const V<R> &v) { return cdd((double)v.x, (double)v.y); }

// one tiled pass on a host state (complex128 storage whatever R is)
template <typename R> static qs_status emulate_pass(qs_state *s, const TileParams<R> &p) {
    constexpr int RB = TileCfg<R>::RB, WB = TileCfg<R>::WB, NR = 1 << RB;
    cdd *psi = (cdd *)s->data;
    const int k = p.k;
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    std::vector<cdd> A(1ull << k);
    for (uint64_t t = 0; t < p.total_tiles; ++t) {
        uint64_t g = t & fmask, tbase = 0;
        {  // expand the free bits around the tile bits (ascending positions)
            uint64_t v = g;
            for (int i = 0; i < p.tins.count; ++i) {
                const int pos = p.tins.pos[i];
                const uint64_t lo = v & ((1ull << pos) - 1ull);
                v = ((v >> pos) << (pos + 1)) | lo;
            }
            tbase = ((t >> p.n_free) << p.n) | v;
        }
        auto gidx = [&](uint32_t li) {
            uint64_t x = tbase;
            for (int i = 0; i < k; ++i)
                if ((li >> i) & 1u) x |= 1ull << p.gbit[i];
            return x;
        };
        for (uint32_t li = 0; li < (1u << k); ++li) A[li] = psi[gidx(li)];
        for (int si = 0; si < p.n_stages; ++si) {
            const TileStage &st = p.st[si];
            auto local_of = [&](uint32_t thread, int r) {  // thread = lane | warp << 5
                uint32_t li = 0;
                for (int i = 0; i < kTileLaneBits; ++i)
                    if ((thread >> i) & 1u) li |= 1u << st.lloc[i];
                for (int w = 0; w < WB; ++w)
                    if ((thread >> (kTileLaneBits + w)) & 1u) li |= 1u << st.wloc[w];
                for (int j = 0; j < RB; ++j)
                    if ((r >> j) & 1) li |= 1u << st.rloc[j];
                return li;
            };
            const uint32_t nthreads = 32u << WB;
            std::vector<cdd> REG((size_t)nthreads * NR);
            for (uint32_t th = 0; th < nthreads; ++th)
                for (int r = 0; r < NR; ++r) REG[(size_t)th * NR + r] = A[local_of(th, r)];
            for (int o = st.op_begin; o < st.op_end; ++o) {
                const TileOp &op = p.op[o];
                const V<R> *M = &p.mat[op.m];
                for (uint32_t th = 0; th < nthreads; ++th) {
                    const uint32_t lt = local_of(th, 0);
                    const bool ok = ((tbase & op.mo) == op.mo) && ((lt & op.mt) == op.mt);
                    cdd *a[NR];
                    for (int r = 0; r < NR; ++r) a[r] = &REG[(size_t)th * NR + r];
                    const uint32_t mr = op.mr;
                    switch (op.type) {
                    case TOP_DENSE1_R:
                        if (!ok) break;
                        for (int r = 0; r < NR; ++r) {
                            if ((r >> op.a) & 1 || (r & mr) != mr) continue;
                            const cdd x = *a[r], y = *a[r | (1 << op.a)];
                            *a[r] = C<R>(M[0]) * x + C<R>(M[1]) * y;
                            *a[r | (1 << op.a)] = C<R>(M[2]) * x + C<R>(M[3]) * y;
                        }
                        break;
                    case TOP_PHASE:
                        if (!ok) break;
                        for (int r = 0; r < NR; ++r)
                            if ((r & mr) == mr) *a[r] *= C<R>(M[0]);
                        break;
                    case TOP_DIAG1:
                        if (!ok) break;
                        for (int r = 0; r < NR; ++r) {
                            if ((r & mr) != mr) continue;
                            bool bit;
                            if (op.tkind == TB_REG) bit = (r >> op.a) & 1;
                            else if (op.tkind == TB_THREAD) bit = (lt & (uint32_t)op.tmask) != 0;
                            else bit = (tbase & op.tmask) != 0;
                            *a[r] *= bit ? C<R>(M[1]) : C<R>(M[0]);
                        }
                        break;
                    case TOP_DENSE2_RR:
                        if (!ok) break;
                        for (int r = 0; r < NR; ++r) {
                            if (r & ((1 << op.a) | (1 << op.b)) || (r & mr) != mr) continue;
                            const int i[4] = {r, r | (1 << op.b), r | (1 << op.a), r | (1 << op.a) | (1 << op.b)};
                            cdd x[4];
                            for (int c = 0; c < 4; ++c) x[c] = *a[i[c]];
                            for (int q = 0; q < 4; ++q) {
                                cdd acc = 0.0;
                                for (int c = 0; c < 4; ++c) acc += C<R>(M[q * 4 + c]) * x[c];
                                *a[i[q]] = acc;
                            }
                        }
                        break;
                    case TOP_SWAP_RR:
                        if (!ok) break;
                        for (int r = 0; r < NR; ++r) {
                            if (!((r >> op.a) & 1) || ((r >> op.b) & 1) || (r & mr) != mr) continue;
                            std::swap(*a[r], *a[r ^ (1 << op.a) ^ (1 << op.b)]);
                        }
                        break;
                    case TOP_ROTS_R:
                        // in-place shears x += s1 y, y += s2 x
                        for (int j = 0; j < RB; ++j) {
                            if (!((op.a >> j) & 1)) continue;
                            const double s1 = (double)M[j].x, s2 = (double)M[j].y;
                            for (int r = 0; r < NR; ++r) {
                                if ((r >> j) & 1) continue;
                                cdd &x = *a[r], &y = *a[r | (1 << j)];
                                x += s1 * y;
                                y += s2 * x;
                            }
                        }
                        break;
                    case TOP_FLIP: {
                        // bits a and b equal to 1 in the frame's terms (tkind: frame on a, b)
                        if (!ok) break;
                        const int va = 1 - (op.tkind & 1), vb = 1 - ((op.tkind >> 1) & 1);
                        for (int r = 0; r < NR; ++r)
                            if (((r >> op.a) & 1) == va && ((r >> op.b) & 1) == vb && ((r ^ op.fx) & mr) == mr)
                                *a[r] = -*a[r];
                        break;
                    }
                    case TOP_DBLOCK: {
                        const int f0 = (int)op.mo, nf = op.b, np = op.a, no = op.gl, ns = op.tkind;
                        cdd base = C<R>(M[0]);
                        cdd u[RB];
                        for (int j = 0; j < RB; ++j) u[j] = C<R>(M[1 + j]);
                        for (int f = f0; f < f0 + no; ++f) {  // outside-only factors
                            const TileDFac<R> &d = p.dfac[f];
                            if (d.type == DF_BIT) base *= (tbase & d.tmask) ? C<R>(d.v1) : C<R>(d.v0);
                            else if ((tbase & d.mo) == d.mo) base *= C<R>(d.v0);
                        }
                        uint32_t neg = 0;
                        for (int f = f0 + no; f < f0 + no + ns; ++f) {
                            const TileDFac<R> &d = p.dfac[f];
                            if ((tbase & d.mo) == d.mo && (lt & d.mt) == d.mt) neg ^= d.a;
                        }
                        if (neg & 0x80u) base = -base;
                        for (int j = 0; j < RB; ++j)
                            if ((neg >> j) & 1u) u[j] = -u[j];
                        for (int f = f0 + no + ns; f < f0 + nf - np; ++f) {
                            const TileDFac<R> &d = p.dfac[f];
                            if (d.type == DF_BIT) {
                                base *= (lt & (uint32_t)d.tmask) ? C<R>(d.v1) : C<R>(d.v0);
                                continue;
                            }
                            if ((tbase & d.mo) != d.mo || (lt & d.mt) != d.mt) continue;
                            if (d.mr == 0) {
                                base *= C<R>(d.v0);
                            } else {
                                for (int j = 0; j < RB; ++j)
                                    if (d.mr == (1u << j)) u[j] *= C<R>(d.v0);
                            }
                        }
                        for (int r = 0; r < NR; ++r) {
                            cdd ph = base;
                            for (int j = 0; j < RB; ++j)
                                if ((r >> j) & 1) ph *= u[j];
                            *a[r] *= ph;
                        }
                        for (int f = f0 + nf - np; f < f0 + nf; ++f) {
                            const TileDFac<R> &d = p.dfac[f];
                            if ((tbase & d.mo) != d.mo || (lt & d.mt) != d.mt) continue;
                            for (int r = 0; r < NR; ++r)
                                if ((d.tmask >> r) & 1ull) *a[r] *= C<R>(d.v0);
                        }
                        break;
                    }
                    case TOP_GRAD: {
                        // phi in registers r < NR/2, lambda in r + NR/2 (top register bit)
                        if (!ok || !g_gpart) break;
                        constexpr int H = NR / 2;
                        double acc = 0.0;
                        for (int r = 0; r < H; ++r) {
                            if ((r & mr) != mr) continue;
                            const cdd la = *a[r + H];
                            cdd ph;
                            if (op.b == GEN_X || op.b == GEN_Y) {
                                if (op.tkind == TB_REG) {
                                    ph = *a[r ^ (1 << op.a)];
                                    const cdd v = std::conj(la) * ph;
                                    acc += op.b == GEN_X ? v.imag() : (((r >> op.a) & 1) ? v.real() : -v.real());
                                } else {
                                    // target on lane bit op.a: the partner is the lane's neighbour
                                    const uint32_t partner = th ^ (1u << op.a);
                                    ph = REG[(size_t)partner * NR + r];
                                    const cdd v = std::conj(la) * ph;
                                    const int bit = (th >> op.a) & 1;
                                    acc += op.b == GEN_X ? v.imag() : (bit ? v.real() : -v.real());
                                }
                            } else {
                                const cdd v = std::conj(la) * *a[r];
                                bool neg = false;
                                if (op.b == GEN_Z) {
                                    if (op.tkind == TB_REG) neg = (r >> op.a) & 1;
                                    else if (op.tkind == TB_THREAD) neg = (lt & (uint32_t)op.tmask) != 0;
                                    else neg = (tbase & op.tmask) != 0;
                                }
                                acc += neg ? -v.imag() : v.imag();
                            }
                        }
                        (*g_gpart)[(size_t)p.gslot[op.gl] * p.total_tiles + t] += acc;
                        break;
                    }
                    case TOP_ISING: {
                        // psi_x *= exp(-i tau E(x)), E from the member's table (host memory here)
                        double tau;
                        std::memcpy(&tau, &op.tmask, sizeof(double));
                        const int nq = p.nq;
                        const double *J = p.ising + (t >> p.n_free) * p.ising_stride;
                        const double *hv = J + (size_t)nq * nq;
                        for (int r = 0; r < NR; ++r) {
                            const uint64_t x = gidx(local_of(th, r));
                            double e = hv[nq];
                            for (int b = 0; b < nq; ++b) {
                                const double zb = ((x >> b) & 1ull) ? -1.0 : 1.0;
                                e += hv[b] * zb;
                                for (int c = b + 1; c < nq; ++c) e += J[b * nq + c] * zb * (((x >> c) & 1ull) ? -1.0 : 1.0);
                            }
                            *a[r] *= std::polar(1.0, -tau * e);
                        }
                        break;
                    }
                    default:
                        set_error("op type %d is not emulated", (int)op.type);
                        return QS_ERR_UNSUPPORTED;
                    }
                }
            }
            // the transpose (or the store) writes register r where r ^ rflip belongs
            for (uint32_t th = 0; th < nthreads; ++th)
                for (int r = 0; r < NR; ++r) A[local_of(th, r ^ st.rflip)] = REG[(size_t)th * NR + r];
        }
        for (uint32_t li = 0; li < (1u << k); ++li) psi[gidx(li)] = A[li];
    }
    return QS_OK;
}

namespace qsim {
static int g_passes = 0;  // tiled passes emulated
qs_status k_tiled_pass_c64(qs_state *s, const TileParams<float> &p) {
    ++g_passes;
    return emulate_pass<float>(s, p);
}
qs_status k_tiled_pass_c128(qs_state *s, const TileParams<double> &p) {
    ++g_passes;
    return emulate_pass<double>(s, p);
}
}  // namespace qsim

static int g_calls = 0;

extern "C" {

int emu_apply_flags(int n, int dtype, const qs_gate *gates, int count, double *psi, int flags);

// psi (complex128, 2^n) <- circuit(psi) through the planner's tiled passes,
// planned for complex64 (dtype 0) or complex128 (dtype 1) descriptors
int emu_apply(int n, int dtype, const qs_gate *gates, int count, double *psi) {
    return emu_apply_flags(n, dtype, gates, count, psi, 0);
}

// the same with RY gates marked for three in-place shears (flags & 1), as the
// Trotter queue marks its layers
int emu_apply_flags(int n, int dtype, const qs_gate *gates, int count, double *psi, int flags) {
    qs_state s;
    s.n = n;
    s.ms = n;
    s.batch = 1;
    s.dtype = (qs_dtype)dtype;
    s.data = psi;
    std::vector<LGate> G(count);
    for (int i = 0; i < count; ++i) {
        if (lower_gate(n, gates[i], &G[i]) != QS_OK) return -1;
        G[i].paeth = (flags & 1) && gates[i].kind == QS_GATE_RY;
    }
    ++g_calls;
    return (int)run_tiled(&s, G, nullptr, 0);
}

// the same under a pass schedule of the planner (the autotuner's variants);
// *passes receives the number of tiled passes it ran
int emu_apply_schedule(int n, int dtype, const qs_gate *gates, int count, double *psi, int select, int max_gates,
                       int *passes) {
    const TileSchedule saved = tile_schedule();
    set_tile_schedule(TileSchedule{select, max_gates});
    const int p0 = g_passes;
    const int st = emu_apply_flags(n, dtype, gates, count, psi, 0);
    *passes = g_passes - p0;
    set_tile_schedule(saved);
    return st;
}

// The adjoint reverse sweep as the library's driver builds it, over a
// (phi, lambda) buffer of 2^(n+1) amplitudes (phi first): for each gate from
// the last, a gradient op (generator of a rotation) before the inverse gate.
// grad[j] receives Im <lambda|P_j|phi> (times -2 for phase gates) for every
// gate j with param_index >= 0 (the gates carry their angles; no batch table).
int emu_sweep(int n, int dtype, const qs_gate *gates, int count, double *buf, double *grad) {
    std::vector<LGate> G(count);
    for (int i = 0; i < count; ++i)
        if (lower_gate(n, gates[i], &G[i]) != QS_OK) return -1;
    std::vector<LGate> rev;
    std::vector<int> slot_gate;
    std::vector<double> coef;
    for (int j = count - 1; j >= 0; --j) {
        LGate g = G[j];
        const bool param = g.param_index >= 0;
        g.param_index = -1;
        if (param) {
            int gen = -1;
            switch (g.kind) {
            case QS_GATE_RX: gen = GEN_X; break;
            case QS_GATE_RY: gen = GEN_Y; break;
            case QS_GATE_RZ: gen = GEN_Z; break;
            case QS_GATE_U1: case QS_GATE_CU1: gen = GEN_PROJ; break;
            default: return -2;
            }
            LGate d = g;
            d.kind = kKindGrad;
            d.grad_gen = gen;
            d.grad_slot = (int)slot_gate.size();
            slot_gate.push_back(j);
            coef.push_back(gen == GEN_PROJ ? -2.0 : 1.0);
            rev.push_back(d);
        }
        LGate h = g;
        const int K = 1 << g.k;
        for (int r = 0; r < K; ++r)
            for (int c = 0; c < K; ++c) h.m[r * K + c] = std::conj(g.m[c * K + r]);
        rev.push_back(h);
    }
    qs_state s;
    s.n = n + 1;
    s.ms = n + 1;
    s.batch = 1;
    s.dtype = (qs_dtype)dtype;
    s.data = buf;
    const int k = tile_bits(s.dtype);
    const uint64_t tiles = (uint64_t)1 << (n + 1 - k);
    std::vector<double> part(slot_gate.size() * tiles, 0.0);
    g_gpart = &part;
    const qs_status st = run_tiled(&s, rev, nullptr, 0, n, part.data(), -1.0);
    g_gpart = nullptr;
    if (st != QS_OK) return (int)st;
    for (int j = 0; j < count; ++j) grad[j] = 0.0;
    for (size_t sl = 0; sl < slot_gate.size(); ++sl) {
        double sum = 0.0;
        for (uint64_t t = 0; t < tiles; ++t) sum += part[sl * tiles + t];
        grad[slot_gate[sl]] += coef[sl] * sum;
    }
    return 0;
}

// Adiabatic evolution through the library's tiled Trotter queue (trotter_queue:
// per step k, s_k = (k + 1/2) dt / T, an Ising phase with the merged half steps,
// then RX(2 dt a_q(s_k)) on every qubit, a_q(s) = (1 - s) a0[q] + s a1[q],
// written as RY layers in the frame of S on every qubit); the Ising table
// (index bits: J[a n + b], h[n], constant) is shared by the state.
int emu_trotter(int n, int dtype, const double *a0, const double *a1, const double *table, double T, double dt,
                int steps, double *psi) {
    std::vector<double> svals, taus;
    for (int k = 0; k < steps; ++k) svals.push_back((k + 0.5) * dt / T);
    taus.push_back(0.5 * dt * svals[0]);
    for (int k = 0; k + 1 < steps; ++k) taus.push_back(0.5 * dt * (svals[k] + svals[k + 1]));
    taus.push_back(0.5 * dt * svals[steps - 1]);
    std::vector<LGate> G;
    if (trotter_queue(n, std::vector<double>(a0, a0 + n), std::vector<double>(a1, a1 + n), taus, svals, dt, true,
                      &G) != QS_OK)
        return -1;
    qs_state s;
    s.n = n;
    s.ms = n;
    s.batch = 1;
    s.dtype = (qs_dtype)dtype;
    s.data = psi;
    s.itab = const_cast<double *>(table);
    s.ising_stride = 0;
    const qs_status st = run_tiled(&s, G, nullptr, 0);
    s.itab = nullptr;
    return (int)st;
}

const char *emu_last_error(void) { return last_error(); }
}
