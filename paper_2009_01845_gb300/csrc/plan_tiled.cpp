// Planner for the tiled multi-gate passes (see tiled.h).
//
// Pass selection is greedy in queue order. A gate joins the current pass when
//   * it commutes past every gate skipped so far (it shares no qubit with them),
//   * its dense targets fit in the tile (5 lane bits + k-5 chosen bits); diagonal
//     gates need no tile bits at all, since a tile knows every index bit of
//     every amplitude it holds.
// A gate the tile cannot express (dense on 3+ qubits, a 2-qubit dense gate
// touching a lane bit, a general 2+-qubit diagonal, a batched parameter) is
// applied by its own unfused pass when it reaches the front of the queue.
// Within a pass, stages re-split the k-5 high tile bits between registers and
// warps; the register set of a new stage is the needed bits plus the bits used
// soonest afterwards (furthest-next-use eviction).
#include <algorithm>
#include <cstring>
#include <limits>

#include "plan.h"
#include "prof.h"
#include "tiled.h"

namespace qsim {

qs_status k_tiled_pass_c64(qs_state *s, const TileParams<float> &p);
qs_status k_tiled_pass_c128(qs_state *s, const TileParams<double> &p);

namespace {

enum GClass { G_PHASE, G_DIAG1, G_DENSE1, G_DENSE2, G_SWAP, G_GRAD, G_ISING, G_SINGLE };

GClass classify(const LGate &g) {
    if (g.kind == kKindGrad) return G_GRAD;
    if (g.kind == kKindIsing) return G_ISING;
    if (g.param_index >= 0) {
        // batched parameters: the class follows the kind (the matrix differs per member)
        switch (g.kind) {
        case QS_GATE_RX: case QS_GATE_RY: return G_DENSE1;
        case QS_GATE_RZ: return G_DIAG1;
        case QS_GATE_U1: case QS_GATE_CU1: return G_PHASE;
        default: return G_SINGLE;
        }
    }
    if (g.phase_only) return G_PHASE;
    if (g.diagonal) return g.k == 1 ? G_DIAG1 : G_SINGLE;
    if (g.is_swap) return (g.tbit[0] >= kTileLaneBits && g.tbit[1] >= kTileLaneBits) ? G_SWAP : G_SINGLE;
    if (g.k == 1) return G_DENSE1;
    if (g.k == 2) return (g.tbit[0] >= kTileLaneBits && g.tbit[1] >= kTileLaneBits) ? G_DENSE2 : G_SINGLE;
    return G_SINGLE;
}

uint64_t qubit_bits(const LGate &g) {
    uint64_t m = g.cmask;
    for (int j = 0; j < g.k; ++j) m |= 1ull << g.tbit[j];
    return m;
}

// high (non-lane) global bits a gate needs inside the tile
uint64_t need_bits(const LGate &g, GClass c) {
    if (c == G_DENSE1) return g.tbit[0] >= kTileLaneBits ? (1ull << g.tbit[0]) : 0;
    if (c == G_GRAD && (g.grad_gen == GEN_X || g.grad_gen == GEN_Y))
        return g.tbit[0] >= kTileLaneBits ? (1ull << g.tbit[0]) : 0;
    if (c == G_DENSE2 || c == G_SWAP) return (1ull << g.tbit[0]) | (1ull << g.tbit[1]);
    return 0;
}

int mat_entries(GClass c) {
    switch (c) {
    case G_PHASE: return 1;
    case G_DIAG1: return 2;
    case G_DENSE1: return 4;
    case G_DENSE2: return 16;
    default: return 0;
    }
}

struct PassPlan {
    std::vector<int> gates;  // indices into the queue, in order
    uint64_t high = 0;       // chosen high tile bits (global)
};

}  // namespace

// slot[i]: per-member table slot of gate i (batched parameters) or -1
template <typename R>
static qs_status emit_and_run(qs_state *s, const std::vector<LGate> &G, const std::vector<GClass> &cls,
                              const std::vector<int> &slot, uint32_t pm_stride, const PassPlan &pp,
                              int force_bit, double *gpart, int *consumed) {
    const int n = s->n;
    const int RB = TileCfg<R>::RB;
    const int k = RB + kTileLaneBits + kTileWarpBits;
    // local <-> global bit maps
    int gbit[16], loc_of[64];
    for (int i = 0; i < 64; ++i) loc_of[i] = -1;
    int nl = 0;
    for (int b = 0; b < kTileLaneBits; ++b) gbit[nl++] = b;
    for (int b = kTileLaneBits; b < n; ++b)
        if ((pp.high >> b) & 1ull) gbit[nl++] = b;
    for (int i = 0; i < k; ++i) loc_of[gbit[i]] = i;

    // per-gate needed local register bits
    const int ng = (int)pp.gates.size();
    std::vector<uint32_t> needl(ng, 0);
    for (int i = 0; i < ng; ++i) {
        const uint64_t nb = need_bits(G[pp.gates[i]], cls[pp.gates[i]]);
        for (int b = 0; b < 64; ++b)
            if ((nb >> b) & 1ull) needl[i] |= 1u << loc_of[b];
    }
    const uint32_t force_loc = force_bit >= 0 ? (1u << loc_of[force_bit]) : 0u;
    auto choose = [&](int from, uint32_t forced) {
        forced |= force_loc;
        // forced bits plus the high local bits used soonest from op `from` on
        std::vector<std::pair<int, int>> rank;  // (next use, local bit)
        for (int lb = kTileLaneBits; lb < k; ++lb) {
            if ((forced >> lb) & 1u) continue;
            int nu = std::numeric_limits<int>::max();
            for (int i = from; i < ng; ++i)
                if ((needl[i] >> lb) & 1u) {
                    nu = i;
                    break;
                }
            rank.push_back({nu, lb});
        }
        std::sort(rank.begin(), rank.end());
        uint32_t r = forced;
        for (auto &pr : rank) {
            if (__builtin_popcount(r) >= RB) break;
            r |= 1u << pr.second;
        }
        return r;
    };

    TileParams<R> P;
    std::memset(&P, 0, sizeof(P));
    P.n = s->ms;  // member shift: tiles of member b start at b << ms
    P.k = k;
    P.n_free = n - k;
    P.total_tiles = (uint64_t)s->batch << P.n_free;
    P.tins.count = 0;
    {
        uint64_t tb = 0;
        for (int i = 0; i < k; ++i) tb |= 1ull << gbit[i];
        for (int b = 0; b < 64; ++b)
            if ((tb >> b) & 1ull) P.tins.pos[P.tins.count++] = (int8_t)b;
    }
    for (int i = 0; i < k; ++i) P.gbit[i] = (uint8_t)gbit[i];
    P.pmat = (const V<R> *)s->ptab;
    P.pm_stride = pm_stride;
    P.gpart = gpart;
    P.ising = s->itab;
    P.ising_stride = s->ising_stride;
    P.nq = n;
    for (int i = 0; i < k; ++i) P.tile_mask |= 1ull << gbit[i];
    int ngrad = 0;

    int nops = 0, nmat = 0, nst = 0, taken = 0;
    uint32_t cur = 0;
    const uint32_t highmask = ((1u << k) - 1u) & ~((1u << kTileLaneBits) - 1u);
    auto open_stage = [&](uint32_t rset) {
        TileStage &st = P.st[nst];
        int j = 0, w = 0;
        for (int lb = kTileLaneBits; lb < k; ++lb) {
            if ((rset >> lb) & 1u)
                st.rloc[j++] = (uint8_t)lb;
            else
                st.wloc[w++] = (uint8_t)lb;
        }
        st.op_begin = st.op_end = (uint16_t)nops;
        ++nst;
        cur = rset;
    };
    auto regidx = [&](int lb) {
        const TileStage &st = P.st[nst - 1];
        for (int j = 0; j < RB; ++j)
            if (st.rloc[j] == lb) return j;
        return -1;
    };
    // split a global required-bit mask into (register, thread-local, outside)
    auto split = [&](uint64_t gm, uint8_t *mr, uint32_t *mt, uint64_t *mo) {
        *mr = 0;
        *mt = 0;
        *mo = 0;
        for (int b = 0; b < 64; ++b) {
            if (!((gm >> b) & 1ull)) continue;
            const int lb = b < n ? loc_of[b] : -1;
            if (lb < 0) {
                *mo |= 1ull << b;
            } else if (lb >= kTileLaneBits && ((cur >> lb) & 1u)) {
                *mr |= (uint8_t)(1u << regidx(lb));
            } else {
                *mt |= 1u << lb;
            }
        }
    };
    auto put = [&](const std::complex<double> &v) {
        P.mat[nmat++] = mkc<R>((R)v.real(), (R)v.imag());
    };

    open_stage(choose(0, needl.empty() ? 0u : needl[0]) & highmask);
    for (int i = 0; i < ng; ++i) {
        const LGate &g = G[pp.gates[i]];
        const GClass c = cls[pp.gates[i]];
        const int ops_needed = 1;
        if ((needl[i] & ~cur) != 0) {
            if (nst >= kTileMaxStages) break;
            open_stage(choose(i, needl[i]));
        }
        const int sl = slot[pp.gates[i]];
        if (nops + ops_needed > kTileMaxOps || nmat + (sl >= 0 ? 0 : mat_entries(c)) > kTileMaxMat) break;
        if (c == G_GRAD && ngrad >= kTileMaxGrad) break;
        TileOp op;
        std::memset(&op, 0, sizeof(op));
        const int K = 1 << g.k;
        switch (c) {
        case G_PHASE: {
            op.type = TOP_PHASE;
            uint64_t req = g.cmask;
            for (int j = 0; j < g.k; ++j) req |= 1ull << g.tbit[j];
            split(req, &op.mr, &op.mt, &op.mo);
            if (sl >= 0) {
                op.pm = 1;
                op.m = 4 * sl;
            } else {
                op.m = nmat;
                put(g.m[(K - 1) * K + (K - 1)]);
            }
            break;
        }
        case G_DIAG1: {
            op.type = TOP_DIAG1;
            split(g.cmask, &op.mr, &op.mt, &op.mo);
            const int b = g.tbit[0];
            const int lb = loc_of[b];
            if (lb < 0) {
                op.tkind = TB_OUTSIDE;
                op.tmask = 1ull << b;
            } else if (lb >= kTileLaneBits && ((cur >> lb) & 1u)) {
                op.tkind = TB_REG;
                op.a = (uint8_t)regidx(lb);
            } else {
                op.tkind = TB_THREAD;
                op.tmask = 1ull << lb;
            }
            if (sl >= 0) {
                op.pm = 1;
                op.m = 4 * sl;
            } else {
                op.m = nmat;
                put(g.m[0]);
                put(g.m[3]);
            }
            break;
        }
        case G_DENSE1: {
            const int lb = loc_of[g.tbit[0]];
            if (lb < kTileLaneBits) {
                op.type = TOP_DENSE1_L;
                op.a = (uint8_t)lb;
            } else {
                op.type = TOP_DENSE1_R;
                op.a = (uint8_t)regidx(lb);
            }
            split(g.cmask, &op.mr, &op.mt, &op.mo);
            if (sl >= 0) {
                op.pm = 1;
                op.m = 4 * sl;
            } else {
                op.m = nmat;
                for (int e = 0; e < 4; ++e) put(g.m[e]);
            }
            break;
        }
        case G_DENSE2:
        case G_SWAP: {
            int A = regidx(loc_of[g.tbit[0]]), B = regidx(loc_of[g.tbit[1]]);
            op.type = c == G_SWAP ? TOP_SWAP_RR : TOP_DENSE2_RR;
            split(g.cmask, &op.mr, &op.mt, &op.mo);
            if (c == G_DENSE2) {
                // local index l = 2*bit(A) + bit(B); with A > B swap the roles
                // by exchanging local indices 1 and 2 on both sides
                op.m = nmat;
                const bool sw = A > B;
                for (int r = 0; r < 4; ++r)
                    for (int cc = 0; cc < 4; ++cc) {
                        auto perm = [&](int l) { return sw ? (((l & 1) << 1) | (l >> 1)) : l; };
                        put(g.m[perm(r) * 4 + perm(cc)]);
                    }
            }
            if (A > B) std::swap(A, B);
            op.a = (uint8_t)A;
            op.b = (uint8_t)B;
            break;
        }
        case G_ISING: {
            op.type = TOP_ISING;
            const double tau = g.m[0].real();
            std::memcpy(&op.tmask, &tau, sizeof(double));
            break;
        }
        case G_GRAD: {
            op.type = TOP_GRAD;
            op.b = (uint8_t)g.grad_gen;
            op.gl = (uint8_t)ngrad;
            P.gslot[ngrad++] = (uint16_t)g.grad_slot;
            if (g.grad_gen == GEN_PROJ) {
                uint64_t req = g.cmask;
                for (int j = 0; j < g.k; ++j) req |= 1ull << g.tbit[j];
                split(req, &op.mr, &op.mt, &op.mo);
                break;
            }
            split(g.cmask, &op.mr, &op.mt, &op.mo);
            const int b = g.tbit[0];
            const int lb = loc_of[b];
            if (g.grad_gen == GEN_Z) {
                if (lb < 0) {
                    op.tkind = TB_OUTSIDE;
                    op.tmask = 1ull << b;
                } else if (lb >= kTileLaneBits && ((cur >> lb) & 1u)) {
                    op.tkind = TB_REG;
                    op.a = (uint8_t)regidx(lb);
                } else {
                    op.tkind = TB_THREAD;
                    op.tmask = 1ull << lb;
                }
            } else if (lb < kTileLaneBits) {
                op.tkind = TB_THREAD;  // lane bit: shuffles
                op.a = (uint8_t)lb;
            } else {
                op.tkind = TB_REG;
                op.a = (uint8_t)regidx(lb);
            }
            break;
        }
        default:
            break;
        }
        P.op[nops++] = op;
        P.st[nst - 1].op_end = (uint16_t)nops;
        ++taken;
    }
    P.n_stages = nst;
    P.n_grad = ngrad;
    *consumed = taken;
    if (taken == 0) return QS_OK;
    if (prof_enabled()) {
        // algorithmic flops: per touched amplitude 16 for a 2x2 complex gate,
        // 64 for 4x4, 6 for a diagonal factor, 0 for a swap; the touched
        // fraction is 2^-(number of required bits)
        const double amps = (double)((uint64_t)s->batch << n);
        double fl = 0.0;
        for (int i = 0; i < taken; ++i) {
            const LGate &g = G[pp.gates[i]];
            const GClass c = cls[pp.gates[i]];
            int req = __builtin_popcountll(g.cmask);
            double per = 0.0;
            if (c == G_PHASE) {
                req += g.k;
                per = 6.0;
            } else if (c == G_DIAG1) {
                per = 6.0;
            } else if (c == G_DENSE1) {
                per = 16.0;
            } else if (c == G_DENSE2) {
                per = 64.0;
            } else if (c == G_GRAD) {
                per = 4.0;  // 8 per phi amplitude, phi is half the (phi, lambda) tile
            } else if (c == G_ISING) {
                per = 18.0; // three complex products per amplitude
            }
            fl += amps * per / (double)(1ull << req);
        }
        prof_add_work(KC_TILED, 2.0 * amps * sizeof(V<R>), fl);
    }
    if constexpr (sizeof(R) == 4)
        return k_tiled_pass_c64(s, P);
    else
        return k_tiled_pass_c128(s, P);
}

qs_status run_tiled(qs_state *s, const std::vector<LGate> &G, const double *params, int n_params, int force_bit,
                    double *gpart, double param_sign) {
    const int n = s->n;
    const int k = tile_bits(s->dtype);
    if (n < k) {
        if (force_bit >= 0) {
            set_error("adjoint sweep needs n + 1 >= %d", k);
            return QS_ERR_UNSUPPORTED;
        }
        for (const LGate &g : G) {
            if (g.param_index >= 0)
                QS_TRY(k_apply_param_gate(s, g, params, n_params));
            else
                QS_TRY(k_apply_unfused(s, g));
        }
        return QS_OK;
    }
    const int nh = k - kTileLaneBits;  // chosen high tile bits
    const uint64_t force = force_bit >= 0 ? (1ull << force_bit) : 0ull;
    std::vector<GClass> cls(G.size());
    for (size_t i = 0; i < G.size(); ++i) cls[i] = classify(G[i]);
    // per-member matrices of every batched-parameter gate, built once on the device
    std::vector<int> slot(G.size(), -1), spidx, skind;
    for (size_t i = 0; i < G.size(); ++i)
        if (G[i].param_index >= 0 && cls[i] != G_SINGLE) {
            slot[i] = (int)spidx.size();
            spidx.push_back(G[i].param_index);
            skind.push_back(G[i].kind);
        }
    uint32_t pm_stride = 0;
    if (!spidx.empty()) QS_TRY(k_param_table(s, spidx, skind, params, n_params, param_sign, &pm_stride));
    std::vector<char> done(G.size(), 0);
    size_t first = 0;
    while (true) {
        while (first < G.size() && done[first]) ++first;
        if (first >= G.size()) break;
        PassPlan pp;
        pp.high = force;
        uint64_t blocked = 0;
        const uint64_t all_bits = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
        for (size_t i = first; i < G.size(); ++i) {
            if (done[i]) continue;
            if (blocked == all_bits) break;  // nothing later can join this pass
            const uint64_t qb = cls[i] == G_ISING ? all_bits : qubit_bits(G[i]);
            if (qb & blocked) {
                blocked |= qb;
                continue;
            }
            if (cls[i] == G_SINGLE) {
                blocked |= qb;
                continue;
            }
            const uint64_t nb = need_bits(G[i], cls[i]);
            if (__builtin_popcountll(pp.high | nb) > nh) {
                blocked |= qb;
                continue;
            }
            pp.high |= nb;
            pp.gates.push_back((int)i);
            if ((int)pp.gates.size() >= kTileMaxOps) break;
        }
        if (pp.gates.empty()) {
            // the front gate cannot run in a tile
            // (in the adjoint sweep it acts on phi and lambda alike: neither the
            // gate nor its controls touch the top bit that tells them apart)
            const LGate &g = G[first];
            if (g.param_index >= 0)
                QS_TRY(k_apply_param_gate(s, g, params, n_params, param_sign));
            else
                QS_TRY(k_apply_unfused(s, g));
            done[first] = 1;
            continue;
        }
        // complete the tile with unused high bits
        for (int b = kTileLaneBits; b < n && __builtin_popcountll(pp.high) < nh; ++b) pp.high |= 1ull << b;
        int consumed = 0;
        if (s->dtype == QS_C64)
            QS_TRY(emit_and_run<float>(s, G, cls, slot, pm_stride, pp, force_bit, gpart, &consumed));
        else
            QS_TRY(emit_and_run<double>(s, G, cls, slot, pm_stride, pp, force_bit, gpart, &consumed));
        if (consumed <= 0) {
            set_error("tiled planner made no progress");
            return QS_ERR_CUDA;
        }
        for (int i = 0; i < consumed; ++i) done[pp.gates[i]] = 1;
    }
    return QS_OK;
}

}  // namespace qsim
