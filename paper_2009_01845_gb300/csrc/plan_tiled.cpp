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
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <unordered_map>
#include <utility>

#include "plan.h"
#include "prof.h"
#include "tiled.h"

namespace qsim {

qs_status k_tiled_pass_c64(qs_state *s, const TileParams<float> &p);
qs_status k_ising_table(qs_state *s, const IsingTabP &tp);
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

// ------------------------------------------------------------------ entries
// A pass is emitted from a list of entries: original gates, rotations (the
// real rotation of an uncontrolled one-qubit gate, see split_1q and rot_plan),
// and diagonal blocks (products of one-bit diagonals and phase factors).
namespace {

enum EKind { E_GATE, E_ROT, E_BLOCK };

struct Factor {
    int type;        // DF_BIT or DF_PHASE
    int bit;         // DF_BIT: index bit
    uint64_t mask;   // DF_PHASE: required index bits
    cd v0, v1;       // DF_BIT: diag(v0, v1); DF_PHASE: v0
    int rot = -1;    // the D_L of rotation gate `rot`: also times that rotation's diagonal
};

struct Entry {
    EKind kind;
    int gi = -1;              // E_GATE / E_ROT: gate index
    int bit = -1;             // E_ROT: index bit
    double cg = 0.0, sg = 0.0;  // E_ROT: cos h, sin h of R = [[cos h, -sin h], [sin h, cos h]]
    bool paeth = false;       // E_ROT: U = R (no diagonal factors), three shears
    std::vector<Factor> fac;  // E_BLOCK
};

// U = D_L R D_R with R = [[cos h, -sin h], [sin h, cos h]], 0 <= h <= pi/2,
// D_R = diag(1, e^{i b1}), D_L = diag(e^{i a0}, e^{i a1}). How R is applied
// (see rot_plan) adds a real diagonal to D_L when the stage is emitted.
// Returns false if U is diagonal.
bool split_1q(const std::vector<cd> &m, cd *dr, cd *dl, double *cg, double *sg) {
    *cg = std::abs(m[0]);
    *sg = std::abs(m[2]);
    if (*sg == 0.0) return false;
    const double a0 = *cg > 0.0 ? std::arg(m[0]) : 0.0;
    const double a1 = std::arg(m[2]);
    const double b1 = std::arg(-m[1]) - a0;
    dr[0] = 1.0;
    dr[1] = std::polar(1.0, b1);
    dl[0] = std::polar(1.0, a0);
    dl[1] = std::polar(1.0, a1);
    return true;
}

// How the rotation R (cos h = cg, sin h = sg) runs on a register bit whose
// halves are (frame = 0) or are not (frame = 1) in natural order: physical
// shears x += s1 y, y += s2 x (and x += s1 y again if `three`), with x the
// register half where the bit is 0, then R = dd * [swap] * (those shears) in
// the bit's own terms, the swap (`swap`: the frame flips) left to the frame.
//   h <= pi/4, t = tan h:  R = diag(cos h, sec h) Sy(sin h cos h) Sx(-t)
//                            = diag(sec h, cos h) Sx(-sin h cos h) Sy(t);
//   h >  pi/4, psi = pi/2 - h, u = tan psi, with the frame:
//                          R = diag(-sec psi, cos psi) X Sy(-sin psi cos psi) Sx(u)
//                            = diag(-cos psi, sec psi) X Sx(sin psi cos psi) Sy(-u);
//   h >  pi/4 without it:  R = Sx(-tan h/2) Sy(sin h) Sx(-tan h/2)
//                            = Sy(tan h/2) Sx(-sin h) Sy(tan h/2),
// where Sx(c): x += c y, Sy(c): y += c x, X swaps x and y; the first form of
// each pair starts with x (frame 0), the second with y (frame 1, where the
// physical x holds the bit's 1 half). Every coefficient and diagonal entry is
// at most sqrt(2) in magnitude.
struct RotPlan {
    double s1, s2;
    bool three, swap;
    cd dd0, dd1;
};
RotPlan rot_plan(double cg, double sg, int frame, bool allow_swap, bool paeth) {
    RotPlan q{};
    const double sc = sg * cg;
    if (paeth) {
        allow_swap = false;
    } else if (cg >= sg) {
        const double t = sg / cg;
        q.s1 = frame ? t : -t;
        q.s2 = frame ? -sc : sc;
        q.dd0 = frame ? 1.0 / cg : cg;
        q.dd1 = frame ? cg : 1.0 / cg;
    } else if (allow_swap) {
        const double u = cg / sg;
        q.swap = true;
        q.s1 = frame ? -u : u;
        q.s2 = frame ? sc : -sc;
        q.dd0 = frame ? -sg : -1.0 / sg;
        q.dd1 = frame ? 1.0 / sg : sg;
    }
    if (paeth || (cg < sg && !allow_swap)) {
        const double th = sg / (1.0 + cg);  // tan(h/2)
        q.three = true;
        q.s1 = frame ? th : -th;
        q.s2 = frame ? -sg : sg;
        q.dd0 = q.dd1 = 1.0;
    }
    return q;
}

uint64_t factor_bits(const Factor &f) { return f.type == DF_BIT ? (1ull << f.bit) : f.mask; }

}  // namespace

// Split the gates of a pass into entries. With `algebra`, uncontrolled
// one-qubit gates become D_R, a real rotation and D_L; those diagonals,
// uncontrolled one-bit diagonal gates and phase gates become factors. Returns
// the other entries in queue order and, in *facs, every factor with the range
// of positions it may be applied at: a cut at position p means "just before
// entry p" (p = size: after the last), valid for left < p <= right, where left
// and right are the last and next entries that do not commute with the factor
// (a rotation or a dense gate on one of its bits). The caller places the cuts
// (diagonal blocks) and assigns the factors to them.
struct FactorSpan {
    Factor f;
    int left, right;
};

static std::vector<Entry> build_entries(const std::vector<LGate> &G, const std::vector<GClass> &cls,
                                        const std::vector<int> &slot, const std::vector<int> &gates, bool algebra,
                                        std::vector<FactorSpan> *facs) {
    facs->clear();
    std::vector<Entry> base;                  // non-factor entries in order
    std::vector<uint64_t> blocks_bits;        // bits each base entry does not commute on
    std::vector<char> is_grad;                // base entry is a gradient op
    struct PF { Factor f; int pos; };         // factor and the base position it precedes
    std::vector<PF> pf;
    for (int gi : gates) {
        const LGate &g = G[gi];
        const GClass c = cls[gi];
        const bool plain = algebra && slot[gi] < 0 && g.cmask == 0;
        if (plain && c == G_DENSE1) {
            cd dr[2], dl[2];
            double cg = 0.0, sg = 0.0;
            if (!split_1q(g.m, dr, dl, &cg, &sg)) {
                pf.push_back({Factor{DF_BIT, g.tbit[0], 0, g.m[0], g.m[3]}, (int)base.size()});
                continue;
            }
            // a real rotation marked for three shears has no factors at all (the
            // lanes are free, so it always runs on a register bit)
            const auto one = [](const cd &v) { return std::abs(v - cd(1.0)) < 1e-15; };
            const bool paeth = g.paeth && one(dr[1]) && one(dl[0]) && one(dl[1]);
            if (!paeth) pf.push_back({Factor{DF_BIT, g.tbit[0], 0, dr[0], dr[1]}, (int)base.size()});
            Entry e{E_ROT};
            e.gi = gi;
            e.bit = g.tbit[0];
            e.cg = cg;
            e.sg = sg;
            e.paeth = paeth;
            base.push_back(e);
            blocks_bits.push_back(1ull << g.tbit[0]);
            is_grad.push_back(0);
            if (paeth) continue;
            Factor fl{DF_BIT, g.tbit[0], 0, dl[0], dl[1]};
            fl.rot = gi;
            pf.push_back({fl, (int)base.size()});
            continue;
        }
        if (plain && c == G_DIAG1) {
            pf.push_back({Factor{DF_BIT, g.tbit[0], 0, g.m[0], g.m[3]}, (int)base.size()});
            continue;
        }
        if (algebra && slot[gi] < 0 && c == G_PHASE) {
            uint64_t req = g.cmask;
            for (int j = 0; j < g.k; ++j) req |= 1ull << g.tbit[j];
            const int K = 1 << g.k;
            pf.push_back({Factor{DF_PHASE, -1, req, g.m[(K - 1) * K + K - 1], 0.0}, (int)base.size()});
            continue;
        }
        Entry e{E_GATE};
        e.gi = gi;
        base.push_back(e);
        uint64_t nb = 0;
        if (c == G_DENSE1 || c == G_DENSE2 || c == G_SWAP)
            for (int j = 0; j < g.k; ++j) nb |= 1ull << g.tbit[j];
        is_grad.push_back(c == G_GRAD ? 1 : 0);
        if (c == G_SINGLE) nb = ~0ull;  // barrier
        // a gradient op <lambda|P|phi> is unchanged by a unitary diagonal
        // applied to both phi and lambda when the diagonal commutes with P: Z
        // and projector generators commute with every diagonal, X and Y with
        // the diagonals that do not involve their target. (The D_L of a
        // factored gate, which carries the real diagonal of its rotation's
        // shears, never crosses a gradient op: the readout is bilinear in the
        // state.)
        if (c == G_GRAD) nb = (g.grad_gen == GEN_X || g.grad_gen == GEN_Y) ? (1ull << g.tbit[0]) : 0ull;
        blocks_bits.push_back(nb);
    }
    const int nbase = (int)base.size();
    for (const PF &q : pf) {
        const uint64_t fb = factor_bits(q.f);
        const bool unitary = q.f.rot < 0 && std::abs(std::abs(q.f.v0) - 1.0) < 1e-12 &&
                             (q.f.type != DF_BIT || std::abs(std::abs(q.f.v1) - 1.0) < 1e-12);
        auto blocks = [&](int p) { return (blocks_bits[p] & fb) != 0 || (is_grad[p] && !unitary); };
        int left = -1, right = nbase;
        for (int p = q.pos - 1; p >= 0; --p)
            if (blocks(p)) {
                left = p;
                break;
            }
        for (int p = q.pos; p < nbase; ++p)
            if (blocks(p)) {
                right = p;
                break;
            }
        facs->push_back(FactorSpan{q.f, left, right});
    }
    return base;
}

// slot[i]: per-member table slot of gate i (batched parameters) or -1.
// Emits one tiled pass for the gates pp.gates; *fits = false (nothing launched)
// when the pass exceeds the descriptor's capacity.
// Swizzle of the transpose from stage a into stage b (see tiled.h): the
// images of the high local bits are chosen so that, for both stages, the
// lanes of one wavefront (lane bits 0 .. h-1) land on h independent low-bit
// patterns, i.e. distinct banks. The fold of the high bits onto bit (p mod h)
// is kept when it already works; otherwise images of the wavefront lanes'
// high bits are drawn from a fixed-seed generator until both stages pass.
// Then the byte offsets of both stages' register bits under that swizzle.
template <typename R> static void set_transpose(const TileStage &a, TileStage &b, int k, uint64_t *rng) {
    constexpr int h = swizzle_low_bits<R>();
    constexpr int RB = TileCfg<R>::RB;
    const int nh = k - h;
    uint8_t f[9];
    for (int i = 0; i < 9; ++i) f[i] = (uint8_t)(i < nh ? 1u << ((h + i) % h) : 0u);
    auto img = [&](int p) -> uint32_t { return p < h ? (1u << p) : f[p - h]; };
    auto full_rank = [&](const uint8_t *lanes) {
        uint32_t v[8];
        for (int x = 0; x < h; ++x) v[x] = img(lanes[x]);
        int rank = 0;
        for (int bit = h - 1; bit >= 0; --bit) {
            int piv = -1;
            for (int x = rank; x < h; ++x)
                if ((v[x] >> bit) & 1u) {
                    piv = x;
                    break;
                }
            if (piv < 0) continue;
            std::swap(v[rank], v[piv]);
            for (int x = 0; x < h; ++x)
                if (x != rank && ((v[x] >> bit) & 1u)) v[x] ^= v[rank];
            ++rank;
        }
        return rank == h;
    };
    if (!(full_rank(a.lloc) && full_rank(b.lloc))) {
        uint32_t free_hi = 0;
        for (int x = 0; x < h; ++x) {
            if (a.lloc[x] >= h) free_hi |= 1u << (a.lloc[x] - h);
            if (b.lloc[x] >= h) free_hi |= 1u << (b.lloc[x] - h);
        }
        uint8_t fold[9];
        std::memcpy(fold, f, sizeof(f));
        bool found = false;
        for (int tries = 0; tries < 4096 && !found; ++tries) {
            for (int i = 0; i < nh; ++i)
                if ((free_hi >> i) & 1u) {
                    *rng = *rng * 6364136223846793005ull + 1442695040888963407ull;
                    f[i] = (uint8_t)((*rng >> 33) & ((1u << h) - 1u));
                }
            found = full_rank(a.lloc) && full_rank(b.lloc);
        }
        if (!found) std::memcpy(f, fold, sizeof(f));
    }
    std::memcpy(b.fcol, f, sizeof(f));
    auto pos = [&](uint32_t x) {
        uint32_t y = x;
        for (int i = 0; i < nh; ++i)
            if ((x >> (h + i)) & 1u) y ^= f[i];
        return y;
    };
    for (int j = 0; j < 6; ++j) {
        b.rw[j] = j < RB ? (uint16_t)(pos(1u << a.rloc[j]) * sizeof(V<R>)) : 0;
        b.rr[j] = j < RB ? (uint16_t)(pos(1u << b.rloc[j]) * sizeof(V<R>)) : 0;
    }
}

template <typename R>
static qs_status emit_and_run(qs_state *s, const std::vector<LGate> &G, const std::vector<GClass> &cls,
                              const std::vector<int> &slot, uint32_t pm_stride, const PassPlan &pp,
                              int force_bit, double *gpart, bool *fits, int *dry_stages = nullptr) {
    const int n = s->n;
    const int RB = TileCfg<R>::RB;
    const int k = RB + kTileLaneBits + TileCfg<R>::WB;
    *fits = true;
    // local <-> global bit maps
    int gbit[16], loc_of[64];
    for (int i = 0; i < 64; ++i) loc_of[i] = -1;
    int nl = 0;
    for (int b = 0; b < kTileLaneBits; ++b) gbit[nl++] = b;
    for (int b = kTileLaneBits; b < n; ++b)
        if ((pp.high >> b) & 1ull) gbit[nl++] = b;
    for (int i = 0; i < k; ++i) loc_of[gbit[i]] = i;

    // Free lanes: dense targets, lane bits included, must be register bits;
    // stages move lanes to any bits. (In the adjoint sweep the forced bit that
    // tells phi from lambda is the highest tile bit, so it is always the top
    // register bit, as the gradient ops require.)
    const bool free_lanes = true;
    std::vector<FactorSpan> facs;
    const std::vector<Entry> base = build_entries(G, cls, slot, pp.gates, free_lanes, &facs);
    // needed local register bits of an entry
    auto need_of = [&](const Entry &e) {
        uint64_t nb = 0;
        if (e.kind == E_GATE) {
            const LGate &g = G[e.gi];
            const GClass c = cls[e.gi];
            nb = need_bits(g, c);
            if (free_lanes && (c == G_DENSE1 || (c == G_GRAD && (g.grad_gen == GEN_X || g.grad_gen == GEN_Y))))
                nb = 1ull << g.tbit[0];
        }
        if (e.kind == E_ROT && (free_lanes || e.bit >= kTileLaneBits)) nb = 1ull << e.bit;
        uint32_t l = 0;
        for (int b = 0; b < 64; ++b)
            if ((nb >> b) & 1ull) l |= 1u << loc_of[b];
        return l;
    };
    // the stage choices below read needl/ne: first over the entries without
    // diagonal blocks (blocks need no bits, so the stages are the same), then
    // over the final list
    std::vector<Entry> ent;
    int ne = (int)base.size();
    std::vector<uint32_t> needl(ne, 0);
    for (int i = 0; i < ne; ++i) needl[i] = need_of(base[i]);
    const uint32_t force_loc = force_bit >= 0 ? (1u << loc_of[force_bit]) : 0u;
    const uint32_t low5 = (1u << kTileLaneBits) - 1u;
    auto next_use = [&](int from, int lb) {
        for (int i = from; i < ne; ++i)
            if ((needl[i] >> lb) & 1u) return i;
        return std::numeric_limits<int>::max();
    };
    // register set: forced bits plus the candidate bits used soonest from entry
    // `from` on (furthest-next-use eviction)
    auto choose = [&](int from, uint32_t forced, uint32_t candidates) {
        forced |= force_loc;
        std::vector<std::pair<int, int>> rank;  // (next use, local bit)
        for (int lb = 0; lb < k; ++lb) {
            if (((forced >> lb) & 1u) || !((candidates >> lb) & 1u)) continue;
            rank.push_back({next_use(from, lb), lb});
        }
        std::sort(rank.begin(), rank.end());
        uint32_t r = forced;
        for (auto &pr : rank) {
            if (__builtin_popcount(r) >= RB) break;
            r |= 1u << pr.second;
        }
        return r;
    };
    // lanes: the 5 lowest bits that are not registers (ops never act on lane
    // bits; keeping index bits 0 and 1 on lanes lets the last stage store whole
    // 32-byte sectors from any lane map), ordered, where possible, so that the
    // lanes of a half-warp (complex64) / quarter-warp (complex128) have
    // distinct residues, which the default swizzle then serves
    const int half = sizeof(R) == 4 ? 4 : 3;
    auto lanes_for = [&](int, uint32_t rset) {
        std::vector<int> L;
        for (int lb = 0; lb < k && (int)L.size() < kTileLaneBits; ++lb)
            if (!((rset >> lb) & 1u)) L.push_back(lb);
        std::vector<int> best = L;
        do {
            bool okr = true;
            for (int x = 0; x < half && okr; ++x)
                for (int y = x + 1; y < half; ++y)
                    if (L[x] % half == L[y] % half) okr = false;
            if (okr) {
                best = L;
                break;
            }
        } while (std::next_permutation(L.begin(), L.end()));
        return best;
    };

    const uint32_t low5_mask = (1u << kTileLaneBits) - 1u;
    const uint32_t high_bits = ((1u << k) - 1u) & ~low5_mask;

    // Diagonal blocks. The register set in effect at every entry (a stage
    // opens at an entry whose needed bits are not all registers). Costs in
    // instructions per thread: a block's phase walk (kWalk; paid by a cut
    // holding any factor but register sign flips), and per factor: on register
    // bits alone 0 (folds into the block's constants), a register sign flip 16
    // (its own op), a sign under thread/outside bits 10, a complex product 25,
    // a pair factor 60. Cuts start as the fewest points that meet every
    // factor's range (greedy interval stabbing: sort by right end, cut at the
    // first right end, repeat), each factor at its cheapest open cut; then,
    // while it lowers the total, the stage opening (or pass end) whose opening
    // saves most is added, factors moving to it where cheaper.
    {
        const int nbase = (int)base.size();
        std::vector<uint32_t> reg_base(nbase + 1, 0u);
        std::vector<char> cand(nbase + 1, 0), open(nbase + 1, 0);
        uint32_t c = choose(0, (ne ? needl[0] : 0u) & high_bits, high_bits);
        cand[0] = 1;
        for (int i = 0; i < nbase; ++i) {
            if ((needl[i] & ~c) != 0) {
                c = free_lanes ? choose(i, needl[i], (1u << k) - 1u) : choose(i, needl[i], high_bits);
                cand[i] = 1;
            }
            reg_base[i] = c;
        }
        reg_base[nbase] = c;
        cand[nbase] = 1;
        const int nf = (int)facs.size();
        {
            std::vector<int> order(nf);
            for (int j = 0; j < nf; ++j) order[j] = j;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return facs[x].right < facs[y].right; });
            for (int j : order) {
                bool met = false;
                for (int p = facs[j].left + 1; p <= facs[j].right && !met; ++p) met = open[p] != 0;
                if (!met) open[facs[j].right] = 1;
            }
        }
        constexpr int kWalk = 280;
        // cost of factor f at a cut with register set regs; *walk: needs the phase walk
        auto cost = [&](const Factor &f, uint32_t regs, bool *walk) {
            int nr = 0, nt = 0, no = 0;
            const uint64_t m = factor_bits(f);
            for (int b = 0; b < 64; ++b) {
                if (!((m >> b) & 1ull)) continue;
                const int lb = b < n ? loc_of[b] : -1;
                if (lb < 0) ++no;
                else if ((regs >> lb) & 1u) ++nr;
                else ++nt;
            }
            *walk = true;
            if (f.type == DF_BIT) return nr ? 0 : 25;
            const bool sign = f.v0 == cd(-1.0, 0.0);
            if (sign && nr >= 2) {
                *walk = false;
                return 16;
            }
            if (nt == 0 && no == 0) return nr <= 1 ? 0 : 60;
            if (sign) return 10;
            return nr >= 2 ? 60 : 25;
        };
        std::vector<int> where(nf, -1), fc(nf, 0);
        std::vector<char> fw(nf, 0);
        for (int j = 0; j < nf; ++j) {
            int bc = std::numeric_limits<int>::max();
            for (int p = facs[j].left + 1; p <= facs[j].right; ++p) {
                if (!open[p]) continue;
                bool w;
                const int cc = cost(facs[j].f, reg_base[p], &w);
                if (cc < bc) {
                    bc = cc;
                    where[j] = p;
                    fc[j] = cc;
                    fw[j] = w;
                }
            }
        }
        for (;;) {
            // walkers per open cut
            std::vector<int> walkers(nbase + 1, 0);
            for (int j = 0; j < nf; ++j) walkers[where[j]] += fw[j];
            int best_q = -1, best_delta = 0;
            for (int q = 0; q <= nbase; ++q) {
                if (!cand[q] || open[q]) continue;
                int delta = 0;
                bool q_walks = false;
                std::vector<int> left_walkers = walkers;
                for (int j = 0; j < nf; ++j) {
                    if (!(facs[j].left < q && q <= facs[j].right)) continue;
                    bool w;
                    const int cc = cost(facs[j].f, reg_base[q], &w);
                    if (cc >= fc[j]) continue;
                    delta += cc - fc[j];
                    q_walks = q_walks || w;
                    if (fw[j] && --left_walkers[where[j]] == 0) delta -= kWalk;  // a block emptied of walkers
                }
                if (q_walks) delta += kWalk;
                if (delta < best_delta) {
                    best_delta = delta;
                    best_q = q;
                }
            }
            if (best_q < 0) break;
            open[best_q] = 1;
            for (int j = 0; j < nf; ++j) {
                if (!(facs[j].left < best_q && best_q <= facs[j].right)) continue;
                bool w;
                const int cc = cost(facs[j].f, reg_base[best_q], &w);
                if (cc >= fc[j]) continue;
                where[j] = best_q;
                fc[j] = cc;
                fw[j] = w;
            }
        }
        std::vector<std::vector<Factor>> at(nbase + 1);
        for (int j = 0; j < nf; ++j) at[where[j]].push_back(facs[j].f);  // in queue order
        for (int p = 0; p <= nbase; ++p) {
            if (!at[p].empty()) {
                Entry b{E_BLOCK};
                b.fac = std::move(at[p]);
                ent.push_back(std::move(b));
            }
            if (p < nbase) ent.push_back(base[p]);
        }
        ne = (int)ent.size();
        needl.assign(ne, 0u);
        for (int i = 0; i < ne; ++i) needl[i] = need_of(ent[i]);
    }
    // a diagonal block is placed in the stage of the next non-block entry
    // (that stage opens before the block)
    auto opener = [&](int i) {
        while (i < ne && ent[i].kind == E_BLOCK) ++i;
        return i;
    };

    TileParams<R> &P = *new TileParams<R>();
    std::unique_ptr<TileParams<R>> hold(&P);
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
    int ngrad = 0, ndf = 0, nising = 0;

    int nops = 0, nmat = 0, nst = 0;
    uint32_t cur = 0, curL = 0;
    uint32_t curF = 0;  // register frame of the open stage (see tiled.h)
    std::unordered_map<int, std::pair<cd, cd>> rot_dd;  // rotation gate -> diagonal joining its D_L
    const uint32_t highmask = ((1u << k) - 1u) & ~low5;
    auto open_stage = [&](uint32_t rset, const std::vector<int> &L) {
        if (nst > 0) P.st[nst - 1].rflip = (uint8_t)curF;  // the transpose undoes the frame
        curF = 0;
        TileStage &st = P.st[nst];
        uint32_t lset = 0;
        for (int x = 0; x < kTileLaneBits; ++x) {
            st.lloc[x] = (uint8_t)L[x];
            lset |= 1u << L[x];
        }
        int j = 0, w = 0;
        for (int lb = 0; lb < k; ++lb) {
            if ((rset >> lb) & 1u)
                st.rloc[j++] = (uint8_t)lb;
            else if (!((lset >> lb) & 1u))
                st.wloc[w++] = (uint8_t)lb;
        }
        st.op_begin = st.op_end = (uint16_t)nops;
        ++nst;
        cur = rset;
        curL = lset;
    };
    const std::vector<int> natural = {0, 1, 2, 3, 4};
    auto lane_index = [&](int lb) {
        const TileStage &st = P.st[nst - 1];
        for (int x = 0; x < kTileLaneBits; ++x)
            if (st.lloc[x] == lb) return x;
        return -1;
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
            } else if ((cur >> lb) & 1u) {
                *mr |= (uint8_t)(1u << regidx(lb));
            } else {
                *mt |= 1u << lb;
            }
        }
    };
    auto put = [&](const std::complex<double> &v) {
        P.mat[nmat++] = mkc<R>((R)v.real(), (R)v.imag());
    };
    auto locate = [&](int b, uint8_t *tkind, uint8_t *a, uint64_t *tmask) {
        const int lb = loc_of[b];
        if (lb < 0) {
            *tkind = TB_OUTSIDE;
            *tmask = 1ull << b;
        } else if ((cur >> lb) & 1u) {
            *tkind = TB_REG;
            *a = (uint8_t)regidx(lb);
        } else {
            *tkind = TB_THREAD;
            *tmask = 1ull << lb;
        }
    };
    auto overflow = [&]() {
        *fits = false;
        return QS_OK;
    };

    // Third shears of three-shear rotations wait (slot, coefficient) until an
    // entry other than a rotation on another register bit comes, or the stage
    // ends; then they go out as one op (rotations on other bits commute with
    // them, so a run of rotations costs two ops, not one per rotation).
    std::vector<std::pair<int, R>> third;
    auto flush_third = [&]() {
        if (third.empty()) return true;
        if (nops + 1 > kTileMaxOps || nmat + RB > kTileMaxMat) return false;
        TileOp ro;
        std::memset(&ro, 0, sizeof(ro));
        ro.type = TOP_ROTS_R;
        ro.m = nmat;
        for (int x = 0; x < RB; ++x) put(cd(0.0, 0.0));
        for (const auto &t3 : third) {
            ro.a |= (uint8_t)(1u << t3.first);
            P.mat[ro.m + t3.first] = mkc<R>(t3.second, (R)0);
        }
        P.op[nops++] = ro;
        P.st[nst - 1].op_end = (uint16_t)nops;
        third.clear();
        return true;
    };
    // the first stage reads the tile with lanes on the 5 lowest bits
    open_stage(choose(0, (ne ? needl[0] : 0u) & highmask, highmask), natural);
    for (int i = 0; i < ne; ++i) {
        const Entry &e = ent[i];
        const int oi = opener(i);
        if (!third.empty()) {
            bool keep = e.kind == E_ROT && !(oi < ne && (needl[oi] & ~cur) != 0);
            if (keep) {
                const int lb3 = loc_of[e.bit];
                keep = ((cur >> lb3) & 1u) != 0;
                for (const auto &t3 : third) keep = keep && t3.first != regidx(lb3);
            }
            if (!keep && !flush_third()) return overflow();
        }
        if (oi < ne && (needl[oi] & ~cur) != 0) {
            if (nst >= kTileMaxStages) return overflow();
            if (free_lanes) {
                const uint32_t rset = choose(oi, needl[oi], (1u << k) - 1u);
                open_stage(rset, lanes_for(oi, rset));
            } else {
                open_stage(choose(oi, needl[oi], highmask), natural);
            }
        }
        if (nops + 1 > kTileMaxOps) return overflow();
        TileOp op;
        std::memset(&op, 0, sizeof(op));
        if (e.kind == E_ROT) {
            // rotations on distinct bits commute: consecutive ones of one stage
            // share an op (register bits or lane bits)
            const int lb = loc_of[e.bit];
            const bool lane = !((cur >> lb) & 1u);
            const int j = lane ? lane_index(lb) : regidx(lb);
            const uint8_t want = lane ? TOP_ROTS_L : TOP_ROTS_R;
            const int width = lane ? kTileLaneBits : RB;
            // place rotation coefficients in slot j: into the stage's last op when
            // it is a rotation op of this kind with slot j free, else a new op
            auto push_rot = [&](const V<R> &cf) {
                if (nops > P.st[nst - 1].op_begin && P.op[nops - 1].type == want) {
                    TileOp &prev = P.op[nops - 1];
                    const bool free_slot = lane ? P.mat[prev.m + j].y == (R)0 : !((prev.a >> j) & 1u);
                    if (free_slot) {
                        P.mat[prev.m + j] = cf;
                        if (!lane) prev.a |= (uint8_t)(1u << j);
                        return true;
                    }
                }
                if (nops + 1 > kTileMaxOps || nmat + width > kTileMaxMat) return false;
                TileOp ro;
                std::memset(&ro, 0, sizeof(ro));
                ro.type = want;
                ro.m = nmat;
                ro.a = lane ? (uint8_t)0 : (uint8_t)(1u << j);
                for (int x = 0; x < width; ++x) put(cd(0.0, 0.0));
                P.mat[ro.m + j] = cf;
                P.op[nops++] = ro;
                P.st[nst - 1].op_end = (uint16_t)nops;
                return true;
            };
            if (lane) {  // scaled forms (see TileRotForm); the scalar and sign join D_L
                const bool tanf = e.cg >= e.sg;
                rot_dd[e.gi] = tanf ? std::make_pair(cd(e.cg), cd(e.cg)) : std::make_pair(cd(-e.sg), cd(e.sg));
                if (!push_rot(mkc<R>((R)(tanf ? e.sg / e.cg : e.cg / e.sg), (R)((tanf ? ROT_TAN : ROT_COT) + 1))))
                    return overflow();
                continue;
            }
            // the swap of a near-swap rotation may stay in the frame when no later
            // op of this stage, other than rotations and diagonal blocks (which the
            // frame rewrites), touches the bit
            bool allow = true;
            for (int i2 = i + 1; i2 < ne && allow; ++i2) {
                const int o2 = opener(i2);
                if (o2 < ne && (needl[o2] & ~cur) != 0) break;  // the next stage opens
                const Entry &e2 = ent[i2];
                if (e2.kind != E_GATE) continue;
                allow = cls[e2.gi] != G_ISING && !((qubit_bits(G[e2.gi]) >> e.bit) & 1ull);
            }
            const RotPlan q = rot_plan(e.cg, e.sg, (int)((curF >> j) & 1u), allow, e.paeth);
            if (q.swap) curF ^= 1u << j;
            rot_dd[e.gi] = std::make_pair(q.dd0, q.dd1);
            // (a swap alone, cos h = 0, is all frame: no op)
            if ((q.s1 != 0.0 || q.s2 != 0.0) && !push_rot(mkc<R>((R)q.s1, (R)q.s2))) return overflow();
            // the third shear of the three-shear form: one more x += s1 y
            if (q.three) third.push_back({j, (R)q.s1});
            continue;
        } else if (e.kind == E_BLOCK) {
            // constants (base, per-register-bit ratios) for the factors on
            // register bits alone; sign flips on two or more register bits become
            // TOP_FLIP ops; the others go to the factor table: outside-only
            // complex factors first, then sign factors (a negation of the base or
            // of one ratio under conditions), then thread/mixed complex factors,
            // pairs last
            // Everything on register bits is written for the stage's register
            // frame F (register r holds register index r ^ F): a condition "bit
            // j is 1" on a register bit of F reads "bit j is 0".
            cd cbase = 1.0;
            std::vector<cd> cu(RB, cd(1.0));
            std::vector<TileDFac<R>> outside, signs, single, pair;
            std::vector<TileOp> flips;
            auto reg_pattern = [&](uint8_t mr) {
                uint64_t pat = 0;
                for (int r = 0; r < (1 << RB); ++r)
                    if (((r ^ curF) & mr) == mr) pat |= 1ull << r;
                return pat;
            };
            auto is_pm1 = [](const cd &v) { return v == cd(1.0, 0.0) || v == cd(-1.0, 0.0); };
            // the rotations' diagonals join their D_L factors; one-bit diagonals
            // on the same bit multiply
            std::vector<Factor> facl;
            for (Factor f : e.fac) {
                if (f.rot >= 0) {
                    const auto it = rot_dd.find(f.rot);
                    if (it != rot_dd.end()) {
                        f.v0 *= it->second.first;
                        f.v1 *= it->second.second;
                    }
                }
                bool merged = false;
                if (f.type == DF_BIT)
                    for (Factor &g : facl)
                        if (g.type == DF_BIT && g.bit == f.bit) {
                            g.v0 *= f.v0;
                            g.v1 *= f.v1;
                            merged = true;
                            break;
                        }
                if (!merged) facl.push_back(f);
            }
            for (const Factor &f : facl) {
                TileDFac<R> d;
                std::memset(&d, 0, sizeof(d));
                d.type = (uint8_t)f.type;
                if (f.type == DF_BIT) {
                    locate(f.bit, &d.tkind, &d.a, &d.tmask);
                    if (d.tkind == TB_REG) {
                        const bool fl = (curF >> d.a) & 1u;
                        cbase *= fl ? f.v1 : f.v0;
                        cu[d.a] *= fl ? f.v0 / f.v1 : f.v1 / f.v0;
                        continue;
                    }
                    if (is_pm1(f.v0) && is_pm1(f.v1)) {  // +-1 values: a sign under the bit
                        cbase *= f.v0;
                        if (f.v1 != f.v0) {
                            TileDFac<R> sg;
                            std::memset(&sg, 0, sizeof(sg));
                            sg.type = DF_SIGN;
                            sg.a = 0x80;
                            if (d.tkind == TB_THREAD) sg.mt = (uint32_t)d.tmask;
                            else sg.mo = d.tmask;
                            signs.push_back(sg);
                        }
                        continue;
                    }
                    d.v0 = mkc<R>((R)f.v0.real(), (R)f.v0.imag());
                    d.v1 = mkc<R>((R)f.v1.real(), (R)f.v1.imag());
                    (d.tkind == TB_OUTSIDE ? outside : single).push_back(d);
                } else {
                    split(f.mask, &d.mr, &d.mt, &d.mo);
                    const int nr = __builtin_popcount(d.mr);
                    const bool sign = f.v0 == cd(-1.0, 0.0);
                    if (nr >= 2 && sign) {  // a sign flip of registers
                        TileOp fo;
                        std::memset(&fo, 0, sizeof(fo));
                        fo.type = TOP_FLIP;
                        fo.a = (uint8_t)__builtin_ctz(d.mr);
                        const uint8_t rest = (uint8_t)(d.mr & (d.mr - 1));
                        fo.b = (uint8_t)__builtin_ctz(rest);
                        fo.mr = (uint8_t)(rest & (rest - 1));
                        fo.tkind = (uint8_t)(((curF >> fo.a) & 1u) | (((curF >> fo.b) & 1u) << 1));
                        fo.fx = (uint8_t)(curF & fo.mr);
                        fo.mt = d.mt;
                        fo.mo = d.mo;
                        flips.push_back(fo);
                        continue;
                    }
                    const bool fl1 = nr == 1 && (curF & d.mr) != 0;  // one register bit, in the frame
                    if (d.mt == 0 && d.mo == 0) {        // register bits alone
                        if (nr == 0) {
                            cbase *= f.v0;
                        } else if (nr == 1) {
                            if (fl1) {
                                cbase *= f.v0;
                                cu[__builtin_ctz(d.mr)] /= f.v0;
                            } else {
                                cu[__builtin_ctz(d.mr)] *= f.v0;
                            }
                        } else {
                            d.v0 = mkc<R>((R)f.v0.real(), (R)f.v0.imag());
                            d.tmask = reg_pattern(d.mr);
                            pair.push_back(d);
                        }
                        continue;
                    }
                    if (sign && nr <= 1) {                // negate the base or one ratio
                        d.type = DF_SIGN;
                        d.a = nr ? (uint8_t)(d.mr | (fl1 ? 0x80 : 0)) : (uint8_t)0x80;
                        d.mr = 0;
                        signs.push_back(d);
                        continue;
                    }
                    d.v0 = mkc<R>((R)f.v0.real(), (R)f.v0.imag());
                    if (d.mr == 0 && d.mt == 0) {         // outside bits alone
                        outside.push_back(d);
                        continue;
                    }
                    if (fl1) {  // v0 where the register bit is 0: v0 on all, 1 / v0 where it is 1
                        TileDFac<R> d0 = d;
                        d0.mr = 0;
                        d0.tmask = reg_pattern(0);
                        single.push_back(d0);
                        const cd iv = 1.0 / f.v0;
                        d.v0 = mkc<R>((R)iv.real(), (R)iv.imag());
                        d.tmask = 0;
                        single.push_back(d);
                        continue;
                    }
                    d.tmask = reg_pattern(d.mr);
                    (nr >= 2 ? pair : single).push_back(d);
                }
            }
            const int nf = (int)(outside.size() + signs.size() + single.size() + pair.size());
            if (ndf + nf > kTileMaxDFac || nf > 255 || (int)outside.size() > 255 || (int)signs.size() > 255)
                return overflow();
            if (nmat + 1 + RB > kTileMaxMat) return overflow();
            if (nops + 1 + (int)flips.size() > kTileMaxOps) return overflow();
            bool trivial = nf == 0 && cbase == cd(1.0);
            for (int x = 0; x < RB; ++x) trivial = trivial && cu[x] == cd(1.0);
            for (const TileOp &fo : flips) P.op[nops++] = fo;
            P.st[nst - 1].op_end = (uint16_t)nops;
            if (trivial) continue;                // flips only
            op.type = TOP_DBLOCK;
            op.m = nmat;                     // constants: base, ratios u[0..RB)
            put(cbase);
            for (int x = 0; x < RB; ++x) put(cu[x]);
            op.mo = (uint64_t)ndf;           // first factor
            op.b = (uint8_t)nf;
            op.a = (uint8_t)pair.size();
            op.gl = (uint8_t)outside.size();
            op.tkind = (uint8_t)signs.size();
            for (auto &d : outside) P.dfac[ndf++] = d;
            for (auto &d : signs) P.dfac[ndf++] = d;
            for (auto &d : single) P.dfac[ndf++] = d;
            for (auto &d : pair) P.dfac[ndf++] = d;
        } else {
            const LGate &g = G[e.gi];
            const GClass c = cls[e.gi];
            const int sl = slot[e.gi];
            if (nmat + (sl >= 0 ? 0 : mat_entries(c)) > kTileMaxMat) return overflow();
            if (c == G_GRAD && ngrad >= kTileMaxGrad) return overflow();
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
                locate(g.tbit[0], &op.tkind, &op.a, &op.tmask);
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
                if (sl >= 0 && ((cur >> lb) & 1u) && (g.kind == QS_GATE_RY || g.kind == QS_GATE_RX)) {
                    // per-member rotation: cos and sin from the member's table
                    op.type = TOP_PROT;
                    op.a = (uint8_t)regidx(lb);
                    op.b = g.kind == QS_GATE_RX ? 1 : 0;
                    split(g.cmask, &op.mr, &op.mt, &op.mo);
                    op.pm = 1;
                    op.m = 4 * sl;
                    break;
                }
                if (!((cur >> lb) & 1u)) {
                    op.type = TOP_DENSE1_L;
                    op.a = (uint8_t)lane_index(lb);
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
                    for (int x = 0; x < 4; ++x) put(g.m[x]);
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
                    auto perm = [&](int l) { return sw ? (((l & 1) << 1) | (l >> 1)) : l; };
                    for (int r = 0; r < 4; ++r)
                        for (int cc = 0; cc < 4; ++cc) put(g.m[perm(r) * 4 + perm(cc)]);
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
                op.m = (uint32_t)nising++;  // index of the op's table
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
                const int lb = loc_of[g.tbit[0]];
                if (g.grad_gen == GEN_Z) {
                    locate(g.tbit[0], &op.tkind, &op.a, &op.tmask);
                } else if (!((cur >> lb) & 1u)) {
                    op.tkind = TB_THREAD;  // lane bit: shuffles
                    op.a = (uint8_t)lane_index(lb);
                } else {
                    op.tkind = TB_REG;
                    op.a = (uint8_t)regidx(lb);
                }
                break;
            }
            default:
                break;
            }
        }
        P.op[nops++] = op;
        P.st[nst - 1].op_end = (uint16_t)nops;
    }
    if (!flush_third()) return overflow();
    // the last stage stores the tile through its own lane map when every warp
    // store covers whole 32-byte sectors (index bits 0 and 1 on lanes for
    // complex64, bit 0 for complex128); otherwise one more stage puts the lanes
    // back on the 5 lowest bits
    {
        const TileStage &last = P.st[nst - 1];
        const uint32_t sector_bits = sizeof(R) == 4 ? 3u : 1u;
        uint32_t lanes = 0;
        for (int x = 0; x < kTileLaneBits; ++x) lanes |= 1u << last.lloc[x];
        if ((lanes & sector_bits) != sector_bits) {
            if (nst >= kTileMaxStages) return overflow();
            open_stage(choose(ne, 0u, highmask), natural);
        }
    }
    P.st[nst - 1].rflip = (uint8_t)curF;  // the store undoes the last stage's frame
    P.n_stages = nst;
    P.n_grad = ngrad;
    if (dry_stages) {  // planning only: report the stage count
        *dry_stages = nst;
        return QS_OK;
    }
    // per-transpose swizzles and register offsets; which stages test thread bits
    uint64_t rng = 0x9e3779b97f4a7c15ull;
    for (int t = 1; t < nst; ++t) set_transpose<R>(P.st[t - 1], P.st[t], k, &rng);
    for (int t = 0; t < nst; ++t) {
        TileStage &st = P.st[t];
        st.need_lt = 0;
        for (int o = st.op_begin; o < st.op_end; ++o) {
            const TileOp &op = P.op[o];
            bool uses = op.mt != 0;
            if (op.type == TOP_DBLOCK) uses = uses || op.b > op.gl;  // thread, mixed or pair factors
            else if (op.type != TOP_ROTS_R && op.type != TOP_ROTS_L && op.type != TOP_FLIP) uses = true;
            st.need_lt |= uses ? 1 : 0;
        }
    }
    static const bool stats = std::getenv("QSIM_PLAN_STATS") != nullptr;
    if (stats) {
        int cnt[16] = {0};
        for (int o = 0; o < nops; ++o) cnt[P.op[o].type & 15]++;
        int rots = 0, threes = 0, frames = 0;
        for (int o = 0; o < nops; ++o) {
            if (P.op[o].type == TOP_ROTS_R)
                for (int j = 0; j < RB; ++j) {
                    if (!((P.op[o].a >> j) & 1u)) continue;
                    ++rots;
                    threes += P.mat[P.op[o].m + j].y == (R)0;  // third shears
                }
            if (P.op[o].type == TOP_ROTS_L)
                for (int j = 0; j < 5; ++j) rots += P.mat[P.op[o].m + j].y != (R)0;
        }
        for (int t = 0; t < nst; ++t) frames += __builtin_popcount(P.st[t].rflip);
        std::fprintf(stderr,
                     "[qsim plan] gates %zu entries %d stages %d ops %d: rots_r %d rots_l %d (rotations %d) "
                     "third shears %d, frame bits at stage ends %d dblock %d (factors %d) dense1 %d phase %d diag1 %d other %d\n",
                     pp.gates.size(), ne, nst, nops, cnt[TOP_ROTS_R], cnt[TOP_ROTS_L], rots, threes, frames,
                     cnt[TOP_DBLOCK], ndf,
                     cnt[TOP_DENSE1_R] + cnt[TOP_DENSE1_L], cnt[TOP_PHASE], cnt[TOP_DIAG1],
                     nops - cnt[TOP_ROTS_R] - cnt[TOP_ROTS_L] - cnt[TOP_DBLOCK] - cnt[TOP_DENSE1_R] -
                         cnt[TOP_DENSE1_L] - cnt[TOP_PHASE] - cnt[TOP_DIAG1]);
    }
    if (prof_enabled()) {
        // algorithmic flops per amplitude: 16 for a 2x2 complex gate, 64 for 4x4,
        // 6 for a diagonal factor, 4 for a rotation, 12 for a diagonal
        // block; scaled by the touched fraction 2^-(required bits)
        const double amps = (double)((uint64_t)s->batch << n);
        double fl = 0.0;
        for (int i = 0; i < ne; ++i) {
            if (ent[i].kind == E_ROT) {
                fl += 4.0 * amps;
                continue;
            }
            if (ent[i].kind == E_BLOCK) {
                if (!ent[i].fac.empty()) fl += 12.0 * amps;
                continue;
            }
            const LGate &g = G[ent[i].gi];
            const GClass c = cls[ent[i].gi];
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
    if (nising > 0) {
        // the Ising ops' tile-independent tables, once per pass
        const int threads = tile_threads(s->dtype);
        const uint32_t stride = ising_thr_stride(RB, threads, k, P.n_free);
        const size_t doubles = (size_t)nising * s->batch * stride;
        if (s->ithr_bytes < doubles * sizeof(double)) {
            if (s->ithr) {
                QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
                cudaFree(s->ithr);
                s->ithr = nullptr;
                s->ithr_bytes = 0;
            }
            QS_CUDA_TRY(cudaMalloc(&s->ithr, doubles * sizeof(double)));
            s->ithr_bytes = doubles * sizeof(double);
        }
        P.ising_thr = s->ithr;
        P.ising_thr_stride = stride;
        for (int st = 0; st < nst; ++st)
            for (int o = P.st[st].op_begin; o < P.st[st].op_end; ++o) {
                const TileOp &op = P.op[o];
                if (op.type != TOP_ISING) continue;
                IsingTabP tp;
                std::memset(&tp, 0, sizeof(tp));
                tp.tb = kTileLaneBits + TileCfg<R>::WB;
                tp.rb = RB;
                for (int i = 0; i < kTileLaneBits; ++i) tp.tg[i] = (int8_t)P.gbit[P.st[st].lloc[i]];
                for (int w = 0; w < TileCfg<R>::WB; ++w) tp.tg[kTileLaneBits + w] = (int8_t)P.gbit[P.st[st].wloc[w]];
                for (int j = 0; j < RB; ++j) tp.rg[j] = (int8_t)P.gbit[P.st[st].rloc[j]];
                tp.k = k;
                tp.n_free = P.n_free;
                for (int i = 0; i < k; ++i) tp.gb[i] = (int8_t)P.gbit[i];
                tp.tins = P.tins;
                std::memcpy(&tp.tau, &op.tmask, sizeof(double));
                tp.ising = s->itab;
                tp.ising_stride = s->ising_stride;
                tp.nq = n;
                tp.stride = stride;
                tp.members = s->batch;
                tp.single = sizeof(R) == 4 ? 1 : 0;
                tp.out = s->ithr + (size_t)op.m * s->batch * stride;
                QS_TRY(k_ising_table(s, tp));
            }
    }
    if constexpr (sizeof(R) == 4)
        return k_tiled_pass_c64(s, P);
    else
        return k_tiled_pass_c128(s, P);
}

// Orders of a pass's gates that keep every dependency: the queue order, then
// the gates split into maximal runs of mutually commuting gates (disjoint
// qubits, or both diagonal; gradient ops end a run) with alternate runs
// reversed, once with the last run reversed and once with the second. Which
// bits a pass's first and last stages hold, and how consecutive runs share
// register bits, depends on these orders.
static std::vector<std::vector<int>> run_orders(const std::vector<LGate> &G, const std::vector<GClass> &cls,
                                                const std::vector<int> &gates) {
    auto diag = [&](int i) { return cls[i] == G_PHASE || cls[i] == G_DIAG1 || cls[i] == G_ISING; };
    // the Ising phase acts on every bit (its gate lists none)
    auto bits = [&](int i) { return cls[i] == G_ISING ? ~0ull : qubit_bits(G[i]); };
    std::vector<std::vector<int>> runs;
    for (int gi : gates) {
        bool joins = !runs.empty() && cls[gi] != G_GRAD;
        if (joins)
            for (int h : runs.back()) {
                const bool commute = cls[h] != G_GRAD && ((bits(gi) & bits(h)) == 0 || (diag(gi) && diag(h)));
                if (!commute) {
                    joins = false;
                    break;
                }
            }
        if (joins)
            runs.back().push_back(gi);
        else
            runs.push_back({gi});
    }
    std::vector<std::vector<int>> out = {gates};
    const int nr = (int)runs.size();
    for (int variant = 0; variant < 2; ++variant) {
        std::vector<int> o;
        for (int r = 0; r < nr; ++r) {
            const bool rev = variant == 0 ? ((nr - 1 - r) % 2 == 0) : (r % 2 == 1);
            if (rev)
                o.insert(o.end(), runs[r].rbegin(), runs[r].rend());
            else
                o.insert(o.end(), runs[r].begin(), runs[r].end());
        }
        if (o != gates) out.push_back(o);
    }
    return out;
}

qs_status trotter_queue(int n, const std::vector<double> &a0, const std::vector<double> &a1,
                        const std::vector<double> &taus, const std::vector<double> &svals, double dt, bool ising,
                        std::vector<LGate> *G) {
    G->clear();
    auto one_qubit = [&](int kind, int q, double angle) {
        qs_gate g;
        std::memset(&g, 0, sizeof(g));
        g.kind = kind;
        g.n_targets = 1;
        g.targets[0] = q;
        g.param_index = -1;
        g.params[0] = angle;
        LGate lg;
        QS_TRY(lower_gate(n, g, &lg));
        lg.paeth = kind == QS_GATE_RY;
        G->push_back(lg);
        return QS_OK;
    };
    auto ising_phase = [&](double tau) {
        if (tau == 0.0 || !ising) return;
        LGate g;
        g.kind = kKindIsing;
        g.k = 0;
        g.diagonal = true;
        g.m.assign(1, cd(tau, 0.0));
        G->push_back(g);
    };
    for (int q = 0; q < n; ++q) QS_TRY(one_qubit(QS_GATE_S, q, 0.0));
    for (size_t k = 0; k < svals.size(); ++k) {
        ising_phase(taus[k]);
        for (int q = 0; q < n; ++q) {
            const double a = (1.0 - svals[k]) * a0[q] + svals[k] * a1[q];
            if (a != 0.0) QS_TRY(one_qubit(QS_GATE_RY, q, 2.0 * dt * a));
        }
    }
    ising_phase(taus[svals.size()]);
    for (int q = 0; q < n; ++q) QS_TRY(one_qubit(QS_GATE_SDG, q, 0.0));
    return QS_OK;
}

thread_local TileSchedule t_schedule;
TileSchedule tile_schedule() { return t_schedule; }
void set_tile_schedule(TileSchedule s) { t_schedule = s; }

qs_status run_tiled(qs_state *s, const std::vector<LGate> &G, const double *params, int n_params, int force_bit,
                    double *gpart, double param_sign) {
    const TileSchedule sched = t_schedule;
    const int max_gates = sched.max_gates > 0 ? std::min(sched.max_gates, kTileMaxOps) : kTileMaxOps;
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
    // complex128 passes read a double-float table (their kernels are
    // double-float unless FP64 is asked for)
    if (!spidx.empty())
        QS_TRY(k_param_table(s, spidx, skind, params, n_params, param_sign, &pm_stride,
                             s->dtype == QS_C128 && !c128_fp64()));
    std::vector<char> done(G.size(), 0);
    size_t first = 0;
    while (true) {
        while (first < G.size() && done[first]) ++first;
        if (first >= G.size()) break;
        // gates from `first` on that can join a pass: a gate joins if it commutes
        // past the gates skipped so far and its dense targets fit the tile's high
        // bits, which are either taken greedily as gates need them or fixed
        const uint64_t all_bits = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
        auto select = [&](bool fixed, uint64_t fixed_high, PassPlan *out) {
            out->high = force | fixed_high;
            out->gates.clear();
            uint64_t blocked = 0;
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
                if (fixed ? (nb & ~out->high) != 0 : __builtin_popcountll(out->high | nb) > nh) {
                    blocked |= qb;
                    continue;
                }
                out->high |= nb;
                out->gates.push_back((int)i);
                if ((int)out->gates.size() >= max_gates) break;
            }
        };
        PassPlan pp;
        if (sched.select != 2) select(false, 0, &pp);
        // high bits fixed to a window of consecutive index bits: circuits with
        // nearest-neighbour structure keep a whole light cone inside one window;
        // the window (or the greedy choice) that takes the most gates wins
        if (sched.select != 1) {
            const int w = nh - __builtin_popcountll(force);
            const int top = force_bit >= 0 ? force_bit : n;
            for (int b = kTileLaneBits; w > 0 && b + w <= top; ++b) {
                PassPlan q;
                select(true, ((1ull << w) - 1ull) << b, &q);
                if (q.gates.size() > pp.gates.size()) pp = std::move(q);
            }
            if (pp.gates.empty() && sched.select == 2) select(false, 0, &pp);
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
        // order: the fewest stages among the queue order and two orders that
        // reverse alternate runs of mutually commuting gates
        if (pp.gates.size() > 1) {
            std::vector<std::vector<int>> cand = run_orders(G, cls, pp.gates);
            int best = -1, best_stages = std::numeric_limits<int>::max();
            for (size_t c = 0; c < cand.size(); ++c) {
                PassPlan q = pp;
                q.gates = cand[c];
                bool fits = true;
                int stages = 0;
                if (s->dtype == QS_C64)
                    QS_TRY(emit_and_run<float>(s, G, cls, slot, pm_stride, q, force_bit, gpart, &fits, &stages));
                else
                    QS_TRY(emit_and_run<double>(s, G, cls, slot, pm_stride, q, force_bit, gpart, &fits, &stages));
                if (fits && stages < best_stages) {
                    best_stages = stages;
                    best = (int)c;
                }
            }
            if (best > 0) pp.gates = cand[best];
        }
        // emit; a pass over the descriptor's capacity is retried with a prefix of
        // its gates (a prefix keeps every dependency)
        while (true) {
            bool fits = true;
            if (s->dtype == QS_C64)
                QS_TRY(emit_and_run<float>(s, G, cls, slot, pm_stride, pp, force_bit, gpart, &fits));
            else
                QS_TRY(emit_and_run<double>(s, G, cls, slot, pm_stride, pp, force_bit, gpart, &fits));
            if (fits) break;
            if (pp.gates.size() <= 1) {
                set_error("tiled planner cannot fit a single gate");
                return QS_ERR_CUDA;
            }
            pp.gates.resize(pp.gates.size() * 3 / 4);
        }
        for (int gi : pp.gates) done[gi] = 1;
    }
    return QS_OK;
}

}  // namespace qsim
