// Fusion planner for the tensor-core block path (see fused.h).
#include <algorithm>
#include <cstring>

#include "fused.h"
#include "plan.h"

namespace qsim {

namespace {

uint64_t gate_bits(const LGate &g) {
    uint64_t m = g.cmask;
    for (int j = 0; j < g.k; ++j) m |= 1ull << g.tbit[j];
    return m;
}

struct Item {
    bool block;
    uint64_t bits;            // block: its qubits (index bits)
    std::vector<int> gates;   // gate indices in queue order
};

// v <- g v on a 32-amplitude register whose local bit (4 - j) is index bit bits[j]
void apply_local(const LGate &g, const int *bits, std::vector<cd> &v) {
    auto local = [&](int b) {
        for (int j = 0; j < 5; ++j)
            if (bits[j] == b) return 4 - j;
        return -1;
    };
    const int K = 1 << g.k;
    int tl[QS_MAX_TARGETS];
    uint64_t tmask = 0, cmask = 0;
    for (int j = 0; j < g.k; ++j) {
        tl[j] = local(g.tbit[j]);
        tmask |= 1ull << tl[j];
    }
    for (int b = 0; b < 64; ++b)
        if ((g.cmask >> b) & 1ull) cmask |= 1ull << local(b);
    std::vector<cd> in(K), out(K);
    for (int base = 0; base < 32; ++base) {
        if (base & tmask) continue;
        if ((base & cmask) != cmask) continue;
        auto idx = [&](int l) {
            int x = base;
            for (int j = 0; j < g.k; ++j)
                if ((l >> (g.k - 1 - j)) & 1) x |= 1 << tl[j];
            return x;
        };
        for (int c = 0; c < K; ++c) in[c] = v[idx(c)];
        for (int r = 0; r < K; ++r) {
            cd acc = 0.0;
            for (int c = 0; c < K; ++c) acc += g.m[r * K + c] * in[c];
            out[r] = acc;
        }
        for (int r = 0; r < K; ++r) v[idx(r)] = out[r];
    }
}

}  // namespace

qs_status run_fused(qs_state *s, const std::vector<LGate> &G, int width, const double *params, int n_params) {
    if (s->dtype != QS_C64 || s->n < 11) return run_tiled(s, G, params, n_params);
    if (width <= 0 || width > 5) width = 5;
    const int n = s->n;
    std::vector<Item> items;
    std::vector<int> last(64, -1);  // latest item touching each index bit
    for (size_t i = 0; i < G.size(); ++i) {
        const LGate &g = G[i];
        const uint64_t gb = gate_bits(g);
        int after = -1;
        for (int b = 0; b < 64; ++b)
            if ((gb >> b) & 1ull) after = std::max(after, last[b]);
        const bool fusable = g.param_index < 0 && __builtin_popcountll(gb) <= width;
        int target = -1;
        if (fusable) {
            // the block at or after `after` with room that shares the most qubits
            int best_overlap = -1;
            for (int it = (int)items.size() - 1; it >= std::max(after, 0); --it) {
                if (!items[it].block) continue;
                if (__builtin_popcountll(items[it].bits | gb) > width) continue;
                const int ov = __builtin_popcountll(items[it].bits & gb);
                if (ov > best_overlap) {
                    best_overlap = ov;
                    target = it;
                }
            }
            if (target < after) target = -1;
        }
        if (target < 0) {
            items.push_back(Item{fusable, fusable ? gb : 0ull, {}});
            target = (int)items.size() - 1;
        }
        items[target].bits |= fusable ? gb : 0ull;
        items[target].gates.push_back((int)i);
        for (int b = 0; b < 64; ++b)
            if ((gb >> b) & 1ull) last[b] = target;
    }
    for (const Item &it : items) {
        if (!it.block) {
            for (int gi : it.gates) {
                const LGate &g = G[gi];
                if (g.param_index >= 0)
                    QS_TRY(k_apply_param_gate(s, g, params, n_params));
                else
                    QS_TRY(k_apply_unfused(s, g));
            }
            continue;
        }
        // exactly five bits: pad with the lowest bits outside the block
        int bits[5], nb = 0;
        for (int b = n - 1; b >= 0 && nb < 5; --b)
            if ((it.bits >> b) & 1ull) bits[nb++] = b;
        for (int b = 0; b < n && nb < 5; ++b)
            if (!((it.bits >> b) & 1ull)) {
                bool used = false;
                for (int j = 0; j < nb; ++j) used |= bits[j] == b;
                if (!used) bits[nb++] = b;
            }
        std::vector<cd> U(1024, 0.0), v(32);
        for (int c = 0; c < 32; ++c) {
            std::fill(v.begin(), v.end(), cd(0.0));
            v[c] = 1.0;
            for (int gi : it.gates) apply_local(G[gi], bits, v);
            for (int r = 0; r < 32; ++r) U[r * 32 + c] = v[r];
        }
        QS_TRY(k_fused5(s, U, bits));
    }
    return QS_OK;
}

}  // namespace qsim
