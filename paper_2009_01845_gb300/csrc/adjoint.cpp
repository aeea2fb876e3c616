// Adjoint gradient driver: qs_energy_gradient.
//
// For E(theta) = Re <psi(theta)|H|psi(theta)>, psi = U_N .. U_1 |psi_0>:
//   forward: phi = psi (tiled passes, per-member angles);
//   seed:    lambda = H phi, E = Re <phi|lambda>;
//   sweep:   for j = N .. 1: if U_j = exp(-i theta_j P_j / 2) is parametrised,
//            dE/dtheta_j = Im <lambda|P_j|phi> (P_j with U_j's controls);
//            for U1/CU1 (exp(i theta Pi)) dE/dtheta_j = -2 Im <lambda|Pi|phi>;
//            then phi <- U_j^dag phi, lambda <- U_j^dag lambda.
// phi and lambda of member b are the two halves of a (B, 2, 2^n) buffer, i.e.
// one (n+1)-qubit state whose top index bit tells them apart, so every U_j^dag
// of the sweep is one ordinary tiled op on both, and a gradient op sees phi_x
// and lambda_x in the same thread's registers. Checkpoints (every k gates)
// store phi during the forward pass and replace the uncomputed phi at each
// segment boundary of the sweep, bounding uncompute drift.
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "adjoint.h"
#include "plan.h"
#include "prof.h"
#include "tiled.h"

namespace qsim {

static size_t amp_size(qs_dtype d) { return d == QS_C64 ? 8 : 16; }

// run `fn` on a shallow copy of `base` re-shaped as a view; buffers the copy
// (re)allocates are handed back to `base`
template <typename F>
static qs_status with_view(qs_state *base, int n, int ms, size_t offset_amps, F fn) {
    qs_state v = *base;
    v.n = n;
    v.ms = ms;
    v.data = (char *)base->data + offset_amps * amp_size(base->dtype);
    v.owns = false;
    const qs_status st = fn(&v);
    base->scratch = v.scratch;
    base->scratch_doubles = v.scratch_doubles;
    base->gtab = v.gtab;
    base->gtab_bytes = v.gtab_bytes;
    base->ptab = v.ptab;
    base->ptab_bytes = v.ptab_bytes;
    base->ptab_dd = v.ptab_dd;
    base->itab = v.itab;
    base->itab_bytes = v.itab_bytes;
    base->ithr = v.ithr;
    base->ithr_bytes = v.ithr_bytes;
    base->host_pinned = v.host_pinned;
    base->host_pinned_doubles = v.host_pinned_doubles;
    return st;
}

static int generator_of(int kind) {
    switch (kind) {
    case QS_GATE_RX: return GEN_X;
    case QS_GATE_RY: return GEN_Y;
    case QS_GATE_RZ: return GEN_Z;
    case QS_GATE_U1: case QS_GATE_CU1: return GEN_PROJ;
    default: return -1;
    }
}

static LGate inverse_of(const LGate &g) {
    LGate h = g;
    const int K = 1 << g.k;
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) h.m[r * K + c] = std::conj(g.m[c * K + r]);
    return h;
}

// copy phi (member stride 2^(n+1)) to / from a contiguous checkpoint
static qs_status copy_phi(qs_state *w, void *ckpt, bool to_ckpt) {
    const size_t row = ((size_t)1 << (w->n - 1)) * amp_size(w->dtype);
    const size_t pitch = 2 * row;
    if (to_ckpt)
        QS_CUDA_TRY(cudaMemcpy2DAsync(ckpt, row, w->data, pitch, row, w->batch, cudaMemcpyDeviceToDevice, w->stream));
    else
        QS_CUDA_TRY(cudaMemcpy2DAsync(w->data, pitch, ckpt, row, row, w->batch, cudaMemcpyDeviceToDevice, w->stream));
    return QS_OK;
}

qs_status energy_gradient(qs_state *w, const std::vector<LGate> &G, const double *params, int n_params,
                          const qs_pauli_term *terms, size_t n_terms, int init_zero, double *energy,
                          double *grad, int ckpt_every, int mode) {
    const int n = w->n - 1;  // qubits of the circuit
    const int B = w->batch;
    const size_t half = (size_t)1 << n;
    const int N = (int)G.size();
    const int seg = ckpt_every > 0 ? ckpt_every : N;
    const int nseg = N > 0 ? (N + seg - 1) / seg : 0;
    std::vector<void *> ckpt;
    auto cleanup = [&]() {
        for (void *p : ckpt)
            if (p) cudaFreeAsync(p, w->stream);
    };
    const size_t ckpt_bytes = half * amp_size(w->dtype) * (size_t)B;
    for (int c = 1; c < nseg; ++c) {
        void *p = nullptr;
        const cudaError_t e = cudaMallocAsync(&p, ckpt_bytes, w->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_status(e, "cudaMallocAsync(checkpoint)");
        }
        ckpt.push_back(p);
    }
    qs_status st = QS_OK;
    if (mode != QS_GRAD_SWEEP) {
    // ---------------- forward on phi, checkpoint at segment ends
    st = with_view(w, n, n + 1, 0, [&](qs_state *phi) -> qs_status {
        if (init_zero) QS_TRY(k_init_basis(phi, 0));
        for (int c = 0; c < nseg; ++c) {
            std::vector<LGate> part(G.begin() + (size_t)c * seg, G.begin() + std::min<size_t>(N, (size_t)(c + 1) * seg));
            QS_TRY(run_tiled(phi, part, params, n_params));
            if (c + 1 < nseg) QS_TRY(copy_phi(w, ckpt[c], true));
        }
        return QS_OK;
    });
    if (st != QS_OK) {
        cleanup();
        return st;
    }
    // ---------------- lambda = H phi, E = Re <phi|lambda>
    const StateView vphi{w->data, n, n + 1, B, w->dtype};
    const StateView vlam{(char *)w->data + half * amp_size(w->dtype), n, n + 1, B, w->dtype};
    st = k_pauli_apply(vphi, vlam, terms, n_terms, w->stream);
    if (st == QS_OK) st = ensure_scratch(w, (size_t)2 * B * 1024 + 2 * (size_t)B);
    if (st == QS_OK) {
        double *dotout = w->scratch + (size_t)2 * B * 1024;
        st = k_dot(vphi, vlam, w->scratch, (size_t)2 * B * 1024, dotout, w->stream);
        if (st == QS_OK && energy) {
            const cudaError_t e = cudaMemcpy2DAsync(energy, sizeof(double), dotout, 2 * sizeof(double),
                                                    sizeof(double), B, cudaMemcpyDeviceToDevice, w->stream);
            if (e != cudaSuccess) st = cuda_status(e, "energy copy");
        }
    }
    if (st != QS_OK || mode == QS_GRAD_FORWARD) {
        cleanup();
        return st;
    }
    }  // forward
    // ---------------- reverse sweep with gradient ops, segment by segment
    std::vector<int> slot_param;        // gradient slot -> parameter column
    std::vector<float> slot_coef;
    std::vector<std::vector<LGate>> rev(nseg);
    for (int j = N - 1; j >= 0; --j) {
        const LGate &g = G[j];
        const int c = j / seg;
        if (g.param_index >= 0) {
            LGate d = g;
            d.kind = kKindGrad;
            d.grad_gen = generator_of(g.kind);
            d.grad_slot = (int)slot_param.size();
            d.param_index = -1;
            slot_param.push_back(g.param_index);
            slot_coef.push_back(d.grad_gen == GEN_PROJ ? -2.0f : 1.0f);
            rev[c].push_back(d);
            rev[c].push_back(g);  // angle negated through the sweep's parameter sign
        } else {
            rev[c].push_back(inverse_of(g));
        }
    }
    const int k = tile_bits(w->dtype);
    const bool small = n + 1 < k;  // below one tile: unfused sweep
    const uint64_t total_tiles = small ? (uint64_t)B : (uint64_t)B << (n + 1 - k);
    double *gpart = nullptr;
    const size_t nslot = slot_param.size();
    if (nslot) {
        const cudaError_t e = cudaMallocAsync(&gpart, sizeof(double) * nslot * total_tiles, w->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_status(e, "cudaMallocAsync(gradient partials)");
        }
    }
    for (int c = nseg - 1; c >= 0 && st == QS_OK; --c) {
        if (small) {
            for (const LGate &g : rev[c]) {
                if (g.kind == kKindGrad)
                    st = k_grad_small(w, g, gpart + (size_t)g.grad_slot * total_tiles);
                else if (g.param_index >= 0)
                    st = k_apply_param_gate(w, g, params, n_params, -1.0);
                else
                    st = k_apply_unfused(w, g);
                if (st != QS_OK) break;
            }
        } else {
            st = run_tiled(w, rev[c], params, n_params, /*force_bit=*/n, gpart, /*param_sign=*/-1.0);
        }
        if (st == QS_OK && c > 0) st = copy_phi(w, ckpt[c - 1], false);
    }
    // ---------------- dE/dtheta, deterministic reduction per parameter
    if (st == QS_OK) {
        std::vector<std::vector<int>> rows(n_params);
        for (size_t sl = 0; sl < nslot; ++sl) rows[slot_param[sl]].push_back((int)sl);
        for (int p0 = 0; p0 < n_params && st == QS_OK;) {
            GradReduceP rp;
            std::memset(&rp, 0, sizeof(rp));
            int nr = 0, ns = 0;
            while (p0 + nr < n_params && nr < kGRMaxRows && ns + (int)rows[p0 + nr].size() <= kGRMaxSlots) {
                rp.beg[nr] = ns;
                for (int sl : rows[p0 + nr]) {
                    rp.slot[ns] = sl;
                    rp.coef[ns] = slot_coef[sl];
                    ++ns;
                }
                ++nr;
            }
            rp.beg[nr] = ns;
            if (nr == 0) {
                st = QS_ERR_UNSUPPORTED;
                set_error("too many gates share one parameter");
                break;
            }
            rp.total_tiles = total_tiles;
            rp.tiles_per_member = total_tiles / B;
            rp.n_params = n_params;
            rp.param0 = p0;
            st = k_grad_reduce(gpart, rp, nr, B, grad, w->stream);
            p0 += nr;
        }
    }
    if (gpart) cudaFreeAsync(gpart, w->stream);
    cleanup();
    return st;
}

}  // namespace qsim
