// Exact time evolution (Sec. 2.6: the "exp" solver and the Runge-Kutta
// integrators of i d/dt psi = H(t) psi) and the schedule gradient of the
// Trotterised adiabatic evolution (Sec. 4: the schedule is optimised for the
// final energy).
//
// H(t) = (1 - s) H0 + s H1 with s = t / T. H is never a matrix here: every
// solver step is a few applications of the Pauli sum to a state (the adjoint
// module's H psi kernel) and linear combinations of states (kernels_evolve.cu),
// so the solvers run at any n the memory holds.
//   exp:  psi <- exp(-i dt H(s_mid)) psi, s_mid at the step's midpoint, by its
//         Taylor series on the state: the step is cut into m pieces of length
//         tau with ||H|| tau <= 1 (||H|| <= sum |c|), each summed to the order K
//         where the remainder bound (||H|| tau)^(K+1) / (K+1)! falls below the
//         precision's unit roundoff;
//   rk4:  the classical fourth-order Runge-Kutta step;
//   rk45: the fifth-order solution of the Dormand-Prince 5(4) pair, fixed step.
// The schedule gradient runs K Trotter steps with the given s_k, then one
// reverse sweep over (phi, lambda = H1 phi) that undoes each factor of each
// step on both and reads <lambda|G|phi> for the generators G that the
// factor's derivative inserts (see qs_schedule_gradient in qsim.h).
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "adjoint.h"
#include "internal.h"
#include "plan.h"

namespace qsim {

qs_status k_combine(qs_dtype dtype, void *out, const std::vector<const void *> &in, const std::vector<cd> &c,
                    uint64_t total, cudaStream_t st);

namespace {

size_t amp_bytes_of(qs_dtype d) { return d == QS_C64 ? 8 : 16; }

// device scratch states owned by one call
struct Work {
    cudaStream_t st;
    std::vector<void *> bufs;
    ~Work() {
        for (void *p : bufs)
            if (p) cudaFreeAsync(p, st);
    }
    qs_status alloc(size_t bytes, int count) {
        for (int i = 0; i < count; ++i) {
            void *p = nullptr;
            QS_CUDA_TRY(cudaMallocAsync(&p, bytes, st));
            bufs.push_back(p);
        }
        return QS_OK;
    }
};

// the terms of (1 - s) H0 + s H1
std::vector<qs_pauli_term> mix(const qs_pauli_term *h0, size_t n0, const qs_pauli_term *h1, size_t n1, double s) {
    std::vector<qs_pauli_term> t;
    for (size_t i = 0; i < n0; ++i) t.push_back({(1.0 - s) * h0[i].coeff, h0[i].x_mask, h0[i].z_mask});
    for (size_t i = 0; i < n1; ++i) t.push_back({s * h1[i].coeff, h1[i].x_mask, h1[i].z_mask});
    return t;
}

double norm_bound(const std::vector<qs_pauli_term> &t) {
    double v = 0.0;
    for (const auto &x : t) v += std::fabs(x.coeff);
    return v;
}

StateView view(const qs_state *s, void *data) { return StateView{data, s->n, s->n, s->batch, s->dtype}; }

}  // namespace

qs_status run_evolve(qs_state *s, const qs_pauli_term *h0, size_t n0, const qs_pauli_term *h1, size_t n1, double T,
                     double dt, int steps, int solver) {
    const uint64_t total = (uint64_t)s->batch << s->n;
    const size_t bytes = total * amp_bytes_of(s->dtype);
    Work w{s->stream, {}};
    const double eps = s->dtype == QS_C64 ? 6e-8 : 1.2e-16;  // unit roundoff of the state's precision
    auto applyH = [&](const std::vector<qs_pauli_term> &t, void *src, void *dst) {
        return k_pauli_apply(view(s, src), view(s, dst), t.data(), t.size(), s->stream);
    };
    auto comb = [&](void *out, std::vector<const void *> in, std::vector<cd> c) {
        return k_combine(s->dtype, out, in, c, total, s->stream);
    };
    const cd mi(0.0, -1.0);
    if (solver == QS_SOLVER_EXP) {
        QS_TRY(w.alloc(bytes, 2));
        void *term = w.bufs[0], *tmp = w.bufs[1];
        for (int k = 0; k < steps; ++k) {
            const std::vector<qs_pauli_term> H = mix(h0, n0, h1, n1, (k + 0.5) * dt / T);
            const double nu = norm_bound(H);
            const int m = std::max(1, (int)std::ceil(nu * dt));
            const double tau = dt / m;
            // order: the first K with (nu tau)^(K+1) / (K+1)! <= eps
            int K = 1;
            double r = nu * tau;
            for (double b = r; K < 60; ++K) {
                b *= r / (K + 1);
                if (b <= eps) break;
            }
            for (int piece = 0; piece < m; ++piece) {
                QS_TRY(comb(term, {s->data}, {1.0}));
                for (int j = 1; j <= K; ++j) {
                    QS_TRY(applyH(H, term, tmp));
                    QS_TRY(comb(term, {tmp}, {mi * (tau / j)}));
                    QS_TRY(comb(s->data, {s->data, term}, {1.0, 1.0}));
                }
            }
        }
        return QS_OK;
    }
    if (solver == QS_SOLVER_RK4) {
        QS_TRY(w.alloc(bytes, 3));
        void *acc = w.bufs[0], *yt = w.bufs[1], *hk = w.bufs[2];
        void *y = s->data;
        for (int k = 0; k < steps; ++k) {
            const double t = k * dt;
            // stage i: hk = H(t_i) y_i, k_i = -i hk; acc gathers y + dt sum b_i k_i
            QS_TRY(applyH(mix(h0, n0, h1, n1, t / T), y, hk));
            QS_TRY(comb(acc, {y, hk}, {1.0, mi * (dt / 6)}));
            QS_TRY(comb(yt, {y, hk}, {1.0, mi * (dt / 2)}));
            QS_TRY(applyH(mix(h0, n0, h1, n1, (t + dt / 2) / T), yt, hk));
            QS_TRY(comb(acc, {acc, hk}, {1.0, mi * (dt / 3)}));
            QS_TRY(comb(yt, {y, hk}, {1.0, mi * (dt / 2)}));
            QS_TRY(applyH(mix(h0, n0, h1, n1, (t + dt / 2) / T), yt, hk));
            QS_TRY(comb(acc, {acc, hk}, {1.0, mi * (dt / 3)}));
            QS_TRY(comb(yt, {y, hk}, {1.0, mi * dt}));
            QS_TRY(applyH(mix(h0, n0, h1, n1, (t + dt) / T), yt, hk));
            QS_TRY(comb(y, {acc, hk}, {1.0, mi * (dt / 6)}));
        }
        return QS_OK;
    }
    // rk45: Dormand-Prince 5(4) nodes, stage matrix and fifth-order weights
    static const double C[6] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0};
    static const double A[6][5] = {{0, 0, 0, 0, 0},
                                   {1.0 / 5, 0, 0, 0, 0},
                                   {3.0 / 40, 9.0 / 40, 0, 0, 0},
                                   {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0},
                                   {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0},
                                   {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656}};
    static const double Bw[6] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84};
    QS_TRY(w.alloc(bytes, 7));
    void *yt = w.bufs[6];
    void *y = s->data;
    for (int k = 0; k < steps; ++k) {
        const double t = k * dt;
        for (int i = 0; i < 6; ++i) {
            const void *src = y;
            if (i > 0) {
                std::vector<const void *> in = {y};
                std::vector<cd> c = {1.0};
                for (int j = 0; j < i; ++j)
                    if (A[i][j] != 0.0) {
                        in.push_back(w.bufs[j]);
                        c.push_back(mi * (dt * A[i][j]));
                    }
                QS_TRY(comb(yt, in, c));
                src = yt;
            }
            QS_TRY(applyH(mix(h0, n0, h1, n1, (t + C[i] * dt) / T), const_cast<void *>(src), w.bufs[i]));
        }
        std::vector<const void *> in = {y};
        std::vector<cd> c = {1.0};
        for (int j = 0; j < 6; ++j)
            if (Bw[j] != 0.0) {
                in.push_back(w.bufs[j]);
                c.push_back(mi * (dt * Bw[j]));
            }
        QS_TRY(comb(y, in, c));
    }
    return QS_OK;
}

// ------------------------------------------------------------------ schedule gradient
namespace {

struct SplitH {
    std::vector<qs_pauli_term> d0, d1, x0, x1;  // diagonal (Z strings) and X parts of H0, H1
};

qs_status split_for_trotter(int n, const qs_pauli_term *h, size_t count, std::vector<qs_pauli_term> *d,
                            std::vector<qs_pauli_term> *x) {
    for (size_t i = 0; i < count; ++i) {
        if (h[i].x_mask == 0)
            d->push_back(h[i]);
        else if (h[i].z_mask == 0 && __builtin_popcountll(h[i].x_mask) == 1)
            x->push_back(h[i]);
        else {
            set_error("term %zu: the Trotter step takes Z strings and single-qubit X terms", i);
            return QS_ERR_UNSUPPORTED;
        }
    }
    (void)n;
    return QS_OK;
}

// exp(-i tau [(1 - s) D0 + s D1]) on every member of s
qs_status diag_step(qs_state *s, const SplitH &h, double sv, double tau) {
    std::vector<double> c;
    std::vector<uint64_t> z;
    auto add = [&](const std::vector<qs_pauli_term> &t, double w) {
        for (const auto &x : t) {
            uint64_t zb = 0;
            for (int q = 0; q < s->n; ++q)
                if ((x.z_mask >> q) & 1ull) zb |= qbit(s->n, q);
            c.push_back(w * x.coeff);
            z.push_back(zb);
        }
    };
    add(h.d0, 1.0 - sv);
    add(h.d1, sv);
    if (c.empty()) return QS_OK;
    return k_diagonal_evolution(s, c, z, tau);
}

// exp(-i dt X(s)) = prod_q RX(2 dt a_q(s)) on every member of s
qs_status x_step(qs_state *s, const SplitH &h, double sv, double dt) {
    std::vector<double> a(s->n, 0.0);
    for (const auto &t : h.x0) a[__builtin_ctzll(t.x_mask)] += (1.0 - sv) * t.coeff;
    for (const auto &t : h.x1) a[__builtin_ctzll(t.x_mask)] += sv * t.coeff;
    std::vector<LGate> G;
    for (int q = 0; q < s->n; ++q) {
        if (a[q] == 0.0) continue;
        qs_gate g;
        std::memset(&g, 0, sizeof(g));
        g.kind = QS_GATE_RX;
        g.n_targets = 1;
        g.targets[0] = q;
        g.param_index = -1;
        g.params[0] = 2.0 * dt * a[q];
        LGate lg;
        QS_TRY(lower_gate(s->n, g, &lg));
        G.push_back(lg);
    }
    if (G.empty()) return QS_OK;
    return run_gates(s, G, QS_MODE_AUTO, nullptr, nullptr, 0);
}

}  // namespace

qs_status run_schedule_gradient(qs_state *s, const qs_pauli_term *h0, size_t n0, const qs_pauli_term *h1, size_t n1,
                                const double *svals, int K, double dt, double *energy, double *dE_ds, double *dE_ddt) {
    const int n = s->n, B = s->batch;
    SplitH h;
    QS_TRY(split_for_trotter(n, h0, n0, &h.d0, &h.x0));
    QS_TRY(split_for_trotter(n, h1, n1, &h.d1, &h.x1));
    const uint64_t per = (uint64_t)B << n;
    const size_t ab = amp_bytes_of(s->dtype);
    Work w{s->stream, {}};
    // pair: 2B members, phi_b then lambda_b; tmp: B members; sand: the sandwiches
    QS_TRY(w.alloc(2 * per * ab, 1));
    QS_TRY(w.alloc(per * ab, 1));
    const size_t points = 2 * (size_t)K + 1;  // after each step (and before the first), and mid-step
    const size_t sand_doubles = points * 2 * 2 * (size_t)B;  // per point: two generators, (re, im) per member
    QS_TRY(w.alloc(sand_doubles * sizeof(double) + 64, 1));
    size_t scratch_doubles = (size_t)2 * B * 1024;
    QS_TRY(w.alloc(scratch_doubles * sizeof(double), 1));
    void *pairbuf = w.bufs[0], *tmp = w.bufs[1];
    double *sand = (double *)w.bufs[2], *scr = (double *)w.bufs[3];
    qs_state pair = *s;
    pair.data = pairbuf;
    pair.batch = 2 * B;
    pair.ms = n;
    pair.owns = false;
    pair.scratch = nullptr;
    pair.scratch_doubles = 0;
    pair.host_pinned = nullptr;
    pair.host_pinned_doubles = 0;
    pair.gtab = pair.ptab = nullptr;
    pair.gtab_bytes = pair.ptab_bytes = 0;
    pair.itab = pair.ithr = nullptr;
    pair.itab_bytes = pair.ithr_bytes = 0;
    qs_state phi = pair;
    phi.batch = B;
    auto release = [&]() {
        for (qs_state *v : {&pair, &phi}) {
            if (v->scratch) cudaFreeAsync(v->scratch, s->stream);
            if (v->gtab) cudaFreeAsync(v->gtab, s->stream);
            if (v->ptab) cudaFreeAsync(v->ptab, s->stream);
            if (v->itab) cudaFreeAsync(v->itab, s->stream);
            if (v->ithr) cudaFreeAsync(v->ithr, s->stream);
        }
    };
    const StateView vphi{pairbuf, n, n, B, s->dtype};
    const StateView vlam{(char *)pairbuf + per * ab, n, n, B, s->dtype};
    const StateView vtmp{tmp, n, n, B, s->dtype};
    // <lambda|G phi> for G = the diagonal or X parts of H0 and H1 at point p
    auto sandwich = [&](size_t p, const std::vector<qs_pauli_term> &g0, const std::vector<qs_pauli_term> &g1) {
        const std::vector<qs_pauli_term> *gs[2] = {&g0, &g1};
        for (int j = 0; j < 2; ++j) {
            double *out = sand + (p * 2 + j) * 2 * (size_t)B;
            if (gs[j]->empty()) {
                QS_CUDA_TRY(cudaMemsetAsync(out, 0, 2 * B * sizeof(double), s->stream));
                continue;
            }
            QS_TRY(k_pauli_apply(vphi, vtmp, gs[j]->data(), gs[j]->size(), s->stream));
            QS_TRY(k_dot(vlam, vtmp, scr, scratch_doubles, out, s->stream));
        }
        return QS_OK;
    };
    qs_status st = QS_OK;
    auto run = [&]() -> qs_status {
        // forward: phi = the K steps applied to psi_0 (adjacent half diagonals merged)
        QS_CUDA_TRY(cudaMemcpyAsync(pairbuf, s->data, per * ab, cudaMemcpyDeviceToDevice, s->stream));
        for (int k = 0; k < K; ++k) {
            if (k == 0) QS_TRY(diag_step(&phi, h, svals[0], 0.5 * dt));
            QS_TRY(x_step(&phi, h, svals[k], dt));
            if (k + 1 < K) {
                // exp(-i dt/2 D(s_k)) exp(-i dt/2 D(s_k+1)) in one pass: D is linear in s
                QS_TRY(diag_step(&phi, h, 0.5 * (svals[k] + svals[k + 1]), dt));
            } else {
                QS_TRY(diag_step(&phi, h, svals[k], 0.5 * dt));
            }
        }
        QS_CUDA_TRY(cudaMemcpyAsync(s->data, pairbuf, per * ab, cudaMemcpyDeviceToDevice, s->stream));
        // lambda = H1 phi, E = Re <phi|lambda>
        std::vector<qs_pauli_term> H1(h1, h1 + n1);
        if (H1.empty()) {
            QS_CUDA_TRY(cudaMemsetAsync((char *)pairbuf + per * ab, 0, per * ab, s->stream));
        } else {
            QS_TRY(k_pauli_apply(vphi, vlam, H1.data(), H1.size(), s->stream));
        }
        double *eout = sand + sand_doubles;  // (re, im) per member follow the sandwiches
        (void)eout;
        // reverse sweep: point 2k+2 after step k, 2k+1 its middle, 0 before step 0
        for (int k = K - 1; k >= 0; --k) {
            QS_TRY(sandwich(2 * (size_t)k + 2, h.d0, h.d1));
            QS_TRY(diag_step(&pair, h, svals[k], -0.5 * dt));
            QS_TRY(sandwich(2 * (size_t)k + 1, h.x0, h.x1));
            QS_TRY(x_step(&pair, h, svals[k], -dt));
            QS_TRY(diag_step(&pair, h, svals[k], -0.5 * dt));
        }
        QS_TRY(sandwich(0, h.d0, h.d1));
        return QS_OK;
    };
    st = run();
    // the energy from psi_K (still in s)
    std::vector<double> host(sand_doubles);
    if (st == QS_OK) {
        const cudaError_t e =
            cudaMemcpyAsync(host.data(), sand, sand_doubles * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) st = cuda_status(e, "sandwich copy");
    }
    release();
    if (st == QS_OK) {
        const cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_status(e, "schedule gradient");
    }
    if (st != QS_OK) return st;
    // Im <lambda|G|phi> at point p, generator j (0: H0 part, 1: H1 part), member b
    auto im = [&](size_t p, int j, int b) { return host[((p * 2 + j) * 2 * B) + 2 * b + 1]; };
    for (int b = 0; b < B; ++b) {
        double gdt = 0.0;
        for (int k = 0; k < K; ++k) {
            const size_t pa = 2 * (size_t)k + 2, pm = 2 * (size_t)k + 1, pb = 2 * (size_t)k;
            const double sk = svals[k];
            const double dD = (im(pa, 1, b) - im(pa, 0, b)) + (im(pb, 1, b) - im(pb, 0, b));
            const double dX = im(pm, 1, b) - im(pm, 0, b);
            dE_ds[(size_t)b * K + k] = dt * dD + 2.0 * dt * dX;
            const double hd = (1.0 - sk) * (im(pa, 0, b) + im(pb, 0, b)) + sk * (im(pa, 1, b) + im(pb, 1, b));
            const double hx = (1.0 - sk) * im(pm, 0, b) + sk * im(pm, 1, b);
            gdt += hd + 2.0 * hx;
        }
        dE_ddt[b] = gdt;
    }
    // energy: Re <phi_K|H1|phi_K>, from the final state kept in s
    if (energy) {
        double *dev = nullptr;
        std::vector<qs_pauli_term> H1(h1, h1 + n1);
        QS_TRY(k_expectation(s, H1.data(), H1.size(), &dev));
        std::vector<double> e2(2 * (size_t)B);
        QS_CUDA_TRY(cudaMemcpyAsync(e2.data(), dev, 2 * B * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        for (int b = 0; b < B; ++b) energy[b] = e2[2 * b];
    }
    return QS_OK;
}

}  // namespace qsim
