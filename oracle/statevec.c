/*
 * Oracle: plain, slow, obviously correct complex128 state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header or table with the CUDA library.
 *
 * Conventions (Qibo paper, Sec. 2.3 and Sec. 2.5):
 *   - the state psi(sigma_1..sigma_N) is a flat array of 2^n complex numbers;
 *     qubit q is stored in bit (n-1-q) of the basis index, so qubit 0 is the
 *     most significant bit (Sec. 2.5: fixing the first qubit selects one of two
 *     contiguous halves of the state);
 *   - a k-target gate G is a row-major 2^k x 2^k matrix whose local row/column
 *     index is sum_j bit(target_j) * 2^(k-1-j): the first target is the most
 *     significant local bit, as in G(tau_1..tau_k, tau'_1..tau'_k) of Eq. (1);
 *   - a controlled gate acts only on the index groups whose control bits are all
 *     1 (Sec. 2.4, "Controlled gates").
 * Every routine below is the textbook definition written out with plain loops:
 * no blocking, no fusion, no reordering. Gate application may split its loop
 * over index groups across threads (orc_set_threads; default 1): every group
 * is read and written by one thread, so the result does not depend on the
 * thread count. The reductions stay single-threaded (fixed summation order).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef double complex cplx;

static int orc_threads = 1;

/* Threads for gate application (the CPU baseline's all-cores run); returns
   the number in effect (1 where the build has no OpenMP). */
int orc_set_threads(int t)
{
#ifdef _OPENMP
    orc_threads = t > 0 ? t : 1;
#else
    (void)t;
    orc_threads = 1;
#endif
    return orc_threads;
}

static uint64_t qubit_bit(int n, int q) { return 1ull << (n - 1 - q); }

static int popcount64(uint64_t v)
{
    int c = 0;
    while (v) { c += (int)(v & 1ull); v >>= 1; }
    return c;
}

/*
 * Eq. (1): psi'(.. tau ..) = sum_tau' G(tau, tau') psi(.. tau' ..), the sum
 * running over the target qubits, for every assignment of the other qubits
 * whose control qubits are all 1. Returns 0, or -1 on a bad argument.
 */
int orc_apply_matrix(cplx *psi, int n, int k, const int *targets,
                     int n_controls, const int *controls, const cplx *G)
{
    if (k < 1 || k > 6 || n < k || n > 40) return -1;
    const uint64_t dim = 1ull << n;
    const int K = 1 << k;
    uint64_t tmask = 0, cmask = 0;
    for (int j = 0; j < k; ++j) tmask |= qubit_bit(n, targets[j]);
    for (int j = 0; j < n_controls; ++j) cmask |= qubit_bit(n, controls[j]);
    if (tmask & cmask) return -1;

    /* offset[l]: the index bits that local index l sets on the target qubits */
    uint64_t offset[64];
    for (int l = 0; l < K; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < k; ++j)
            if ((l >> (k - 1 - j)) & 1) o |= qubit_bit(n, targets[j]);
        offset[l] = o;
    }

#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(orc_threads) if (orc_threads > 1)
#endif
    for (uint64_t i = 0; i < dim; ++i) {
        cplx in[64], out[64];
        if (i & tmask) continue;             /* i is the group's base index */
        if ((i & cmask) != cmask) continue;  /* controls not all 1: unchanged */
        for (int c = 0; c < K; ++c) in[c] = psi[i | offset[c]];
        for (int r = 0; r < K; ++r) {
            cplx acc = 0.0;
            for (int c = 0; c < K; ++c) acc += G[r * K + c] * in[c];
            out[r] = acc;
        }
        for (int r = 0; r < K; ++r) psi[i | offset[r]] = out[r];
    }
    return 0;
}

/* Outcome probabilities |psi_x|^2, indexed by the basis integer (Sec. 2.4,
   "Measurements": the distribution sampled from the final state). */
void orc_probabilities(const cplx *psi, int n, double *p)
{
    const uint64_t dim = 1ull << n;
    for (uint64_t x = 0; x < dim; ++x) {
        double re = creal(psi[x]), im = cimag(psi[x]);
        p[x] = re * re + im * im;
    }
}

/* Squared norm sum_x |psi_x|^2. */
double orc_norm2(const cplx *psi, int n)
{
    const uint64_t dim = 1ull << n;
    double s = 0.0;
    for (uint64_t x = 0; x < dim; ++x) {
        double re = creal(psi[x]), im = cimag(psi[x]);
        s += re * re + im * im;
    }
    return s;
}

/*
 * <psi| sum_t c_t P_t |psi> for Pauli strings (the Energy callback of Sec. 2.4).
 * Term t is given by qubit masks (bit q <-> qubit q): X on x-only qubits, Z on
 * z-only qubits, Y where both bits are set. With Y = i X Z,
 *   P|x> = i^{#Y} (-1)^{popcount(x & zbits)} |x xor xbits>,
 * so <psi|P|psi> = sum_x conj(psi[x xor xbits]) * phase(x) * psi[x].
 * Writes the real and imaginary parts of the sum.
 */
void orc_pauli_expectation(const cplx *psi, int n, int n_terms,
                           const double *coeff, const uint64_t *x_mask,
                           const uint64_t *z_mask, double *out_re, double *out_im)
{
    const uint64_t dim = 1ull << n;
    cplx total = 0.0;
    for (int t = 0; t < n_terms; ++t) {
        uint64_t xb = 0, zb = 0;
        for (int q = 0; q < n; ++q) {
            if ((x_mask[t] >> q) & 1ull) xb |= qubit_bit(n, q);
            if ((z_mask[t] >> q) & 1ull) zb |= qubit_bit(n, q);
        }
        int n_y = popcount64(x_mask[t] & z_mask[t]);
        cplx iy = 1.0;
        for (int j = 0; j < n_y; ++j) iy *= I;
        cplx acc = 0.0;
        for (uint64_t x = 0; x < dim; ++x) {
            double sign = (popcount64(x & zb) & 1) ? -1.0 : 1.0;
            acc += conj(psi[x ^ xb]) * (iy * sign) * psi[x];
        }
        total += coeff[t] * acc;
    }
    *out_re = creal(total);
    *out_im = cimag(total);
}

/*
 * Multiply every amplitude by exp(-i * tau * E(x)) where
 * E(x) = sum_t c_t (-1)^{popcount(x & z_t)} is the eigenvalue of a diagonal
 * (Z-string) Hamiltonian on basis state |x>. This is the exact exponential of
 * the diagonal part of H(s) used in a Trotter step (Sec. 2.6).
 */
void orc_apply_diagonal_evolution(cplx *psi, int n, int n_terms,
                                  const double *coeff, const uint64_t *z_mask,
                                  double tau)
{
    const uint64_t dim = 1ull << n;
    uint64_t *zb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_terms > 0 ? n_terms : 1));
    if (!zb) return;
    for (int t = 0; t < n_terms; ++t) {
        zb[t] = 0;
        for (int q = 0; q < n; ++q)
            if ((z_mask[t] >> q) & 1ull) zb[t] |= qubit_bit(n, q);
    }
    for (uint64_t x = 0; x < dim; ++x) {
        double e = 0.0;
        for (int t = 0; t < n_terms; ++t)
            e += coeff[t] * ((popcount64(x & zb[t]) & 1) ? -1.0 : 1.0);
        psi[x] *= cexp(-I * tau * e);
    }
    free(zb);
}
