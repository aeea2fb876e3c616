// complex128 one-gate passes in double-float arithmetic on the FP32 pipes.
//
// GB300's FP64 rate (1.19 TFLOP/s measured) makes a complex128 dense gate pass
// FP64-bound at ~0.31 of the HBM peak (8 FP64 FMAs per amplitude for a 2x2
// gate). Here every double is split into a pair of floats h + l (df_split in
// device.cuh: 47 of its 53 significant bits), the gate is applied in
// double-float arithmetic (device.cuh: exact paired FMA products, exact
// two-sums of their high parts, the low parts summed in FP32; the real and
// imaginary parts share each paired .f32x2 instruction), and the result is
// joined back into a double (df_join). The split and
// the join are integer operations on the IEEE bit patterns, so no FP64
// instruction remains. The error per gate is a few 2^-47 (~1e-14) of the
// amplitudes' magnitude, which keeps the complex128 tolerance (1e-12 on
// amplitudes) over the circuits here.
#include <algorithm>
#include <complex>
#include <cstring>

#include "device.cuh"
#include "dd_sum.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

namespace {

template <int K> struct DenseDFP {
    PairFactor m[(1 << K) * (1 << K)];  // row-major, split and arranged on the host
    uint64_t off[1 << K];
    uint64_t setmask;
    InsertBits ib;
    int n;
    int n_free;
    uint64_t total;
};

// zero bits inserted at ib's positions into g, in I-bit arithmetic (every
// shift below the width)
template <typename I> __device__ __forceinline__ I expand_bits_i(I g, const InsertBits &ib) {
    for (int i = 0; i < ib.count; ++i) {
        const int q = ib.pos[i];
        const I lo = g & ((I(1) << q) - I(1));
        g = (((g >> q) << q) << 1) | lo;
    }
    return g;
}

// I: the index type, 32-bit where every amplitude index of the batch fits
template <int K, typename I>
__global__ void __launch_bounds__(256) dense_df_kernel(double2 *__restrict__ psi,
                                                       const __grid_constant__ DenseDFP<K> p) {
    constexpr int D = 1 << K;
    const I fmask = (I(1) << p.n_free) - I(1);
    const I total = (I)p.total;
    for (I g = (I)global_tid(); g < total; g += (I)global_stride()) {
        const I b = g >> p.n_free;
        // b > 0 only in a batch, whose member stride is then below the width
        const I base = (b << (p.n & (int)(8 * sizeof(I) - 1))) | expand_bits_i<I>(g & fmask, p.ib) | (I)p.setmask;
        ddc a[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double2 v = psi[base | (I)p.off[c]];
            a[c] = mkc<dd>(dd(v.x), dd(v.y));
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            ProdSum acc = prod_first(p.m[r * D], a[0]);
#pragma unroll
            for (int c = 1; c < D; ++c) prod_add(acc, p.m[r * D + c], a[c]);
            const ddc w = prod_result(acc);
            psi[base | (I)p.off[r]] = make_double2(to_double(re_of<dd>(w)), to_double(im_of<dd>(w)));
        }
    }
}

unsigned grid_for_df(const qs_state *s, uint64_t work) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 8));
}

template <int K> qs_status launch_dense_df(qs_state *s, const LGate &g) {
    constexpr int D = 1 << K;
    DenseDFP<K> p;
    std::memset(&p, 0, sizeof(p));
    for (int i = 0; i < D * D; ++i) p.m[i] = pair_factor(mkc<dd>(dd(g.m[i].real()), dd(g.m[i].imag())));
    uint64_t tmask = 0;
    for (int j = 0; j < K; ++j) tmask |= 1ull << g.tbit[j];
    for (int l = 0; l < D; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((l >> (K - 1 - j)) & 1) o |= 1ull << g.tbit[j];
        p.off[l] = o;
    }
    p.setmask = g.cmask;
    // zero bits inserted at the target and control positions (ascending)
    const uint64_t ins = tmask | g.cmask;
    p.ib.count = 0;
    for (int b = 0; b < 64; ++b)
        if ((ins >> b) & 1ull) p.ib.pos[p.ib.count++] = (int8_t)b;
    p.n = s->ms;
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    const double amps = (double)p.total * D;
    ProfScope _ps(s->stream, KC_DENSE, amps * 2.0 * 16.0, amps * 8.0 * D);
    if (((uint64_t)s->batch << s->ms) <= (1ull << 32))
        dense_df_kernel<K, uint32_t><<<grid_for_df(s, p.total), 256, 0, s->stream>>>((double2 *)s->data, p);
    else
        dense_df_kernel<K, uint64_t><<<grid_for_df(s, p.total), 256, 0, s->stream>>>((double2 *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace

// complex128 dense 1- and 2-qubit gates on the double-float kernel; false:
// the caller runs the gate in FP64
bool k_dense_df(qs_state *s, const LGate &g, qs_status *st) {
    if (s->dtype != QS_C128 || g.diagonal || g.is_swap || g.k > 2) return false;
    *st = g.k == 1 ? launch_dense_df<1>(s, g) : launch_dense_df<2>(s, g);
    return true;
}

}  // namespace qsim
