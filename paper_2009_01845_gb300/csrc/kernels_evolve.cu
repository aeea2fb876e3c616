// Linear combinations of states for the exact time-evolution solvers
// (evolve.cpp): out = sum_j c_j in_j with complex FP64 coefficients, summed in
// FP64 per amplitude and stored in the state's precision. An input may be the
// output (each amplitude is read before it is written, by the same thread).
#include <algorithm>
#include <complex>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

namespace {

constexpr int kCombMax = 8;

struct CombineP {
    int nin;
    double cre[kCombMax], cim[kCombMax];
    const void *in[kCombMax];
    void *out;
    uint64_t total;
};

template <typename R> __global__ void __launch_bounds__(256) combine_kernel(const CombineP p) {
    for (uint64_t i = global_tid(); i < p.total; i += global_stride()) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int j = 0; j < kCombMax; ++j) {
            if (j >= p.nin) break;
            const V<R> v = reinterpret_cast<const V<R> *>(p.in[j])[i];
            re += p.cre[j] * (double)v.x - p.cim[j] * (double)v.y;
            im += p.cre[j] * (double)v.y + p.cim[j] * (double)v.x;
        }
        reinterpret_cast<V<R> *>(p.out)[i] = mkc<R>((R)re, (R)im);
    }
}

}  // namespace

qs_status k_combine(qs_dtype dtype, void *out, const std::vector<const void *> &in, const std::vector<cd> &c,
                    uint64_t total, cudaStream_t st) {
    if (in.empty() || in.size() > (size_t)kCombMax || in.size() != c.size()) {
        set_error("combination of %zu states (1 to %d)", in.size(), kCombMax);
        return QS_ERR_ARG;
    }
    CombineP p;
    std::memset(&p, 0, sizeof(p));
    p.nin = (int)in.size();
    for (int j = 0; j < p.nin; ++j) {
        p.cre[j] = c[j].real();
        p.cim[j] = c[j].imag();
        p.in[j] = in[j];
    }
    p.out = out;
    p.total = total;
    const size_t b = dtype == QS_C64 ? 8 : 16;
    ProfScope _ps(st, KC_EVOLVE, (double)total * b * (p.nin + 1), 8.0 * (double)total * p.nin);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + 255) / 256, 152ull * 16));
    if (dtype == QS_C64)
        combine_kernel<float><<<grid, 256, 0, st>>>(p);
    else
        combine_kernel<double><<<grid, 256, 0, st>>>(p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
