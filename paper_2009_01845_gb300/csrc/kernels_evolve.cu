// Linear combinations of states for the exact time-evolution solvers
// (evolve.cpp): out = sum_j c_j in_j, complex coefficients given in FP64.
// complex64: FP32 products and sums (FP32 coefficients, relative rounding
// 6e-8 per term, far inside the complex64 bound); complex128: double-float
// products summed before one renormalisation (no FP64 instruction). An input
// may be the output (each amplitude is read before it is written, by the same
// thread).
#include <algorithm>
#include <complex>
#include <cstring>
#include <vector>

#include "dd_sum.cuh"
#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

namespace {

constexpr int kCombMax = 8;

struct CombineP {
    int nin;
    float2 cf[kCombMax];  // complex64: the coefficients in FP32
    ddc cd[kCombMax];     // complex128: the coefficients as double-float pairs
    const void *in[kCombMax];
    void *out;
    uint64_t total;
};

__global__ void __launch_bounds__(256) combine_c64_kernel(const __grid_constant__ CombineP p) {
    for (uint64_t i = global_tid(); i < p.total; i += global_stride()) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kCombMax; ++j) {
            if (j >= p.nin) break;
            acc = cmadd<float>(p.cf[j], reinterpret_cast<const float2 *>(p.in[j])[i], acc);
        }
        reinterpret_cast<float2 *>(p.out)[i] = acc;
    }
}

__global__ void __launch_bounds__(256) combine_c128_kernel(const __grid_constant__ CombineP p) {
    for (uint64_t i = global_tid(); i < p.total; i += global_stride()) {
        const double2 v0 = reinterpret_cast<const double2 *>(p.in[0])[i];
        ProdSum acc = prod_first(p.cd[0], mkc<dd>(dd(v0.x), dd(v0.y)));
#pragma unroll
        for (int j = 1; j < kCombMax; ++j) {
            if (j >= p.nin) break;
            const double2 v = reinterpret_cast<const double2 *>(p.in[j])[i];
            prod_add(acc, p.cd[j], mkc<dd>(dd(v.x), dd(v.y)));
        }
        const ddc w = prod_result(acc);
        reinterpret_cast<double2 *>(p.out)[i] = make_double2(to_double(re_of<dd>(w)), to_double(im_of<dd>(w)));
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
        p.cf[j] = make_float2((float)c[j].real(), (float)c[j].imag());
        p.cd[j] = mkc<dd>(dd(c[j].real()), dd(c[j].imag()));
        p.in[j] = in[j];
    }
    p.out = out;
    p.total = total;
    const size_t b = dtype == QS_C64 ? 8 : 16;
    ProfScope _ps(st, KC_EVOLVE, (double)total * b * (p.nin + 1), 8.0 * (double)total * p.nin);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + 255) / 256, 152ull * 16));
    if (dtype == QS_C64)
        combine_c64_kernel<<<grid, 256, 0, st>>>(p);
    else
        combine_c128_kernel<<<grid, 256, 0, st>>>(p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
