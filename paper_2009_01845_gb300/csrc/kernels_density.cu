// Density matrices (Sec. 2.4, "Density matrices and noise"): a density matrix
// rho of dm qubits is held as the vector of its 4^dm entries, entry (r, c) at
// index r 2^dm + c: a state of 2 dm qubits whose first dm qubits index the row
// and last dm the column. Gates and channels run on the ordinary gate kernels
// (api.cpp lowers them); this file holds what is specific to the layout: the
// outer product |psi><psi|, the diagonal (outcome probabilities), the trace
// and Tr(rho H) for a Pauli sum H.
#include <algorithm>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

namespace {

constexpr int kDmThreads = 256;
constexpr int kDmMaxTerms = 64;  // terms of one X mask per launch

template <typename R> __device__ __forceinline__ V<R> conj_c(V<R> v) { return mkc<R>(v.x, -v.y); }

// rho_b[r, c] = psi_b[r] conj(psi_b[c])
template <typename R>
__global__ void __launch_bounds__(kDmThreads) dm_outer_kernel(V<R> *__restrict__ rho, const V<R> *__restrict__ psi,
                                                              int dm, uint64_t total) {
    const uint64_t per = 1ull << dm;
    for (uint64_t i = global_tid(); i < total; i += global_stride()) {
        const uint64_t b = i >> (2 * dm), rc = i & (per * per - 1ull);
        const V<R> *p = psi + (b << dm);
        rho[i] = cmul<R>(p[rc >> dm], conj_c<R>(p[rc & (per - 1ull)]));
    }
}

// out[b 2^dm + x] = Re rho_b[x, x]
template <typename R>
__global__ void __launch_bounds__(kDmThreads) dm_diag_kernel(const V<R> *__restrict__ rho, int dm, uint64_t total,
                                                             double *__restrict__ out) {
    const uint64_t per = 1ull << dm;
    for (uint64_t i = global_tid(); i < total; i += global_stride()) {
        const uint64_t b = i >> dm, x = i & (per - 1ull);
        out[i] = (double)rho[(b << (2 * dm)) + x * (per + 1ull)].x;
    }
}

// Terms c_t P_t sharing the X mask xb (row index bits): per term the
// coefficient times i^(number of Y) and the Z mask in row index bits.
struct DmTerms {
    int nt;
    int dm;
    uint64_t xb;
    double cre[kDmMaxTerms], cim[kDmMaxTerms];
    uint64_t zb[kDmMaxTerms];
};

// Per block (blockIdx.x of gridDim.x over the rows, member blockIdx.y): the
// partial sum of rho[r, r ^ xb] f(r), f(r) = sum_t c_t (-1)^popcount(r & zb_t),
// which is Tr(rho P) summed over the group's terms, accumulated in FP64.
template <typename R>
__global__ void __launch_bounds__(kDmThreads) dm_pauli_partial_kernel(const V<R> *__restrict__ rho, const DmTerms p,
                                                                      double2 *__restrict__ part, int accumulate) {
    __shared__ double sre[kDmThreads / 32], sim[kDmThreads / 32];
    const uint64_t per = 1ull << p.dm;
    const V<R> *rb = rho + ((uint64_t)blockIdx.y << (2 * p.dm));
    double are = 0.0, aim = 0.0;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < per;
         r += (uint64_t)gridDim.x * blockDim.x) {
        double fre = 0.0, fim = 0.0;
        for (int t = 0; t < p.nt; ++t) {
            const double sg = (__popcll(r & p.zb[t]) & 1) ? -1.0 : 1.0;
            fre += sg * p.cre[t];
            fim += sg * p.cim[t];
        }
        const V<R> v = rb[r * per + (r ^ p.xb)];
        are += (double)v.x * fre - (double)v.y * fim;
        aim += (double)v.x * fim + (double)v.y * fre;
    }
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_down_sync(0xffffffffu, are, o);
        aim += __shfl_down_sync(0xffffffffu, aim, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sre[threadIdx.x >> 5] = are;
        sim[threadIdx.x >> 5] = aim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tr += sre[w];
            ti += sim[w];
        }
        double2 &slot = part[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x];
        if (accumulate) {
            slot.x += tr;
            slot.y += ti;
        } else {
            slot = make_double2(tr, ti);
        }
    }
}

// out[2 b], out[2 b + 1] = the fixed-order sum of member b's P partials
__global__ void dm_finalize_kernel(const double2 *__restrict__ part, int P, double *__restrict__ out) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < P; ++i) {
        re += part[(uint64_t)b * P + i].x;
        im += part[(uint64_t)b * P + i].y;
    }
    out[2 * b] = re;
    out[2 * b + 1] = im;
}

// out[b] = sum_x Re rho_b[x, x], FP64, fixed order (one CTA per member)
template <typename R>
__global__ void __launch_bounds__(kDmThreads) dm_trace_kernel(const V<R> *__restrict__ rho, int dm,
                                                              double *__restrict__ out) {
    __shared__ double sh[kDmThreads / 32];
    const uint64_t per = 1ull << dm;
    const V<R> *rb = rho + ((uint64_t)blockIdx.x << (2 * dm));
    double acc = 0.0;
    for (uint64_t x = threadIdx.x; x < per; x += blockDim.x) acc += (double)rb[x * (per + 1ull)].x;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

unsigned grid_for(uint64_t work) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + kDmThreads - 1) / kDmThreads, 152ull * 16));
}

}  // namespace

qs_status k_dm_init_pure(qs_state *s, const void *psi_dev) {
    const uint64_t total = (uint64_t)s->batch << s->n;
    ProfScope _ps(s->stream, KC_INIT, (double)total * (s->dtype == QS_C64 ? 8 : 16));
    if (s->dtype == QS_C64)
        dm_outer_kernel<float><<<grid_for(total), kDmThreads, 0, s->stream>>>((float2 *)s->data,
                                                                              (const float2 *)psi_dev, s->dm, total);
    else
        dm_outer_kernel<double><<<grid_for(total), kDmThreads, 0, s->stream>>>(
            (double2 *)s->data, (const double2 *)psi_dev, s->dm, total);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

qs_status k_dm_probabilities(qs_state *s, double *out_dev) {
    const uint64_t total = (uint64_t)s->batch << s->dm;
    ProfScope _ps(s->stream, KC_REDUCE);
    if (s->dtype == QS_C64)
        dm_diag_kernel<float><<<grid_for(total), kDmThreads, 0, s->stream>>>((const float2 *)s->data, s->dm, total,
                                                                             out_dev);
    else
        dm_diag_kernel<double><<<grid_for(total), kDmThreads, 0, s->stream>>>((const double2 *)s->data, s->dm,
                                                                              total, out_dev);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

qs_status k_dm_trace(qs_state *s, double **out_dev) {
    QS_TRY(ensure_scratch(s, (size_t)s->batch));
    ProfScope _ps(s->stream, KC_REDUCE);
    if (s->dtype == QS_C64)
        dm_trace_kernel<float><<<s->batch, kDmThreads, 0, s->stream>>>((const float2 *)s->data, s->dm, s->scratch);
    else
        dm_trace_kernel<double><<<s->batch, kDmThreads, 0, s->stream>>>((const double2 *)s->data, s->dm,
                                                                         s->scratch);
    QS_CUDA_TRY(cudaGetLastError());
    *out_dev = s->scratch;
    return QS_OK;
}

// Tr(rho_b H) per member into the scratch: (re, im) pairs
qs_status k_dm_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double **out_dev) {
    const int dm = s->dm;
    const uint64_t per = 1ull << dm;
    const int P = (int)std::max<uint64_t>(1, std::min<uint64_t>((per + kDmThreads - 1) / kDmThreads,
                                                                 std::max(1, 2 * 152 / s->batch)));
    QS_TRY(ensure_scratch(s, (size_t)2 * P * s->batch + 2 * (size_t)s->batch));
    double2 *part = (double2 *)s->scratch;
    double *out = s->scratch + (size_t)2 * P * s->batch;
    *out_dev = out;
    ProfScope _ps(s->stream, KC_REDUCE);
    // groups of terms by X mask (row index bits), in order of first appearance
    std::vector<uint64_t> masks;
    for (size_t i = 0; i < count; ++i) {
        uint64_t xb = 0;
        for (int q = 0; q < dm; ++q)
            if ((terms[i].x_mask >> q) & 1ull) xb |= qbit(dm, q);
        if (std::find(masks.begin(), masks.end(), xb) == masks.end()) masks.push_back(xb);
    }
    bool first = true;
    for (uint64_t xb : masks) {
        DmTerms p;
        std::memset(&p, 0, sizeof(p));
        p.dm = dm;
        p.xb = xb;
        for (size_t i = 0; i <= count; ++i) {
            const bool flush = i == count || p.nt == kDmMaxTerms;
            if (flush && p.nt > 0) {
                const dim3 grid((unsigned)P, (unsigned)s->batch);
                if (s->dtype == QS_C64)
                    dm_pauli_partial_kernel<float><<<grid, kDmThreads, 0, s->stream>>>((const float2 *)s->data, p,
                                                                                       part, first ? 0 : 1);
                else
                    dm_pauli_partial_kernel<double><<<grid, kDmThreads, 0, s->stream>>>((const double2 *)s->data,
                                                                                        p, part, first ? 0 : 1);
                QS_CUDA_TRY(cudaGetLastError());
                first = false;
                p.nt = 0;
            }
            if (i == count) break;
            uint64_t tx = 0, zb = 0;
            for (int q = 0; q < dm; ++q) {
                if ((terms[i].x_mask >> q) & 1ull) tx |= qbit(dm, q);
                if ((terms[i].z_mask >> q) & 1ull) zb |= qbit(dm, q);
            }
            if (tx != xb) continue;
            const int ny = __builtin_popcountll(terms[i].x_mask & terms[i].z_mask) & 3;
            const double c = terms[i].coeff;
            const double re[4] = {c, 0.0, -c, 0.0}, im[4] = {0.0, c, 0.0, -c};  // c i^ny
            p.cre[p.nt] = re[ny];
            p.cim[p.nt] = im[ny];
            p.zb[p.nt] = zb;
            ++p.nt;
        }
    }
    if (first) {
        QS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * 2 * s->batch, s->stream));
        return QS_OK;
    }
    dm_finalize_kernel<<<s->batch, 32, 0, s->stream>>>(part, P, out);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
