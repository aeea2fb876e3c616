// Device-side helpers shared by the qsim kernels: complex arithmetic on
// interleaved float2/double2 amplitudes and index-bit manipulation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qsim.h"

namespace qsim {

template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename R> using V = typename cvec<R>::type;

template <typename R> __host__ __device__ __forceinline__ V<R> mkc(R re, R im) {
    V<R> v;
    v.x = re;
    v.y = im;
    return v;
}

#ifdef __CUDACC__
// a * b
template <typename R> __device__ __forceinline__ V<R> cmul(V<R> a, V<R> b) {
    return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// a * b + c (four fused multiply-adds)
template <typename R> __device__ __forceinline__ V<R> cmadd(V<R> a, V<R> b, V<R> c) {
    R re = fma(a.x, b.x, c.x);
    re = fma(-a.y, b.y, re);
    R im = fma(a.x, b.y, c.y);
    im = fma(a.y, b.x, im);
    return mkc<R>(re, im);
}

#endif  // __CUDACC__

// Sorted (ascending) bit positions at which zero bits are inserted into a
// compact counter to enumerate the index groups of a gate.
struct InsertBits {
    int8_t pos[QS_MAX_QUBITS + 8];
    int32_t count;
};

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t expand_bits(uint64_t g, const InsertBits &ib) {
    for (int i = 0; i < ib.count; ++i) {
        const int p = ib.pos[i];
        const uint64_t lo = g & ((1ull << p) - 1ull);
        g = ((g >> p) << (p + 1)) | lo;
    }
    return g;
}

__device__ __forceinline__ uint64_t global_tid() {
    return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ uint64_t global_stride() {
    return (uint64_t)gridDim.x * blockDim.x;
}

#endif  // __CUDACC__

}  // namespace qsim
