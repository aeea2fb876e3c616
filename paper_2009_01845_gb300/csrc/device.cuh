// Device-side helpers shared by the qsim kernels: complex arithmetic on
// interleaved float2/double2 amplitudes and index-bit manipulation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qsim.h"

namespace qsim {

// ------------------------------------------------------------------ double-float
// A real number as the unevaluated sum h + l of two floats (|l| <= ulp(h)/2
// after every operation): complex128 amplitudes are computed in this form on
// the FP32 pipes (GB300's FP64 rate is 1/64 of its FP32 rate), loaded from and
// stored to memory as doubles. A double becomes h + l with 47 of its 53
// significant bits (values below 2^-103 keep h alone, below 2^-126 flush to
// zero); an operation's error is a few 2^-47 of its operands' magnitude.
// Products use the exact FMA product (Dekker's method with a fused
// multiply-add), sums Knuth's exact two-sum.

#ifdef __CUDACC__
// d = h + l from the bit pattern: h takes the implicit bit and the top 23
// fraction bits, l the remaining 29 rounded to 23 (integer operations only)
__device__ __forceinline__ void df_split(double d, float &h, float &l) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    const unsigned f23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    h = e >= -126 ? __uint_as_float(sign | ((unsigned)(e + 127) << 23) | f23) : 0.f;
    // l = rem 2^(e-52) ~ round(rem / 64) 2^(e-46): a float of exponent e+104
    // and fraction round(rem / 64), less the same float with fraction 0
    // (exact; a fraction of 2^23 carries into the exponent, still exact)
    const unsigned eb = (unsigned)(e + 104) << 23;
    const float t = __uint_as_float(eb + ((rem + 32u) >> 6)) - __uint_as_float(eb);
    l = e >= -103 ? __uint_as_float(__float_as_uint(t) | sign) : 0.f;
}

// the double nearest h + l, for |l| <= ulp(h): h's bits widened to a double,
// then l added as a whole number of the double's ulps
__device__ __forceinline__ double df_join(float h, float l) {
    const unsigned hb = __float_as_uint(h);
    const unsigned sign = hb & 0x80000000u;
    const int eh = (int)((hb >> 23) & 0xffu);
    if (eh == 0) return 0.0;
    unsigned long long db =
        ((unsigned long long)(sign | ((unsigned)(eh + 896) << 20) | ((hb & 0x7fffffu) >> 3)) << 32) |
        ((unsigned long long)(hb & 7u) << 29);
    if (eh >= 52) {
        // l in units of the double's ulp 2^(eh - 127 - 52): l 2^(179 - eh)
        const float q = l * __uint_as_float((unsigned)(306 - eh) << 23);
        long long k = __float2int_rn(q);
        if (sign) k = -k;  // the ulps count in the magnitude's direction
        // below a power of two the binade's ulp is half as large
        if (k < 0 && (hb & 0x7fffffu) == 0) k *= 2;
        db += (unsigned long long)k;
    }
    return __longlong_as_double((long long)db);
}

// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a + b = s + e for |a| >= |b| (three operations); otherwise off by at most
// 2^-24 |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}
#endif  // __CUDACC__

struct dd {
    float h, l;
    dd() = default;
    __host__ __device__ constexpr dd(float hh, float ll) : h(hh), l(ll) {}
    __host__ __device__ dd(double d) {
#ifdef __CUDA_ARCH__
        df_split(d, h, l);
#else
        h = (float)d;
        l = (float)(d - (double)h);
#endif
    }
};

struct __align__(16) ddc {
    dd x, y;
};

template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<dd> { using type = ddc; };
template <typename R> using V = typename cvec<R>::type;
template <typename R> constexpr bool is_dd = false;
template <> constexpr bool is_dd<dd> = true;

#ifdef __CUDACC__
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.h, -a.l); }
__device__ __forceinline__ bool operator==(dd a, dd b) { return a.h == b.h && a.l == b.l; }
__device__ __forceinline__ dd operator+(dd a, dd b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    dd r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.h * b.h;
    float q = fmaf(a.h, b.h, -p);  // p + q = a.h b.h exactly
    q = fmaf(a.h, b.l, q);
    q = fmaf(a.l, b.h, q);
    dd r;
    fast_two_sum(p, q, r.h, r.l);
    return r;
}
__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
// c + a b
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
    const float p = a.h * b.h;
    float q = fmaf(a.h, b.h, -p);
    q = fmaf(a.h, b.l, q);
    q = fmaf(a.l, b.h, q);
    float s, e;
    two_sum(c.h, p, s, e);
    e += q + c.l;
    dd r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}
// a b + c d (one renormalisation)
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
    const float p1 = a.h * b.h, p2 = c.h * d.h;
    float q = fmaf(a.h, b.h, -p1) + fmaf(c.h, d.h, -p2);  // the two products' low parts
    q = fmaf(a.h, b.l, q);
    q = fmaf(a.l, b.h, q);
    q = fmaf(c.h, d.l, q);
    q = fmaf(c.l, d.h, q);
    float s, e;
    two_sum(p1, p2, s, e);
    e += q;
    dd r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}
__device__ __forceinline__ double to_double(dd a) { return df_join(a.h, a.l); }
#endif  // __CUDACC__

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

// double-float complex products: each component one two-product sum
template <> __device__ __forceinline__ ddc cmul<dd>(ddc a, ddc b) {
    return mkc<dd>(dd_dot2(a.x, b.x, -a.y, b.y), dd_dot2(a.x, b.y, a.y, b.x));
}
template <> __device__ __forceinline__ ddc cmadd<dd>(ddc a, ddc b, ddc c) {
    return mkc<dd>(dd_dot2(a.x, b.x, -a.y, b.y) + c.x, dd_dot2(a.x, b.y, a.y, b.x) + c.y);
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
