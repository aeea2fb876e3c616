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
// significant bits (the rest dropped: < 2^-46 relative; values below 2^-103
// keep h alone, below 2^-126 flush to zero); an operation's error is a few
// 2^-47 of its operands' magnitude.
// Products use the exact FMA product (Dekker's method with a fused
// multiply-add), sums Knuth's exact two-sum.

#ifdef __CUDACC__
// d = h + l from the bit pattern (integer operations only): h takes the
// implicit bit and the top 23 fraction bits, the exponent re-biased in place;
// l the next 23 fraction bits (the last 6 dropped: |d - h - l| < 2^-46 |d|).
// Exact range 2^-126 <= |d| < 2^128; below it h is 0 (and l below 2^-103).
__device__ __forceinline__ void df_split(double d, float &h, float &l) {
    const unsigned lo = (unsigned)__double2loint(d), hi = (unsigned)__double2hiint(d);
    const unsigned ex = hi & 0x7ff00000u;  // biased exponent field, in place
    const unsigned sign = hi & 0x80000000u;
    // (hi - (896 << 20)) << 3 | lo >> 29: the float exponent (double bias
    // 1023, float bias 127) and the fraction's top 23 bits; bit 31 is 0 in range
    const unsigned hb = __funnelshift_l(lo, hi - (896u << 20), 3);
    h = ex >= (897u << 20) ? __uint_as_float(hb | sign) : 0.f;
    // l = (fraction bits 28..6) 2^(e-46): a float of exponent e + 104 and
    // those bits as its fraction, less the same float with fraction 0 (exact)
    const unsigned eb = ex * 8u - (919u << 23);  // (biased e - 919) << 23 = (e + 104 + 127 - 127) << 23
    const float t = __uint_as_float(eb | ((lo >> 6) & 0x7fffffu)) - __uint_as_float(eb);
    l = ex >= (920u << 20) ? __uint_as_float(__float_as_uint(t) | sign) : 0.f;
}

// the double nearest h + l, for |l| <= ulp(h): h's bits widened to a double,
// then l added as a whole number of the double's ulps
__device__ __forceinline__ double df_join(float h, float l) {
    const unsigned hb = __float_as_uint(h);
    const unsigned ef = hb & 0x7f800000u;  // float exponent field, in place
    if (ef == 0u) return 0.0;
    const unsigned sign = hb & 0x80000000u;
    // hi: sign, exponent + 896, the fraction's top 20 bits; lo: its last 3
    const unsigned hi = (((hb & 0x7fffffffu) >> 3) + (896u << 20)) | sign;
    const unsigned lo = hb << 29;
    long long k = 0;
    if (ef >= (52u << 23)) {
        // l in units of the double's ulp 2^(eh - 127 - 52): l 2^(179 - eh),
        // the scale's exponent field 306 - eh
        const float q = l * __uint_as_float((306u << 23) - ef);
        k = __float2int_rn(q);
        if (sign) k = -k;  // the ulps count in the magnitude's direction
        // below a power of two the binade's ulp is half as large
        if (k < 0 && (hb & 0x7fffffu) == 0u) k *= 2;
    }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo) + k);
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

// A complex double-float number, laid out for the paired FP32 instructions
// (add/sub/mul/fma .f32x2, two lanes per instruction): h = (re.h, im.h),
// l = (re.l, im.l).
struct __align__(16) ddc {
    float2 h, l;
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
__device__ __forceinline__ double to_double(dd a) { return df_join(a.h, a.l); }

// ---- paired FP32 operations (round to nearest, never contracted)
__device__ __forceinline__ unsigned long long pbits(float2 v) { return *reinterpret_cast<unsigned long long *>(&v); }
__device__ __forceinline__ float2 pfloat(unsigned long long b) { return *reinterpret_cast<float2 *>(&b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
    return pfloat(r);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
    return pfloat(r);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
    return pfloat(r);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)), "l"(pbits(c)));
    return pfloat(r);
}
// sign flips by bit operations (exact, no FP instruction)
__device__ __forceinline__ float2 pneg(float2 a) { return pfloat(pbits(a) ^ 0x8000000080000000ull); }
__device__ __forceinline__ float2 pneg_hi(float2 a) { return pfloat(pbits(a) ^ 0x8000000000000000ull); }

// ---- complex double-float arithmetic on the lane pairs
// The exact sums below are Knuth's two-sum (s = a + b, bb = s - a,
// e = (a - (s - bb)) + (b - bb): a + b = s + e exactly, six operations) and
// the renormalisations its three-operation form for |a| >= |b|.
// a + b: exact two-sum of the high parts, then the low parts, renormalised
__device__ __forceinline__ ddc dd_cadd(ddc a, ddc b) {
    const float2 s = padd(a.h, b.h);
    const float2 bb = psub(s, a.h);
    float2 e = padd(psub(a.h, psub(s, bb)), psub(b.h, bb));
    e = padd(e, padd(a.l, b.l));
    ddc r;
    r.h = padd(s, e);
    r.l = psub(e, psub(r.h, s));
    return r;
}

// c + x v for a real double-float x (both components)
__device__ __forceinline__ ddc dd_fma_c2(dd x, ddc v, ddc c) {
    const float2 xh = make_float2(x.h, x.h), xl = make_float2(x.l, x.l);
    const float2 np = pmul(pneg(xh), v.h);  // -p, p = xh v.h rounded
    float2 q = pfma(xh, v.h, np);           // xh v.h - p, exactly
    q = pfma(xh, v.l, q);
    q = pfma(xl, v.h, q);
    // c.h + p = s + e exactly (two-sum with b = -np)
    const float2 s = psub(c.h, np);
    const float2 bb = psub(s, c.h);
    float2 e = psub(psub(c.h, psub(s, bb)), padd(np, bb));
    e = padd(e, padd(q, c.l));
    ddc r;
    r.h = padd(s, e);
    r.l = psub(e, psub(r.h, s));
    return r;
}

// a b = a.re (b.re, b.im) + (-a.im, a.im) (b.im, b.re): two paired exact
// products, an exact two-sum of their high parts, the low parts in FP32
__device__ __forceinline__ ddc dd_cmul(ddc a, ddc b) {
    const float2 xh = make_float2(a.h.x, a.h.x), xl = make_float2(a.l.x, a.l.x);
    const float2 yh = make_float2(-a.h.y, a.h.y), yl = make_float2(-a.l.y, a.l.y);
    const float2 sh = make_float2(b.h.y, b.h.x), sl = make_float2(b.l.y, b.l.x);
    const float2 np1 = pmul(pneg(xh), b.h);
    const float2 np2 = pmul(pneg(yh), sh);
    float2 q = padd(pfma(xh, b.h, np1), pfma(yh, sh, np2));
    q = pfma(xh, b.l, q);
    q = pfma(xl, b.h, q);
    q = pfma(yh, sl, q);
    q = pfma(yl, sh, q);
    // np1 + np2 = ns + ne exactly; the product is -(ns + ne) + q
    const float2 ns = padd(np1, np2);
    const float2 bb = psub(ns, np1);
    const float2 ne = padd(psub(np1, psub(ns, bb)), psub(np2, bb));
    const float2 e = psub(q, ne);
    ddc r;
    r.h = psub(e, ns);
    r.l = psub(e, padd(r.h, ns));
    return r;
}
#endif  // __CUDACC__

template <typename R> __host__ __device__ __forceinline__ V<R> mkc(R re, R im) {
    V<R> v;
    v.x = re;
    v.y = im;
    return v;
}
template <> __host__ __device__ __forceinline__ ddc mkc<dd>(dd re, dd im) {
    ddc v;
    v.h = make_float2(re.h, im.h);
    v.l = make_float2(re.l, im.l);
    return v;
}

// real and imaginary parts as scalars of the arithmetic
template <typename R> __host__ __device__ __forceinline__ R re_of(V<R> v) { return v.x; }
template <typename R> __host__ __device__ __forceinline__ R im_of(V<R> v) { return v.y; }
template <> __host__ __device__ __forceinline__ dd re_of<dd>(ddc v) { return dd(v.h.x, v.l.x); }
template <> __host__ __device__ __forceinline__ dd im_of<dd>(ddc v) { return dd(v.h.y, v.l.y); }

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

template <> __device__ __forceinline__ ddc cmul<dd>(ddc a, ddc b) { return dd_cmul(a, b); }
template <> __device__ __forceinline__ ddc cmadd<dd>(ddc a, ddc b, ddc c) { return dd_cadd(dd_cmul(a, b), c); }

// -v and conj(v)
template <typename R> __device__ __forceinline__ V<R> cneg(V<R> v) { return mkc<R>(-v.x, -v.y); }
template <> __device__ __forceinline__ ddc cneg<dd>(ddc v) {
    ddc r;
    r.h = pneg(v.h);
    r.l = pneg(v.l);
    return r;
}
template <typename R> __device__ __forceinline__ V<R> conjc(V<R> v) { return mkc<R>(v.x, -v.y); }
template <> __device__ __forceinline__ ddc conjc<dd>(ddc v) {
    ddc r;
    r.h = pneg_hi(v.h);
    r.l = pneg_hi(v.l);
    return r;
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
