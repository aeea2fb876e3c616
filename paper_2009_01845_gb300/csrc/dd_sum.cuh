// Sums of complex double-float products (device.cuh's paired arithmetic),
// kept unnormalised until the end: the one-gate double-float kernel and the
// state combinations of the exact solvers.
#pragma once

#include "device.cuh"

namespace qsim {

// A sum of complex double-float products kept unnormalised: S holds the
// exact running sum of the products' high parts (two-sums), E the low parts
// and the two-sums' errors in FP32; one renormalisation at the end.
struct ProdSum {
    float2 S, E;
};

// A complex double-float factor a arranged for the paired products of a sum:
// a.re in both lanes (x), (-a.im, a.im) (y), high and low parts, and the
// negated high pairs. A factor shared by every thread of a launch (a gate's
// matrix entry) is arranged once on the host.
struct PairFactor {
    float2 xh, xl, yh, yl, nxh, nyh;
};

__host__ __device__ inline PairFactor pair_factor(ddc a) {
    PairFactor f;
    f.xh = make_float2(a.h.x, a.h.x);
    f.xl = make_float2(a.l.x, a.l.x);
    f.yh = make_float2(-a.h.y, a.h.y);
    f.yl = make_float2(-a.l.y, a.l.y);
    f.nxh = make_float2(-a.h.x, -a.h.x);
    f.nyh = make_float2(a.h.y, -a.h.y);
    return f;
}

// The paired products of a b (as in dd_cmul): -p1, -p2 (the rounded high
// products a.re b and (-a.im, a.im) (b.im, b.re)) and q, their rounding errors
// plus the cross terms in FP32.
__device__ __forceinline__ void prod_parts(const PairFactor &f, ddc b, float2 &np1, float2 &np2, float2 &q) {
    const float2 sh = make_float2(b.h.y, b.h.x), sl = make_float2(b.l.y, b.l.x);
    np1 = pmul(f.nxh, b.h);
    np2 = pmul(f.nyh, sh);
    q = padd(pfma(f.xh, b.h, np1), pfma(f.yh, sh, np2));
    q = pfma(f.xh, b.l, q);
    q = pfma(f.xl, b.h, q);
    q = pfma(f.yh, sl, q);
    q = pfma(f.yl, sh, q);
}

// the product a b as a first sum
__device__ __forceinline__ ProdSum prod_first(const PairFactor &f, ddc b) {
    float2 np1, np2, q;
    prod_parts(f, b, np1, np2, q);
    const float2 ns = padd(np1, np2);
    const float2 bb = psub(ns, np1);
    const float2 ne = padd(psub(np1, psub(ns, bb)), psub(np2, bb));
    return ProdSum{pneg(ns), psub(q, ne)};
}

// acc + a b
__device__ __forceinline__ void prod_add(ProdSum &acc, const PairFactor &f, ddc b) {
    float2 np1, np2, q;
    prod_parts(f, b, np1, np2, q);
    // S - np1 - np2 by two exact two-sums
    const float2 s1 = psub(acc.S, np1);
    const float2 b1 = psub(s1, acc.S);
    const float2 e1 = psub(psub(acc.S, psub(s1, b1)), padd(np1, b1));
    const float2 s2 = psub(s1, np2);
    const float2 b2 = psub(s2, s1);
    const float2 e2 = psub(psub(s1, psub(s2, b2)), padd(np2, b2));
    acc.E = padd(acc.E, padd(padd(e1, e2), q));
    acc.S = s2;
}

__device__ __forceinline__ ProdSum prod_first(ddc a, ddc b) { return prod_first(pair_factor(a), b); }
__device__ __forceinline__ void prod_add(ProdSum &acc, ddc a, ddc b) { prod_add(acc, pair_factor(a), b); }

__device__ __forceinline__ ddc prod_result(const ProdSum &acc) {
    ddc r;
    r.h = padd(acc.S, acc.E);
    r.l = psub(acc.E, psub(r.h, acc.S));
    return r;
}

}  // namespace qsim
