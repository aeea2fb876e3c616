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

// the product a b as a first sum (the paired products of dd_cmul)
__device__ __forceinline__ ProdSum prod_first(ddc a, ddc b) {
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
    const float2 ns = padd(np1, np2);
    const float2 bb = psub(ns, np1);
    const float2 ne = padd(psub(np1, psub(ns, bb)), psub(np2, bb));
    return ProdSum{pneg(ns), psub(q, ne)};
}

// acc + a b
__device__ __forceinline__ void prod_add(ProdSum &acc, ddc a, ddc b) {
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

__device__ __forceinline__ ddc prod_result(const ProdSum &acc) {
    ddc r;
    r.h = padd(acc.S, acc.E);
    r.l = psub(acc.E, psub(r.h, acc.S));
    return r;
}

}  // namespace qsim
