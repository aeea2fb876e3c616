// Device code of the tiled multi-gate pass (see tiled.h for the data layout):
// the register-level gate operations, and the pieces a pass kernel is made of
// (per-CTA tables, tile load, stage transpose, one op, tile store, gradient
// partials).
//
// Two kernels are built from these pieces. The generic kernel (kernels_tiled.cu)
// reads a pass descriptor from its parameters and loops over its stages and
// ops, decoding each op at run time. A pass kernel specialised for one
// descriptor (tile_jit.cpp) is the same pieces called in a straight line with
// the descriptor as a compile-time constant, so every op's decode, its loop
// bounds and its constants fold away. Both run the same arithmetic.
#pragma once

#include "device.cuh"
#include "tiled.h"

namespace qsim {

template <typename R> __device__ __forceinline__ V<R> shfl_xor_c(V<R> v, int m) {
    V<R> o;
    if constexpr (is_dd<R>) {
        o.h.x = __shfl_xor_sync(0xffffffffu, v.h.x, m);
        o.h.y = __shfl_xor_sync(0xffffffffu, v.h.y, m);
        o.l.x = __shfl_xor_sync(0xffffffffu, v.l.x, m);
        o.l.y = __shfl_xor_sync(0xffffffffu, v.l.y, m);
    } else {
        o.x = __shfl_xor_sync(0xffffffffu, v.x, m);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, m);
    }
    return o;
}

// 2x2 gate on register bit J for every register pair whose required register
// bits (mr) are set.
template <typename R, int RB, int J>
__device__ __forceinline__ void dense1_reg(V<R> *a, V<R> m00, V<R> m01, V<R> m10, V<R> m11, uint32_t mr) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if (r & (1 << J)) continue;
        if ((r & mr) != mr) continue;
        const V<R> x = a[r], y = a[r | (1 << J)];
        a[r] = cmadd<R>(m01, y, cmul<R>(m00, x));
        a[r | (1 << J)] = cmadd<R>(m11, y, cmul<R>(m10, x));
    }
}

// 4x4 gate on register bits (A = local MSB, B), A != B
template <typename R, int RB, int A, int B>
__device__ __forceinline__ void dense2_reg(V<R> *a, const V<R> *m, uint32_t mr) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if (r & ((1 << A) | (1 << B))) continue;
        if ((r & mr) != mr) continue;
        const int i[4] = {r, r | (1 << B), r | (1 << A), r | (1 << A) | (1 << B)};
        V<R> x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = a[i[c]];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            V<R> acc = cmul<R>(m[o * 4], x[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = cmadd<R>(m[o * 4 + c], x[c], acc);
            a[i[o]] = acc;
        }
    }
}

template <typename R, int RB, int A, int B>
__device__ __forceinline__ void swap_reg(V<R> *a, uint32_t mr) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if (!(r & (1 << A)) || (r & (1 << B))) continue;
        if ((r & mr) != mr) continue;
        const int q = r ^ (1 << A) ^ (1 << B);
        const V<R> t = a[r];
        a[r] = a[q];
        a[q] = t;
    }
}

template <typename R, int RB>
__device__ __forceinline__ void dispatch_dense1(V<R> *a, int j, V<R> m00, V<R> m01, V<R> m10, V<R> m11,
                                                uint32_t mr) {
    switch (j) {
    case 0: dense1_reg<R, RB, 0>(a, m00, m01, m10, m11, mr); break;
    case 1: dense1_reg<R, RB, 1>(a, m00, m01, m10, m11, mr); break;
    case 2: dense1_reg<R, RB, 2>(a, m00, m01, m10, m11, mr); break;
    case 3: dense1_reg<R, RB, 3>(a, m00, m01, m10, m11, mr); break;
    case 4:
        if constexpr (RB > 4) dense1_reg<R, RB, (RB > 4 ? 4 : 0)>(a, m00, m01, m10, m11, mr);
        break;
    default:
        if constexpr (RB > 5) dense1_reg<R, RB, (RB > 5 ? 5 : 0)>(a, m00, m01, m10, m11, mr);
        break;
    }
}

#define QS_PAIR_CASES(FN, ...)                                                  \
    switch (A * 8 + B) {                                                        \
    case 0 * 8 + 1: FN<R, RB, 0, 1>(__VA_ARGS__); break;                        \
    case 0 * 8 + 2: FN<R, RB, 0, 2>(__VA_ARGS__); break;                        \
    case 0 * 8 + 3: FN<R, RB, 0, 3>(__VA_ARGS__); break;                        \
    case 1 * 8 + 2: FN<R, RB, 1, 2>(__VA_ARGS__); break;                        \
    case 1 * 8 + 3: FN<R, RB, 1, 3>(__VA_ARGS__); break;                        \
    case 2 * 8 + 3: FN<R, RB, 2, 3>(__VA_ARGS__); break;                        \
    default:                                                                    \
        if constexpr (RB > 4) {                                                 \
            constexpr int F = RB > 4 ? 4 : 1;                                   \
            switch (A * 8 + B) {                                                \
            case 0 * 8 + 4: FN<R, RB, 0, F>(__VA_ARGS__); break;                \
            case 1 * 8 + 4: FN<R, RB, 1, F>(__VA_ARGS__); break;                \
            case 2 * 8 + 4: FN<R, RB, 2, F>(__VA_ARGS__); break;                \
            case 3 * 8 + 4: FN<R, RB, 3, F>(__VA_ARGS__); break;                \
            default:                                                            \
                if constexpr (RB > 5) {                                         \
                    constexpr int S = RB > 5 ? 5 : 2;                           \
                    switch (A * 8 + B) {                                        \
                    case 0 * 8 + 5: FN<R, RB, 0, S>(__VA_ARGS__); break;        \
                    case 1 * 8 + 5: FN<R, RB, 1, S>(__VA_ARGS__); break;        \
                    case 2 * 8 + 5: FN<R, RB, 2, S>(__VA_ARGS__); break;        \
                    case 3 * 8 + 5: FN<R, RB, 3, S>(__VA_ARGS__); break;        \
                    case 4 * 8 + 5: FN<R, RB, (RB > 5 ? 4 : 0), S>(__VA_ARGS__); break; \
                    default: break;                                             \
                    }                                                           \
                }                                                               \
                break;                                                          \
            }                                                                   \
        }                                                                       \
    }

template <typename R, int RB>
__device__ __forceinline__ void dispatch_dense2(V<R> *a, int A, int B, const V<R> *m, uint32_t mr) {
    QS_PAIR_CASES(dense2_reg, a, m, mr)
}

template <typename R, int RB>
__device__ __forceinline__ void dispatch_swap(V<R> *a, int A, int B, uint32_t mr) {
    QS_PAIR_CASES(swap_reg, a, mr)
}

// Im<lambda|P|phi> over this thread's registers for P = X or Y on register bit
// J; phi in registers r < NR/2, lambda in r + NR/2 (the top register bit).
template <typename R, int RB, int J>
__device__ __forceinline__ R grad_xy_reg(const V<R> *a, int gen, uint32_t mr) {
    constexpr int H = 1 << (RB - 1);
    R acc = 0;
#pragma unroll
    for (int r = 0; r < H; ++r) {
        if ((r & mr) != mr) continue;
        const V<R> ph = a[r ^ (1 << J)], la = a[r + H];
        // X: Im(conj(la) ph); Y: (r_J ? +1 : -1) * Re(conj(la) ph)
        const R im = la.x * ph.y - la.y * ph.x;
        const R re = la.x * ph.x + la.y * ph.y;
        acc += gen == GEN_X ? im : (((r >> J) & 1) ? re : -re);
    }
    return acc;
}

template <typename R, int RB>
__device__ __forceinline__ R dispatch_grad_xy(const V<R> *a, int j, int gen, uint32_t mr) {
    switch (j) {
    case 0: return grad_xy_reg<R, RB, 0>(a, gen, mr);
    case 1: return grad_xy_reg<R, RB, 1>(a, gen, mr);
    case 2: return grad_xy_reg<R, RB, 2>(a, gen, mr);
    case 3:
        if constexpr (RB > 4) return grad_xy_reg<R, RB, (RB > 4 ? 3 : 0)>(a, gen, mr);
        return 0;
    default:
        if constexpr (RB > 5) return grad_xy_reg<R, RB, (RB > 5 ? 4 : 0)>(a, gen, mr);
        return 0;
    }
}

// exp(i angle) with the angle reduced to [-pi, pi] in FP64 first
template <typename R> __device__ __forceinline__ V<R> expi(double angle) {
    const double two_pi = 6.283185307179586476925286766559;
    const double inv_two_pi = 0.15915494309189533576888376337251;  // multiply: no FP64 division
    const double a = angle - two_pi * rint(angle * inv_two_pi);
    if constexpr (sizeof(R) == 4) {
        float sn, cs;
        sincosf((float)a, &sn, &cs);
        return mkc<float>(cs, sn);
    } else {
        double sn, cs;
        sincos(a, &sn, &cs);
        return mkc<double>(cs, sn);
    }
}


// psi_x *= exp(-i tau E(x)) for an Ising energy E(x) = c + sum_i h_i z_i +
// sum_{i<j} J_ij z_i z_j, z_i = 1 - 2 x_i. Split over the tile: the outside bits
// give fields s_g on the tile bits and an energy of their own (per tile); the
// thread's lane/warp bits add their mutual coupling and their fields on the
// register bits (per thread pattern); the register bits couple among
// themselves (per register index). With w_j the whole field on register bit j,
// E = C + sum_j w_j - 2 sum_{j: r_j = 1} w_j + Q[r], so the phase is a base
// times a factor u_j per set register bit times q[r]. The op's table (filled
// once per pass by ising_table_kernel) holds every part as a unit complex
// number; here they are only multiplied, with no angle or energy in the loop.
template <typename R, int RB>
__device__ __forceinline__ void ising_phase(V<R> *a, const TileParams<R> &p, const double *ising_thr, const TileOp &op,
                                            const TileStage &st, uint64_t tile, uint64_t member, int lane, int warp,
                                            V<R> *s_e, V<R> *s_qp) {
    constexpr int NR = 1 << RB;
    constexpr int WB = TileCfg<R>::WB;
    constexpr int T = 32 << WB;
    const double2 *tab = reinterpret_cast<const double2 *>(
        ising_thr + ((size_t)op.m * (p.total_tiles >> p.n_free) + member) * p.ising_thr_stride);
    const double2 *qp = tab + (size_t)T * (1 + RB);
    const double2 *tile_row = qp + NR + (size_t)(tile & ((1ull << p.n_free) - 1ull)) * (p.k + 1);
    const int tid = threadIdx.x;
    if (tid <= p.k) {
        const double2 v = tile_row[tid];
        s_e[tid] = mkc<R>((R)v.x, (R)v.y);
    } else if (tid >= 32 && tid < 32 + NR) {
        const double2 v = qp[tid - 32];
        s_qp[tid - 32] = mkc<R>((R)v.x, (R)v.y);
    }
    __syncthreads();
    const double2 *row = tab + (size_t)tid * (1 + RB);
    V<R> base = cmul<R>(s_e[p.k], mkc<R>((R)row[0].x, (R)row[0].y));
#pragma unroll
    for (int i = 0; i < kTileLaneBits; ++i) {
        const V<R> e = s_e[st.lloc[i]];
        base = cmul<R>(base, ((lane >> i) & 1) ? conjc<R>(e) : e);
    }
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        const V<R> e = s_e[st.wloc[w]];
        base = cmul<R>(base, ((warp >> w) & 1) ? conjc<R>(e) : e);
    }
    V<R> u[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        const V<R> e = s_e[st.rloc[j]];
        base = cmul<R>(base, e);
        const V<R> ec = conjc<R>(e);
        u[j] = cmul<R>(cmul<R>(ec, ec), mkc<R>((R)row[1 + j].x, (R)row[1 + j].y));
    }
#pragma unroll
    for (int hb = 0; hb < NR / 8; ++hb) {
        V<R> q = base;
#pragma unroll
        for (int j = 3; j < RB; ++j)
            if ((hb >> (j - 3)) & 1) q = cmul<R>(q, u[j]);
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
            const int gk = k8 ^ (k8 >> 1);
            const int r = hb * 8 + gk;
            a[r] = cmul<R>(a[r], cmul<R>(q, s_qp[r]));
            if (k8 < 7) {
                const int gn = (k8 + 1) ^ ((k8 + 1) >> 1);
                const int bit = __ffs(gk ^ gn) - 1;
                q = (gn >> bit) & 1 ? cmul<R>(q, u[bit]) : cmul<R>(q, conjc<R>(u[bit]));
            }
        }
    }
    __syncthreads();
}


// acc + c * v on both components: one packed FMA for float pairs
__device__ __forceinline__ float2 fma_c2(float c, float2 v, float2 acc) {
    uint64_t out;
    const float2 cc = make_float2(c, c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(out)
        : "l"(*reinterpret_cast<const uint64_t *>(&cc)), "l"(*reinterpret_cast<const uint64_t *>(&v)),
          "l"(*reinterpret_cast<const uint64_t *>(&acc)));
    return *reinterpret_cast<float2 *>(&out);
}
__device__ __forceinline__ double2 fma_c2(double c, double2 v, double2 acc) {
    return make_double2(fma(c, v.x, acc.x), fma(c, v.y, acc.y));
}
__device__ __forceinline__ ddc fma_c2(dd c, ddc v, ddc acc) { return dd_fma_c2(c, v, acc); }

// real rotation on register bit J as in-place shears (TOP_ROTS_R): x += s1 y,
// then y += s2 x over the register pairs (x, y) that differ in bit J. Each
// update reads the pair and overwrites one of its members, so no register is
// copied.
template <typename R, int RB, int J>
__device__ __forceinline__ void rot_reg(V<R> *a, R s1, R s2) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if (r & (1 << J)) continue;
        a[r] = fma_c2(s1, a[r | (1 << J)], a[r]);
        a[r | (1 << J)] = fma_c2(s2, a[r], a[r | (1 << J)]);
    }
}

// -i v for a double-float complex v: (v.im, -v.re), lanes swapped, the new
// imaginary lane negated
__device__ __forceinline__ ddc mul_minus_i(ddc v) {
    ddc r;
    r.h = make_float2(v.h.y, -v.h.x);
    r.l = make_float2(v.l.y, -v.l.x);
    return r;
}

// Value of an outside-only factor for this tile.
template <typename R>
__device__ __forceinline__ V<R> outside_factor(const TileDFac<R> &d, const TileDFac<R> &dv, uint64_t tbase) {
    if (d.type == DF_BIT) return (tbase & d.tmask) ? dv.v1 : dv.v0;
    return (tbase & d.mo) == d.mo ? dv.v0 : mkc<R>(1, 0);
}

// A diagonal block (TOP_DBLOCK). The planner folded the factors on register
// bits alone into constants C[0] (base) and C[1 + j] (ratio applied when
// register bit j is 1); sign flips on two register bits are TOP_FLIP ops. The
// factor table holds, in order, `no` complex factors on outside bits alone (a
// per-tile product, formed by each warp), `ns` sign factors (negate the base
// or one ratio where their required bits are 1), complex factors involving
// thread bits or one register bit, and `np` factors on two or more register
// bits. Per thread: base and ratios, then each register's phase as base times
// the ratios of its set bits (prefix products shared by the compiler), then
// the remaining pair factors.
template <typename R, int RB>
__device__ __forceinline__ void diag_block(V<R> *a, const TileParams<R> &p, const V<R> *mat, const TileDFac<R> *dfv,
                                           const TileOp &op, uint64_t tbase, uint32_t lt) {
    constexpr int NR = 1 << RB;
    const V<R> *C = &mat[op.m];
    const int f0 = (int)op.mo, nf = op.b, np = op.a, no = op.gl, ns = op.tkind;
    V<R> base = C[0];
    V<R> u[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) u[j] = C[1 + j];
    if (no > 0) {
        // every warp forms the tile's product of outside factors itself (lanes
        // over factors, then a shuffle product): no barrier
        const int lane = threadIdx.x & 31;
        V<R> v = mkc<R>(1, 0);
        for (int f = f0 + lane; f < f0 + no; f += 32) v = cmul<R>(v, outside_factor<R>(p.dfac[f], dfv[f], tbase));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = cmul<R>(v, shfl_xor_c<R>(v, off));
        base = cmul<R>(base, v);
    }
    if (ns > 0) {
        // sign factors: XOR of negation bits (bit j: ratio j, bit 7: base)
        uint32_t neg = 0;
        for (int f = f0 + no; f < f0 + no + ns; ++f) {
            const TileDFac<R> &d = p.dfac[f];
            if ((tbase & d.mo) == d.mo && (lt & d.mt) == d.mt) neg ^= d.a;
        }
        if (neg & 0x80u) base = cneg<R>(base);
#pragma unroll
        for (int j = 0; j < RB; ++j)
            if ((neg >> j) & 1u) u[j] = cneg<R>(u[j]);
    }
    // thread and mixed factors (two independent product chains)
    V<R> b2 = mkc<R>(1, 0);
    for (int f = f0 + no + ns; f < f0 + nf - np; ++f) {
        const TileDFac<R> &d = p.dfac[f];
        if (d.type == DF_BIT) {
            const V<R> v = (lt & (uint32_t)d.tmask) ? dfv[f].v1 : dfv[f].v0;
            if ((f - f0) & 1) b2 = cmul<R>(b2, v);
            else base = cmul<R>(base, v);
            continue;
        }
        if ((tbase & d.mo) != d.mo || (lt & d.mt) != d.mt) continue;
        if (d.mr == 0) {
            if ((f - f0) & 1) b2 = cmul<R>(b2, dfv[f].v0);
            else base = cmul<R>(base, dfv[f].v0);
        } else {
#pragma unroll
            for (int j = 0; j < RB; ++j)
                if (d.mr == (1u << j)) u[j] = cmul<R>(u[j], dfv[f].v0);
        }
    }
    base = cmul<R>(base, b2);
#pragma unroll
    for (int hb = 0; hb < NR / 8; ++hb) {
        V<R> q = base;
#pragma unroll
        for (int j = 3; j < RB; ++j)
            if ((hb >> (j - 3)) & 1) q = cmul<R>(q, u[j]);
#pragma unroll
        for (int lo = 0; lo < 8; ++lo) {
            V<R> ph = q;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((lo >> j) & 1) ph = cmul<R>(ph, u[j]);
            a[hb * 8 + lo] = cmul<R>(a[hb * 8 + lo], ph);
        }
    }
    // factors on two or more register bits (rare: controlled phases inside a block)
    for (int f = f0 + nf - np; f < f0 + nf; ++f) {
        const TileDFac<R> &d = p.dfac[f];
        if ((tbase & d.mo) != d.mo || (lt & d.mt) != d.mt) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if ((d.tmask >> r) & 1ull) a[r] = cmul<R>(a[r], dfv[f].v0);
    }
}

// per-member rotation on register bit J: RY [[c, -s], [s, c]] (real, packed
// FMAs) or RX [[c, -i s], [-i s, c]], for the registers whose bits of mr are 1
template <typename R, int RB, int J>
__device__ __forceinline__ void prot_reg(V<R> *a, R c, R s, bool rx, uint32_t mr) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if (r & (1 << J)) continue;
        if ((r & mr) != mr) continue;
        const V<R> x = a[r], y = a[r | (1 << J)];
        if (!rx) {
            a[r] = fma_c2(c, x, fma_c2(-s, y, mkc<R>(0, 0)));
            a[r | (1 << J)] = fma_c2(c, y, fma_c2(s, x, mkc<R>(0, 0)));
        } else if constexpr (is_dd<R>) {
            // c x - i s y and c y - i s x: -i v = (v.im, -v.re)
            a[r] = fma_c2(s, mul_minus_i(y), fma_c2(c, x, mkc<R>(0, 0)));
            a[r | (1 << J)] = fma_c2(s, mul_minus_i(x), fma_c2(c, y, mkc<R>(0, 0)));
        } else {
            a[r] = mkc<R>(c * x.x + s * y.y, c * x.y - s * y.x);
            a[r | (1 << J)] = mkc<R>(c * y.x + s * x.y, c * y.y - s * x.x);
        }
    }
}

template <typename R, int RB>
__device__ __forceinline__ void dispatch_prot(V<R> *a, int j, R c, R s, bool rx, uint32_t mr) {
    switch (j) {
    case 0: prot_reg<R, RB, 0>(a, c, s, rx, mr); break;
    case 1: prot_reg<R, RB, 1>(a, c, s, rx, mr); break;
    case 2: prot_reg<R, RB, 2>(a, c, s, rx, mr); break;
    case 3: prot_reg<R, RB, 3>(a, c, s, rx, mr); break;
    default:
        if constexpr (RB > 4) prot_reg<R, RB, (RB > 4 ? 4 : 0)>(a, c, s, rx, mr);
        break;
    }
}

// negate the registers whose bit A is 1 - PA and bit B is 1 - PB (PA, PB: the
// register frame on A and B)
template <typename R, int RB, int A, int B, int PA, int PB>
__device__ __forceinline__ void flip_pat(V<R> *a) {
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r)
        if (((r >> A) & 1) != PA && ((r >> B) & 1) != PB) a[r] = cneg<R>(a[r]);
}

template <typename R, int RB, int A, int B>
__device__ __forceinline__ void flip_reg(V<R> *a, uint32_t pat) {
    switch (pat) {
    case 0: flip_pat<R, RB, A, B, 0, 0>(a); break;
    case 1: flip_pat<R, RB, A, B, 1, 0>(a); break;
    case 2: flip_pat<R, RB, A, B, 0, 1>(a); break;
    default: flip_pat<R, RB, A, B, 1, 1>(a); break;
    }
}

// TOP_FLIP: with further required register bits mr (a sign on three or more
// register bits, rare) every register is tested
template <typename R, int RB>
__device__ __forceinline__ void dispatch_flip(V<R> *a, int A, int B, uint32_t mr, uint32_t pat, uint32_t fx) {
    if (mr == 0) {
        QS_PAIR_CASES(flip_reg, a, pat)
        return;
    }
    const uint32_t m = mr | (1u << A) | (1u << B);
    const uint32_t x = fx | ((pat & 1u) << A) | (((pat >> 1) & 1u) << B);
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r)
        if ((((uint32_t)r ^ x) & m) == m) a[r] = cneg<R>(a[r]);
}

// Shared-memory position of tile-local index x under a transpose's swizzle
// (see tiled.h): the images f[i] of its high bits h + i XORed into its low bits.
template <typename R> __device__ __forceinline__ uint32_t swizzle_pos(uint32_t x, const uint8_t *f, int k) {
    constexpr int h = swizzle_low_bits<R>();
    uint32_t y = x;
    for (int i = 0; i < k - h; ++i)
        if ((x >> (h + i)) & 1u) y ^= f[i];
    return y;
}

// tile-local index of this thread's lane and warp bits under a stage mapping
template <int WB>
__device__ __forceinline__ uint32_t thread_local_index(const TileStage &st, int lane, int warp) {
    uint32_t lt = 0;
#pragma unroll
    for (int i = 0; i < kTileLaneBits; ++i)
        if ((lane >> i) & 1) lt |= 1u << st.lloc[i];
#pragma unroll
    for (int w = 0; w < WB; ++w)
        if ((warp >> w) & 1) lt |= 1u << st.wloc[w];
    return lt;
}

template <int RB>
__device__ __forceinline__ uint64_t reg_offset(int r, const uint64_t *g) {
    uint64_t o = 0;
#pragma unroll
    for (int j = 0; j < RB; ++j)
        if ((r >> j) & 1) o |= g[j];
    return o;
}

// XOR of l[j] over the set bits j of r (swizzled positions are not disjoint)
template <int RB>
__device__ __forceinline__ uint32_t reg_local(int r, const uint32_t *l) {
    uint32_t o = 0;
#pragma unroll
    for (int j = 0; j < RB; ++j)
        if ((r >> j) & 1) o ^= l[j];
    return o;
}


// Per-CTA tables, once per launch: this thread's byte offsets for every
// transpose (written and read by this thread only): low half under the
// previous stage's mapping (write), high half under the new stage's (read),
// both in the transpose's swizzle; and its tile-local lane/warp bits per stage.
template <typename R, int RB>
__device__ __forceinline__ void tile_tables(const TileParams<R> &p, uint32_t *tab, uint16_t *ltab, int lane,
                                            int warp) {
    constexpr int WB = TileCfg<R>::WB;
    constexpr int NT = 32 << WB;
    for (int s = 0; s < p.n_stages; ++s) {
        const TileStage &st = p.st[s];
        const uint32_t lt = thread_local_index<WB>(st, lane, warp);
        ltab[s * NT + threadIdx.x] = (uint16_t)lt;
        if (s == 0) continue;
        uint32_t w = swizzle_pos<R>(thread_local_index<WB>(p.st[s - 1], lane, warp), st.fcol, p.k) * sizeof(V<R>);
        // the previous stage's register frame: register r is written where r ^ rflip belongs
        for (int j = 0; j < RB; ++j)
            if ((p.st[s - 1].rflip >> j) & 1u) w ^= st.rw[j];
        const uint32_t r = swizzle_pos<R>(lt, st.fcol, p.k) * sizeof(V<R>);
        tab[s * NT + threadIdx.x] = w | (r << 16);
    }
}

// The global index bits every amplitude of tile t shares.
template <typename R>
__device__ __forceinline__ uint64_t tile_base(const TileParams<R> &p, uint64_t t) {
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    return ((t >> p.n_free) << p.n) | expand_bits(t & fmask, p.tins);
}

// Load a tile straight into registers under stage 0's mapping (lane = the 5
// lowest index bits: every warp-wide load is 32 consecutive amplitudes).
template <typename R, int RB>
__device__ __forceinline__ void tile_load(V<R> *a, const V<R> *__restrict__ psi, const TileParams<R> &p,
                                          uint64_t tbase, int lane, int warp) {
    constexpr int WB = TileCfg<R>::WB;
    const TileStage &s0 = p.st[0];
    uint64_t gt = tbase | (uint64_t)lane;
#pragma unroll
    for (int w = 0; w < WB; ++w)
        if ((warp >> w) & 1) gt |= 1ull << p.gbit[s0.wloc[w]];
    uint64_t gr[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) gr[j] = 1ull << p.gbit[s0.rloc[j]];
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if constexpr (is_dd<R>) {  // complex128 in memory, split into double-float pairs
            const double2 v = reinterpret_cast<const double2 *>(psi)[gt | reg_offset<RB>(r, gr)];
            a[r] = mkc<dd>(dd(v.x), dd(v.y));
        } else {
            a[r] = psi[gt | reg_offset<RB>(r, gr)];
        }
    }
}

// Transpose into stage s (s > 0): write under the previous mapping, read under
// this one (positions are linear over XOR: thread offset ^ register offsets).
template <typename R, int RB>
__device__ __forceinline__ void tile_transpose(V<R> *a, unsigned char *smem, const uint32_t *tab,
                                               const TileParams<R> &p, int s) {
    constexpr int NT = 32 << TileCfg<R>::WB;
    const TileStage &st = p.st[s];
    const uint32_t e = tab[s * NT + threadIdx.x];
    uint32_t ro[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) ro[j] = st.rw[j];
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r)
        *reinterpret_cast<V<R> *>(smem + ((e & 0xffffu) ^ reg_local<RB>(r, ro))) = a[r];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RB; ++j) ro[j] = st.rr[j];
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r)
        a[r] = *reinterpret_cast<const V<R> *>(smem + ((e >> 16) ^ reg_local<RB>(r, ro)));
    __syncthreads();
}

// Per-warp gradient sums: in the state's precision, double for double-float.
template <typename R> struct GradType { using type = R; };
template <> struct GradType<dd> { using type = double; };
template <typename R> using GradT = typename GradType<R>::type;

// Gradient op (TOP_GRAD) in double-float: sum_r w_r conj(lambda_r) phi_r over
// the thread's registers as a complex double-float sum (w_r = +-1: the Y
// generator's sign by the target bit, Z's by the target bit; phi the partner
// across the target for X and Y), summed over the warp, then the generator's
// component (X, Z, projector: the imaginary part; Y: the real part) as a
// double into the warp's slot.
__device__ __forceinline__ ddc grad_term_dd(ddc la, ddc ph, bool neg) {
    const ddc t = dd_cmul(conjc<dd>(la), ph);
    return neg ? cneg<dd>(t) : t;
}

template <int RB, int J>
__device__ __forceinline__ ddc grad_xy_reg_dd(const ddc *a, int gen, uint32_t mr) {
    constexpr int H = 1 << (RB - 1);
    ddc acc = mkc<dd>(dd(0.f, 0.f), dd(0.f, 0.f));
#pragma unroll
    for (int r = 0; r < H; ++r) {
        if ((r & mr) != mr) continue;
        acc = dd_cadd(acc, grad_term_dd(a[r + H], a[r ^ (1 << J)], gen == GEN_Y && !((r >> J) & 1)));
    }
    return acc;
}

template <int RB>
__device__ __forceinline__ void grad_dd(const ddc *a, const TileOp &op, bool ok, uint32_t lt, uint64_t tbase,
                                        int lane, int warp, double (*gsm)[1 << TileCfg<dd>::WB]) {
    constexpr int H = 1 << (RB - 1);
    const uint32_t mr = op.mr;
    ddc acc = mkc<dd>(dd(0.f, 0.f), dd(0.f, 0.f));
    if (op.b == GEN_X || op.b == GEN_Y) {
        if (op.tkind == TB_REG) {
            if (ok) {
                switch (op.a) {
                case 0: acc = grad_xy_reg_dd<RB, 0>(a, op.b, mr); break;
                case 1: acc = grad_xy_reg_dd<RB, 1>(a, op.b, mr); break;
                case 2: acc = grad_xy_reg_dd<RB, 2>(a, op.b, mr); break;
                default:
                    if constexpr (RB > 4) acc = grad_xy_reg_dd<RB, (RB > 4 ? 3 : 0)>(a, op.b, mr);
                    break;
                }
            }
        } else {
            // target on lane bit op.a: partner phi by shuffle (every lane takes part)
            const int bit = (lane >> op.a) & 1;
#pragma unroll
            for (int r = 0; r < H; ++r) {
                const ddc ph = shfl_xor_c<dd>(a[r], 1 << op.a);
                if (ok && (r & mr) == mr) acc = dd_cadd(acc, grad_term_dd(a[r + H], ph, op.b == GEN_Y && !bit));
            }
        }
    } else if (ok) {
        // diagonal generator: Z on one bit, or the all-ones projector
        bool tz = false;
        if (op.b == GEN_Z && op.tkind != TB_REG)
            tz = op.tkind == TB_THREAD ? ((lt & (uint32_t)op.tmask) != 0) : ((tbase & op.tmask) != 0);
#pragma unroll
        for (int r = 0; r < H; ++r) {
            if ((r & mr) != mr) continue;
            bool neg = false;
            if (op.b == GEN_Z) neg = op.tkind == TB_REG ? (((r >> op.a) & 1) != 0) : tz;
            acc = dd_cadd(acc, grad_term_dd(a[r + H], a[r], neg));
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        ddc other;
        other.h.x = __shfl_down_sync(0xffffffffu, acc.h.x, o2);
        other.h.y = __shfl_down_sync(0xffffffffu, acc.h.y, o2);
        other.l.x = __shfl_down_sync(0xffffffffu, acc.l.x, o2);
        other.l.y = __shfl_down_sync(0xffffffffu, acc.l.y, o2);
        acc = dd_cadd(acc, other);
    }
    if (lane == 0) gsm[op.gl][warp] = to_double(op.b == GEN_Y ? re_of<dd>(acc) : im_of<dd>(acc));
}

// Scratch a CTA's ops share: per-warp gradient sums, the Ising op's per-tile
// factors and register-pair factors.
template <typename R> struct TileScratch {
    GradT<R> (*gsm)[1 << TileCfg<R>::WB];
    V<R> *s_e;
    V<R> *s_qp;
};

// Op o of the pass on this thread's registers. The pass's values (matrix
// entries, diagonal-block factors) come from mat[] and dfv[] (the descriptor's
// own arrays in the generic kernel, a separate parameter block in a
// specialised kernel), everything else from p. MODE selects the ops the
// generic kernel compiles in (less code, fewer instruction-fetch stalls): 0:
// rotations on register bits, diagonal blocks, sign flips, phase and one-bit
// diagonal gates; 1: also dense one-qubit gates, lane rotations and per-member
// rotations; 2: also 4x4 gates, swaps, Ising phases and gradients.
template <typename R, int RB, int MODE>
__device__ __forceinline__ void tile_op(V<R> *a, const TileParams<R> &p, const V<R> *mat, const TileDFac<R> *dfv,
                                        const TilePtrs<R> &q, int o, const TileStage &st, uint64_t t, uint64_t tbase,
                                        uint32_t lt, int lane, int warp, const TileScratch<R> &sc) {
    constexpr bool FULL = MODE == 2;
    constexpr int NR = 1 << RB;
    const TileOp &op = p.op[o];
    // decoded per case: the common ops read only the fields they use
    auto req_ok = [&]() { return ((tbase & op.mo) == op.mo) && ((lt & op.mt) == op.mt); };
    auto mat_of = [&]() { return op.pm ? (q.pmat + (t >> p.n_free) * p.pm_stride + op.m) : &mat[op.m]; };
    switch (op.type) {
    case TOP_DENSE1_L: {
        if constexpr (MODE < 1) break;
        // every lane takes part in the shuffles; only `ok` lanes update
        const bool ok = req_ok();
        const uint32_t mr = op.mr;
        const V<R> *M = mat_of();
        const int bit = (lane >> op.a) & 1;
        const V<R> cs = bit ? M[3] : M[0];
        const V<R> co = bit ? M[2] : M[1];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const V<R> v = shfl_xor_c<R>(a[r], 1 << op.a);
            if (ok && (r & mr) == mr) a[r] = cmadd<R>(co, v, cmul<R>(cs, a[r]));
        }
        break;
    }
    case TOP_DENSE1_R:
        if constexpr (MODE < 1) break;
        if (req_ok()) {
            const V<R> *M = mat_of();
            dispatch_dense1<R, RB>(a, op.a, M[0], M[1], M[2], M[3], op.mr);
        }
        break;
    case TOP_PHASE:
        if (req_ok()) {
            const uint32_t mr = op.mr;
            const V<R> ph = mat_of()[0];
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if ((r & mr) == mr) a[r] = cmul<R>(a[r], ph);
        }
        break;
    case TOP_DIAG1:
        if (req_ok()) {
            const uint32_t mr = op.mr;
            const V<R> *M = mat_of();
            const V<R> d0 = M[0], d1 = M[1];
            if (op.tkind == TB_REG) {
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if ((r & mr) == mr) a[r] = cmul<R>(a[r], ((r >> op.a) & 1) ? d1 : d0);
            } else {
                const bool bit = op.tkind == TB_THREAD ? ((lt & (uint32_t)op.tmask) != 0)
                                                       : ((tbase & op.tmask) != 0);
                const V<R> d = bit ? d1 : d0;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if ((r & mr) == mr) a[r] = cmul<R>(a[r], d);
            }
        }
        break;
    case TOP_DENSE2_RR:
        if constexpr (FULL)
            if (req_ok()) dispatch_dense2<R, RB>(a, op.a, op.b, mat_of(), op.mr);
        break;
    case TOP_SWAP_RR:
        if constexpr (FULL)
            if (req_ok()) dispatch_swap<R, RB>(a, op.a, op.b, op.mr);
        break;
    case TOP_ISING:
        if constexpr (FULL)
            ising_phase<R, RB>(a, p, q.ising_thr, op, st, t, t >> p.n_free, lane, warp, sc.s_e, sc.s_qp);
        break;
    case TOP_ROTS_R: {
        // rotations on distinct register bits (they commute): bit j of op.a
        // marks an active one
        const V<R> *M = &mat[op.m];
        const uint32_t am = op.a;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            if (!((am >> j) & 1u)) continue;
            switch (j) {
            case 0: rot_reg<R, RB, 0>(a, re_of<R>(M[0]), im_of<R>(M[0])); break;
            case 1: rot_reg<R, RB, 1>(a, re_of<R>(M[1]), im_of<R>(M[1])); break;
            case 2: rot_reg<R, RB, 2>(a, re_of<R>(M[2]), im_of<R>(M[2])); break;
            case 3: rot_reg<R, RB, 3>(a, re_of<R>(M[3]), im_of<R>(M[3])); break;
            case 4:
                if constexpr (RB > 4) rot_reg<R, RB, (RB > 4 ? 4 : 0)>(a, re_of<R>(M[4]), im_of<R>(M[4]));
                break;
            default:
                if constexpr (RB > 5) rot_reg<R, RB, (RB > 5 ? 5 : 0)>(a, re_of<R>(M[5]), im_of<R>(M[5]));
            }
        }
        break;
    }
    case TOP_ROTS_L: {
        if constexpr (MODE < 1) break;
        // own value in row `bit`, partner value v from lane ^ (1 << j)
        const V<R> *M = &mat[op.m];
#pragma unroll
        for (int j = 0; j < kTileLaneBits; ++j) {
            const R cfx = re_of<R>(M[j]), cfy = im_of<R>(M[j]);
            if (cfy == (R)0) continue;
            const int bit = (lane >> j) & 1;
            const R cc = bit ? cfx : -cfx;
            const bool tan_form = cfy == (R)(ROT_TAN + 1);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const V<R> v = shfl_xor_c<R>(a[r], 1 << j);
                a[r] = tan_form ? fma_c2(cc, v, a[r]) : fma_c2(cc, a[r], v);
            }
        }
        break;
    }
    case TOP_DBLOCK:
        diag_block<R, RB>(a, p, mat, dfv, op, tbase, lt);
        break;
    case TOP_FLIP:
        if (req_ok()) dispatch_flip<R, RB>(a, op.a, op.b, op.mr, op.tkind, op.fx);
        break;
    case TOP_PROT:
        if constexpr (MODE < 1) break;
        if (req_ok()) {
            const V<R> *M = mat_of();
            // table: RY m[2] = (s, 0); RX m[2] = (0, -s)
            const R c = re_of<R>(M[0]), sn = op.b ? -im_of<R>(M[2]) : re_of<R>(M[2]);
            dispatch_prot<R, RB>(a, op.a, c, sn, op.b != 0, op.mr);
        }
        break;
    case TOP_GRAD: {
        if constexpr (FULL && is_dd<R>) {
            grad_dd<RB>(a, op, req_ok(), lt, tbase, lane, warp, sc.gsm);
        } else if constexpr (FULL) {
        const bool ok = req_ok();
        const uint32_t mr = op.mr;
        constexpr int H = NR / 2;
        R acc = 0;
        if (op.b == GEN_X || op.b == GEN_Y) {
            if (op.tkind == TB_REG) {
                if (ok) acc = dispatch_grad_xy<R, RB>(a, op.a, op.b, mr);
            } else {
                // target on lane bit op.a: partner phi by shuffle
                const int bit = (lane >> op.a) & 1;
#pragma unroll
                for (int r = 0; r < H; ++r) {
                    const V<R> ph = shfl_xor_c<R>(a[r], 1 << op.a);
                    const V<R> la = a[r + H];
                    const R im = la.x * ph.y - la.y * ph.x;
                    const R re = la.x * ph.x + la.y * ph.y;
                    if (ok && (r & mr) == mr) acc += op.b == GEN_X ? im : (bit ? re : -re);
                }
            }
        } else if (ok) {
            // diagonal generator: Z on one bit, or the all-ones projector
            bool tz = false;
            if (op.b == GEN_Z && op.tkind != TB_REG)
                tz = op.tkind == TB_THREAD ? ((lt & (uint32_t)op.tmask) != 0) : ((tbase & op.tmask) != 0);
#pragma unroll
            for (int r = 0; r < H; ++r) {
                if ((r & mr) != mr) continue;
                const V<R> ph = a[r], la = a[r + H];
                const R im = la.x * ph.y - la.y * ph.x;
                bool neg = false;
                if (op.b == GEN_Z) neg = op.tkind == TB_REG ? (((r >> op.a) & 1) != 0) : tz;
                acc += neg ? -im : im;
            }
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o2);
        if (lane == 0) sc.gsm[op.gl][warp] = acc;
        }
        break;
    }
    default:
        break;
    }
}

// Store the tile under the last stage's mapping: its lanes hold index bits 0
// and 1 (bit 0 for complex128), so every warp store covers whole sectors.
template <typename R, int RB>
__device__ __forceinline__ void tile_store(V<R> *__restrict__ psi, const V<R> *a, const TileParams<R> &p,
                                           uint64_t tbase, int lane, int warp) {
    constexpr int WB = TileCfg<R>::WB;
    const TileStage &sl = p.st[p.n_stages - 1];
    uint64_t gt = tbase;
#pragma unroll
    for (int i = 0; i < kTileLaneBits; ++i)
        if ((lane >> i) & 1) gt |= 1ull << p.gbit[sl.lloc[i]];
#pragma unroll
    for (int w = 0; w < WB; ++w)
        if ((warp >> w) & 1) gt |= 1ull << p.gbit[sl.wloc[w]];
    uint64_t gr[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        gr[j] = 1ull << p.gbit[sl.rloc[j]];
        if ((sl.rflip >> j) & 1u) gt |= gr[j];  // register frame: r holds r ^ rflip
    }
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) {
        if constexpr (is_dd<R>)
            reinterpret_cast<double2 *>(psi)[gt ^ reg_offset<RB>(r, gr)] =
                make_double2(to_double(re_of<dd>(a[r])), to_double(im_of<dd>(a[r])));
        else
            psi[gt ^ reg_offset<RB>(r, gr)] = a[r];
    }
}

// Gradient partials of this tile (adjoint sweep), summed over the warps in a
// fixed order.
template <typename R>
__device__ __forceinline__ void tile_grad_flush(const TileParams<R> &p, const TilePtrs<R> &q, uint64_t t,
                                                const TileScratch<R> &sc) {
    constexpr int NW = 1 << TileCfg<R>::WB;
    __syncthreads();
    if ((int)threadIdx.x < p.n_grad) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += (double)sc.gsm[threadIdx.x][w];
        q.gpart[(uint64_t)p.gslot[threadIdx.x] * p.total_tiles + t] = sum;
    }
    __syncthreads();
}

}  // namespace qsim
