// Kernels of the adjoint gradient (no counterpart in the paper, which
// differentiates through its TensorFlow backends only, Sec. 2.3):
//   * pauli_apply_kernel: lambda = H phi for a Pauli sum H (the costate seed);
//   * dot_partial_kernel: <phi|lambda> per member (the energy), FP64 across runs;
//   * grad_reduce_kernel: per-tile gradient partials -> dE/dtheta, FP64, fixed order.
// The reverse sweep itself runs in the tiled pass kernel (TOP_GRAD ops).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "adjoint.h"
#include "device.cuh"
#include "prof.h"

namespace qsim {

static unsigned grid_cap(uint64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t need = (work + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)sms * 32));
}

// ------------------------------------------------------------------ lambda = H phi
// (P phi)[y] = i^{#Y} (-1)^{popcount((y ^ m) & z)} phi[y ^ m] for a term (c, m, z).
// U: the index type within a member (32-bit while n <= 32); groups of terms
// without Z bits (pure X) add a constant coefficient.
template <typename R, typename U>
__global__ void __launch_bounds__(256) pauli_apply_kernel(const V<R> *__restrict__ src, V<R> *__restrict__ dst,
                                                          const __grid_constant__ PauliApplyP<R> p) {
    const uint64_t mask = (1ull << p.n) - 1ull;
    for (uint64_t i = global_tid(); i < p.total; i += global_stride()) {
        const U y = (U)(i & mask);
        const V<R> *sm = src + ((i >> p.n) << p.ms);
        V<R> *dm = dst + ((i >> p.n) << p.ms);
        V<R> acc = p.accumulate ? dm[y] : mkc<R>(0, 0);
        for (int g = 0; g < p.ng; ++g) {
            const U x = y ^ (U)p.gx[g];
            R fr, fi;
            if (p.gconst[g]) {
                fr = p.gcre[g];
                fi = p.gcim[g];
            } else {
                fr = 0;
                fi = 0;
                for (int t = p.gbeg[g]; t < p.gbeg[g + 1]; ++t) {
                    const bool odd = (sizeof(U) == 4 ? __popc((uint32_t)(x & (U)p.zb[t]))
                                                     : __popcll((uint64_t)(x & (U)p.zb[t]))) & 1;
                    fr += odd ? -p.cre[t] : p.cre[t];
                    fi += odd ? -p.cim[t] : p.cim[t];
                }
            }
            acc = cmadd<R>(mkc<R>(fr, fi), sm[x], acc);
        }
        dm[y] = acc;
    }
}

// The same over tiles of 2^kPATileBits consecutive amplitudes of a member held
// in shared memory: partners y ^ m whose mask m stays inside the tile's bits
// come from shared memory, the others from global memory (for a transverse
// field on n qubits, n - kPATileBits of the n X groups), so DRAM and L2 see
// far fewer partner reads. Loads and stores are coalesced (thread tid takes
// offsets tid + 256 j).
template <typename R> struct PATile { static constexpr int kBits = sizeof(R) == 4 ? 12 : 11; };

// Amplitude arithmetic A of the tile kernel: the state's own (complex64), or
// double-float for complex128 (loads split, stores joined; the coefficients,
// R = double, are summed in FP64 and converted per use).
template <typename A, typename R> __device__ __forceinline__ V<A> amp_in(const V<R> *p, uint64_t i) {
    if constexpr (is_dd<A>) {
        const double2 v = p[i];
        return mkc<dd>(dd(v.x), dd(v.y));
    } else {
        return p[i];
    }
}
template <typename A, typename R> __device__ __forceinline__ void amp_out(V<R> *p, uint64_t i, V<A> v) {
    if constexpr (is_dd<A>)
        p[i] = make_double2(to_double(re_of<dd>(v)), to_double(im_of<dd>(v)));
    else
        p[i] = v;
}
template <typename A> __device__ __forceinline__ V<A> coef(double re, double im) {
    if constexpr (is_dd<A>)
        return mkc<dd>(dd(re), dd(im));
    else
        return mkc<A>((A)re, (A)im);
}
template <typename A> __device__ __forceinline__ V<A> cadd(V<A> a, V<A> b) {
    if constexpr (is_dd<A>)
        return dd_cadd(a, b);
    else
        return mkc<A>(a.x + b.x, a.y + b.y);
}

template <typename R, typename A>
__global__ void __launch_bounds__(256, 2) pauli_apply_tile_kernel(const V<R> *__restrict__ src, V<R> *__restrict__ dst,
                                                               const __grid_constant__ PauliApplyP<R> p) {
    constexpr int K = PATile<R>::kBits;
    constexpr int PER = (1 << K) / 256;
    constexpr int CB = K - 8;  // chunk bits: bits 8 .. K-1 tell a thread's outputs apart
    __shared__ V<A> tile[1 << K];
    __shared__ R s_f[K];       // Ising fields of the outside bits on the tile bits
    __shared__ R s_eout;       // the outside bits' own energy
    // per thread, once: the thread bits' pair energy and their fields on the chunk bits
    R e_bb = 0, g_b[CB];
    if (p.quad) {
        const uint32_t tb = threadIdx.x;
#pragma unroll
        for (int j = 0; j < CB; ++j) g_b[j] = 0;
        for (int i = 0; i < 8; ++i) {
            const R zi = ((tb >> i) & 1u) ? R(-1) : R(1);
            R half = 0;
            for (int j = 0; j < 8; ++j) half += ((tb >> j) & 1u) ? -p.qJ[i][j] : p.qJ[i][j];
            e_bb += R(0.5) * zi * half;
#pragma unroll
            for (int j = 0; j < CB; ++j) g_b[j] += zi * p.qJ[8 + j][i];
        }
    }
    const uint32_t lowm = (1u << K) - 1u;
    const uint64_t tiles = p.total >> K;
    const int tshift = p.n - K;  // tiles per member: 2^tshift
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t moff = (t >> tshift) << p.ms;
        const uint32_t yb = (uint32_t)((t & ((1ull << tshift) - 1ull)) << K);
        const V<R> *sm = src + moff;
        V<R> *dm = dst + moff;
        __syncthreads();  // the previous tile's readers are done
        if (p.quad) {
            // warp 0: the outside bits' fields on tile bit j (lanes j < K);
            // warp 1: the outside energy, one outside bit per lane, summed
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (warp == 0 && lane < K) {
                R f = p.qh[lane];
                for (int i = K; i < p.n; ++i) f += ((yb >> i) & 1u) ? -p.qJ[lane][i] : p.qJ[lane][i];
                s_f[lane] = f;
            } else if (warp == 1) {
                R u = 0;
                const int i = K + lane;
                if (i < p.n) {
                    R half = 0;
                    for (int j = K; j < p.n; ++j) half += ((yb >> j) & 1u) ? -p.qJ[i][j] : p.qJ[i][j];
                    u = (((yb >> i) & 1u) ? R(-1) : R(1)) * (p.qh[i] + R(0.5) * half);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
                if (lane == 0) s_eout = p.qc0 + u;
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) tile[threadIdx.x + 256 * j] = amp_in<A, R>(sm, yb + threadIdx.x + 256 * j);
        __syncthreads();
        // Z-only group: coefficient of output j = f(j), from the terms' signs on
        // the other bits summed per mask of bits 8.. and a Walsh-Hadamard
        // transform over the PER outputs of this thread
        R Dr[PER], Di[PER];
        if (p.gdiag >= 0) {
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                R ar = 0, ai = 0;
                for (int k = p.dmb[m]; k < p.dmb[m + 1]; ++k) {
                    const int tt = p.dord[k];
                    const bool odd = __popc((yb | threadIdx.x) & (uint32_t)p.zb[tt]) & 1;
                    ar += odd ? -p.cre[tt] : p.cre[tt];
                    ai += odd ? -p.cim[tt] : p.cim[tt];
                }
                Dr[m] = ar;
                Di[m] = ai;
            }
#pragma unroll
            for (int h = 1; h < PER; h <<= 1)
#pragma unroll
                for (int i = 0; i < PER; ++i)
                    if (!(i & h)) {
                        const R ur = Dr[i], vr = Dr[i | h], ui = Di[i], vi = Di[i | h];
                        Dr[i] = ur + vr;
                        Dr[i | h] = ur - vr;
                        Di[i] = ui + vi;
                        Di[i | h] = ui - vi;
                    }
            if (p.quad) {
                // E = outside energy + thread bits (their fields from outside,
                // their pairs) + chunk bits (fields from outside and from the
                // thread bits, their pairs)
                R base = s_eout + e_bb, g[CB];
#pragma unroll
                for (int i = 0; i < 8; ++i) base += ((threadIdx.x >> i) & 1u) ? -s_f[i] : s_f[i];
#pragma unroll
                for (int j = 0; j < CB; ++j) g[j] = s_f[8 + j] + g_b[j];
#pragma unroll
                for (int c = 0; c < PER; ++c) {
                    R e = base + p.qecc[c];
#pragma unroll
                    for (int j = 0; j < CB; ++j) e += ((c >> j) & 1) ? -g[j] : g[j];
                    Dr[c] += e;
                }
            }
        }
        // groups outer, this thread's PER outputs inner: the PER partner loads of
        // one X mask are independent and in flight together
        V<A> acc[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j)
            acc[j] = p.accumulate ? amp_in<A, R>(dm, yb | (threadIdx.x + 256 * j)) : coef<A>(0.0, 0.0);
        for (int g = 0; g < p.ng; ++g) {
            const uint32_t m = (uint32_t)p.gx[g];
            V<A> v[PER];
            if ((m & ~lowm) == 0) {
#pragma unroll
                for (int j = 0; j < PER; ++j) v[j] = tile[(threadIdx.x + 256 * j) ^ m];
            } else {
#pragma unroll
                for (int j = 0; j < PER; ++j) v[j] = amp_in<A, R>(sm, (yb | (threadIdx.x + 256 * j)) ^ m);
            }
            if (g == p.gdiag) {
#pragma unroll
                for (int j = 0; j < PER; ++j) acc[j] = cmadd<A>(coef<A>(Dr[j], Di[j]), v[j], acc[j]);
            } else if (g < p.run0) {
                // the leading run of groups with one coefficient: partners
                // summed, then multiplied once
#pragma unroll
                for (int j = 0; j < PER; ++j) acc[j] = cadd<A>(acc[j], v[j]);
                if (g + 1 == p.run0) {
                    const V<A> c = coef<A>(p.gcre[g], p.gcim[g]);
#pragma unroll
                    for (int j = 0; j < PER; ++j) acc[j] = cmul<A>(c, acc[j]);
                }
            } else if (p.gconst[g]) {
                const V<A> c = coef<A>(p.gcre[g], p.gcim[g]);
#pragma unroll
                for (int j = 0; j < PER; ++j) acc[j] = cmadd<A>(c, v[j], acc[j]);
            } else {
#pragma unroll
                for (int j = 0; j < PER; ++j) {
                    const uint32_t x = (yb | (threadIdx.x + 256 * j)) ^ m;
                    R fr = 0, fi = 0;
                    for (int tt = p.gbeg[g]; tt < p.gbeg[g + 1]; ++tt) {
                        const bool odd = __popc(x & (uint32_t)p.zb[tt]) & 1;
                        fr += odd ? -p.cre[tt] : p.cre[tt];
                        fi += odd ? -p.cim[tt] : p.cim[tt];
                    }
                    acc[j] = cmadd<A>(coef<A>(fr, fi), v[j], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) amp_out<A, R>(dm, yb | (threadIdx.x + 256 * j), acc[j]);
    }
}

template <typename R>
static qs_status pauli_apply_t(const StateView &src, const StateView &dst, const qs_pauli_term *terms, size_t count,
                               cudaStream_t st) {
    const int n = src.n;
    // group by X mask, first-seen order
    std::vector<uint64_t> masks;
    std::vector<std::vector<size_t>> groups;
    for (size_t t = 0; t < count; ++t) {
        uint64_t xb = 0;
        for (int q = 0; q < n; ++q)
            if ((terms[t].x_mask >> q) & 1ull) xb |= 1ull << (n - 1 - q);
        size_t gi = 0;
        while (gi < masks.size() && masks[gi] != xb) ++gi;
        if (gi == masks.size()) {
            masks.push_back(xb);
            groups.emplace_back();
        }
        groups[gi].push_back(t);
    }
    // constant groups (no Z bits) first, the largest set with one coefficient
    // leading, then the others in their order
    {
        auto coef = [&](size_t gi, double *re, double *im, bool *cst) {
            *re = *im = 0.0;
            *cst = true;
            for (size_t t : groups[gi]) {
                const qs_pauli_term &tm = terms[t];
                const int ny = __builtin_popcountll(tm.x_mask & tm.z_mask) & 3;
                const double c = tm.coeff;
                *re += ny == 0 ? c : ny == 2 ? -c : 0.0;
                *im += ny == 1 ? c : ny == 3 ? -c : 0.0;
                if (tm.z_mask) *cst = false;
            }
        };
        std::vector<size_t> ord(masks.size());
        std::vector<double> cre(masks.size()), cim(masks.size());
        std::vector<int> cst(masks.size());
        for (size_t gi = 0; gi < masks.size(); ++gi) {
            bool c;
            coef(gi, &cre[gi], &cim[gi], &c);
            cst[gi] = c;
            ord[gi] = gi;
        }
        // the coefficient shared by the most constant groups
        size_t lead = masks.size(), lead_n = 0;
        for (size_t a = 0; a < masks.size(); ++a) {
            if (!cst[a]) continue;
            size_t c = 0;
            for (size_t b = 0; b < masks.size(); ++b) c += cst[b] && cre[b] == cre[a] && cim[b] == cim[a];
            if (c > lead_n) {
                lead_n = c;
                lead = a;
            }
        }
        auto in_lead = [&](size_t a) {
            return lead < masks.size() && cst[a] && cre[a] == cre[lead] && cim[a] == cim[lead];
        };
        std::stable_partition(ord.begin(), ord.end(), in_lead);
        std::vector<uint64_t> m2;
        std::vector<std::vector<size_t>> g2;
        for (size_t i : ord) {
            m2.push_back(masks[i]);
            g2.push_back(std::move(groups[i]));
        }
        masks.swap(m2);
        groups.swap(g2);
    }
    const uint64_t total = (uint64_t)src.batch << n;
    ProfScope _ps(st, KC_HPSI, 2.0 * total * sizeof(V<R>), 8.0 * total * (double)count);
    bool first = true;
    size_t gi = 0;
    while (gi < masks.size() || first) {
        PauliApplyP<R> p;
        std::memset(&p, 0, sizeof(p));
        int nt = 0;
        while (gi < masks.size() && p.ng < kPAMaxGroups &&
               nt + (int)groups[gi].size() <= kPAMaxTerms) {
            p.gx[p.ng] = masks[gi];
            p.gbeg[p.ng] = nt;
            p.gconst[p.ng] = 1;
            double sre = 0.0, sim = 0.0;
            for (size_t t : groups[gi]) {
                const qs_pauli_term &tm = terms[t];
                const int ny = __builtin_popcountll(tm.x_mask & tm.z_mask) & 3;
                const double c = tm.coeff;
                const double re[4] = {c, 0.0, -c, 0.0}, im[4] = {0.0, c, 0.0, -c};
                p.cre[nt] = (R)re[ny];
                p.cim[nt] = (R)im[ny];
                uint64_t zb = 0;
                for (int q = 0; q < n; ++q)
                    if ((tm.z_mask >> q) & 1ull) zb |= 1ull << (n - 1 - q);
                p.zb[nt] = zb;
                if (zb != 0) p.gconst[p.ng] = 0;
                sre += re[ny];
                sim += im[ny];
                ++nt;
            }
            p.gcre[p.ng] = (R)sre;
            p.gcim[p.ng] = (R)sim;
            ++p.ng;
            ++gi;
        }
        if (p.ng == 0 && gi < masks.size()) {
            set_error("a Pauli group has more than %d terms", kPAMaxTerms);
            return QS_ERR_UNSUPPORTED;
        }
        p.gbeg[p.ng] = nt;
        p.run0 = 0;
        if (first)
            while (p.run0 < p.ng && p.gconst[p.run0] && p.gcre[p.run0] == p.gcre[0] && p.gcim[p.run0] == p.gcim[0] &&
                   p.gx[p.run0] != 0)
                ++p.run0;
        p.gdiag = -1;
        for (int g = 0; g < p.ng; ++g)
            if (p.gx[g] == 0 && !p.gconst[g]) p.gdiag = g;
        if (p.gdiag >= 0) {
            constexpr int cb = PATile<R>::kBits - 8;  // log2 of outputs per thread
            // weight 0-2 terms of the Z-only group: the Ising form (tile kernel
            // only, n <= 32); the others by their parities per chunk mask
            const bool tiled = n >= PATile<R>::kBits && n <= 32;
            std::vector<char> quad(kPAMaxTerms, 0);
            if (tiled) {
                std::vector<double> h(32, 0.0), J(32 * 32, 0.0);
                double c0 = 0.0;
                for (int t = p.gbeg[p.gdiag]; t < p.gbeg[p.gdiag + 1]; ++t) {
                    const uint64_t zb = p.zb[t];
                    const int w = __builtin_popcountll(zb);
                    if (w > 2) continue;
                    quad[t] = 1;
                    p.quad = 1;
                    const double c = (double)p.cre[t];  // Z-only terms: real coefficients
                    if (w == 0) {
                        c0 += c;
                    } else if (w == 1) {
                        h[__builtin_ctzll(zb)] += c;
                    } else {
                        const int i = __builtin_ctzll(zb), j = 63 - __builtin_clzll(zb);
                        J[i * 32 + j] += c;
                        J[j * 32 + i] += c;
                    }
                }
                p.qc0 = (R)c0;
                for (int i = 0; i < 32; ++i) {
                    p.qh[i] = (R)h[i];
                    for (int j = 0; j < 32; ++j) p.qJ[i][j] = (R)J[i * 32 + j];
                }
                for (int c = 0; c < (1 << cb); ++c) {
                    double e = 0.0;
                    for (int i = 0; i < cb; ++i)
                        for (int j = i + 1; j < cb; ++j)
                            e += ((((c >> i) ^ (c >> j)) & 1) ? -1.0 : 1.0) * J[(8 + i) * 32 + 8 + j];
                    p.qecc[c] = (R)e;
                }
            }
            int k2 = 0;
            for (int m = 0; m < (1 << cb); ++m) {
                p.dmb[m] = k2;
                for (int t = p.gbeg[p.gdiag]; t < p.gbeg[p.gdiag + 1]; ++t)
                    if (!quad[t] && (int)((p.zb[t] >> 8) & ((1u << cb) - 1u)) == m) p.dord[k2++] = (uint16_t)t;
            }
            p.dmb[1 << cb] = k2;
        }
        p.n = n;
        p.ms = src.ms;
        p.total = total;
        p.accumulate = first ? 0 : 1;
        first = false;
        // complex128 partner arithmetic in double-float
        using A = typename std::conditional<sizeof(R) == 4, float, dd>::type;
        if (n >= PATile<R>::kBits && n <= 32)
            pauli_apply_tile_kernel<R, A>
                <<<grid_cap(total >> PATile<R>::kBits, 1), 256, 0, st>>>((const V<R> *)src.data, (V<R> *)dst.data, p);
        else if (n <= 32)
            pauli_apply_kernel<R, uint32_t>
                <<<grid_cap(total, 256), 256, 0, st>>>((const V<R> *)src.data, (V<R> *)dst.data, p);
        else
            pauli_apply_kernel<R, uint64_t>
                <<<grid_cap(total, 256), 256, 0, st>>>((const V<R> *)src.data, (V<R> *)dst.data, p);
        QS_CUDA_TRY(cudaGetLastError());
    }
    return QS_OK;
}

qs_status k_pauli_apply(const StateView &src, const StateView &dst, const qs_pauli_term *terms, size_t count,
                        cudaStream_t st) {
    return src.dtype == QS_C64 ? pauli_apply_t<float>(src, dst, terms, count, st)
                               : pauli_apply_t<double>(src, dst, terms, count, st);
}

// ------------------------------------------------------------------ <a|b> per member
__device__ __forceinline__ double2 block_sum2_adj(double a, double b) {
    __shared__ double2 sh[32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = make_double2(a, b);
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        r = lane < nw ? sh[lane] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            r.x += __shfl_down_sync(0xffffffffu, r.x, o);
            r.y += __shfl_down_sync(0xffffffffu, r.y, o);
        }
    }
    __syncthreads();
    return r;
}

template <typename R>
__global__ void __launch_bounds__(256) dot_partial_kernel(const V<R> *__restrict__ a, const V<R> *__restrict__ b,
                                                          int n, int ms, double2 *__restrict__ part) {
    const uint64_t per = 1ull << n;
    const V<R> *pa = a + ((uint64_t)blockIdx.y << ms);
    const V<R> *pb = b + ((uint64_t)blockIdx.y << ms);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double sr = 0.0, si = 0.0;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    while (i < per) {
        R rr = 0, ri = 0;
        for (int c = 0; c < 16 && i < per; ++c, i += stride) {
            const V<R> x = pa[i], y = pb[i];
            rr = fma(x.x, y.x, fma(x.y, y.y, rr));   // Re conj(x) y
            ri = fma(x.x, y.y, fma(-x.y, y.x, ri));  // Im conj(x) y
        }
        sr += (double)rr;
        si += (double)ri;
    }
    const double2 r = block_sum2_adj(sr, si);
    if (threadIdx.x == 0) part[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
}

__global__ void dot_finalize_kernel(const double2 *__restrict__ part, int per_member, double *__restrict__ out) {
    const int b = blockIdx.x;
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < per_member; i += blockDim.x) {
        x += part[(uint64_t)b * per_member + i].x;
        y += part[(uint64_t)b * per_member + i].y;
    }
    const double2 r = block_sum2_adj(x, y);
    if (threadIdx.x == 0) {
        out[2 * b] = r.x;
        out[2 * b + 1] = r.y;
    }
}

qs_status k_dot(const StateView &a, const StateView &b, double *scratch, size_t scratch_doubles, double *out,
                cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t per = 1ull << a.n;
    int P = (int)std::min<uint64_t>(std::max<uint64_t>(1, per / (256 * 16)),
                                    std::max<uint64_t>(1, (uint64_t)sms * 8 / a.batch));
    P = (int)std::min<size_t>((size_t)P, std::max<size_t>(1, scratch_doubles / (2 * (size_t)a.batch)));
    ProfScope _ps(st, KC_ADJOINT, 2.0 * (double)((uint64_t)a.batch << a.n) * (a.dtype == QS_C64 ? 8 : 16),
                  8.0 * (double)((uint64_t)a.batch << a.n));
    dim3 grid(P, a.batch);
    if (a.dtype == QS_C64)
        dot_partial_kernel<float><<<grid, 256, 0, st>>>((const float2 *)a.data, (const float2 *)b.data, a.n, a.ms,
                                                        (double2 *)scratch);
    else
        dot_partial_kernel<double><<<grid, 256, 0, st>>>((const double2 *)a.data, (const double2 *)b.data, a.n,
                                                         a.ms, (double2 *)scratch);
    QS_CUDA_TRY(cudaGetLastError());
    dot_finalize_kernel<<<a.batch, 256, 0, st>>>((const double2 *)scratch, P, out);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ------------------------------------------------------------------ gradient reduction
// grad[b * n_params + p] = sum over the gradient slots s of parameter p of
// coef[s] * sum over member b's tiles of part[s * total_tiles + tile], in a fixed
// order (slot list order, then a block reduction over tiles).
__global__ void __launch_bounds__(256) grad_reduce_kernel(const double *__restrict__ part,
                                                          const __grid_constant__ GradReduceP p,
                                                          double *__restrict__ grad) {
    const int pi = blockIdx.x, b = blockIdx.y;
    double total = 0.0;
    for (int k = p.beg[pi]; k < p.beg[pi + 1]; ++k) {
        const int s = p.slot[k];
        const double *row = part + (uint64_t)s * p.total_tiles + (uint64_t)b * p.tiles_per_member;
        double acc = 0.0;
        for (uint64_t t = threadIdx.x; t < p.tiles_per_member; t += blockDim.x) acc += row[t];
        const double2 r = block_sum2_adj(acc, 0.0);
        total += p.coef[k] * r.x;   // thread 0 holds the block sum
    }
    if (threadIdx.x == 0) grad[(uint64_t)b * p.n_params + p.param0 + pi] = total;
}

qs_status k_grad_reduce(const double *part, const GradReduceP &p, int n_param_rows, int batch, double *grad,
                        cudaStream_t st) {
    if (n_param_rows <= 0) return QS_OK;
    ProfScope _ps(st, KC_ADJOINT);
    dim3 grid(n_param_rows, batch);
    grad_reduce_kernel<<<grid, 256, 0, st>>>(part, p, grad);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ------------------------------------------------------------------ small states
// Gradient op for states too small for the sweep's tiles: one block per member
// sums Im<lambda|P|phi> (see adjoint.cpp) over the member and writes out[b].
template <typename R>
__global__ void __launch_bounds__(256) grad_small_kernel(const V<R> *__restrict__ psi, int n, int gen, int tbit,
                                                         uint64_t req, double *__restrict__ out) {
    const int b = blockIdx.x;
    const uint64_t half = 1ull << n;
    const V<R> *ph = psi + ((uint64_t)b << (n + 1));
    const V<R> *la = ph + half;
    double acc = 0.0;
    for (uint64_t x = threadIdx.x; x < half; x += blockDim.x) {
        if ((x & req) != req) continue;
        const bool tb = (x >> tbit) & 1ull;
        const uint64_t xp = (gen == 0 || gen == 1) ? (x ^ (1ull << tbit)) : x;
        const V<R> f = ph[xp], l = la[x];
        const double im = (double)l.x * f.y - (double)l.y * f.x;
        const double re = (double)l.x * f.x + (double)l.y * f.y;
        if (gen == 0) acc += im;
        else if (gen == 1) acc += tb ? re : -re;
        else if (gen == 2) acc += tb ? -im : im;
        else acc += im;
    }
    const double2 r = block_sum2_adj(acc, 0.0);
    if (threadIdx.x == 0) out[b] = r.x;
}

qs_status k_grad_small(qs_state *w, const LGate &g, double *out) {
    uint64_t req = g.cmask;
    if (g.grad_gen == 3)
        for (int j = 0; j < g.k; ++j) req |= 1ull << g.tbit[j];
    ProfScope _ps(w->stream, KC_ADJOINT);
    if (w->dtype == QS_C64)
        grad_small_kernel<float><<<w->batch, 256, 0, w->stream>>>((const float2 *)w->data, w->n - 1, g.grad_gen,
                                                                  g.tbit[0], req, out);
    else
        grad_small_kernel<double><<<w->batch, 256, 0, w->stream>>>((const double2 *)w->data, w->n - 1, g.grad_gen,
                                                                   g.tbit[0], req, out);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
