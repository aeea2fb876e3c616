// Tiled multi-gate pass kernel (see tiled.h for the data layout and
// tile_device.cuh for the pieces).
//
// One CTA (256 threads) processes tiles of 2^k amplitudes in a grid-stride
// loop. Per tile: load from HBM straight into registers (lane = the 5 lowest
// index bits, so every warp-wide load is 32 consecutive amplitudes), run the
// pass's stages (register/shuffle gate application, shared-memory transposes
// between stages), and store back once. HBM traffic per pass: one read and one
// write of the state, whatever the number of gates. This generic kernel reads
// the pass descriptor from its parameters and decodes every op at run time; a
// pass kernel specialised for its descriptor (tile_jit.cpp) runs the same
// pieces with the decode folded away.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.h"
#include "prof.h"
#include "tile_device.cuh"
#include "tiled.h"

namespace qsim {

template <typename R> qs_status tile_jit_launch_t(qs_state *s, const TileParams<R> &p, bool *launched);

// The Ising op's tables (see ising_thr_stride), per member (blockIdx.y), in
// FP64: block 0, one thread per thread pattern (lane bits, then warp bits), the
// pattern's coupling energy and fields, and the register-pair energies; blocks
// 1.., one thread per tile, the fields of the outside bits on the tile bits and
// the outside energy. Every energy x is stored as exp(-i tau x).
__global__ void __launch_bounds__(256) ising_table_kernel(const __grid_constant__ IsingTabP tp) {
    const int member = blockIdx.y, tid = threadIdx.x;
    const int nq = tp.nq;
    const double *J = tp.ising + (size_t)member * tp.ising_stride;
    const double *hv = J + (size_t)nq * nq;
    double2 *base = reinterpret_cast<double2 *>(tp.out + (size_t)member * tp.stride);
    auto put = [&](double2 *dst, double x) {
        if (tp.single) {
            const V<float> v = expi<float>(-tp.tau * x);
            *dst = make_double2(v.x, v.y);
        } else {
            const V<double> v = expi<double>(-tp.tau * x);
            *dst = make_double2(v.x, v.y);
        }
    };
    if (blockIdx.x == 0) {
        double z[kTileLaneBits + kTileMaxWarpBits];
        for (int i = 0; i < tp.tb; ++i) z[i] = ((tid >> i) & 1) ? -1.0 : 1.0;
        double e = 0.0;
        for (int i = 0; i < tp.tb; ++i)
            for (int j = i + 1; j < tp.tb; ++j) e += J[tp.tg[i] * nq + tp.tg[j]] * z[i] * z[j];
        double2 *row = base + (size_t)tid * (1 + tp.rb);
        double wsum = 0.0;
        for (int j = 0; j < tp.rb; ++j) {
            double w = 0.0;
            for (int i = 0; i < tp.tb; ++i) w += J[tp.rg[j] * nq + tp.tg[i]] * z[i];
            wsum += w;
            put(&row[1 + j], -2.0 * w);
        }
        put(&row[0], e + wsum);
        if (tid < (1 << tp.rb)) {
            double q = 0.0;
            for (int i = 0; i < tp.rb; ++i)
                for (int j = i + 1; j < tp.rb; ++j) {
                    const double c = J[tp.rg[i] * nq + tp.rg[j]];
                    q += (((tid >> i) ^ (tid >> j)) & 1) ? -c : c;
                }
            put(base + (size_t)blockDim.x * (1 + tp.rb) + tid, q);
        }
        return;
    }
    const uint64_t t = (uint64_t)(blockIdx.x - 1) * blockDim.x + tid;
    if (t >= (1ull << tp.n_free)) return;
    const uint64_t tbase = expand_bits(t, tp.tins);  // the tile's outside bits
    uint64_t tmask = 0;
    for (int i = 0; i < tp.k; ++i) tmask |= 1ull << tp.gb[i];
    double2 *row = base + (size_t)blockDim.x * (1 + tp.rb) + (1 << tp.rb) + t * (tp.k + 1);
    for (int i = 0; i < tp.k; ++i) {
        const int g = tp.gb[i];
        double acc = hv[g];
        for (int o = 0; o < nq; ++o)
            if (!((tmask >> o) & 1ull)) acc += ((tbase >> o) & 1ull) ? -J[g * nq + o] : J[g * nq + o];
        put(&row[i], acc);
    }
    double eo = hv[nq];
    for (int o = 0; o < nq; ++o) {
        if ((tmask >> o) & 1ull) continue;
        const double zo = ((tbase >> o) & 1ull) ? -1.0 : 1.0;
        double r = hv[o];
        for (int o2 = o + 1; o2 < nq; ++o2)
            if (!((tmask >> o2) & 1ull)) r += ((tbase >> o2) & 1ull) ? -J[o * nq + o2] : J[o * nq + o2];
        eo += zo * r;
    }
    put(&row[tp.k], eo);
}

qs_status k_ising_table(qs_state *s, const IsingTabP &tp) {
    if (tp.members <= 0) return QS_OK;
    ProfScope _ps(s->stream, KC_TROTTER_DIAG);
    const dim3 grid(1 + (unsigned)(((1ull << tp.n_free) + 255) / 256), (unsigned)tp.members);
    ising_table_kernel<<<grid, 256, 0, s->stream>>>(tp);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}


// MODE selects the ops compiled in (see tile_op).
template <typename R, int RB, int MODE>
__global__ void __launch_bounds__(32 << TileCfg<R>::WB, TileCfg<R>::kMinBlocks)
    tiled_kernel(V<R> *__restrict__ psi, const __grid_constant__ TileParams<R> p) {
    constexpr int NR = 1 << RB;
    constexpr int WB = TileCfg<R>::WB;
    constexpr int NW = 1 << WB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem_raw + (sizeof(V<R>) << p.k));
    uint16_t *ltab = reinterpret_cast<uint16_t *>(tab + p.n_stages * (NW * 32));
    __shared__ GradT<R> gsm[kTileMaxGrad][NW];
    __shared__ V<R> s_e[16];
    __shared__ V<R> s_qp[NR];
    const TileScratch<R> sc{gsm, s_e, s_qp};
    const TilePtrs<R> q{p.pmat, p.gpart, p.ising_thr};
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    V<R> a[NR];
    tile_tables<R, RB>(p, tab, ltab, lane, warp);
    for (uint64_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
        const uint64_t tbase = tile_base<R>(p, t);
        tile_load<R, RB>(a, psi, p, tbase, lane, warp);
        for (int s = 0; s < p.n_stages; ++s) {
            const TileStage &st = p.st[s];
            if (s > 0) tile_transpose<R, RB>(a, smem_raw, tab, p, s);
            const uint32_t lt = st.need_lt ? (uint32_t)ltab[s * (NW * 32) + threadIdx.x] : 0u;
            for (int o = st.op_begin; o < st.op_end; ++o)
                tile_op<R, RB, MODE>(a, p, p.mat, p.dfac, q, o, st, t, tbase, lt, lane, warp, sc);
        }
        tile_store<R, RB>(psi, a, p, tbase, lane, warp);
        if (MODE == 2 && p.n_grad > 0) tile_grad_flush<R>(p, q, t, sc);
    }
}

template <typename R>
static qs_status launch_tiled_t(qs_state *s, const TileParams<R> &p, int mode) {
    constexpr int RB = TileCfg<R>::RB;
    constexpr int threads = 32 << TileCfg<R>::WB;
    // the tile, then the transpose-offset and local-index tables (6 bytes per
    // stage and thread)
    constexpr size_t per_stage = threads * (sizeof(uint32_t) + sizeof(uint16_t));
    const size_t smem = (sizeof(V<R>) << p.k) + (size_t)std::max(p.n_stages, 1) * per_stage;
    const size_t smem_max = (sizeof(V<R>) << tile_bits(sizeof(R) == 4 ? QS_C64 : QS_C128)) +
                            (size_t)kTileMaxStages * per_stage;
    static int configured[64] = {0};
    const int dev = (s->device >= 0 && s->device < 64) ? s->device : 0;
    static int blocks_per_sm[64] = {0};
    if (!configured[dev]) {
        QS_CUDA_TRY(cudaFuncSetAttribute(tiled_kernel<R, RB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max));
        QS_CUDA_TRY(cudaFuncSetAttribute(tiled_kernel<R, RB, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max));
        QS_CUDA_TRY(cudaFuncSetAttribute(tiled_kernel<R, RB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max));
        int bps = 0;
        QS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tiled_kernel<R, RB, 2>, threads,
                                                                  smem_max));
        int sms = 0;
        QS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        blocks_per_sm[dev] = std::max(1, bps) * sms;
        configured[dev] = 1;
    }
    const uint64_t grid = std::min<uint64_t>(p.total_tiles, (uint64_t)blocks_per_sm[dev]);
    if (grid == 0) return QS_OK;
    ProfScope _ps(s->stream, KC_TILED);
    bool launched = false;
    QS_TRY(tile_jit_launch_t<R>(s, p, &launched));  // the pass's specialised kernel, if ready
    if (launched) return QS_OK;
    if (mode == 2)
        tiled_kernel<R, RB, 2><<<(unsigned)grid, threads, smem, s->stream>>>((V<R> *)s->data, p);
    else if (mode == 1)
        tiled_kernel<R, RB, 1><<<(unsigned)grid, threads, smem, s->stream>>>((V<R> *)s->data, p);
    else
        tiled_kernel<R, RB, 0><<<(unsigned)grid, threads, smem, s->stream>>>((V<R> *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// one-time per-device kernel attributes (done before any graph capture)
qs_status tiled_configure(qs_state *s) {
    TileParams<float> pf;
    std::memset(&pf, 0, sizeof(pf));
    pf.k = tile_bits(QS_C64);
    // total_tiles = 0: the launches configure the attributes and do no work
    QS_TRY(launch_tiled_t<float>(s, pf, 2));
    static thread_local TileParams<double> pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.k = tile_bits(QS_C128);
    QS_TRY(launch_tiled_t<double>(s, pd, 2));
    static thread_local TileParams<dd> pq;
    std::memset(&pq, 0, sizeof(pq));
    pq.k = tile_bits(QS_C128);
    return launch_tiled_t<dd>(s, pq, 2);
}

// the smallest kernel MODE that holds every op of the pass
template <typename R> static int kernel_mode(const TileParams<R> &p) {
    int mode = p.n_grad > 0 ? 2 : 0;
    for (int st = 0; st < p.n_stages; ++st)
        for (int o = p.st[st].op_begin; o < p.st[st].op_end; ++o) {
            const int t = p.op[o].type;
            if (t == TOP_DENSE2_RR || t == TOP_SWAP_RR || t == TOP_ISING || t == TOP_GRAD) return 2;
            if (t == TOP_DENSE1_R || t == TOP_DENSE1_L || t == TOP_ROTS_L || t == TOP_PROT) mode = 1;
        }
    return mode;
}

qs_status k_tiled_pass_c64(qs_state *s, const TileParams<float> &p) {
    return launch_tiled_t<float>(s, p, kernel_mode(p));
}
// A complex128 pass runs in double-float arithmetic unless FP64 is asked for;
// per-member matrices must then be in a double-float table (s->ptab_dd). The
// descriptor converts in place: its values (matrix entries, diagonal factors)
// become float pairs, everything else is copied.
static bool double_float_pass(const qs_state *s, const TileParams<double> &p) {
    if (c128_fp64()) return false;
    for (int st = 0; st < p.n_stages; ++st)
        for (int o = p.st[st].op_begin; o < p.st[st].op_end; ++o)
            if (p.op[o].pm && !s->ptab_dd) return false;
    return true;
}

qs_status k_tiled_pass_c128(qs_state *s, const TileParams<double> &p) {
    if (!double_float_pass(s, p)) return launch_tiled_t<double>(s, p, kernel_mode(p));
    static thread_local TileParams<dd> q;
    std::memcpy(&q, &p, sizeof(p));
    q.pmat = s->ptab_dd ? reinterpret_cast<const ddc *>(p.pmat) : nullptr;
    auto cv = [](double2 v) { return mkc<dd>(dd(v.x), dd(v.y)); };
    for (int i = 0; i < kTileMaxMat; ++i) q.mat[i] = cv(p.mat[i]);
    for (int f = 0; f < kTileMaxDFac; ++f) {
        const TileDFac<double> &d = p.dfac[f];
        q.dfac[f].v0 = cv(d.v0);
        q.dfac[f].v1 = cv(d.v1);
        q.dfac[f].v2 = cv(d.v2);
    }
    return launch_tiled_t<dd>(s, q, kernel_mode(q));
}

}  // namespace qsim
