// One-gate-per-pass kernels (the plain, unfused simulator) and the read-out
// reductions.
//
//  * dense k-qubit gate (k = 1..5) with controls: Eq. (1), Sec. 2.3-2.4; every
//    thread owns one index group of 2^k amplitudes whose control bits are 1,
//    so controlled gates touch only the 2^(n-c) amplitudes they change;
//  * diagonal gates: only the amplitudes a diagonal changes are touched
//    (Sec. 2.3: "Z flips the sign of half the components"); a phase gate
//    (Z, S, T, U1, CZ, CU1, multi-controlled Z) touches 2^(n-c) amplitudes;
//  * SWAP exchanges the |01> and |10> sub-blocks (QFT, Sec. 3.1);
//  * probabilities |psi_x|^2 (Sec. 2.4, "Measurements"), squared norm and
//    Pauli-sum expectation values (Sec. 2.4, Energy callback), all with FP64
//    accumulation and a fixed reduction order (run-to-run deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

static int sm_count(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 148;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
            v = 148;
        cached[device] = v;
    }
    return cached[device];
}

static unsigned grid_for(const qs_state *s, uint64_t work, int threads, int waves = 8) {
    const uint64_t need = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sm_count(s->device) * (uint64_t)waves * (2048 / threads);
    return (unsigned)std::max<uint64_t>(1, std::min(need, cap));
}

static void fill_insert(InsertBits *ib, uint64_t bits) {
    ib->count = 0;
    for (int p = 0; p < 64; ++p)
        if ((bits >> p) & 1ull) ib->pos[ib->count++] = (int8_t)p;
}

// ================================================================== init
// psi = (re, 0) everywhere, then 1 at index x of every member if x is valid
template <typename R>
__global__ void fill_kernel(V<R> *psi, uint64_t total, int n, int ms, R re, uint64_t x) {
    const uint64_t mask = (1ull << n) - 1ull;
    for (uint64_t i = global_tid(); i < total; i += global_stride()) {
        const uint64_t xi = i & mask;
        psi[((i >> n) << ms) | xi] = mkc<R>(xi == x ? (R)1 : re, 0);
    }
}

static size_t amp_bytes(const qs_state *s) { return s->dtype == QS_C64 ? 8 : 16; }

// algorithmic work of a launch over `touched` amplitudes, each read and written once
static void tally(int cls, const qs_state *s, double touched, double flops_per_amp) {
    if (prof_enabled()) prof_add_work(cls, 2.0 * touched * (double)amp_bytes(s), touched * flops_per_amp);
}

qs_status k_init_basis(qs_state *s, uint64_t x) {
    const uint64_t total = (uint64_t)s->batch << s->n;
    ProfScope _ps(s->stream, KC_INIT, (double)total * amp_bytes(s));
    const unsigned g = grid_for(s, total, 256);
    if (s->dtype == QS_C64)
        fill_kernel<float><<<g, 256, 0, s->stream>>>((float2 *)s->data, total, s->n, s->ms, 0.f, x);
    else
        fill_kernel<double><<<g, 256, 0, s->stream>>>((double2 *)s->data, total, s->n, s->ms, 0.0, x);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

qs_status k_init_plus(qs_state *s) {
    const uint64_t total = (uint64_t)s->batch << s->n;
    ProfScope _ps(s->stream, KC_INIT, (double)total * amp_bytes(s));
    const double a = std::pow(2.0, -0.5 * s->n);
    const unsigned g = grid_for(s, total, 256);
    if (s->dtype == QS_C64)
        fill_kernel<float><<<g, 256, 0, s->stream>>>((float2 *)s->data, total, s->n, s->ms, (float)a, ~0ull);
    else
        fill_kernel<double><<<g, 256, 0, s->stream>>>((double2 *)s->data, total, s->n, s->ms, a, ~0ull);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ================================================================== dense k-qubit gate
template <typename R, int K> struct DenseP {
    V<R> m[(1 << K) * (1 << K)];
    uint64_t off[1 << K];
    uint64_t setmask;
    InsertBits ib;
    int n;
    int n_free;
    uint64_t total;
};

template <typename R, int K>
__global__ void __launch_bounds__(256) dense_kernel(V<R> *__restrict__ psi,
                                                    const __grid_constant__ DenseP<R, K> p) {
    constexpr int D = 1 << K;
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    for (uint64_t g = global_tid(); g < p.total; g += global_stride()) {
        const uint64_t b = g >> p.n_free;
        const uint64_t base = (b << p.n) | expand_bits(g & fmask, p.ib) | p.setmask;
        V<R> a[D];
#pragma unroll
        for (int l = 0; l < D; ++l) a[l] = psi[base | p.off[l]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            V<R> acc = mkc<R>(0, 0);
#pragma unroll
            for (int c = 0; c < D; ++c) acc = cmadd<R>(p.m[r * D + c], a[c], acc);
            psi[base | p.off[r]] = acc;
        }
    }
}

template <typename R, int K>
static qs_status launch_dense(qs_state *s, const LGate &g) {
    ProfScope _ps(s->stream, KC_DENSE);
    DenseP<R, K> p;
    constexpr int D = 1 << K;
    for (int i = 0; i < D * D; ++i) p.m[i] = mkc<R>((R)g.m[i].real(), (R)g.m[i].imag());
    uint64_t tmask = 0;
    for (int j = 0; j < K; ++j) tmask |= 1ull << g.tbit[j];
    for (int l = 0; l < D; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((l >> (K - 1 - j)) & 1) o |= 1ull << g.tbit[j];
        p.off[l] = o;
    }
    p.setmask = g.cmask;
    fill_insert(&p.ib, tmask | g.cmask);
    p.n = s->ms;  // member shift
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    tally(KC_DENSE, s, (double)p.total * D, 8.0 * D);
    dense_kernel<R, K><<<grid_for(s, p.total, 256), 256, 0, s->stream>>>((V<R> *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ================================================================== diagonal gates
template <typename R> struct PhaseP {
    V<R> ph;
    uint64_t setmask;
    InsertBits ib;
    int n;
    int n_free;
    uint64_t total;
};

// psi[x] *= ph for every x whose `setmask` bits are all 1
template <typename R>
__global__ void __launch_bounds__(256) phase_kernel(V<R> *__restrict__ psi,
                                                    const __grid_constant__ PhaseP<R> p) {
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    for (uint64_t g = global_tid(); g < p.total; g += global_stride()) {
        const uint64_t x = ((g >> p.n_free) << p.n) | expand_bits(g & fmask, p.ib) | p.setmask;
        psi[x] = cmul<R>(psi[x], p.ph);
    }
}

template <typename R, int K> struct DiagP {
    V<R> d[1 << K];
    int tbit[K];
    uint64_t setmask;
    InsertBits ib;
    int n;
    int n_free;
    uint64_t total;
};

// psi[x] *= d[local(x)] for every x whose control bits are all 1
template <typename R, int K>
__global__ void __launch_bounds__(256) diag_kernel(V<R> *__restrict__ psi,
                                                   const __grid_constant__ DiagP<R, K> p) {
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    for (uint64_t g = global_tid(); g < p.total; g += global_stride()) {
        const uint64_t x = ((g >> p.n_free) << p.n) | expand_bits(g & fmask, p.ib) | p.setmask;
        int l = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) l |= (int)((x >> p.tbit[j]) & 1ull) << (K - 1 - j);
        psi[x] = cmul<R>(psi[x], p.d[l]);
    }
}

template <typename R>
static qs_status launch_phase(qs_state *s, uint64_t setmask, std::complex<double> ph) {
    ProfScope _ps(s->stream, KC_PHASE);
    PhaseP<R> p;
    p.ph = mkc<R>((R)ph.real(), (R)ph.imag());
    p.setmask = setmask;
    fill_insert(&p.ib, setmask);
    p.n = s->ms;  // member shift
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    tally(KC_PHASE, s, (double)p.total, 6.0);
    phase_kernel<R><<<grid_for(s, p.total, 256), 256, 0, s->stream>>>((V<R> *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

template <typename R, int K>
static qs_status launch_diag(qs_state *s, const LGate &g) {
    ProfScope _ps(s->stream, KC_DIAG);
    DiagP<R, K> p;
    constexpr int D = 1 << K;
    for (int l = 0; l < D; ++l) p.d[l] = mkc<R>((R)g.m[l * D + l].real(), (R)g.m[l * D + l].imag());
    for (int j = 0; j < K; ++j) p.tbit[j] = g.tbit[j];
    p.setmask = g.cmask;
    fill_insert(&p.ib, g.cmask);
    p.n = s->ms;  // member shift
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    tally(KC_DIAG, s, (double)p.total, 6.0);
    diag_kernel<R, K><<<grid_for(s, p.total, 256), 256, 0, s->stream>>>((V<R> *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ================================================================== SWAP
struct SwapP {
    uint64_t A, B, setmask;
    InsertBits ib;
    int n;
    int n_free;
    uint64_t total;
};

template <typename R>
__global__ void __launch_bounds__(256) swap_kernel(V<R> *__restrict__ psi,
                                                   const __grid_constant__ SwapP p) {
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    for (uint64_t g = global_tid(); g < p.total; g += global_stride()) {
        const uint64_t x = ((g >> p.n_free) << p.n) | expand_bits(g & fmask, p.ib) | p.setmask;
        const V<R> a = psi[x | p.A];
        const V<R> b = psi[x | p.B];
        psi[x | p.A] = b;
        psi[x | p.B] = a;
    }
}

template <typename R>
static qs_status launch_swap(qs_state *s, const LGate &g) {
    ProfScope _ps(s->stream, KC_SWAP);
    SwapP p;
    p.A = 1ull << g.tbit[0];
    p.B = 1ull << g.tbit[1];
    p.setmask = g.cmask;
    fill_insert(&p.ib, p.A | p.B | g.cmask);
    p.n = s->ms;  // member shift
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    tally(KC_SWAP, s, 2.0 * (double)p.total, 0.0);
    swap_kernel<R><<<grid_for(s, p.total, 256), 256, 0, s->stream>>>((V<R> *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

bool k_dense_df(qs_state *s, const LGate &g, qs_status *st);

thread_local bool t_c128_fp64 = false;
void set_c128_fp64(bool on) { t_c128_fp64 = on; }
bool c128_fp64() { return t_c128_fp64; }

template <typename R>
static qs_status apply_unfused_t(qs_state *s, const LGate &g) {
    const int K = 1 << g.k;
    if (g.is_swap) return launch_swap<R>(s, g);
    if (g.phase_only) {
        uint64_t setmask = g.cmask;
        for (int j = 0; j < g.k; ++j) setmask |= 1ull << g.tbit[j];
        const std::complex<double> ph = g.m[(K - 1) * K + (K - 1)];
        if (ph == std::complex<double>(1.0, 0.0)) return QS_OK;  // identity
        return launch_phase<R>(s, setmask, ph);
    }
    if (g.diagonal) {
        switch (g.k) {
        case 1: return launch_diag<R, 1>(s, g);
        case 2: return launch_diag<R, 2>(s, g);
        case 3: return launch_diag<R, 3>(s, g);
        case 4: return launch_diag<R, 4>(s, g);
        case 5: return launch_diag<R, 5>(s, g);
        }
    }
    if (sizeof(R) == 8 && !t_c128_fp64) {  // complex128 dense gates: double-float on the FP32 pipes
        qs_status st = QS_OK;
        if (k_dense_df(s, g, &st)) return st;
    }
    switch (g.k) {
    case 1: return launch_dense<R, 1>(s, g);
    case 2: return launch_dense<R, 2>(s, g);
    case 3: return launch_dense<R, 3>(s, g);
    case 4: return launch_dense<R, 4>(s, g);
    case 5: return launch_dense<R, 5>(s, g);
    }
    set_error("gate with %d targets", g.k);
    return QS_ERR_ARG;
}

qs_status k_apply_unfused(qs_state *s, const LGate &g) {
    return s->dtype == QS_C64 ? apply_unfused_t<float>(s, g) : apply_unfused_t<double>(s, g);
}

// ================================================================== reductions
qs_status ensure_scratch(qs_state *s, size_t doubles) {
    if (s->scratch_doubles >= doubles) return QS_OK;
    if (s->scratch) {
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_doubles = 0;
    }
    QS_CUDA_TRY(cudaMalloc(&s->scratch, doubles * sizeof(double)));
    s->scratch_doubles = doubles;
    return QS_OK;
}

qs_status ensure_host_pinned(qs_state *s, size_t doubles) {
    if (s->host_pinned_doubles >= doubles) return QS_OK;
    if (s->host_pinned) {
        cudaFreeHost(s->host_pinned);
        s->host_pinned = nullptr;
        s->host_pinned_doubles = 0;
    }
    QS_CUDA_TRY(cudaMallocHost(&s->host_pinned, doubles * sizeof(double)));
    s->host_pinned_doubles = doubles;
    return QS_OK;
}

template <typename R>
__global__ void probs_kernel(const V<R> *__restrict__ psi, double *__restrict__ out, uint64_t total) {
    for (uint64_t i = global_tid(); i < total; i += global_stride()) {
        const V<R> a = psi[i];
        const double re = (double)a.x, im = (double)a.y;
        out[i] = re * re + im * im;
    }
}

qs_status k_probabilities(qs_state *s, double *out_dev) {
    const uint64_t total = (uint64_t)s->batch << s->n;
    ProfScope _ps(s->stream, KC_REDUCE, (double)total * (amp_bytes(s) + 8), 3.0 * total);
    const unsigned g = grid_for(s, total, 256);
    if (s->dtype == QS_C64)
        probs_kernel<float><<<g, 256, 0, s->stream>>>((const float2 *)s->data, out_dev, total);
    else
        probs_kernel<double><<<g, 256, 0, s->stream>>>((const double2 *)s->data, out_dev, total);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// Block-wide sum of two doubles; result valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
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

constexpr int kRedThreads = 256;

static int red_blocks_per_member(const qs_state *s) {
    const uint64_t per = 1ull << s->n;
    const uint64_t want = std::max<uint64_t>(1, per / (kRedThreads * 16));
    const uint64_t cap = std::max<uint64_t>(1, (uint64_t)sm_count(s->device) * 8 / s->batch);
    return (int)std::min<uint64_t>(std::min<uint64_t>(want, cap), 4096);
}

// Each thread sums runs of kChunk amplitudes and adds every run to an FP64
// accumulator, so FP64 carries the reduction across the state while the
// per-amplitude work stays off GB300's FP64 pipe (about 1/60 of the FP32
// rate). For complex64 the run sum is error-free to float-float precision:
// squares are split exactly with a fused multiply-add (x*x = p + e) and the
// large parts are added with Knuth's TwoSum, so a run's value carries ~48
// significant bits, like the FP64 sum it replaces.
constexpr int kChunk = 16;

template <typename R> struct RunSum {
    R s = 0;
    __device__ __forceinline__ void add_sq(R x, R y) { s = fma(x, x, fma(y, y, s)); }
    __device__ __forceinline__ double value() const { return (double)s; }
};

template <> struct RunSum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void two_sum(float v) {
        const float t = hi + v;
        const float bv = t - hi;
        lo += (hi - (t - bv)) + (v - bv);
        hi = t;
    }
    __device__ __forceinline__ void add_sq(float x, float y) {
        const float px = x * x, py = y * y;
        lo += fmaf(x, x, -px) + fmaf(y, y, -py);
        two_sum(px);
        two_sum(py);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename R>
__global__ void __launch_bounds__(kRedThreads) norm2_partial_kernel(const V<R> *__restrict__ psi, int n, int ms,
                                                                    double2 *__restrict__ part) {
    const uint64_t per = 1ull << n;
    const V<R> *p = psi + ((uint64_t)blockIdx.y << ms);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // full runs: all kChunk loads in flight before the arithmetic
    while (i + (kChunk - 1) * stride < per) {
        V<R> av[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) av[c] = p[i + c * stride];
        RunSum<R> run;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) run.add_sq(av[c].x, av[c].y);
        acc += run.value();
        i += kChunk * stride;
    }
    {
        RunSum<R> run;
        for (; i < per; i += stride) {
            const V<R> a = p[i];
            run.add_sq(a.x, a.y);
        }
        acc += run.value();
    }
    const double2 r = block_sum2(acc, 0.0);
    if (threadIdx.x == 0) part[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
}

// out[b] = sum of the member's partials (x and y parts), in a fixed order
__global__ void finalize_kernel(const double2 *__restrict__ part, int per_member, double *__restrict__ out,
                                int two) {
    const int b = blockIdx.x;
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < per_member; i += blockDim.x) {
        x += part[(uint64_t)b * per_member + i].x;
        y += part[(uint64_t)b * per_member + i].y;
    }
    const double2 r = block_sum2(x, y);
    if (threadIdx.x == 0) {
        if (two) {
            out[2 * b] = r.x;
            out[2 * b + 1] = r.y;
        } else {
            out[b] = r.x;
        }
    }
}

qs_status k_norm2(qs_state *s, double **out) {
    const int P = red_blocks_per_member(s);
    QS_TRY(ensure_scratch(s, (size_t)2 * P * s->batch + 2 * (size_t)s->batch));
    double *out_dev = s->scratch + (size_t)2 * P * s->batch;
    *out = out_dev;
    ProfScope _ps(s->stream, KC_REDUCE, (double)((uint64_t)s->batch << s->n) * amp_bytes(s),
                  4.0 * (double)((uint64_t)s->batch << s->n));
    dim3 grid(P, s->batch);
    if (s->dtype == QS_C64)
        norm2_partial_kernel<float><<<grid, kRedThreads, 0, s->stream>>>((const float2 *)s->data, s->n, s->ms,
                                                                          (double2 *)s->scratch);
    else
        norm2_partial_kernel<double><<<grid, kRedThreads, 0, s->stream>>>((const double2 *)s->data, s->n, s->ms,
                                                                           (double2 *)s->scratch);
    QS_CUDA_TRY(cudaGetLastError());
    finalize_kernel<<<s->batch, kRedThreads, 0, s->stream>>>((const double2 *)s->scratch, P, out_dev, 0);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ------------------------------------------------------------------ Pauli expectation
// Terms sharing one X mask m form f_m(x) = sum_t c_t i^{#Y_t} (-1)^{popcount(x & z_t)},
// and <psi|H|psi> = sum_m sum_x conj(psi[x ^ m]) f_m(x) psi[x].
constexpr int kMaxTermsPerLaunch = 256;

template <typename R> struct ExpP {
    R cre[kMaxTermsPerLaunch];
    R cim[kMaxTermsPerLaunch];
    uint64_t zb[kMaxTermsPerLaunch];
    int8_t za[kMaxTermsPerLaunch];   // first Z bit, or -1
    int8_t zc[kMaxTermsPerLaunch];   // second Z bit, or -1
    int8_t zn[kMaxTermsPerLaunch];   // number of Z bits: 0, 1, 2 or 3 (= more)
    int8_t ys[kMaxTermsPerLaunch];   // (-1)^{popcount(z_t & xb)}: the term's sign at x ^ xb relative to x
    // one- and two-bit terms: bits 0-7 first Z bit a, 8-15 second bit b (= a
    // for one bit), bit 16: two bits; parity = ((x >> a) ^ ((x >> b) & two)) & 1
    uint32_t zw[kMaxTermsPerLaunch];
    // diagonal group (xb = 0), chunked: the varying terms sorted by cm, the
    // chunk bits their Z bits include (bit i = index bit kExpChunkLo + i);
    // vord[vmb[m] .. vmb[m+1]) are the ones with cm = m
    uint8_t cm[kMaxTermsPerLaunch];
    uint8_t vord[kMaxTermsPerLaunch];
    int vmb[17];
    int nt;
    int nv;           // terms [0, nv) touch the chunk bits (see expect_partial_kernel)
    int nvf, nff;     // [0, nvf) and [nv, nff): one- and two-bit terms; the rest general
    uint64_t xb;      // X mask in index bits (0 for the diagonal group)
    int n;
    int ms;           // member shift
    int n_free;       // n (diagonal group) or n - 1 (pairs)
    int hb;           // highest bit of xb (pairs)
    int accumulate;   // add to the partials instead of overwriting
};

// (-1)^{popcount(x & z_t)}, with shift-and-xor for one- and two-bit masks
template <typename R>
__device__ __forceinline__ bool term_odd(const ExpP<R> &p, int t, uint64_t x) {
    switch (p.zn[t]) {
    case 0: return false;
    case 1: return (x >> p.za[t]) & 1ull;
    case 2: return ((x >> p.za[t]) ^ (x >> p.zc[t])) & 1ull;
    default: return __popcll(x & p.zb[t]) & 1;
    }
}

// Free-index bits that vary inside one thread's chunk: 16 amplitudes at
// j = chunk * 4096 + c * 256 + thread, c = 0..15 (bits 8..11 of j).
constexpr int kExpChunkLo = 8, kExpChunkBits = 4;

// Host: order the terms so that those whose Z bits meet the chunk bits come
// first (p->nv of them); the others are constant over a chunk and are summed
// once per chunk. Within each part the one- and two-bit terms come first
// (evaluated by shifts), then the others (popcount). Also the per-term sign
// between x and x ^ xb.
template <typename R> static void exp_order_terms(ExpP<R> *p) {
    uint64_t cx = 0;
    for (int b = kExpChunkLo; b < kExpChunkLo + kExpChunkBits; ++b)
        cx |= 1ull << ((p->xb && b >= p->hb) ? b + 1 : b);
    ExpP<R> q = *p;
    int k = 0;
    for (int pass = 0; pass < 4; ++pass) {
        for (int t = 0; t < p->nt; ++t) {
            const bool varying = (p->zb[t] & cx) != 0;
            const bool fast = p->zn[t] == 1 || p->zn[t] == 2;
            if (varying != (pass < 2) || fast != (pass % 2 == 0)) continue;
            q.cre[k] = p->cre[t];
            q.cim[k] = p->cim[t];
            q.zb[k] = p->zb[t];
            q.za[k] = p->za[t];
            q.zc[k] = p->zc[t];
            q.zn[k] = p->zn[t];
            q.ys[k] = (int8_t)(__builtin_popcountll(p->zb[t] & p->xb) & 1);
            q.zw[k] = fast ? ((uint32_t)p->za[t] | ((uint32_t)(p->zn[t] == 2 ? p->zc[t] : p->za[t]) << 8) |
                              ((uint32_t)(p->zn[t] == 2) << 16))
                           : 0u;
            ++k;
        }
        if (pass == 0) q.nvf = k;
        if (pass == 1) q.nv = k;
        if (pass == 2) q.nff = k;
    }
    if (q.xb == 0) {
        for (int t = 0; t < q.nv; ++t)
            q.cm[t] = (uint8_t)((q.zb[t] >> kExpChunkLo) & ((1u << kExpChunkBits) - 1u));
        int k2 = 0;
        for (int m = 0; m < (1 << kExpChunkBits); ++m) {
            q.vmb[m] = k2;
            for (int t = 0; t < q.nv; ++t)
                if (q.cm[t] == m) q.vord[k2++] = (uint8_t)t;
        }
        q.vmb[1 << kExpChunkBits] = k2;
    }
    *p = q;
}

// f_m at x (fr, fi) and at x ^ xb (gr, gi), adding terms [t0, t1)
template <typename R>
__device__ __forceinline__ void exp_terms(const ExpP<R> &p, int t0, int t1, uint64_t x, R &fr, R &fi, R &gr,
                                          R &gi) {
    for (int t = t0; t < t1; ++t) {
        const bool sx = term_odd(p, t, x);
        const R cr = sx ? -p.cre[t] : p.cre[t], ci = sx ? -p.cim[t] : p.cim[t];
        fr += cr;
        fi += ci;
        gr += p.ys[t] ? -cr : cr;
        gi += p.ys[t] ? -ci : ci;
    }
}

// the same for one- and two-bit terms, by shifts on an index of type U
template <typename R, typename U>
__device__ __forceinline__ void exp_terms_fast(const ExpP<R> &p, int t0, int t1, U x, R &fr, R &fi, R &gr,
                                               R &gi) {
    for (int t = t0; t < t1; ++t) {
        const uint32_t w = p.zw[t];
        const bool sx = ((x >> (w & 0xffu)) ^ ((x >> ((w >> 8) & 0xffu)) & (U)((w >> 16) & 1u))) & 1u;
        const R cr = sx ? -p.cre[t] : p.cre[t], ci = sx ? -p.cim[t] : p.cim[t];
        fr += cr;
        fi += ci;
        gr += p.ys[t] ? -cr : cr;
        gi += p.ys[t] ? -ci : ci;
    }
}

// all terms of [t0, t1) that the ordering put in a fast or general run
template <typename R, typename U>
__device__ __forceinline__ void exp_range(const ExpP<R> &p, bool varying, U x, R &fr, R &fi, R &gr, R &gi) {
    if (varying) {
        exp_terms_fast<R, U>(p, 0, p.nvf, x, fr, fi, gr, gi);
        exp_terms(p, p.nvf, p.nv, (uint64_t)x, fr, fi, gr, gi);
    } else {
        exp_terms_fast<R, U>(p, p.nv, p.nff, x, fr, fi, gr, gi);
        exp_terms(p, p.nff, p.nt, (uint64_t)x, fr, fi, gr, gi);
    }
}

// Per member: sum_x |psi[x]|^2 f_0(x) (diagonal group), or sum over the pairs
// (x, y = x ^ xb) with bit hb of x clear of conj(psi[y]) psi[x] f(x) +
// conj(psi[x]) psi[y] f(y). For 2^12 or more free indices a thread takes
// chunks of 16 amplitudes (consecutive threads on consecutive addresses for
// each c); terms that do not touch the chunk bits are summed once per chunk,
// the others per amplitude. Runs of 16 are summed in R, then in FP64. U: the
// index type (32-bit while the indices fit).
template <typename R, typename U>
__device__ __forceinline__ double2 expect_body(const V<R> *__restrict__ q, const ExpP<R> &p) {
    const uint64_t cnt = 1ull << p.n_free;
    double ar = 0.0, ai = 0.0;
    const U lo = (U)((1ull << p.hb) - 1ull);
    const U xb = (U)p.xb;
    auto insert0 = [&](U j) { return p.xb ? (U)(((j >> p.hb) << (p.hb + 1)) | (j & lo)) : j; };
    if (p.n_free >= kExpChunkLo + kExpChunkBits) {
        const uint64_t nchunks = cnt >> (kExpChunkLo + kExpChunkBits);
        for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
            const U j0 = (U)((ch << (kExpChunkLo + kExpChunkBits)) | threadIdx.x);
            R f0r = 0, f0i = 0, g0r = 0, g0i = 0;
            exp_range<R, U>(p, false, insert0(j0), f0r, f0i, g0r, g0i);
            R rr = 0, ri = 0;
            if (p.xb == 0) {
                // all 16 loads in flight before the arithmetic
                V<R> av[1 << kExpChunkBits];
#pragma unroll
                for (int c = 0; c < (1 << kExpChunkBits); ++c) av[c] = q[j0 | ((U)c << kExpChunkLo)];
                // varying terms: sign from the bits outside the chunk (x with chunk
                // bits 0), summed per chunk-bit mask m into F[m]; then
                // f(c) = f0 + sum_m F[m] (-1)^{popcount(c & m)}, the Walsh-Hadamard
                // transform of F (no per-amplitude term evaluation)
                R F[1 << kExpChunkBits];
#pragma unroll
                for (int m = 0; m < (1 << kExpChunkBits); ++m) {
                    R acc = 0;
                    for (int k = p.vmb[m]; k < p.vmb[m + 1]; ++k) {
                        const int t = p.vord[k];
                        acc += term_odd(p, t, (uint64_t)j0) ? -p.cre[t] : p.cre[t];
                    }
                    F[m] = acc;
                }
#pragma unroll
                for (int h = 1; h < (1 << kExpChunkBits); h <<= 1)
#pragma unroll
                    for (int i = 0; i < (1 << kExpChunkBits); ++i)
                        if (!(i & h)) {
                            const R u = F[i], v = F[i | h];
                            F[i] = u + v;
                            F[i | h] = u - v;
                        }
#pragma unroll
                for (int c = 0; c < (1 << kExpChunkBits); ++c)
                    rr = fma(f0r + F[c], fma(av[c].x, av[c].x, av[c].y * av[c].y), rr);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    constexpr int H = (1 << kExpChunkBits) / 2;
                    V<R> av[H], bv[H];
#pragma unroll
                    for (int c = 0; c < H; ++c) {
                        const U x = insert0(j0 | ((U)(h * H + c) << kExpChunkLo));
                        av[c] = q[x];
                        bv[c] = q[x ^ xb];
                    }
#pragma unroll
                    for (int c = 0; c < H; ++c) {
                        const U x = insert0(j0 | ((U)(h * H + c) << kExpChunkLo));
                        R fxr = f0r, fxi = f0i, fyr = g0r, fyi = g0i;
                        exp_range<R, U>(p, true, x, fxr, fxi, fyr, fyi);
                        const V<R> a = av[c], b = bv[c];
                        // conj(b) a f(x) + conj(a) b f(y), with conj(a) b = conj(conj(b) a)
                        const R abr = b.x * a.x + b.y * a.y;
                        const R abi = b.x * a.y - b.y * a.x;
                        rr += abr * (fxr + fyr) - abi * (fxi - fyi);
                        ri += abr * (fxi + fyi) + abi * (fxr - fyr);
                    }
                }
            }
            ar += (double)rr;
            ai += (double)ri;
        }
    } else {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t jj = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; jj < cnt; jj += stride) {
            const U x = insert0((U)jj);
            R fxr = 0, fxi = 0, fyr = 0, fyi = 0;
            exp_range<R, U>(p, true, x, fxr, fxi, fyr, fyi);
            exp_range<R, U>(p, false, x, fxr, fxi, fyr, fyi);
            if (p.xb == 0) {
                const V<R> a = q[x];
                ar += (double)(fxr * fma(a.x, a.x, a.y * a.y));
            } else {
                const V<R> a = q[x], b = q[x ^ xb];
                const R abr = b.x * a.x + b.y * a.y;
                const R abi = b.x * a.y - b.y * a.x;
                ar += (double)(abr * (fxr + fyr) - abi * (fxi - fyi));
                ai += (double)(abr * (fxi + fyi) + abi * (fxr - fyr));
            }
        }
    }
    return make_double2(ar, ai);
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads, 2) expect_partial_kernel(const V<R> *__restrict__ psi,
                                                                     const __grid_constant__ ExpP<R> p,
                                                                     double2 *__restrict__ part) {
    const V<R> *q = psi + ((uint64_t)blockIdx.y << p.ms);
    // indices within a member fit 32 bits up to n = 32
    const double2 acc = p.n <= 32 ? expect_body<R, uint32_t>(q, p) : expect_body<R, uint64_t>(q, p);
    const double2 r = block_sum2(acc.x, acc.y);
    if (threadIdx.x == 0) {
        double2 *slot = &part[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x];
        if (p.accumulate) {
            double2 v = *slot;
            v.x += r.x;
            v.y += r.y;
            *slot = v;
        } else {
            *slot = r;
        }
    }
}

qs_status k_expectation(qs_state *s, const qs_pauli_term *terms, size_t count, double **out) {
    const int n = s->n;
    const int P = red_blocks_per_member(s);
    QS_TRY(ensure_scratch(s, (size_t)2 * P * s->batch + 2 * (size_t)s->batch));
    double *out_dev = s->scratch + (size_t)2 * P * s->batch;
    *out = out_dev;
    // group the terms by X mask (in index bits), keeping first-seen order
    std::vector<uint64_t> masks;
    std::vector<std::vector<size_t>> groups;
    for (size_t t = 0; t < count; ++t) {
        uint64_t xb = 0;
        for (int q = 0; q < n; ++q)
            if ((terms[t].x_mask >> q) & 1ull) xb |= qbit(n, q);
        size_t gi = 0;
        while (gi < masks.size() && masks[gi] != xb) ++gi;
        if (gi == masks.size()) {
            masks.push_back(xb);
            groups.emplace_back();
        }
        groups[gi].push_back(t);
    }
    bool first = true;
    ProfScope _ps(s->stream, KC_REDUCE);
    dim3 grid(P, s->batch);
    for (size_t gi = 0; gi < masks.size(); ++gi) {
        const auto &idx = groups[gi];
        for (size_t c0 = 0; c0 < idx.size(); c0 += kMaxTermsPerLaunch) {
            ExpP<double> p;
            std::memset(&p, 0, sizeof(p));
            p.nt = (int)std::min<size_t>(kMaxTermsPerLaunch, idx.size() - c0);
            for (int j = 0; j < p.nt; ++j) {
                const qs_pauli_term &t = terms[idx[c0 + j]];
                int ny = __builtin_popcountll(t.x_mask & t.z_mask) & 3;
                // c * i^ny
                const double c = t.coeff;
                const double re[4] = {c, 0.0, -c, 0.0}, im[4] = {0.0, c, 0.0, -c};
                p.cre[j] = re[ny];
                p.cim[j] = im[ny];
                uint64_t zb = 0;
                for (int q = 0; q < n; ++q)
                    if ((t.z_mask >> q) & 1ull) zb |= qbit(n, q);
                p.zb[j] = zb;
                const int nz = __builtin_popcountll(zb);
                p.zn[j] = (int8_t)std::min(nz, 3);
                p.za[j] = (int8_t)(nz ? __builtin_ctzll(zb) : -1);
                p.zc[j] = (int8_t)(nz >= 2 ? 63 - __builtin_clzll(zb) : -1);
            }
            p.xb = masks[gi];
            p.n = n;
            p.ms = s->ms;
            p.hb = p.xb ? 63 - __builtin_clzll(p.xb) : 0;
            p.n_free = p.xb ? n - 1 : n;
            p.accumulate = first ? 0 : 1;
            first = false;
            exp_order_terms(&p);
            if (prof_enabled())
                prof_add_work(KC_REDUCE, (double)((uint64_t)s->batch << n) * amp_bytes(s),
                              (double)((uint64_t)s->batch << n) * (2.0 * p.nt + 6.0));
            if (s->dtype == QS_C64) {
                ExpP<float> pf;
                std::memcpy(&pf.zb, &p.zb, sizeof(p.zb));
                std::memcpy(&pf.za, &p.za, sizeof(p.za));
                std::memcpy(&pf.zc, &p.zc, sizeof(p.zc));
                std::memcpy(&pf.zn, &p.zn, sizeof(p.zn));
                std::memcpy(&pf.ys, &p.ys, sizeof(p.ys));
                std::memcpy(&pf.zw, &p.zw, sizeof(p.zw));
                std::memcpy(&pf.cm, &p.cm, sizeof(p.cm));
                std::memcpy(&pf.vord, &p.vord, sizeof(p.vord));
                std::memcpy(&pf.vmb, &p.vmb, sizeof(p.vmb));
                pf.nv = p.nv;
                pf.nvf = p.nvf;
                pf.nff = p.nff;
                for (int j = 0; j < kMaxTermsPerLaunch; ++j) {
                    pf.cre[j] = (float)p.cre[j];
                    pf.cim[j] = (float)p.cim[j];
                }
                pf.nt = p.nt;
                pf.xb = p.xb;
                pf.n = p.n;
                pf.ms = p.ms;
                pf.n_free = p.n_free;
                pf.hb = p.hb;
                pf.accumulate = p.accumulate;
                expect_partial_kernel<float><<<grid, kRedThreads, 0, s->stream>>>(
                    (const float2 *)s->data, pf, (double2 *)s->scratch);
            } else {
                expect_partial_kernel<double><<<grid, kRedThreads, 0, s->stream>>>(
                    (const double2 *)s->data, p, (double2 *)s->scratch);
            }
            QS_CUDA_TRY(cudaGetLastError());
        }
    }
    if (first) {  // no terms: the zero operator
        QS_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * s->batch, s->stream));
        return QS_OK;
    }
    finalize_kernel<<<s->batch, kRedThreads, 0, s->stream>>>((const double2 *)s->scratch, P, out_dev, 1);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ================================================================== diagonal evolution
// psi[x] *= exp(-i tau E(x)), E(x) = sum_t c_t (-1)^{popcount(x & z_t)}: the exact
// exponential of a Z-string Hamiltonian (one factor of the Trotter step, Sec. 2.6).
// The angle tau E(x) is evaluated in FP64.
struct DiagEvoP {
    double c[kMaxTermsPerLaunch];
    uint64_t zb[kMaxTermsPerLaunch];
    int nt;
    int n;
    int ms;
    double tau;
    uint64_t total;
};

template <typename R>
__global__ void __launch_bounds__(256) diag_evo_kernel(V<R> *__restrict__ psi,
                                                       const __grid_constant__ DiagEvoP p) {
    const uint64_t mask = (1ull << p.n) - 1ull;
    for (uint64_t i0 = global_tid(); i0 < p.total; i0 += global_stride()) {
        const uint64_t x = i0 & mask;
        const uint64_t i = ((i0 >> p.n) << p.ms) | x;
        double e = 0.0;
        for (int t = 0; t < p.nt; ++t) e += (__popcll(x & p.zb[t]) & 1) ? -p.c[t] : p.c[t];
        double sn, cs;
        sincos(-p.tau * e, &sn, &cs);
        psi[i] = cmul<R>(psi[i], mkc<R>((R)cs, (R)sn));
    }
}

qs_status k_diagonal_evolution(qs_state *s, const std::vector<double> &coeff,
                               const std::vector<uint64_t> &zbits, double tau) {
    ProfScope _ps(s->stream, KC_TROTTER_DIAG);
    for (size_t c0 = 0; c0 < coeff.size(); c0 += kMaxTermsPerLaunch) {
        DiagEvoP p;
        std::memset(&p, 0, sizeof(p));
        p.nt = (int)std::min<size_t>(kMaxTermsPerLaunch, coeff.size() - c0);
        for (int j = 0; j < p.nt; ++j) {
            p.c[j] = coeff[c0 + j];
            p.zb[j] = zbits[c0 + j];
        }
        p.n = s->n;
        p.ms = s->ms;
        p.tau = tau;
        p.total = (uint64_t)s->batch << s->n;
        tally(KC_TROTTER_DIAG, s, (double)p.total, 2.0 * p.nt + 26.0);
        const unsigned g = grid_for(s, p.total, 256);
        if (s->dtype == QS_C64)
            diag_evo_kernel<float><<<g, 256, 0, s->stream>>>((float2 *)s->data, p);
        else
            diag_evo_kernel<double><<<g, 256, 0, s->stream>>>((double2 *)s->data, p);
        QS_CUDA_TRY(cudaGetLastError());
    }
    return QS_OK;
}

}  // namespace qsim

namespace qsim {

// ================================================================== batched-parameter rotations
// A gate whose angle comes from a device table params[b * n_params + p] (one
// row per batch member). The member's 2x2 matrix (or CU1 phase) is built once
// per member in FP64 by param_matrix_kernel, then applied by dense/phase passes
// that pick the member's entry.
qs_status ensure_gtab(qs_state *s, size_t bytes) {
    if (s->gtab_bytes >= bytes) return QS_OK;
    if (s->gtab) {
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        cudaFree(s->gtab);
        s->gtab = nullptr;
        s->gtab_bytes = 0;
    }
    QS_CUDA_TRY(cudaMalloc(&s->gtab, bytes));
    s->gtab_bytes = bytes;
    return QS_OK;
}

template <typename R>
__global__ void param_matrix_kernel(const double *__restrict__ params, int n_params, int pidx, int kind,
                                    int batch, double sign, V<R> *__restrict__ mats) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double th = sign * params[(uint64_t)b * n_params + pidx];
    double s, c;
    sincos(0.5 * th, &s, &c);
    V<R> *m = mats + 4 * (uint64_t)b;
    switch (kind) {
    case QS_GATE_RX:  // [[c, -is], [-is, c]]
        m[0] = mkc<R>(c, 0); m[1] = mkc<R>(0, -s); m[2] = mkc<R>(0, -s); m[3] = mkc<R>(c, 0);
        break;
    case QS_GATE_RY:  // [[c, -s], [s, c]]
        m[0] = mkc<R>(c, 0); m[1] = mkc<R>(-s, 0); m[2] = mkc<R>(s, 0); m[3] = mkc<R>(c, 0);
        break;
    case QS_GATE_RZ:  // diag(e^{-i th/2}, e^{i th/2})
        m[0] = mkc<R>(c, -s); m[1] = mkc<R>(0, 0); m[2] = mkc<R>(0, 0); m[3] = mkc<R>(c, s);
        break;
    default: {        // U1 / CU1: phase e^{i th} on the all-ones block
        double s2, c2;
        sincos(th, &s2, &c2);
        m[0] = mkc<R>(1, 0); m[1] = mkc<R>(0, 0); m[2] = mkc<R>(0, 0); m[3] = mkc<R>(c2, s2);
    }
    }
}

struct PDenseP {
    uint64_t off1;     // target bit
    uint64_t setmask;  // control bits (and, for phase gates, target bits)
    InsertBits ib;
    int n;
    int n_free;
    int phase_only;
    uint64_t total;
};

template <typename R>
__global__ void __launch_bounds__(256) pdense_kernel(V<R> *__restrict__ psi, const V<R> *__restrict__ mats,
                                                     const __grid_constant__ PDenseP p) {
    const uint64_t fmask = (1ull << p.n_free) - 1ull;
    for (uint64_t g = global_tid(); g < p.total; g += global_stride()) {
        const uint64_t b = g >> p.n_free;
        const uint64_t x = (b << p.n) | expand_bits(g & fmask, p.ib) | p.setmask;
        const V<R> *m = mats + 4 * b;
        if (p.phase_only) {
            psi[x] = cmul<R>(psi[x], m[3]);
        } else {
            const V<R> a0 = psi[x], a1 = psi[x | p.off1];
            psi[x] = cmadd<R>(m[1], a1, cmul<R>(m[0], a0));
            psi[x | p.off1] = cmadd<R>(m[3], a1, cmul<R>(m[2], a0));
        }
    }
}

template <typename R>
static qs_status apply_param_t(qs_state *s, const LGate &g, const double *params, int n_params, double sign) {
    ProfScope _ps(s->stream, KC_PARAM);
    QS_TRY(ensure_gtab(s, sizeof(V<R>) * 4 * (size_t)s->batch));
    param_matrix_kernel<R><<<(s->batch + 127) / 128, 128, 0, s->stream>>>(params, n_params, g.param_index,
                                                                          g.kind, s->batch, sign, (V<R> *)s->gtab);
    QS_CUDA_TRY(cudaGetLastError());
    PDenseP p;
    const bool phase = (g.kind == QS_GATE_U1 || g.kind == QS_GATE_CU1);
    uint64_t tmask = 0;
    for (int j = 0; j < g.k; ++j) tmask |= 1ull << g.tbit[j];
    p.off1 = 1ull << g.tbit[0];
    p.phase_only = phase ? 1 : 0;
    p.setmask = g.cmask | (phase ? tmask : 0);
    fill_insert(&p.ib, tmask | g.cmask);
    p.n = s->ms;  // member shift
    p.n_free = s->n - p.ib.count;
    p.total = (uint64_t)s->batch << p.n_free;
    tally(KC_PARAM, s, (double)p.total * (phase ? 1 : 2), phase ? 6.0 : 16.0);
    pdense_kernel<R><<<grid_for(s, p.total, 256), 256, 0, s->stream>>>((V<R> *)s->data,
                                                                       (const V<R> *)s->gtab, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

constexpr int kPTabSlotsPerLaunch = 512;
struct PTabP {
    int16_t pidx[kPTabSlotsPerLaunch];
    int8_t kind[kPTabSlotsPerLaunch];
    int n_slots;     // slots in this launch
    int slot0;       // first slot index of this launch
    int stride;      // entries per member
    int n_params;
    int batch;
    double sign;
};

template <typename R>
__global__ void param_table_kernel(const double *__restrict__ params, const __grid_constant__ PTabP p,
                                   V<R> *__restrict__ tab) {
    const uint64_t total = (uint64_t)p.batch * p.n_slots;
    for (uint64_t i = global_tid(); i < total; i += global_stride()) {
        const int b = (int)(i / p.n_slots), j = (int)(i % p.n_slots);
        const double th = p.sign * params[(uint64_t)b * p.n_params + p.pidx[j]];
        double sn, cs;
        sincos(0.5 * th, &sn, &cs);
        V<R> *m = tab + (uint64_t)b * p.stride + 4 * (uint64_t)(p.slot0 + j);
        switch (p.kind[j]) {
        case QS_GATE_RX:
            m[0] = mkc<R>(cs, 0); m[1] = mkc<R>(0, -sn); m[2] = mkc<R>(0, -sn); m[3] = mkc<R>(cs, 0);
            break;
        case QS_GATE_RY:
            m[0] = mkc<R>(cs, 0); m[1] = mkc<R>(-sn, 0); m[2] = mkc<R>(sn, 0); m[3] = mkc<R>(cs, 0);
            break;
        case QS_GATE_RZ:  // diagonal (d0, d1)
            m[0] = mkc<R>(cs, -sn); m[1] = mkc<R>(cs, sn); m[2] = mkc<R>(0, 0); m[3] = mkc<R>(0, 0);
            break;
        default: {         // U1 / CU1: the phase on the all-ones block
            double s2, c2;
            sincos(th, &s2, &c2);
            m[0] = mkc<R>(c2, s2); m[1] = mkc<R>(0, 0); m[2] = mkc<R>(0, 0); m[3] = mkc<R>(0, 0);
        }
        }
    }
}

template <typename R>
static qs_status param_table_t(qs_state *s, const std::vector<int> &pidx, const std::vector<int> &kind,
                               const double *params, int n_params, double sign, uint32_t *stride) {
    const int ns = (int)pidx.size();
    const size_t need = sizeof(V<R>) * 4 * (size_t)ns * s->batch;
    if (s->ptab_bytes < need) {
        if (s->ptab) {
            QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
            cudaFree(s->ptab);
            s->ptab = nullptr;
            s->ptab_bytes = 0;
        }
        QS_CUDA_TRY(cudaMalloc(&s->ptab, need));
        s->ptab_bytes = need;
    }
    *stride = (uint32_t)(4 * ns);
    ProfScope _ps(s->stream, KC_PARAM);
    for (int j0 = 0; j0 < ns; j0 += kPTabSlotsPerLaunch) {
        PTabP p;
        std::memset(&p, 0, sizeof(p));
        p.n_slots = std::min(kPTabSlotsPerLaunch, ns - j0);
        for (int j = 0; j < p.n_slots; ++j) {
            p.pidx[j] = (int16_t)pidx[j0 + j];
            p.kind[j] = (int8_t)kind[j0 + j];
        }
        p.slot0 = j0;
        p.stride = 4 * ns;
        p.n_params = n_params;
        p.batch = s->batch;
        p.sign = sign;
        const uint64_t total = (uint64_t)s->batch * p.n_slots;
        param_table_kernel<R><<<grid_for(s, total, 256), 256, 0, s->stream>>>(params, p, (V<R> *)s->ptab);
        QS_CUDA_TRY(cudaGetLastError());
    }
    return QS_OK;
}

qs_status k_param_table(qs_state *s, const std::vector<int> &pidx, const std::vector<int> &kind,
                        const double *params, int n_params, double sign, uint32_t *stride, bool dd_table) {
    if (pidx.size() > 32767) {
        set_error("too many batched-parameter gates");
        return QS_ERR_ARG;
    }
    s->ptab_dd = s->dtype == QS_C128 && dd_table;
    if (s->dtype == QS_C64) return param_table_t<float>(s, pidx, kind, params, n_params, sign, stride);
    return dd_table ? param_table_t<dd>(s, pidx, kind, params, n_params, sign, stride)
                    : param_table_t<double>(s, pidx, kind, params, n_params, sign, stride);
}

qs_status k_apply_param_gate(qs_state *s, const LGate &g, const double *params, int n_params, double sign) {
    return s->dtype == QS_C64 ? apply_param_t<float>(s, g, params, n_params, sign)
                              : apply_param_t<double>(s, g, params, n_params, sign);
}

}  // namespace qsim

// ================================================================== allocation-free expectation
// qs_expectation_noalloc: the Pauli-sum expectation for callers that cannot
// allocate device memory (see qsim.h). Its reduction scratch is a fixed
// file-scope device array instead of the per-handle buffer of qs_expectation.
namespace qsim {

constexpr int kNoAllocMaxPartials = QS_NOALLOC_MAX_PARTIALS;

// Shared by every call on a device, it keeps the last call's partial sums; each
// call overwrites the slots it uses with its first launch before accumulating.
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxPartials];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};  // device address of g_noalloc_partials, per device
}  // namespace

// Device address of the scratch array on the current device, looked up once per
// device (host code may not use the symbol itself as a device pointer).
static qs_status noalloc_scratch(int device, double2 **out) {
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d not supported", device);
        return QS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[device] = p;
    }
    *out = (double2 *)g_noalloc_ptr[device];
    return QS_OK;
}

template <typename R>
static void fill_exp_params(ExpP<R> *p, int n, const qs_pauli_term *terms, size_t count, uint64_t xb,
                            size_t *cursor) {
    p->nt = 0;
    for (; *cursor < count && p->nt < kMaxTermsPerLaunch; ++*cursor) {
        const qs_pauli_term &t = terms[*cursor];
        uint64_t tx = 0, zb = 0;
        for (int q = 0; q < n; ++q) {
            if ((t.x_mask >> q) & 1ull) tx |= qbit(n, q);
            if ((t.z_mask >> q) & 1ull) zb |= qbit(n, q);
        }
        if (tx != xb) continue;
        const int ny = __builtin_popcountll(t.x_mask & t.z_mask) & 3;
        const double c = t.coeff;
        const double re[4] = {c, 0.0, -c, 0.0}, im[4] = {0.0, c, 0.0, -c};
        const int j = p->nt++;
        p->cre[j] = (R)re[ny];
        p->cim[j] = (R)im[ny];
        p->zb[j] = zb;
        const int nz = __builtin_popcountll(zb);
        p->zn[j] = (int8_t)std::min(nz, 3);
        p->za[j] = (int8_t)(nz ? __builtin_ctzll(zb) : -1);
        p->zc[j] = (int8_t)(nz >= 2 ? 63 - __builtin_clzll(zb) : -1);
    }
}

template <typename R>
static qs_status expectation_noalloc_t(const V<R> *psi, int n, int batch, const qs_pauli_term *terms,
                                       size_t count, double *out_dev, cudaStream_t stream, int device) {
    double2 *part = nullptr;
    QS_TRY(noalloc_scratch(device, &part));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint64_t want = std::max<uint64_t>(1, (1ull << n) / (kRedThreads * 16));
    const uint64_t cap = std::max<uint64_t>(1, (uint64_t)sms * 8 / batch);
    const int P = (int)std::min<uint64_t>(std::min<uint64_t>(want, cap),
                                          (uint64_t)(kNoAllocMaxPartials / batch));
    const dim3 grid(P, batch);
    bool first = true;
    ExpP<R> p;  // on the host stack: passed by value as kernel parameters
    for (size_t lead = 0; lead < count; ++lead) {
        // one group per distinct X mask, handled at its first occurrence
        uint64_t xb = 0;
        for (int q = 0; q < n; ++q)
            if ((terms[lead].x_mask >> q) & 1ull) xb |= qbit(n, q);
        bool seen = false;
        for (size_t e = 0; e < lead && !seen; ++e) {
            uint64_t xe = 0;
            for (int q = 0; q < n; ++q)
                if ((terms[e].x_mask >> q) & 1ull) xe |= qbit(n, q);
            seen = (xe == xb);
        }
        if (seen) continue;
        size_t cursor = lead;
        while (true) {
            std::memset(&p, 0, sizeof(p));
            fill_exp_params(&p, n, terms, count, xb, &cursor);
            if (p.nt == 0) break;
            p.xb = xb;
            p.n = n;
            p.ms = n;
            p.hb = xb ? 63 - __builtin_clzll(xb) : 0;
            p.n_free = xb ? n - 1 : n;
            p.accumulate = first ? 0 : 1;
            first = false;
            exp_order_terms(&p);
            expect_partial_kernel<R><<<grid, kRedThreads, 0, stream>>>(psi, p, part);
            QS_CUDA_TRY(cudaGetLastError());
            if (cursor >= count) break;
        }
    }
    if (first) {
        QS_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * batch, stream));
        return QS_OK;
    }
    finalize_kernel<<<batch, kRedThreads, 0, stream>>>(part, P, out_dev, 1);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim

extern "C" qs_status qs_expectation_noalloc(const void *psi_dev, int n, int batch, qs_dtype dtype,
                                            const qs_pauli_term *terms, size_t count, double *out_dev,
                                            void *cuda_stream) {
    using namespace qsim;
    try {
        clear_error();
        if (!psi_dev || !out_dev || (count && !terms)) {
            set_error("null pointer argument");
            return QS_ERR_ARG;
        }
        if (n < 1 || n > QS_MAX_QUBITS || (dtype != QS_C64 && dtype != QS_C128)) {
            set_error("bad n or dtype");
            return QS_ERR_ARG;
        }
        if (batch < 1 || batch > QS_MAX_BATCH) {
            set_error("batch = %d outside [1, %d] (members are a grid dimension of at most %d)", batch,
                      QS_MAX_BATCH, QS_MAX_BATCH);
            return QS_ERR_ARG;
        }
        if ((uint64_t)batch > (1ull << (46 - n))) {
            set_error("batch * 2^n too large");
            return QS_ERR_ARG;
        }
        for (size_t i = 0; i < count; ++i)
            if ((n < 64 && ((terms[i].x_mask | terms[i].z_mask) >> n) != 0) || !std::isfinite(terms[i].coeff)) {
                set_error("term %zu names a qubit >= n or has a non-finite coefficient", i);
                return QS_ERR_ARG;
            }
        int device = 0;
        QS_CUDA_TRY(cudaGetDevice(&device));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (dtype == QS_C64)
            return expectation_noalloc_t<float>((const float2 *)psi_dev, n, batch, terms, count, out_dev, st,
                                                device);
        return expectation_noalloc_t<double>((const double2 *)psi_dev, n, batch, terms, count, out_dev, st,
                                             device);
    } catch (...) {
        set_error("internal error");
        return QS_ERR_CUDA;
    }
}
