// Measurements (Sec. 2.4, "Measurements": sampling the final state and the
// outcome probabilities of a group of qubits traced over the others; Sec. 3.3
// times the sampling):
//   * marginal_partial_kernel / marginal_finalize_kernel: per-block histograms
//     of |psi|^2 over the group's outcome in shared memory (each thread adds
//     the sum of a run of amplitudes with one outcome), then a fixed-order sum
//     of the blocks' histograms (FP64);
//   * block_sums_kernel, scan kernels, sample_kernel: |psi|^2 summed over
//     blocks of kSampleBlock amplitudes, their exclusive prefix sums in FP64
//     (a two-level scan), and one warp per shot: a binary search over the block
//     prefixes, then a warp scan through the block up to the first amplitude
//     whose cumulative probability exceeds the shot's target.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace qsim {

static int sms_of(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
    return v;
}

// ------------------------------------------------------------------ marginals
struct MargP {
    int pos[kMarginalMaxQubits];  // index bit of the group's qubit j (outcome bit m-1-j)
    int m;
    int ms;        // member shift
    uint64_t per;  // amplitudes per member
};

// Each block takes a contiguous range of the member's amplitudes (a multiple
// of 256 long); thread tid reads x = start + tid + 256 i (coalesced), so its
// index bits 0..7 are fixed and its outcome y changes only where x crosses a
// multiple of 2^pmin, pmin the lowest group bit above bit 7. The thread walks
// those runs: y is formed once per run, the run's |psi|^2 is summed (runs of
// 64 in the state's precision, then FP64; 8 loads in flight) and added to the
// block's shared histogram.
template <typename R>
__global__ void __launch_bounds__(256) marginal_partial_kernel(const V<R> *__restrict__ psi, const MargP p,
                                                               double *__restrict__ part) {
    __shared__ double h[1 << kMarginalMaxQubits];
    const int bins = 1 << p.m;
    for (int i = threadIdx.x; i < bins; i += blockDim.x) h[i] = 0.0;
    __syncthreads();
    const V<R> *q = psi + ((uint64_t)blockIdx.y << p.ms);
    const uint64_t span = ((p.per + gridDim.x - 1) / gridDim.x + 255) & ~255ull;
    const uint64_t start = (uint64_t)blockIdx.x * span;
    const uint64_t end = start + span < p.per ? start + span : p.per;
    int pmin = 63;
    for (int j = 0; j < p.m; ++j)
        if (p.pos[j] >= 8 && p.pos[j] < pmin) pmin = p.pos[j];
    constexpr int U = 8;  // loads in flight per thread
    for (uint64_t x0 = start + threadIdx.x; x0 < end;) {
        uint32_t y = 0;
        for (int j = 0; j < p.m; ++j) y |= (uint32_t)((x0 >> p.pos[j]) & 1ull) << (p.m - 1 - j);
        // the run ends at the next multiple of 2^pmin (or the range's end)
        const uint64_t bound = ((x0 >> pmin) + 1) << pmin;
        const uint64_t rend = bound < end ? bound : end;
        double accd = 0.0;
        R accf = 0;
        int run = 0;
        uint64_t x = x0;
        for (; x < rend; x += (uint64_t)U * blockDim.x) {
            R pr[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const uint64_t xk = x + (uint64_t)k * blockDim.x;
                pr[k] = 0;
                if (xk < rend) {
                    const V<R> a = q[xk];
                    pr[k] = a.x * a.x + a.y * a.y;
                }
            }
#pragma unroll
            for (int k = 0; k < U; ++k) accf += pr[k];
            run += U;
            if (run >= 64) {
                accd += (double)accf;
                accf = 0;
                run = 0;
            }
        }
        atomicAdd(&h[y], accd + (double)accf);
        x0 = rend + threadIdx.x;  // rend is a multiple of 256 unless it is the range's end
    }
    __syncthreads();
    double *out = part + ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * bins;
    for (int i = threadIdx.x; i < bins; i += blockDim.x) out[i] = h[i];
}

__global__ void __launch_bounds__(256) marginal_finalize_kernel(const double *__restrict__ part, int parts,
                                                                int bins, double *__restrict__ out) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= bins) return;
    const double *pp = part + (uint64_t)blockIdx.y * parts * bins + y;
    double acc = 0.0;
    for (int b = 0; b < parts; ++b) acc += pp[(uint64_t)b * bins];
    out[(uint64_t)blockIdx.y * bins + y] = acc;
}

qs_status k_marginal(qs_state *s, const int *bitpos, int m, double *out_dev) {
    MargP p;
    std::memset(&p, 0, sizeof(p));
    for (int j = 0; j < m; ++j) p.pos[j] = bitpos[j];
    p.m = m;
    p.ms = s->ms;
    p.per = 1ull << s->n;
    const int bins = 1 << m;
    const uint64_t want = std::max<uint64_t>(1, p.per / (256 * 32));
    const int parts = (int)std::min<uint64_t>(want, (uint64_t)std::max(1, 4 * sms_of(s->device) / s->batch));
    // one part per member (large batches): the partial histograms are the
    // result, written straight into out_dev with no scratch; otherwise the
    // scratch holds batch * parts <= 4 x SMs histograms
    double *part = out_dev;
    if (parts > 1) {
        QS_TRY(ensure_scratch(s, (size_t)s->batch * parts * bins));
        part = s->scratch;
    }
    ProfScope _ps(s->stream, KC_REDUCE, (double)(s->batch * p.per) * (s->dtype == QS_C64 ? 8 : 16),
                  3.0 * s->batch * p.per);
    const dim3 grid((unsigned)parts, (unsigned)s->batch);
    if (s->dtype == QS_C64)
        marginal_partial_kernel<float><<<grid, 256, 0, s->stream>>>((const float2 *)s->data, p, part);
    else
        marginal_partial_kernel<double><<<grid, 256, 0, s->stream>>>((const double2 *)s->data, p, part);
    QS_CUDA_TRY(cudaGetLastError());
    if (parts == 1) return QS_OK;
    const dim3 g2((unsigned)((bins + 255) / 256), (unsigned)s->batch);
    marginal_finalize_kernel<<<g2, 256, 0, s->stream>>>(s->scratch, parts, bins, out_dev);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

// ------------------------------------------------------------------ sampling
constexpr int kSampleBlock = 4096;  // amplitudes per block of the prefix sums
constexpr int kScanChunk = 1024;    // block sums per CTA of the first scan level

// sum of |psi|^2 over each block of L amplitudes (one CTA of 256 threads per
// block): per-thread sums in the state's precision, the block total in FP64
template <typename R>
__global__ void __launch_bounds__(256) block_sums_kernel(const V<R> *__restrict__ q, uint64_t L,
                                                         double *__restrict__ bsum) {
    __shared__ double sh[8];
    const V<R> *b = q + (uint64_t)blockIdx.x * L;
    R acc = 0;
    for (uint64_t i = threadIdx.x; i < L; i += blockDim.x) {
        const V<R> a = b[i];
        acc += a.x * a.x + a.y * a.y;
    }
    double d = (double)acc;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        bsum[blockIdx.x] = t;
    }
}

// exclusive prefix of v[0..count) within chunks of kScanChunk (one CTA each);
// the chunk's total goes to tot[chunk]
__global__ void __launch_bounds__(kScanChunk) scan_chunks_kernel(const double *__restrict__ v, uint64_t count,
                                                                 double *__restrict__ pre,
                                                                 double *__restrict__ tot) {
    __shared__ double sh[kScanChunk];
    const uint64_t i = (uint64_t)blockIdx.x * kScanChunk + threadIdx.x;
    const double x = i < count ? v[i] : 0.0;
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < kScanChunk; o <<= 1) {  // inclusive Hillis-Steele scan
        const double t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < count) pre[i] = sh[threadIdx.x] - x;
    if (threadIdx.x == kScanChunk - 1) tot[blockIdx.x] = sh[threadIdx.x];
}

// exclusive prefix of the chunk totals in place (one CTA; each thread a run)
__global__ void __launch_bounds__(kScanChunk) scan_totals_kernel(double *__restrict__ tot, uint64_t chunks) {
    __shared__ double sh[kScanChunk];
    const uint64_t per = (chunks + kScanChunk - 1) / kScanChunk;
    const uint64_t b = threadIdx.x * per, e = std::min<uint64_t>(b + per, chunks);
    double run = 0.0;
    for (uint64_t i = b; i < e; ++i) run += tot[i];
    sh[threadIdx.x] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < kScanChunk; ++t) {
            const double r = sh[t];
            sh[t] = acc;
            acc += r;
        }
    }
    __syncthreads();
    double acc = sh[threadIdx.x];
    for (uint64_t i = b; i < e; ++i) {
        const double r = tot[i];
        tot[i] = acc;
        acc += r;
    }
}

__global__ void __launch_bounds__(kScanChunk) add_offsets_kernel(double *__restrict__ pre, uint64_t count,
                                                                 const double *__restrict__ tot) {
    const uint64_t i = (uint64_t)blockIdx.x * kScanChunk + threadIdx.x;
    if (i < count) pre[i] += tot[blockIdx.x];
}

// one warp per shot: the smallest x with cdf(x) > u * total
template <typename R>
__global__ void __launch_bounds__(256) sample_kernel(const V<R> *__restrict__ q, const double *__restrict__ pre,
                                                     const double *__restrict__ bsum, uint64_t nb, uint64_t L,
                                                     const double *__restrict__ u, uint64_t shots,
                                                     unsigned long long *__restrict__ out) {
    const uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= shots) return;
    const int lane = threadIdx.x & 31;
    const double total = pre[nb - 1] + bsum[nb - 1];
    // a uniform outside [0, 1) is clamped: below 0 to 0, 1 or above (or NaN) to 1
    double uu = u[w];
    if (!(uu < 1.0)) uu = 1.0;
    if (uu < 0.0) uu = 0.0;
    const double target = uu * total;
    uint64_t lo = 0, hi = nb - 1;  // the last block whose exclusive prefix is <= target
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= target) lo = mid;
        else hi = mid - 1;
    }
    // the prefix sums are monotone only up to rounding, so the search can end
    // in a block of zero probability: step back to the last block before it
    // that has some (its last nonzero outcome is then the sample)
    while (lo > 0 && !(bsum[lo] > 0.0)) --lo;
    const V<R> *b = q + lo * L;
    double running = pre[lo];
    uint64_t found = ~0ull, last_nz = lo * L;
    for (uint64_t c = 0; c < L; c += 32) {
        R pr = 0;
        if (c + lane < L) {
            const V<R> a = b[c + lane];
            pr = a.x * a.x + a.y * a.y;
        }
        R sc = pr;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const R t = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += t;
        }
        // only a lane of nonzero probability can be the sample: the scan's
        // rounding differs between lanes, so a zero lane after the target's
        // position can compare above it while the nonzero lane before did not
        const unsigned hit = __ballot_sync(0xffffffffu, pr > (R)0 && running + (double)sc > target);
        const unsigned nz = __ballot_sync(0xffffffffu, pr > (R)0);
        if (nz) last_nz = lo * L + c + (31 - __clz(nz));
        if (hit) {
            found = lo * L + c + (__ffs(hit) - 1);
            break;
        }
        running += (double)__shfl_sync(0xffffffffu, sc, 31);
    }
    // the target lies at the block's end only through rounding: its last
    // outcome with nonzero probability
    if (lane == 0) out[w] = found != ~0ull ? found : last_nz;
}

qs_status k_sample(qs_state *s, int member, const double *u_dev, uint64_t shots, uint64_t *out_dev) {
    const uint64_t per = 1ull << s->n;
    const uint64_t L = std::min<uint64_t>(per, kSampleBlock);
    const uint64_t nb = per / L;
    const uint64_t chunks = (nb + kScanChunk - 1) / kScanChunk;
    QS_TRY(ensure_scratch(s, (size_t)(2 * nb + chunks)));
    double *bsum = s->scratch, *pre = s->scratch + nb, *tot = s->scratch + 2 * nb;
    ProfScope _ps(s->stream, KC_REDUCE, (double)per * (s->dtype == QS_C64 ? 8 : 16), 3.0 * per);
    const uint64_t moff = (uint64_t)member << s->ms;
    if (s->dtype == QS_C64)
        block_sums_kernel<float><<<(unsigned)nb, 256, 0, s->stream>>>((const float2 *)s->data + moff, L, bsum);
    else
        block_sums_kernel<double><<<(unsigned)nb, 256, 0, s->stream>>>((const double2 *)s->data + moff, L, bsum);
    QS_CUDA_TRY(cudaGetLastError());
    scan_chunks_kernel<<<(unsigned)chunks, kScanChunk, 0, s->stream>>>(bsum, nb, pre, tot);
    QS_CUDA_TRY(cudaGetLastError());
    scan_totals_kernel<<<1, kScanChunk, 0, s->stream>>>(tot, chunks);
    QS_CUDA_TRY(cudaGetLastError());
    add_offsets_kernel<<<(unsigned)chunks, kScanChunk, 0, s->stream>>>(pre, nb, tot);
    QS_CUDA_TRY(cudaGetLastError());
    if (shots == 0) return QS_OK;
    const uint64_t blocks = (shots + 7) / 8;
    for (uint64_t b0 = 0; b0 < blocks; b0 += 1u << 30) {  // grid.x limit, in whole blocks
        const uint64_t nbk = std::min<uint64_t>(blocks - b0, 1u << 30);
        const uint64_t s0 = b0 * 8, ns = std::min<uint64_t>(shots - s0, nbk * 8);
        if (s->dtype == QS_C64)
            sample_kernel<float><<<(unsigned)nbk, 256, 0, s->stream>>>(
                (const float2 *)s->data + moff, pre, bsum, nb, L, u_dev + s0, ns,
                (unsigned long long *)out_dev + s0);
        else
            sample_kernel<double><<<(unsigned)nbk, 256, 0, s->stream>>>(
                (const double2 *)s->data + moff, pre, bsum, nb, L, u_dev + s0, ns,
                (unsigned long long *)out_dev + s0);
        QS_CUDA_TRY(cudaGetLastError());
    }
    return QS_OK;
}

}  // namespace qsim
