// Fused 5-qubit blocks on tensor cores (Sec. 2.4, "Gate fusion", taken to
// 5-qubit 32x32 blocks; the GEMM form is the paper's matmuleinsum reshape,
// Sec. 2.3).
//
// For a block on index bits (q_0 .. q_4) the state is a 32 x 2^(n-5) complex
// matrix X (row = local index sum_j bit(q_j) 2^(4-j), column = the other bits)
// and the block applies Y = U X. As one real GEMM:
//     [Yr; Yi] = [[Ur, -Ui], [Ui, Ur]] [Xr; Xi]     (M = K = 64, N = columns)
// run on the tensor cores in TF32 with the 3xTF32 split a = a_hi + a_lo,
// b = b_hi + b_lo, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32:
// about FP32 accuracy for complex64 states.
//
// A CTA (8 warps) loops over chunks of 64 columns: the chunk's 2048 amplitudes
// are loaded with consecutive threads on consecutive addresses, split into hi
// and lo TF32 planes in shared memory (column-major, padded against bank
// conflicts), multiplied by warp-level m16n8k8 TF32 MMAs (warp w owns rows
// 16 (w & 3) .. + 15 and columns 32 (w >> 2) .. + 31), and written back.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "fused.h"
#include "internal.h"
#include "prof.h"

namespace qsim {

constexpr int kFCols = 64;           // columns per chunk
constexpr int kFLd = 68;             // padded column stride (floats) in shared memory
constexpr int kFThreads = 256;

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// scatter the low bits of v over the positions of mask (ascending)
__device__ __forceinline__ uint64_t deposit(uint64_t v, uint64_t mask) {
    uint64_t out = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (v & 1ull) out |= low;
        v >>= 1;
        mask &= mask - 1;
    }
    return out;
}

__global__ void __launch_bounds__(kFThreads, 2)
    fused5_tc_kernel(float2 *__restrict__ psi, const __grid_constant__ FusedP p) {
    __shared__ float sb_hi[kFCols * kFLd];
    __shared__ float sb_lo[kFCols * kFLd];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int mt = warp & 3;          // rows 16 mt .. 16 mt + 15
    const int nb = (warp >> 2) * 32;  // columns nb .. nb + 31

    // A fragments of this warp's 16 rows for all 8 k-steps, hi and lo, from the
    // real 64 x 64 form of U (row m, col k):
    //   m < 32, k < 32: Re U[m][k];  m < 32, k >= 32: -Im U[m][k-32]
    //   m >= 32, k < 32: Im U[m-32][k];  m >= 32, k >= 32: Re U[m-32][k-32]
    auto a_elem = [&](int m, int k) -> float {
        const float2 u = p.u[(m & 31) * 32 + (k & 31)];
        if (m < 32) return k < 32 ? u.x : -u.y;
        return k < 32 ? u.y : u.x;
    };
    uint32_t ahi[8][4], alo[8][4];
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
        const int r0 = 16 * mt + gid, c0 = 8 * ks + tig;
        const float v[4] = {a_elem(r0, c0), a_elem(r0 + 8, c0), a_elem(r0, c0 + 4), a_elem(r0 + 8, c0 + 4)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ahi[ks][e] = to_tf32(v[e]);
            alo[ks][e] = to_tf32(v[e] - __uint_as_float(ahi[ks][e]));
        }
    }

    for (uint64_t chunk = blockIdx.x; chunk < p.total_chunks; chunk += gridDim.x) {
        const uint64_t member = chunk >> p.chunk_shift;
        const uint64_t cbase = (member << p.ms) | deposit(chunk & ((1ull << p.chunk_shift) - 1), p.hi_mask);
        // ---- load: thread index bits follow the chunk's 11 address bits in
        // ascending order (consecutive threads -> consecutive addresses)
#pragma unroll
        for (int it = 0; it < (kFCols * 32) / kFThreads; ++it) {
            const uint32_t i = threadIdx.x + it * kFThreads;
            const uint64_t addr = cbase | deposit(i, p.chunk_mask);
            const int row = p.lmap[i];  // local row index
            const int c = p.cmap[i];    // column in the chunk
            const float2 x = psi[addr];
            float hr = __uint_as_float(to_tf32(x.x)), hi = __uint_as_float(to_tf32(x.y));
            sb_hi[c * kFLd + row] = hr;
            sb_hi[c * kFLd + 32 + row] = hi;
            sb_lo[c * kFLd + row] = __uint_as_float(to_tf32(x.x - hr));
            sb_lo[c * kFLd + 32 + row] = __uint_as_float(to_tf32(x.y - hi));
        }
        __syncthreads();
        // ---- 3xTF32 MMAs: D[16 x 32] per warp
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int col = nb + 8 * nt + gid;
                const int k0 = 8 * ks + tig;
                const uint32_t bh0 = __float_as_uint(sb_hi[col * kFLd + k0]);
                const uint32_t bh1 = __float_as_uint(sb_hi[col * kFLd + k0 + 4]);
                const uint32_t bl0 = __float_as_uint(sb_lo[col * kFLd + k0]);
                const uint32_t bl1 = __float_as_uint(sb_lo[col * kFLd + k0 + 4]);
                mma_tf32(acc[nt], alo[ks], bh0, bh1);
                mma_tf32(acc[nt], ahi[ks], bl0, bl1);
                mma_tf32(acc[nt], ahi[ks], bh0, bh1);
            }
        }
        __syncthreads();
        // ---- stage D in the hi plane (row-major by column), then store
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = nb + 8 * nt + 2 * tig;
            const int row = 16 * mt + gid;
            sb_hi[col * kFLd + row] = acc[nt][0];
            sb_hi[(col + 1) * kFLd + row] = acc[nt][1];
            sb_hi[col * kFLd + row + 8] = acc[nt][2];
            sb_hi[(col + 1) * kFLd + row + 8] = acc[nt][3];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < (kFCols * 32) / kFThreads; ++it) {
            const uint32_t i = threadIdx.x + it * kFThreads;
            const uint64_t addr = cbase | deposit(i, p.chunk_mask);
            const int row = p.lmap[i];
            const int c = p.cmap[i];
            psi[addr] = make_float2(sb_hi[c * kFLd + row], sb_hi[c * kFLd + 32 + row]);
        }
        __syncthreads();
    }
}

qs_status k_fused5(qs_state *s, const std::vector<cd> &U, const int *bits) {
    if (s->dtype != QS_C64) {
        set_error("tensor-core blocks take complex64 states");
        return QS_ERR_UNSUPPORTED;
    }
    const int n = s->n;
    if (n < 11) {
        set_error("tensor-core blocks need n >= 11");
        return QS_ERR_UNSUPPORTED;
    }
    FusedP p;
    std::memset(&p, 0, sizeof(p));
    for (int i = 0; i < 1024; ++i) p.u[i] = make_float2((float)U[i].real(), (float)U[i].imag());
    uint64_t qmask = 0;
    for (int j = 0; j < 5; ++j) qmask |= 1ull << bits[j];
    // the chunk's column bits: the 6 lowest index bits outside the block
    uint64_t colmask = 0;
    int got = 0;
    for (int b = 0; b < n && got < 6; ++b)
        if (!((qmask >> b) & 1ull)) {
            colmask |= 1ull << b;
            ++got;
        }
    p.chunk_mask = qmask | colmask;
    uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    p.hi_mask = all & ~p.chunk_mask;
    p.chunk_shift = n - 11;
    p.ms = s->ms;
    p.total_chunks = (uint64_t)s->batch << p.chunk_shift;
    // thread index i (11 bits, over the chunk bits in ascending order) -> (row, column)
    int cb[11], nc = 0;
    for (int b = 0; b < 64 && nc < 11; ++b)
        if ((p.chunk_mask >> b) & 1ull) cb[nc++] = b;
    for (int i = 0; i < 2048; ++i) {
        int row = 0, col = 0, ci = 0;
        for (int t = 0; t < 11; ++t) {
            const int bit = (i >> t) & 1;
            const int g = cb[t];
            int jq = -1;
            for (int j = 0; j < 5; ++j)
                if (bits[j] == g) jq = j;
            if (jq >= 0)
                row |= bit << (4 - jq);
            else
                col |= bit << ci++;
        }
        p.lmap[i] = (uint8_t)row;
        p.cmap[i] = (uint8_t)col;
    }
    int dev = s->device, sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t grid = std::min<uint64_t>(p.total_chunks, (uint64_t)sms * 4);
    const double amps = (double)((uint64_t)s->batch << n);
    ProfScope _ps(s->stream, KC_FUSED_TC, 2.0 * amps * 8.0, amps * 256.0 * 3.0);
    fused5_tc_kernel<<<(unsigned)grid, kFThreads, 0, s->stream>>>((float2 *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
