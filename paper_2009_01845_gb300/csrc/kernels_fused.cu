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
// A CTA (8 warps) loops over chunks of 64 columns (2048 amplitudes). The next
// chunk is fetched with cp.async into a raw staging buffer (consecutive
// threads on consecutive addresses) while the current one is multiplied; each
// chunk is split from the raw buffer into hi and lo TF32 planes (column-major,
// padded, rows XOR-swizzled by column group so that both the staging stores
// and the MMA operand loads hit distinct banks), multiplied by warp-level
// m16n8k8 TF32 MMAs (warp w owns rows 16 (w & 3) .. + 15 and columns
// 32 (w >> 2) .. + 31), staged back and written out.
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
constexpr int kFElems = 2048;        // amplitudes per chunk
constexpr size_t kFSmem = kFElems * sizeof(float2) + 2 * kFCols * kFLd * sizeof(float);

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

// 8-byte asynchronous copy global -> shared, and its group fences
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// row swizzle of a column group (8 columns): XOR into the row's low 2 bits
__device__ __forceinline__ int fswz(int col) { return (col >> 3) & 3; }

__global__ void __launch_bounds__(kFThreads, 2)
    fused5_tc_kernel(float2 *__restrict__ psi, const __grid_constant__ FusedP p) {
    extern __shared__ __align__(16) unsigned char fsm[];
    float2 *raw = reinterpret_cast<float2 *>(fsm);
    float *sb_hi = reinterpret_cast<float *>(fsm + kFElems * sizeof(float2));
    float *sb_lo = sb_hi + kFCols * kFLd;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
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
    // this thread's part of every element's address (the chunk's lowest 8 bits)
    uint64_t dt = 0;
    {
        uint64_t m = p.chunk_mask;
        for (int b = 0; b < 8; ++b) {
            const uint64_t low = m & (~m + 1);
            if ((tid >> b) & 1) dt |= low;
            m &= m - 1;
        }
    }
    const int rt = p.lmap[tid], ct = p.cmap[tid];
    const uint64_t cmask = (1ull << p.chunk_shift) - 1ull;
    auto chunk_base = [&](uint64_t chunk) {
        return ((chunk >> p.chunk_shift) << p.ms) | expand_bits(chunk & cmask, p.cins);
    };
    auto fetch = [&](uint64_t chunk) {
        const uint64_t cb = chunk_base(chunk) | dt;
#pragma unroll
        for (int h = 0; h < 8; ++h) cp_async8(&raw[tid + kFThreads * h], &psi[cb | p.dhi[h]]);
    };

    uint64_t chunk = blockIdx.x;
    if (chunk < p.total_chunks) fetch(chunk);
    cp_async_commit();
    for (; chunk < p.total_chunks; chunk += gridDim.x) {
        const uint64_t cb = chunk_base(chunk) | dt;
        cp_async_wait_all();
        __syncthreads();
        // ---- split the raw chunk into TF32 hi and lo planes
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const float2 x = raw[tid + kFThreads * h];
            const int row = rt | p.rhi[h], c = ct | p.chi[h];
            const int o = c * kFLd + (row ^ fswz(c));
            const float hr = __uint_as_float(to_tf32(x.x)), hi = __uint_as_float(to_tf32(x.y));
            sb_hi[o] = hr;
            sb_hi[o + 32] = hi;
            sb_lo[o] = __uint_as_float(to_tf32(x.x - hr));
            sb_lo[o + 32] = __uint_as_float(to_tf32(x.y - hi));
        }
        __syncthreads();
        // ---- the next chunk streams in while this one is multiplied
        if (chunk + gridDim.x < p.total_chunks) fetch(chunk + gridDim.x);
        cp_async_commit();
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
                const int sw = fswz(col);
                const int k0 = 8 * ks + tig;
                const uint32_t bh0 = __float_as_uint(sb_hi[col * kFLd + (k0 ^ sw)]);
                const uint32_t bh1 = __float_as_uint(sb_hi[col * kFLd + ((k0 + 4) ^ sw)]);
                const uint32_t bl0 = __float_as_uint(sb_lo[col * kFLd + (k0 ^ sw)]);
                const uint32_t bl1 = __float_as_uint(sb_lo[col * kFLd + ((k0 + 4) ^ sw)]);
                mma_tf32(acc[nt], alo[ks], bh0, bh1);
                mma_tf32(acc[nt], ahi[ks], bl0, bl1);
                mma_tf32(acc[nt], ahi[ks], bh0, bh1);
            }
        }
        __syncthreads();
        // ---- stage D in the hi plane (same swizzle), then store
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = nb + 8 * nt + 2 * tig;
            const int row = 16 * mt + gid;
            const int sw = fswz(col);
            sb_hi[col * kFLd + (row ^ sw)] = acc[nt][0];
            sb_hi[(col + 1) * kFLd + (row ^ sw)] = acc[nt][1];
            sb_hi[col * kFLd + ((row + 8) ^ sw)] = acc[nt][2];
            sb_hi[(col + 1) * kFLd + ((row + 8) ^ sw)] = acc[nt][3];
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int row = rt | p.rhi[h], c = ct | p.chi[h];
            const int o = c * kFLd + (row ^ fswz(c));
            psi[cb | p.dhi[h]] = make_float2(sb_hi[o], sb_hi[o + 32]);
        }
    }
    cp_async_wait_all();
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
    p.chunk_shift = n - 11;
    p.ms = s->ms;
    p.total_chunks = (uint64_t)s->batch << p.chunk_shift;
    // chunk bits in ascending order; element index i (11 bits) -> address
    // offset, row and column
    int cb[11], nc = 0;
    for (int b = 0; b < 64 && nc < 11; ++b)
        if ((p.chunk_mask >> b) & 1ull) cb[nc++] = b;
    p.cins.count = 11;
    for (int t = 0; t < 11; ++t) p.cins.pos[t] = (int8_t)cb[t];
    auto row_col = [&](int i, int *row, int *col) {
        *row = 0;
        *col = 0;
        int ci = 0;
        for (int t = 0; t < 11; ++t) {
            const int bit = (i >> t) & 1;
            int jq = -1;
            for (int j = 0; j < 5; ++j)
                if (bits[j] == cb[t]) jq = j;
            if (jq >= 0)
                *row |= bit << (4 - jq);
            else
                *col |= bit << ci++;
        }
    };
    for (int t = 0; t < 256; ++t) {
        int r, c;
        row_col(t, &r, &c);
        p.lmap[t] = (uint8_t)r;
        p.cmap[t] = (uint8_t)c;
    }
    for (int h = 0; h < 8; ++h) {
        int r, c;
        row_col(h << 8, &r, &c);
        p.rhi[h] = (uint8_t)r;
        p.chi[h] = (uint8_t)c;
        uint64_t d = 0;
        for (int t = 8; t < 11; ++t)
            if (((h << 8) >> t) & 1) d |= 1ull << cb[t];
        p.dhi[h] = d;
    }
    static int configured[64] = {0};
    static int blocks_per_sm[64] = {0};
    const int dev = (s->device >= 0 && s->device < 64) ? s->device : 0;
    if (!configured[dev]) {
        QS_CUDA_TRY(cudaFuncSetAttribute(fused5_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem));
        int bps = 0, sms = 0;
        QS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fused5_tc_kernel, kFThreads, kFSmem));
        QS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        blocks_per_sm[dev] = std::max(1, bps) * sms;
        configured[dev] = 1;
    }
    const uint64_t grid = std::min<uint64_t>(p.total_chunks, (uint64_t)blocks_per_sm[dev]);
    const double amps = (double)((uint64_t)s->batch << n);
    ProfScope _ps(s->stream, KC_FUSED_TC, 2.0 * amps * 8.0, amps * 256.0 * 3.0);
    fused5_tc_kernel<<<(unsigned)grid, kFThreads, kFSmem, s->stream>>>((float2 *)s->data, p);
    QS_CUDA_TRY(cudaGetLastError());
    return QS_OK;
}

}  // namespace qsim
