// Tiled multi-gate pass: the pass description shared by the planner and the
// kernel.
//
// A pass loads tiles of 2^k amplitudes whose indices vary over k chosen index
// bits (the "tile bits": always the 5 lowest bits, for coalescing, plus k-5
// others) with every other bit fixed per tile, applies a run of gates to the
// tile while it is on chip, and writes it back once: one HBM round trip for
// many gates (the grouping of local gates of Sec. 2.5, done per tile).
//
// Inside a CTA of 2^WB warps each thread holds 2^RB amplitudes in registers
// (see TileCfg). The tile's k = RB + 5 + WB local bits are split, per stage, into
//   L: 5 local bits     -> lane index (local bits 0..4 in the first and last
//                          stage, so global loads and stores are coalesced),
//   R: RB local bits    -> register index,
//   W: WB local bits    -> warp index.
// Gates whose dense targets lie in R are applied in registers, targets in L
// through warp shuffles; a new stage re-splits the bits through a shared-memory
// transpose. Each transpose has its own XOR swizzle, chosen by the planner so
// that both of its accesses (the write under the previous stage's lanes, the
// read under the new stage's) are free of bank conflicts: the shared-memory
// position of tile-local index j is j with the images fcol[] of its high bits
// XORed into its low h bits (h = 4 for complex64, 3 for complex128, the lanes
// of one 128-byte wavefront), linear over XOR, so register and thread offsets
// combine by XOR. Diagonal gates may act on any bits, inside or outside the tile.
#pragma once

#include <cstdint>

#include "device.cuh"

namespace qsim {

constexpr int kTileLaneBits = 5;
constexpr int kTileMaxWarpBits = 3;
constexpr int kTileMaxStages = 24;  // also sizes the per-CTA offset tables
constexpr int kTileMaxOps = 288;
constexpr int kTileMaxMat = 640;   // complex entries in the matrix pool
constexpr int kTileMaxGrad = 48;   // gradient ops per pass (adjoint sweep)
constexpr int kTileMaxDFac = 96;   // diagonal-block factors per pass

// Per precision: RB register bits per thread, WB warp bits (2^WB warps per
// CTA), kMinBlocks resident CTAs per SM the register budget is sized for.
// complex64: 32 amplitudes per thread, 8 warps, 2 CTAs per SM (k = 13);
// complex128: 16 amplitudes per thread, 8 warps, 1 CTA per SM (k = 12).
// (64 amplitudes per thread with 4 warps and 3 CTAs per SM measured slower:
// fewer transposes, but register spills and fewer warps to hide latency.)
template <typename R> struct TileCfg;
template <> struct TileCfg<float> { static constexpr int RB = 5, WB = 3, kMinBlocks = 2; };
template <> struct TileCfg<double> { static constexpr int RB = 4, WB = 3, kMinBlocks = 1; };
// complex128 computed in double-float: the same tile (16 bytes per amplitude),
// registers capped for 2 CTAs per SM (a few spilled words; 16 warps per SM
// hide the long double-float dependency chains and instruction fetches:
// 1.5x faster than 1 CTA per SM, measured at n = 28)
template <> struct TileCfg<dd> { static constexpr int RB = 4, WB = 3, kMinBlocks = 2; };
inline int tile_reg_bits(qs_dtype dt) { return dt == QS_C64 ? 5 : 4; }
inline int tile_warp_bits(qs_dtype dt) { return 3; }
inline int tile_threads(qs_dtype dt) { return 32 << tile_warp_bits(dt); }
inline int tile_bits(qs_dtype dt) { return tile_reg_bits(dt) + kTileLaneBits + tile_warp_bits(dt); }

enum TileOpType : uint8_t {
    TOP_PHASE = 0,   // multiply by mat[m] where all required bits are 1
    TOP_DIAG1,       // multiply by mat[m + bit] (bit = the target's value), if required bits are 1
    TOP_DENSE1_R,    // 2x2 on register bit a
    TOP_DENSE1_L,    // 2x2 on lane bit a (warp shuffles)
    TOP_DENSE2_RR,   // 4x4 on register bits (a = local MSB, b), a < b
    TOP_SWAP_RR,     // swap register bits a < b
    TOP_GRAD,        // adjoint sweep: accumulate Im<lambda|P|phi> for a generator P
    TOP_ISING,       // psi_x *= exp(-i tau E(x)), E an Ising energy (<= 2-body Z terms)
    TOP_ROTS_R,      // real rotations on register bits as in-place shears: for each bit j of a,
                     // x += s1 y, then y += s2 x, with (s1, s2) = mat[m + j] and (x, y) the
                     // register pairs that differ in bit j (x: bit j is 0)
    TOP_ROTS_L,      // scaled real rotations on the 5 lane bits (warp shuffles):
                     // mat[m + j] = (coef, form + 1) or (0, 0)
    TOP_DBLOCK,      // product of diagonal factors (see diag_block)
    TOP_FLIP,        // negate the registers whose bit a is 1 - (tkind & 1), bit b is
                     // 1 - (tkind >> 1 & 1), and whose bits of mr, XORed with fx, are 1
    TOP_PROT,        // per-member RY (b = 0) or RX (b = 1) on register bit a: (cos, sin) from the member's table
};

// Scaled real rotations on lane bits: form 0: (a, b) <- (a - t b, b + t a)
// with |t| <= 1; form 1: (a, b) <- (b - u a, a + u b) with |u| <= 1. The
// planner moves the scalar and sign that make these equal to the rotation
// into diagonal factors.
enum TileRotForm : uint8_t { ROT_TAN = 0, ROT_COT = 1 };

// Register frame. A rotation closer to a swap than to the identity is applied
// as the shears of the remaining small rotation, and the swap of the two
// register halves is not carried out: from there to the end of the stage
// register r holds the amplitude of register index r ^ rflip (rflip = the
// register bits swapped so far). The planner writes every later op of the
// stage in those terms; the transpose that ends the stage writes register r
// where r ^ rflip belongs (an XOR of the stage's write offsets), and so does
// the last stage's store, so the next stage starts with no frame.

// One factor of a diagonal block, located in the block's stage:
//   DF_BIT: diag(v0, v1) on one thread bit (kind TB_THREAD, local mask tmask)
//           or one outside bit (TB_OUTSIDE, global mask tmask);
//   DF_PHASE: v0 where all required bits (mr register, mt thread, mo outside)
//           are 1; for two or more register bits tmask holds the registers
//           covered;
//   DF_SIGN: where the required bits mt, mo are 1, negate the block's ratio
//           of register bit j (a = 1 << j) or its base (a = 0x80).
// Factors on register bits alone are folded by the planner into the block's
// constants (a base value and one ratio per register bit); sign flips on two
// or more register bits are TOP_FLIP ops.
enum TileDFacType : uint8_t { DF_BIT = 0, DF_PHASE = 1, DF_SIGN = 2 };

// Generators of TOP_GRAD (b field): Pauli X, Y, Z on one target, or the
// projector on the all-ones block of the required bits (U1/CU1).
enum TileGen : uint8_t { GEN_X = 0, GEN_Y = 1, GEN_Z = 2, GEN_PROJ = 3 };

// Where a DIAG1 target bit lives in the current stage.
enum TileBitKind : uint8_t { TB_REG = 0, TB_THREAD = 1, TB_OUTSIDE = 2 };

// Every op may carry required bits (controls, or the bits of a phase gate),
// split by where they live in the op's stage:
//   mr: register-index bits, mt: thread-local (lane/warp) local-index bits,
//   mo: global index bits outside the tile.
struct TileOp {
    uint8_t type;
    uint8_t a, b;
    uint8_t tkind;    // TOP_DIAG1: TileBitKind of the target
    uint8_t mr;
    uint8_t pm;       // 1: matrix entries come from the per-member table (pmat)
    uint8_t gl;       // TOP_GRAD: row of this op in the pass's gradient table
    uint8_t fx;       // TOP_FLIP: register frame bits among mr
    uint32_t mt;
    uint32_t m;       // first matrix-pool entry
    uint64_t mo;
    uint64_t tmask;   // TOP_DIAG1 target: thread-local mask (TB_THREAD) or global mask (TB_OUTSIDE)
};

template <typename R> struct TileDFac {
    uint8_t type;
    uint8_t tkind;
    uint8_t a;
    uint8_t mr;
    uint32_t mt;
    uint64_t mo;
    uint64_t tmask;
    V<R> v0, v1, v2;
};

struct TileStage {
    uint8_t rloc[6];  // local bit of register bit j
    uint8_t wloc[3];  // local bit of warp bit w
    uint8_t lloc[5];  // local bit of lane bit i (the first and last stage: 0..4)
    uint8_t fcol[9];  // swizzle of the transpose into this stage: low-bit image of high local bit h + i
    uint8_t need_lt;  // some op of the stage tests thread-local bits
    uint8_t rflip;    // register frame at the end of the stage (register bits)
    uint16_t rw[6];   // transpose into this stage: byte offset of the previous stage's register bit j
    uint16_t rr[6];   // ... and of this stage's register bit j
    uint16_t op_begin, op_end;
};

// Low bits of a shared-memory position that the swizzle folds into: the lanes
// of one 128-byte wavefront (16 of complex64, 8 of complex128).
template <typename R> constexpr int swizzle_low_bits() { return sizeof(R) == 4 ? 4 : 3; }

template <typename R> struct TileParams {
    int n;            // member shift: member b starts at amplitude b << n
    int k;            // tile bits
    int n_stages;
    int n_free;       // n - k
    uint64_t total_tiles;
    InsertBits tins;  // sorted global positions of the tile bits
    uint8_t gbit[16]; // global bit of local bit i
    const V<R> *pmat; // per-member matrices of batched-parameter gates, or null
    uint32_t pm_stride;
    // adjoint sweep: the state is (phi, lambda) per member, told apart by the
    // member's top index bit, which is always the top register bit; gradient
    // op g of this pass adds its per-tile partial to gpart[gslot[g] * total_tiles + tile]
    int n_grad;
    double *gpart;
    uint16_t gslot[kTileMaxGrad];
    // TOP_ISING: per-member Ising coefficients in index bits, ising_stride
    // doubles per member: J[a * nq + b] (symmetric, zero diagonal), then h[nq],
    // then the constant; nq = qubits per member; tau in the op's tmask bits
    const double *ising;
    uint32_t ising_stride;
    int nq;
    // per Ising op (index in op.m) and member, ising_thr_stride doubles (see
    // ising_thr_stride): the op's phase factors as complex pairs, per thread
    // pattern, per register index and per tile
    const double *ising_thr;
    uint32_t ising_thr_stride;
    uint64_t tile_mask;   // global bits of the tile
    TileDFac<R> dfac[kTileMaxDFac];
    TileStage st[kTileMaxStages];
    TileOp op[kTileMaxOps];
    V<R> mat[kTileMaxMat];
};

static_assert(sizeof(TileParams<double>) <= 32700, "kernel parameter block too large");
// a complex128 pass descriptor converts to its double-float form in place
static_assert(sizeof(TileParams<dd>) == sizeof(TileParams<double>) && sizeof(ddc) == sizeof(double2) &&
                  alignof(ddc) == alignof(double2) && sizeof(TileDFac<dd>) == sizeof(TileDFac<double>),
              "double-float pass descriptor layout");

// Pointers a pass kernel needs at run time (not part of a pass's structure):
// per-member matrices of batched-parameter gates, the gradient partials of the
// adjoint sweep, and the Ising op's factor tables.
template <typename R> struct TilePtrs {
    const V<R> *pmat;
    double *gpart;
    const double *ising_thr;
};

// The values of a pass (matrix entries, diagonal-block factors), passed
// beside a specialised kernel whose descriptor holds only the structure: one
// kernel serves every pass of that structure (e.g. every step of a Trotter
// evolution, whose angles change from step to step).
template <typename R> struct TileVals {
    V<R> mat[kTileMaxMat];
    TileDFac<R> dfac[kTileMaxDFac];  // only v0, v1, v2 are read
};
static_assert(sizeof(TileVals<double>) <= 24576, "pass values exceed the kernel parameter budget");

// Dynamic shared memory of a pass kernel: the tile (sizeof(V<R>) << k bytes),
// then the transpose offsets, one word per (stage, thread), then the threads'
// tile-local lane/warp bits per stage (16 bits per stage and thread).
template <typename R>
__host__ __device__ constexpr size_t tile_smem_bytes(int k, int n_stages) {
    return (sizeof(V<R>) << k) +
           (size_t)(n_stages > 0 ? n_stages : 1) * (32u << TileCfg<R>::WB) * (sizeof(uint32_t) + sizeof(uint16_t));
}

// Inputs of the Ising-table kernel for one op: global bits of the stage's
// thread bits (lanes 0..4, then warps) and register bits, the pass's tile bits
// (k of them, global positions gb, inserted into a tile number by tins), tau,
// and where the op's tables start.
struct IsingTabP {
    int8_t tg[kTileLaneBits + kTileMaxWarpBits];
    int8_t rg[6];
    int8_t gb[16];
    int tb, rb, k, n_free;
    InsertBits tins;
    double tau;
    const double *ising;
    uint32_t ising_stride;
    int nq;
    double *out;
    uint32_t stride;   // doubles per member
    int members;
    int single;        // the state is complex64: sin and cos in FP32 (of the FP64-reduced angle)
};

// The Ising op's tables, per member, as (cos, sin) pairs of exp(-i tau x):
// for each thread pattern (threads of them) x = the coupling energy among its
// lane/warp bits plus the fields those bits put on the register bits, then
// for each register bit j, x = -2 times that field on j; for each register
// index x = its register-pair energy; for each tile (2^n_free) and each of the
// k tile bits, x = the field the outside bits and h put on it, then x = the
// tile's outside energy (couplings among outside bits, their h, the constant).
inline uint32_t ising_thr_stride(int rb, int threads, int k, int n_free) {
    return (uint32_t)(2 * threads * (1 + rb) + 2 * (1 << rb) + ((uint64_t)2 * (k + 1) << n_free));
}

}  // namespace qsim
