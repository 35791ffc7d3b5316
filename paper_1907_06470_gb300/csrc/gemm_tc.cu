// Tensor-core A-passes (Section 2.1 steps 2 and 5, Eq. (3)) on FP32 A with
// BF16 operands and FP32 accumulation in TMEM (tcgen05, sm_103a).
//
//   C[M x N] = Ahat[M x K] * X[K x N],   Ahat = A (forward) or A^T (transposed)
//
// A stays FP32 in HBM and is read exactly once per pass.  Each CTA is a
// persistent, warp-specialised pipeline:
//   warp 0     TMA producer: FP32 tile of A (64 x 128 or 128 x 64) per K
//              step of 64 (a 16-bit A: the A tile and the panel tile, one
//              thread, straight into the operand slot)
//   warp 1     TMEM allocator and single-thread tcgen05.mma issuer
//   warps 2-5  converters: round the FP32 tile to BF16 (and the residual to a
//              second BF16 "lo" tile in split mode), transposing it for A^T,
//              into the K-major 128-byte-swizzled operand layout
//   warps 6-9  epilogue: tcgen05.ld of the FP32 accumulator, stores to C
//   warp 10    TMA producer of the BF16 panel tile (64 x N, 128-byte
//              swizzle) per K step, for the converted sources
// Every producer loop runs in a warp of its own: two lanes of one warp that
// each spin on their own barriers take turns and starve each other.
// Two TMEM accumulators let the epilogue of one 128-row tile overlap the MMAs
// of the next.  The reduction dimension may be split across CTAs for load
// balance; the partial products are then added in a fixed order by a second
// kernel (in split order; with many splits and few outputs, contiguous blocks
// of splits combined by a fixed butterfly), so the result does not depend on
// scheduling.
//
// Split mode (BF16X3): A = A_hi + A_lo and X = X_hi + X_lo, each part BF16,
// C = A_hi X_hi + A_hi X_lo + A_lo X_hi, about 16 significant bits per operand.
//
// FP8 source: A is read as E4M3 codes with one power-of-two scale per
// block-cyclic tile; the converters decode each code to BF16 times its tile's
// scale (exact) -- a quarter of the HBM bytes of the FP32 source.
//
// BF16 source: A is read as a BF16 copy (half the bytes of FP32); the
// converters only move (or, for A^T, transpose) the 16-bit values into the
// operand layout.  The copy is written by the first forward pass over the FP32
// A, whose converters store the BF16 values they form anyway, so the later
// passes see exactly the operands the FP32 source would give.  The same
// kernels read an A the caller stores in 16 bits (Section 3.2: half-precision
// storage), BF16 or IEEE FP16; for FP16 the panel is rounded to FP16 too (one
// tcgen05.mma takes A and B of one type), and the split mode becomes two
// launches, A X_hi then A X_lo added, since A itself is exact.
//
// Every wait is bounded (about one second of global time); a wait that expires
// records DEV_TIMEOUT, every role stops issuing work, and the CTA frees its
// TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128;            // output rows per tile (MMA M)
constexpr int BK = 64;             // K per step: one 128-byte BF16 row
constexpr int A32_BYTES = BM * BK * 4;
constexpr int A8_BYTES = BM * BK;
constexpr int A16_BYTES = BM * BK * 2;
// operand (BF16 A + panel) ring depth: a runtime choice.  Converted sources
// take 2 or 4 slots (4 when the FP32 staging ring keeps at least 3 stages next
// to it); the 16-bit source, whose tiles TMA writes straight into the operand
// slots, takes as many as fit (up to 8).  Deeper rings let the panel tiles,
// which come from L2, be requested further ahead.
constexpr int kMaxSop = 8;
constexpr int kMaxSopConverted = 4;
// source of A: FP32, FP8 (E4M3 codes + tile scales) or 16-bit values (the
// plan's BF16 copy, or an A stored in BF16 / FP16)
constexpr int kSrc32 = 0, kSrc8 = 1, kSrc16 = 2;
constexpr int kSplitMaxNP = 192;   // widest split-mode panel one pass supports
constexpr int64_t kSplitChainSteps = 8;   // split mode: K steps (of 64) per TMEM accumulation chain
constexpr int64_t kPlainChainSteps = 32;  // other modes, when a TMEM running sum fits
constexpr int THREADS = 352;
// epilogue staging: one 32 x 33 float block per epilogue warp (row stride 33:
// no bank conflicts in either direction)
constexpr int kStageFloatsPerWarp = 32 * 33;
constexpr size_t kStageBytes = 4 * kStageFloatsPerWarp * sizeof(float);
constexpr uint64_t kWaitNs = 1000000000ull;

struct TcArgs {
  int64_t M;            // output rows
  int N;                // output columns written (r)
  int NP;               // MMA N: r rounded up to 16
  int acc_stride;       // TMEM column offset of the second accumulator
  int tmem_cols;        // TMEM columns allocated
  int64_t mtiles;
  int ntiles;           // column tiles of NP output columns (wide products; 1 for A-passes)
  int64_t ksteps;       // total K steps
  int64_t ksteps_per_split;
  int nsplit;
  int accumulate;       // 1: C += result (direct write only, nsplit == 1)
  int s32;              // FP32 staging ring depth
  int sop;              // operand ring depth (2 or 4)
  float* C;
  int64_t ldc;
  int64_t c_split_stride;
  int* status;
  const float* qscale;  // FP8 source: per-tile scales, qtn per tile row
  int64_t qm, qn, qtn;  // FP8 source: tile edges (in rows / columns of A)
  uint16_t* a16;        // FP32 forward pass: also store BF16(A) here (row stride ld16), or null
  uint16_t* a16lo;      // FP32 forward pass in split mode: also store BF16(A - BF16(A)) here, or null
  int64_t ld16;
  int a_lo;             // 16-bit source in split mode: 1 when A has a lo part (A = hi + lo)
  int64_t chunk_ks;     // K steps per TMEM accumulation chain (>= 1); chains are added in FP32 by the epilogue
  int sum_col;          // TMEM column of the running sum of a unit's chains (-1: in the output itself)
  int gram;             // 1: C = A^T A with one row tile: the panel operand is the converted A tile
  uint32_t idesc;       // tcgen05 instruction descriptor (operand type BF16 or FP16, FP32 accumulator)
  int c_stage;          // shared-memory offset of the epilogue's staging tiles (kStageBytes), or -1
};

#ifndef RSVD_TC_MAX_S32
#define RSVD_TC_MAX_S32 8
#endif
constexpr int kMaxS32 = RSVD_TC_MAX_S32;  // deepest FP32 staging ring

// Shared-memory plan: BF16 operand slots (A then panel), then the FP32 staging
// ring of depth S32 (a runtime choice: as deep as the 227 KB allow), then the
// barriers and the TMEM address word.
template <bool SPLIT, int SRC = kSrc32>
struct Layout {
  static constexpr int PARTS = SPLIT ? 2 : 1;
  // the 16-bit source needs no staging ring: TMA fills the operand slots
  static constexpr int STAGE_BYTES = SRC == kSrc8 ? A8_BYTES : (SRC == kSrc16 ? 0 : A32_BYTES);
  __host__ __device__ static size_t a16_off(int s, int part) { return ((size_t)s * PARTS + part) * A16_BYTES; }
  __host__ __device__ static size_t b16_base(int sop) { return (size_t)sop * PARTS * A16_BYTES; }
  __host__ __device__ static size_t b16_off(int NP, int sop, int s, int part) {
    return b16_base(sop) + ((size_t)s * PARTS + part) * (size_t)NP * 128;
  }
  __host__ __device__ static size_t a32_off(int NP, int sop, int s) {
    return b16_base(sop) + (size_t)sop * PARTS * NP * 128 + (size_t)s * STAGE_BYTES;
  }
  __host__ __device__ static size_t bar_off(int NP, int sop, int S32) { return a32_off(NP, sop, S32); }
  // barriers: full32, empty32 (kMaxS32 each), fullA, fullB, emptyOp (kMaxSop
  // each), accFull, accEmpty (2 each), drain, then the TMEM address word
  __host__ __device__ static size_t total(int NP, int sop, int S32) {
    return bar_off(NP, sop, S32) + (size_t)(2 * kMaxS32 + 3 * kMaxSop + 5) * 8 + 16 + 1024;
  }
};

// Roles whose waits can expire, recorded with the first expired wait.
enum : int { kWaitAFree = 1, kWaitStageFree = 2, kWaitPanelFree = 3, kWaitAccFree = 4, kWaitAFull = 5,
             kWaitPanelFull = 6, kWaitConvert = 7, kWaitAccFull = 8 };

// Record DEV_TIMEOUT, and in the two words after the status where the first
// expired wait was: role, ring slot and K step, then the unit.
__device__ __forceinline__ void flag_timeout(int* status, int role, int slot, int64_t ks, int64_t unit) {
  if (!status) return;
  if (atomicCAS(status + 1, 0, (role << 24) | ((slot & 255) << 16) | (int)(ks & 0xffff)) == 0)
    status[2] = (int)unit;
  dev_set_status(status, DEV_TIMEOUT);
}

// Position in a ring of n slots (slot, phase parity), advanced once per item.
struct RingPos {
  int slot = 0;
  uint32_t phase = 0;
  __device__ __forceinline__ void next(int n) {
    if (++slot == n) { slot = 0; phase ^= 1u; }
  }
};

// Two E4M3 codes (low byte first) to two floats, each times s.
__device__ __forceinline__ float2 e4m3x2_scaled(uint16_t codes, float s) {
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)codes, __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
  return make_float2(f.x * s, f.y * s);
}

template <bool TRANS, bool SPLIT, int SRC = kSrc32>
__global__ void __launch_bounds__(THREADS, 1)
tc_apass_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapAlo,
                const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapBlo,
                const TcArgs a) {
  static_assert(!(SPLIT && SRC == kSrc8), "the FP8 source has no split mode");
  constexpr bool SRC8 = SRC == kSrc8;
  // 16-bit source: TMA lands A tiles in the operand slots in the MMA's layout
  // (128-byte swizzle; K-major for A, MN-major for A^T) and no converter runs
  constexpr bool DIRECT = SRC == kSrc16;
  using L = Layout<SPLIT, SRC>;
  const int SOP = a.sop;
  const int S32 = a.s32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NP = a.NP;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::bar_off(NP, SOP, S32));
  uint64_t* full32 = bars;
  uint64_t* empty32 = full32 + kMaxS32;
  uint64_t* fullA = empty32 + kMaxS32;
  uint64_t* fullB = fullA + kMaxSop;
  uint64_t* emptyOp = fullB + kMaxSop;
  uint64_t* accFull = emptyOp + kMaxSop;
  uint64_t* accEmpty = accFull + 2;
  uint64_t* drain = accEmpty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const volatile int* vstatus = a.status;
  volatile int* vabort = &s_abort;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S32; ++i) { ptx::mbar_init(&full32[i], 1); ptx::mbar_init(&empty32[i], 4); }
    for (int i = 0; i < SOP; ++i) {
      ptx::mbar_init(&fullA[i], DIRECT ? 1 : 4);
      ptx::mbar_init(&fullB[i], 1);
      ptx::mbar_init(&emptyOp[i], 1);
    }
    for (int i = 0; i < 2; ++i) { ptx::mbar_init(&accFull[i], 1); ptx::mbar_init(&accEmpty[i], 4); }
    ptx::mbar_init(drain, 1);
    ptx::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0 && lane == 0) {
    ptx::prefetch_tensormap(&mapA);
    ptx::prefetch_tensormap(&mapB);
    if (SPLIT) ptx::prefetch_tensormap(&mapBlo);
    if (DIRECT && SPLIT && a.a_lo) ptx::prefetch_tensormap(&mapAlo);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // a unit is one output tile (128 rows x NP columns) over one K split;
  // unit u: row tile u % mtiles, column tile (u / mtiles) % ntiles, split
  // u / (mtiles ntiles)
  const int64_t mn_tiles = a.mtiles * a.ntiles;
  const int64_t units = mn_tiles * a.nsplit;
  const uint32_t b_bytes = (uint32_t)NP * 128u;

  if (warp == 0) {
    // ---------------- TMA producers ----------------
    // Lane 0 streams the FP32 tiles of A into their ring as far ahead as it
    // has free slots; lane 1 loads the panel tiles into the operand slots as
    // the MMAs free them.  Separate lanes, so that a panel slot still in use
    // never holds back the prefetch of A.
    if (lane == 0 && DIRECT) {
      // A tiles straight into the operand slots: forward, one 64 x 128 box
      // (K-major rows of 128 bytes); transposed, two 64 x 64 boxes (the two
      // 64-row halves of the MN-major tile, 8 KB apart).  A and the panel
      // share the slot, so this one thread loads both for each K step (two
      // producer lanes of one warp would take turns at their waits).
      const int nA = (SPLIT && a.a_lo) ? 2 : 1;
      const uint32_t a_bytes = (uint32_t)(A16_BYTES * nA);
      RingPos rop;
      uint32_t issued = 0, parity = 0;  // per slot: loaded at least once, phase of the last load
      for (int64_t u = blockIdx.x; u < units && !*vabort; u += gridDim.x) {
        const int64_t z = u / mn_tiles, mt = u % a.mtiles;
        const int64_t k0 = z * a.ksteps_per_split;
        const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
        const int32_t ny = (int32_t)(((u / a.mtiles) % a.ntiles) * NP);  // first panel column of the tile
        for (int64_t ks = k0; ks < k1; ++ks, rop.next(SOP)) {
          const int sop = rop.slot;
          if (!ptx::mbar_wait(&emptyOp[sop], rop.phase ^ 1, vstatus, kWaitNs)) {
            flag_timeout(a.status, kWaitAFree, sop, ks, u); s_abort = 1; break;
          }
          ptx::mbar_arrive_expect_tx(&fullA[sop], a_bytes);
          ptx::mbar_arrive_expect_tx(&fullB[sop], b_bytes * L::PARTS);
          issued |= 1u << sop;
          parity = (parity & ~(1u << sop)) | (rop.phase << sop);
          ptx::tma_load_2d(smem + L::b16_off(NP, SOP, sop, 0), &mapB, &fullB[sop], (int32_t)(ks * BK), ny);
          if (SPLIT)
            ptx::tma_load_2d(smem + L::b16_off(NP, SOP, sop, 1), &mapBlo, &fullB[sop], (int32_t)(ks * BK), ny);
          for (int part = 0; part < nA; ++part) {
            const CUtensorMap* map = part ? &mapAlo : &mapA;
            uint8_t* dst = smem + L::a16_off(sop, part);
            if (TRANS) {
              ptx::tma_load_2d(dst, map, &fullA[sop], (int32_t)(mt * BM), (int32_t)(ks * BK));
              ptx::tma_load_2d(dst + A16_BYTES / 2, map, &fullA[sop], (int32_t)(mt * BM + BM / 2), (int32_t)(ks * BK));
            } else {
              ptx::tma_load_2d(dst, map, &fullA[sop], (int32_t)(ks * BK), (int32_t)(mt * BM));
            }
          }
        }
      }
      // every load issued has landed before the CTA may exit (immediate unless stopped early)
      for (int i = 0; i < SOP; ++i)
        if (issued >> i & 1) {
          ptx::mbar_wait_drain(&fullA[i], parity >> i & 1, kWaitNs);
          ptx::mbar_wait_drain(&fullB[i], parity >> i & 1, kWaitNs);
        }
    } else if (lane == 0) {
      RingPos r32;
      uint32_t issued = 0, parity = 0;
      for (int64_t u = blockIdx.x; u < units && !*vabort; u += gridDim.x) {
        const int64_t z = u / mn_tiles, mt = u % a.mtiles;
        const int64_t k0 = z * a.ksteps_per_split;
        const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
        for (int64_t ks = k0; ks < k1; ++ks, r32.next(S32)) {
          const int s32 = r32.slot;
          if (!ptx::mbar_wait(&empty32[s32], r32.phase ^ 1, vstatus, kWaitNs)) {
            flag_timeout(a.status, kWaitStageFree, s32, ks, u); s_abort = 1; break;
          }
          ptx::mbar_arrive_expect_tx(&full32[s32], L::STAGE_BYTES);
          issued |= 1u << s32;
          parity = (parity & ~(1u << s32)) | (r32.phase << s32);
          void* dstA = smem + L::a32_off(NP, SOP, s32);
          if (TRANS) ptx::tma_load_2d(dstA, &mapA, &full32[s32], (int32_t)(mt * BM), (int32_t)(ks * BK));
          else ptx::tma_load_2d(dstA, &mapA, &full32[s32], (int32_t)(ks * BK), (int32_t)(mt * BM));
        }
      }
      for (int i = 0; i < S32; ++i)
        if (issued >> i & 1) ptx::mbar_wait_drain(&full32[i], parity >> i & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = a.idesc;
      RingPos rop;
      int64_t ua = 0;  // accumulation chains issued
      bool ok = true;
      for (int64_t u = blockIdx.x; u < units && ok && !*vabort; u += gridDim.x) {
        const int64_t z = u / mn_tiles;
        const int64_t k0 = z * a.ksteps_per_split;
        const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
       for (int64_t c0 = k0; c0 < k1 && ok; c0 += a.chunk_ks, ++ua) {
        const int64_t c1 = min(k1, c0 + a.chunk_ks);
        const int acc = (int)(ua & 1);
        const uint32_t pha = (uint32_t)((ua >> 1) & 1);
        if (!ptx::mbar_wait(&accEmpty[acc], pha ^ 1, vstatus, kWaitNs)) {
          flag_timeout(a.status, kWaitAccFree, acc, c0, u); s_abort = 1; ok = false; break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * a.acc_stride);
        uint32_t accumulate = 0;
        for (int64_t ks = c0; ks < c1; ++ks, rop.next(SOP)) {
          const int sop = rop.slot;
          const uint32_t phop = rop.phase;
          if (!ptx::mbar_wait(&fullA[sop], phop, vstatus, kWaitNs)) {
            flag_timeout(a.status, kWaitAFull, sop, ks, u); s_abort = 1; ok = false; break;
          }
          if (!a.gram && !ptx::mbar_wait(&fullB[sop], phop, vstatus, kWaitNs)) {
            flag_timeout(a.status, kWaitPanelFull, sop, ks, u); s_abort = 1; ok = false; break;
          }
          ptx::tc_fence_after();
          // Gram mode: the K-major tile of A^T is also the panel tile (its first NP rows)
          // A^T from a 16-bit source is MN-major: 16 K values span two 8-row
          // groups of 1024 bytes; K-major operands advance 32 bytes in the row
          constexpr bool MN = DIRECT && TRANS;
          const uint64_t astep = MN ? 2048 >> 4 : 2;
          const uint64_t ad = MN ? ptx::smem_desc_sw128_mn(smem + L::a16_off(sop, 0), A16_BYTES / 2)
                                 : ptx::smem_desc_sw128(smem + L::a16_off(sop, 0));
          const uint64_t bd = a.gram ? ad : ptx::smem_desc_sw128(smem + L::b16_off(NP, SOP, sop, 0));
          const bool alo = SPLIT && (!DIRECT || a.a_lo);
          const uint64_t adl = !alo ? 0
                               : (MN ? ptx::smem_desc_sw128_mn(smem + L::a16_off(sop, 1), A16_BYTES / 2)
                                     : ptx::smem_desc_sw128(smem + L::a16_off(sop, 1)));
          const uint64_t bdl = !SPLIT ? 0 : (a.gram ? adl : ptx::smem_desc_sw128(smem + L::b16_off(NP, SOP, sop, 1)));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            ptx::mma_bf16(d_tmem, ad + astep * kk, bd + 2 * kk, idesc, accumulate);
            accumulate = 1;
            if (SPLIT) {
              ptx::mma_bf16(d_tmem, ad + astep * kk, bdl + 2 * kk, idesc, 1);
              if (alo) ptx::mma_bf16(d_tmem, adl + astep * kk, bd + 2 * kk, idesc, 1);
            }
          }
          ptx::mma_commit(&emptyOp[sop]);
        }
        if (!ok) break;
        ptx::mma_commit(&accFull[acc]);
       }
      }
      // every product issued has completed before TMEM is released
      ptx::mma_commit(drain);
      ptx::mbar_wait_drain(drain, 0, kWaitNs);
    }
  } else if (warp < 6 && !DIRECT) {
    // ---------------- converters ----------------
    const int cw = warp - 2;
    RingPos r32, rop;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
      const int64_t z = u / mn_tiles, mt = u % a.mtiles;
      const int64_t k0 = z * a.ksteps_per_split;
      const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
      bool ok = true;
      for (int64_t ks = k0; ks < k1; ++ks, r32.next(S32), rop.next(SOP)) {
        const int s32 = r32.slot;
        const int sop = rop.slot;
        const bool w = ptx::mbar_wait(&full32[s32], r32.phase, vstatus, kWaitNs) &&
                       ptx::mbar_wait(&emptyOp[sop], rop.phase ^ 1, vstatus, kWaitNs);
        if (!__all_sync(0xffffffffu, w)) { if (lane == 0) flag_timeout(a.status, kWaitConvert, sop, ks, u); ok = false; break; }
        const float* src = reinterpret_cast<const float*>(smem + L::a32_off(NP, SOP, s32));
        uint8_t* hi = smem + L::a16_off(sop, 0);
        uint8_t* lo = smem + L::a16_off(sop, SPLIT ? 1 : 0);
        if (SRC8) {
          const uint8_t* src8 = smem + L::a32_off(NP, SOP, s32);
          if (!TRANS) {
            // codes[i][k], 128 rows of 64 bytes; the block lies in one tile.  Four
            // rows per step: lane l takes the 8 codes of 16-byte chunk c = l & 7
            // of row 4 step + l / 8 and writes the whole BF16 chunk.
            const float sc = a.qscale[(mt * BM / a.qm) * a.qtn + (ks * BK / a.qn)];
            const int c = lane & 7;
#pragma unroll 2
            for (int rr = 0; rr < 32; rr += 4) {
              const int i = cw * 32 + rr + (lane >> 3);
              const uint2 b = *reinterpret_cast<const uint2*>(src8 + i * BK + 8 * c);
              uint32_t hw[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const uint32_t word = t < 2 ? b.x : b.y;
                const __nv_bfloat162 h =
                    __float22bfloat162_rn(e4m3x2_scaled((uint16_t)(word >> (16 * (t & 1))), sc));
                hw[t] = *reinterpret_cast<const uint32_t*>(&h);
              }
              const uint32_t off = (uint32_t)i * 128u + ((((uint32_t)c) ^ ((uint32_t)i & 7u)) << 4);
              *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            }
          } else {
            // codes[k][i], 64 rows of 128 bytes: lane owns output row i
            const float sc = a.qscale[(ks * BK / a.qm) * a.qtn + (mt * BM / a.qn)];
            const int i = cw * 32 + lane;
#pragma unroll 2
            for (int c = 0; c < BK / 8; ++c) {
              uint32_t hw[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const uint16_t c2 = (uint16_t)src8[(c * 8 + 2 * t) * BM + i] |
                                    (uint16_t)((uint16_t)src8[(c * 8 + 2 * t + 1) * BM + i] << 8);
                const __nv_bfloat162 h = __float22bfloat162_rn(e4m3x2_scaled(c2, sc));
                hw[t] = *reinterpret_cast<const uint32_t*>(&h);
              }
              const uint32_t off = (uint32_t)i * 128u + ((((uint32_t)c) ^ ((uint32_t)i & 7u)) << 4);
              *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            }
          }
        } else if (!TRANS) {
          // src[i][k], 128 rows of 64 floats.  Two rows per step: lane l converts
          // the float4 q = l & 15 (k = 4q .. 4q+3) of row 2 step + l / 16, i.e.
          // half of 16-byte BF16 chunk q / 2.
          const int q = lane & 15;
          const uint32_t sub = ((uint32_t)q & 1u) << 3;
#pragma unroll 4
          for (int rr = 0; rr < 32; rr += 2) {
            const int i = cw * 32 + rr + (lane >> 4);
            const float4 v = reinterpret_cast<const float4*>(src + i * BK)[q];
            const __nv_bfloat162 h0 = __float22bfloat162_rn(make_float2(v.x, v.y));
            const __nv_bfloat162 h1 = __float22bfloat162_rn(make_float2(v.z, v.w));
            const uint32_t off = (uint32_t)i * 128u + ((((uint32_t)q >> 1) ^ ((uint32_t)i & 7u)) << 4) + sub;
            const uint2 hv =
                make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
            *reinterpret_cast<uint2*>(hi + off) = hv;
            // the BF16 copy of A for later passes (rows past M are TMA fill; the
            // copy's rows are padded to whole 64-column tiles); split mode: its
            // lo part too
            const bool keep = a.a16 && mt * BM + i < a.M;
            const int64_t coff = (mt * BM + i) * a.ld16 + ks * BK + 4 * q;
            if (keep) *reinterpret_cast<uint2*>(a.a16 + coff) = hv;
            if (SPLIT) {
              const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
              const __nv_bfloat162 l0 = __float22bfloat162_rn(make_float2(v.x - f0.x, v.y - f0.y));
              const __nv_bfloat162 l1 = __float22bfloat162_rn(make_float2(v.z - f1.x, v.w - f1.y));
              const uint2 lv =
                  make_uint2(*reinterpret_cast<const uint32_t*>(&l0), *reinterpret_cast<const uint32_t*>(&l1));
              *reinterpret_cast<uint2*>(lo + off) = lv;
              if (keep && a.a16lo) *reinterpret_cast<uint2*>(a.a16lo + coff) = lv;
            }
          }
        } else {
          // src[k][i], 64 rows of 128 floats: lane owns output row i, 8 K values per chunk
          const int i = cw * 32 + lane;
#pragma unroll 2
          for (int c = 0; c < BK / 8; ++c) {
            float v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = src[(c * 8 + t) * BM + i];
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const __nv_bfloat162 h = __float22bfloat162_rn(make_float2(v[2 * t], v[2 * t + 1]));
              hw[t] = *reinterpret_cast<const uint32_t*>(&h);
              if (SPLIT) {
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l =
                    __float22bfloat162_rn(make_float2(v[2 * t] - hf.x, v[2 * t + 1] - hf.y));
                lw[t] = *reinterpret_cast<const uint32_t*>(&l);
              }
            }
            const uint32_t off = (uint32_t)i * 128u + ((((uint32_t)c) ^ ((uint32_t)i & 7u)) << 4);
            *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (SPLIT) *reinterpret_cast<uint4*>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&fullA[sop]);
          ptx::mbar_arrive(&empty32[s32]);
        }
      }
      if (!ok) break;
    }
  } else if (warp == 10) {
    // ---------------- panel producer ----------------
    // With a converted source (FP32, FP8) the panel tiles load into the
    // operand slots as the MMAs free them, from a warp of their own so that
    // they never wait behind the A prefetch (and the other way round).
    if (lane == 0 && !a.gram && !DIRECT) {
      RingPos rop;
      uint32_t issued = 0, parity = 0;
      for (int64_t u = blockIdx.x; u < units && !*vabort; u += gridDim.x) {
        const int64_t z = u / mn_tiles;
        const int64_t k0 = z * a.ksteps_per_split;
        const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
        for (int64_t ks = k0; ks < k1; ++ks, rop.next(SOP)) {
          const int sop = rop.slot;
          if (!ptx::mbar_wait(&emptyOp[sop], rop.phase ^ 1, vstatus, kWaitNs)) {
            flag_timeout(a.status, kWaitPanelFree, sop, ks, u); s_abort = 1; break;
          }
          ptx::mbar_arrive_expect_tx(&fullB[sop], b_bytes * L::PARTS);
          issued |= 1u << sop;
          parity = (parity & ~(1u << sop)) | (rop.phase << sop);
          const int32_t ny = (int32_t)(((u / a.mtiles) % a.ntiles) * NP);  // first panel column of the tile
          ptx::tma_load_2d(smem + L::b16_off(NP, SOP, sop, 0), &mapB, &fullB[sop], (int32_t)(ks * BK), ny);
          if (SPLIT) ptx::tma_load_2d(smem + L::b16_off(NP, SOP, sop, 1), &mapBlo, &fullB[sop], (int32_t)(ks * BK), ny);
        }
      }
      for (int i = 0; i < SOP; ++i)
        if (issued >> i & 1) ptx::mbar_wait_drain(&fullB[i], parity >> i & 1, kWaitNs);
    }
  } else if (warp >= 6) {
    // ---------------- epilogue ----------------
    // (warps 6-9 only: with a 16-bit source the converter warps 2-5 stay idle)
    // Chains after the first of a unit are added in FP32 (rounded to
    // nearest) -- to a running sum in TMEM, or to the output -- so no TMEM
    // accumulation runs longer than chunk_ks K steps.
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
    int64_t ua = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int64_t z = u / mn_tiles, mt = u % a.mtiles;
      const int64_t k0 = z * a.ksteps_per_split;
      const int64_t k1 = min(a.ksteps, k0 + a.ksteps_per_split);
     for (int64_t ch = k0; ch < k1; ch += a.chunk_ks, ++ua) {
      const int acc = (int)(ua & 1);
      const uint32_t pha = (uint32_t)((ua >> 1) & 1);
      const bool w = ptx::mbar_wait(&accFull[acc], pha, vstatus, kWaitNs);
      if (!__all_sync(0xffffffffu, w)) { if (lane == 0) flag_timeout(a.status, kWaitAccFull, acc, ch, u); ok = false; break; }
      ptx::tc_fence_after();
      const int64_t row = mt * BM + q * 32 + lane;
      const int col0 = (int)((u / a.mtiles) % a.ntiles) * NP;  // first output column of the tile
      float* crow = a.C + z * a.c_split_stride + row * a.ldc + col0;
      const int ncols = a.N - col0;  // output columns left from col0
      const bool first = ch == k0, last = ch + a.chunk_ks >= k1;
      const bool tsum = a.sum_col >= 0;
      if (tsum && !last) {
        // keep the running sum in TMEM: sum = chain (first) or sum + chain
        for (int c0 = 0; c0 < NP; c0 += 32) {
          uint32_t v[32];
          ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)(acc * a.acc_stride + c0), v);
          if (!first) {
            uint32_t t[32];
            ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)(a.sum_col + c0), t);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(t[j]) + __uint_as_float(v[j]));
          } else {
            ptx::tmem_ld_wait();
          }
          ptx::tmem_st_32x32b_x32(lane_base + (uint32_t)(a.sum_col + c0), v);
        }
        ptx::tmem_st_wait();
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&accEmpty[acc]);
        continue;
      }
      // the unit's last chain: its value (plus the running sum) goes out
      const bool add = a.accumulate || (!tsum && !first);
      for (int c0 = 0; c0 < NP; c0 += 32) {
        uint32_t v[32];
        ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)(acc * a.acc_stride + c0), v);
        if (tsum && !first) {
          uint32_t t[32];
          ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)(a.sum_col + c0), t);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(t[j]) + __uint_as_float(v[j]));
        } else {
          ptx::tmem_ld_wait();
        }
        if (a.c_stage >= 0) {
          // through shared memory: the warp's 32 x 32 block goes out one row
          // per store, 32 consecutive columns (128 bytes) per instruction,
          // instead of 32 rows x 16 bytes (large outputs are write bound)
          float* stg = reinterpret_cast<float*>(smem + a.c_stage) + q * kStageFloatsPerWarp;
#pragma unroll
          for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(v[j]);
          __syncwarp();
          const int64_t row0 = mt * BM + q * 32;
          const bool col_ok = c0 + lane < ncols;
          float* cbase = a.C + z * a.c_split_stride + col0 + c0 + lane;
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            if (row0 + rr < a.M && col_ok) {
              float* p = cbase + (row0 + rr) * a.ldc;
              const float x = stg[rr * 33 + lane];
              *p = add ? *p + x : x;
            }
          }
          __syncwarp();
        } else if (row < a.M && c0 < ncols) {
          const int nv = min(32, ncols - c0);
          if (add && nv == 32 && (a.ldc & 3) == 0 && (col0 & 3) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4* p = reinterpret_cast<float4*>(crow + c0 + j);
              const float4 o = *p;
              *p = make_float4(o.x + __uint_as_float(v[j]), o.y + __uint_as_float(v[j + 1]),
                               o.z + __uint_as_float(v[j + 2]), o.w + __uint_as_float(v[j + 3]));
            }
          } else if (add) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv) crow[c0 + j] += __uint_as_float(v[j]);
          } else if (nv == 32 && (a.ldc & 3) == 0 && (col0 & 3) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(crow + c0 + j) =
                  make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                              __uint_as_float(v[j + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv) crow[c0 + j] = __uint_as_float(v[j]);
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&accEmpty[acc]);
     }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, (uint32_t)a.tmem_cols);
  }
}

// Xt[j][k] = bf16(X[k][j]) for j < r, 0 for r <= j < NP (and the residual
// into Xlo): the K-major panel operand of the MMA.
__device__ __forceinline__ uint16_t round16(float v, __nv_bfloat16*) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ uint16_t round16(float v, __half*) { return __half_as_ushort(__float2half_rn(v)); }
__device__ __forceinline__ float widen16(uint16_t h, __nv_bfloat16*) {
  return __bfloat162float(__ushort_as_bfloat16(h));
}
__device__ __forceinline__ float widen16(uint16_t h, __half*) { return __half2float(__ushort_as_half(h)); }

// X (K x r, FP32) -> the K-major 16-bit panel hi = round(X) and, when Xlo is
// set, lo = round(X - hi); H = __nv_bfloat16 or __half; columns r..NP-1 are 0
template <typename H>
__global__ void panel_to_16_kernel(int64_t K, int r, int NP, const float* __restrict__ X, int64_t ldx,
                                   uint16_t* __restrict__ Xhi, uint16_t* __restrict__ Xlo, int64_t ldb) {
  __shared__ float tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int64_t k = k0 + t;
    const int j = j0 + threadIdx.x;
    tile[t][threadIdx.x] = (k < K && j < r) ? X[k * ldx + j] : 0.f;
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int j = j0 + t;
    const int64_t k = k0 + threadIdx.x;
    if (j < NP && k < K) {
      const float v = tile[threadIdx.x][t];
      const uint16_t h = round16(v, (H*)nullptr);
      Xhi[(int64_t)j * ldb + k] = h;
      if (Xlo) Xlo[(int64_t)j * ldb + k] = round16(v - widen16(h, (H*)nullptr), (H*)nullptr);
    }
  }
}

// ---- host side ----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

rsvd_status encode_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                      uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return fail(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(RSVD_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
  return RSVD_OK;
}

struct TcShape {
  int64_t M, K, mtiles, ksteps, ksteps_per_split, ldb;
  int NP, nsplit;
};

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

// Split of the K range chosen for balance over the SMs: minimise
// ceil(units / SMs) * steps_per_unit plus the cost of the partial sums.
TcShape tc_shape(int64_t m, int64_t n, int r, int trans) {
  TcShape s;
  s.M = trans ? n : m;
  s.K = trans ? m : n;
  s.NP = (int)round_up(r, 16);
  s.mtiles = cdiv(s.M, BM);
  s.ksteps = cdiv(s.K, BK);
  s.ldb = round_up(s.K, 8);
  const int64_t sms = num_sms();
  double best = 1e300;
  int bestS = 1;
  for (int S = 1; S <= 256 && S <= s.ksteps; ++S) {
    const int64_t per = cdiv(s.ksteps, S);
    const int64_t used = cdiv(s.ksteps, per);
    const double rounds = (double)cdiv(s.mtiles * used, sms);
    const double partial = used > 1 ? (double)used * s.M * r * 8.0 / ((double)A32_BYTES * sms) : 0.0;
    const double cost = rounds * per + partial;
    if (cost < best - 1e-9) { best = cost; bestS = (int)used; }
  }
  s.ksteps_per_split = cdiv(s.ksteps, bestS);
  s.nsplit = (int)cdiv(s.ksteps, s.ksteps_per_split);
  return s;
}

}  // namespace

size_t tc_apass_ws_bytes(int64_t m, int64_t n, int r, int trans, int prec, int64_t, int64_t) {
  const TcShape s = tc_shape(m, n, r, trans);
  const bool split = prec == RSVD_PREC_BF16X3;
  Sizer z;
  z.take<__nv_bfloat16>((size_t)s.NP * s.ldb);
  if (split) z.take<__nv_bfloat16>((size_t)s.NP * s.ldb);
  if (s.nsplit > 1) z.take<float>((size_t)s.nsplit * round_up(s.M * r, 4));
  z.take<int>(4);
  return z.used + 256;
}

namespace {

// The FP32 source (A), the FP8 source (E4M3 codes of A with tile scales) or
// the BF16 copy of A.
struct TcSource {
  const rsvd_matrix* A = nullptr;   // FP32 source
  const Fp8Source* f8 = nullptr;    // FP8 source
  const Bf16Source* b16 = nullptr;  // 16-bit source (optionally with a lo part)
  uint16_t* copy16 = nullptr;       // FP32 forward pass: write the BF16 copy here
  uint16_t* copy16lo = nullptr;     // FP32 forward pass in split mode: and its lo part here
  int64_t ld16 = 0;
  int64_t kps = 0;                  // K steps per split to use (0: the balanced choice for this shape)
  bool wide = false;                // forward product with any number of output columns, in column tiles
};

rsvd_status tc_apass_run(const TcSource& src, int64_t m, int64_t n, int trans, int prec, int r, const float* X,
                         int64_t ldx, float* Y, int64_t ldy, void* ws, size_t ws_bytes, int* status,
                         cudaStream_t stream, bool accumulate) {
  const bool split = prec == RSVD_PREC_BF16X3;
  const bool src8 = src.f8 != nullptr;
  const bool src16 = src.b16 != nullptr;
  const bool f16 = src16 && src.b16->f16;
  // 16-bit source in split mode: A X_hi + A X_lo, plus A_lo X_hi when A has a
  // lo part (the split copy of an FP32 A)
  const bool a_lo = split && src16 && src.b16->lo != nullptr;
  if (r < 1 || (r > 512 && !src.wide)) return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: r must be in [1, 512]");
  if (src.wide && (trans || !src.A || src.copy16))
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core product: column tiles take a forward product over FP32 A");
  if (split && src8) return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: the FP8 source has no split mode");
  if (src16 && src.b16->lo && f16)
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: a split 16-bit source is BF16");
  if (src.copy16 && (trans || src8 || src16 || round_up(r, 16) > (split ? kSplitMaxNP : 256) ||
                     src.ld16 < round_up(n, BK) || src.ld16 % BK != 0 || (src.copy16lo && !split)))
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: the BF16 copy is written by one forward pass "
                                      "over FP32 A (ld16 a multiple of 64 covering n; its lo part in split mode)");
  if (!src.wide && round_up(r, 16) > (split ? kSplitMaxNP : 256)) {
    // wider than one accumulator (256 columns) or than the split-mode operand
    // ring fits: passes over column halves of the panel (A is read per half)
    const int h = (int)round_up(cdiv(r, 2), 16);
    RSVD_TRY(tc_apass_run(src, m, n, trans, prec, h, X, ldx, Y, ldy, ws, ws_bytes, status, stream, accumulate));
    return tc_apass_run(src, m, n, trans, prec, r - h, X + h, ldx, Y + h, ldy, ws, ws_bytes, status, stream,
                        accumulate);
  }
  if (!src8 && !src16 && (src.A->ld % 4 != 0 || (reinterpret_cast<uintptr_t>(src.A->data) & 15) != 0))
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: A needs a 16-byte aligned base and ld % 4 == 0");
  if (src16 && (src.b16->ld % 8 != 0 || (reinterpret_cast<uintptr_t>(src.b16->data) & 15) != 0 ||
                (reinterpret_cast<uintptr_t>(src.b16->lo) & 15) != 0))
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: a 16-bit A needs a 16-byte aligned base and ld % 8 == 0");
  if (src8 && (src.f8->ldc % 16 != 0 || (reinterpret_cast<uintptr_t>(src.f8->codes) & 15) != 0))
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: FP8 codes need a 16-byte aligned base and ld % 16 == 0");
  // column tiles of a wide product: NP columns each, the K range whole
  const int np_wide = (int)std::min<int64_t>(round_up(r, 16), split ? kSplitMaxNP : 256);
  TcShape s = tc_shape(m, n, src.wide ? np_wide : r, trans);
  const int ntiles = src.wide ? (int)cdiv(r, s.NP) : 1;
  const int64_t np_all = (int64_t)ntiles * s.NP;  // panel rows converted (all column tiles)
  if (src.wide) {
    s.ksteps_per_split = s.ksteps;
    s.nsplit = 1;
  }
  if (src.kps > 0) {  // a row block of a larger pass: that pass's split of the K range
    s.ksteps_per_split = src.kps;
    s.nsplit = (int)cdiv(s.ksteps, s.ksteps_per_split);
  }
  Carver c(ws, ws_bytes);
  auto* Xhi = c.take<uint16_t>((size_t)np_all * s.ldb);
  uint16_t* Xlo = split ? c.take<uint16_t>((size_t)np_all * s.ldb) : nullptr;
  const int64_t slab = round_up(s.M * r, 4);
  float* partial = s.nsplit > 1 ? c.take<float>((size_t)s.nsplit * slab) : nullptr;
  int* own_status = c.take<int>(4);
  if (c.overflow) return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: workspace too small");
  if (!status) {
    status = own_status;
    RSVD_CUDA(cudaMemsetAsync(status, 0, 4 * sizeof(int), stream));
  }

  // Gram C = A^T A of a matrix of at most 128 columns: the converters' K-major
  // tile of A^T (one row tile) already is the panel tile, rounded the same way
  const bool gram = trans && !src8 && !src16 && !src.copy16 && X == static_cast<const float*>(src.A->data) &&
                    ldx == src.A->ld && (int64_t)r == n && s.mtiles == 1;
  if (!gram) {  // panel -> BF16 or FP16 (hi, lo), K-major
    dim3 grid((unsigned)cdiv(s.K, 32), (unsigned)cdiv(np_all, 32));
    if (f16) panel_to_16_kernel<__half><<<grid, dim3(32, 8), 0, stream>>>(s.K, r, (int)np_all, X, ldx, Xhi, Xlo, s.ldb);
    else panel_to_16_kernel<__nv_bfloat16><<<grid, dim3(32, 8), 0, stream>>>(s.K, r, (int)np_all, X, ldx, Xhi, Xlo, s.ldb);
    RSVD_CUDA(after_launch());
  }
  const CUtensorMapDataType t16 = f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap mapA, mapAlo, mapB, mapBlo;
  const uint32_t box_in = trans ? BM : BK, box_out = trans ? BK : BM;
  if (src8) {
    RSVD_TRY(encode_2d(&mapA, CU_TENSOR_MAP_DATA_TYPE_UINT8, src.f8->codes, (uint64_t)n, (uint64_t)m,
                       (uint64_t)src.f8->ldc, box_in, box_out, CU_TENSOR_MAP_SWIZZLE_NONE));
  } else if (src16) {
    // tiles land in the operand slots in the MMA's layout: 128-byte rows
    // (64 values) with the 128-byte swizzle; A^T in two 64-wide halves
    const uint32_t bi = BK, bo = trans ? BK : BM;
    RSVD_TRY(encode_2d(&mapA, t16, src.b16->data, (uint64_t)n, (uint64_t)m, (uint64_t)src.b16->ld * 2, bi, bo,
                       CU_TENSOR_MAP_SWIZZLE_128B));
    if (a_lo)
      RSVD_TRY(encode_2d(&mapAlo, t16, src.b16->lo, (uint64_t)n, (uint64_t)m, (uint64_t)src.b16->ld * 2, bi, bo,
                         CU_TENSOR_MAP_SWIZZLE_128B));
  } else
    RSVD_TRY(encode_2d(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, src.A->data, (uint64_t)n, (uint64_t)m,
                       (uint64_t)src.A->ld * 4, box_in, box_out, CU_TENSOR_MAP_SWIZZLE_NONE));
  if (!a_lo) mapAlo = mapA;
  RSVD_TRY(encode_2d(&mapB, t16, Xhi, (uint64_t)s.K, (uint64_t)np_all, (uint64_t)s.ldb * 2, BK, (uint32_t)s.NP,
                     CU_TENSOR_MAP_SWIZZLE_128B));
  if (split)
    RSVD_TRY(encode_2d(&mapBlo, t16, Xlo, (uint64_t)s.K, (uint64_t)np_all, (uint64_t)s.ldb * 2, BK, (uint32_t)s.NP,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  else
    mapBlo = mapB;

  TcArgs ta;
  ta.M = s.M;
  ta.N = r;
  ta.NP = s.NP;
  ta.acc_stride = (int)round_up(s.NP, 32);
  // two accumulators and a running sum when it fits in the 512 columns of TMEM
  // (else split mode adds its chains to the output, other modes take one chain
  // per output tile)
  const bool tsum = 3 * ta.acc_stride <= 512;
  int cols = 32;
  while (cols < (tsum ? 3 : 2) * ta.acc_stride) cols *= 2;
  ta.tmem_cols = cols;
  ta.mtiles = s.mtiles;
  ta.ntiles = ntiles;
  ta.ksteps = s.ksteps;
  ta.ksteps_per_split = s.ksteps_per_split;
  ta.nsplit = s.nsplit;
  ta.accumulate = (s.nsplit == 1 && accumulate) ? 1 : 0;
  ta.C = s.nsplit > 1 ? partial : Y;
  ta.ldc = s.nsplit > 1 ? r : ldy;
  ta.c_split_stride = s.nsplit > 1 ? slab : 0;
  ta.status = status;
  ta.qscale = src8 ? src.f8->scales : nullptr;
  ta.qm = src8 ? src.f8->qm : 1;
  ta.qn = src8 ? src.f8->qn : 1;
  ta.qtn = src8 ? cdiv(n, src.f8->qn) : 1;
  ta.a16 = src.copy16;
  ta.a16lo = src.copy16lo;
  ta.ld16 = src.ld16;
  ta.a_lo = a_lo ? 1 : 0;
  // The tensor cores' FP32 accumulation truncates: each MMA added to an
  // accumulator shrinks it by about half a unit in 2^-24 on average, a bias
  // that grows with the number of MMAs in the chain (at 700 MMAs per chain it
  // lowered every singular value of the dense workload by 1.3e-5 to 1.9e-5).
  // Split-mode passes, which aim at FP32 accuracy, restart the accumulation
  // every kSplitChainSteps K steps (96 MMAs) and add the chains in FP32,
  // rounded to nearest, on the CUDA cores; other passes every
  // kPlainChainSteps K steps (128 MMAs) where the running sum fits TMEM.
  ta.chunk_ks = split ? kSplitChainSteps : (tsum ? kPlainChainSteps : s.ksteps_per_split);
  ta.sum_col = tsum ? 2 * ta.acc_stride : -1;
  ta.gram = gram ? 1 : 0;
  ta.idesc = f16 ? ptx::idesc_f16_f32(BM, (uint32_t)s.NP) : ptx::idesc_bf16_f32(BM, (uint32_t)s.NP);
  if (src16 && trans) ta.idesc |= ptx::kIdescAMajorMN;

  const int64_t units = s.mtiles * ntiles * s.nsplit;
  const int grid = (int)(units < num_sms() ? units : num_sms());
  constexpr size_t kSmemMax = 232448;
  auto need = [&](int sop, int depth) {
    if (src16)
      return split ? Layout<true, kSrc16>::total(s.NP, sop, depth) : Layout<false, kSrc16>::total(s.NP, sop, depth);
    return split ? Layout<true>::total(s.NP, sop, depth)
                 : (src8 ? Layout<false, kSrc8>::total(s.NP, sop, depth) : Layout<false>::total(s.NP, sop, depth));
  };
  int sop, s32;
  if (src16) {
    // no staging ring: as many operand slots as fit
    s32 = 0;
    sop = kMaxSop;
    while (sop > 2 && need(sop, 0) > kSmemMax) --sop;
  } else {
    // four operand slots when at least three staging stages still fit, else two
    sop = need(kMaxSopConverted, 3) <= kSmemMax ? kMaxSopConverted : 2;
    s32 = kMaxS32;
    while (s32 > 2 && need(sop, s32) > kSmemMax) --s32;
  }
  size_t smem = need(sop, s32);
  if (smem > kSmemMax) return fail(RSVD_ERR_UNSUPPORTED, "tensor-core A-pass: shared memory plan too large");
  // products with a large output (the column tiles of a wide product) stage
  // the epilogue's stores through shared memory, after the barriers; a
  // staging ring one stage shorter if that is what it takes
  ta.c_stage = -1;
  if (src.wide) {
    auto staged = [&](int sp, int d) { return round_up(need(sp, d) - 1024, 128) + kStageBytes + 1024; };
    if (staged(sop, s32) > kSmemMax && s32 > 2) --s32;
    if (staged(sop, s32) <= kSmemMax) {
      ta.c_stage = (int)round_up(need(sop, s32) - 1024, 128);
      smem = staged(sop, s32);
    } else {
      smem = need(sop, s32);
    }
  }
  ta.s32 = s32;
  ta.sop = sop;
  auto launch = [&](auto kern) -> rsvd_status {
    RSVD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, THREADS, smem, stream>>>(mapA, mapAlo, mapB, mapBlo, ta);
    RSVD_CUDA(after_launch());
    return RSVD_OK;
  };
  if (src8) {
    RSVD_TRY(trans ? launch(tc_apass_kernel<true, false, kSrc8>) : launch(tc_apass_kernel<false, false, kSrc8>));
  } else if (src16) {
    if (split)
      RSVD_TRY(trans ? launch(tc_apass_kernel<true, true, kSrc16>) : launch(tc_apass_kernel<false, true, kSrc16>));
    else
      RSVD_TRY(trans ? launch(tc_apass_kernel<true, false, kSrc16>) : launch(tc_apass_kernel<false, false, kSrc16>));
  } else if (trans) {
    RSVD_TRY(split ? launch(tc_apass_kernel<true, true>) : launch(tc_apass_kernel<true, false>));
  } else {
    RSVD_TRY(split ? launch(tc_apass_kernel<false, true>) : launch(tc_apass_kernel<false, false>));
  }
  if (s.nsplit > 1)
    RSVD_TRY(reduce_partials<float>(s.M, r, s.nsplit, partial, r, slab, Y, ldy, accumulate, stream));
  return RSVD_OK;
}

}  // namespace

size_t tc_gemm_wide_ws_bytes(int64_t M, int64_t K, int64_t N, int prec) {
  const int np = (int)std::min<int64_t>(round_up(N, 16), prec == RSVD_PREC_BF16X3 ? kSplitMaxNP : 256);
  const int64_t np_all = cdiv(N, np) * np;
  Sizer z;
  z.take<uint16_t>((size_t)np_all * round_up(K, 8));
  if (prec == RSVD_PREC_BF16X3) z.take<uint16_t>((size_t)np_all * round_up(K, 8));
  z.take<int>(4);
  (void)M;
  return z.used + 256;
}

rsvd_status tc_gemm_wide(const rsvd_matrix& A, int prec, int64_t N, const float* X, int64_t ldx, float* Y,
                         int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream) {
  if (N < 1 || N > 0x7fffffffLL || (prec != RSVD_PREC_BF16 && prec != RSVD_PREC_BF16X3) || A.dtype != RSVD_F32)
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core product: FP32 A, BF16 or BF16X3, N >= 1");
  TcSource src;
  src.A = &A;
  src.wide = true;
  return tc_apass_run(src, A.m, A.n, 0, prec, (int)N, X, ldx, Y, ldy, ws, ws_bytes, status, stream, false);
}

int64_t tc_ksteps_per_split(int64_t m, int64_t n, int r, int trans, int prec) {
  // a pass over column halves of the panel takes each half's own split
  if (round_up(r, 16) > (prec == RSVD_PREC_BF16X3 ? kSplitMaxNP : 256)) return 0;
  return tc_shape(m, n, r, trans).ksteps_per_split;
}

rsvd_status tc_apass_from_f32(const rsvd_matrix& A, int trans, int prec, int r, const float* X, int64_t ldx,
                              float* Y, int64_t ldy, int64_t, int64_t, void* ws, size_t ws_bytes,
                              int* status, cudaStream_t stream, bool accumulate, uint16_t* copy16,
                              int64_t ld16, uint16_t* copy16lo, int64_t kps) {
  TcSource src;
  src.A = &A;
  src.copy16 = copy16;
  src.copy16lo = copy16lo;
  src.ld16 = ld16;
  src.kps = kps;
  return tc_apass_run(src, A.m, A.n, trans, prec, r, X, ldx, Y, ldy, ws, ws_bytes, status, stream, accumulate);
}

rsvd_status tc_apass_from_bf16(const Bf16Source& b16, int trans, int r, const float* X, int64_t ldx, float* Y,
                               int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream) {
  return tc_apass_from_16(b16, trans, RSVD_PREC_BF16, r, X, ldx, Y, ldy, ws, ws_bytes, status, stream);
}

rsvd_status tc_apass_from_16(const Bf16Source& a16, int trans, int prec, int r, const float* X, int64_t ldx,
                             float* Y, int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream,
                             bool accumulate, int64_t kps) {
  if (prec != RSVD_PREC_BF16 && prec != RSVD_PREC_BF16X3)
    return fail(RSVD_ERR_INVALID_ARG, "tensor-core A-pass: a 16-bit A takes BF16 or BF16X3 precision");
  TcSource src;
  src.b16 = &a16;
  src.kps = kps;
  return tc_apass_run(src, a16.m, a16.n, trans, prec, r, X, ldx, Y, ldy, ws, ws_bytes, status, stream,
                      accumulate);
}

rsvd_status tc_apass_from_fp8(const Fp8Source& f8, int trans, int r, const float* X, int64_t ldx, float* Y,
                              int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream,
                              bool accumulate) {
  TcSource src;
  src.f8 = &f8;
  return tc_apass_run(src, f8.m, f8.n, trans, RSVD_PREC_BF16, r, X, ldx, Y, ldy, ws, ws_bytes, status, stream,
                      accumulate);
}

}  // namespace rsvd
