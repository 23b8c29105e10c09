// Tensor-core (tcgen05) parts of the W_H build (Eq. "schur complemnt
// reformulated": W_H = H A^-1 H^T = X^T D^-1 X, X = L^-1 H^T):
//   * the contraction W_H += Y_s^T Y_s for the supernodes whose scaled front
//     Y_s = D_s^-1/2 X_s has at least TC_MIN_COLS columns, and
//   * the forward-solve product of wide fronts, out = G_s F_top with the solve
//     operator G_s = [L_ss^-1; L_Rs L_ss^-1] (3xTF32 only): rows < w give X_s,
//     the others are subtracted from the update rows.
//
// Operands are packed into blocks of 128 rows x 32 K (K-major core-matrix
// layout: 8 rows x 16 bytes per core matrix, no swizzle), converted to the MMA
// operand type: k_pack_tc packs Y_s (contraction, B = A) or F_top (forward
// solve, B operand) once per build, k_pack_g packs G_s once per system.
// k_contract_tc, persistent blocks of 6 warps taking work units (128 x 128
// output tile pair I <= J of supernode s) from a counter, largest fronts first:
//   * a loader thread streams the blocks of tiles I and J through a ring of
//     STAGES shared-memory stages with cp.async.bulk (mbarrier transaction
//     counts), an MMA thread issues tcgen05.mma (M = N = 128) into a
//     128-column TMEM accumulator as stages land, committing each stage to
//     its release barrier;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31, i.e. the tile's rows) and adds the upper-triangle
//     entries into W_H.
// The pipeline's stage and phase come from running load / MMA counters that
// carry over from one unit to the next.
// Modes: TF32X3 splits every operand into a TF32 part and a TF32 remainder and
// accumulates hi*hi + hi*lo + lo*hi (FP32-level error); TF32 and BF16 use one
// rounded part.  Every mbarrier wait is bounded; a wait that runs out sets the
// scene's device error word and the block skips its epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "icr_internal.h"

namespace icr {
namespace {

constexpr int TM = TC_TILE;   // output tile (M = N)
constexpr int KT = TC_KT;     // K rows per stage
// bound of the waits that must not be cut short: copies in flight landing and
// every issued MMA completing before TMEM is freed (microseconds in practice)
constexpr uint64_t DRAIN_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// largest position p in [lo, hi) with P[p] <= u (P a non-decreasing prefix
// array with P[lo] <= u < P[hi]): the supernode owning work unit u
__device__ __forceinline__ int find_unit(const int* __restrict__ P, int lo, int hi, int u) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P[mid] <= u)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// tcgen05 shared-memory descriptor: start >> 4 in bits 0-13, leading (K)
// core-matrix stride >> 4 in bits 16-29, stride between 8-row groups >> 4 in
// bits 32-45, descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: F32 accumulator (bits 4-5 = 1), A and B type in bits
// 7-9 / 10-12 (TF32 = 2 for kind::tf32, BF16 = 1 for kind::f16), K-major A and
// B, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t instr_desc(int ab_type) {
  return (1u << 4) | ((uint32_t)ab_type << 7) | ((uint32_t)ab_type << 10) | ((uint32_t)(TM >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` of an mbarrier: true once the phase has
// completed; false after limit_ns of global time, at once when `alive` (the
// CTA's shared ok flag) has been cleared by the other side of the pipeline,
// or, with limit_ns = 0, after one non-blocking poll (failure injection).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns,
                                          const volatile int* alive = nullptr) {
  uint32_t done;
  if (limit_ns == 0) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
  }
  const uint64_t t0 = global_ns();
  for (;;) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (alive && *alive == 0) return false;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int MODE>
struct TcTraits;
template <>
struct TcTraits<ICR_CONTRACT_TF32X3> {
  static constexpr int EB = 4, PARTS = 2, KMMA = 8, TYPE = 2;
};
template <>
struct TcTraits<ICR_CONTRACT_TF32> {
  static constexpr int EB = 4, PARTS = 1, KMMA = 8, TYPE = 2;
};
template <>
struct TcTraits<ICR_CONTRACT_BF16> {
  static constexpr int EB = 2, PARTS = 1, KMMA = 16, TYPE = 1;
};

template <int MODE>
__host__ __device__ constexpr int tile_bytes() {
  return TM * KT * TcTraits<MODE>::EB;
}
// byte offset of element (r, k) of a K-major TM x KT tile: core matrix (r/8, k/C)
// with C elements per 16 bytes; core matrices contiguous along K, 8-row groups
// KT/C core matrices apart
template <int EB>
__host__ __device__ constexpr int tile_off(int r, int k) {
  return (r >> 3) * ((KT / (16 / EB)) * 128) + (k / (16 / EB)) * 128 + (r & 7) * 16 + (k % (16 / EB)) * EB;
}

constexpr int STAGES = 3;

// Packs the scaled front Y_s into operand blocks: block (s, I, kt) holds rows
// kt*KT.. of Y_s restricted to columns I*TM.., as PARTS planes of a K-major
// TM x KT tile (tile row r = front column I*TM + r, tile k = front row kt*KT + k).
// Staged through shared memory so that global reads and writes are coalesced.
// Writes the KT x TM staging tile sy (sy[k][r]) as one K-major operand block:
// PARTS planes of TM x KT, 16-byte chunk q = core matrix (g, j), row r8.
template <int MODE>
__device__ __forceinline__ void pack_tile(const float (*sy)[TM + 1], unsigned char* blk) {
  using TR = TcTraits<MODE>;
  constexpr int C = 16 / TR::EB;
  constexpr int CHUNKS = TM * KT / C;
  for (int q = threadIdx.x; q < CHUNKS; q += blockDim.x) {
    const int cm = q >> 3, r8 = q & 7;                 // core matrix index, row inside it
    const int g = cm / (KT / C), j = cm % (KT / C);
    const int r = g * 8 + r8;
    if constexpr (MODE == ICR_CONTRACT_BF16) {
      unsigned short h[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) h[c] = __bfloat16_as_ushort(__float2bfloat16_rn(sy[j * C + c][r]));
      *(uint4*)(blk + q * 16) = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                                           h[6] | (h[7] << 16));
    } else {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float x = sy[j * C + c][r];
        hi[c] = to_tf32(x);
        lo[c] = to_tf32(x - __uint_as_float(hi[c]));
      }
      *(uint4*)(blk + q * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      if constexpr (TR::PARTS == 2)
        *(uint4*)(blk + tile_bytes<MODE>() + q * 16) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// Packs, for the work units [plan[pa], plan[pb]) of a list over level_list
// positions, 128-column x KT-row blocks of a front: unit (s, I, kt) holds rows
// kt*KT.. of the source restricted to columns I*TM.., as PARTS planes of a
// K-major TM x KT tile (tile row r = column I*TM + r, tile k = row kt*KT + k).
// The source is the scaled front Y_s (rows from fr_ptr[s]) or the assembled top
// rows F_top (rows from super_ptr[s]).  Staged through shared memory so that
// global reads and writes are coalesced.
template <int MODE>
__device__ __forceinline__ void d_pack_tc(const VB& vb, const int* __restrict__ plan, int pa, int pb,
                                          const int* __restrict__ level_list, const int* __restrict__ super_ptr,
                                          const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                                          const int64_t* __restrict__ boff, const float* __restrict__ src,
                                          int from_ftop, int64_t ldx, unsigned char* pk, float* X,
                                          const int* __restrict__ gsplit_p) {
  using TR = TcTraits<MODE>;
  __shared__ float sy[KT][TM + 1];
  const int u1 = plan[pb];
  const int gsplit = from_ftop ? *gsplit_p : 1;   // read once: the unit loop has no other dependent load on it
  for (int u = plan[pa] + vb.bx; u < u1; u += vb.gx) {   // block-uniform
    const int pos = find_unit(plan, pa, pb, u);
    const int s = level_list[pos];
    const int ncol = 3 * qcount[s];
    const int w = super_ptr[s + 1] - super_ptr[s];
    const int nk = (w + KT - 1) / KT;
    const int local = u - plan[pos];
    const int I = local / nk, kt = local % nk;
    const float* Ys = src + (from_ftop ? (int64_t)super_ptr[s] : fr_ptr[s]) * ldx;
    // F_top of a level whose units are split over K (gsplit_p: the level's
    // split factor): the K parts add the product's rows < w (X_s) into X, so
    // those rows start at zero; unsplit units store them
    float* Xz = from_ftop && tc_parts(gsplit, nk) > 1 ? X + fr_ptr[s] * ldx : nullptr;
    for (int e = threadIdx.x; e < KT * TM; e += blockDim.x) {
      const int k = e / TM, r = e % TM;
      const int row = kt * KT + k, col = I * TM + r;
      const bool in = row < w && col < ncol;
      sy[k][r] = in ? Ys[(int64_t)row * ldx + col] : 0.f;
      if (Xz && in) Xz[(int64_t)row * ldx + col] = 0.f;
    }
    __syncthreads();
    unsigned char* blk = pk + (boff[s] + (int64_t)I * nk + kt) * (int64_t)(TR::PARTS * tile_bytes<MODE>());
    pack_tile<MODE>(sy, blk);
    __syncthreads();   // sy is refilled by the next unit
  }
}

template <int MODE>
__global__ void __launch_bounds__(256)
    k_pack_tc(const int* __restrict__ plan, int pa, int pb, const int* __restrict__ level_list,
              const int* __restrict__ super_ptr, const int64_t* __restrict__ fr_ptr,
              const int* __restrict__ qcount, const int64_t* __restrict__ boff, const float* __restrict__ src,
              int from_ftop, int64_t ldx, unsigned char* pk, float* X, const int* __restrict__ gsplit_p) {
  pdl_entry();
  d_pack_tc<MODE>(own_block(), plan, pa, pb, level_list, super_ptr, fr_ptr, qcount, boff, src, from_ftop, ldx, pk, X,
                  gsplit_p);
}

template <int MODE>
struct pack_tc_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = true;
  static auto kernel() { return &k_pack_tc<MODE>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_pack_tc<MODE>(vb, a...);
  }
};

// Packs the solve operators G_s of the supernodes at least TC_GEMM_MIN_W wide
// (column-major (w + r) x w panels, ld = w + r) into 128-row x 32-K blocks with
// two TF32 planes; one CTA per block, the blocks listed by the host as
// (supernode, row tile, K tile).
__global__ void __launch_bounds__(256)
    k_pack_g(const int* __restrict__ blocks, int nblocks, const int* __restrict__ super_ptr,
             const int64_t* __restrict__ rowpat_ptr, const int64_t* __restrict__ val_ptr,
             const int64_t* __restrict__ goff, const float* __restrict__ G, unsigned char* pk) {
  pdl_entry();
  __shared__ float sy[KT][TM + 1];
  for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int s = blocks[3 * b], rt = blocks[3 * b + 1], kt = blocks[3 * b + 2];
    const int w = super_ptr[s + 1] - super_ptr[s];
    const int nrows = w + (int)(rowpat_ptr[s + 1] - rowpat_ptr[s]);
    const int nk = (w + KT - 1) / KT;
    const float* Gs = G + val_ptr[s];
    for (int e = threadIdx.x; e < KT * TM; e += blockDim.x) {
      const int k = e / TM, r = e % TM;   // consecutive threads: consecutive rows of one column
      const int row = rt * TM + r, col = kt * KT + k;
      sy[k][r] = (row < nrows && col < w) ? Gs[(int64_t)col * nrows + row] : 0.f;
    }
    __syncthreads();
    pack_tile<ICR_CONTRACT_TF32X3>(sy, pk + (goff[s] + (int64_t)rt * nk + kt) * (int64_t)(2 * tile_bytes<ICR_CONTRACT_TF32X3>()));
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pipeline
// CTA of 6 warps.  Warp 5 (lane 0) streams the nk K-blocks of A and B (B = A
// when same) through the STAGES-deep shared-memory ring with cp.async.bulk,
// refilling a stage as soon as the MMAs that read it have completed; warp 4
// (lane 0) issues the MMAs (M = N = 128) as soon as a stage has landed, so the
// tensor pipe holds the MMAs of every landed stage while copies run ahead;
// warps 0-3 own the tile's rows (warp w reads TMEM lanes 32w..32w+31).  The tensor cores accumulate at most PROMOTE_KB
// K-blocks (128 K) into one of two 128-column TMEM buffers; the row warps then
// add that partial tile into FP32 registers (IEEE adds) and free the buffer, so
// the MMA's own accumulation never runs over more than 128 products.  Load,
// MMA-chunk and buffer counters run over the CTA's whole life: stage or buffer
// = count % depth, phase parity = (count / depth) & 1.  Every wait is bounded.
constexpr int PROMOTE_KB = 128 / KT;   // K-blocks per TMEM chunk: 128 K
constexpr int TC_THREADS = 192;
// TMEM accumulator buffers of 128 columns: four (all 512 columns of the SM)
// in 3xTF32 mode, where the shared-memory ring keeps one CTA per SM, so that
// the MMA thread can run up to four chunks ahead of a unit's epilogue; two
// in the TF32 and BF16 modes, which fit two CTAs per SM
template <int MODE>
__host__ __device__ constexpr int tmem_bufs() {
  return TcTraits<MODE>::PARTS == 2 ? 4 : 2;
}
constexpr int TMEM_MAX_BUFS = 4;

constexpr int UQ = 4;   // slots of the unit ring from the MMA-issuing thread to the accumulator warps

struct TcBars {
  uint64_t full[STAGES], empty[STAGES];   // shared-memory ring
  uint64_t tfull[TMEM_MAX_BUFS], tfree[TMEM_MAX_BUFS];   // TMEM buffers: MMAs done / drained
  uint64_t fin;                           // teardown: every MMA issued has completed
  uint64_t qfull[UQ], qfree[UQ];          // unit ring: unit published / taken by the four accumulator warps
  int uq[UQ];                             // unit ring: the work-list counter value of each unit (>= total: end)
};

// The MMA-issuing thread takes work units from the list counter and publishes
// each in the unit ring before it issues the unit's MMAs; the loader warp and
// the accumulator warps take the units from the ring in the same order.
// The producer thus runs ahead into the next unit while the accumulator warps
// still drain the last one (the TMEM buffers and the operand ring bound how
// far).  Every wait is bounded and gives up when the other side has.
__device__ __forceinline__ bool uq_push(TcBars& br, uint32_t i, int ur, uint64_t wait_ns, const volatile int* alive) {
  const int slot = (int)(i % UQ);
  if (i >= UQ && !mbar_wait(smem_u32(&br.qfree[slot]), ((i / UQ) - 1) & 1, wait_ns, alive)) return false;
  *(volatile int*)&br.uq[slot] = ur;
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&br.qfull[slot])) : "memory");
  return true;
}

// one accumulator warp: the counter value of unit i, or -1 when the wait gave up
__device__ __forceinline__ int uq_pop(TcBars& br, uint32_t i, int lane, uint64_t wait_ns, const volatile int* alive) {
  const int slot = (int)(i % UQ);
  const int fine = mbar_wait(smem_u32(&br.qfull[slot]), (i / UQ) & 1, wait_ns, alive);
  if (!__all_sync(0xffffffffu, fine)) return -1;
  const int ur = *(volatile int*)&br.uq[slot];
  __syncwarp();
  if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&br.qfree[slot])) : "memory");
  return ur;
}

// warp 5, lane 0: the copies of one unit's nk K-blocks into the ring, each
// into the next stage once the MMAs of its last use have completed (gl: the
// CTA's running count of copies)
template <int MODE>
__device__ bool tc_load(const unsigned char* blkA, const unsigned char* blkB, bool same, int nk,
                        unsigned char* smem, TcBars& br, uint32_t& gl, uint64_t wait_ns, const volatile int* alive) {
  using TR = TcTraits<MODE>;
  constexpr int BLK = TR::PARTS * tile_bytes<MODE>();
  const uint32_t bytes = same ? BLK : 2 * BLK;
  for (int kt = 0; kt < nk; ++kt) {
    const uint32_t g = gl;
    const int st = g % STAGES;
    if (g >= STAGES && !mbar_wait(smem_u32(&br.empty[st]), ((g / STAGES) - 1) & 1, wait_ns, alive)) return false;
    unsigned char* dA = smem + st * 2 * BLK;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&br.full[st])),
                 "r"(bytes));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dA)),
        "l"(blkA + (int64_t)kt * BLK), "r"((uint32_t)BLK), "r"(smem_u32(&br.full[st]))
        : "memory");
    if (!same)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              smem_u32(dA + BLK)),
          "l"(blkB + (int64_t)kt * BLK), "r"((uint32_t)BLK), "r"(smem_u32(&br.full[st]))
          : "memory");
    ++gl;
  }
  return true;
}

// warp 5, lane 0, before the CTA exits: the last copy into every stage has
// landed (bounded; no later copy reuses those stages, so each wait names one
// phase), so no copy writes shared memory after the CTA is gone
__device__ __forceinline__ void tc_load_drain(TcBars& br, uint32_t gl) {
  for (uint32_t g = gl > (uint32_t)STAGES ? gl - STAGES : 0u; g < gl; ++g)
    mbar_wait(smem_u32(&br.full[g % STAGES]), (g / STAGES) & 1, DRAIN_NS);
}

// warp 4, lane 0: the MMAs of one unit's nk K-blocks (gm: running count of
// K-blocks multiplied, gc: of TMEM chunks); each stage is released to the
// loader by a commit when its MMAs complete, each chunk's TMEM buffer handed
// to the accumulator warps by a commit after its last K-block
template <int MODE>
__device__ bool tc_mma(bool same, int nk, unsigned char* smem, TcBars& br, uint32_t tmem, uint32_t& gm, uint32_t& gc,
                       uint64_t wait_ns, const volatile int* alive) {
  using TR = TcTraits<MODE>;
  constexpr int BLK = TR::PARTS * tile_bytes<MODE>();
  const uint32_t idesc = instr_desc(TR::TYPE);
  constexpr int SBO = (KT / (16 / TR::EB)) * 128;
  const int nchunks = (nk + PROMOTE_KB - 1) / PROMOTE_KB;
  for (int kc = 0; kc < nk; ++kc) {
    const int ch = kc / PROMOTE_KB, first = kc % PROMOTE_KB == 0;
    const bool last = kc % PROMOTE_KB == PROMOTE_KB - 1 || kc == nk - 1;
    const uint32_t gb = gc + ch;                 // buffer use counter of this chunk
    constexpr int NB = tmem_bufs<MODE>();
    const uint32_t tb = tmem + (gb % NB) * TM;   // its 128 TMEM columns
    if (first && gb >= NB && !mbar_wait(smem_u32(&br.tfree[gb % NB]), ((gb / NB) - 1) & 1, wait_ns, alive))
      return false;
    const uint32_t g = gm + kc;
    const int st = g % STAGES;
    if (!mbar_wait(smem_u32(&br.full[st]), (g / STAGES) & 1, wait_ns, alive)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const unsigned char* sA = smem + st * 2 * BLK;
    const unsigned char* sB = same ? sA : sA + BLK;
#pragma unroll
    for (int kk = 0; kk < KT / TR::KMMA; ++kk) {
      const uint32_t off = kk * 256;   // two core matrices along K per MMA
#pragma unroll
      for (int term = 0; term < (TR::PARTS == 2 ? 3 : 1); ++term) {
        const int ai = term == 2 ? 1 : 0, bi = term == 1 ? 1 : 0;
        const uint64_t ad = smem_desc(smem_u32(sA + ai * tile_bytes<MODE>()) + off, 128, SBO);
        const uint64_t bd = smem_desc(smem_u32(sB + bi * tile_bytes<MODE>()) + off, 128, SBO);
        const uint32_t acc = (!first || kk > 0 || term > 0) ? 1u : 0u;
        if constexpr (MODE == ICR_CONTRACT_BF16)
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                  tb),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                  tb),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_u32(&br.empty[st])));
    if (last)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&br.tfull[gb % NB])));
  }
  gm += nk;
  gc += nchunks;
  return true;
}

// warps 0-3: acc[0..127] <- sum over the unit's chunks of the row's TMEM columns
template <int NB>
__device__ bool tc_drain(int nk, TcBars& br, uint32_t tmem, int warp, int lane, uint32_t& gc, float* acc,
                         uint64_t wait_ns, const volatile int* alive) {
  const int nchunks = (nk + PROMOTE_KB - 1) / PROMOTE_KB;
  bool ok = true;
  for (int ch = 0; ch < nchunks; ++ch) {
    const uint32_t gb = gc + ch;
    const int fine = ok && mbar_wait(smem_u32(&br.tfull[gb % NB]), (gb / NB) & 1, wait_ns, alive);
    if (!__all_sync(0xffffffffu, fine)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t base = tmem + (gb % NB) * TM + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int c0j = 0; c0j < TM; c0j += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(base + (uint32_t)c0j));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[c0j + j] = ch == 0 ? __uint_as_float(v[j]) : acc[c0j + j] + __uint_as_float(v[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&br.tfree[gb % NB])));
  }
  gc += nchunks;
  return ok;
}

template <int NB>
__device__ __forceinline__ void tc_setup(uint32_t* tmem_base, TcBars& br, volatile int* ok_sh) {
  const int tid = threadIdx.x;
  if ((tid >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_base)),
                 "r"((uint32_t)(NB * TM)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.empty[i])), "r"(1));
    }
    for (int i = 0; i < NB; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.tfull[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.tfree[i])), "r"(4));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.fin)), "r"(1));
    for (int i = 0; i < UQ; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.qfull[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&br.qfree[i])), "r"(5));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n");
    *ok_sh = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
}

// every MMA the CTA issued has completed (bounded) before TMEM is freed
template <int NB>
__device__ __forceinline__ void tc_teardown(uint32_t tmem, TcBars& br) {
  if (threadIdx.x == 128) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_u32(&br.fin)));
    mbar_wait(smem_u32(&br.fin), 0, DRAIN_NS);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)(NB * TM)));
}

// Contraction: persistent CTAs take units (128 x 128 output tile pair I <= J
// of supernode s) from a counter, largest fronts first; the row warps add the
// tile's upper-triangle entries into W_H.
template <int MODE>
__device__ __forceinline__ void d_contract_tc(const VB& vb, const int* __restrict__ plan, int* counter, int ns,
                                              const int* __restrict__ level_list, const int* __restrict__ super_ptr,
                                              const int* __restrict__ qcount, const int* __restrict__ qidx,
                                              const int64_t* __restrict__ boff, int m,
                                              const unsigned char* __restrict__ pk, float* WH, int64_t ldw,
                                              int* dev_err, int cache_plan, const int* __restrict__ tsplit_p,
                                              uint64_t wait_ns) {
  using TR = TcTraits<MODE>;
  constexpr int BLK = TR::PARTS * tile_bytes<MODE>();
  extern __shared__ __align__(1024) unsigned char smem[];   // STAGES x (A block, B block), then the list's prefix
  __shared__ __align__(8) TcBars br;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int ok_sh;   // cleared by the side of the pipeline whose wait ran out
  const int total = plan[ns];
  if ((int)vb.bx >= total) return;   // uniform: before any allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tsplit = *tsplit_p;
  // the unit search reads the list's prefix sums from shared memory when they fit
  const int* plan_s = plan;
  if (cache_plan) {
    int* ps = reinterpret_cast<int*>(smem + STAGES * 2 * BLK);
    for (int i = tid; i <= ns; i += TC_THREADS) ps[i] = plan[i];
    plan_s = ps;
  }
  tc_setup<tmem_bufs<MODE>()>(&tmem_base, br, &ok_sh);
  const uint32_t tmem = tmem_base;
  uint32_t gl = 0, gm = 0, gc = 0;
  // unit ur (counter value): supernode s, tile pair I <= J, K part [k0, k0 + nku)
  auto decode = [&](int ur, int& s, int& ncol, int& I, int& J, int& nk, int& k0, int& nku) {
    const int u = total - 1 - ur;
    const int pos = find_unit(plan_s, 0, ns, u);
    s = level_list[pos];
    ncol = 3 * qcount[s];
    const int nI = (ncol + TM - 1) / TM;
    const int w = super_ptr[s + 1] - super_ptr[s];
    nk = (w + KT - 1) / KT;
    const int nsk = tc_parts(tsplit, nk);   // unit = (tile pair, K part)
    const int kc = (u - plan_s[pos]) % nsk;
    int rem = (u - plan_s[pos]) / nsk;
    I = 0;
    while (rem >= nI - I) {
      rem -= nI - I;
      ++I;
    }
    J = I + rem;
    k0 = kc * nk / nsk;
    nku = (kc + 1) * nk / nsk - k0;
  };
  if (warp == 4) {
    if (lane == 0) {
      for (uint32_t i = 0;; ++i) {
        const int ur = ok_sh ? atomicAdd(counter, 1) : total;   // a pipeline that gave up takes no more
        if (!uq_push(br, i, ur < total ? ur : total, wait_ns, &ok_sh)) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
          break;
        }
        if (ur >= total) break;
        int s, ncol, I, J, nk, k0, nku;
        decode(ur, s, ncol, I, J, nk, k0, nku);
        if (!tc_mma<MODE>(I == J, nku, smem, br, tmem, gm, gc, wait_ns, &ok_sh)) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
          break;
        }
      }
    }
  } else if (warp == 5) {   // the loader
    for (uint32_t i = 0;; ++i) {
      const int ur = uq_pop(br, i, lane, wait_ns, &ok_sh);
      if (ur < 0) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      if (ur >= total) break;
      int fine = 1;
      if (lane == 0) {
        int s, ncol, I, J, nk, k0, nku;
        decode(ur, s, ncol, I, J, nk, k0, nku);
        fine = tc_load<MODE>(pk + (boff[s] + (int64_t)I * nk + k0) * BLK, pk + (boff[s] + (int64_t)J * nk + k0) * BLK,
                             I == J, nku, smem, br, gl, wait_ns, &ok_sh);
        if (!fine) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
      }
      if (!__shfl_sync(0xffffffffu, fine, 0)) break;
    }
    if (lane == 0) tc_load_drain(br, gl);
  } else {
    for (uint32_t i = 0;; ++i) {
      const int ur = uq_pop(br, i, lane, wait_ns, &ok_sh);
      if (ur < 0) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      if (ur >= total) break;
      int s, ncol, I, J, nk, k0, nku;
      decode(ur, s, ncol, I, J, nk, k0, nku);
      float acc[TM];
      if (!tc_drain<tmem_bufs<MODE>()>(nku, br, tmem, warp, lane, gc, acc, wait_ns, &ok_sh)) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      const int li = I * TM + 32 * warp + lane;   // tile row owned by this thread
      if (li < ncol) {
        const int64_t gi = 3 * (int64_t)qidx[(size_t)s * m + li / 3] + li % 3;
        float* Wrow = WH + gi * ldw;
        // four columns at a time: one 16-byte atomic add when they are four
        // consecutive, aligned entries of W_H's row (consecutive contacts, e.g.
        // a front every contact reaches), else one add per entry
#pragma unroll
        for (int j0 = 0; j0 < TM; j0 += 4) {
          int64_t g[4];
          bool ok[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int lj = J * TM + j0 + k;
            ok[k] = lj < ncol && li <= lj;
            g[k] = ok[k] ? 3 * (int64_t)qidx[(size_t)s * m + lj / 3] + lj % 3 : 0;
          }
          const bool vec = ok[0] && ok[1] && ok[2] && ok[3] && g[1] == g[0] + 1 && g[2] == g[0] + 2 &&
                           g[3] == g[0] + 3 && (((uintptr_t)(Wrow + g[0])) & 15) == 0;
          if (vec) {
            atomicAdd((float4*)(Wrow + g[0]), make_float4(acc[j0], acc[j0 + 1], acc[j0 + 2], acc[j0 + 3]));
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (ok[k]) atomicAdd(Wrow + g[k], acc[j0 + k]);
          }
        }
      }
    }
  }
  tc_teardown<tmem_bufs<MODE>()>(tmem, br);
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_contract_tc(const int* __restrict__ plan, int* counter, int ns, const int* __restrict__ level_list,
                  const int* __restrict__ super_ptr, const int* __restrict__ qcount, const int* __restrict__ qidx,
                  const int64_t* __restrict__ boff, int m, const unsigned char* __restrict__ pk, float* WH,
                  int64_t ldw, int* dev_err, int cache_plan, const int* __restrict__ tsplit_p, uint64_t wait_ns) {
  pdl_entry();
  d_contract_tc<MODE>(own_block(), plan, counter, ns, level_list, super_ptr, qcount, qidx, boff, m, pk, WH, ldw,
                      dev_err, cache_plan, tsplit_p, wait_ns);
}

template <int MODE>
struct contract_tc_body {
  static constexpr int threads = TC_THREADS, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_contract_tc<MODE>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_contract_tc<MODE>(vb, a...);
  }
};

// Forward-solve product of the wide fronts of one level (3xTF32): persistent
// CTAs take units (supernode s, 128-row tile rt of its w + r front rows,
// 128-column tile ct of its 3|Q_s| columns) from the level's counter, largest
// fronts first, and form out = G_s[rt rows, :] F_top[:, ct columns]; rows < w
// store X_s = out, the update rows take U_s -= out.
__device__ __forceinline__ void d_front_gemm_tc(const VB& vb, const int* __restrict__ plan, int pa, int pb,
                                                int* counter, const int* __restrict__ level_list,
                                                const int* __restrict__ super_ptr,
                                                const int64_t* __restrict__ rowpat_ptr,
                                                const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                                                const int64_t* __restrict__ goff,
                                                const unsigned char* __restrict__ gpk,
                                                const int64_t* __restrict__ boff,
                                                const unsigned char* __restrict__ fpk, float* X, int64_t ldx,
                                                int* dev_err, const int* __restrict__ gsplit_p, uint64_t wait_ns) {
  constexpr int MODE = ICR_CONTRACT_TF32X3;
  constexpr int BLK = TcTraits<MODE>::PARTS * tile_bytes<MODE>();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) TcBars br;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int ok_sh;   // cleared by the side of the pipeline whose wait ran out
  const int u0 = plan[pa], total = plan[pb] - u0;
  if ((int)vb.bx >= total) return;   // uniform: before any allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gsplit = *gsplit_p;
  tc_setup<tmem_bufs<MODE>()>(&tmem_base, br, &ok_sh);
  const uint32_t tmem = tmem_base;
  uint32_t gl = 0, gm = 0, gc = 0;
  // unit ur (counter value): supernode s, 128-row tile rt, 128-column tile ct, K part [k0, k0 + nku)
  struct Unit {
    int s, ncol, w, nrows, nk, nsk, rt, ct, k0, nku;
  };
  auto decode = [&](int ur) {
    Unit x;
    const int u = u0 + total - 1 - ur;
    const int pos = find_unit(plan, pa, pb, u);
    x.s = level_list[pos];
    x.ncol = 3 * qcount[x.s];
    const int nJ = (x.ncol + TM - 1) / TM;
    x.w = super_ptr[x.s + 1] - super_ptr[x.s];
    x.nrows = x.w + (int)(rowpat_ptr[x.s + 1] - rowpat_ptr[x.s]);
    x.nk = (x.w + KT - 1) / KT;
    x.nsk = tc_parts(gsplit, x.nk);   // unit = (tile, K part)
    const int local = (u - plan[pos]) / x.nsk, kc = (u - plan[pos]) % x.nsk;
    x.rt = local / nJ;
    x.ct = local % nJ;
    x.k0 = kc * x.nk / x.nsk;
    x.nku = (kc + 1) * x.nk / x.nsk - x.k0;
    return x;
  };
  if (warp == 4) {
    if (lane == 0) {
      for (uint32_t i = 0;; ++i) {
        const int ur = ok_sh ? atomicAdd(counter, 1) : total;   // a pipeline that gave up takes no more
        if (!uq_push(br, i, ur < total ? ur : total, wait_ns, &ok_sh)) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
          break;
        }
        if (ur >= total) break;
        const Unit x = decode(ur);
        if (!tc_mma<MODE>(false, x.nku, smem, br, tmem, gm, gc, wait_ns, &ok_sh)) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
          break;
        }
      }
    }
  } else if (warp == 5) {   // the loader
    for (uint32_t i = 0;; ++i) {
      const int ur = uq_pop(br, i, lane, wait_ns, &ok_sh);
      if (ur < 0) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      if (ur >= total) break;
      int fine = 1;
      if (lane == 0) {
        const Unit x = decode(ur);
        fine = tc_load<MODE>(gpk + (goff[x.s] + (int64_t)x.rt * x.nk + x.k0) * BLK,
                             fpk + (boff[x.s] + (int64_t)x.ct * x.nk + x.k0) * BLK, false, x.nku, smem, br, gl,
                             wait_ns, &ok_sh);
        if (!fine) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
      }
      if (!__shfl_sync(0xffffffffu, fine, 0)) break;
    }
    if (lane == 0) tc_load_drain(br, gl);
  } else {
    for (uint32_t i = 0;; ++i) {
      const int ur = uq_pop(br, i, lane, wait_ns, &ok_sh);
      if (ur < 0) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      if (ur >= total) break;
      const Unit x = decode(ur);
      float acc[TM];
      if (!tc_drain<tmem_bufs<MODE>()>(x.nku, br, tmem, warp, lane, gc, acc, wait_ns, &ok_sh)) {
        if (lane == 0) {
          ok_sh = 0;
          atomicExch(dev_err, 1);
        }
        break;
      }
      const int row = x.rt * TM + 32 * warp + lane;   // front row owned by this thread
      const int cmax = x.ncol - x.ct * TM;            // columns of this tile inside the front
      if (row < x.nrows && x.nsk > 1) {
        // K parts add up: X_s (zeroed when F_top was packed) += out, U_s -= out
        float* F = X + (fr_ptr[x.s] + row) * ldx + x.ct * TM;
        const float sg = row < x.w ? 1.f : -1.f;
#pragma unroll
        for (int c0j = 0; c0j < TM; c0j += 4) {
          if (c0j >= cmax) break;
          if (c0j + 4 <= cmax) {
            atomicAdd((float4*)(F + c0j),
                      make_float4(sg * acc[c0j], sg * acc[c0j + 1], sg * acc[c0j + 2], sg * acc[c0j + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (c0j + j < cmax) atomicAdd(F + c0j + j, sg * acc[c0j + j]);
          }
        }
      } else if (row < x.nrows) {
        float* F = X + (fr_ptr[x.s] + row) * ldx + x.ct * TM;
#pragma unroll
        for (int c0j = 0; c0j < TM; c0j += 4) {
          if (c0j >= cmax) break;
          if (c0j + 4 <= cmax) {
            float4* F4 = (float4*)(F + c0j);
            float4 o = make_float4(acc[c0j], acc[c0j + 1], acc[c0j + 2], acc[c0j + 3]);
            if (row >= x.w) {
              const float4 y = *F4;
              o = make_float4(y.x - o.x, y.y - o.y, y.z - o.z, y.w - o.w);
            }
            *F4 = o;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (c0j + j < cmax) F[c0j + j] = row < x.w ? acc[c0j + j] : F[c0j + j] - acc[c0j + j];
          }
        }
      }
    }
  }
  tc_teardown<tmem_bufs<MODE>()>(tmem, br);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_front_gemm_tc(const int* __restrict__ plan, int pa, int pb, int* counter, const int* __restrict__ level_list,
                    const int* __restrict__ super_ptr, const int64_t* __restrict__ rowpat_ptr,
                    const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                    const int64_t* __restrict__ goff, const unsigned char* __restrict__ gpk,
                    const int64_t* __restrict__ boff, const unsigned char* __restrict__ fpk, float* X, int64_t ldx,
                    int* dev_err, const int* __restrict__ gsplit_p, uint64_t wait_ns) {
  pdl_entry();
  d_front_gemm_tc(own_block(), plan, pa, pb, counter, level_list, super_ptr, rowpat_ptr, fr_ptr, qcount, goff, gpk,
                  boff, fpk, X, ldx, dev_err, gsplit_p, wait_ns);
}

struct front_gemm_tc_body {
  static constexpr int threads = TC_THREADS, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_front_gemm_tc; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_front_gemm_tc(vb, a...);
  }
};

// dynamic shared memory of a tensor-core CTA: the ring, padded so that at most
// two CTAs share an SM (2 x 256 TMEM columns fill its 512)
template <int MODE>
static size_t tc_smem_bytes() {
  return std::max<size_t>(STAGES * 2 * (size_t)(TcTraits<MODE>::PARTS * tile_bytes<MODE>()), 100 * 1024);
}

template <int MODE>
int contract_tc_T(Scene* s) {
  const int m = s->m, ns = s->ns;
  const int64_t nr = 3 * (int64_t)m;
  // the ring, then the contraction list's prefix sums (up to 24 KiB of them)
  const size_t ring = (size_t)STAGES * 2 * TcTraits<MODE>::PARTS * tile_bytes<MODE>();
  const int cache_plan = (ns + 1) * (int)sizeof(int) <= 24 * 1024;
  const size_t smem = std::max(tc_smem_bytes<MODE>(), ring + (cache_plan ? (size_t)(ns + 1) * sizeof(int) : 0));
  static SmemLimit lim;
  static DevInt occ_dev;
  const int dev = s->ctx->device;
  cudaError_t e0 = ensure_smem(k_contract_tc<MODE>, lim, dev, (int)smem);
  if (e0 != cudaSuccess) return cuda_fail(e0, "cudaFuncSetAttribute(k_contract_tc)");
  int occ = occ_dev.get(dev);
  if (occ == 0) {
    e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_contract_tc<MODE>, TC_THREADS, smem);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_contract_tc)");
    occ = std::max(1, std::min(occ, 2));   // 2 x 256 TMEM columns fill an SM's 512
    occ_dev.put(dev, occ);
  }
  const int* plan = (const int*)s->plan.p;
  const int nsm = s->ctx->sm_count;
  const int tmax = s->tc_tmax;
  const int64_t ub_pack = (int64_t)ns * tmax * ((s->wmax + KT - 1) / KT);
  PDL("k_pack_tc", pack_tc_body<MODE>, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ub_pack, 4 * nsm)), 256, 0, s->ctx->stream,
      plan + PLAN_PACK * (ns + 1), 0, ns, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
      (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, (const int64_t*)s->tc_boff.p, (const float*)s->X.p, 0,
      s->ldx, (unsigned char*)s->Ypk.p, (float*)nullptr, (const int*)nullptr);
  const int64_t ub_tc = (int64_t)ns * tmax * (tmax + 1) / 2 * TC_MAX_SPLIT;
  const int nlev = (int)s->levels.size();
  PDL("k_contract_tc", contract_tc_body<MODE>, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ub_tc, (int64_t)occ * nsm)), TC_THREADS, smem, s->ctx->stream,
      plan + PLAN_TC * (ns + 1), (int*)plan + PLAN_LISTS * (ns + 1) + PLAN_CNT_TC, ns, (const int*)s->level_list.p,
      (const int*)s->super_ptr.p, (const int*)s->qcount.p, (const int*)s->qidx.p, (const int64_t*)s->tc_boff.p, m,
      (const unsigned char*)s->Ypk.p, (float*)s->WH.p, nr, (int*)s->dev_err.p, cache_plan,
      plan + PLAN_LISTS * (ns + 1) + 2 + 2 * nlev, s->ctx->wait_ns);
  return ICR_OK;
}

}  // namespace

int launch_contract_tc(Scene* s, int mode) {
  switch (mode) {
    case ICR_CONTRACT_TF32X3: return contract_tc_T<ICR_CONTRACT_TF32X3>(s);
    case ICR_CONTRACT_TF32: return contract_tc_T<ICR_CONTRACT_TF32>(s);
    case ICR_CONTRACT_BF16: return contract_tc_T<ICR_CONTRACT_BF16>(s);
    default: set_error("launch_contract_tc: mode %d is not a tensor-core mode", mode); return ICR_EINVAL;
  }
}

int launch_pack_g(Scene* s, const int32_t* blocks, int nblocks) {
  if (nblocks == 0) return ICR_OK;
  k_pack_g<<<(unsigned)std::min(nblocks, 8 * s->ctx->sm_count), 256, 0, s->ctx->stream>>>(
      blocks, nblocks, (const int*)s->super_ptr.p, (const int64_t*)s->rowpat_ptr.p, (const int64_t*)s->val_ptr.p,
      (const int64_t*)s->gpk_off.p, (const float*)s->G.p, (unsigned char*)s->Gpk.p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_pack_g");
  return ICR_OK;
}

int launch_front_gemm_tc(Scene* s, int level) {
  constexpr int MODE = ICR_CONTRACT_TF32X3;
  const size_t smem = tc_smem_bytes<MODE>();
  static SmemLimit lim;
  const cudaError_t e0 = ensure_smem(k_front_gemm_tc, lim, s->ctx->device, (int)smem);
  if (e0 != cudaSuccess) return cuda_fail(e0, "cudaFuncSetAttribute(k_front_gemm_tc)");
  const Level& lv = s->levels[level];
  const int ns = s->ns, pa = lv.first, pb = lv.first + lv.count;
  int* plan = (int*)s->plan.p;
  const int nsm = s->ctx->sm_count;
  const int tmax = s->tc_tmax;
  const int64_t ub_pack = (int64_t)lv.count * tmax * ((lv.wmax + KT - 1) / KT);
  PDL("k_pack_tc", pack_tc_body<MODE>, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ub_pack, 4 * nsm)), 256, 0, s->ctx->stream,
      plan + PLAN_FPACK * (ns + 1), pa, pb, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
      (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, (const int64_t*)s->tc_boff.p, (const float*)s->Ftop.p, 1,
      s->ldx, (unsigned char*)s->Ypk.p, (float*)s->X.p,
      (const int*)plan + PLAN_LISTS * (ns + 1) + 2 + (int)s->levels.size() + level);
  const int64_t ub = (int64_t)lv.count * ((lv.wmax + lv.rmax + TM - 1) / TM) * tmax * TC_MAX_SPLIT;
  const int nlev = (int)s->levels.size();
  PDL("k_front_gemm_tc", front_gemm_tc_body, (unsigned)std::max<int64_t>(1, std::min<int64_t>(ub, nsm)), TC_THREADS, smem, s->ctx->stream,
      plan + PLAN_GTC * (ns + 1), pa, pb, plan + PLAN_LISTS * (ns + 1) + PLAN_CNT_GTC + level,
      (const int*)s->level_list.p, (const int*)s->super_ptr.p, (const int64_t*)s->rowpat_ptr.p,
      (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, (const int64_t*)s->gpk_off.p,
      (const unsigned char*)s->Gpk.p, (const int64_t*)s->tc_boff.p, (const unsigned char*)s->Ypk.p, (float*)s->X.p,
      s->ldx, (int*)s->dev_err.p, plan + PLAN_LISTS * (ns + 1) + 2 + nlev + level, s->ctx->wait_ns);
  return ICR_OK;
}

}  // namespace icr
