// Tensor-core (tcgen05) contraction W_H += Y_s^T Y_s for the supernodes whose
// scaled front Y_s = D_s^-1/2 X_s has at least TC_MIN_COLS columns
// (Eq. "schur complemnt reformulated": W_H = H A^-1 H^T = X^T D^-1 X).
//
// Block (128 x 128 output tile pair I <= J, supernode s), 4 warps:
//   * the K dimension (the w_s rows of Y_s) is streamed in 32-row chunks
//     through two shared-memory stages; all threads convert their share of
//     the chunk to the MMA operand type and store it in the K-major
//     core-matrix layout (8 rows x 16 bytes per core matrix, no swizzle);
//   * one thread issues tcgen05.mma (M = N = 128) into a 128-column TMEM
//     accumulator and commits to the stage's mbarrier, which releases the
//     stage two chunks later;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31, i.e. the tile's rows) and adds the upper-triangle
//     entries into W_H.
// Modes: TF32X3 splits every operand into a TF32 part and a TF32 remainder and
// accumulates hi*hi + hi*lo + lo*hi (FP32-level error); TF32 and BF16 use one
// rounded part.  Every mbarrier wait is bounded; a wait that runs out sets the
// scene's device error word and the block skips its epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "icr_internal.h"

namespace icr {
namespace {

constexpr int TM = 128;   // output tile (M = N)
constexpr int KT = 32;    // K rows per stage
constexpr long long WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
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
template <int MODE>
__host__ __device__ constexpr int stage_bytes() {
  return 2 * TcTraits<MODE>::PARTS * tile_bytes<MODE>();   // A and B parts
}

// byte offset of element (r, k) of a K-major TM x KT tile: core matrix (r/8, k/C)
// with C elements per 16 bytes; core matrices contiguous along K, 8-row groups
// KT/C core matrices apart
template <int EB>
__device__ __forceinline__ int tile_off(int r, int k) {
  constexpr int C = 16 / EB;
  constexpr int SBO = (KT / C) * 128;
  return (r >> 3) * SBO + (k / C) * 128 + (r & 7) * 16 + (k % C) * EB;
}

template <int MODE>
__global__ void __launch_bounds__(128, 1)
    k_contract_tc(int ntc, int min_cols, const int* __restrict__ super_ptr, const int64_t* __restrict__ fr_ptr,
                  const int* __restrict__ qcount, const int* __restrict__ qidx, int m, const float* __restrict__ Y,
                  int64_t ldx, float* WH, int64_t ldw, int* dev_err) {
  using TR = TcTraits<MODE>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  const int s = blockIdx.y;
  int rem = blockIdx.x, I = 0;
  while (rem >= ntc - I) {
    rem -= ntc - I;
    ++I;
  }
  const int J = I + rem;
  const int ncol = 3 * qcount[s];
  if (ncol < min_cols || J * TM >= ncol) return;   // uniform: before any allocation
  const int c0 = super_ptr[s], w = super_ptr[s + 1] - c0;
  const float* Ys = Y + fr_ptr[s] * ldx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&bars[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&bars[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc(TR::TYPE);
  constexpr int SBO = (KT / (16 / TR::EB)) * 128;
  const int nk = (w + KT - 1) / KT;
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    unsigned char* st = smem + buf * stage_bytes<MODE>();
    unsigned char* sA = st;                                   // PARTS tiles
    unsigned char* sB = st + TR::PARTS * tile_bytes<MODE>();  // PARTS tiles
    if (kt >= 2 && !mbar_wait(smem_u32(&bars[buf]), ((kt - 2) >> 1) & 1)) {
      ok = false;
      break;
    }
    // stage: element (r, k) of A is Y[k0 + k, I*TM + r], of B is Y[k0 + k, J*TM + r]
    const int k0 = kt * KT;
    for (int e = tid; e < TM * KT; e += 128) {
      const int k = e / TM, r = e % TM;
      const bool kin = k0 + k < w;
      const int ca = I * TM + r, cb = J * TM + r;
      const float a = (kin && ca < ncol) ? Ys[(int64_t)(k0 + k) * ldx + ca] : 0.f;
      const float b = (kin && cb < ncol) ? Ys[(int64_t)(k0 + k) * ldx + cb] : 0.f;
      const int o = tile_off<TR::EB>(r, k);
      if constexpr (MODE == ICR_CONTRACT_BF16) {
        const unsigned short ah = __bfloat16_as_ushort(__float2bfloat16_rn(a));
        const unsigned short bh = __bfloat16_as_ushort(__float2bfloat16_rn(b));
        *(unsigned short*)(sA + o) = ah;
        *(unsigned short*)(sB + o) = bh;
      } else {
        const uint32_t ah = to_tf32(a), bh = to_tf32(b);
        *(uint32_t*)(sA + o) = ah;
        *(uint32_t*)(sB + o) = bh;
        if constexpr (TR::PARTS == 2) {
          *(uint32_t*)(sA + tile_bytes<MODE>() + o) = to_tf32(a - __uint_as_float(ah));
          *(uint32_t*)(sB + tile_bytes<MODE>() + o) = to_tf32(b - __uint_as_float(bh));
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
      for (int kk = 0; kk < KT / TR::KMMA; ++kk) {
        const uint32_t off = kk * 256;   // two core matrices along K per MMA
#pragma unroll
        for (int term = 0; term < (TR::PARTS == 2 ? 3 : 1); ++term) {
          const int ai = term == 2 ? 1 : 0, bi = term == 1 ? 1 : 0;
          const uint64_t ad = smem_desc(smem_u32(sA + ai * tile_bytes<MODE>()) + off, 128, SBO);
          const uint64_t bd = smem_desc(smem_u32(sB + bi * tile_bytes<MODE>()) + off, 128, SBO);
          const uint32_t acc = (kt > 0 || kk > 0 || term > 0) ? 1u : 0u;
          if constexpr (MODE == ICR_CONTRACT_BF16)
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          else
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                    tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&bars[buf])));
    }
  }
  // all MMAs done: the last commit tracks every earlier MMA of this thread
  if (ok && nk > 0 && !mbar_wait(smem_u32(&bars[(nk - 1) & 1]), ((nk - 1) >> 1) & 1)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (ok && nk > 0) {
    const int li = I * TM + 32 * warp + lane;   // tile row owned by this thread (TMEM lane)
    const bool row_ok = li < ncol;
    const int64_t gi = row_ok ? 3 * (int64_t)qidx[(size_t)s * m + li / 3] + li % 3 : 0;
    for (int c0j = 0; c0j < TM; c0j += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0j;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
      if (!row_ok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int lj = J * TM + c0j + j;
        if (lj >= ncol || li > lj) continue;
        const int64_t gj = 3 * (int64_t)qidx[(size_t)s * m + lj / 3] + lj % 3;
        atomicAdd(&WH[gi * ldw + gj], __uint_as_float(v[j]));
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(dev_err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TM));
}

template <int MODE>
int contract_tc_T(Scene* s, int min_cols) {
  const int m = s->m;
  const int64_t nr = 3 * (int64_t)m;
  const int ntc = (int)((nr + TM - 1) / TM);
  const int npairs = ntc * (ntc + 1) / 2;
  const size_t smem = 2 * (size_t)stage_bytes<MODE>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_contract_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_contract_tc)");
    attr = true;
  }
  k_contract_tc<MODE><<<dim3(npairs, s->ns), 128, smem, s->ctx->stream>>>(
      ntc, min_cols, (const int*)s->super_ptr.p, (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p,
      (const int*)s->qidx.p, m, (const float*)s->X.p, s->ldx, (float*)s->WH.p, nr, (int*)s->dev_err.p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_contract_tc");
  ++s->launches;
  return ICR_OK;
}

}  // namespace

int launch_contract_tc(Scene* s, int mode, int min_cols) {
  switch (mode) {
    case ICR_CONTRACT_TF32X3: return contract_tc_T<ICR_CONTRACT_TF32X3>(s, min_cols);
    case ICR_CONTRACT_TF32: return contract_tc_T<ICR_CONTRACT_TF32>(s, min_cols);
    case ICR_CONTRACT_BF16: return contract_tc_T<ICR_CONTRACT_BF16>(s, min_cols);
    default: set_error("launch_contract_tc: mode %d is not a tensor-core mode", mode); return ICR_EINVAL;
  }
}

}  // namespace icr
