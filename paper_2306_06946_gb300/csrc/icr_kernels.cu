// libicr device side: the kernels of the constraint-resolution hot path and
// their launchers.  Every kernel is templated on the storage / arithmetic type
// T (float or double); D^-1 and D^-1/2 are always applied in FP64.
//
// Build of W_H = H A^-1 H^T = X^T D^-1 X, X = L^-1 H^T
// (Eq. "schur complemnt reformulated" with A = L D L^T):
//   a1  k_reach_*      which contacts' columns of H^T reach each supernode
//                      (etree ancestors of the supernodes owning their nodes)
//   a2  k_assemble     one thread per front element: its H^T entry plus the
//                      children's update entries (extend-add as a gather)
//       k_front_gemm   X_s = L_ss^-1 F_top and U_s = F_R - L_Rs L_ss^-1 F_top,
//                      one register-tiled product with the precomputed
//                      G_s = [L_ss^-1; L_Rs L_ss^-1] (per level, all tiles)
//   a3+a4 k_contract   W_H += Y_s^T Y_s with Y_s = D_s^-1/2 X_s (FP64 scaling)
// Newton iteration (Alg. 3):
//   a6  k_update_W     W = C W_H C^T, one 3x3 block pair per thread
//   a7  k_pgs          projected Gauss-Seidel (Eq. "PGS"), one CTA
//       k_pgs_residual FP64 complementarity / cone residuals
//   a8  k_prox         p += W_H C^T lambda~, u += C^T lambda~ (k_prox_u and
//                      k_prox_p when C^T lambda~ does not fit shared memory)
// End of step:
//   a9  k_xu, k_bsolve dq = L^-T D^-1 X u, the backward solve as
//                      dq_s = G_s^T [y_s; -dq_R] per level, top-down
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "icr_internal.h"

namespace icr {

// checks a launch and counts it in the scene (every launcher has `s` in scope)
#define LAUNCH_OK(where)                                  \
  do {                                                    \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, where);   \
    ++s->launches;                                        \
  } while (0)

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int TCC = 32;            // contacts per column tile of the forward solve
static constexpr int TCOLS = 3 * TCC;     // columns per tile
static constexpr int KB = 32;             // diagonal block of the triangular solves
static constexpr int SOLVE_THREADS = 192; // 2 x 96 columns
static constexpr int CT = 64;             // contraction output tile
static constexpr int CK_ = 16;            // contraction k-chunk
static constexpr int TC_MIN_COLS = 64;    // fronts this wide use the tensor-core contraction


template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// The Newton loop of a device-resident step has ended (icr_params.newton_tol):
// the kernels of the remaining iterations return at entry.  NULL outside it.
__device__ __forceinline__ bool newton_stopped(const int* stop) { return stop && *(const volatile int*)stop; }

__device__ __forceinline__ int lower_bound_dev(const int* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------ a1 reach
// One thread per (contact, node): mark the contact in every supernode on the
// etree path from the node's supernode to the root.  A thread stops at the
// first supernode already marked for its contact: whoever marked it walks on.
__device__ __forceinline__ void d_reach_mark(const VB& vb, const int* __restrict__ nodes, int m,
                                             const int* __restrict__ node_super, const int* __restrict__ parent,
                                             int ns, uint32_t* bitmap, int words) {
  int t = vb.bx * blockDim.x + threadIdx.x;
  if (t >= 4 * m) return;
  int a = t >> 2;
  int s = node_super[nodes[t]];
  uint32_t bit = 1u << (a & 31);
  int w = a >> 5;
  for (int guard = 0; s >= 0 && guard < ns; ++guard) {
    uint32_t old = atomicOr(&bitmap[(size_t)s * words + w], bit);
    if (old & bit) break;
    s = parent[s];
  }
}

__global__ void k_reach_mark(const int* __restrict__ nodes, int m, const int* __restrict__ node_super,
                             const int* __restrict__ parent, int ns, uint32_t* bitmap, int words) {
  pdl_entry();
  d_reach_mark(own_block(), nodes, m, node_super, parent, ns, bitmap, words);
}

struct reach_mark_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_reach_mark; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_reach_mark(vb, a...);
  }
};

// One block per supernode: count its contacts, prefix the per-word counts and
// list the contacts in ascending order.
__device__ __forceinline__ void d_reach_rows(const VB& vb, const uint32_t* __restrict__ bitmap, int words, int m,
                                             int* wprefix, int* qcount, int* qidx) {
  extern __shared__ int sh[];
  int s = vb.bx;
  int w = threadIdx.x;
  uint32_t bits = (w < words) ? bitmap[(size_t)s * words + w] : 0u;
  int c = __popc(bits);
  sh[w] = c;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int v = (w >= off) ? sh[w - off] : 0;
    __syncthreads();
    sh[w] += v;
    __syncthreads();
  }
  int excl = sh[w] - c;
  if (w < words) wprefix[(size_t)s * words + w] = excl;
  if (w == blockDim.x - 1) qcount[s] = sh[w];
  int* out = qidx + (size_t)s * m + excl;
  while (bits) {
    int b = __ffs(bits) - 1;
    *out++ = 32 * w + b;
    bits &= bits - 1;
  }
}

__global__ void k_reach_rows(const uint32_t* __restrict__ bitmap, int words, int m, int* wprefix, int* qcount,
                             int* qidx) {
  pdl_entry();
  d_reach_rows(own_block(), bitmap, words, m, wprefix, qcount, qidx);
}

struct reach_rows_body {
  static constexpr int threads = 1024, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_reach_rows; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_reach_rows(vb, a...);
  }
};

// Position of each of a supernode's contacts in its parent's contact list.
__device__ __forceinline__ void d_reach_parentpos(const VB& vb, const uint32_t* __restrict__ bitmap,
                                                  const int* __restrict__ wprefix, int words, int m,
                                                  const int* __restrict__ parent, const int* __restrict__ qcount,
                                                  const int* __restrict__ qidx, int* qpos) {
  int s = vb.by;
  int j = vb.bx * blockDim.x + threadIdx.x;
  if (j >= qcount[s]) return;
  int p = parent[s];
  int a = qidx[(size_t)s * m + j];
  int pos = -1;
  if (p >= 0) {
    int w = a >> 5;
    pos = wprefix[(size_t)p * words + w] + __popc(bitmap[(size_t)p * words + w] & ((1u << (a & 31)) - 1u));
  }
  qpos[(size_t)s * m + j] = pos;
}

__global__ void k_reach_parentpos(const uint32_t* __restrict__ bitmap, const int* __restrict__ wprefix, int words,
                                  int m, const int* __restrict__ parent, const int* __restrict__ qcount,
                                  const int* __restrict__ qidx, int* qpos) {
  pdl_entry();
  d_reach_parentpos(own_block(), bitmap, wprefix, words, m, parent, qcount, qidx, qpos);
}

struct reach_parentpos_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_reach_parentpos; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_reach_parentpos(vb, a...);
  }
};

// For every supernode c: the local position in c's contact list of each
// contact of its parent's list (-1 when the contact does not reach c).
__device__ __forceinline__ void d_reach_inv(const VB& vb, int m, const int* __restrict__ parent,
                                            const int* __restrict__ qcount, const int* __restrict__ qpos, int* qinv) {
  const int c = vb.bx;
  const int p = parent[c];
  if (p < 0) return;
  const int np = qcount[p], nc = qcount[c];
  int* inv = qinv + (size_t)c * m;
  for (int k = threadIdx.x; k < np; k += blockDim.x) inv[k] = -1;
  __syncthreads();
  for (int j = threadIdx.x; j < nc; j += blockDim.x) inv[qpos[(size_t)c * m + j]] = j;
}

__global__ void k_reach_inv(int m, const int* __restrict__ parent, const int* __restrict__ qcount,
                            const int* __restrict__ qpos, int* qinv) {
  pdl_entry();
  d_reach_inv(own_block(), m, parent, qcount, qpos, qinv);
}

struct reach_inv_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_reach_inv; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_reach_inv(vb, a...);
  }
};

// ------------------------------------------------------------------ a2 forward solve
// The front of supernode s has w + r rows (its DOF columns, then R_s) and
// 3 |Q_s| columns (the contacts of Q_s in ascending order, 3 axes each).
// Its first w rows are assembled in Ftop (indexed by DOF row), the last r rows
// in the front itself; after the solve the front holds X_s then U_s:
//   X_s = L_ss^-1 F_top,  U_s = F_R - (L_Rs L_ss^-1) F_top,
// one dense product with the precomputed operator G_s = [L_ss^-1; L_Rs L_ss^-1].

// Block (supernode s of the level, 4-row tile of its front, 32-contact tile),
// one thread per front element: the H^T entry plus the children's update
// entries listed for that row (extend-add as a gather, children in ascending
// order).  Rows < w go to Ftop, rows >= w to the front's update rows.
static constexpr int AR = 4;          // threads per column of an assembly block
static constexpr int ASM_ROWS = 16;   // front rows per assembly unit (AR threads, 4 rows each)


__device__ __forceinline__ int cdiv(int a, int b) { return (a + b - 1) / b; }

// The position p in [lo, hi) with P[p] <= u < P[p + 1], for a non-decreasing
// prefix array P with P[lo] <= u < P[hi]: the supernode that owns work unit u.
__device__ __forceinline__ int find_pos(const int* __restrict__ P, int lo, int hi, int u) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P[mid] <= u)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// find_pos by the whole block, for kernels with few, large units: thread t
// tests position lo + t (+ multiples of the block size), one round of loads
// instead of log2 dependent ones.  Block-uniform call; sh is a shared int.
__device__ __forceinline__ int block_find_pos(const int* __restrict__ P, int lo, int hi, int u, int* sh) {
  const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int p = lo + tid; p < hi; p += nt)
    if (P[p] <= u && u < P[p + 1]) *sh = p;   // exactly one p: P non-decreasing, P[lo] <= u < P[hi]
  __syncthreads();
  const int r = *sh;
  __syncthreads();   // sh is reused by the next search
  return r;
}

// Work units per supernode for the lists of one build (PlanList order):
// assembly tiles; front-GEMM tiles, on the tensor cores (with their packed
// F_top blocks) for fronts at least TC_GEMM_MIN_W wide with TC_GEMM_MIN_COLS
// columns when tc_gemm is set and the supernode's level runs on the tensor
// cores (tc_super), on CUDA cores otherwise; SIMT contraction tile
// pairs of fronts narrower than simt_max columns; packed operand blocks and
// tensor-core tile pairs of fronts at least tc_min columns wide.  Tensor-core
// units are split over K into tc_parts(gsplit or tsplit, K blocks) parts
// (gsplit: the level's front GEMM, tsplit: the contraction; 0 counts the
// unsplit tiles).
__device__ __forceinline__ void plan_counts(int s, const int* __restrict__ super_ptr,
                                            const int64_t* __restrict__ rowpat_ptr, const int* __restrict__ qcount,
                                            int simt_max, int tc_min, int tc_gemm,
                                            const unsigned char* __restrict__ tc_super, int gsplit, int tsplit,
                                            int* c) {
  const int q = qcount[s];
  const int w = super_ptr[s + 1] - super_ptr[s];
  const int nrows = w + (int)(rowpat_ptr[s + 1] - rowpat_ptr[s]);
  const int nt = cdiv(q, TCC);
  const int ncol = 3 * q;
  const bool tcg = tc_gemm && tc_super[s] == FWD_TC && q > 0 && w >= TC_GEMM_MIN_W && ncol >= TC_GEMM_MIN_COLS;
  c[PLAN_ASM] = cdiv(nrows, ASM_ROWS) * nt;
  c[PLAN_GEMM] = tcg ? 0 : cdiv(nrows, tc_super[s] == FWD_SIMT_SHORT ? GR_SHORT : GR_LONG) * nt;
  const int nkb = cdiv(w, TC_KT);   // K blocks of a tensor-core unit
  c[PLAN_GTC] = tcg ? cdiv(nrows, TC_TILE) * cdiv(ncol, TC_TILE) * tc_parts(gsplit, nkb) : 0;
  c[PLAN_FPACK] = tcg ? cdiv(ncol, TC_TILE) * cdiv(w, TC_KT) : 0;
  const int ns_ = cdiv(ncol, CT);
  c[PLAN_SIMT] = (q > 0 && ncol < simt_max) ? ns_ * (ns_ + 1) / 2 : 0;
  const int nI = cdiv(ncol, TC_TILE);
  const bool tc = q > 0 && ncol >= tc_min;
  c[PLAN_PACK] = tc ? nI * cdiv(w, TC_KT) : 0;
  c[PLAN_TC] = tc ? nI * (nI + 1) / 2 * tc_parts(tsplit, nkb) : 0;
}

// One block: exclusive prefix sums of the per-supernode unit counts over the
// positions of level_list, and the scheduling counters reset to zero.  First
// the K split factors: a level's tensor-core front GEMM, and the
// tensor-core contraction, with fewer tiles than target (one per SM) split
// their units over K into about target / tiles parts (plan counters area,
// after the 2 + nlev counters: nlev level factors, then the contraction's).
__device__ __forceinline__ void d_plan(const VB& vb, int ns, const int* __restrict__ level_list,
                                       const int* __restrict__ super_ptr, const int64_t* __restrict__ rowpat_ptr,
                                       const int* __restrict__ qcount, int simt_max, int tc_min, int tc_gemm,
                                       const unsigned char* __restrict__ tc_super,
                                       const int* __restrict__ level_first, int nlev, int target, int* plan) {
  __shared__ int wsum[PLAN_LISTS][32];
  __shared__ int tiles[PLAN_MAX_LEV + 1];   // unsplit tensor-core tiles per level; [PLAN_MAX_LEV]: contraction
  __shared__ int split[PLAN_MAX_LEV + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int per = cdiv(ns, blockDim.x);
  const int p0 = min(ns, tid * per), p1 = min(ns, p0 + per);
  const int nl = min(nlev, PLAN_MAX_LEV);
  for (int l = tid; l <= PLAN_MAX_LEV; l += blockDim.x) tiles[l] = 0;
  __syncthreads();
  int lv0 = 0;   // level of position p0
  while (lv0 + 1 < nlev && level_first[lv0 + 1] <= p0) ++lv0;
  for (int p = p0, lv = lv0; p < p1; ++p) {
    while (lv + 1 < nlev && level_first[lv + 1] <= p) ++lv;
    int c[PLAN_LISTS];
    plan_counts(level_list[p], super_ptr, rowpat_ptr, qcount, simt_max, tc_min, tc_gemm, tc_super, 1, 1, c);
    if (c[PLAN_GTC] && lv < nl) atomicAdd(&tiles[lv], c[PLAN_GTC]);
    if (c[PLAN_TC]) atomicAdd(&tiles[PLAN_MAX_LEV], c[PLAN_TC]);
  }
  __syncthreads();
  for (int l = tid; l <= PLAN_MAX_LEV; l += blockDim.x) {
    const int t = tiles[l];
    split[l] = t > 0 ? max(1, min(TC_MAX_SPLIT, target / t)) : 1;
  }
  __syncthreads();
  int* splits = plan + PLAN_LISTS * (ns + 1) + 2 + nlev;
  for (int l = tid; l <= nlev; l += blockDim.x) splits[l] = l == nlev ? split[PLAN_MAX_LEV] : (l < nl ? split[l] : 1);
  const int tsplit = split[PLAN_MAX_LEV];
  int tot[PLAN_LISTS];
#pragma unroll
  for (int l = 0; l < PLAN_LISTS; ++l) tot[l] = 0;
  for (int p = p0, lv = lv0; p < p1; ++p) {
    while (lv + 1 < nlev && level_first[lv + 1] <= p) ++lv;
    int c[PLAN_LISTS];
    plan_counts(level_list[p], super_ptr, rowpat_ptr, qcount, simt_max, tc_min, tc_gemm, tc_super,
                lv < nl ? split[lv] : 1, tsplit, c);
#pragma unroll
    for (int l = 0; l < PLAN_LISTS; ++l) tot[l] += c[l];
  }
  int off[PLAN_LISTS];
#pragma unroll
  for (int l = 0; l < PLAN_LISTS; ++l) {   // inclusive scan inside the warp
    int v = tot[l];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, v, o);
      if (lane >= o) v += y;
    }
    off[l] = v - tot[l];
    if (lane == 31) wsum[l][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int l = 0; l < PLAN_LISTS; ++l) {   // exclusive scan of the warp totals
      const int t = lane < nw ? wsum[l][lane] : 0;
      int v = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
      }
      if (lane < nw) wsum[l][lane] = v - t;
      if (lane == 31) plan[l * (ns + 1) + ns] = v;   // list total
    }
  }
  __syncthreads();
#pragma unroll
  for (int l = 0; l < PLAN_LISTS; ++l) off[l] += wsum[l][warp];
  for (int p = p0, lv = lv0; p < p1; ++p) {
    while (lv + 1 < nlev && level_first[lv + 1] <= p) ++lv;
    int c[PLAN_LISTS];
    plan_counts(level_list[p], super_ptr, rowpat_ptr, qcount, simt_max, tc_min, tc_gemm, tc_super,
                lv < nl ? split[lv] : 1, tsplit, c);
#pragma unroll
    for (int l = 0; l < PLAN_LISTS; ++l) {
      plan[l * (ns + 1) + p] = off[l];
      off[l] += c[l];
    }
  }
  for (int i = tid; i < 2 + nlev; i += blockDim.x) plan[PLAN_LISTS * (ns + 1) + i] = 0;
}

__global__ void __launch_bounds__(1024)
    k_plan(int ns, const int* __restrict__ level_list, const int* __restrict__ super_ptr,
           const int64_t* __restrict__ rowpat_ptr, const int* __restrict__ qcount, int simt_max, int tc_min,
           int tc_gemm, const unsigned char* __restrict__ tc_super, const int* __restrict__ level_first, int nlev,
           int target, int* plan) {
  pdl_entry();
  d_plan(own_block(), ns, level_list, super_ptr, rowpat_ptr, qcount, simt_max, tc_min, tc_gemm, tc_super, level_first,
         nlev, target, plan);
}

struct plan_body {
  static constexpr int threads = 1024, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_plan; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_plan(vb, a...);
  }
};

// Entry (row, column 3*kl + d) of supernode s's front: its H^T entry (rows < w)
// plus the children's update entries listed for that row (extend-add as a
// gather, children in ascending order; ctr_row holds each child row's index
// in the front storage).
template <class T>
__device__ __forceinline__ T assemble_entry(int s, int row, int kl, int d, int c0, int w, int m,
                                           const int64_t* __restrict__ fr_ptr,
                                           const int* __restrict__ ctr_ptr, const int* __restrict__ ctr_child,
                                           const int* __restrict__ ctr_row, const int* __restrict__ nodes,
                                           const T* __restrict__ bary, const int* __restrict__ qidx,
                                           const int* __restrict__ qinv, const T* X, int64_t ldx) {
  T v = T(0);
  if (row < w && (c0 + row) % 3 == d) {
    // column 3k+d of contact a holds bary[a,i] at DOF 3*node_i + d
    const int node = (c0 + row) / 3;
    const int a = qidx[(size_t)s * m + kl];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (nodes[4 * a + i] == node) v += bary[4 * a + i];
  }
  const int64_t fr = fr_ptr[s] + row;
  const int e1 = ctr_ptr[fr + 1];
#pragma unroll 2
  for (int e = ctr_ptr[fr]; e < e1; ++e) {
    const int jl = qinv[(size_t)ctr_child[e] * m + kl];
    if (jl >= 0) v += X[(int64_t)ctr_row[e] * ldx + 3 * jl + d];
  }
  return v;
}

// Assembly of the fronts of one level (positions [pa, pb) of level_list).
// Work unit (supernode, ASM_ROWS-row tile, TCC-contact tile), found once per
// unit; a block of TCOLS x AR threads, each thread assembling the front
// elements of its column in ASM_ROWS / AR rows (independent gathers in
// flight): the H^T entry, plus the children's update entries listed for that
// row (extend-add as a gather, children in ascending order).  Rows < w go to
// Ftop, rows >= w to the front's update rows.
template <class T>
__device__ __forceinline__ void d_assemble(const VB& vb, const int* __restrict__ plan, int pa, int pb,
                                           const int* __restrict__ level_list, const int* __restrict__ super_ptr,
                                           const int64_t* __restrict__ rowpat_ptr, const int64_t* __restrict__ fr_ptr,
                                           const int* __restrict__ ctr_ptr, const int* __restrict__ ctr_child,
                                           const int* __restrict__ ctr_row, const int* __restrict__ nodes,
                                           const T* __restrict__ bary, const int* __restrict__ qcount,
                                           const int* __restrict__ qidx, const int* __restrict__ qinv, int m, T* X,
                                           T* Ftop, int64_t ldx) {
  const int u1 = plan[pb];
  for (int u = plan[pa] + vb.bx; u < u1; u += vb.gx) {
    const int pos = find_pos(plan, pa, pb, u);
    const int s = level_list[pos];
    const int nq = qcount[s];
    const int local = u - plan[pos];
    const int nt = cdiv(nq, TCC);
    const int rt = local / nt, t = local % nt;
    const int k0 = t * TCC;
    const int ncols = 3 * min(TCC, nq - k0);
    const int col = threadIdx.x;
    if (col >= ncols) continue;
    const int c0 = super_ptr[s], w = super_ptr[s + 1] - c0;
    const int nrows = w + (int)(rowpat_ptr[s + 1] - rowpat_ptr[s]);
#pragma unroll
    for (int rr = 0; rr < ASM_ROWS / AR; ++rr) {
      const int row = rt * ASM_ROWS + rr * AR + threadIdx.y;
      if (row >= nrows) break;
      const T v = assemble_entry<T>(s, row, k0 + col / 3, col % 3, c0, w, m, fr_ptr, ctr_ptr, ctr_child, ctr_row,
                                    nodes, bary, qidx, qinv, X, ldx);
      if (row < w)
        Ftop[(int64_t)(c0 + row) * ldx + 3 * k0 + col] = v;
      else
        X[(fr_ptr[s] + row) * ldx + 3 * k0 + col] = v;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(AR * TCOLS)
    k_assemble(const int* __restrict__ plan, int pa, int pb, const int* __restrict__ level_list,
               const int* __restrict__ super_ptr, const int64_t* __restrict__ rowpat_ptr,
               const int64_t* __restrict__ fr_ptr, const int* __restrict__ ctr_ptr,
               const int* __restrict__ ctr_child, const int* __restrict__ ctr_row, const int* __restrict__ nodes,
               const T* __restrict__ bary, const int* __restrict__ qcount, const int* __restrict__ qidx,
               const int* __restrict__ qinv, int m, T* X, T* Ftop, int64_t ldx) {
  pdl_entry();
  d_assemble<T>(own_block(), plan, pa, pb, level_list, super_ptr, rowpat_ptr, fr_ptr, ctr_ptr, ctr_child, ctr_row,
                nodes, bary, qcount, qidx, qinv, m, X, Ftop, ldx);
}

template <class T>
struct assemble_body {
  static constexpr int threads = AR * TCOLS, minb = 1;
  static constexpr bool stride = true;
  static auto kernel() { return &k_assemble<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_assemble<T>(vb, a...);
  }
};

// Block (supernode, GR-row tile of the w + r front rows, 32-contact tile):
// out = G_s[rows, :] F_top; top rows store X_s = out, bottom rows U_s -= out.
// K is streamed in 32-wide chunks through a double-buffered cp.async pipeline.
// 256 threads as 16 x 16, each RPT rows x 6 columns: GR = 16 RPT front rows
// (RPT = 4: 64-row tiles; RPT = 2: 32-row tiles for short fronts).
static constexpr int FLD = TCOLS + 4;
template <int RPT>
struct GemmTile {
  static constexpr int GR = 16 * RPT, GLD = GR + 4;
};
template <class T>
__device__ __forceinline__ void cp_async_zfill(T* smem, const T* gmem, bool ok) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = ok ? (int)sizeof(T) : 0;   // 0 bytes read: the element is zero-filled
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}

template <class T, int RPT>
__device__ __forceinline__ void front_gemm_tile(int s, int rt, int t, int nq, const int* __restrict__ super_ptr,
                                                const int64_t* __restrict__ rowpat_ptr,
                                                const int64_t* __restrict__ val_ptr, const T* __restrict__ G,
                                                const int64_t* __restrict__ fr_ptr, T* X,
                                                const T* __restrict__ Ftop, int64_t ldx, T* sG, T* sF) {
  const int k0 = t * TCC;
  const int ncols = 3 * min(TCC, nq - k0);
  const int c0 = super_ptr[s], w = super_ptr[s + 1] - c0;
  const int nrows = w + (int)(rowpat_ptr[s + 1] - rowpat_ptr[s]);
  constexpr int GR = GemmTile<RPT>::GR, GLD = GemmTile<RPT>::GLD;
  const int row0 = rt * GR;
  const int64_t ldG = nrows;
  const T* Gs = G + val_ptr[s];
  const T* Ft = Ftop + (int64_t)c0 * ldx + 3 * k0;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  auto load = [&](int kb, int buf) {
    const int nb = min(KB, w - kb);
    T* dG = sG + buf * KB * GLD;
    T* dF = sF + buf * KB * FLD;
    for (int e = tid; e < KB * GR; e += 256) {
      const int k = e / GR, i = e % GR;
      const bool ok = k < nb && row0 + i < nrows;
      cp_async_zfill(&dG[k * GLD + i], ok ? &Gs[(int64_t)(kb + k) * ldG + row0 + i] : Gs, ok);
    }
    for (int e = tid; e < KB * TCOLS; e += 256) {
      const int k = e / TCOLS, jj = e % TCOLS;
      const bool ok = k < nb && jj < ncols;
      cp_async_zfill(&dF[k * FLD + jj], ok ? &Ft[(int64_t)(kb + k) * ldx + jj] : Ft, ok);
    }
    cp_async_commit();
  };
  T acc[RPT][6];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[q][c] = T(0);
  load(0, 0);
  int buf = 0;
  for (int kb = 0; kb < w; kb += KB) {
    if (kb + KB < w) {
      load(kb + KB, buf ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const T* cG = sG + buf * KB * GLD;
    const T* cF = sF + buf * KB * FLD;
#pragma unroll 8
    for (int k = 0; k < KB; ++k) {
      T a[RPT], bv[6];
#pragma unroll
      for (int q = 0; q < RPT; ++q) a[q] = cG[k * GLD + RPT * ty + q];
#pragma unroll
      for (int c = 0; c < 6; ++c) bv[c] = cF[k * FLD + 6 * tx + c];
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[q][c] += a[q] * bv[c];
    }
    __syncthreads();
    buf ^= 1;
  }
  T* F = X + fr_ptr[s] * ldx + 3 * k0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int row = row0 + RPT * ty + q;
    if (row >= nrows) continue;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int col = 6 * tx + c;
      if (col >= ncols) continue;
      if (row < w)
        F[(int64_t)row * ldx + col] = acc[q][c];
      else
        F[(int64_t)row * ldx + col] -= acc[q][c];
    }
  }
}

template <class T, int RPT>
__device__ __forceinline__ void d_front_gemm(const VB& vb, const int* __restrict__ plan, int pa, int pb,
                                             const int* __restrict__ level_list, const int* __restrict__ super_ptr,
                                             const int64_t* __restrict__ rowpat_ptr,
                                             const int64_t* __restrict__ val_ptr, const T* __restrict__ G,
                                             const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount, T* X,
                                             const T* __restrict__ Ftop, int64_t ldx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sG = (T*)smraw;                                  // 2 x KB x GLD
  T* sF = sG + 2 * KB * GemmTile<RPT>::GLD;           // 2 x KB x FLD
  __shared__ int pos_sh;
  const int u1 = plan[pb];
  for (int u = plan[pa] + vb.bx; u < u1; u += vb.gx) {   // block-uniform
    const int pos = block_find_pos(plan, pa, pb, u, &pos_sh);
    const int s = level_list[pos];
    const int nq = qcount[s];
    const int local = u - plan[pos];
    const int nt = cdiv(nq, TCC);
    const int rt = local / nt, t = local % nt;
    front_gemm_tile<T, RPT>(s, rt, t, nq, super_ptr, rowpat_ptr, val_ptr, G, fr_ptr, X, Ftop, ldx, sG, sF);
  }
}

template <class T, int RPT>
__global__ void __launch_bounds__(256)
    k_front_gemm(const int* __restrict__ plan, int pa, int pb, const int* __restrict__ level_list,
                 const int* __restrict__ super_ptr, const int64_t* __restrict__ rowpat_ptr,
                 const int64_t* __restrict__ val_ptr, const T* __restrict__ G, const int64_t* __restrict__ fr_ptr,
                 const int* __restrict__ qcount, T* X, const T* __restrict__ Ftop, int64_t ldx) {
  pdl_entry();
  d_front_gemm<T, RPT>(own_block(), plan, pa, pb, level_list, super_ptr, rowpat_ptr, val_ptr, G, fr_ptr, qcount, X,
                       Ftop, ldx);
}

template <class T, int RPT>
struct front_gemm_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = true;
  static auto kernel() { return &k_front_gemm<T, RPT>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_front_gemm<T, RPT>(vb, a...);
  }
};

template <class T, int RPT>
static size_t gemm_smem_bytes() {
  return 2 * (size_t)KB * (GemmTile<RPT>::GLD + FLD) * sizeof(T);
}

// ------------------------------------------------------------------ a3 pivot scaling
// Y = D^-1/2 X in place on the first w rows of every front (one warp per DOF
// row), with D^-1/2 kept in FP64.  FP32 scenes split the FP64 value once per
// row into FP32 parts hi + lo (hi = D^-1/2 rounded, lo = the remainder
// rounded) and form x hi + (x lo) with one fused rounding: the error of x lo
// is below 2^-48 of the product, so the result is the FP64 product rounded to
// FP32 except within 2^-48 (relative) of a rounding midpoint, where the FP64
// route rounds twice as well.  The FP32 units do it at their full rate.
template <class T>
__device__ __forceinline__ void d_scale(const VB& vb, int n, const int* __restrict__ dof_super,
                                        const int* __restrict__ super_ptr, const int64_t* __restrict__ fr_ptr,
                                        const int* __restrict__ qcount, const double* __restrict__ dinvsqrt, T* X,
                                        int64_t ldx) {
  const int row = vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int s = dof_super[row];
  const int ncol = 3 * qcount[s];
  const double ds = dinvsqrt[row];
  T* F = X + (fr_ptr[s] + row - super_ptr[s]) * ldx;
  if constexpr (sizeof(T) == 8) {
    for (int c = lane; c < ncol; c += 32) F[c] *= ds;
  } else {
    const float hi = (float)ds, lo = (float)(ds - (double)hi);
    for (int c = lane; c < ncol; c += 32) F[c] = __fmaf_rn(F[c], hi, F[c] * lo);
  }
}

template <class T>
__global__ void k_scale(int n, const int* __restrict__ dof_super, const int* __restrict__ super_ptr,
                        const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                        const double* __restrict__ dinvsqrt, T* X, int64_t ldx) {
  pdl_entry();
  d_scale<T>(own_block(), n, dof_super, super_ptr, fr_ptr, qcount, dinvsqrt, X, ldx);
}

template <class T>
struct scale_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_scale<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_scale<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ a4 contraction
// Work unit (supernode s, tile pair I <= J of its local columns), for the
// fronts narrower than the tensor-core threshold (all fronts in SIMT mode):
// W_H[g(i), g(j)] += sum_k Y[k,i] Y[k,j] over the scaled fronts Y = D^-1/2 X.
// Only the upper triangle (g(i) <= g(j)) is accumulated; k_symmetrize mirrors
// it.  Blocks take units from a counter, largest supernodes (the end of
// level_list) first.
template <class T>
__device__ __forceinline__ void d_contract(const VB& vb, const int* __restrict__ plan, int* counter, int ns,
                                           const int* __restrict__ level_list, const int* __restrict__ super_ptr,
                                           const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                                           const int* __restrict__ qidx, int m, const T* __restrict__ X, int64_t ldx,
                                           T* WH, int64_t ldw) {
  __shared__ T sA[CK_][CT + 1];
  __shared__ T sB[CK_][CT + 1];
  __shared__ int unit_sh, pos_sh;
  const int total = plan[ns];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (;;) {
    if (tid == 0) unit_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int ur = unit_sh;
    __syncthreads();
    if (ur >= total) break;
    const int u = total - 1 - ur;
    const int pos = block_find_pos(plan, 0, ns, u, &pos_sh);
    const int s = level_list[pos];
    const int ncol = 3 * qcount[s];
    const int nt = cdiv(ncol, CT);
    int rem = u - plan[pos], I = 0;
    while (rem >= nt - I) {
      rem -= nt - I;
      ++I;
    }
    const int J = I + rem;
    const int c0 = super_ptr[s], w = super_ptr[s + 1] - c0;
    const T* Xs = X + fr_ptr[s] * ldx;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int kb = 0; kb < w; kb += CK_) {
      const int nb = min(CK_, w - kb);
      for (int e = tid; e < CK_ * CT; e += blockDim.x) {
        int k = e / CT, c = e % CT;
        int ca = I * CT + c, cb = J * CT + c;
        sA[k][c] = (k < nb && ca < ncol) ? Xs[(int64_t)(kb + k) * ldx + ca] : T(0);
        sB[k][c] = (k < nb && cb < ncol) ? Xs[(int64_t)(kb + k) * ldx + cb] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < CK_; ++k) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = sA[k][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = sB[k][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
      }
      __syncthreads();
    }
    const int* q = qidx + (size_t)s * m;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int li = I * CT + ty * 4 + a;
      if (li >= ncol) continue;
      int64_t gi = 3 * (int64_t)q[li / 3] + li % 3;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int lj = J * CT + tx * 4 + b;
        if (lj >= ncol || li > lj) continue;
        int64_t gj = 3 * (int64_t)q[lj / 3] + lj % 3;
        atomicAdd(&WH[gi * ldw + gj], acc[a][b]);
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256)
    k_contract(const int* __restrict__ plan, int* counter, int ns, const int* __restrict__ level_list,
               const int* __restrict__ super_ptr, const int64_t* __restrict__ fr_ptr,
               const int* __restrict__ qcount, const int* __restrict__ qidx, int m,
               const T* __restrict__ X, int64_t ldx, T* WH, int64_t ldw) {
  pdl_entry();
  d_contract<T>(own_block(), plan, counter, ns, level_list, super_ptr, fr_ptr, qcount, qidx, m, X, ldx, WH, ldw);
}

template <class T>
struct contract_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = true;
  static auto kernel() { return &k_contract<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_contract<T>(vb, a...);
  }
};

// Mirrors the upper triangle of the nr x nr matrix A into its lower one, by
// 32 x 32 tiles (block (32, 8)): a tile at or below the diagonal reads its
// mirror tile's rows, transposes them in shared memory and writes its own
// rows, both coalesced.  With A16, also writes the BF16 copy of every entry
// (tiles above the diagonal copy their own entries).
template <class T>
__device__ __forceinline__ void d_symmetrize(const VB& vb, int nr, T* A, __nv_bfloat16* A16) {
  __shared__ T tile[32][33];
  const int ti = vb.by, tj = vb.bx;   // tile row, tile column
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tj > ti) {
    if (!A16) return;
    for (int r = ty; r < 32; r += 8) {
      const int i = ti * 32 + r, j = tj * 32 + tx;
      if (i < nr && j < nr) A16[(int64_t)i * nr + j] = __float2bfloat16_rn((float)A[(int64_t)i * nr + j]);
    }
    return;
  }
  // tile[c][r] = A[tj*32 + r][ti*32 + c] (the mirror tile's rows)
  for (int r = ty; r < 32; r += 8) {
    const int i = tj * 32 + r, j = ti * 32 + tx;
    if (i < nr && j < nr) tile[tx][r] = A[(int64_t)i * nr + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + tx;
    if (i >= nr || j >= nr) continue;
    if (j < i) {
      const T v = tile[r][tx];   // A[j][i]
      A[(int64_t)i * nr + j] = v;
      if (A16) A16[(int64_t)i * nr + j] = __float2bfloat16_rn((float)v);
    } else if (A16) {   // the diagonal tile's upper part: its own entries
      A16[(int64_t)i * nr + j] = __float2bfloat16_rn((float)tile[tx][r]);
    }
  }
}

template <class T>
__global__ void k_symmetrize(int nr, T* A, __nv_bfloat16* A16) {
  pdl_entry();
  d_symmetrize<T>(own_block(), nr, A, A16);
}

template <class T>
struct symmetrize_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_symmetrize<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_symmetrize<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ a6 W = C W_H C^T
// Also raises wblk[a][B] to the largest |W[3a, j]| over the columns j of PGS
// block B other than contact a's own (the normal row's coupling to that block;
// wblk is zeroed before the launch): the bound PGS uses to pass over separated
// contacts, taken over the blocks that may change only.
__device__ __forceinline__ void atomic_max_nonneg(unsigned* addr, float v) { atomicMax(addr, __float_as_uint(v)); }
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}
template <class T>
using bits_t = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
__device__ __forceinline__ unsigned to_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long to_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ float from_bits(unsigned u) { return __uint_as_float(u); }
__device__ __forceinline__ double from_bits(unsigned long long u) { return __longlong_as_double((long long)u); }
// max of non-negative values that keeps a NaN (its bits order above +inf)
template <class T>
__device__ __forceinline__ T nmax(T a, T b) {
  return a != a ? a : ((b > a || b != b) ? b : a);
}

// WM: operand precision (enum icr_w_update; FP32 scenes): W_H and C as stored,
// rounded to TF32, or W_H from its BF16 copy and C rounded to BF16; the
// products are accumulated in T.
template <class T, int WM>
__device__ __forceinline__ T w_operand(T x) {
  if constexpr (WM == ICR_W_TF32) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)x));
    return (T)__uint_as_float(r);
  } else if constexpr (WM == ICR_W_BF16) {
    return (T)__bfloat162float(__float2bfloat16_rn((float)x));
  } else {
    return x;
  }
}

template <class T, int WM>
__device__ __forceinline__ void d_update_W(const VB& vb, int m, const T* __restrict__ C, const T* __restrict__ WH,
                                           const __nv_bfloat16* __restrict__ WH16, T* W, int64_t ldw, T* wblk, int bc,
                                           const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;
  if (vb.bx < vb.by) return;   // the block pairs of the upper triangle only (uniform)
  __shared__ bits_t<T> mxa[16], mxb[16];
  __shared__ T sC[2][16][9];             // directions of the block's a and b contacts
  __shared__ T tile[48][49];             // W[3b + j, 3a + i] of the block, for coalesced mirror rows
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int b = vb.bx * 16 + tx, a = vb.by * 16 + ty;
  if (ty == 0) mxb[tx] = 0;
  if (tx == 0) mxa[ty] = 0;
  for (int e = tid; e < 2 * 16 * 9; e += 256) {
    const int w = e / 144, k = (e % 144) / 9, q = e % 9;
    const int c = (w == 0 ? vb.by : vb.bx) * 16 + k;
    sC[w][k][q] = c < m ? w_operand<T, WM>(C[9 * c + q]) : T(0);
  }
  __syncthreads();
  if (a < m && b < m && a <= b) {
    const int64_t ld = 3 * (int64_t)m;
    T M[3][3], t[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int64_t at = (3 * a + i) * ld + 3 * b + j;
        if constexpr (WM == ICR_W_BF16)
          M[i][j] = (T)__bfloat162float(WH16[at]);
        else
          M[i][j] = w_operand<T, WM>(WH[at]);
      }
    const T(*Ca)[3] = reinterpret_cast<const T(*)[3]>(&sC[0][ty][0]);
    const T(*Cb)[3] = reinterpret_cast<const T(*)[3]>(&sC[1][tx][0]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) t[i][j] = M[i][0] * Cb[j][0] + M[i][1] * Cb[j][1] + M[i][2] * Cb[j][2];
    T ra = T(0), rb = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T v = Ca[i][0] * t[0][j] + Ca[i][1] * t[1][j] + Ca[i][2] * t[2][j];
        W[(3 * a + i) * ldw + 3 * b + j] = v;
        if (a == b) W[(3 * b + j) * ldw + 3 * a + i] = v;   // the diagonal block, made symmetric
        tile[3 * tx + j][3 * ty + i] = v;
        if (i == 0) ra = nmax(ra, fabs(v));   // W[3a, 3b + j]
        if (j == 0) rb = nmax(rb, fabs(v));   // W[3b, 3a + i]
      }
    if (a != b) {
      atomic_max_nonneg(&mxa[ty], ra);
      atomic_max_nonneg(&mxb[tx], rb);
    }
  }
  __syncthreads();
  // the mirror W[3b + j, 3a + i] (a < b), 48 consecutive columns per row
  for (int e = tid; e < 48 * 48; e += 256) {
    const int rr = e / 48, cc = e % 48;
    const int bg = vb.bx * 16 + rr / 3, ag = vb.by * 16 + cc / 3;
    if (bg < m && ag < bg) W[(3 * bg + rr % 3) * ldw + 3 * ag + cc % 3] = tile[rr][cc];
  }
  // the tile's 16 columns lie in one PGS block of bc contacts (16 divides bc):
  // per contact, the largest |W[3a, j]| over that block's other columns
  const int nb = (m + bc - 1) / bc;
  const int ga = vb.by * 16 + tx, gb = vb.bx * 16 + tx;
  const int Ba = vb.by * 16 / bc, Bb = vb.bx * 16 / bc;
  if (ty == 0 && ga < m && mxa[tx] != 0)
    atomicMax(reinterpret_cast<bits_t<T>*>(wblk) + (int64_t)ga * nb + Bb, mxa[tx]);
  if (ty == 1 && gb < m && mxb[tx] != 0)
    atomicMax(reinterpret_cast<bits_t<T>*>(wblk) + (int64_t)gb * nb + Ba, mxb[tx]);
}

template <class T, int WM>
__global__ void k_update_W(int m, const T* __restrict__ C, const T* __restrict__ WH,
                           const __nv_bfloat16* __restrict__ WH16, T* W, int64_t ldw, T* wblk, int bc,
                           const int* __restrict__ stop) {
  pdl_entry();
  d_update_W<T, WM>(own_block(), m, C, WH, WH16, W, ldw, wblk, bc, stop);
}

template <class T, int WM>
struct update_W_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_update_W<T, WM>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_update_W<T, WM>(vb, a...);
  }
};

// The per-block coupling bounds (wblk) of a W given directly: one warp per
// contact's normal row
template <class T>
__device__ __forceinline__ void d_wcoup(const VB& vb, int m, const T* __restrict__ W, int64_t ldw, T* wblk, int bc) {
  const int a = (int)((vb.bx * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (a >= m) return;
  const T* row = W + (int64_t)(3 * a) * ldw;
  const int nb = (m + bc - 1) / bc;
  for (int B = 0; B < nb; ++B) {   // per PGS block: max |W[3a, j]| over its columns (not a's own)
    T mx = T(0);
    const int j1 = 3 * min(m, (B + 1) * bc);
    for (int j = 3 * B * bc + lane; j < j1; j += 32)
      if (j / 3 != a) mx = nmax(mx, fabs(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = nmax(mx, __shfl_xor_sync(FULL, mx, o));
    if (lane == 0) wblk[(int64_t)a * nb + B] = mx;
  }
}

template <class T>
__global__ void k_wcoup(int m, const T* __restrict__ W, int64_t ldw, T* wblk, int bc) {
  pdl_entry();
  d_wcoup<T>(own_block(), m, W, ldw, wblk, bc);
}

template <class T>
struct wcoup_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_wcoup<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_wcoup<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ a7 PGS
// One CTA of PGS_THREADS threads.  The residual r = delta + W lambda~ of every
// row is kept in shared memory.  Contacts are taken in blocks of BC; for each
// block, with one barrier per block:
//       warp 0 runs the block's contacts in order (lane = contact); the lane
//       of contact i solves it and every lane folds the change into its own
//       residual and into the next block's contact of the same lane, while the
//       other warps fold the previous block's non-zero changes into all other
//       residuals (streaming those rows of W) and prefetch, with cp.async,
//       the next block's rows of W (its diagonal block and the block to its right).
// A block whose contacts all have lambda~ = 0 and non-negative normal
// residuals is a no-op and is passed without reading W.  After a block that
// changed nothing every residual is complete, so the CTA looks ahead (one
// warp per block) and jumps over the run of no-op blocks that follows.
// With every residual complete, sweeps may visit only the blocks that can
// change (S-only sweeps, pgs_defer_enter), folding their changes into the
// other rows later in one pass, while a bound shows that no other contact
// can change.
// The solve stops when eps <= tol (tol > 0) or after a sweep that changed
// nothing, a fixed point of the iteration (Alg. 1's test with PGS_error = 0).
// Visiting order, residual definition and local rule are those of Eq. "PGS"
// with contacts in ascending order; the local rule uses reciprocals and an
// rsqrt scale, so results differ from the plain formulas by rounding only.
template <class T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) {
  return rsqrtf(x);
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) {
  return 1.0 / sqrt(x);
}
// correctly rounded reciprocal (the value of 1 / x)
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return __drcp_rn(x); }



static constexpr int PGS_MAX_BLOCKS = 1024;   // contact blocks per scene (m <= 1024 BC)
static constexpr int PGS_THREADS = 512;       // one CTA: warp 0 solves, the others stream
static constexpr int PGS_WARPS = PGS_THREADS / 32;
static constexpr int PGS_MAX_DEFER = 16;      // most blocks that may change while the others are passed over

// acc[q] += w[q] * d for one 16-byte chunk of a W row (16-byte aligned)
__device__ __forceinline__ void fma_chunk(float* acc, const float* w, float d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(w));
  acc[0] += v.x * d;
  acc[1] += v.y * d;
  acc[2] += v.z * d;
  acc[3] += v.w * d;
}
__device__ __forceinline__ void fma_chunk(double* acc, const double* w, double d) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(w));
  acc[0] += v.x * d;
  acc[1] += v.y * d;
}

// clears bits [lo, hi) of a bit array, one atomic per 32-bit word
__device__ __forceinline__ void clear_bits(unsigned* bits, int lo, int hi, int tid, int nthr) {
  for (int w = (lo >> 5) + tid; w <= ((hi - 1) >> 5) && lo < hi; w += nthr) {
    const int a = max(lo, w << 5) - (w << 5), e = min(hi, (w + 1) << 5) - (w << 5);   // bits [a, e) of word w
    const unsigned msk = (e - a == 32) ? ~0u : (((1u << (e - a)) - 1u) << a);
    atomicAnd(&bits[w], ~msk);
  }
}

// State of the S-only sweeps (deferred folds), in shared memory.
template <class T>
struct PgsDefer {
  int slist[PGS_MAX_DEFER];            // the blocks of S in ascending order
  unsigned sbits[PGS_MAX_BLOCKS / 32]; // S as a bit set
  int on, ns;                          // S-only sweeps start; |S|
  int xf[2];                           // leave them after step t (slot t & 1)
  T nb[PGS_MAX_DEFER];                 // sum of |D| over block slist[k]
  T th;                                // the bound sum |D| must stay below
  bits_t<T> thq;                       // theta being formed (bits of a non-negative value)
  int cnt;                             // entries of the compact list of non-zero D
  int sweeps, folds, rechecks, joins;  // statistics: S-only sweeps, deferred folds, rechecks, joins
  int xs[2];                           // sweeps warp 0 ended itself in step t (slot t & 1)
  unsigned jbits[PGS_MAX_BLOCKS / 32]; // blocks a recheck found that may change: they join S
};

// Largest coupling of contact a's normal row to the columns of the blocks of
// S: the bound on how far the changes D of S move its normal residual per unit
// of sum |D| (wblk: per contact and PGS block, from the W update).
template <class T>
__device__ __forceinline__ T s_coupling(const T* __restrict__ wblk, int nb, int a, const int* slist, int ns) {
  T w = T(0);
  for (int k = 0; k < ns; ++k) w = nmax(w, wblk[(int64_t)a * nb + slist[k]]);
  return w;
}

// Entered with every residual complete, at the end of a sweep.  S = the
// blocks that may change in the next sweep; every other contact has
// lambda~ = 0 and r_n >= 0 and keeps lambda~ = 0 while r_n stays
// non-negative.  The changes D of S move its r_n by at most ws * sum |D|, ws
// its largest coupling to the columns of S's blocks (s_coupling), so while
// sum |D| stays below theta = min r_n / ws over those contacts,
// sweeps can visit S only and fold S's changes into S's rows; the other rows
// wait for one fold of D.  Returns |S| when the S-only sweeps start, else 0.
// Out of line: its temporaries stay out of the solve loop's registers.
template <class T, int BC>
__device__ __noinline__ int pgs_defer_enter(PgsDefer<T>* d, int m, const T* lam, const T* r,
                                            const T* __restrict__ wblk, T* beta, T* dacc, T* dsnap) {
  constexpr int BR = 3 * BC;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nblk = (m + BC - 1) / BC;
  if (tid < PGS_MAX_BLOCKS / 32) d->sbits[tid] = 0u;
  if (tid == 0) d->thq = to_bits(T(INFINITY));
  __syncthreads();
  for (int bb = wid; bb < nblk; bb += PGS_WARPS) {
    const int i0 = 3 * bb * BC, nbb = min(BC, m - bb * BC);
    const bool a = lane < nbb && (lam[i0 + 3 * lane] != T(0) || lam[i0 + 3 * lane + 1] != T(0) ||
                                  lam[i0 + 3 * lane + 2] != T(0) || r[i0 + 3 * lane] < T(0));
    if (__ballot_sync(FULL, a) != 0u && lane == 0) atomicOr(&d->sbits[bb >> 5], 1u << (bb & 31));
  }
  __syncthreads();
  // S in ascending order (when it is small enough to sweep alone)
  if (wid == 0) {
    const unsigned wd = d->sbits[lane];
    const int c = __popc(wd);
    int off = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, off, o);
      if (lane >= o) off += y;
    }
    const int total = __shfl_sync(FULL, off, 31);
    off -= c;
    if (total <= PGS_MAX_DEFER && total < nblk)
      for (unsigned w = wd; w != 0u; w &= w - 1u) d->slist[off++] = lane * 32 + __ffs(w) - 1;
    if (lane == 0) d->ns = total;
  }
  __syncthreads();
  const int total = d->ns;
  if (total <= PGS_MAX_DEFER && total < nblk) {
    // theta = min over the other contacts of r_n / (their coupling to the blocks of S)
    for (int bb = wid; bb < nblk; bb += PGS_WARPS) {
      if ((d->sbits[bb >> 5] >> (bb & 31)) & 1u) continue;
      const int i0 = 3 * bb * BC, nbb = min(BC, m - bb * BC);
      T v = T(INFINITY);
      if (lane < nbb) {
        const T rn = r[i0 + 3 * lane], wm = s_coupling(wblk, nblk, bb * BC + lane, d->slist, total);
        beta[bb * BC + lane] = rn;       // the residual at the base (complete here)
        beta[m + bb * BC + lane] = wm;   // its coupling to S
        v = (wm > T(0) && rn > T(0)) ? rn / wm : (wm == T(0) ? T(INFINITY) : T(0));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL, v, o));
      if (lane == 0) atomicMin(&d->thq, to_bits(v));
    }
  }
  __syncthreads();
  if (wid == 0) {
    const T th = from_bits(d->thq);
    const bool on = total <= PGS_MAX_DEFER && total < nblk && th > T(0);
    if (on) {
      for (int i = lane; i < total * BR; i += 32) dacc[i] = dsnap[i] = T(0);
      if (lane < total) d->nb[lane] = T(0);
    }
    if (lane == 0) {
      d->on = on ? 1 : 0;
      d->th = th * T(1.0 - 1.0 / 1024.0);   // margin for the rounding of the bound
    }
  }
  __syncthreads();
  return d->on ? d->ns : 0;
}

// The bound on the changes of S since the last base ran out: every contact
// outside S gets its normal residual with all deferred changes D,
// r_n + W[n, S] D (W's symmetry: column n of the rows of D, from the list of
// D's non-zero rows built in drow / dval, stage 0's space), kept in beta.  If
// all stay positive, no contact outside S changes at its passed-over visit,
// and the bound starts again from this base (dsnap = D, theta from these
// residuals): returns 1.  Else the blocks of the contacts that may change are
// in jbits, and it returns 2 when S can take them (S-only sweeps with those
// blocks joined) or 0 (the caller leaves the S-only sweeps).
template <class T, int BC>
__device__ __noinline__ int pgs_defer_recheck(PgsDefer<T>* d, int m, int nsd, const T* __restrict__ W, int64_t ldw,
                                              const T* r, const T* dacc, T* dsnap, T* beta, int* drow, T* dval) {
  constexpr int BR = 3 * BC;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x;
  if (tid < PGS_MAX_BLOCKS / 32) d->jbits[tid] = 0u;
  if (wid == 0) {
    int cnt = 0;
    for (int k = 0; k < nsd; ++k) {
      const int R = 3 * d->slist[k] * BC;
      for (int w0 = 0; w0 < BR; w0 += 32) {
        const T v = w0 + lane < BR ? dacc[k * BR + w0 + lane] : T(0);
        const bool nz = v != T(0);
        const unsigned msk = __ballot_sync(FULL, nz);
        if (nz) {
          const int q = cnt + __popc(msk & ((1u << lane) - 1u));
          drow[q] = R + w0 + lane;
          dval[q] = v;
        }
        cnt += __popc(msk);
      }
    }
    if (lane == 0) {
      d->cnt = cnt;
      d->thq = to_bits(T(INFINITY));
    }
  }
  __syncthreads();
  const int nd = d->cnt;
  for (int a = tid; a < m; a += nthr) {
    const int blk = a / BC;
    if ((d->sbits[blk >> 5] >> (blk & 31)) & 1u) continue;
    T v = r[3 * a];
    for (int k = 0; k < nd; ++k) v += W[(int64_t)drow[k] * ldw + 3 * a] * dval[k];
    beta[a] = v;
    if (!(v > T(0))) {
      atomicOr(&d->jbits[blk >> 5], 1u << (blk & 31));
    } else {
      const T ws = beta[m + a];
      atomicMin(&d->thq, to_bits(ws > T(0) ? v / ws : T(INFINITY)));
    }
  }
  __syncthreads();
  int nj = 0;
#pragma unroll 4
  for (int w = 0; w < PGS_MAX_BLOCKS / 32; ++w) nj += __popc(d->jbits[w]);
  const int ok = nj == 0;
  if (ok) {
    for (int i = tid; i < nsd * BR; i += nthr) dsnap[i] = dacc[i];
    if (tid < nsd) d->nb[tid] = T(0);
    if (tid == 0) d->th = from_bits(d->thq) * T(1.0 - 1.0 / 1024.0);
  }
  __syncthreads();
  return ok ? 1 : (nsd + nj <= PGS_MAX_DEFER ? 2 : 0);
}

// After the deferred changes reached the rows of the blocks in jbits: S takes
// those blocks.  The new S in ascending order; D moved to its blocks' new
// positions (a position never moves down, so from the end), the joined blocks'
// D start at zero; a new base (dsnap = D, nb = 0); each other contact's
// coupling to S widened by the joined blocks and theta = min beta / ws.
// Returns the position in the new S of the block after pb (pb is in S).
template <class T, int BC>
__device__ __noinline__ int pgs_defer_merge(PgsDefer<T>* d, int m, int pb, T* dacc, T* dsnap,
                                            const T* __restrict__ wblk, T* beta) {
  constexpr int BR = 3 * BC;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x;
  const int nblk = (m + BC - 1) / BC;
  if (wid == 0) {
    const int nold = d->ns;
    const int oldb = lane < nold ? d->slist[lane] : -1;
    const unsigned wd = d->sbits[lane] | d->jbits[lane];
    const int c = __popc(wd);
    int off = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, off, o);
      if (lane >= o) off += y;
    }
    const int total = __shfl_sync(FULL, off, 31);
    off -= c;
    __syncwarp();
    for (unsigned w = wd; w != 0u; w &= w - 1u) d->slist[off++] = lane * 32 + __ffs(w) - 1;
    __syncwarp();
    for (int kp = total - 1; kp >= 0; --kp) {
      const int B = d->slist[kp];
      const unsigned mk = __ballot_sync(FULL, oldb == B);
      const int k = mk ? __ffs(mk) - 1 : -1;
      if (k != kp)
        for (int i = lane; i < BR; i += 32) dacc[kp * BR + i] = k >= 0 ? dacc[k * BR + i] : T(0);
      __syncwarp();
    }
    for (int i = lane; i < total * BR; i += 32) dsnap[i] = dacc[i];
    if (lane < total) d->nb[lane] = T(0);
    d->sbits[lane] = wd;
    if (lane == 0) {
      d->ns = total;
      d->thq = to_bits(T(INFINITY));
    }
  }
  __syncthreads();
  const int ns = d->ns;
  for (int a = tid; a < m; a += nthr) {
    const int blk = a / BC;
    if ((d->sbits[blk >> 5] >> (blk & 31)) & 1u) continue;
    T ws = beta[m + a];
    for (int k = 0; k < ns; ++k) {
      const int B = d->slist[k];
      if ((d->jbits[B >> 5] >> (B & 31)) & 1u) ws = nmax(ws, wblk[(int64_t)a * nblk + B]);
    }
    beta[m + a] = ws;
    const T v = beta[a];
    const T q = (ws > T(0) && v > T(0)) ? v / ws : (ws == T(0) ? T(INFINITY) : T(0));
    atomicMin(&d->thq, to_bits(q));
  }
  __syncthreads();
  int kp = 0;
  while (kp < ns - 1 && d->slist[kp] != pb) ++kp;
  if (tid < PGS_MAX_BLOCKS / 32) d->jbits[tid] = 0u;
  if (tid == 0) {
    d->th = from_bits(d->thq) * T(1.0 - 1.0 / 1024.0);
    ++d->joins;
  }
  __syncthreads();
  return kp + 1 == ns ? 0 : kp + 1;
}

// Leaves the S-only sweeps after block pb, whose changes are dlp: they are
// folded into the rows of S (its successor's pending share included, which
// warp 0 drops) and the deferred changes D of S into every other row.  Then
// every residual is complete.  Out of line, like pgs_defer_enter.
// With `only` (a block bit set) the deferred changes reach the rows of those
// blocks alone (a join), else every row outside S (a leave).
template <class T, int BC>
__device__ __noinline__ void pgs_defer_leave(PgsDefer<T>* d, int m, int pb, int nsd, const T* dlp,
                                             const T* __restrict__ W, int64_t ldw, T* r, const T* dacc,
                                             int* nzl, int* drow, T* dval, const unsigned* only) {
  constexpr int BR = 3 * BC;
  constexpr int CH = 16 / (int)sizeof(T);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x;
  const int n3 = 3 * m;
  const int pR0 = 3 * pb * BC, pnr = 3 * min(BC, m - pb * BC);
  int cnt = 0;
  if (wid == 0) {
    // compact list of the non-zero D rows, in order
    for (int k = 0; k < nsd; ++k) {
      const int R = 3 * d->slist[k] * BC;
      for (int w0 = 0; w0 < BR; w0 += 32) {
        const T v = w0 + lane < BR ? dacc[k * BR + w0 + lane] : T(0);
        const bool nz = v != T(0);
        const unsigned msk = __ballot_sync(FULL, nz);
        if (nz) {
          const int q = cnt + __popc(msk & ((1u << lane) - 1u));
          drow[q] = R + w0 + lane;
          dval[q] = v;
        }
        cnt += __popc(msk);
      }
    }
    if (lane == 0) d->cnt = cnt;
  } else {
    int* lst = nzl + (wid - 1) * BR;
#pragma unroll
    for (int w0 = 0; w0 < BR; w0 += 32) {
      const bool nz = w0 + lane < pnr && dlp[w0 + lane] != T(0);
      const unsigned msk = __ballot_sync(FULL, nz);
      if (nz) lst[cnt + __popc(msk & ((1u << lane) - 1u))] = w0 + lane;
      cnt += __popc(msk);
    }
  }
  __syncthreads();
  if (wid > 0) {
    const int t2 = tid - 32, n2 = nthr - 32, nd = d->cnt;
    const int* lst = nzl + (wid - 1) * BR;
    const int nch = (n3 + CH - 1) / CH;
    for (int c = t2; c < nch; c += n2) {
      const int j0 = c * CH;
      if (j0 >= pR0 && j0 < pR0 + pnr) continue;
      const int blk = j0 / BR;
      T acc[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) acc[q] = T(0);
      if ((d->sbits[blk >> 5] >> (blk & 31)) & 1u) {
        const T* Wc = W + (int64_t)pR0 * ldw + j0;
        for (int k = 0; k < cnt; ++k) fma_chunk(acc, Wc + (int64_t)lst[k] * ldw, dlp[lst[k]]);
      } else if (!only || ((only[blk >> 5] >> (blk & 31)) & 1u)) {
        for (int k = 0; k < nd; ++k) fma_chunk(acc, W + (int64_t)drow[k] * ldw + j0, dval[k]);
      } else {
        continue;
      }
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (j0 + q < n3) r[j0 + q] += acc[q];
    }
  }
  __syncthreads();
}


template <class T, int BC>
__device__ __forceinline__ void d_pgs(const VB& vb, int m, int sweeps, double tol, const T* __restrict__ W,
                                      int64_t ldw, const T* __restrict__ delta, const T* __restrict__ mu,
                                      const T* __restrict__ wblk, T* pgsb, T* lam_g, int warm, PgsDevStats* st,
                                      const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;   // uniform, before any shared memory or barrier
  constexpr int BR = 3 * BC;
  constexpr int CH = 16 / (int)sizeof(T);      // elements per 16-byte copy
  constexpr int RCH = BR / CH;                 // 16-byte copies per block row
  extern __shared__ __align__(16) unsigned char smraw[];
  // stage k holds, for the block it was loaded for, WD = W[block rows, block
  // cols] and WR = W[block rows, next block's cols] (row-major, ld BR); warp 0
  // reads them through the symmetry of W as W[cols, rows], bank-conflict free.
  T* WD = (T*)smraw;               // 2 x BR x BR
  T* WR = WD + 2 * BR * BR;        // 2 x BR x BR
  T* lam = WR + 2 * BR * BR;       // 3m
  T* r = lam + 3 * m;              // 3m
  T* dl = r + 3 * m;               // 2 x BR: lambda~ changes of the last two blocks
  T* dacc = dl + 2 * BR;           // PGS_MAX_DEFER x BR: changes of the blocks in S not yet folded elsewhere
  T* dsnap = dacc + PGS_MAX_DEFER * BR;   // PGS_MAX_DEFER x BR: dacc at the bound's base
  int* nzl = (int*)(dsnap + PGS_MAX_DEFER * BR);  // (PGS_WARPS - 1) x BR: per streaming warp, rows with a non-zero change
  __shared__ T red[PGS_WARPS];
  __shared__ int pref[2];            // block whose rows stage k holds (-1: none)
  __shared__ int psuc[2];            // the block whose columns stage k's WR holds
  __shared__ int chg_sweep[2];       // some lambda~ changed in sweep (done & 1)
  __shared__ int chg_it[2];          // block processed at step t changed some lambda~ (slot t & 1)
  __shared__ int nxt[2][2];          // look-ahead results (two slots, alternating): from b on, from 0
  __shared__ T cst[2][5][BC];        // per-contact local-rule constants of the block in stage k
  __shared__ int cst_blk[2];         // block whose constants cst[k] holds (-1: none)
  __shared__ unsigned actb[PGS_MAX_BLOCKS / 32];   // block had a changing contact in its last visit
  __shared__ PgsDefer<T> dfs;       // S-only sweeps (deferred folds)
  static_assert(PGS_MAX_BLOCKS / 32 == 32 && PGS_MAX_DEFER <= 32, "one warp scans the block bits");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x;
  const int n3 = 3 * m;
  const int nblk = (m + BC - 1) / BC;
  // W[rows of block bn, cols of block bn and of its successor bn1] -> stage k
  auto prefetch = [&](int bn, int bn1, int k, int t0, int nt) {
    const int n0 = 3 * bn * BC, nnr = 3 * min(BC, m - bn * BC), c1 = 3 * bn1 * BC;
    T* D = WD + k * BR * BR;
    T* Rr = WR + k * BR * BR;
    for (int e = t0; e < nnr * RCH; e += nt) {
      const int i = e / RCH, c = (e % RCH) * CH;
      const T* src = W + (int64_t)(n0 + i) * ldw;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(&D[i * BR + c])),
                   "l"(src + n0 + c));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(&Rr[i * BR + c])),
                   "l"(src + c1 + c));
    }
    cp_async_commit();
  };
  for (int i = tid; i < n3; i += nthr) lam[i] = warm ? lam_g[i] : T(0);
  for (int i = tid; i < 2 * BR; i += nthr) dl[i] = T(0);
  for (int i = tid; i < PGS_MAX_BLOCKS / 32; i += nthr) actb[i] = 0u;
  if (tid == 0) {
    pref[1] = -1;
    psuc[0] = 1 % nblk;
    psuc[1] = -1;
    dfs.on = dfs.ns = 0;
    dfs.sweeps = dfs.folds = dfs.rechecks = dfs.joins = 0;
    dfs.xs[0] = dfs.xs[1] = 0;
    dfs.xf[0] = dfs.xf[1] = 0;
    chg_sweep[0] = chg_sweep[1] = 0;
    chg_it[0] = chg_it[1] = 1;   // no look-ahead before the first block
    nxt[0][0] = nxt[0][1] = nxt[1][0] = nxt[1][1] = nblk;
    cst_blk[0] = cst_blk[1] = -1;
  }
  __syncthreads();
  if (warm) {
    for (int row = wid; row < n3; row += PGS_WARPS) {
      const T* Wr = W + (int64_t)row * ldw;
      T acc = T(0);
#pragma unroll 4
      for (int j = lane; j < n3; j += 32) acc += Wr[j] * lam[j];
      acc = warp_sum(acc);
      if (lane == 0) r[row] = delta[row] + acc;
    }
  } else {
    for (int i = tid; i < n3; i += nthr) r[i] = delta[i];
  }
  __syncthreads();
  // a block starts active when one of its contacts has lambda~ != 0 or a
  // negative normal residual; only active blocks have their rows prefetched
  for (int bb = wid; bb < nblk; bb += PGS_WARPS) {
    const int i0 = 3 * bb * BC, nbb = min(BC, m - bb * BC);
    const bool a = lane < nbb && (lam[i0 + 3 * lane] != T(0) || lam[i0 + 3 * lane + 1] != T(0) ||
                                  lam[i0 + 3 * lane + 2] != T(0) || r[i0 + 3 * lane] < T(0));
    if (__ballot_sync(FULL, a) != 0u && lane == 0) atomicOr(&actb[bb >> 5], 1u << (bb & 31));
  }
  // No block holds a contact with lambda~ != 0 or a negative normal residual:
  // the first sweep changes nothing, a fixed point (lambda~ = 0) after one
  // sweep, as the loop below would find.
  if (!__syncthreads_or(tid < PGS_MAX_BLOCKS / 32 && actb[tid] != 0u)) {
    for (int i = tid; i < n3; i += nthr) lam_g[i] = T(0);
    if (tid == 0) {
      st->sweeps = sweeps > 0 ? 1 : 0;
      st->eps = 0.0;
      st->s_only = 0;
      st->folds = 0;
      st->rechecks = 0;
      st->joins = 0;
    }
    return;
  }
  const bool act0 = nblk <= 2 || (actb[0] & 1u);
  if (act0) prefetch(0, 1 % nblk, 0, tid, nthr);
  if (tid == 0) pref[0] = act0 ? 0 : -1;
  cp_async_wait_all();
  __syncthreads();

  // warp 0: lane l holds the residual (q) of contact l of the current block and
  // the pending changes (p) of contact l of the next block
  T p0 = 0, p1 = 0, p2 = 0, dsum = T(0), dlast = T(0);
  int done = 0, b = 0, pb = -1, look = 0;
  bool known = false;   // b was found by a look-ahead: no second look needed
  unsigned t = 0;   // blocks processed (its parity selects double-buffered slots)
  const bool want_eps = tol > 0.0;   // eps of a sweep is formed into red[0]
  // S-only sweeps: |S| (0: off), position of b in slist, may start in this
  // sweep; a sweep end waits for a recheck; S-block visits since the bound's base
  int nsd = 0, kpos = 0, tryd = 1, since = 0;
  bool pend = false;
  // end of a sweep: eps = ||lambda^i - lambda^(i-1)|| / ||lambda^i|| (Alg. 1),
  // formed only when a positive tol needs it; returns 1 to stop at eps <= tol
  // or after a sweep that changed nothing (a fixed point: every later sweep
  // would repeat it exactly)
  auto end_sweep = [&]() -> int {
    if (want_eps) {
      T nrm = T(0);
      for (int i = tid; i < n3; i += nthr) nrm += lam[i] * lam[i];
      nrm = warp_sum(nrm);
      if (lane == 0) red[wid] = nrm;
      const T ds = wid == 0 ? warp_sum(dsum) : T(0);
      __syncthreads();
      if (tid == 0) {
        T tot = T(0);
        for (int k = 0; k < PGS_WARPS; ++k) tot += red[k];
        red[0] = tot > T(0) ? sqrt(ds / tot) : T(0);
      }
      __syncthreads();
    }
    const int brk = !chg_sweep[done & 1] || (want_eps && (double)red[0] <= tol);
    if (wid == 0) {
      dlast = dsum;
      dsum = T(0);
    }
    if (tid == 0) {
      chg_sweep[(done + 1) & 1] = 0;
      if (nsd) ++dfs.sweeps;
    }
    ++done;
    tryd = 1;
    __syncthreads();
    return brk;
  };
  while (done < sweeps) {
    if (nsd && dfs.xf[(t + 1) & 1]) {   // set in the previous step
      // The bound on the changes of S ran out after block pb: the passed-over
      // contacts' normal residuals are formed with the deferred changes.  If
      // none would change, the S-only sweeps go on from this new base; if
      // some would, their blocks join S when it can take them; else fold what
      // was deferred and go on in order after pb.  (The list of D's non-zero
      // rows is built in stage 0: its rows are fetched again.)
      if (tid == 0 && since >= nsd) ++dfs.rechecks;
      const int rc = since >= nsd ? pgs_defer_recheck<T, BC>(&dfs, m, nsd, W, ldw, r, dacc, dsnap, pgsb, (int*)WD, WR)
                                  : 0;
      __syncthreads();   // every thread has read the flag before it is cleared
      if (tid == 0) {
        dfs.xf[0] = dfs.xf[1] = 0;
        pref[0] = -1;
        cst_blk[0] = -1;
      }
      __syncthreads();
      if (rc == 1) {
        since = 0;
        if (pend) {
          pend = false;
          if (end_sweep()) break;
        }
        continue;
      }
      if (rc == 2) {
        // The blocks holding contacts that may change join S: the deferred
        // changes reach their rows, pb's changes the rows of S (warp 0 drops
        // its pending share), and the S-only sweeps go on after pb in order,
        // the joined blocks included (a plain sweep visits them there too).
        if (wid == 0) p0 = p1 = p2 = T(0);
        pgs_defer_leave<T, BC>(&dfs, m, pb, nsd, dl + (1 - (int)(t & 1)) * BR, W, ldw, r, dacc, nzl, (int*)WD, WR,
                               dfs.jbits);
        kpos = pgs_defer_merge<T, BC>(&dfs, m, pb, dacc, dsnap, wblk, pgsb);
        nsd = dfs.ns;
        since = 0;
        pend = false;
        const int bnext = dfs.slist[kpos];
        const bool wrap = bnext <= pb;   // no joined block after pb: the sweep ends here
        pb = -1;
        b = bnext;
        if (wrap && end_sweep()) break;
        continue;
      }
      pend = false;
      if (wid == 0) p0 = p1 = p2 = T(0);
      pgs_defer_leave<T, BC>(&dfs, m, pb, nsd, dl + (1 - (int)(t & 1)) * BR, W, ldw, r, dacc, nzl,
                             (int*)WD, WR, nullptr);   // scratch in stage 0
      if (tid == 0) {
        ++dfs.folds;
        dfs.xf[0] = dfs.xf[1] = 0;
        pref[0] = -1;
        cst_blk[0] = -1;
        chg_it[(t + 1) & 1] = 0;   // nothing pending: look ahead from b
      }
      __syncthreads();
      // every residual is complete again: the look-ahead from b may start
      // S-only sweeps over the new S at once (as a sweep's first look-ahead does)
      nsd = 0;
      tryd = 1;
      b = pb + 1;
      pb = -1;
      known = false;
      continue;
    }
    if (!nsd && !known && !chg_it[(t + 1) & 1]) {   // the previous step's slot
      // the last block changed nothing: every residual is complete and nothing
      // is pending, so blocks that hold lambda~ = 0 and non-negative normal
      // residuals stay unchanged.  One warp per block finds the first other
      // block from b on, and the first from 0 on (the next sweep's start when
      // this sweep has none left).
      int* nx = nxt[look & 1];
      for (int bb = wid; bb < nblk; bb += PGS_WARPS) {
        const int i0 = 3 * bb * BC, nbb = min(BC, m - bb * BC);
        const bool a = lane < nbb && (lam[i0 + 3 * lane] != T(0) || lam[i0 + 3 * lane + 1] != T(0) ||
                                      lam[i0 + 3 * lane + 2] != T(0) || r[i0 + 3 * lane] < T(0));
        if (__ballot_sync(FULL, a) != 0u && lane == 0) {
          if (bb >= b) atomicMin(&nx[0], bb);
          atomicMin(&nx[1], bb);
        }
      }
      __syncthreads();
      const int nb_ = nx[0], nw_ = nx[1];
      if (tid == 0) nxt[(look + 1) & 1][0] = nxt[(look + 1) & 1][1] = nblk;   // the other slot, for the next look-ahead
      ++look;
      // blocks passed over hold no active contact (a prefetch hint, no barrier needed)
      clear_bits(actb, b, nb_, tid, nthr);
      b = nb_;
      if (tryd && b < nblk) {
        // every residual is complete: the rest of the sweep and the next
        // sweeps may visit S only, starting at b (the first block of S from b)
        tryd = 0;
        nsd = pgs_defer_enter<T, BC>(&dfs, m, lam, r, wblk, pgsb, dacc, dsnap);
        kpos = since = 0;
        while (kpos < nsd - 1 && dfs.slist[kpos] != b) ++kpos;
      }
      if (b == nblk) {   // the rest of the sweep is unchanged: end of sweep
        if (want_eps) {
          T nrm = T(0);
          for (int i = tid; i < n3; i += nthr) nrm += lam[i] * lam[i];
          nrm = warp_sum(nrm);
          if (lane == 0) red[wid] = nrm;
          const T ds = wid == 0 ? warp_sum(dsum) : T(0);
          __syncthreads();
          if (tid == 0) {
            T tot = T(0);
            for (int k = 0; k < PGS_WARPS; ++k) tot += red[k];
            red[0] = tot > T(0) ? sqrt(ds / tot) : T(0);
          }
          __syncthreads();
        }
        int brk = !chg_sweep[done & 1] || (want_eps && (double)red[0] <= tol);
        if (wid == 0) {
          dlast = dsum;
          dsum = T(0);
        }
        if (tid == 0) chg_sweep[(done + 1) & 1] = 0;
        ++done;
        if (!brk && nw_ == nblk && done < sweeps) {
          // no block can change in the next sweep: it is a sweep without
          // change, after which the iteration stops at its fixed point
          if (wid == 0) {
            dlast = T(0);
          }
          ++done;
          brk = 1;
        }
        clear_bits(actb, 0, nw_, tid, nthr);
        tryd = 1;
        if (!brk && nw_ < nblk && done < sweeps) {
          tryd = 0;
          nsd = pgs_defer_enter<T, BC>(&dfs, m, lam, r, wblk, pgsb, dacc, dsnap);
          kpos = since = 0;
        }
        b = nw_;
        known = true;   // the next sweep starts at a block that may change
        __syncthreads();
        if (brk) break;
        continue;
      }
    }
    known = false;
    const int a0 = b * BC, nb = min(BC, m - a0), R0 = 3 * a0;
    // the next block visited: the next one in order, or the next one of S
    const int bn = nsd ? dfs.slist[kpos + 1 == nsd ? 0 : kpos + 1] : (b + 1 == nblk ? 0 : b + 1);
    const int dc = (int)(t & 1);   // slot of this block's changes in dl
    // stage of this block's rows: alternating, so that the next block's rows
    // can be prefetched into the other one; when S is one block, whichever
    // stage holds it (nothing is prefetched then)
    int stg = dc;
    if (nsd == 1 && pref[stg] != b && pref[1 - stg] == b) stg = 1 - stg;
    if (wid == 0) {
      const T* WDc = WD + stg * BR * BR;
      const T* WRc = WR + stg * BR * BR;
      const bool valid = lane < nb;
      const int ll = lane < BC ? lane : BC - 1;   // lanes past the block read a valid column
      // lane l: contact l of this block (residual q, lambda~ l, its 3x3 diagonal data)
      T q0 = T(0), q1 = T(0), q2 = T(0), l0 = T(0), l1 = T(0), l2 = T(0);
      T iWnn = T(0), Wt1n = T(0), Wt2n = T(0), iwt = T(0), mua = T(0);
      if (valid) {
        q0 = r[R0 + 3 * lane] + p0;
        q1 = r[R0 + 3 * lane + 1] + p1;
        q2 = r[R0 + 3 * lane + 2] + p2;
        l0 = lam[R0 + 3 * lane];
        l1 = lam[R0 + 3 * lane + 1];
        l2 = lam[R0 + 3 * lane + 2];
      }
      p0 = p1 = p2 = T(0);
      T e0 = 0, e1 = 0, e2 = 0;
      // No contact of the block can change unless one starts active (changes
      // only come from active contacts): such a block needs no rows of W.
      const bool any = __ballot_sync(FULL, valid && (l0 != T(0) || l1 != T(0) || l2 != T(0) || q0 < T(0))) != 0u;
      if (lane == 0) {
        if (any)
          atomicOr(&actb[b >> 5], 1u << (b & 31));
        else
          atomicAnd(&actb[b >> 5], ~(1u << (b & 31)));
      }
      if (any && (pref[stg] != b || (bn != b && psuc[stg] != bn))) {
        // rows not prefetched: warp 0 fetches them now
        T* D = WD + stg * BR * BR;
        T* Rr = WR + stg * BR * BR;
        const int c1 = 3 * bn * BC, nr = 3 * nb;
        for (int e = lane; e < nr * RCH; e += 32) {
          const int i = e / RCH, c = (e % RCH) * CH;
          const T* src = W + (int64_t)(R0 + i) * ldw;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(&D[i * BR + c])),
                       "l"(src + R0 + c));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(&Rr[i * BR + c])),
                       "l"(src + c1 + c));
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        if (lane == 0) {
          pref[stg] = b;
          psuc[stg] = bn;
          cst_blk[stg] = -1;
        }
      }
      if (any) {
        // the local rule's constants, kept with the stage's rows: a block that
        // comes back to the same stage reuses them
        if (cst_blk[stg] == b) {
          if (valid) {
            iWnn = cst[stg][0][lane];
            Wt1n = cst[stg][1][lane];
            Wt2n = cst[stg][2][lane];
            iwt = cst[stg][3][lane];
            mua = cst[stg][4][lane];
          }
        } else {
          if (valid) {
            const T* Wo = WDc + (3 * lane) * BR + 3 * lane;
            iWnn = rcp_t(Wo[0]);
            Wt1n = Wo[BR];
            Wt2n = Wo[2 * BR];
            iwt = rcp_t(T(0.5) * (Wo[BR + 1] + Wo[2 * BR + 2]));
            mua = mu[a0 + lane];
            cst[stg][0][lane] = iWnn;
            cst[stg][1][lane] = Wt1n;
            cst[stg][2][lane] = Wt2n;
            cst[stg][3][lane] = iwt;
            cst[stg][4][lane] = mua;
          }
          __syncwarp();
          if (lane == 0) cst_blk[stg] = b;
        }
      }
      // Every lane forms the update its own contact would take from its current
      // residual (the local rule); the next contact in order whose update is
      // not zero is applied and folded into every lane's residual.  The contacts
      // passed over have zero updates (among them every contact with lambda~ = 0
      // and a non-negative normal residual), so the iterate is exactly that of
      // visiting them in order.
      int xs = 0;          // sweeps warp 0 ends itself (S is this block alone)
      bool lv = false;     // the bound on the changes of S ran out
      bool chg;
      for (bool go = any;;) {
      int i = -1;
      while (go) {
        // without branches: lanes past the block hold zeros and get zero updates
        T ln = l0 - q0 * iWnn;
        ln = ln > T(0) ? ln : T(0);
        const T dn = ln - l0;
        const T rt1 = q1 + Wt1n * dn, rt2 = q2 + Wt2n * dn;
        T lt1 = l1 - rt1 * iwt, lt2 = l2 - rt2 * iwt;
        const T lim = mua * ln;
        const T s2 = lt1 * lt1 + lt2 * lt2;
        const bool out = s2 > lim * lim;            // outside the friction disc: project
        const T sc = lim * rsqrt_t(out ? s2 : T(1));
        lt1 = ln <= T(0) ? T(0) : (out ? lt1 * sc : lt1);
        lt2 = ln <= T(0) ? T(0) : (out ? lt2 * sc : lt2);
        const T c0 = ln - l0, c1 = lt1 - l1, c2 = lt2 - l2;
        const unsigned act = __ballot_sync(FULL, valid && lane > i && (c0 != T(0) || c1 != T(0) || c2 != T(0)));
        if (act == 0u) break;
        i = __ffs(act) - 1;
        // couplings W[3i+c, 3l+q] (this block) and W[3i+c, next block's 3l+q]
        const T* Wl = WDc + (3 * i) * BR + 3 * ll;
        const T* Xl = WRc + (3 * i) * BR + 3 * ll;
        const T w00 = Wl[0], w01 = Wl[1], w02 = Wl[2], w10 = Wl[BR], w11 = Wl[BR + 1], w12 = Wl[BR + 2],
                w20 = Wl[2 * BR], w21 = Wl[2 * BR + 1], w22 = Wl[2 * BR + 2];
        const T d0 = __shfl_sync(FULL, c0, i), d1 = __shfl_sync(FULL, c1, i), d2 = __shfl_sync(FULL, c2, i);
        if (lane == i) {
          l0 = ln;
          l1 = lt1;
          l2 = lt2;
          e0 = d0;
          e1 = d1;
          e2 = d2;
          dsum += d0 * d0 + d1 * d1 + d2 * d2;
        }
        q0 += w00 * d0 + w10 * d1 + w20 * d2;
        q1 += w01 * d0 + w11 * d1 + w21 * d2;
        q2 += w02 * d0 + w12 * d1 + w22 * d2;
        if (bn != b) {   // pending changes for the next block (none when it is this block)
          const T x00 = Xl[0], x01 = Xl[1], x02 = Xl[2], x10 = Xl[BR], x11 = Xl[BR + 1], x12 = Xl[BR + 2],
                  x20 = Xl[2 * BR], x21 = Xl[2 * BR + 1], x22 = Xl[2 * BR + 2];
          p0 += x00 * d0 + x10 * d1 + x20 * d2;
          p1 += x01 * d0 + x11 * d1 + x21 * d2;
          p2 += x02 * d0 + x12 * d1 + x22 * d2;
        }
      }
      if (nsd) {
        // accumulate this visit's changes into D and test the bound: the
        // blocks outside S up to the next block of S see the state after it
        T* Dk = dacc + kpos * BR;
        const T* Sk = dsnap + kpos * BR;
        T part = T(0);
        if (valid) {
          const T D0 = Dk[3 * lane] + e0, D1 = Dk[3 * lane + 1] + e1, D2 = Dk[3 * lane + 2] + e2;
          Dk[3 * lane] = D0;
          Dk[3 * lane + 1] = D1;
          Dk[3 * lane + 2] = D2;
          part = fabs(D0 - Sk[3 * lane]) + fabs(D1 - Sk[3 * lane + 1]) + fabs(D2 - Sk[3 * lane + 2]);
        }
        part = warp_sum(part);
        T tot = lane < nsd ? (lane == kpos ? part : dfs.nb[lane]) : T(0);
        tot = warp_sum(tot);
        lv = !(tot <= dfs.th);
        if (lane == 0) {
          dfs.nb[kpos] = part;
          if (lv) dfs.xf[t & 1] = 1;
        }
      }
      chg = __any_sync(FULL, e0 != T(0) || e1 != T(0) || e2 != T(0));
      // When S is this block alone, the visit ends a sweep.  Warp 0 ends it
      // and starts the next one itself, residuals kept in registers, while
      // the other warps wait at the barrier; the main loop ends the last
      // sweep (no change, eps <= tol, the sweep cap or the bound running out).
      if (nsd != 1 || !chg || lv || done + xs + 1 >= sweeps) break;
      if (want_eps) {
        // lambda~ outside S is zero, so ||lambda^i|| is this block's
        T nl = valid ? l0 * l0 + l1 * l1 + l2 * l2 : T(0);
        nl = warp_sum(nl);
        const T ds = warp_sum(dsum);
        if ((nl > T(0) ? (double)sqrt(ds / nl) : 0.0) <= tol) break;
      }
      dlast = dsum;
      dsum = T(0);
      ++xs;
      e0 = e1 = e2 = T(0);
      go = __ballot_sync(FULL, valid && (l0 != T(0) || l1 != T(0) || l2 != T(0) || q0 < T(0))) != 0u;
      }
      if (valid) {
        lam[R0 + 3 * lane] = l0;
        lam[R0 + 3 * lane + 1] = l1;
        lam[R0 + 3 * lane + 2] = l2;
        r[R0 + 3 * lane] = q0;       // complete residual of this block's rows
        r[R0 + 3 * lane + 1] = q1;
        r[R0 + 3 * lane + 2] = q2;
      }
      if (lane == 0) {
        chg_it[t & 1] = chg ? 1 : 0;
        if (xs) {
          chg_sweep[(done + xs) & 1] = chg ? 1 : 0;   // the slot of the sweep now running
          dfs.sweeps += xs;
        } else if (chg) {
          chg_sweep[done & 1] = 1;
        }
        dfs.xs[t & 1] = xs;
      }
      if (lane < BC) {                // lanes without a change write zeros
        dl[dc * BR + 3 * lane] = e0;
        dl[dc * BR + 3 * lane + 1] = e1;
        dl[dc * BR + 3 * lane + 2] = e2;
      }
      if (bn == b) p0 = p1 = p2 = T(0);   // single block: the residual already has them
    } else if (wid & 3) {
      // the streaming warps: the twelve of the three sub-partitions other than
      // warp 0's (warps are spread over the SM's four schedulers by id mod 4),
      // so that the serial chain has its scheduler to itself
      const int t2 = (wid - 1 - (wid >> 2)) * 32 + lane, n2 = (PGS_WARPS - PGS_WARPS / 4) * 32;
      {
        // prefetch the next block's rows when it has a non-zero lambda~ or
        // changed in its last visit (data no streaming warp writes, so every
        // warp takes the same decision); a block that needs rows it did not
        // get has them fetched by warp 0
        const int nbn = min(BC, m - bn * BC), bn0 = 3 * bn * BC;
        bool need = nsd > 1 || (!nsd && (nblk <= 2 || ((actb[bn >> 5] >> (bn & 31)) & 1u)));
        if (!need && !nsd) {
          const bool nz = lane < nbn && (lam[bn0 + 3 * lane] != T(0) || lam[bn0 + 3 * lane + 1] != T(0) ||
                                         lam[bn0 + 3 * lane + 2] != T(0));
          need = __ballot_sync(FULL, nz) != 0u;
        }
        const int bn1 = nsd ? dfs.slist[(kpos + 2) % nsd] : (bn + 1) % nblk;
        if (need) prefetch(bn, bn1, 1 - stg, t2, n2);
        // a stage not refilled keeps the rows it holds: a block that comes back
        // to the same stage (the next sweep's first active block) reuses them
        if (t2 == 0 && need) {
          pref[1 - stg] = bn;
          psuc[1 - stg] = bn1;
          cst_blk[1 - stg] = -1;
        }
      }
      if (pb >= 0) {
        // fold the previous block's non-zero changes into every row but this
        // block's and its own; each warp lists the non-zero rows by ballot
        const T* dlp = dl + (1 - dc) * BR;
        const int pR0 = 3 * pb * BC, pnr = 3 * min(BC, m - pb * BC);
        int* lst = nzl + (wid - 1) * BR;
        int cnt = 0;
#pragma unroll
        for (int w0 = 0; w0 < BR; w0 += 32) {
          const bool nz = w0 + lane < pnr && dlp[w0 + lane] != T(0);
          const unsigned msk = __ballot_sync(FULL, nz);
          if (nz) lst[cnt + __popc(msk & ((1u << lane) - 1u))] = w0 + lane;
          cnt += __popc(msk);
        }
        __syncwarp();
        if (cnt > 0) {
          // rows in 16-byte chunks (block starts are multiples of the chunk, so a
          // chunk is inside or outside a block; W's padding columns are zero);
          // during S-only sweeps only the rows of S
          const int nch = nsd ? nsd * RCH : (n3 + CH - 1) / CH;
          for (int c = t2; c < nch; c += n2) {
            const int j0 = nsd ? 3 * dfs.slist[c / RCH] * BC + (c % RCH) * CH : c * CH;
            if (j0 >= n3) continue;
            if ((j0 >= R0 && j0 < R0 + 3 * nb) || (j0 >= pR0 && j0 < pR0 + pnr)) continue;
            T acc[CH];
#pragma unroll
            for (int q = 0; q < CH; ++q) acc[q] = T(0);
            const T* Wc = W + (int64_t)pR0 * ldw + j0;
            constexpr int UNR = sizeof(T) == 4 ? 8 : 4;   // loads in flight per group, within 64 registers
            for (int k0 = 0; k0 < cnt; k0 += UNR) {
              // a whole group is issued at once (predicated), so a short tail
              // does not fall back to one load latency per row
#pragma unroll
              for (int u = 0; u < UNR; ++u)
                if (k0 + u < cnt) {
                  const int i = lst[k0 + u];
                  fma_chunk(acc, Wc + (int64_t)i * ldw, dlp[i]);
                }
            }
#pragma unroll
            for (int q = 0; q < CH; ++q)
              if (j0 + q < n3) r[j0 + q] += acc[q];
          }
        }
      }
      cp_async_wait_all();
    }
    __syncthreads();
    pb = b;
    const bool leave = nsd && dfs.xf[t & 1];
    done += dfs.xs[t & 1];   // sweeps warp 0 ended itself
    ++t;
    pend = leave && bn <= b;   // the sweep ends once the passed-over blocks are shown unchanged
    if (bn <= b && !leave && end_sweep()) break;
    b = bn;
    if (nsd) {
      kpos = kpos + 1 == nsd ? 0 : kpos + 1;
      ++since;
    }
  }
  // eps of the last sweep, for the statistics
  double eps = 0.0;
  {
    T nrm = T(0);
    for (int i = tid; i < n3; i += nthr) nrm += lam[i] * lam[i];
    nrm = warp_sum(nrm);
    if (lane == 0) red[wid] = nrm;
    const T ds = wid == 0 ? warp_sum(dlast) : T(0);
    __syncthreads();
    if (tid == 0) {
      T tot = T(0);
      for (int k = 0; k < PGS_WARPS; ++k) tot += red[k];
      eps = tot > T(0) ? (double)sqrt(ds / tot) : 0.0;
    }
  }
  for (int i = tid; i < n3; i += nthr) lam_g[i] = lam[i];
  if (tid == 0) {
    st->sweeps = done;
    st->eps = eps;
    st->s_only = dfs.sweeps;
    st->folds = dfs.folds;
    st->rechecks = dfs.rechecks;
    st->joins = dfs.joins;
  }
}

template <class T, int BC>
__global__ void __launch_bounds__(PGS_THREADS, 1)
    k_pgs(int m, int sweeps, double tol, const T* __restrict__ W, int64_t ldw, const T* __restrict__ delta,
          const T* __restrict__ mu, const T* __restrict__ wblk, T* pgsb, T* lam_g, int warm, PgsDevStats* st,
          const int* __restrict__ stop) {
  pdl_entry();
  d_pgs<T, BC>(own_block(), m, sweeps, tol, W, ldw, delta, mu, wblk, pgsb, lam_g, warm, st, stop);
}

template <class T, int BC>
struct pgs_body {
  static constexpr int threads = PGS_THREADS, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_pgs<T, BC>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_pgs<T, BC>(vb, a...);
  }
};

template <class T, int BC>
static size_t pgs_smem_bytes(int m) {
  const size_t BR = 3 * BC;
  return (4 * BR * BR + 6 * (size_t)m + 2 * BR + 2 * PGS_MAX_DEFER * BR) * sizeof(T) +
         (PGS_WARPS - 1) * BR * sizeof(int);
}

// FP64 residuals of the final iterate: one warp per contact.
template <class T>
__device__ __forceinline__ void d_pgs_residual(const VB& vb, int m, const T* __restrict__ W, int64_t ldw,
                                               const T* __restrict__ delta, const T* __restrict__ mu,
                                               const T* __restrict__ lam, double rel, PgsDevStats* st) {
  const int a = vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= m) return;
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T* Wr = W + (3 * (int64_t)a + k) * ldw;
    double acc = 0.0;
    for (int j = lane; j < 3 * m; j += 32) acc += (double)Wr[j] * (double)lam[j];
    acc = warp_sum(acc);
    d[k] = (double)delta[3 * a + k] + acc;
  }
  if (lane != 0) return;
  const double L0 = lam[3 * a], L1 = lam[3 * a + 1], L2 = lam[3 * a + 2];
  const double lim = (double)mu[a] * L0;
  const double nt = hypot(L1, L2);
  atomic_max_nonneg(&st->res_bits[0], fabs(fmin(d[0], L0)));
  atomic_max_nonneg(&st->res_bits[1], fmax(0.0, nt - lim));
  // slip: on the cone within rel, which includes a frictionless contact
  // (mu lambda_n = 0, lambda_t = 0) whose sliding Coulomb's law leaves free
  const bool on_cone = L0 > 0 && nt >= lim * (1.0 - rel);
  const bool stick = L0 > 0 && !on_cone;
  if (L0 <= 0) {
    atomicAdd(&st->n_sep, 1);
  } else if (on_cone) {
    atomicAdd(&st->n_slip, 1);
    if (nt > 0) {
      const double tx = L1 / nt, ty = L2 / nt;
      const double along = d[1] * tx + d[2] * ty;
      const double px = d[1] - along * tx, py = d[2] - along * ty;
      atomic_max_nonneg(&st->res_bits[3], hypot(px, py) + fmax(0.0, along));
    }
  } else if (stick) {
    atomicAdd(&st->n_stick, 1);
    atomic_max_nonneg(&st->res_bits[2], hypot(d[1], d[2]));
  }
}

template <class T>
__global__ void k_pgs_residual(int m, const T* __restrict__ W, int64_t ldw, const T* __restrict__ delta,
                               const T* __restrict__ mu, const T* __restrict__ lam, double rel, PgsDevStats* st) {
  pdl_entry();
  d_pgs_residual<T>(own_block(), m, W, ldw, delta, mu, lam, rel, st);
}

template <class T>
struct pgs_residual_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_pgs_residual<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_pgs_residual<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ Newton stop
// After the linearisation for the next Newton iteration: the FP64
// complementarity residual of a zero increment at the new gaps,
// max over contacts of max(0, -delta_n).  At most tol: the next solve has
// nothing to correct, the loop ends (nw[0] = 1); else one more iteration runs
// (nw[1] counts the iterations after the first).  One block.
template <class T>
__device__ __forceinline__ void d_newton_check(const VB& vb, int m, const T* __restrict__ delta, double tol, int* nw) {
  if (nw[0]) return;
  __shared__ double red[32];
  double v = 0.0;
  for (int a = threadIdx.x; a < m; a += blockDim.x) v = fmax(v, -(double)delta[3 * a]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    if (mx <= tol)
      nw[0] = 1;
    else
      nw[1] += 1;
  }
}

template <class T>
__global__ void k_newton_check(int m, const T* __restrict__ delta, double tol, int* nw) {
  pdl_entry();
  d_newton_check<T>(own_block(), m, delta, tol, nw);
}

template <class T>
struct newton_check_body {
  static constexpr int threads = 1024, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_newton_check<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_newton_check<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ a8 proximity update
template <class T>
__device__ __forceinline__ void d_prox_u(const VB& vb, int m, const T* __restrict__ C, const T* __restrict__ lam,
                                         T* uk, double* u, const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;
  int a = vb.bx * blockDim.x + threadIdx.x;
  if (a >= m) return;
  const T l0 = lam[3 * a], l1 = lam[3 * a + 1], l2 = lam[3 * a + 2];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T v = C[9 * a + j] * l0 + C[9 * a + 3 + j] * l1 + C[9 * a + 6 + j] * l2;
    uk[3 * a + j] = v;
    u[3 * a + j] += (double)v;
  }
}

template <class T>
__global__ void k_prox_u(int m, const T* __restrict__ C, const T* __restrict__ lam, T* uk, double* u,
                         const int* __restrict__ stop) {
  pdl_entry();
  d_prox_u<T>(own_block(), m, C, lam, uk, u, stop);
}

template <class T>
struct prox_u_body {
  static constexpr int threads = 128, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_prox_u<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_prox_u<T>(vb, a...);
  }
};

// u_k = C_k^T lambda~_k and p += W_H u_k in one launch: every CTA forms u_k in
// shared memory (12 flops per contact), CTA 0 also adds it to u (FP64), and
// each warp takes one row of W_H.
template <class T>
__device__ __forceinline__ void d_prox(const VB& vb, int m, const T* __restrict__ C, const T* __restrict__ lam,
                                       const T* __restrict__ WH, double* u, double* p, double* dp,
                                       const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* uk = (T*)smraw;   // 3m
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    const T l0 = lam[3 * a], l1 = lam[3 * a + 1], l2 = lam[3 * a + 2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T v = C[9 * a + j] * l0 + C[9 * a + 3 + j] * l1 + C[9 * a + 6 + j] * l2;
      uk[3 * a + j] = v;
      if (vb.bx == 0) u[3 * a + j] += (double)v;
    }
  }
  __syncthreads();
  bool nz = false;
  for (int a = threadIdx.x; a < 3 * m; a += blockDim.x) nz |= uk[a] != T(0);
  nz = __syncthreads_or(nz);
  const int i = vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= 3 * m) return;
  if (!nz) {   // C^T lambda~ = 0: p stays, dp = 0 (no row of W_H is read)
    if (lane == 0) dp[i] = 0.0;
    return;
  }
  const T* Wr = WH + (int64_t)i * 3 * m;
  T acc = T(0);
  for (int j = lane; j < 3 * m; j += 32) acc += Wr[j] * uk[j];
  acc = warp_sum(acc);
  if (lane == 0) {
    p[i] += (double)acc;
    dp[i] = (double)acc;
  }
}

template <class T>
__global__ void k_prox(int m, const T* __restrict__ C, const T* __restrict__ lam, const T* __restrict__ WH,
                       double* u, double* p, double* dp, const int* __restrict__ stop) {
  pdl_entry();
  d_prox<T>(own_block(), m, C, lam, WH, u, p, dp, stop);
}

template <class T>
struct prox_body {
  static constexpr int threads = 512, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_prox<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_prox<T>(vb, a...);
  }
};

template <class T>
__device__ __forceinline__ void d_prox_p(const VB& vb, int m, const T* __restrict__ WH, const T* __restrict__ uk,
                                         double* p, double* dp, const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;
  const int i = vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= 3 * m) return;
  const T* Wr = WH + (int64_t)i * 3 * m;
  T acc = T(0);
  for (int j = lane; j < 3 * m; j += 32) acc += Wr[j] * uk[j];
  acc = warp_sum(acc);
  if (lane == 0) {
    p[i] += (double)acc;
    dp[i] = (double)acc;
  }
}

template <class T>
__global__ void k_prox_p(int m, const T* __restrict__ WH, const T* __restrict__ uk, double* p, double* dp,
                         const int* __restrict__ stop) {
  pdl_entry();
  d_prox_p<T>(own_block(), m, WH, uk, p, dp, stop);
}

template <class T>
struct prox_p_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_prox_p<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_prox_p<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ a9 corrective motion
// y = D^-1 X u = D^-1/2 (Y u), one warp per DOF row (Y holds the scaled front
// rows, restricted to the contacts reaching them); u in the working precision
template <class T>
__device__ __forceinline__ void d_xu(const VB& vb, int n, const int* __restrict__ dof_super,
                                     const int* __restrict__ super_ptr, const int64_t* __restrict__ fr_ptr,
                                     const int* __restrict__ qcount, const int* __restrict__ qidx, int m,
                                     const T* __restrict__ X, int64_t ldx, const T* __restrict__ u,
                                     const double* __restrict__ dinvsqrt, T* y) {
  const int row = vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int s = dof_super[row];
  const int nq = qcount[s];
  const T* F = X + (fr_ptr[s] + row - super_ptr[s]) * ldx;
  const int* q = qidx + (size_t)s * m;
  T acc = T(0);
  for (int k = lane; k < nq; k += 32) {
    const T* ua = u + 3 * q[k];
    acc += F[3 * k] * ua[0] + F[3 * k + 1] * ua[1] + F[3 * k + 2] * ua[2];
  }
  acc = warp_sum(acc);
  if (lane == 0) y[row] = (T)(dinvsqrt[row] * (double)acc);
}

template <class T>
__global__ void k_xu(int n, const int* __restrict__ dof_super, const int* __restrict__ super_ptr,
                     const int64_t* __restrict__ fr_ptr, const int* __restrict__ qcount,
                     const int* __restrict__ qidx, int m, const T* __restrict__ X, int64_t ldx,
                     const T* __restrict__ u, const double* __restrict__ dinvsqrt, T* y) {
  pdl_entry();
  d_xu<T>(own_block(), n, dof_super, super_ptr, fr_ptr, qcount, qidx, m, X, ldx, u, dinvsqrt, y);
}

template <class T>
struct xu_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_xu<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_xu<T>(vb, a...);
  }
};

// u in the working precision for k_xu
template <class T>
__device__ __forceinline__ void d_u_round(const VB& vb, int n3, const double* __restrict__ u, T* ut) {
  const int i = vb.bx * blockDim.x + threadIdx.x;
  if (i < n3) ut[i] = (T)u[i];
}

template <class T>
__global__ void k_u_round(int n3, const double* __restrict__ u, T* ut) {
  pdl_entry();
  d_u_round<T>(own_block(), n3, u, ut);
}

template <class T>
struct u_round_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_u_round<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_u_round<T>(vb, a...);
  }
};

// Backward solve L^T dq = y for the supernodes of one level (top-down):
// dq_s = G_s^T [y_s ; -dq_R], one warp per DOF column of the supernode.
template <class T>
__device__ __forceinline__ void d_bsolve(const VB& vb, const int* __restrict__ level_list, int lvl_first, int nchunk,
                                         const int* __restrict__ super_ptr, const int64_t* __restrict__ rowpat_ptr,
                                         const int* __restrict__ rowpat, const int64_t* __restrict__ val_ptr,
                                         const T* __restrict__ G, const T* __restrict__ y, T* dq) {
  const int s = level_list[lvl_first + vb.bx / nchunk];
  const int k = (vb.bx % nchunk) * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int c0 = super_ptr[s], w = super_ptr[s + 1] - c0;
  if (k >= w) return;
  const int r = (int)(rowpat_ptr[s + 1] - rowpat_ptr[s]);
  const T* Gk = G + val_ptr[s] + (int64_t)k * (w + r);
  const int* R = rowpat + rowpat_ptr[s];
  T acc = T(0);
  for (int i = (k & ~31) + lane; i < w; i += 32) acc += Gk[i] * y[c0 + i];
  for (int i = lane; i < r; i += 32) acc -= Gk[w + i] * dq[R[i]];
  acc = warp_sum(acc);
  if (lane == 0) dq[c0 + k] = acc;
}

template <class T>
__global__ void __launch_bounds__(256)
    k_bsolve(const int* __restrict__ level_list, int lvl_first, int nchunk, const int* __restrict__ super_ptr,
             const int64_t* __restrict__ rowpat_ptr, const int* __restrict__ rowpat,
             const int64_t* __restrict__ val_ptr, const T* __restrict__ G, const T* __restrict__ y, T* dq) {
  pdl_entry();
  d_bsolve<T>(own_block(), level_list, lvl_first, nchunk, super_ptr, rowpat_ptr, rowpat, val_ptr, G, y, dq);
}

template <class T>
struct bsolve_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_bsolve<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_bsolve<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ linearisation
// C rows n, t1, t2 and the gaps from the current proximity positions.  The
// normal, the choice of the tangent axis and the normal gap are formed in
// FP64 (the gap is a small difference of large distances); in the FP32 path
// the tangent frame and the tangential gaps are formed in FP32, the precision
// C and delta are stored in (FP64 arithmetic is a slow path on this part).
template <class T>
__device__ __forceinline__ void d_linearize(const VB& vb, int m, int kind, const double* __restrict__ normals_k,
                                            const double* __restrict__ anchors, const double* __restrict__ spheres,
                                            const int* __restrict__ sphere_of, const double* __restrict__ p, T* C,
                                            T* delta, const int* __restrict__ stop) {
  if (newton_stopped(stop)) return;
  int a = vb.bx * blockDim.x + threadIdx.x;
  if (a >= m) return;
  const double px = p[3 * a], py = p[3 * a + 1], pz = p[3 * a + 2];
  const double rx = px - anchors[3 * a], ry = py - anchors[3 * a + 1], rz = pz - anchors[3 * a + 2];
  double n0, n1, n2, dn;
  if (kind == 1) {
    n0 = normals_k[3 * a];
    n1 = normals_k[3 * a + 1];
    n2 = normals_k[3 * a + 2];
    dn = n0 * rx + n1 * ry + n2 * rz;
  } else {
    const double* sp = spheres + 4 * sphere_of[a];
    const double dx = px - sp[0], dy = py - sp[1], dz = pz - sp[2];
    const double dist = sqrt(dx * dx + dy * dy + dz * dz);
    if (sizeof(T) == 8) {
      n0 = dx / dist;
      n1 = dy / dist;
      n2 = dz / dist;
    } else {
      const double inv = 1.0 / dist;
      n0 = dx * inv;
      n1 = dy * inv;
      n2 = dz * inv;
    }
    dn = dist - sp[3];
  }
  // tangent t1 = n x e, e the axis of the smallest |n| component; t2 = n x t1
  int ax = 0;
  double best = fabs(n0);
  if (fabs(n1) < best) {
    ax = 1;
    best = fabs(n1);
  }
  if (fabs(n2) < best) ax = 2;
  const T m0 = (T)n0, m1 = (T)n1, m2 = (T)n2;
  const T e0 = ax == 0, e1 = ax == 1, e2 = ax == 2;
  T t10 = m1 * e2 - m2 * e1, t11 = m2 * e0 - m0 * e2, t12 = m0 * e1 - m1 * e0;
  const T nt = sqrt(t10 * t10 + t11 * t11 + t12 * t12);
  t10 /= nt;
  t11 /= nt;
  t12 /= nt;
  const T t20 = m1 * t12 - m2 * t11, t21 = m2 * t10 - m0 * t12, t22 = m0 * t11 - m1 * t10;
  const T qx = (T)rx, qy = (T)ry, qz = (T)rz;
  T* Ca = C + 9 * a;
  Ca[0] = m0;
  Ca[1] = m1;
  Ca[2] = m2;
  Ca[3] = t10;
  Ca[4] = t11;
  Ca[5] = t12;
  Ca[6] = t20;
  Ca[7] = t21;
  Ca[8] = t22;
  delta[3 * a] = (T)dn;
  delta[3 * a + 1] = t10 * qx + t11 * qy + t12 * qz;
  delta[3 * a + 2] = t20 * qx + t21 * qy + t22 * qz;
}

template <class T>
__global__ void k_linearize(int m, int kind, const double* __restrict__ normals_k,
                            const double* __restrict__ anchors, const double* __restrict__ spheres,
                            const int* __restrict__ sphere_of, const double* __restrict__ p, T* C, T* delta,
                            const int* __restrict__ stop) {
  pdl_entry();
  d_linearize<T>(own_block(), m, kind, normals_k, anchors, spheres, sphere_of, p, C, delta, stop);
}

template <class T>
struct linearize_body {
  static constexpr int threads = 128, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_linearize<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_linearize<T>(vb, a...);
  }
};

// ------------------------------------------------------------------ launchers
// the front GEMM's dynamic shared memory set up on the device, and its
// resident blocks per SM (cached per device)
template <class T, int RPT>
static int gemm_occupancy(int dev, int* occ) {
  static SmemLimit lim;
  static DevInt occ_dev;
  cudaError_t e = ensure_smem(k_front_gemm<T, RPT>, lim, dev, (int)gemm_smem_bytes<T, RPT>());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_front_gemm)");
  int o = occ_dev.get(dev);
  if (o == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_front_gemm<T, RPT>, 256, gemm_smem_bytes<T, RPT>());
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_front_gemm)");
    o = std::max(1, o);
    occ_dev.put(dev, o);
  }
  *occ = o;
  return ICR_OK;
}

template <class T>
static int build_WH_T(Scene* s) {
  cudaStream_t st = s->ctx->stream;
  const int m = s->m, ns = s->ns, words = s->words;
  const int64_t ldx = s->ldx;
  T* X = (T*)s->X.p;
  if (m == 0) return ICR_OK;
  RET(dzero(s, s->bitmap.p, (size_t)ns * words * sizeof(uint32_t), "memset bitmap"));
  cudaError_t e = cudaSuccess;
  PDL("k_reach_mark", reach_mark_body, (4 * m + 255) / 256, 256, 0, st,
      (const int*)s->nodes.p, m, (const int*)s->node_super.p,
                                                     (const int*)s->parent.p, ns, (uint32_t*)s->bitmap.p, words);
  const int bt = ((words + 31) / 32) * 32;
  PDL("k_reach_rows", reach_rows_body, ns, bt, bt * sizeof(int), st,
      (const uint32_t*)s->bitmap.p, words, m, (int*)s->wprefix.p,
                                                  (int*)s->qcount.p, (int*)s->qidx.p);
  PDL("k_reach_parentpos", reach_parentpos_body, dim3((m + 255) / 256, ns), 256, 0, st,
      (const uint32_t*)s->bitmap.p, (const int*)s->wprefix.p, words, m, (const int*)s->parent.p,
      (const int*)s->qcount.p, (const int*)s->qidx.p, (int*)s->qpos.p);
  PDL("k_reach_inv", reach_inv_body, ns, 256, 0, st,
      m, (const int*)s->parent.p, (const int*)s->qcount.p, (const int*)s->qpos.p,
                                  (int*)s->qinv.p);
  const int dev = s->ctx->device;
  int gemm_occ[2] = {0, 0};   // resident blocks per SM of the 64-row and the 32-row front GEMM
  RET((gemm_occupancy<T, 4>(dev, &gemm_occ[0])));
  RET((gemm_occupancy<T, 2>(dev, &gemm_occ[1])));
  using KGemmLong = front_gemm_body<T, 4>;
  using KGemmShort = front_gemm_body<T, 2>;
  // contraction: FP32 scenes put fronts of TC_MIN_COLS or more columns on the
  // tensor cores (unless SIMT is asked for), the rest on CUDA cores
  int mode = s->params.contraction;
  if (sizeof(T) == 8) mode = ICR_CONTRACT_SIMT;
  if (mode == ICR_CONTRACT_AUTO) mode = ICR_CONTRACT_TF32X3;
  const int simt_max = mode == ICR_CONTRACT_SIMT ? (1 << 30) : TC_MIN_COLS;
  const int tc_min = mode == ICR_CONTRACT_SIMT ? (1 << 30) : TC_MIN_COLS;
  // the forward solve of wide fronts goes to the tensor cores (3xTF32) in FP32
  // scenes, except in the all-SIMT mode
  const int tc_gemm = mode != ICR_CONTRACT_SIMT ? 1 : 0;
  int* plan = (int*)s->plan.p;
  const int nlev = (int)s->levels.size();
  PDL("k_plan", plan_body, 1, 1024, 0, st,
      ns, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
                             (const int64_t*)s->rowpat_ptr.p, (const int*)s->qcount.p, simt_max, tc_min, tc_gemm,
                             (const unsigned char*)s->tc_super.p, (const int*)s->level_first.p, nlev,
                             s->ctx->sm_count, plan);
  const int nsm = s->ctx->sm_count;
  const int ntiles = (m + TCC - 1) / TCC;
  for (int li = 0; li < nlev; ++li) {
    const Level& lv = s->levels[li];
    const int pa = lv.first, pb = lv.first + lv.count;
    if (s->level_events) {
      e = cudaEventRecord(s->level_events[li], st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(level)");
    }
    const int64_t ub_a = (int64_t)lv.count * ((lv.wmax + lv.rmax + ASM_ROWS - 1) / ASM_ROWS) * ntiles;
    PDL("k_assemble", assemble_body<T>, (unsigned)std::min<int64_t>(ub_a, 4 * nsm), dim3(TCOLS, AR), 0, st,
        plan + PLAN_ASM * (ns + 1), pa, pb, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
        (const int64_t*)s->rowpat_ptr.p, (const int64_t*)s->fr_ptr.p, (const int*)s->ctr_ptr.p,
        (const int*)s->ctr_child.p, (const int*)s->ctr_row.p, (const int*)s->nodes.p, (const T*)s->bary.p,
        (const int*)s->qcount.p, (const int*)s->qidx.p, (const int*)s->qinv.p, m, X, (T*)s->Ftop.p, ldx);
    const bool short_rows = s->tc_level[li] == FWD_SIMT_SHORT;
    const int gr = short_rows ? GR_SHORT : GR_LONG;
    const int64_t ub_g = (int64_t)lv.count * ((lv.wmax + lv.rmax + gr - 1) / gr) * ntiles;
    const unsigned grid_g = (unsigned)std::min<int64_t>(ub_g, (int64_t)gemm_occ[short_rows ? 1 : 0] * nsm);
    if (short_rows)
      PDL("k_front_gemm", KGemmShort, grid_g, 256, (gemm_smem_bytes<T, 2>()), st,
          plan + PLAN_GEMM * (ns + 1), pa, pb, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
          (const int64_t*)s->rowpat_ptr.p, (const int64_t*)s->val_ptr.p, (const T*)s->G.p,
          (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, X, (const T*)s->Ftop.p, ldx);
    else
      PDL("k_front_gemm", KGemmLong, grid_g, 256, (gemm_smem_bytes<T, 4>()), st,
          plan + PLAN_GEMM * (ns + 1), pa, pb, (const int*)s->level_list.p, (const int*)s->super_ptr.p,
          (const int64_t*)s->rowpat_ptr.p, (const int64_t*)s->val_ptr.p, (const T*)s->G.p,
          (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, X, (const T*)s->Ftop.p, ldx);
    if (tc_gemm && s->tc_level[li] == FWD_TC && lv.wmax >= TC_GEMM_MIN_W) {
      const int rc = launch_front_gemm_tc(s, li);
      if (rc != ICR_OK) return rc;
    }
  }
  if (s->level_events) {
    e = cudaEventRecord(s->level_events[nlev], st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(level)");
  }
  PDL("k_scale", scale_body<T>, (s->n + 7) / 8, 256, 0, st,
      s->n, (const int*)s->dof_super.p, (const int*)s->super_ptr.p,
                                             (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p,
                                             (const double*)s->dinvsqrt.p, X, ldx);
  const int64_t nr = 3 * (int64_t)m;
  RET(dzero(s, s->WH.p, (size_t)nr * nr * sizeof(T), "memset WH"));
  {
    const int64_t ntc = (nr + CT - 1) / CT;
    const int64_t ub = (int64_t)ns * (ntc * (ntc + 1) / 2);
    PDL("k_contract", contract_body<T>, (unsigned)std::min<int64_t>(ub, 4 * nsm), 256, 0, st,
        plan + PLAN_SIMT * (ns + 1), plan + PLAN_LISTS * (ns + 1), ns, (const int*)s->level_list.p,
        (const int*)s->super_ptr.p, (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, (const int*)s->qidx.p, m,
        X, ldx, (T*)s->WH.p, nr);
  }
  if (mode != ICR_CONTRACT_SIMT) {
    const int rc = launch_contract_tc(s, mode);
    if (rc != ICR_OK) return rc;
  }
  // FP32 scenes with the BF16 W update also get W_H's BF16 copy
  __nv_bfloat16* wh16 = (sizeof(T) == 4 && s->params.w_update == ICR_W_BF16) ? (__nv_bfloat16*)s->WH16.p : nullptr;
  const unsigned nt32 = (unsigned)((nr + 31) / 32);
  PDL("k_symmetrize", symmetrize_body<T>, dim3(nt32, nt32), dim3(32, 8), 0, st, (int)nr, (T*)s->WH.p, wh16);
  return ICR_OK;
}

int launch_build_WH(Scene* s) { return s->prec == ICR_FP64 ? build_WH_T<double>(s) : build_WH_T<float>(s); }

template <class T, int WM>
static int update_W_mode(Scene* s, dim3 grid, int bc) {
  using K = update_W_body<T, WM>;
  PDL("k_update_W", K, grid, dim3(16, 16), 0, s->ctx->stream, s->m, (const T*)s->C.p, (const T*)s->WH.p,
      (const __nv_bfloat16*)s->WH16.p, (T*)s->W.p, s->ldw, (T*)s->wblk.p, bc, s->step_stop);
  return ICR_OK;
}

template <class T>
static int update_W_T(Scene* s) {
  const int m = s->m;
  if (m == 0) return ICR_OK;
  dim3 grid((m + 15) / 16, (m + 15) / 16);
  const int bc = sizeof(T) == 8 ? 16 : 32;   // the PGS block size of the scene's precision
  const size_t nb = (size_t)(m + bc - 1) / bc;
  RET(dzero(s, s->wblk.p, (size_t)m * nb * sizeof(T), "memset wblk"));
  const int wm = sizeof(T) == 4 ? s->params.w_update : ICR_W_FP32;
  if (wm == ICR_W_TF32) return update_W_mode<T, ICR_W_TF32>(s, grid, bc);
  if (wm == ICR_W_BF16) return update_W_mode<T, ICR_W_BF16>(s, grid, bc);
  return update_W_mode<T, ICR_W_FP32>(s, grid, bc);
}

int launch_update_W(Scene* s) { return s->prec == ICR_FP64 ? update_W_T<double>(s) : update_W_T<float>(s); }

template <class T>
static int wcoup_T(Scene* s) {
  const int m = s->m;
  if (m == 0) return ICR_OK;
  PDL("k_wcoup", wcoup_body<T>, (unsigned)((m + 7) / 8), 256, 0, s->ctx->stream,
      m, (const T*)s->W.p, s->ldw, (T*)s->wblk.p, sizeof(T) == 8 ? 16 : 32);
  return ICR_OK;
}

int launch_wcoup(Scene* s) { return s->prec == ICR_FP64 ? wcoup_T<double>(s) : wcoup_T<float>(s); }

template <class T, int BC>
static int pgs_T(Scene* s, int warm, int want_res) {
  cudaStream_t st = s->ctx->stream;
  const int m = s->m;
  PgsDevStats* ds = (PgsDevStats*)s->stats.p;
  RET(dzero(s, ds, sizeof(PgsDevStats), "memset stats"));
  cudaError_t e = cudaSuccess;
  if (m == 0) return ICR_OK;
  const size_t smem = pgs_smem_bytes<T, BC>(m);
  // the opt-in limit covers static plus dynamic shared memory
  static SmemLimit pgs_lim;
  int room = 0;
  if ((m + BC - 1) / BC > PGS_MAX_BLOCKS) {
    set_error("solve_friction: %d contacts exceed the single-CTA PGS block capacity", m);
    return ICR_EINVAL;
  }
  e = ensure_smem(k_pgs<T, BC>, pgs_lim, s->ctx->device, 0, &room);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes(k_pgs)");
  if (smem > (size_t)room) {
    set_error("solve_friction: %d contacts need %zu bytes of shared memory, the device allows %d", m, smem, room);
    return ICR_EINVAL;
  }
  e = ensure_smem(k_pgs<T, BC>, pgs_lim, s->ctx->device, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_pgs)");
  using KP = pgs_body<T, BC>;
  PDL("k_pgs", KP, 1, PGS_THREADS, smem, st,
      m, s->params.n_sweeps, s->params.tol, (const T*)s->W.p, s->ldw,
      (const T*)s->delta.p, (const T*)s->mu.p, (const T*)s->wblk.p, (T*)s->pgsb.p, (T*)s->lam.p, warm, ds,
      s->step_stop);
  if (want_res) {
    const double rel = sizeof(T) == 8 ? 1e-9 : 1e-5;
    PDL("k_pgs_residual", pgs_residual_body<T>, (m + 7) / 8, 256, 0, st,
        m, (const T*)s->W.p, s->ldw, (const T*)s->delta.p, (const T*)s->mu.p,
                                                   (const T*)s->lam.p, rel, ds);
  }
  return ICR_OK;
}

int launch_pgs(Scene* s, int warm, int want_res) {
  return s->prec == ICR_FP64 ? pgs_T<double, 16>(s, warm, want_res) : pgs_T<float, 32>(s, warm, want_res);
}

template <class T>
static int prox_T(Scene* s) {
  cudaStream_t st = s->ctx->stream;
  const int m = s->m;
  if (m == 0) return ICR_OK;
  double* u = (double*)s->u.p;
  const size_t smem = 3 * (size_t)m * sizeof(T);
  if (smem <= 48 * 1024) {   // u_k fits the default shared memory: one launch
    PDL("k_prox", prox_body<T>, (3 * m + 15) / 16, 512, smem, st, m, (const T*)s->C.p, (const T*)s->lam.p,
        (const T*)s->WH.p, u, (double*)s->p.p, u + 3 * (size_t)m, s->step_stop);
    return ICR_OK;
  }
  PDL("k_prox_u", prox_u_body<T>, (m + 127) / 128, 128, 0, st,
      m, (const T*)s->C.p, (const T*)s->lam.p, (T*)s->uk.p, u, s->step_stop);
  PDL("k_prox_p", prox_p_body<T>, (3 * m + 7) / 8, 256, 0, st,
      m, (const T*)s->WH.p, (const T*)s->uk.p, (double*)s->p.p, u + 3 * (size_t)m, s->step_stop);
  return ICR_OK;
}

// one thread per contact: its entries of every per-contact buffer
template <class T>
__device__ __forceinline__ void d_reset_contacts(const VB& vb, int mm, T* lam, T* lam0, T* mu, T* delta, T* C,
                                                 double* p, double* p0, double* u, int* stats, int nstats,
                                                 int* dev_err) {
  const int a = vb.bx * blockDim.x + threadIdx.x;
  if (a < mm) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lam[3 * a + j] = T(0);
      lam0[3 * a + j] = T(0);
      delta[3 * a + j] = T(0);
      p[3 * a + j] = 0.0;
      p0[3 * a + j] = 0.0;
      u[3 * a + j] = 0.0;
      u[3 * (size_t)mm + 3 * a + j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) C[9 * a + j] = T(0);
    mu[a] = T(0);
  }
  if (a < nstats) stats[a] = 0;
  if (a == 0) *dev_err = 0;
}

template <class T>
__global__ void k_reset_contacts(int mm, T* lam, T* lam0, T* mu, T* delta, T* C, double* p, double* p0, double* u,
                                 int* stats, int nstats, int* dev_err) {
  pdl_entry();
  d_reset_contacts<T>(own_block(), mm, lam, lam0, mu, delta, C, p, p0, u, stats, nstats, dev_err);
}

template <class T>
struct reset_contacts_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_reset_contacts<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_reset_contacts<T>(vb, a...);
  }
};

// one thread per contact: the inputs of icr_set_step_inputs from the staging
// buffer, and the contact state reset as in k_reset_contacts
template <class T>
__device__ __forceinline__ void d_unpack_inputs(const VB& vb, int m, int nsph, const unsigned char* __restrict__ stg,
                                                int64_t o_nodes, int64_t o_of, int64_t o_bary, int64_t o_mu,
                                                int64_t o_p0, int64_t o_anch, int64_t o_sph, int* nodes,
                                                int* sphere_of, T* bary, T* mu, double* p, double* p0,
                                                double* anchors, double* spheres, T* lam, T* lam0, T* delta, T* C,
                                                double* u, int* stats, int nstats, int* dev_err) {
  const int a = vb.bx * blockDim.x + threadIdx.x;
  if (a < m) {
    const int* sn = (const int*)(stg + o_nodes);
    const T* sb = (const T*)(stg + o_bary);
    const double* sp = (const double*)(stg + o_p0);
    const double* sa = (const double*)(stg + o_anch);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      nodes[4 * a + j] = sn[4 * a + j];
      bary[4 * a + j] = sb[4 * a + j];
    }
    sphere_of[a] = ((const int*)(stg + o_of))[a];
    mu[a] = ((const T*)(stg + o_mu))[a];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      p[3 * a + j] = sp[3 * a + j];
      p0[3 * a + j] = sp[3 * a + j];
      anchors[3 * a + j] = sa[3 * a + j];
      lam[3 * a + j] = T(0);
      lam0[3 * a + j] = T(0);
      delta[3 * a + j] = T(0);
      u[3 * a + j] = 0.0;
      u[3 * (size_t)m + 3 * a + j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) C[9 * a + j] = T(0);
  }
  if (a < 4 * nsph) spheres[a] = ((const double*)(stg + o_sph))[a];
  if (a < nstats) stats[a] = 0;
  if (a == 0) *dev_err = 0;
}

template <class T>
__global__ void k_unpack_inputs(int m, int nsph, const unsigned char* __restrict__ stg, int64_t o_nodes,
                                int64_t o_of, int64_t o_bary, int64_t o_mu, int64_t o_p0, int64_t o_anch,
                                int64_t o_sph, int* nodes, int* sphere_of, T* bary, T* mu, double* p, double* p0,
                                double* anchors, double* spheres, T* lam, T* lam0, T* delta, T* C, double* u,
                                int* stats, int nstats, int* dev_err) {
  pdl_entry();
  d_unpack_inputs<T>(own_block(), m, nsph, stg, o_nodes, o_of, o_bary, o_mu, o_p0, o_anch, o_sph, nodes, sphere_of,
                     bary, mu, p, p0, anchors, spheres, lam, lam0, delta, C, u, stats, nstats, dev_err);
}

template <class T>
struct unpack_inputs_body {
  static constexpr int threads = 256, minb = 1;
  static constexpr bool stride = false;
  static auto kernel() { return &k_unpack_inputs<T>; }
  template <class... A>
  __device__ __forceinline__ static void run(const VB& vb, A... a) {
    d_unpack_inputs<T>(vb, a...);
  }
};

template <class T>
static int unpack_T(Scene* s, int nsph, const int64_t* o) {
  const int m = s->m;
  const int nstats = (int)(sizeof(PgsDevStats) / sizeof(int));
  const int n = std::max(std::max(m, 4 * nsph), nstats);
  PDL("k_unpack_inputs", unpack_inputs_body<T>, (n + 255) / 256, 256, 0, s->ctx->stream, m, nsph,
      (const unsigned char*)s->stage_dev.p, o[0], o[1], o[2], o[3], o[4], o[5], o[6], (int*)s->nodes.p,
      (int*)s->obst_of.p, (T*)s->bary.p, (T*)s->mu.p, (double*)s->p.p, (double*)s->p0.p,
      (double*)s->obst_anchors.p, (double*)s->obst_spheres.p, (T*)s->lam.p, (T*)s->lam0.p, (T*)s->delta.p,
      (T*)s->C.p, (double*)s->u.p, (int*)s->stats.p, nstats, (int*)s->dev_err.p);
  return ICR_OK;
}

int launch_unpack_inputs(Scene* s, int n_spheres, const int64_t* off) {
  return s->prec == ICR_FP64 ? unpack_T<double>(s, n_spheres, off) : unpack_T<float>(s, n_spheres, off);
}

template <class T>
static int reset_T(Scene* s, int mm) {
  const int nstats = (int)(sizeof(PgsDevStats) / sizeof(int));
  PDL("k_reset_contacts", reset_contacts_body<T>, (std::max(mm, nstats) + 255) / 256, 256, 0, s->ctx->stream, mm,
      (T*)s->lam.p, (T*)s->lam0.p, (T*)s->mu.p, (T*)s->delta.p, (T*)s->C.p, (double*)s->p.p, (double*)s->p0.p,
      (double*)s->u.p, (int*)s->stats.p, nstats, (int*)s->dev_err.p);
  return ICR_OK;
}

int launch_reset_contacts(Scene* s, int mm) {
  return s->prec == ICR_FP64 ? reset_T<double>(s, mm) : reset_T<float>(s, mm);
}

int launch_update_proximity(Scene* s) { return s->prec == ICR_FP64 ? prox_T<double>(s) : prox_T<float>(s); }

template <class T>
static int correct_T(Scene* s) {
  cudaStream_t st = s->ctx->stream;
  const int m = s->m, n = s->n;
  if (m == 0) {
    return dzero(s, s->dq.p, (size_t)n * sizeof(T), "memset dq");
  }
  const T* uw = (const T*)s->u.p;   // FP64: u as it is
  if (sizeof(T) == 4) {
    PDL("k_u_round", u_round_body<T>, (3 * m + 255) / 256, 256, 0, st, 3 * m, (const double*)s->u.p, (T*)s->uk.p);
    uw = (const T*)s->uk.p;
  }
  PDL("k_xu", xu_body<T>, (n + 7) / 8, 256, 0, st,
      n, (const int*)s->dof_super.p, (const int*)s->super_ptr.p,
                                       (const int64_t*)s->fr_ptr.p, (const int*)s->qcount.p, (const int*)s->qidx.p,
                                       m, (const T*)s->X.p, s->ldx, uw, (const double*)s->dinvsqrt.p,
                                       (T*)s->y.p);
  for (int l = (int)s->levels.size() - 1; l >= 0; --l) {
    const Level& lv = s->levels[l];
    const int nchunk = (lv.wmax + 7) / 8;
    PDL("k_bsolve", bsolve_body<T>, lv.count * nchunk, 256, 0, st,
        (const int*)s->level_list.p, lv.first, nchunk,
                                                   (const int*)s->super_ptr.p, (const int64_t*)s->rowpat_ptr.p,
                                                   (const int*)s->rowpat.p, (const int64_t*)s->val_ptr.p,
                                                   (const T*)s->G.p, (const T*)s->y.p, (T*)s->dq.p);
  }
  return ICR_OK;
}

int launch_correct_motion(Scene* s) { return s->prec == ICR_FP64 ? correct_T<double>(s) : correct_T<float>(s); }

template <class T>
static int linearize_T(Scene* s, int k) {
  const int m = s->m;
  if (m == 0) return ICR_OK;
  const double* nk = s->obst_kind == 1 ? (const double*)s->obst_normals.p + (size_t)k * m * 3 : nullptr;
  PDL("k_linearize", linearize_body<T>, (m + 127) / 128, 128, 0, s->ctx->stream,
      m, s->obst_kind, nk, (const double*)s->obst_anchors.p, (const double*)s->obst_spheres.p,
      (const int*)s->obst_of.p, (const double*)s->p.p, (T*)s->C.p, (T*)s->delta.p, s->step_stop);
  return ICR_OK;
}

template <class T>
static int newton_check_T(Scene* s) {
  const int m = s->m;
  if (m == 0) return ICR_OK;
  PDL("k_newton_check", newton_check_body<T>, 1, 1024, 0, s->ctx->stream, m, (const T*)s->delta.p,
      s->params.newton_tol, (int*)s->newton.p);
  return ICR_OK;
}

int launch_newton_check(Scene* s) {
  return s->prec == ICR_FP64 ? newton_check_T<double>(s) : newton_check_T<float>(s);
}

int launch_linearize(Scene* s, int k) { return s->prec == ICR_FP64 ? linearize_T<double>(s, k) : linearize_T<float>(s, k); }

}  // namespace icr
