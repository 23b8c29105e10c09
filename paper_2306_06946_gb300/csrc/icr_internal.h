// Internal declarations of libicr: scene state and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "icr.h"

namespace icr {

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);

struct Ctx {
  int device = 0;
  int sm_count = 1;
  cudaStream_t stream = nullptr;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  uint64_t wait_ns = 1000000000ull;   // bound of the tensor-core kernels' pipeline waits
  int64_t fail_alloc_after = -1;      // failure injection: allocations left before one fails (-1: off)
  int scenes = 0;          // live scenes; the context is freed after the last one
  bool destroyed = false;  // icr_ctx_destroy was called while scenes were alive
};

// Device buffer owned by a scene, accounted against the context budget.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  uint64_t gen = 0;   // allocation generation (changes with every cudaMalloc behind it)
};

// Work lists of one W_H build, written on the device by the planner right
// after the reach pass: for every position p of level_list (p = 0..ns), the
// exclusive prefix sum of the work units the supernodes before p contribute to
// each list.  A kernel over a level range [a, b) of positions covers units
// plan[a] .. plan[b] - 1; the unit's supernode is found by binary search.
// Lists: assembly tiles, SIMT front-GEMM tiles, tensor-core front-GEMM tiles,
// packed F_top blocks, SIMT contraction tile pairs, packed Y blocks,
// tensor-core contraction tile pairs.  After the lists come the scheduling
// counters: SIMT contraction, tensor-core contraction, then one per level for
// the tensor-core front GEMM.
enum PlanList {
  PLAN_ASM = 0, PLAN_GEMM = 1, PLAN_GTC = 2, PLAN_FPACK = 3, PLAN_SIMT = 4, PLAN_PACK = 5, PLAN_TC = 6,
  PLAN_LISTS = 7
};
enum PlanCounter { PLAN_CNT_SIMT = 0, PLAN_CNT_TC = 1, PLAN_CNT_GTC = 2 };
// Forward-solve tile shape of an etree level (icr_autotune / icr_set_forward_plan):
// CUDA-core tiles of 64 front rows x 96 columns, tcgen05 tiles of 128 x 128 for
// the level's fronts at least TC_GEMM_MIN_W wide (the others on 64-row tiles),
// or CUDA-core tiles of 32 front rows x 96 columns.
enum FwdTile { FWD_SIMT = 0, FWD_TC = 1, FWD_SIMT_SHORT = 2, FWD_TILES = 3 };
constexpr int GR_LONG = 64, GR_SHORT = 32;   // front rows of the two CUDA-core tiles
constexpr int TC_TILE = 128;         // tensor-core output tile (M = N)
constexpr int TC_KT = 32;            // front rows (K) per packed operand block
// bytes of one packed operand block in the widest mode (3xTF32: two TF32 planes)
constexpr size_t TC_BLOCK_BYTES = (size_t)TC_TILE * TC_KT * 4 * 2;
constexpr int TC_GEMM_MIN_W = 64;    // fronts at least this wide ...
constexpr int TC_GEMM_MIN_COLS = 64; // ... and with this many columns take the tensor-core forward solve
constexpr int TC_PART_KB = 2;        // fewest K blocks (64 K) in a part of a split tensor-core unit
constexpr int TC_MAX_SPLIT = 8;      // most K parts of a tensor-core unit
constexpr int PLAN_MAX_LEV = 128;    // levels with their own K split (deeper ones are not split)
// K parts of a tensor-core unit over nk K blocks, given the split factor of
// its list (k_plan: about one unit per SM when the list has few tiles)
__host__ __device__ inline int tc_parts(int split, int nk) {
  const int most = nk / TC_PART_KB;
  const int n = split < most ? split : most;
  return n < 1 ? 1 : n;
}

// Per-level launch geometry of the supernodal elimination tree.
struct Level {
  int first = 0;   // offset into level_list
  int count = 0;   // supernodes in the level
  int wmax = 0;    // widest supernode
  int rmax = 0;    // most below-diagonal rows
};

// Opt-in per-launch timing of a scene (icr_profile_begin / icr_profile_end):
// an event pair around every eagerly launched kernel, tagged with its name.
// Never active while a stream is captured.
struct Profiler {
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;   // events of earlier profiles, reused
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
  }
  void recycle() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  ~Profiler() {
    recycle();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct BatchRec;

// parameters compared field by field: the struct has padding, whose bytes a
// copy need not keep
static_assert(sizeof(icr_params) == 40, "a new icr_params field must be compared in same_params");
inline bool same_params(const icr_params& a, const icr_params& b) {
  return a.precision == b.precision && a.n_sweeps == b.n_sweeps && a.tol == b.tol && a.contraction == b.contraction &&
         a.warm_start == b.warm_start && a.w_update == b.w_update && a.newton_tol == b.newton_tol;
}

struct Scene {
  Ctx* ctx = nullptr;
  Profiler* prof = nullptr;   // per-launch timing while profiling
  BatchRec* rec = nullptr;    // while an icr_batch records the scene's step: launches are recorded, not made
  int batches = 0;            // live icr_batch objects that hold this scene
  icr_params params{};
  int prec = ICR_FP32;
  size_t tsize = 4;

  // ---- system (set_system)
  bool has_system = false;
  int n = 0, ns = 0, n_nodes = 0;
  std::vector<int32_t> h_super_ptr, h_parent, h_qcount;
  std::vector<int64_t> h_rowpat_ptr, h_val_ptr, h_fr_ptr;
  std::vector<Level> levels;
  int64_t total_front_rows = 0;
  int wmax = 0, rmax = 0;
  DBuf super_ptr, rowpat_ptr, rowpat, val_ptr, G, dinv, dinvsqrt, parent;  // G: per-supernode solve operators
  DBuf child_ptr, child_list, relidx, level_list, node_super, dof_super, fr_ptr;
  DBuf ctr_ptr, ctr_child, ctr_row;   // per front row: (child, child row) pairs of the extend-add

  // ---- mapping (set_mapping)
  bool has_mapping = false;
  int m = 0, words = 0;
  int64_t ldx = 0;     // leading dimension (columns) of every front
  int64_t ldw = 0;     // leading dimension of W: 3m rounded up to 96 (16-byte aligned row blocks)
  DBuf nodes, bary, bitmap, wprefix, qcount, qidx, qpos, qinv, X, Ftop;  // Ftop: assembled top rows (n x ldx)
  DBuf WH, W, C, delta, mu, lam, lam0, p, p0, u, uk, y, dq, stats;
  DBuf wblk;    // per contact a and PGS block B (m x ceil(m / block)): max |W[3a, j]| over B's columns
                //   other than a's own (the coupling bound of the PGS's S-only sweeps)
  DBuf WH16;    // BF16 copy of W_H (FP32 scenes with the BF16 W update)
  DBuf pgsb;    // PGS S-only sweeps (2m): each passed-over contact's residual bound at the base, its coupling to S
  DBuf newton;  // device Newton stop: [0] the loop has ended, [1] iterations run after the first
  const int* step_stop = nullptr;   // while a device-resident step is enqueued with newton_tol: newton.p
  int last_newton = 0;              // n_newton of the last device-resident step
  bool last_newton_tol = false;     // ... and whether newton_tol could end it early
  DBuf plan;   // PLAN_LISTS x (ns + 1) prefix sums, 2 + levels counters, levels + 1 K splits (int32)
  DBuf level_first;   // (levels + 1) offsets of the levels in level_list
  // icr_set_step_inputs: device staging buffer, two pinned host slots, their copy events
  DBuf stage_dev;
  unsigned char* stage_host[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  bool stage_used[2] = {false, false};
  int stage_slot = 0;
  DBuf Gpk, gpk_off;   // G_s of the wide supernodes as 3xTF32 operand blocks; first block per supernode
  // forward-solve engine per etree level: 1 puts the level's wide fronts on the
  // tensor cores (chosen by icr_autotune), mirrored per supernode for the planner
  std::vector<uint8_t> tc_level;
  std::vector<int32_t> h_level_list;
  DBuf tc_super;
  bool tuned = false;
  cudaEvent_t* level_events = nullptr;   // while tuning: recorded before every level and after the last
  DBuf dev_err;            // int set by a kernel whose bounded wait ran out
  DBuf Ypk, tc_boff;       // packed tensor-core operand blocks and each supernode's first block
  int tc_tmax = 0;         // 128-column tiles of the widest possible front
  uint64_t W_zeroed = 0;   // allocation generation of W whose padding is known to be zero, for ld and rows
  int64_t W_zeroed_ld = 0, W_zeroed_rows = 0;
  uint64_t launches = 0;   // kernels launched by this scene
  cudaGraphExec_t step_graph = nullptr;   // captured icr_step
  uint64_t graph_kernels = 0;             // kernels in the captured step
  // the graph holds device addresses and launch shapes: it stays valid while no
  // buffer has been reallocated (alloc_epoch), and the contact count, obstacle
  // kind, parameters and Newton count are those it was captured with
  uint64_t alloc_epoch = 0, graph_epoch = 0;
  int graph_m = -1, graph_obst = -1, graph_newton = -1;
  icr_params graph_params{};
  bool has_WH = false, has_dirs = false, has_W = false, has_lam = false;

  // ---- eviction (icr_scene_evict / icr_scene_readmit)
  bool evicted = false;
  struct Saved {
    DBuf* b;
    void* host;   // pinned copy of a kept buffer
    size_t bytes;
  };
  std::vector<Saved> saved;                              // kept buffers' contents while evicted
  std::vector<std::pair<DBuf*, size_t>> evicted_sizes;   // every buffer's size while evicted
  uint64_t resident_bytes = 0;                           // device bytes the scene held when evicted
  bool recapture = false;                                // a step graph existed when it was evicted

  // ---- obstacle (device linearisation)
  int obst_kind = 0;   // 0 none, 1 plane, 2 sphere
  int obst_iters = 0;
  DBuf obst_normals, obst_anchors;
  DBuf obst_spheres, obst_of;   // sphere tools (n x 4 doubles) and each contact's tool (m int32)
};

int dalloc(Scene* s, DBuf& b, size_t bytes);
void dfree(Scene* s, DBuf& b);
// every device buffer of a scene (not the input staging buffer), with
// whether an eviction keeps its contents (the rest is rebuilt by every step)
void scene_buffers(Scene* s, std::vector<std::pair<DBuf*, bool>>& out);
int scene_evict(Scene* s);
int scene_readmit(Scene* s);

// Device statistics written by the PGS kernels (FP64 residual check).
struct PgsDevStats {
  int32_t sweeps;
  int32_t n_sep, n_stick, n_slip;
  int32_t s_only, folds;   // sweeps over S only; deferred folds
  int32_t rechecks;        // rechecks of the passed-over contacts when the coupling bound ran out
  int32_t joins;           // rechecks after which blocks joined S
  double eps;
  unsigned long long res_bits[4];   // normal, cone, stick, slip as non-negative double bits
};

// ---- launchers (icr_kernels.cu); every one enqueues on s->ctx->stream
int launch_build_WH(Scene* s);
int launch_update_W(Scene* s);
int launch_wcoup(Scene* s);   // the coupling bounds (wblk) of a W given directly
// scatter a packed staging buffer into the per-contact inputs and reset the
// contact state (offsets in bytes: nodes, sphere ids, bary, mu, p0, anchors, spheres)
int launch_unpack_inputs(Scene* s, int n_spheres, const int64_t* off);
int launch_pgs(Scene* s, int warm_start, int want_residuals);
int launch_update_proximity(Scene* s);
int launch_correct_motion(Scene* s);
int launch_linearize(Scene* s, int k);
int launch_newton_check(Scene* s);
// tcgen05 contraction for supernodes with at least min_cols front columns (icr_tc.cu)
int launch_contract_tc(Scene* s, int mode);
int launch_pack_g(Scene* s, const int32_t* blocks, int nblocks);
int launch_front_gemm_tc(Scene* s, int level);
// zero lambda~, its warm start, mu, delta, C, p, p_0, u, the PGS stats and the
// device error word of mm contacts in one launch
int launch_reset_contacts(Scene* s, int mm);
int check_step_graph(Scene* s, const char* where);

// Kernel launches of the time step use programmatic dependent launch outside
// graph capture: a kernel's CTAs may be scheduled while the previous kernel on
// the stream finishes.  Every library kernel therefore starts with pdl_entry():
// griddepcontrol.wait returns once the preceding kernels have completed and
// their writes are visible, and launch_dependents lets the next kernel be
// scheduled early.  Without a programmatic dependency both return at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <class... KArgs, class... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  // inside a captured graph the nodes are already launched back to back, and
  // programmatic edges measured slower there: plain edges when capturing
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Per-device set-up of a kernel's dynamic shared-memory limit (the attribute
// belongs to the current device); thread-safe, a driver call only when the
// limit grows.  `room` (may be NULL) receives the dynamic bytes the device
// allows next to the kernel's static shared memory.
struct SmemLimit {
  std::atomic<int> bytes[64];
};
template <class K>
cudaError_t ensure_smem(K kernel, SmemLimit& lim, int device, int bytes, int* room = nullptr) {
  if (room) {
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    *room = optin - (int)fa.sharedSizeBytes;
  }
  const bool cached = device >= 0 && device < 64;
  if (cached && lim.bytes[device].load() >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && cached) {
    int cur = lim.bytes[device].load();
    while (cur < bytes && !lim.bytes[device].compare_exchange_weak(cur, bytes)) {
    }
  }
  return e;
}

// Per-device cache of an occupancy figure (0: not yet known).
struct DevInt {
  std::atomic<int> v[64];
  int get(int device) const { return device >= 0 && device < 64 ? v[device].load() : 0; }
  void put(int device, int x) {
    if (device >= 0 && device < 64) v[device].store(x);
  }
};

// events around a launch while the scene is profiled (not during capture)
int prof_mark(Scene* s, const char* name, bool after);

// ---------------------------------------------------------------- batched launches
// A kernel body reads its block index and grid size from a VB instead of
// blockIdx / gridDim.  A single-scene launch passes its own (own_block());
// a batched launch (icr_batch) runs the bodies of many scenes in one flat
// grid, each scene's blocks numbered as in that scene's own launch.
struct VB {
  unsigned bx, by, gx, gy;
};
__device__ __forceinline__ VB own_block() { return VB{blockIdx.x, blockIdx.y, gridDim.x, gridDim.y}; }

// The arguments of one launch, stored by value (a small tuple whose layout is
// the same on the host and the device: it is copied into device memory).
template <class... A>
struct Args;
template <>
struct Args<> {};
template <class H, class... R>
struct Args<H, R...> {
  H h;
  Args<R...> r;
};
inline Args<> make_args() { return Args<>{}; }
template <class H, class... R>
Args<H, R...> make_args(H h, R... r) {
  return Args<H, R...>{h, make_args(r...)};
}
// K::run(d..., the stored arguments in order)
template <class K, class... D>
__device__ __forceinline__ void apply_args(const Args<>&, D... d) {
  K::run(d...);
}
template <class K, class H, class... R, class... D>
__device__ __forceinline__ void apply_args(const Args<H, R...>& a, D... d) {
  apply_args<K>(a.r, d..., a.h);
}

// One scene's part of a batched launch: its own grid and its arguments.
template <class P>
struct BatchSlot {
  unsigned gx, gy;
  P args;
};

// Batched launch of body K.  Bodies whose work units any grid covers
// (K::stride: a grid-stride loop or a counter over the scene's device work
// list) run persistently: every block serves every slot in turn, heaviest
// scene first, as block bx of a grid of gridDim.x.  Otherwise slot i owns the
// flat blocks [first[i], first[i+1]) and its blocks run K's body with the
// block index of the scene's own launch.
template <class K, class P>
__global__ void __launch_bounds__(K::threads, K::minb)
    k_batch(const BatchSlot<P>* __restrict__ slots, const unsigned* __restrict__ first, int nslots) {
  pdl_entry();
  if constexpr (K::stride) {
    for (int i = 0; i < nslots; ++i) {
      apply_args<K>(slots[i].args, VB{blockIdx.x, 0u, gridDim.x, 1u});
      __syncthreads();   // the next scene's units reuse the shared memory
    }
    return;
  }
  __shared__ int slot_sh;
  const unsigned b = blockIdx.x;
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0) slot_sh = -1;
  __syncthreads();
  for (int i = tid; i < nslots; i += nt)
    if (first[i] <= b && b < first[i + 1]) slot_sh = i;   // exactly one slot
  __syncthreads();
  const int i = slot_sh;
  if (i < 0) return;   // uniform; cannot happen with the offsets the host checked
  const BatchSlot<P>& sl = slots[i];
  const unsigned local = b - first[i];
  apply_args<K>(sl.args, VB{local % sl.gx, local / sl.gx, sl.gx, sl.gy});
}

// A device-to-device copy (src != NULL) or a zero fill of `bytes` bytes.
struct MemOp {
  void* dst;
  const void* src;
  unsigned long long bytes;
};

using BatchLaunchFn = cudaError_t (*)(const void* slots, const unsigned* first, int nslots, unsigned nblocks,
                                      dim3 block, size_t smem, cudaStream_t st, int device);

template <class K, class P>
cudaError_t batch_launch(const void* slots, const unsigned* first, int nslots, unsigned nblocks, dim3 block,
                         size_t smem, cudaStream_t st, int device) {
  static SmemLimit lim;
  if (smem > 48 * 1024) {
    const cudaError_t e = ensure_smem(k_batch<K, P>, lim, device, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_batch<K, P><<<nblocks, block, smem, st>>>(static_cast<const BatchSlot<P>*>(slots), first, nslots);
  return cudaGetLastError();
}

// One recorded launch of a scene's step: a kernel (launch != NULL, one slot)
// or a group of independent copies and fills (launch == NULL).
struct BatchEntry {
  const char* name = nullptr;
  BatchLaunchFn launch = nullptr;
  dim3 block;
  size_t smem = 0;
  unsigned blocks = 0;                // blocks of the scene's own launch
  size_t slot_align = 0;
  bool stride = false;                // K::stride: one persistent grid serves every slot
  std::vector<unsigned char> slot;    // the BatchSlot<P> bytes
  std::vector<MemOp> ops;
};
struct BatchRec {
  std::vector<BatchEntry> entries;
};

template <class K, class... KArgs, class... A>
int batch_record(BatchRec* rec, const char* where, void (*)(KArgs...), dim3 grid, dim3 block, size_t smem,
                 A... a) {
  using P = Args<KArgs...>;
  if (grid.z != 1) {
    set_error("%s: a batched launch takes a 1-D or 2-D grid", where);
    return ICR_EINVAL;
  }
  if ((uint64_t)grid.x * grid.y == 0) return ICR_OK;   // nothing to run
  const BatchSlot<P> sl{grid.x, grid.y, make_args(static_cast<KArgs>(a)...)};
  BatchEntry e;
  e.name = where;
  e.launch = &batch_launch<K, P>;
  e.block = block;
  e.smem = smem;
  e.blocks = grid.x * grid.y;
  e.slot_align = alignof(BatchSlot<P>);
  e.stride = K::stride;
  e.slot.assign(reinterpret_cast<const unsigned char*>(&sl), reinterpret_cast<const unsigned char*>(&sl) + sizeof(sl));
  rec->entries.push_back(std::move(e));
  return ICR_OK;
}

// Zero fill and device-to-device copy on the scene's stream (recorded while a
// batch records the scene's step).
int dzero(Scene* s, void* p, size_t bytes, const char* where);
int dcopy(Scene* s, void* dst, const void* src, size_t bytes, const char* where);
// the device-resident time step (icr_step), enqueued or recorded
int step_enqueue(Scene* s, int n_newton);

// Launch body tag K (K::kernel() is its single-scene kernel) through
// pdl_launch, check it and count it in the scene `s` in scope; while the
// scene is recorded by a batch, record the launch instead.
#define PDL(where, K, grid, block, smem, st, ...)                                                          \
  do {                                                                                                  \
    if (s->rec) {                                                                                       \
      const int rc_ = batch_record<K>(s->rec, where, K::kernel(), dim3(grid), dim3(block), (size_t)(smem), \
                                      __VA_ARGS__);                                                     \
      if (rc_ != ICR_OK) return rc_;                                                                    \
      break;                                                                                            \
    }                                                                                                   \
    if (s->prof) {                                                                                      \
      const int rc_ = prof_mark(s, where, false);                                                       \
      if (rc_ != ICR_OK) return rc_;                                                                    \
    }                                                                                                   \
    const cudaError_t e_ = pdl_launch(K::kernel(), grid, block, smem, st, __VA_ARGS__);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, where);                                                 \
    ++s->launches;                                                                                      \
    if (s->prof) {                                                                                      \
      const int rc_ = prof_mark(s, where, true);                                                        \
      if (rc_ != ICR_OK) return rc_;                                                                    \
    }                                                                                                   \
  } while (0)
// return a non-OK status of a call
#define RET(call)                \
  do {                           \
    int r_ = (call);             \
    if (r_ != ICR_OK) return r_; \
  } while (0)

// ICR_ETIMEOUT when a kernel reported a bounded wait that ran out (synchronises)
int check_device_error(Scene* s);

}  // namespace icr
