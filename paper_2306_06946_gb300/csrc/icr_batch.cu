// Batched time steps: many scenes stepped by one captured CUDA graph in which
// every kernel launch covers many of them (Alg. 3 per scene; the scenes are
// independent problems).
//
// A batch records the device-resident step of each of its scenes (the launch
// sequence icr_step would make: kernels with their grids and arguments, plus
// device copies and fills) instead of launching it.  The scenes are split into
// cost-balanced groups; within a group the per-scene sequences are merged into
// one, and a launch of the merged sequence runs one kernel body for every
// scene whose recorded launch it takes over (k_batch): either one flat grid in
// which each scene's blocks see the block index of the scene's own launch, or,
// for bodies whose work units any grid covers, one persistent grid that serves
// every scene in turn.  So each scene runs exactly its own step, and the
// kernels of different scenes share launches, waves and SMs.  Each scene's
// launches stay in its own order; scenes never wait on one another inside a
// launch.  The groups run as parallel branches of the graph.
//
// The merge (merge_sequences) builds a common supersequence of the scenes'
// sequences by pairwise longest-common-subsequence alignment.  The merged
// sequence and its argument slots are fixed at creation; the graph replays
// them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "icr_internal.h"

struct icr_scene : icr::Scene {};

namespace icr {
namespace {

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// appends op to the scene's recorded step: into the last entry when that is
// a group of copies and fills none of which touches op's bytes
int rec_memop(BatchRec* rec, const MemOp& op, const char* where) {
  if (!rec->entries.empty() && rec->entries.back().launch == nullptr) {
    bool free_of = true;
    for (const MemOp& o : rec->entries.back().ops)
      free_of = free_of && !overlaps(o.dst, o.bytes, op.dst, op.bytes) && !overlaps(o.dst, o.bytes, op.src, op.bytes) &&
                !overlaps(o.src, o.bytes, op.dst, op.bytes);
    if (free_of) {
      rec->entries.back().ops.push_back(op);
      return ICR_OK;
    }
  }
  BatchEntry e;
  e.name = where;
  e.ops.push_back(op);
  rec->entries.push_back(std::move(e));
  return ICR_OK;
}

constexpr int MEMOP_THREADS = 256;
// blocks of a copy or fill: about four 16-byte words per thread, at most 512
unsigned memop_blocks(unsigned long long bytes) {
  const unsigned long long per = (unsigned long long)MEMOP_THREADS * 16 * 4;
  return (unsigned)std::min<unsigned long long>(512, std::max<unsigned long long>(1, (bytes + per - 1) / per));
}

// The copies and fills of one merged launch: op i owns the flat blocks
// [first[i], first[i+1]); 16-byte words when both ends and the size allow,
// else 4-byte words, else bytes.
__global__ void __launch_bounds__(MEMOP_THREADS)
    k_batch_memops(const MemOp* __restrict__ ops, const unsigned* __restrict__ first, int nops) {
  pdl_entry();
  __shared__ int op_sh;
  if (threadIdx.x == 0) op_sh = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nops; i += blockDim.x)
    if (first[i] <= blockIdx.x && blockIdx.x < first[i + 1]) op_sh = i;
  __syncthreads();
  const int k = op_sh;
  if (k < 0) return;   // uniform; cannot happen with the offsets the host checked
  const MemOp op = ops[k];
  const unsigned long long nthr = (unsigned long long)(first[k + 1] - first[k]) * blockDim.x;
  const unsigned long long t0 = (unsigned long long)(blockIdx.x - first[k]) * blockDim.x + threadIdx.x;
  const uintptr_t al = (uintptr_t)op.dst | (uintptr_t)op.src | (uintptr_t)op.bytes;
  if ((al & 15) == 0) {
    uint4* d = static_cast<uint4*>(op.dst);
    const uint4* s = static_cast<const uint4*>(op.src);
    for (unsigned long long i = t0; i < op.bytes / 16; i += nthr) d[i] = s ? s[i] : make_uint4(0u, 0u, 0u, 0u);
  } else if ((al & 3) == 0) {
    uint32_t* d = static_cast<uint32_t*>(op.dst);
    const uint32_t* s = static_cast<const uint32_t*>(op.src);
    for (unsigned long long i = t0; i < op.bytes / 4; i += nthr) d[i] = s ? s[i] : 0u;
  } else {
    unsigned char* d = static_cast<unsigned char*>(op.dst);
    const unsigned char* s = static_cast<const unsigned char*>(op.src);
    for (unsigned long long i = t0; i < op.bytes; i += nthr) d[i] = s ? s[i] : (unsigned char)0;
  }
}

// relative cost of a scene's step: the dense bound of the forward solve's
// right-hand sides (n x 3m) plus the PGS sweep work ((3m)^2)
double scene_cost(const Scene* s) { return (double)s->n * 3.0 * s->m + 9.0 * (double)s->m * s->m; }

// identity of a recorded launch for merging: its batched launcher and block
// shape (NULL launcher: copies and fills)
struct Key {
  BatchLaunchFn fn;
  unsigned x, y, z;
  bool operator==(const Key& o) const { return fn == o.fn && x == o.x && y == o.y && z == o.z; }
};
Key key_of(const BatchEntry& e) {
  if (!e.launch) return Key{nullptr, 0, 0, 0};
  return Key{e.launch, e.block.x, e.block.y, e.block.z};
}

}  // namespace

int dzero(Scene* s, void* p, size_t bytes, const char* where) {
  if (bytes == 0) return ICR_OK;
  if (s->rec) return rec_memop(s->rec, MemOp{p, nullptr, bytes}, where);
  const cudaError_t e = cudaMemsetAsync(p, 0, bytes, s->ctx->stream);
  return e == cudaSuccess ? ICR_OK : cuda_fail(e, where);
}

int dcopy(Scene* s, void* dst, const void* src, size_t bytes, const char* where) {
  if (bytes == 0) return ICR_OK;
  if (s->rec) return rec_memop(s->rec, MemOp{dst, src, bytes}, where);
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s->ctx->stream);
  return e == cudaSuccess ? ICR_OK : cuda_fail(e, where);
}

// Merge of per-scene launch sequences (keys[s] in order) into one sequence of
// shared launches: a common supersequence of all of them, built progressively.
// The sequences are taken longest first; each is merged into the supersequence
// so far through a longest common subsequence of the two (dynamic programming:
// the shortest common supersequence of the pair), so that a launch of the new
// sequence joins an existing launch of the same key wherever the orders allow.
// Every output launch lists the scenes it covers, in ascending order; each
// scene's launches appear in its own order, one per output launch.
void merge_sequences(const std::vector<std::vector<int>>& keys, std::vector<std::vector<int>>& out_scenes,
                     std::vector<int>& out_key) {
  const int n = (int)keys.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return keys[a].size() > keys[b].size(); });
  std::vector<int> S;                  // supersequence so far
  std::vector<std::vector<int>> cov;   // scenes covered by each of its launches
  std::vector<int> L;
  for (int s : order) {
    const std::vector<int>& q = keys[s];
    const size_t a = S.size(), b = q.size();
    // L[i][j]: longest common subsequence of S[i:] and q[j:]
    L.assign((a + 1) * (b + 1), 0);
    auto at = [&](size_t i, size_t j) -> int& { return L[i * (b + 1) + j]; };
    for (size_t i = a; i-- > 0;)
      for (size_t j = b; j-- > 0;)
        at(i, j) = S[i] == q[j] ? at(i + 1, j + 1) + 1 : std::max(at(i + 1, j), at(i, j + 1));
    std::vector<int> S2;
    std::vector<std::vector<int>> cov2;
    size_t i = 0, j = 0;
    while (i < a || j < b) {
      if (i < a && j < b && S[i] == q[j] && at(i, j) == at(i + 1, j + 1) + 1) {   // shared launch
        S2.push_back(S[i]);
        cov2.push_back(cov[i]);
        cov2.back().push_back(s);
        ++i;
        ++j;
      } else if (j >= b || (i < a && at(i + 1, j) >= at(i, j + 1))) {   // a launch of the merged scenes only
        S2.push_back(S[i]);
        cov2.push_back(std::move(cov[i]));
        ++i;
      } else {   // a launch of scene s only
        S2.push_back(q[j]);
        cov2.push_back({s});
        ++j;
      }
    }
    S.swap(S2);
    cov.swap(cov2);
  }
  for (auto& c : cov) std::sort(c.begin(), c.end());
  out_scenes.swap(cov);
  out_key.swap(S);
}

}  // namespace icr

using namespace icr;

struct icr_batch {
  Ctx* ctx = nullptr;
  std::vector<Scene*> scenes;
  int n_newton = 0;
  int n_groups = 1;
  std::vector<int> group;                  // group of each scene
  std::vector<cudaStream_t> streams;       // groups 1.. (group 0 runs on the context's stream)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  // one merged launch: a kernel body over its slots, or copies and fills
  struct Launch {
    const char* name = nullptr;
    int group = 0;
    BatchLaunchFn fn = nullptr;   // NULL: k_batch_memops
    dim3 block;
    size_t smem = 0;
    int nslots = 0;
    unsigned nblocks = 0;
    size_t off_first = 0, off_slots = 0;   // in the arena
  };
  std::vector<Launch> launches;
  unsigned char* arena = nullptr;   // device: every launch's block offsets and argument slots
  size_t arena_bytes = 0;
  cudaGraphExec_t graph = nullptr;
  int64_t recorded = 0;   // kernel launches the scenes' own steps would make
  uint64_t steps = 0;
  struct Snap {
    uint64_t epoch;
    int m, obst;
    icr_params params;
  };
  std::vector<Snap> snaps;
};

namespace {

#define CKB(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

// The merged launches of every group, each group on its own stream, forked
// from and joined back into the context's stream (inside a capture: parallel
// branches of one graph).
int run_launches(icr_batch* b, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev = nullptr) {
  cudaStream_t st0 = b->ctx->stream;
  if (b->n_groups > 1) {
    CKB(cudaEventRecord(b->fork, st0));
    for (cudaStream_t g : b->streams) CKB(cudaStreamWaitEvent(g, b->fork, 0));
  }
  for (size_t l = 0; l < b->launches.size(); ++l) {
    const icr_batch::Launch& L = b->launches[l];
    cudaStream_t st = L.group == 0 ? st0 : b->streams[L.group - 1];
    if (ev) CKB(cudaEventRecord((*ev)[l].first, st));
    const unsigned* first = reinterpret_cast<const unsigned*>(b->arena + L.off_first);
    if (L.fn) {
      CKB(L.fn(b->arena + L.off_slots, first, L.nslots, L.nblocks, L.block, L.smem, st, b->ctx->device));
    } else {
      k_batch_memops<<<L.nblocks, MEMOP_THREADS, 0, st>>>(reinterpret_cast<const MemOp*>(b->arena + L.off_slots),
                                                          first, L.nslots);
      CKB(cudaGetLastError());
    }
    if (ev) CKB(cudaEventRecord((*ev)[l].second, st));
  }
  if (b->n_groups > 1) {
    for (size_t g = 0; g < b->streams.size(); ++g) {
      CKB(cudaEventRecord(b->joins[g], b->streams[g]));
      CKB(cudaStreamWaitEvent(st0, b->joins[g], 0));
    }
  }
  return ICR_OK;
}

void free_batch(icr_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaStream_t g : b->streams) cudaStreamDestroy(g);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->arena) {
    cudaFree(b->arena);
    b->ctx->in_use -= b->arena_bytes;
  }
  for (Scene* s : b->scenes) --s->batches;
  delete b;
}

// the recorded launches hold the scenes' device addresses and launch shapes:
// ICR_ESTATE once a scene was evicted, reallocated a buffer, or changed its
// contact count, obstacle kind or parameters
int check_batch(const icr_batch* b, const char* where) {
  for (size_t i = 0; i < b->scenes.size(); ++i) {
    const Scene* s = b->scenes[i];
    const icr_batch::Snap& sn = b->snaps[i];
    if (s->evicted || s->alloc_epoch != sn.epoch || s->m != sn.m || s->obst_kind != sn.obst ||
        !same_params(s->params, sn.params)) {
      set_error("%s: scene %zu changed since the batch was created (evicted, buffers, contact count, obstacle or "
                "parameters); create the batch again",
                where, i);
      return ICR_ESTATE;
    }
  }
  return ICR_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int build_batch(icr_batch* b) {
  const int n = (int)b->scenes.size();
  // 1. every scene's step, recorded
  std::vector<BatchRec> recs(n);
  for (int i = 0; i < n; ++i) {
    Scene* s = b->scenes[i];
    s->rec = &recs[i];
    const int rc = step_enqueue(s, b->n_newton);
    s->rec = nullptr;
    if (rc != ICR_OK) return rc;
    for (const BatchEntry& e : recs[i].entries) b->recorded += e.launch ? 1 : 0;
  }
  // 2. keys and the merged sequence
  std::vector<Key> keys;
  std::vector<std::vector<int>> seq(n);
  for (int i = 0; i < n; ++i)
    for (const BatchEntry& e : recs[i].entries) {
      const Key k = key_of(e);
      auto it = std::find(keys.begin(), keys.end(), k);
      if (it == keys.end()) {
        keys.push_back(k);
        it = keys.end() - 1;
      }
      seq[i].push_back((int)(it - keys.begin()));
    }
  // every group's sequences merged on their own (cover: scene indices of the batch)
  std::vector<std::vector<int>> cover;
  std::vector<int> cover_group;
  for (int g = 0; g < b->n_groups; ++g) {
    std::vector<int> members;
    std::vector<std::vector<int>> gseq;
    for (int i = 0; i < n; ++i)
      if (b->group[i] == g) {
        members.push_back(i);
        gseq.push_back(seq[i]);
      }
    std::vector<std::vector<int>> gcover;
    std::vector<int> gkey;
    merge_sequences(gseq, gcover, gkey);
    for (auto& c : gcover) {
      for (int& x : c) x = members[x];
      cover.push_back(std::move(c));
      cover_group.push_back(g);
    }
  }
  // 3. the arena: per launch, the block offsets of its slots, then the slots
  std::vector<unsigned char> host;
  std::vector<size_t> next(n, 0);
  for (size_t l = 0; l < cover.size(); ++l) {
    icr_batch::Launch L;
    L.group = cover_group[l];
    const std::vector<int>& sc = cover[l];
    L.nslots = (int)sc.size();
    std::vector<unsigned> first;   // block offset of every slot, then the total
    std::vector<const BatchEntry*> ent;
    std::vector<MemOp> ops;
    // the covered scenes' entries, heaviest scene first: its blocks are
    // dispatched first, so the longest part of the launch starts earliest
    std::vector<int> by_cost(sc.begin(), sc.end());
    std::stable_sort(by_cost.begin(), by_cost.end(),
                     [&](int x, int y) { return scene_cost(b->scenes[x]) > scene_cost(b->scenes[y]); });
    for (int i : sc) ++next[i];
    for (int i : by_cost) ent.push_back(&recs[i].entries[next[i] - 1]);
    const BatchEntry& e0 = *ent[0];
    L.fn = e0.launch;
    L.name = e0.name;
    L.block = e0.block;
    uint64_t total = 0;
    if (L.fn) {
      for (size_t j = 0; j < ent.size(); ++j) {
        first.push_back((unsigned)total);
        total += ent[j]->blocks;
        L.smem = std::max(L.smem, ent[j]->smem);
      }
    } else {   // the ops of every covered scene, one slot each
      for (const BatchEntry* e : ent)
        for (const MemOp& o : e->ops) {
          first.push_back((unsigned)total);
          total += memop_blocks(o.bytes);
          ops.push_back(o);
        }
      L.nslots = (int)ops.size();
    }
    first.push_back((unsigned)total);
    bool ok = first.size() == (size_t)L.nslots + 1 && first[0] == 0;
    for (size_t j = 0; ok && j + 1 < first.size(); ++j) ok = first[j] < first[j + 1];
    if (!ok) {
      set_error("batch_create: block offsets of launch %zu (%s) are not increasing", l, e0.name);
      return ICR_EINVAL;
    }
    if (total == 0 || total > 0x7fffffffull) {
      set_error("batch_create: launch %zu (%s) has %llu blocks", l, e0.name, (unsigned long long)total);
      return ICR_EINVAL;
    }
    L.nblocks = (unsigned)total;
    if (L.fn && e0.stride) {   // one persistent grid, as large as the largest scene's own
      unsigned most = 0;
      for (const BatchEntry* e : ent) most = std::max(most, e->blocks);
      L.nblocks = most;
    }
    L.off_first = align_up(host.size(), 16);
    host.resize(L.off_first + first.size() * sizeof(unsigned));
    std::memcpy(host.data() + L.off_first, first.data(), first.size() * sizeof(unsigned));
    if (L.fn) {
      const size_t sz = e0.slot.size();
      L.off_slots = align_up(host.size(), std::max<size_t>(16, e0.slot_align));
      host.resize(L.off_slots + sz * ent.size());
      for (size_t j = 0; j < ent.size(); ++j) {
        if (ent[j]->slot.size() != sz) {
          set_error("batch_create: argument slots of %s differ in size", e0.name);
          return ICR_EINVAL;
        }
        std::memcpy(host.data() + L.off_slots + j * sz, ent[j]->slot.data(), sz);
      }
    } else {
      L.off_slots = align_up(host.size(), 16);
      host.resize(L.off_slots + ops.size() * sizeof(MemOp));
      std::memcpy(host.data() + L.off_slots, ops.data(), ops.size() * sizeof(MemOp));
    }
    b->launches.push_back(L);
  }
  // 4. the arena on the device, under the context's budget
  b->arena_bytes = align_up(std::max<size_t>(host.size(), 16), 256);
  Ctx* c = b->ctx;
  if (c->budget && c->in_use + b->arena_bytes > c->budget) {
    set_error("batch_create: %zu bytes of launch arguments exceed the HBM budget", b->arena_bytes);
    b->arena_bytes = 0;
    return ICR_ENOMEM;
  }
  const cudaError_t ea = cudaMalloc(&b->arena, b->arena_bytes);
  if (ea != cudaSuccess) {
    b->arena = nullptr;
    b->arena_bytes = 0;
    return cuda_fail(ea, "cudaMalloc(batch arguments)");
  }
  c->in_use += b->arena_bytes;
  CKB(cudaMemcpyAsync(b->arena, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream));
  // 5. one eager step (sets every kernel up), then the captured graph
  RET(run_launches(b));
  CKB(cudaStreamSynchronize(c->stream));
  for (Scene* s : b->scenes) RET(check_device_error(s));
  CKB(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = run_launches(b);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
  if (rc != ICR_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture(batch)");
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    b->graph = nullptr;
    return cuda_fail(ei, "cudaGraphInstantiate(batch)");
  }
  return ICR_OK;
}

}  // namespace

extern "C" {

int icr_batch_create(icr_batch** out, icr_scene* const* scenes, int32_t n_scenes, int32_t n_newton,
                     int32_t n_groups) {
  if (!out || !scenes || n_scenes <= 0 || n_groups <= 0) {
    set_error("batch_create: need an output pointer, at least one scene and at least one group");
    return ICR_EINVAL;
  }
  *out = nullptr;
  Ctx* ctx = nullptr;
  for (int i = 0; i < n_scenes; ++i) {
    Scene* s = scenes[i];
    if (!s) {
      set_error("batch_create: scene %d is NULL", i);
      return ICR_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (scenes[j] == scenes[i]) {
        set_error("batch_create: scene %d appears twice", i);
        return ICR_EINVAL;
      }
    if (!ctx) ctx = s->ctx;
    if (s->ctx != ctx) {
      set_error("batch_create: all scenes must share one context (one device and stream)");
      return ICR_EINVAL;
    }
    if (s->evicted || !s->has_system || !s->has_mapping || s->obst_kind == 0) {
      set_error("batch_create: scene %d needs to be resident with a system, a mapping and an obstacle", i);
      return ICR_ESTATE;
    }
    if (n_newton < 0 || (s->obst_kind == 1 && n_newton > s->obst_iters)) {
      set_error("batch_create: %d Newton iterations not available for scene %d", n_newton, i);
      return ICR_EINVAL;
    }
  }
  cudaStream_t st = ctx->stream;
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
    set_error("batch_create: the context needs its own CUDA stream to capture a graph");
    return ICR_EINVAL;
  }
  CKB(cudaSetDevice(ctx->device));
  for (int i = 0; i < n_scenes; ++i)
    if (!scenes[i]->tuned) RET(icr_autotune(scenes[i], nullptr, nullptr, 0));
  icr_batch* b = new icr_batch;
  b->ctx = ctx;
  b->n_newton = n_newton;
  b->n_groups = std::min<int>(n_groups, n_scenes);
  for (int i = 0; i < n_scenes; ++i) {
    b->scenes.push_back(scenes[i]);
    ++scenes[i]->batches;
  }
  // groups balanced by cost (longest processing time first: scenes in
  // decreasing cost, ties by index, each to the least loaded group, ties to the
  // lower group), so that every group's chain carries about one heavy scene
  // and the lighter scenes' kernels ride in its launches
  std::vector<int> order(n_scenes);
  for (int i = 0; i < n_scenes; ++i) order[i] = i;
  auto cost = [&](int i) { return scene_cost(b->scenes[i]); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  b->group.assign(n_scenes, 0);
  std::vector<double> load(b->n_groups, 0.0);
  for (int i : order) {
    const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->group[i] = g;
    load[g] += cost(i);
  }
  int rc = ICR_OK;
  if (b->n_groups > 1) {
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int g = 1; g < b->n_groups && e == cudaSuccess; ++g) {
      cudaStream_t gs = nullptr;
      cudaEvent_t je = nullptr;
      e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->streams.push_back(gs);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&je, cudaEventDisableTiming);
      if (e == cudaSuccess) b->joins.push_back(je);
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "batch_create: group streams");
  }
  if (rc == ICR_OK) rc = build_batch(b);
  if (rc != ICR_OK) {
    cudaStreamSynchronize(st);
    free_batch(b);
    return rc;
  }
  for (Scene* s : b->scenes) b->snaps.push_back({s->alloc_epoch, s->m, s->obst_kind, s->params});
  *out = b;
  return ICR_OK;
}

int icr_batch_launch(icr_batch* b) {
  if (!b) {
    set_error("batch_launch: NULL batch");
    return ICR_EINVAL;
  }
  RET(check_batch(b, "batch_launch"));
  CKB(cudaSetDevice(b->ctx->device));
  CKB(cudaGraphLaunch(b->graph, b->ctx->stream));
  ++b->steps;
  for (Scene* s : b->scenes) {
    s->last_newton = b->n_newton;
    s->last_newton_tol = s->params.newton_tol > 0 && b->n_newton > 1 && s->m > 0;
    s->has_WH = s->has_dirs = s->has_W = s->has_lam = true;
  }
  return ICR_OK;
}

int icr_batch_info(icr_batch* b, icr_batch_info_t* out) {
  if (!b || !out) {
    set_error("batch_info: NULL argument");
    return ICR_EINVAL;
  }
  out->n_scenes = (int32_t)b->scenes.size();
  out->n_groups = b->n_groups;
  out->launches_per_step = (int32_t)b->launches.size();
  int32_t k = 0;
  for (const icr_batch::Launch& L : b->launches) k += L.fn ? 1 : 0;
  out->kernel_launches_per_step = k;
  out->scene_launches_per_step = b->recorded;
  out->argument_bytes = (uint64_t)b->arena_bytes;
  out->steps = b->steps;
  return ICR_OK;
}

int icr_batch_profile(icr_batch* b, icr_batch_launch_time* out, int32_t max_out, int32_t* n_out) {
  if (!b || !n_out || max_out < 0 || (max_out > 0 && !out)) {
    set_error("batch_profile: invalid arguments");
    return ICR_EINVAL;
  }
  RET(check_batch(b, "batch_profile"));
  CKB(cudaSetDevice(b->ctx->device));
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev(b->launches.size(), {nullptr, nullptr});
  auto release = [&](int rc) {
    for (auto& p : ev) {
      if (p.first) cudaEventDestroy(p.first);
      if (p.second) cudaEventDestroy(p.second);
    }
    return rc;
  };
  for (auto& p : ev) {
    cudaError_t e = cudaEventCreate(&p.first);
    if (e == cudaSuccess) e = cudaEventCreate(&p.second);
    if (e != cudaSuccess) return release(cuda_fail(e, "batch_profile: cudaEventCreate"));
  }
  int rc = run_launches(b, &ev);
  if (rc != ICR_OK) return release(rc);
  const cudaError_t es = cudaStreamSynchronize(b->ctx->stream);
  if (es != cudaSuccess) return release(cuda_fail(es, "batch_profile: cudaStreamSynchronize"));
  ++b->steps;
  *n_out = (int32_t)b->launches.size();
  for (size_t l = 0; l < b->launches.size() && (int32_t)l < max_out; ++l) {
    const icr_batch::Launch& L = b->launches[l];
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, ev[l].first, ev[l].second);
    if (e != cudaSuccess) return release(cuda_fail(e, "batch_profile: cudaEventElapsedTime"));
    std::memset(out[l].name, 0, sizeof(out[l].name));
    std::strncpy(out[l].name, L.fn ? L.name : "copies/fills", sizeof(out[l].name) - 1);
    out[l].group = L.group;
    out[l].slots = L.nslots;
    out[l].blocks = (int32_t)L.nblocks;
    out[l].ms = ms;
  }
  return release(ICR_OK);
}

int icr_batch_destroy(icr_batch* b) {
  if (!b) return ICR_OK;
  cudaSetDevice(b->ctx->device);
  cudaStreamSynchronize(b->ctx->stream);
  free_batch(b);
  return ICR_OK;
}

int icr_batch_merge_plan(const int32_t* keys, const int32_t* lengths, int32_t n_seq, int32_t* out_key,
                         int32_t* out_count, int32_t* out_cover, int32_t max_out, int32_t* n_out) {
  if (!keys || !lengths || n_seq <= 0 || !out_key || !out_count || !out_cover || !n_out || max_out < 0) {
    set_error("batch_merge_plan: invalid arguments");
    return ICR_EINVAL;
  }
  std::vector<std::vector<int>> seq(n_seq);
  int64_t off = 0;
  for (int i = 0; i < n_seq; ++i) {
    if (lengths[i] < 0) {
      set_error("batch_merge_plan: negative length of sequence %d", i);
      return ICR_EINVAL;
    }
    seq[i].assign(keys + off, keys + off + lengths[i]);
    off += lengths[i];
    for (int k : seq[i])
      if (k < 0) {
        set_error("batch_merge_plan: negative key in sequence %d", i);
        return ICR_EINVAL;
      }
  }
  std::vector<std::vector<int>> cover;
  std::vector<int> mkey;
  merge_sequences(seq, cover, mkey);
  *n_out = (int32_t)cover.size();
  if ((int64_t)cover.size() > max_out) {
    set_error("batch_merge_plan: %zu merged launches exceed max_out = %d", cover.size(), max_out);
    return ICR_EINVAL;
  }
  int64_t c = 0;
  for (size_t l = 0; l < cover.size(); ++l) {
    out_key[l] = mkey[l];
    out_count[l] = (int32_t)cover[l].size();
    for (int s : cover[l]) out_cover[c++] = s;
  }
  return ICR_OK;
}

}  // extern "C"
