// Allocation-free variant of the elimination-tree reach (the contacts whose
// columns of H^T reach each supernode), for callers that cannot allocate
// device memory: a real-time simulation or haptics loop that forbids any
// allocation after start-up, or a host framework that owns every device
// allocation through its own pool.  The caller passes device buffers for all
// inputs and outputs; the only working memory is the fixed static array below.
//
// The scratch array is a file-scope __device__ array, so every GPU that loads
// the library holds its ICR_NOALLOC_SCRATCH_WORDS words until the process
// exits.  In host code its name is only a host-side stand-in, not a device
// address: the device address is looked up with cudaGetSymbolAddress once per
// device (on the first call made with that device current) and passed to the
// kernels.  The cached address belongs to the device's context at that time:
// after cudaDeviceReset the module is loaded again elsewhere, so the call must
// not be used across a device reset in one process.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "icr.h"
#include "icr_internal.h"

namespace icr {
namespace {

constexpr int kMaxDevices = 64;

// reach bitmap: nsuper rows of ceil(m / 32) words
static __device__ __align__(256) uint32_t g_reach_scratch[ICR_NOALLOC_SCRATCH_WORDS];
static __device__ int g_reach_status;   // set to 1 by a kernel that met an out-of-range id

std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};
int* g_status_ptr[kMaxDevices] = {};

// Device addresses of the scratch array and the status word on the current
// device, looked up on the first call for that device.
int scratch_for_current_device(uint32_t** scratch, int** status) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("reach_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return ICR_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reach_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: cudaGetSymbolAddress(scratch)");
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_reach_status);
    if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: cudaGetSymbolAddress(status)");
    g_scratch_ptr[dev] = (uint32_t*)p;
    g_status_ptr[dev] = (int*)q;
  }
  *scratch = g_scratch_ptr[dev];
  *status = g_status_ptr[dev];
  return ICR_OK;
}

__global__ void k_na_clear(uint32_t* bitmap, size_t words, int* status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
    bitmap[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// One thread per (contact, node): mark the contact on the etree path from the
// node's supernode to the root, stopping where another thread already marked
// it.  Every id is checked before it is used as an index: a node id outside
// [0, n_nodes), a supernode id outside [0, ns), or a parent that is neither -1
// nor above its child sets the status word and ends the walk (parents above
// their children also bound the walk by ns steps).
__global__ void k_na_mark(const int* __restrict__ nodes, int m, int n_nodes, const int* __restrict__ node_super,
                          const int* __restrict__ parent, int ns, uint32_t* bitmap, int words, int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * m) return;
  const int a = t >> 2;
  const int node = nodes[t];
  if (node < 0 || node >= n_nodes) {
    *status = 1;
    return;
  }
  int s = node_super[node];
  if (s < 0 || s >= ns) {
    *status = 1;
    return;
  }
  const uint32_t bit = 1u << (a & 31);
  const int w = a >> 5;
  for (int guard = 0; guard < ns; ++guard) {
    const uint32_t old = atomicOr(&bitmap[(size_t)s * words + w], bit);
    if (old & bit) return;
    const int p = parent[s];
    if (p == -1) return;
    if (p <= s || p >= ns) {
      *status = 1;
      return;
    }
    s = p;
  }
  *status = 1;   // not reached with valid parents (each step climbs)
}

// One block per supernode: count its contacts and list them in ascending order.
__global__ void k_na_rows(const uint32_t* __restrict__ bitmap, int words, int m, int* qcount, int* qidx) {
  extern __shared__ int sh[];
  const int s = blockIdx.x;
  const int w = threadIdx.x;
  uint32_t bits = (w < words) ? bitmap[(size_t)s * words + w] : 0u;
  const int c = __popc(bits);
  sh[w] = c;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    const int v = (w >= off) ? sh[w - off] : 0;
    __syncthreads();
    sh[w] += v;
    __syncthreads();
  }
  if (w == blockDim.x - 1) qcount[s] = sh[w];
  int* out = qidx + (size_t)s * m + (sh[w] - c);
  while (bits) {
    *out++ = 32 * w + __ffs(bits) - 1;
    bits &= bits - 1;
  }
}

}  // namespace
}  // namespace icr

extern "C" int icr_reach_noalloc(int32_t m, int32_t nsuper, int32_t n_nodes, const int32_t* nodes,
                                 const int32_t* node_super, const int32_t* parent, int32_t* qcount, int32_t* qidx,
                                 void* cuda_stream) {
  using namespace icr;
  if (m < 0 || m > 32768 || nsuper <= 0 || n_nodes <= 0 || !node_super || !parent || !qcount ||
      (m > 0 && (!nodes || !qidx))) {
    set_error("reach_noalloc: need 0 <= m <= 32768, nsuper > 0, n_nodes > 0 and non-NULL device buffers");
    return ICR_EINVAL;
  }
  const int words = (m + 31) / 32 > 0 ? (m + 31) / 32 : 1;
  const size_t need = (size_t)nsuper * words;
  if (need > (size_t)ICR_NOALLOC_SCRATCH_WORDS) {
    set_error("reach_noalloc: nsuper x ceil(m/32) = %zu words exceeds the static scratch of %d words", need,
              (int)ICR_NOALLOC_SCRATCH_WORDS);
    return ICR_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the call reads its status back and synchronises: it cannot be captured
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cs);
  if (ce != cudaSuccess) return cuda_fail(ce, "reach_noalloc: cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) {
    set_error("reach_noalloc: the stream is being captured; this call synchronises and cannot be captured");
    return ICR_ESTATE;
  }
  uint32_t* bitmap = nullptr;
  int* status = nullptr;
  int rc = scratch_for_current_device(&bitmap, &status);
  if (rc != ICR_OK) return rc;
  const int grid_clear = (int)((need + 255) / 256 < 1024 ? (need + 255) / 256 : 1024);
  k_na_clear<<<grid_clear, 256, 0, st>>>(bitmap, need, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: k_na_clear");
  if (m > 0) {
    k_na_mark<<<(4 * m + 255) / 256, 256, 0, st>>>((const int*)nodes, m, n_nodes, (const int*)node_super,
                                                  (const int*)parent, nsuper, bitmap, words, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: k_na_mark");
  }
  const int bt = ((words + 31) / 32) * 32;
  k_na_rows<<<nsuper, bt, bt * sizeof(int), st>>>(bitmap, words, m > 0 ? m : 1, (int*)qcount, (int*)qidx);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: k_na_rows");
  int h_status = 0;
  e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: status copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reach_noalloc: synchronize");
  if (h_status) {
    set_error("reach_noalloc: a node id, a supernode id or a parent was out of range (a parent must be -1 or "
              "above its child); the outputs are incomplete");
    return ICR_EINVAL;
  }
  return ICR_OK;
}
