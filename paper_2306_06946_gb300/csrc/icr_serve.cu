// Request loop for many scenes: continuous batching of time steps with
// admission under the contexts' HBM budgets.
//
// Every scene has a captured step graph (icr_step_capture).  A resident scene
// keeps its system, mapping, obstacle and graph on the device; an evicted one
// (icr_scene_evict) keeps them in pinned host memory.  A request asks for one
// time step of one scene at a given arrival time.  The loop replays the
// arrival schedule in real time: a request is admitted once it has arrived,
// waits while its scene already has a step in flight (a scene's steps share
// its buffers), and is started on the first free slot stream; slots complete
// independently, so requests that arrive while others run on the GPU overlap
// with them.  A request for an evicted scene first readmits it; while its
// context's budget is short, the least recently used idle resident scenes of
// that context are evicted.  If the scene cannot fit even then, the request
// waits while other steps of the context are in flight, and is rejected
// (latency -1) when none are.  The latency of a request is the time from its
// arrival to the moment its slot's completion event is seen.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <deque>
#include <string>
#include <vector>

#include "icr_internal.h"

struct icr_scene : icr::Scene {};

using namespace icr;

namespace {

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int request = -1;   // request running on the slot, -1 when free
};

int serve_fail(std::vector<Slot>& slots, int code) {
  for (Slot& sl : slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.done) cudaEventDestroy(sl.done);
  }
  return code;
}

}  // namespace

extern "C" int icr_serve_ex(icr_scene* const* scenes, int32_t n_scenes, const int32_t* req_scene,
                            const double* req_arrival_s, int32_t n_req, int32_t n_slots, double timeout_s,
                            double* latency_s, double* makespan_s, icr_serve_stats* stats) {
  if (!scenes || n_scenes <= 0 || n_req < 0 || (n_req > 0 && (!req_scene || !req_arrival_s || !latency_s)) ||
      n_slots <= 0 || !(timeout_s > 0)) {
    set_error("serve: need scenes, a request schedule, n_slots > 0 and a positive timeout");
    return ICR_EINVAL;
  }
  int device = -1;
  for (int i = 0; i < n_scenes; ++i) {
    if (!scenes[i]) {
      set_error("serve: scene %d is NULL", i);
      return ICR_EINVAL;
    }
    if (scenes[i]->evicted) {
      if (!scenes[i]->recapture) {
        set_error("serve: scene %d was evicted without a captured step", i);
        return ICR_ESTATE;
      }
    } else {
      const int rc = check_step_graph(scenes[i], "serve");
      if (rc != ICR_OK) return rc;
    }
    if (device < 0) device = scenes[i]->ctx->device;
    if (scenes[i]->ctx->device != device) {
      set_error("serve: all scenes must live on one device");
      return ICR_EINVAL;
    }
  }
  for (int r = 0; r < n_req; ++r) {
    if (req_scene[r] < 0 || req_scene[r] >= n_scenes || !(req_arrival_s[r] >= 0)) {
      set_error("serve: request %d has a bad scene id or arrival time", r);
      return ICR_EINVAL;
    }
    if (r > 0 && req_arrival_s[r] < req_arrival_s[r - 1]) {
      set_error("serve: arrival times must be non-decreasing");
      return ICR_EINVAL;
    }
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "serve: cudaSetDevice");
  // scenes' own streams must be idle before their graphs move to slot streams
  for (int i = 0; i < n_scenes; ++i) {
    e = cudaStreamSynchronize(scenes[i]->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve: scene stream");
  }
  icr_serve_stats st{};
  std::vector<Slot> slots(n_slots);
  for (Slot& sl : slots) {
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return serve_fail(slots, cuda_fail(e, "serve: cudaStreamCreate"));
    e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return serve_fail(slots, cuda_fail(e, "serve: cudaEventCreate"));
  }
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
  std::vector<char> busy(n_scenes, 0);
  std::vector<double> last_used(n_scenes, -1.0);
  std::deque<int> pending;   // arrived, not yet started, in arrival order
  int next = 0, finished = 0;
  // Makes scene i resident: 1 when it is, 0 when it must wait (other steps of
  // its context are in flight and may free budget), -1 when it cannot fit
  // (rejected), or a negative status below -1 (minus the error code).
  auto admit = [&](int i) -> int {
    Scene* sc = scenes[i];
    if (!sc->evicted) return 1;
    Ctx* c = sc->ctx;
    const double a0 = now_s();
    while (c->budget && c->in_use + sc->resident_bytes > c->budget) {
      int victim = -1;
      for (int j = 0; j < n_scenes; ++j)
        if (j != i && !busy[j] && !scenes[j]->evicted && scenes[j]->ctx == c &&
            (victim < 0 || last_used[j] < last_used[victim]))
          victim = j;
      if (victim < 0) break;
      const int rc = scene_evict(scenes[victim]);
      if (rc != ICR_OK) return -1 - rc;
      ++st.evictions;
    }
    if (c->budget && c->in_use + sc->resident_bytes > c->budget) {
      for (int j = 0; j < n_scenes; ++j)
        if (busy[j] && scenes[j]->ctx == c) return 0;
      return -1;
    }
    const int rc = scene_readmit(sc);
    if (rc != ICR_OK) return -1 - rc;
    ++st.readmissions;
    st.admit_s += now_s() - a0;
    return 1;
  };
  while (finished < n_req) {
    const double t = now_s();
    if (t > timeout_s) {
      set_error("serve: %d of %d requests unfinished after %g s", n_req - finished, n_req, timeout_s);
      return serve_fail(slots, ICR_ETIMEOUT);
    }
    while (next < n_req && req_arrival_s[next] <= t) pending.push_back(next++);
    // completions
    for (Slot& sl : slots) {
      if (sl.request < 0) continue;
      e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) return serve_fail(slots, cuda_fail(e, "serve: step"));
      latency_s[sl.request] = now_s() - req_arrival_s[sl.request];
      busy[req_scene[sl.request]] = 0;
      sl.request = -1;
      ++finished;
    }
    // starts: oldest pending request whose scene is idle (and fits), on a free slot
    for (Slot& sl : slots) {
      if (sl.request >= 0) continue;
      int r = -1;
      for (auto it = pending.begin(); it != pending.end();) {
        if (busy[req_scene[*it]]) {
          ++it;
          continue;
        }
        const int a = admit(req_scene[*it]);
        if (a < -1) {
          const std::string why = icr_last_error();
          set_error("serve: admitting scene %d: %s", req_scene[*it], why.c_str());
          return serve_fail(slots, -1 - a);
        }
        if (a == -1) {   // cannot fit under the budget even alone: rejected
          latency_s[*it] = -1.0;
          ++st.rejected;
          ++finished;
          it = pending.erase(it);
          continue;
        }
        if (a == 0) {
          ++it;
          continue;
        }
        r = *it;
        pending.erase(it);
        break;
      }
      if (r < 0) break;
      Scene* s = scenes[req_scene[r]];
      e = cudaGraphLaunch(s->step_graph, sl.stream);
      if (e != cudaSuccess) return serve_fail(slots, cuda_fail(e, "serve: cudaGraphLaunch"));
      e = cudaEventRecord(sl.done, sl.stream);
      if (e != cudaSuccess) return serve_fail(slots, cuda_fail(e, "serve: cudaEventRecord"));
      s->launches += s->graph_kernels;
      busy[req_scene[r]] = 1;
      last_used[req_scene[r]] = now_s();
      sl.request = r;
    }
  }
  if (makespan_s) *makespan_s = now_s();
  for (Slot& sl : slots) {
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  if (stats) *stats = st;
  for (int i = 0; i < n_scenes; ++i) {
    if (scenes[i]->evicted) continue;   // its device error word was checked when it was evicted
    const int rc = check_device_error(scenes[i]);
    if (rc != ICR_OK) return rc;
  }
  return ICR_OK;
}

extern "C" int icr_serve(icr_scene* const* scenes, int32_t n_scenes, const int32_t* req_scene,
                         const double* req_arrival_s, int32_t n_req, int32_t n_slots, double timeout_s,
                         double* latency_s, double* makespan_s) {
  return icr_serve_ex(scenes, n_scenes, req_scene, req_arrival_s, n_req, n_slots, timeout_s, latency_s, makespan_s,
                      nullptr);
}
