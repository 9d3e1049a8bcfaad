// Serving loop with continuous batching (gnntrk_serve_run).
//
// The calling thread replays the request stream against a steady clock: every
// event whose arrival time has passed waits in a queue; whenever a slot (its
// own stream, handle and staging buffers) is free, the slot takes every queued
// event (up to the batch caps), copies them to pinned memory, and enqueues
// host-to-device copies, the hot path and the device-to-host copy of the labels
// on its stream, followed by a host callback that stamps the completion time.
// Slots run concurrently on the device, so events arriving while other batches
// are in flight are admitted as soon as a slot frees up.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gnntrk.h"
#include "internal.cuh"

namespace gnntrk {
void set_global_error(const std::string& msg);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  gnntrk_handle* h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* h_xyz = nullptr;  // pinned staging
  uint8_t* h_plane = nullptr;
  int64_t* h_off = nullptr;
  int32_t* h_lab = nullptr;
  float* d_xyz = nullptr;  // device
  uint8_t* d_plane = nullptr;
  int64_t* d_off = nullptr;
  int32_t* d_lab = nullptr;
  bool busy = false;
  int first = 0, count = 0;  // events of the batch in flight
  int64_t hits = 0;
  std::atomic<double> t_done{0.0};
  Clock::time_point t0;
};

void CUDART_CB stamp_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->t_done.store(std::chrono::duration<double>(Clock::now() - s->t0).count());
}

gnntrk_status err(gnntrk_status st, const std::string& m) {
  gnntrk::set_global_error("gnntrk_serve_run: " + m);
  return st;
}

}  // namespace

extern "C" gnntrk_status gnntrk_serve_run(const void* weights, size_t weights_bytes,
                                          const gnntrk_cfg* model, const gnntrk_serve_cfg* scfg,
                                          int32_t n_events, const int64_t* offsets,
                                          const float* hits_xyz, const uint8_t* plane,
                                          const double* arrival_s, int32_t* out_labels,
                                          double* done_s, int64_t* stats) {
  if (!model || !scfg || n_events < 0 || !offsets || !arrival_s || !done_s)
    return err(GNNTRK_ERR_INVALID_ARG, "NULL argument or negative event count");
  if (scfg->n_slots < 1 || scfg->n_slots > 16 || scfg->max_events_per_batch < 1 ||
      scfg->max_hits_per_batch < 1 || scfg->memory_budget_bytes < 1)
    return err(GNNTRK_ERR_INVALID_ARG, "serve cfg out of range");
  const int64_t n_hits = n_events ? offsets[n_events] : 0;
  if (n_hits > 0 && (!hits_xyz || !plane || !out_labels))
    return err(GNNTRK_ERR_INVALID_ARG, "NULL hit arrays");
  for (int e = 0; e < n_events; ++e) {
    if (offsets[e + 1] < offsets[e] || offsets[e + 1] - offsets[e] > scfg->max_hits_per_batch)
      return err(GNNTRK_ERR_INVALID_ARG,
                 "offsets must be non-decreasing and every event must fit a batch");
    if (e > 0 && arrival_s[e] < arrival_s[e - 1])
      return err(GNNTRK_ERR_INVALID_ARG, "arrival times must be non-decreasing");
  }
  if (offsets[0] != 0) return err(GNNTRK_ERR_INVALID_ARG, "offsets[0] must be 0");

  gnntrk_cfg c = *model;
  c.max_hits = scfg->max_hits_per_batch;
  c.max_events = scfg->max_events_per_batch;
  c.use_graph = 0;  // batch shapes change from batch to batch
  const int64_t ws = gnntrk_workspace_bytes(&c);
  if (ws <= 0) return err(GNNTRK_ERR_INVALID_ARG, "invalid model cfg");
  const int64_t per_slot = ws + c.max_hits * 17 + (c.max_events + 1) * 8;
  const int n_slots = int(std::min<int64_t>(scfg->n_slots, scfg->memory_budget_bytes / per_slot));
  if (n_slots < 1) return err(GNNTRK_ERR_OOM, "one slot needs " + std::to_string(per_slot) +
                                                  " bytes, more than the budget");

  std::vector<Slot> slots(n_slots);
  gnntrk_status st = GNNTRK_OK;
  auto cleanup = [&]() {
    for (auto& s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      gnntrk_destroy(s.h);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
      cudaFreeHost(s.h_xyz);
      cudaFreeHost(s.h_plane);
      cudaFreeHost(s.h_off);
      cudaFreeHost(s.h_lab);
      cudaFree(s.d_xyz);
      cudaFree(s.d_plane);
      cudaFree(s.d_off);
      cudaFree(s.d_lab);
    }
  };
  for (auto& s : slots) {
    st = gnntrk_create(weights, weights_bytes, &c, &s.h);
    if (st) {
      cleanup();
      return err(st, std::string("slot handle: ") + gnntrk_last_error(nullptr));
    }
    if (scfg->apply_tuning && (st = gnntrk_set_tuning(s.h, scfg->tuning)) != GNNTRK_OK) {
      const std::string m = gnntrk_last_error(s.h);
      cleanup();
      return err(st, "tuning: " + m);
    }
    const int64_t H = c.max_hits, Ev = c.max_events;
    bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost(&s.h_xyz, 12 * H) == cudaSuccess &&
              cudaMallocHost(&s.h_plane, H) == cudaSuccess &&
              cudaMallocHost(&s.h_off, 8 * (Ev + 1)) == cudaSuccess &&
              cudaMallocHost(&s.h_lab, 4 * H) == cudaSuccess &&
              cudaMalloc(&s.d_xyz, 12 * H) == cudaSuccess &&
              cudaMalloc(&s.d_plane, H) == cudaSuccess &&
              cudaMalloc(&s.d_off, 8 * (Ev + 1)) == cudaSuccess &&
              cudaMalloc(&s.d_lab, 4 * H) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cleanup();
      return err(GNNTRK_ERR_OOM, "slot buffers");
    }
  }

  const Clock::time_point t0 = Clock::now();
  for (auto& s : slots) s.t0 = t0;
  auto now_s = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  int next = 0, finished = 0;
  int64_t n_batches = 0, failed = 0, max_inflight = 0, largest = 0;
  const float* X = hits_xyz;
  const float* Y = hits_xyz + n_hits;
  const float* Z = hits_xyz + 2 * n_hits;

  while (finished < n_events) {
    bool progress = false;
    // 1. completed batches
    for (auto& s : slots) {
      if (!s.busy || cudaEventQuery(s.done) != cudaSuccess) continue;
      gnntrk_status bst = gnntrk_sync_status(s.h, s.stream);
      const double t = s.t_done.load();
      for (int e = s.first; e < s.first + s.count; ++e) {
        done_s[e] = t;
        const int64_t a = offsets[e], z = offsets[e + 1], base = offsets[s.first];
        if (bst == GNNTRK_OK)
          std::memcpy(out_labels + a, s.h_lab + (a - base), 4 * (z - a));
        else
          for (int64_t i = a; i < z; ++i) out_labels[i] = -1;
      }
      if (bst != GNNTRK_OK) ++failed;
      finished += s.count;
      s.busy = false;
      progress = true;
    }
    // 2. admit every arrived event into free slots
    const double now = now_s();
    for (auto& s : slots) {
      if (s.busy || next >= n_events || arrival_s[next] > now) continue;
      int cnt = 0;
      int64_t hits = 0;
      while (next + cnt < n_events && cnt < c.max_events && arrival_s[next + cnt] <= now) {
        const int64_t nh = offsets[next + cnt + 1] - offsets[next + cnt];
        if (hits + nh > c.max_hits) break;
        hits += nh;
        ++cnt;
      }
      const int64_t base = offsets[next];
      std::memcpy(s.h_xyz, X + base, 4 * hits);
      std::memcpy(s.h_xyz + hits, Y + base, 4 * hits);
      std::memcpy(s.h_xyz + 2 * hits, Z + base, 4 * hits);
      std::memcpy(s.h_plane, plane + base, hits);
      for (int e = 0; e <= cnt; ++e) s.h_off[e] = offsets[next + e] - base;
      cudaMemcpyAsync(s.d_xyz, s.h_xyz, 12 * hits, cudaMemcpyHostToDevice, s.stream);
      cudaMemcpyAsync(s.d_plane, s.h_plane, hits, cudaMemcpyHostToDevice, s.stream);
      cudaMemcpyAsync(s.d_off, s.h_off, 8 * (cnt + 1), cudaMemcpyHostToDevice, s.stream);
      gnntrk_status lst =
          gnntrk_find_tracks(s.h, cnt, hits, s.d_xyz, s.d_plane, s.d_off, s.d_lab, s.stream);
      if (lst != GNNTRK_OK) {
        std::string m = gnntrk_last_error(s.h);
        cleanup();
        return err(lst, "launch: " + m);
      }
      cudaMemcpyAsync(s.h_lab, s.d_lab, 4 * hits, cudaMemcpyDeviceToHost, s.stream);
      cudaLaunchHostFunc(s.stream, stamp_done, &s);
      cudaEventRecord(s.done, s.stream);
      s.busy = true;
      s.first = next;
      s.count = cnt;
      s.hits = hits;
      next += cnt;
      ++n_batches;
      largest = std::max<int64_t>(largest, cnt);
      progress = true;
    }
    int64_t inflight = 0;
    for (auto& s : slots) inflight += s.busy;
    max_inflight = std::max(max_inflight, inflight);
    if (!progress) std::this_thread::yield();
  }
  const double wall = now_s();
  cudaError_t ce = cudaGetLastError();
  cleanup();
  if (ce != cudaSuccess) return err(GNNTRK_ERR_CUDA, cudaGetErrorString(ce));
  if (stats) {
    stats[0] = n_batches;
    stats[1] = n_slots;
    stats[2] = failed;
    stats[3] = max_inflight;
    stats[4] = per_slot;
    stats[5] = largest;
    stats[6] = int64_t(wall * 1e6);
    stats[7] = 0;
  }
  return GNNTRK_OK;
}
