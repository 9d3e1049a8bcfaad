// Weakly connected components of the purified hit graph (Sec. "WCC
// Implementation"): track candidates are the components left after the edge
// cut. Instead of the thesis's plane sweeps, an exact lock-free union-find over
// global input indices:
//   * parent[i] <= i always; a union hooks the larger root under the smaller
//     one with a compare-and-swap, so every root is the smallest input index of
//     its component and the result does not depend on the order of unions;
//   * finds halve paths with plain stores (each store moves a pointer to an
//     ancestor, which keeps parent[i] <= i).
// A label is the root minus the event's first index: the smallest event-local
// input index of the component.
#include <algorithm>
#include <mutex>

#include "../../include/gnntrk.h"
#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kUnionRetries = 1 << 20;

__device__ __forceinline__ int uf_find(volatile int32_t* P, int x) {
  int cur = P[x];
  if (cur == x) return x;
  int prev = x;
  int next;
  while (cur > (next = P[cur])) {
    P[prev] = next;
    prev = cur;
    cur = next;
  }
  return cur;
}

__device__ __forceinline__ void uf_union(volatile int32_t* P, int a, int b, int32_t* counters) {
  int ra = uf_find(P, a), rb = uf_find(P, b);
  for (int it = 0; it < kUnionRetries; ++it) {
    if (ra == rb) return;
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    const int old = atomicCAS((int32_t*)&P[rb], rb, ra);
    if (old == rb) return;
    rb = uf_find(P, old);
    ra = uf_find(P, ra);
  }
  set_status(counters, ST_TIMEOUT);
}

__global__ void k_cc_union(Ws w) {
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  for (int base = blockIdx.x * blockDim.x; base < E; base += gridDim.x * blockDim.x) {
    const int e = base + threadIdx.x;
    const bool k = e < E && w.keep[e];
    const unsigned m = __ballot_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&w.counters[C_KEPT], __popc(m));
    if (k) uf_union(w.parent, w.perm[w.src[e]], w.perm[w.col[e]], w.counters);
  }
}

__global__ void k_cc_label(Batch b, Ws w) {
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < b.n_hits;
       v += gridDim.x * blockDim.x) {
    const int i = w.perm[v];
    const int r = uf_find(w.parent, i);
    b.labels[i] = r - int(b.offsets[w.node_event[v]]);
  }
}

// ---------------------------------------------------------------------------
// Component labelling without allocation (gnntrk_components_noalloc).
//
// For callers that may not allocate device memory, the union-find parents live
// in one file-scope device array of fixed size instead of a handle's
// workspace. The array exists on every device that loads the library and
// stays until the process exits. Every call on a device reuses it, so each
// call first rewrites the part it needs (status word and parents); calls whose
// work overlaps on the GPU would race on it.
// ---------------------------------------------------------------------------
constexpr int kNoAllocHeader = 64;  // ints: [C_STATUS] status word, rest padding
constexpr int kMaxDevices = 64;
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocHeader + GNNTRK_NOALLOC_MAX_HITS];

std::mutex g_noalloc_mu;
int32_t* g_noalloc_ptr[kMaxDevices] = {};

__global__ void k_na_init(int32_t* scratch, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kNoAllocHeader) scratch[t] = 0;
  int32_t* P = scratch + kNoAllocHeader;
  for (int v = t; v < n; v += gridDim.x * blockDim.x) P[v] = v;
}

__global__ void k_na_union(int32_t* scratch, int n, int ne, const int32_t* src,
                           const int32_t* dst, const uint8_t* kept) {
  int32_t* P = scratch + kNoAllocHeader;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    if (kept != nullptr && !kept[e]) continue;
    const int a = src[e], b = dst[e];
    if (a < 0 || a >= n || b < 0 || b >= n) {
      set_status(scratch, ST_INPUT);
      continue;
    }
    uf_union(P, a, b, scratch);
  }
}

__global__ void k_na_label(const int32_t* scratch, int n, int32_t* labels) {
  const bool bad = *(volatile const int32_t*)&scratch[C_STATUS] != 0;
  int32_t* P = const_cast<int32_t*>(scratch) + kNoAllocHeader;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    labels[v] = bad ? -1 : uf_find(P, v);
}

// ---------------------------------------------------------------------------
// One block per event: events are independent and their hits and edges are
// contiguous (sorted positions are event-major, edges are CSR rows), so the
// union-find runs in shared memory over event-local input indices, with the
// same hooking rule. An event with more than kCcSmemHits hits runs the same
// steps on its slice of the global parent array.
// ---------------------------------------------------------------------------
constexpr int kCcThreads = 512;
constexpr int kCcSmemHits = 6144;

__global__ void __launch_bounds__(kCcThreads) k_cc_event(Batch b, Ws w) {
  extern __shared__ int32_t sm_cc[];
  int32_t* sP = sm_cc;                // [kCcSmemHits] parents (event-local input index)
  int32_t* sL = sm_cc + kCcSmemHits;  // [kCcSmemHits] local input index of sorted position
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  int kept = 0;
  for (int ev = blockIdx.x; ev < b.n_events; ev += gridDim.x) {
    const int v0 = int(w.ev_off[ev]), v1 = int(w.ev_off[ev + 1]);
    const int n = v1 - v0;
    const int e0 = min(w.row_ptr[v0], E), e1 = min(w.row_ptr[v1], E);
    const bool small = n <= kCcSmemHits;
    int32_t* P = small ? sP : w.parent + v0;  // local index -> parent
    for (int i = threadIdx.x; i < n; i += kCcThreads) {
      P[i] = i;
      if (small) sL[i] = w.perm[v0 + i] - v0;
    }
    __syncthreads();
    for (int e = e0 + threadIdx.x; e < e1; e += kCcThreads) {
      if (!w.keep[e]) continue;
      ++kept;
      const int a = w.src[e] - v0, c = w.col[e] - v0;
      uf_union(P, small ? sL[a] : w.perm[v0 + a] - v0, small ? sL[c] : w.perm[v0 + c] - v0,
               w.counters);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kCcThreads) {
      const int li = small ? sL[i] : w.perm[v0 + i] - v0;
      b.labels[v0 + li] = uf_find(P, li);
    }
    __syncthreads();  // P and L are reused by the next event
  }
  // kept-edge count
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&w.counters[C_KEPT], kept);
}

}  // namespace

void set_global_error(const std::string& msg);

// Device address of the scratch array on the current device. Looked up on
// every call made outside a stream capture (a device reset may reload the
// module at another address), and remembered per device for calls made while
// `s` is being captured, where the last uncaptured lookup is used.
static cudaError_t noalloc_scratch(cudaStream_t s, int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    int32_t* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  } else if (g_noalloc_ptr[dev] == nullptr) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

void launch_cc(const Batch& b, const Ws& w, cudaStream_t s) {
  if (b.n_events <= 0 || b.n_hits <= 0) {
    k_cc_union<<<device_sms() * 8, 256, 0, s>>>(w);
    return;
  }
  // set once per process (thread-safe initialisation of a local static)
  static const bool attr_set = [] {
    cudaFuncSetAttribute(k_cc_event, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * kCcSmemHits * int(sizeof(int32_t)));
    return true;
  }();
  (void)attr_set;
  k_cc_event<<<std::min(b.n_events, device_sms() * 16), kCcThreads,
               2 * kCcSmemHits * sizeof(int32_t), s>>>(b, w);
}

}  // namespace gnntrk

extern "C" gnntrk_status gnntrk_components_noalloc(int64_t n_hits, int64_t n_edges,
                                                   const int32_t* src, const int32_t* dst,
                                                   const uint8_t* kept, int32_t* out_labels,
                                                   void* stream) {
  using namespace gnntrk;
  if (n_hits < 0 || n_hits > GNNTRK_NOALLOC_MAX_HITS) {
    set_global_error("gnntrk_components_noalloc: n_hits " + std::to_string(n_hits) +
                     " outside 0.." + std::to_string(GNNTRK_NOALLOC_MAX_HITS) +
                     " (the fixed scratch array holds at most that many vertices)");
    return GNNTRK_ERR_INVALID_ARG;
  }
  if (n_edges < 0 || n_edges > 0x7fffffffLL) {
    set_global_error("gnntrk_components_noalloc: n_edges outside 0..2^31-1");
    return GNNTRK_ERR_INVALID_ARG;
  }
  if ((n_hits > 0 && out_labels == nullptr) || (n_edges > 0 && (src == nullptr || dst == nullptr))) {
    set_global_error("gnntrk_components_noalloc: NULL pointer");
    return GNNTRK_ERR_INVALID_ARG;
  }
  if (n_hits == 0 && n_edges > 0) {
    set_global_error("gnntrk_components_noalloc: edges given with n_hits == 0");
    return GNNTRK_ERR_INVALID_ARG;
  }
  if (n_hits == 0) return GNNTRK_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* scratch = nullptr;
  cudaError_t e = noalloc_scratch(s, &scratch);
  if (e != cudaSuccess) {
    set_global_error(std::string("gnntrk_components_noalloc: scratch address: ") +
                     cudaGetErrorString(e));
    return GNNTRK_ERR_CUDA;
  }
  const int n = int(n_hits), ne = int(n_edges);
  k_na_init<<<div_up(n > kNoAllocHeader ? n : kNoAllocHeader, 256), 256, 0, s>>>(scratch, n);
  if (ne > 0) k_na_union<<<device_sms() * 8, 256, 0, s>>>(scratch, n, ne, src, dst, kept);
  k_na_label<<<div_up(n, 256), 256, 0, s>>>(scratch, n, out_labels);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("gnntrk_components_noalloc: launch: ") + cudaGetErrorString(e));
    return GNNTRK_ERR_CUDA;
  }
  return GNNTRK_OK;
}
