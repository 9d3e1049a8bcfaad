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

}  // namespace

void launch_cc(const Batch& b, const Ws& w, cudaStream_t s) {
  k_cc_union<<<device_sms() * 8, 256, 0, s>>>(w);
  if (b.n_hits > 0) k_cc_label<<<div_up(b.n_hits, 256), 256, 0, s>>>(b, w);
}

}  // namespace gnntrk
