// Exact receptive field of the near-cut edges, for the FP32 re-score.
//
// The logit of an edge after K message-passing steps depends on a K-hop
// neighbourhood; working backwards from the band edges B gives, per step, the
// rows whose FP32 values are needed (sets nest, so one level per row says up
// to which step the row is computed):
//   edge step K-1 : E_{K-1} = B
//   node step k   : V_k = V_{k+1} + endpoints(E_k)          (V_K empty)
//   edge step k-1 : E_{k-1} = edges incident to V_k       (their e^k feeds the sums)
//   node encoder  : V_{-1} = V_0 + endpoints(E_{-1}); edge encoder: E_{-1}
// Recomputing exactly these rows in FP32 gives the band edges the same logits
// as an FP32 run of the whole event. A counting sort by level (descending)
// turns the levels into one row list whose prefix [0, cnt_ge[k]) is the set of
// step k.
#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

__device__ __forceinline__ bool input_bad(const Ws& w) {
  return (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) != 0;
}

// band edges get level K-1 (or -1 when K = 0), all others -2; nodes -2
__global__ void k_rs_init(Batch b, Ws w, float lo, float hi, int K) {
  if (input_bad(w)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int n = max(E, b.n_hits);
  const int top = K > 0 ? K - 1 : -1;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    bool in = false;
    if (i < E) {
      const float l = w.logit[i];
      in = l > lo && l < hi;
      w.rs_elev[i] = in ? top : -2;
      if (in) w.ev_flag[w.node_event[w.src[i]]] = 1;
    }
    if (i < b.n_hits) w.rs_nlev[i] = -2;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&w.counters[C_BAND], __popc(m));
  }
}

// V_k grows by the endpoints of E_k (edges with level >= k)
__global__ void k_rs_nodes(Ws w, int k) {
  if (input_bad(w)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    if (w.rs_elev[e] >= k) {
      atomicMax(&w.rs_nlev[w.src[e]], k);
      atomicMax(&w.rs_nlev[w.col[e]], k);
    }
}

// E_{k-1}: edges incident to a node of V_k (level >= k)
__global__ void k_rs_edges(Ws w, int k) {
  if (input_bad(w)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    if (w.rs_elev[e] < k - 1 && (w.rs_nlev[w.src[e]] >= k || w.rs_nlev[w.col[e]] >= k))
      w.rs_elev[e] = k - 1;
}

// histogram of levels -1 .. K-1 into buckets K-1-level (so bucket 0 = top)
__global__ void k_rs_count(const int32_t* lev, const int32_t* n_ptr, int n_fixed, int32_t* hist,
                           int K, const int32_t* counters) {
  __shared__ int h[kMaxIters + 2];
  if ((*(volatile const int32_t*)&counters[C_STATUS]) & ST_INPUT) return;
  const int nb = K + 1;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int n = n_ptr ? min(*n_ptr, n_fixed) : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = lev[i];
    if (l >= -1) atomicAdd(&h[K - 1 - l], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// cursors (exclusive prefix over buckets) and cnt_ge[k + 1] = rows with
// level >= k, for k = -1 .. K-1
__global__ void k_rs_offsets(int32_t* rs, int K, int32_t* counters) {
  if ((*(volatile int32_t*)&counters[C_STATUS]) & ST_INPUT) return;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int NL = kMaxIters + 2;
  for (int side = 0; side < 2; ++side) {  // 0 edges, 1 nodes
    int32_t* hist = rs + side * 3 * NL;
    int32_t* cur = hist + NL;
    int32_t* cge = hist + 2 * NL;
    int run = 0;
    for (int bkt = 0; bkt <= K; ++bkt) {  // level K-1-bkt
      cur[bkt] = run;
      run += hist[bkt];
      cge[K - 1 - bkt + 1] = run;  // rows with level >= K-1-bkt
    }
    counters[side == 0 ? C_RERUN_EDGES : C_RERUN_HITS] = run;
  }
}

__global__ void k_rs_scatter(const int32_t* lev, const int32_t* n_ptr, int n_fixed, int32_t* cur,
                             int32_t* list, int K, const int32_t* counters) {
  if ((*(volatile const int32_t*)&counters[C_STATUS]) & ST_INPUT) return;
  const int n = n_ptr ? min(*n_ptr, n_fixed) : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = lev[i];
    if (l >= -1) list[atomicAdd(&cur[K - 1 - l], 1)] = i;
  }
}

}  // namespace

int launch_rescore_sets(const Batch& b, const Ws& w, float band_lo, float band_hi, int K,
                        cudaStream_t s) {
  const int NL = kMaxIters + 2;
  const int grid = device_sms() * 8;
  int launches = 0;
  cudaMemsetAsync(w.ev_flag, 0, sizeof(int32_t) * b.n_events, s);
  cudaMemsetAsync(w.rs_counts, 0, sizeof(int32_t) * 6 * NL, s);
  k_rs_init<<<grid, 256, 0, s>>>(b, w, band_lo, band_hi, K);
  ++launches;
  for (int k = K - 1; k >= 0; --k) {
    k_rs_nodes<<<grid, 256, 0, s>>>(w, k);
    k_rs_edges<<<grid, 256, 0, s>>>(w, k);
    launches += 2;
  }
  k_rs_nodes<<<grid, 256, 0, s>>>(w, -1);
  ++launches;
  int32_t* he = w.rs_counts;
  int32_t* hn = w.rs_counts + 3 * NL;
  k_rs_count<<<grid, 256, 0, s>>>(w.rs_elev, w.counters + C_EDGES, int(w.e_cap), he, K, w.counters);
  k_rs_count<<<grid, 256, 0, s>>>(w.rs_nlev, nullptr, b.n_hits, hn, K, w.counters);
  k_rs_offsets<<<1, 32, 0, s>>>(w.rs_counts, K, w.counters);
  k_rs_scatter<<<grid, 256, 0, s>>>(w.rs_elev, w.counters + C_EDGES, int(w.e_cap), he + NL,
                                    w.rs_elist, K, w.counters);
  k_rs_scatter<<<grid, 256, 0, s>>>(w.rs_nlev, nullptr, b.n_hits, hn + NL, w.rs_nlist, K,
                                    w.counters);
  launches += 5;
  return launches;
}

}  // namespace gnntrk
