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
// as an FP32 run of the whole event. Before each step a stable compaction
// lists that step's rows (level >= k) in index order.
//
// Levels are stored as int8 shifted by +2 (0 = not needed, 1 = encoders only,
// k + 2 = up to step k), so a memset clears them.
#include <algorithm>

#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ bool input_bad(const int32_t* counters) {
  return (*(volatile const int32_t*)&counters[C_STATUS] & ST_INPUT) != 0;
}

// E_{K-1} = band edges, V_{K-1} = their endpoints. Returns 1 for a band edge.
__device__ __forceinline__ int rs_init_edge(const Ws& w, int e, float l, float lo, float hi,
                                            int8_t top) {
  if (!(l > lo && l < hi)) return 0;
  w.rs_elev[e] = top;
  w.rs_nlev[w.src[e]] = top;  // every writer stores the same value
  w.rs_nlev[w.col[e]] = top;
  return 1;
}

// Step k of the backward walk for one edge: the edge joins E_{k-1} if an
// endpoint is in V_k (level >= k + 2); an edge of E_{k-1} puts its endpoints
// in V_{k-1}. Within one sweep a hit level only rises to k + 1, which no
// other edge of the same sweep tests for, so the sweep does not depend on
// the order of its edges.
__device__ __forceinline__ void rs_step_edge(const Ws& w, int e, int8_t ge_k, int8_t km1) {
  int8_t L = w.rs_elev[e];
  const int a = w.src[e], c = w.col[e];
  const int8_t la = w.rs_nlev[a], lc = w.rs_nlev[c];
  if (L < km1 && (la >= ge_k || lc >= ge_k)) {
    L = km1;
    w.rs_elev[e] = L;
  }
  if (L >= km1) {
    if (la < km1) w.rs_nlev[a] = km1;
    if (lc < km1) w.rs_nlev[c] = km1;
  }
}

// The whole receptive field, one block per event (events share no hits and
// no edges): clear the event's levels, mark the band edges and their
// endpoints, then the K backward steps with a block barrier between them;
// counts the band edges into counters[C_BAND] and the events holding one
// into counters[C_RERUN].
constexpr int kRsEvThreads = 512;

__global__ void __launch_bounds__(kRsEvThreads) k_rs_event(Batch b, Ws w, float lo, float hi, int K) {
  if (input_bad(w.counters)) return;
  __shared__ int wsum[kRsEvThreads / 32];
  const int E = clamp_edges(w.counters, w.e_cap);
  const int8_t top = int8_t((K > 0 ? K - 1 : -1) + 2);
  const int tid = threadIdx.x;
  int band_total = 0, band_events = 0;
  for (int ev = blockIdx.x; ev < b.n_events; ev += gridDim.x) {
    const int v0 = int(w.ev_off[ev]), v1 = int(w.ev_off[ev + 1]);
    const int e0 = min(w.row_ptr[v0], E), e1 = min(w.row_ptr[v1], E);
    for (int i = v0 + tid; i < v1; i += kRsEvThreads) w.rs_nlev[i] = 0;
    for (int e = e0 + tid; e < e1; e += kRsEvThreads) w.rs_elev[e] = 0;
    __syncthreads();
    int n = 0;
    for (int e = e0 + tid; e < e1; e += kRsEvThreads) n += rs_init_edge(w, e, w.logit[e], lo, hi, top);
    __syncthreads();
    for (int k = K - 1; k >= 0; --k) {
      const int8_t ge_k = int8_t(k + 2), km1 = int8_t(k + 1);
      for (int e = e0 + tid; e < e1; e += kRsEvThreads) rs_step_edge(w, e, ge_k, km1);
      __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((tid & 31) == 0) wsum[tid >> 5] = n;
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int q = 0; q < kRsEvThreads / 32; ++q) t += wsum[q];
      band_total += t;
      band_events += t > 0;
    }
    __syncthreads();  // wsum is reused by the next event
  }
  if (tid == 0 && band_total) {
    atomicAdd(&w.counters[C_BAND], band_total);
    atomicAdd(&w.counters[C_RERUN], band_events);
  }
}

// Row lists of all steps in one sweep: list t (t = 0 .. K, step k = t - 1)
// holds the rows with level >= k in index order (so a step's kernels visit
// rows in the batch's event order, as the full FP32 path does). Each block
// takes one contiguous chunk of rows; counts per list by ballots, offsets by
// one warp per list, placement in the same order (stable).
struct SortSide {
  const int8_t* lev;
  int32_t* list;         // [K + 1][stride]
  int64_t stride;
  int32_t* blk_cnt;      // [K + 1][gridDim.x] rows per block, then block offsets
  const int32_t* n_ptr;  // row count on the device (edges) or null
  int n_fixed;
  int32_t* cge;          // [K + 1]: rows of step k at [k + 1]
  int counter;           // counters index receiving the encoder step's total
};

constexpr int kRsTile = 4 * kRsThreads;  // rows per block and iteration (4 per thread)

// the block's chunk of rows, a multiple of kRsTile (so every 4-row group is
// 4-byte aligned)
__device__ __forceinline__ void chunk_of(int n, int& lo, int& hi) {
  const int per = (((n + gridDim.x - 1) / gridDim.x) + kRsTile - 1) / kRsTile * kRsTile;
  lo = min(n, int(blockIdx.x) * per);
  hi = min(n, lo + per);
}

__device__ __forceinline__ int side_rows(const SortSide& sd) {
  return sd.n_ptr ? min(*sd.n_ptr, sd.n_fixed) : sd.n_fixed;
}

// shifted levels of the 4 rows i0 .. i0+3 (0 past hi)
__device__ __forceinline__ void levels4(const int8_t* lev, int i0, int hi, int (&l)[4]) {
  if (i0 + 3 < hi) {
    const char4 v = *reinterpret_cast<const char4*>(lev + i0);
    l[0] = v.x;
    l[1] = v.y;
    l[2] = v.z;
    l[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) l[j] = i0 + j < hi ? lev[i0 + j] : 0;
  }
}

// rows of this block's chunk in each list (level >= t - 1, i.e. shifted >= t + 1)
__global__ void __launch_bounds__(kRsThreads) k_rs_count(SortSide se, SortSide sn, int K,
                                                         const int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.y == 0 ? se : sn;
  __shared__ int cnt[kRsWarps][kMaxIters + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lo, hi;
  chunk_of(side_rows(sd), lo, hi);
  int c[kMaxIters + 1];
#pragma unroll
  for (int t = 0; t <= kMaxIters; ++t) c[t] = 0;
  for (int base = lo; base < hi; base += kRsTile) {
    int l[4];
    levels4(sd.lev, base + 4 * threadIdx.x, hi, l);
#pragma unroll
    for (int t = 0; t <= kMaxIters; ++t)
      if (t <= K) c[t] += (l[0] >= t + 1) + (l[1] >= t + 1) + (l[2] >= t + 1) + (l[3] >= t + 1);
  }
#pragma unroll
  for (int t = 0; t <= kMaxIters; ++t) {
    if (t > K) break;
    int v = c[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) cnt[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    int tot = 0;
    for (int q = 0; q < kRsWarps; ++q) tot += cnt[q][threadIdx.x];
    sd.blk_cnt[threadIdx.x * gridDim.x + blockIdx.x] = tot;
  }
}

// exclusive offsets per (list, block); warp t of block `side` scans list t;
// the totals are the steps' row counts, list 0's also the re-score total
__global__ void k_rs_offsets(SortSide se, SortSide sn, int nblk, int K, int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.x == 0 ? se : sn;
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  if (t > K) return;
  int32_t* row = sd.blk_cnt + t * nblk;
  int run = 0;
  for (int b0 = 0; b0 < nblk; b0 += 32) {
    const int v = b0 + lane < nblk ? row[b0 + lane] : 0;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (b0 + lane < nblk) row[b0 + lane] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) {
    sd.cge[t] = run;
    if (t == 0) counters[sd.counter] = run;
  }
}

// placement in the same chunk order as the count (stable): per tile and list,
// each thread's rows ranked by a warp scan and the block's warp totals
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(SortSide se, SortSide sn, int K,
                                                           const int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.y == 0 ? se : sn;
  __shared__ int wtot[2][kMaxIters + 1][kRsWarps];
  __shared__ int run[kMaxIters + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x <= K) run[threadIdx.x] = sd.blk_cnt[threadIdx.x * gridDim.x + blockIdx.x];
  int lo, hi;
  chunk_of(side_rows(sd), lo, hi);
  int par = 0;
  for (int base = lo; base < hi; base += kRsTile, par ^= 1) {
    const int i0 = base + 4 * threadIdx.x;
    int l[4];
    levels4(sd.lev, i0, hi, l);
    int xs[kMaxIters + 1];
#pragma unroll
    for (int t = 0; t <= kMaxIters; ++t) {
      if (t > K) break;
      const int c = (l[0] >= t + 1) + (l[1] >= t + 1) + (l[2] >= t + 1) + (l[3] >= t + 1);
      int x = c;  // inclusive scan over the warp
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      if (lane == 31) wtot[par][t][warp] = x;
      xs[t] = x - c;
    }
    __syncthreads();  // wtot[par] complete; run[] from the previous tile visible
#pragma unroll
    for (int t = 0; t <= kMaxIters; ++t) {
      if (t > K) break;
      int off = run[t] + xs[t];
      for (int q = 0; q < warp; ++q) off += wtot[par][t][q];
      int32_t* list = sd.list + t * sd.stride;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (l[j] >= t + 1) list[off++] = i0 + j;
    }
    __syncthreads();  // every thread has read run[] of this tile
    if (threadIdx.x <= K) {
      int tot = 0;
      for (int q = 0; q < kRsWarps; ++q) tot += wtot[par][threadIdx.x][q];
      run[threadIdx.x] += tot;
    }
  }
}

}  // namespace

int rescore_sort_blocks() { return std::min(device_sms() * 4, kRsMaxBlocks); }

int launch_rescore_sets(const Batch& b, const Ws& w, float band_lo, float band_hi, int K,
                        cudaStream_t s) {
  const int NL = kMaxIters + 2;
  cudaMemsetAsync(w.rs_counts, 0, sizeof(int32_t) * 6 * NL, s);
  if (b.n_events <= 0) return 0;
  k_rs_event<<<std::min(b.n_events, device_sms() * 4), kRsEvThreads, 0, s>>>(b, w, band_lo,
                                                                           band_hi, K);
  return 1;
}

int launch_rescore_lists(const Batch& b, const Ws& w, int K, cudaStream_t s) {
  const int NL = kMaxIters + 2;
  const int nblk = rescore_sort_blocks();
  SortSide se{w.rs_elev, w.rs_elist, w.e_cap, w.rs_blk, w.counters + C_EDGES, int(w.e_cap),
              w.rs_counts + 2 * NL, C_RERUN_EDGES};
  SortSide sn{w.rs_nlev, w.rs_nlist, w.h_cap, w.rs_blk + (kMaxIters + 1) * kRsMaxBlocks, nullptr,
              b.n_hits, w.rs_counts + 5 * NL, C_RERUN_HITS};
  k_rs_count<<<dim3(nblk, 2), kRsThreads, 0, s>>>(se, sn, K, w.counters);
  k_rs_offsets<<<2, 32 * (K + 1), 0, s>>>(se, sn, nblk, K, w.counters);
  k_rs_scatter<<<dim3(nblk, 2), kRsThreads, 0, s>>>(se, sn, K, w.counters);
  return 3;
}

}  // namespace gnntrk
