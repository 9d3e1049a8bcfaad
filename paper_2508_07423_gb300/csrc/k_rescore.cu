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
// as an FP32 run of the whole event. A stable counting sort by level
// (descending) turns the levels into one row list whose prefix [0, cnt_ge[k])
// is the set of step k, rows in index order within a level.
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

// E_{K-1} = band edges, V_{K-1} = their endpoints; flags the events. Four
// edges per thread and iteration; the band count is summed per thread and
// added once per warp.
__device__ __forceinline__ int rs_init_edge(const Ws& w, int e, float l, float lo, float hi,
                                            int8_t top) {
  if (!(l > lo && l < hi)) return 0;
  w.rs_elev[e] = top;
  const int a = w.src[e], c = w.col[e];
  w.rs_nlev[a] = top;  // every writer stores the same value
  w.rs_nlev[c] = top;
  w.ev_flag[w.node_event[a]] = 1;
  return 1;
}

__global__ void k_rs_init(Ws w, float lo, float hi, int K) {
  if (input_bad(w.counters)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int8_t top = int8_t((K > 0 ? K - 1 : -1) + 2);
  const int stride = gridDim.x * blockDim.x;
  const int E4 = E / 4;
  int n = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E4; i += stride) {
    const float4 l = reinterpret_cast<const float4*>(w.logit)[i];
    n += rs_init_edge(w, 4 * i, l.x, lo, hi, top);
    n += rs_init_edge(w, 4 * i + 1, l.y, lo, hi, top);
    n += rs_init_edge(w, 4 * i + 2, l.z, lo, hi, top);
    n += rs_init_edge(w, 4 * i + 3, l.w, lo, hi, top);
  }
  for (int e = 4 * E4 + blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride)
    n += rs_init_edge(w, e, w.logit[e], lo, hi, top);
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&w.counters[C_BAND], n);
}

__device__ __forceinline__ void rs_step_edge(const Ws& w, int8_t& L, int a, int c, int8_t la,
                                             int8_t lc, int8_t ge_k, int8_t km1, bool& changed) {
  if (L < km1 && (la >= ge_k || lc >= ge_k)) {
    L = km1;
    changed = true;
  }
  if (L >= km1) {
    if (la < km1) w.rs_nlev[a] = km1;
    if (lc < km1) w.rs_nlev[c] = km1;
  }
}

// four consecutive edges per thread and iteration: their levels, sources and
// targets in one 4-byte and two 16-byte loads, the eight hit-level gathers in
// flight together
__global__ void k_rs_step(Ws w, int k) {
  if (input_bad(w.counters)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int8_t ge_k = int8_t(k + 2), km1 = int8_t(k + 1);
  const int stride = gridDim.x * blockDim.x;
  const int E4 = E / 4;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E4; i += stride) {
    char4 L4 = reinterpret_cast<const char4*>(w.rs_elev)[i];
    const int4 a4 = reinterpret_cast<const int4*>(w.src)[i];
    const int4 c4 = reinterpret_cast<const int4*>(w.col)[i];
    const int8_t la0 = w.rs_nlev[a4.x], la1 = w.rs_nlev[a4.y], la2 = w.rs_nlev[a4.z], la3 = w.rs_nlev[a4.w];
    const int8_t lc0 = w.rs_nlev[c4.x], lc1 = w.rs_nlev[c4.y], lc2 = w.rs_nlev[c4.z], lc3 = w.rs_nlev[c4.w];
    int8_t L0 = L4.x, L1 = L4.y, L2 = L4.z, L3 = L4.w;
    bool changed = false;
    rs_step_edge(w, L0, a4.x, c4.x, la0, lc0, ge_k, km1, changed);
    rs_step_edge(w, L1, a4.y, c4.y, la1, lc1, ge_k, km1, changed);
    rs_step_edge(w, L2, a4.z, c4.z, la2, lc2, ge_k, km1, changed);
    rs_step_edge(w, L3, a4.w, c4.w, la3, lc3, ge_k, km1, changed);
    if (changed) reinterpret_cast<char4*>(w.rs_elev)[i] = make_char4(L0, L1, L2, L3);
  }
  for (int e = 4 * E4 + blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    int8_t L = w.rs_elev[e];
    const int a = w.src[e], c = w.col[e];
    bool changed = false;
    rs_step_edge(w, L, a, c, w.rs_nlev[a], w.rs_nlev[c], ge_k, km1, changed);
    if (changed) w.rs_elev[e] = L;
  }
}

// Stable counting sort of the levels. Bucket = top - shifted level (bucket 0
// holds the highest level); rows at level 0 (not needed) are dropped.
struct SortSide {
  const int8_t* lev;
  int32_t* list;
  int32_t* blk_cnt;      // [nb][gridDim.x] rows per bucket per block, then block offsets
  const int32_t* n_ptr;  // row count on the device (edges) or null
  int n_fixed;
  int32_t* cge;          // [K + 1]: rows with level >= k at [k + 1]
  int counter;           // counters index receiving the total
};

__device__ __forceinline__ void chunk_of(int n, int& lo, int& hi) {
  const int per = (((n + gridDim.x - 1) / gridDim.x) + kRsThreads - 1) / kRsThreads * kRsThreads;
  lo = min(n, int(blockIdx.x) * per);
  hi = min(n, lo + per);
}

__device__ __forceinline__ int side_rows(const SortSide& sd) {
  return sd.n_ptr ? min(*sd.n_ptr, sd.n_fixed) : sd.n_fixed;
}

// per block and bucket, the number of rows (ballot counts, no atomics)
__global__ void __launch_bounds__(kRsThreads) k_rs_count(SortSide se, SortSide sn, int K,
                                                         const int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.y == 0 ? se : sn;
  const int nb = K + 1, top = K + 1;
  __shared__ int cnt[kRsWarps][kMaxIters + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int mine = 0;  // lane j of each warp counts bucket j
  int lo, hi;
  chunk_of(side_rows(sd), lo, hi);
  for (int base = lo; base < hi; base += kRsThreads) {
    const int i = base + threadIdx.x;
    const int bk = i < hi ? top - sd.lev[i] : -1;  // level 0 -> bucket K + 1 (dropped)
    for (int j = 0; j < nb; ++j) {
      const int c = __popc(__ballot_sync(0xffffffffu, bk == j));
      if (lane == j) mine += c;
    }
  }
  if (lane < nb) cnt[warp][lane] = mine;
  __syncthreads();
  if (threadIdx.x < nb) {
    int t = 0;
    for (int q = 0; q < kRsWarps; ++q) t += cnt[q][threadIdx.x];
    sd.blk_cnt[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// exclusive offsets per (bucket, block) in bucket-major order; one block per side
__global__ void __launch_bounds__(1024) k_rs_offsets(SortSide se, SortSide sn, int K, int nblk,
                                                     int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.x == 0 ? se : sn;
  const int nb = K + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int tot[kMaxIters + 2];
  // warp j scans bucket j over the blocks
  if (warp < nb) {
    int32_t* row = sd.blk_cnt + warp * nblk;
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
    if (lane == 0) tot[warp] = run;
  }
  __syncthreads();
  __shared__ int base[kMaxIters + 2];
  if (threadIdx.x == 0) {
    int run = 0;
    for (int j = 0; j < nb; ++j) {  // bucket j = level K-1-j
      base[j] = run;
      run += tot[j];
      sd.cge[K - 1 - j + 1] = run;  // rows with level >= K-1-j
    }
    counters[sd.counter] = run;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j)
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) sd.blk_cnt[j * nblk + b] += base[j];
}

// scatter in the same chunk and tile order as the count: stable
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(SortSide se, SortSide sn, int K,
                                                           const int32_t* counters) {
  if (input_bad(counters)) return;
  const SortSide& sd = blockIdx.y == 0 ? se : sn;
  const int nb = K + 1, top = K + 1;
  __shared__ int wtot[kRsWarps][kMaxIters + 2];
  __shared__ int run[kMaxIters + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x < nb) run[threadIdx.x] = sd.blk_cnt[threadIdx.x * gridDim.x + blockIdx.x];
  int lo, hi;
  chunk_of(side_rows(sd), lo, hi);
  for (int base = lo; base < hi; base += kRsThreads) {
    const int i = base + threadIdx.x;
    const int bk = i < hi ? top - sd.lev[i] : -1;
    int rank = 0;
    for (int j = 0; j < nb; ++j) {
      const unsigned m = __ballot_sync(0xffffffffu, bk == j);
      if (bk == j) rank = __popc(m & lt);
      if (lane == 0) wtot[warp][j] = __popc(m);
    }
    __syncthreads();
    if (bk >= 0 && bk < nb) {
      int off = run[bk];
      for (int q = 0; q < warp; ++q) off += wtot[q][bk];
      sd.list[off + rank] = i;
    }
    __syncthreads();
    if (threadIdx.x < nb) {
      int t = 0;
      for (int q = 0; q < kRsWarps; ++q) t += wtot[q][threadIdx.x];
      run[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

}  // namespace

int rescore_sort_blocks() { return std::min(device_sms() * 4, kRsMaxBlocks); }

int launch_rescore_sets(const Batch& b, const Ws& w, float band_lo, float band_hi, int K,
                        cudaStream_t s) {
  const int NL = kMaxIters + 2;
  const int grid = device_sms() * 8;
  const int nblk = rescore_sort_blocks();
  cudaMemsetAsync(w.ev_flag, 0, sizeof(int32_t) * b.n_events, s);
  cudaMemsetAsync(w.rs_counts, 0, sizeof(int32_t) * 6 * NL, s);
  cudaMemsetAsync(w.rs_elev, 0, size_t(w.e_cap), s);
  cudaMemsetAsync(w.rs_nlev, 0, size_t(b.n_hits), s);
  k_rs_init<<<grid, kRsThreads, 0, s>>>(w, band_lo, band_hi, K);
  for (int k = K - 1; k >= 0; --k) k_rs_step<<<grid, kRsThreads, 0, s>>>(w, k);
  SortSide se{w.rs_elev, w.rs_elist, w.rs_blk, w.counters + C_EDGES, int(w.e_cap),
              w.rs_counts + 2 * NL, C_RERUN_EDGES};
  SortSide sn{w.rs_nlev, w.rs_nlist, w.rs_blk + NL * nblk, nullptr, b.n_hits,
              w.rs_counts + 5 * NL, C_RERUN_HITS};
  k_rs_count<<<dim3(nblk, 2), kRsThreads, 0, s>>>(se, sn, K, w.counters);
  k_rs_offsets<<<2, 1024, 0, s>>>(se, sn, K, nblk, w.counters);
  k_rs_scatter<<<dim3(nblk, 2), kRsThreads, 0, s>>>(se, sn, K, w.counters);
  return 1 + K + 3;
}

}  // namespace gnntrk
