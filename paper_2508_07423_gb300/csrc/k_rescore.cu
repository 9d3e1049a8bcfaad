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
// as an FP32 run of the whole event. The same kernel lists each step's rows
// (level >= k) in index order for the FP32 kernels.
//
// Levels are stored as int8 shifted by +2 (0 = not needed, 1 = encoders only,
// k + 2 = up to step k), in shared memory for the event a block works on
// (the workspace arrays rs_elev / rs_nlev for events too large for it).
#include <algorithm>

#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

__device__ __forceinline__ bool input_bad(const int32_t* counters) {
  return (*(volatile const int32_t*)&counters[C_STATUS] & ST_INPUT) != 0;
}

// Levels of one event, indexed event-locally: el[e - e0] for its edges,
// nl[v - v0] for its hits (shared memory when the event fits, else the
// event's slices of the workspace arrays).
struct EvLevels {
  int8_t* el;
  int8_t* nl;
  int e0, v0;
};

// E_{K-1} = band edges, V_{K-1} = their endpoints (event-local a, c). Returns
// 1 for a band edge.
__device__ __forceinline__ int rs_init_edge(const EvLevels& L, int k, int a, int c, float l,
                                            float lo, float hi, int8_t top) {
  if (!(l > lo && l < hi)) return 0;
  L.el[k] = top;
  L.nl[a] = top;  // every writer stores the same value
  L.nl[c] = top;
  return 1;
}

// Step k of the backward walk for one edge (event-local index ke, endpoints
// a, c): the edge joins E_{k-1} if an endpoint is in V_k (level >= k + 2); an
// edge of E_{k-1} puts its endpoints in V_{k-1}. Within one sweep a hit level
// only rises to k + 1, which no other edge of the same sweep tests for, so
// the sweep does not depend on the order of its edges.
__device__ __forceinline__ void rs_step_edge(const EvLevels& L, int ke, int a, int c, int8_t ge_k,
                                             int8_t km1) {
  int8_t le = L.el[ke];
  const int8_t la = L.nl[a], lc = L.nl[c];
  if (le < km1 && (la >= ge_k || lc >= ge_k)) {
    le = km1;
    L.el[ke] = le;
  }
  if (le >= km1) {
    if (la < km1) L.nl[a] = km1;
    if (lc < km1) L.nl[c] = km1;
  }
}

// The whole receptive field and the row lists of every step, one block per
// event (events share no hits and no edges): clear the event's levels, mark
// the band edges and their endpoints, the K backward steps with a block
// barrier between them, then the event's rows of each list. List t (t = 0 ..
// K, step k = t - 1) holds the rows of level >= k in index order, so that a
// step's kernels visit rows in the batch's event order, as the full FP32 path
// does. Events go to blocks in index order by a ticket (counters[C_RS_TICKET])
// and each takes its offsets in the 2 (K + 1) lists from a look-back over the
// counts its predecessors publish (flag 1: the event's own counts, flag 2: the
// counts up to and including it), so a block only waits for blocks that took
// their tickets before it. Counts the band edges into counters[C_BAND] and the
// events holding one into counters[C_RERUN].
constexpr int kRsEvThreads = 512;
constexpr int kRsEvWarps = kRsEvThreads / 32;
constexpr int kRsLists = 2 * (kMaxIters + 1);
constexpr int kRsLookbackSpins = 1 << 22;  // x >= 100 ns sleeps: about half a second
constexpr int kRsSmemBytes = 96 * 1024;  // endpoints and levels: about 19 k edges per event

struct RsDesc {
  int32_t* flag;  // [n_events]
  int32_t* agg;   // [n_events][2 (K + 1)] the event's own counts
  int32_t* inc;   // [n_events][2 (K + 1)] counts up to and including the event
};

__device__ __forceinline__ int ld_vol(const int32_t* p) { return *(volatile const int32_t*)p; }

// The event's rows of one side (edges or hits, [r0, r1)) are cut into one
// contiguous segment per warp, so that counting and placement need no block
// barrier inside their loops: warp q counts its segment's rows per list,
// a block scan over the warps gives each warp its offset in every list, and
// the warp then places its rows in order (ballot ranks).
__device__ __forceinline__ void rs_segment(int r0, int r1, int warp, int& a, int& z) {
  const int len = (((r1 - r0) + kRsEvWarps - 1) / kRsEvWarps + 31) / 32 * 32;
  a = min(r1, r0 + warp * len);
  z = min(r1, a + len);
}

// counts of this warp's rows per list t (t = 0 .. K) into wcnt[t][warp]
__device__ void rs_count_warp(const int8_t* lev, int r0, int r1, int K, int (*wcnt)[kRsEvWarps]) {
  // lev[r - r0]: the level of row r
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int a, z;
  rs_segment(r0, r1, warp, a, z);
  int mine = 0;  // lane t holds the count of list t
  for (int c0 = a; c0 < z; c0 += 32) {
    const int r = c0 + lane;
    const int l = r < z ? lev[r - r0] : 0;
    for (int t = 0; t <= K; ++t) {
      const int n = __popc(__ballot_sync(0xffffffffu, l >= t + 1));
      if (lane == t) mine += n;
    }
  }
  if (lane <= K) wcnt[lane][warp] = mine;
}

// this warp's rows into list t at run[t][warp] (t = 0 .. K), in index order
__device__ void rs_place_warp(const int8_t* lev, int r0, int r1, int K, int32_t* list,
                              int64_t stride, int (*run)[kRsEvWarps]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int a, z;
  rs_segment(r0, r1, warp, a, z);
  int mine = lane <= K ? run[lane][warp] : 0;  // lane t: next position in list t
  for (int c0 = a; c0 < z; c0 += 32) {
    const int r = c0 + lane;
    const int l = r < z ? lev[r - r0] : 0;
    for (int t = 0; t <= K; ++t) {
      const unsigned m = __ballot_sync(0xffffffffu, l >= t + 1);
      const int at = __shfl_sync(0xffffffffu, mine, t);
      if (l >= t + 1) list[t * stride + at + __popc(m & lt)] = r;
      if (lane == t) mine += __popc(m);
    }
  }
}

// Warp 0: publishes the event's counts cnt[0 .. nv) and sets base[v] to the
// counts of all earlier events. A wait that runs out sets ST_TIMEOUT.
__device__ void rs_lookback(const RsDesc& d, int ev, int nv, const int* cnt, int* base,
                            int32_t* counters) {
  const int lane = threadIdx.x & 31;
  for (int v = lane; v < nv; v += 32) {
    base[v] = 0;
    (ev == 0 ? d.inc : d.agg)[size_t(ev) * nv + v] = cnt[v];
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) atomicExch(d.flag + ev, ev == 0 ? 2 : 1);
  int spins = 0;
  bool timed_out = false;
  for (int top = ev - 1; top >= 0 && !timed_out; top -= 32) {
    const int i = top - lane;
    int f = i >= 0 ? ld_vol(d.flag + i) : 2;  // before event 0: counts of 0
    while (__any_sync(0xffffffffu, f == 0)) {
      if (++spins > kRsLookbackSpins) {
        timed_out = true;
        break;
      }
      __nanosleep(100);
      if (f == 0) f = ld_vol(d.flag + i);
    }
    if (timed_out) break;
    __threadfence();  // the counts were written before the flags read above
    const unsigned incm = __ballot_sync(0xffffffffu, f == 2);
    const int stop = incm ? __ffs(incm) - 1 : 31;  // the nearest inclusive counts
    const int32_t* src = f == 2 ? d.inc : d.agg;
    for (int v = 0; v < nv; ++v) {
      int x = (lane <= stop && i >= 0) ? ld_vol(src + size_t(i) * nv + v) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) base[v] += x;
    }
    __syncwarp();
    if (incm) break;
  }
  if (timed_out) {
    if (lane == 0) set_status(counters, ST_TIMEOUT);
    return;
  }
  if (ev > 0) {
    for (int v = lane; v < nv; v += 32) d.inc[size_t(ev) * nv + v] = base[v] + cnt[v];
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(d.flag + ev, 2);
  }
}

__global__ void __launch_bounds__(kRsEvThreads) k_rs_event(Batch b, Ws w, RsDesc d, float lo,
                                                          float hi, int K) {
  extern __shared__ __align__(16) int8_t sm_lev[];  // endpoints and levels of the event
  if (input_bad(w.counters)) return;
  __shared__ int wsum[kRsEvWarps];
  __shared__ int wcnt[kRsLists][kRsEvWarps];  // per list and warp: rows, then offsets
  __shared__ int cnt_s[kRsLists];
  __shared__ int base_s[kRsLists];
  __shared__ int ticket_s;
  const int NL = kMaxIters + 2;
  const int nv = 2 * (K + 1);
  const int E = clamp_edges(w.counters, w.e_cap);
  const int8_t top = int8_t((K > 0 ? K - 1 : -1) + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  int band_total = 0, band_events = 0;
  for (;;) {
    if (tid == 0) ticket_s = atomicAdd(&w.counters[C_RS_TICKET], 1);
    __syncthreads();
    const int ev = ticket_s;
    if (ev >= b.n_events) break;
    const int v0 = int(w.ev_off[ev]), v1 = int(w.ev_off[ev + 1]);
    const int e0 = min(w.row_ptr[v0], E), e1 = min(w.row_ptr[v1], E);
    // shared memory, when the event fits: [endpoints 4 B per edge][hit
    // levels][edge levels]; the endpoints (event-local, 16 bits each) only
    // for events of at most 65536 hits, read once and reused by every sweep
    const int nh = v1 - v0, ne = e1 - e0;
    const bool staged = nh + ne <= kRsSmemBytes;
    const bool eps = staged && nh <= 65536 && 5 * int64_t(ne) + nh <= kRsSmemBytes;
    uint32_t* ep = reinterpret_cast<uint32_t*>(sm_lev);
    int8_t* lev0 = eps ? sm_lev + 4 * ne : sm_lev;
    const EvLevels L{staged ? lev0 + nh : w.rs_elev + e0, staged ? lev0 : w.rs_nlev + v0, e0, v0};
    for (int i = tid; i < nh; i += kRsEvThreads) L.nl[i] = 0;
    for (int e = tid; e < ne; e += kRsEvThreads) L.el[e] = 0;
    __syncthreads();
    int n = 0;
    for (int k = tid; k < ne; k += kRsEvThreads) {
      const int a = w.src[e0 + k] - v0, c = w.col[e0 + k] - v0;
      if (eps) ep[k] = uint32_t(a) | (uint32_t(c) << 16);
      n += rs_init_edge(L, k, a, c, w.logit[e0 + k], lo, hi, top);
    }
    __syncthreads();
    for (int kk = K - 1; kk >= 0; --kk) {
      const int8_t ge_k = int8_t(kk + 2), km1 = int8_t(kk + 1);
      for (int k = tid; k < ne; k += kRsEvThreads) {
        int a, c;
        if (eps) {
          const uint32_t u = ep[k];
          a = int(u & 0xffffu);
          c = int(u >> 16);
        } else {
          a = w.src[e0 + k] - v0;
          c = w.col[e0 + k] - v0;
        }
        rs_step_edge(L, k, a, c, ge_k, km1);
      }
      __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((tid & 31) == 0) wsum[warp] = n;
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int q = 0; q < kRsEvWarps; ++q) t += wsum[q];
      band_total += t;
      band_events += t > 0;
    }
    // the event's rows per list, their offsets, then placement
    rs_count_warp(L.el, e0, e1, K, wcnt);
    rs_count_warp(L.nl, v0, v1, K, wcnt + K + 1);
    __syncthreads();
    if (tid < nv) {  // exclusive scan over the warps, the event's count per list
      int run = 0;
      for (int q = 0; q < kRsEvWarps; ++q) {
        const int c = wcnt[tid][q];
        wcnt[tid][q] = run;
        run += c;
      }
      cnt_s[tid] = run;
    }
    __syncthreads();
    if (warp == 0) rs_lookback(d, ev, nv, cnt_s, base_s, w.counters);
    __syncthreads();
    if (tid < nv)
      for (int q = 0; q < kRsEvWarps; ++q) wcnt[tid][q] += base_s[tid];
    __syncthreads();
    rs_place_warp(L.el, e0, e1, K, w.rs_elist, w.e_cap, wcnt);
    rs_place_warp(L.nl, v0, v1, K, w.rs_nlist, w.h_cap, wcnt + K + 1);
    if (ev == b.n_events - 1 && tid <= K) {
      // the totals of every list
      w.rs_counts[2 * NL + tid] = base_s[tid] + cnt_s[tid];
      w.rs_counts[5 * NL + tid] = base_s[K + 1 + tid] + cnt_s[K + 1 + tid];
      if (tid == 0) {
        w.counters[C_RERUN_EDGES] = base_s[0] + cnt_s[0];
        w.counters[C_RERUN_HITS] = base_s[K + 1] + cnt_s[K + 1];
      }
    }
    __syncthreads();  // shared counts and ticket_s are reused by the next event
  }
  if (tid == 0 && band_total) {
    atomicAdd(&w.counters[C_BAND], band_total);
    atomicAdd(&w.counters[C_RERUN], band_events);
  }
}

}  // namespace

int launch_rescore_sets(const Batch& b, const Ws& w, float band_lo, float band_hi, int K,
                        cudaStream_t s) {
  const int NL = kMaxIters + 2;
  cudaMemsetAsync(w.rs_counts, 0, sizeof(int32_t) * 6 * NL, s);
  if (b.n_events <= 0) return 0;
  cudaMemsetAsync(w.rs_desc, 0, sizeof(int32_t) * b.n_events, s);
  const int nv = 2 * (K + 1);
  const RsDesc d{w.rs_desc, w.rs_desc + b.n_events, w.rs_desc + b.n_events + size_t(b.n_events) * nv};
  // set once per process (thread-safe initialisation of a local static)
  static const bool attr = [] {
    cudaFuncSetAttribute(k_rs_event, cudaFuncAttributeMaxDynamicSharedMemorySize, kRsSmemBytes);
    return true;
  }();
  (void)attr;
  k_rs_event<<<std::min(b.n_events, device_sms() * 2), kRsEvThreads, kRsSmemBytes, s>>>(
      b, w, d, band_lo, band_hi, K);
  return 1;
}

}  // namespace gnntrk
