// Input staging and rough-graph construction.
//
//  k_sort         per event, a stable counting sort of the hits by plane: the
//                 sorted order is (event, plane, input index), so the
//                 candidates of a hit on plane p (planes p+1 and p+2) form one
//                 contiguous range.
//  k_graph_event  per event, the rough graph of Sec. "Hit Embedding and Rough
//                 Graph Construction" in CSR form and its in-edge index (see
//                 the kernel's comment): degrees, offsets (block scan plus a
//                 look-back over the earlier events), fill, in-edge lists.
//  k_scan_*       exclusive scan in two kernels (block sums, with the last
//                 block scanning them; then block scans plus the block offset),
//                 used by the triplet stage.
#include <algorithm>

#include "internal.cuh"

namespace gnntrk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ bool input_bad(const Ws& w) {
  return (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) != 0;
}

// ---------------------------------------------------------------------------
// stable plane sort, one block per event
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_sort(Batch b, Ws w, int P) {
  __shared__ int cnt[kMaxPlanes];
  __shared__ int base[kMaxPlanes];
  __shared__ int wcnt[kSortThreads / 32][kMaxPlanes];
  __shared__ int ctot[kMaxPlanes];
  __shared__ int bad;
  const int ev = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t o0 = b.offsets[ev], o1 = b.offsets[ev + 1];
  if (tid == 0) {
    int f = 0;
    if (o0 < 0 || o1 < o0 || o1 > b.n_hits) f = 1;
    if (ev == 0 && o0 != 0) f = 1;
    if (ev == b.n_events - 1 && o1 != b.n_hits) f = 1;
    if (f) set_status(w.counters, ST_INPUT);
    bad = f;
  }
  for (int i = tid; i < P; i += kSortThreads) cnt[i] = 0;
  for (int i = tid; i < (kSortThreads / 32) * kMaxPlanes; i += kSortThreads)
    (&wcnt[0][0])[i] = 0;
  __syncthreads();
  if (bad) return;
  const int lo = int(o0), hi = int(o1);

  for (int i = lo + tid; i < hi; i += kSortThreads) {
    int p = b.plane[i];
    if (p >= P) {
      set_status(w.counters, ST_INPUT);
      p = P - 1;
    }
    atomicAdd(&cnt[p], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    int32_t* po = w.plane_off + size_t(ev) * (P + 1);
    for (int p = 0; p < P; ++p) {
      base[p] = run;
      po[p] = lo + run;
      run += cnt[p];
    }
    po[P] = hi;
  }
  __syncthreads();

  for (int c0 = lo; c0 < hi; c0 += kSortThreads) {
    const int i = c0 + tid;
    const bool valid = i < hi;
    const int p = valid ? min(int(b.plane[i]), P - 1) : P;
    const unsigned peers = __match_any_sync(kFull, p);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][p] = __popc(peers);
    __syncthreads();
    if (tid < P) {
      int run = 0;
      for (int k = 0; k < kSortThreads / 32; ++k) {
        int t = wcnt[k][tid];
        wcnt[k][tid] = run;
        run += t;
      }
      ctot[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const int d = lo + base[p] + wcnt[warp][p] + rank;
      w.perm[d] = i;
      w.node_event[d] = ev;
      w.pos[d] = make_float4(b.x[i], b.y[i], b.z[i], 0.0f);
      w.in_cnt[d] = 0;
      w.deg[d] = 0;
    }
    __syncthreads();
    if (tid < P) base[tid] += ctot[tid];
    for (int k = tid; k < (kSortThreads / 32) * kMaxPlanes; k += kSortThreads)
      (&wcnt[0][0])[k] = 0;
    __syncthreads();
  }
  for (int i = lo + tid; i < hi; i += kSortThreads) w.parent[i] = i;
}

// ---------------------------------------------------------------------------
// radius search helpers
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ float dist2(const float (&q)[D], const float* c) {
  float cv[D];
  if constexpr (D % 4 == 0) {  // 16-byte loads (rows are 16-byte aligned)
#pragma unroll
    for (int d = 0; d < D; d += 4) {
      const float4 v = *reinterpret_cast<const float4*>(c + d);
      cv[d] = v.x;
      cv[d + 1] = v.y;
      cv[d + 2] = v.z;
      cv[d + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) cv[d] = c[d];
  }
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float t = q[d] - cv[d];
    s = fmaf(t, t, s);
  }
  return s;
}

template <int D>
__device__ __forceinline__ void load_row(const float* r, float (&q)[D]) {
  if constexpr (D % 4 == 0) {
#pragma unroll
    for (int d = 0; d < D; d += 4) {
      const float4 v = *reinterpret_cast<const float4*>(r + d);
      q[d] = v.x;
      q[d + 1] = v.y;
      q[d + 2] = v.z;
      q[d + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) q[d] = r[d];
  }
}

// Candidate rows of an event, by event-local index c. Both forms give d^2 =
// sum_d (q_d - c_d)^2 accumulated by fmaf in increasing d, bit for bit:
//  CandRows  rows of D floats (global memory, events too large to stage);
//  CandNegT  the event staged in shared memory transposed and negated,
//            t[d * ns + c] = -e_c[d], so that two candidates c, c + 1 of one
//            dimension are one 8-byte load and q_d + (-c_d) (exactly q_d - c_d)
//            runs as a packed FP32 add, two candidates per instruction.
template <int D>
struct CandRows {
  const float* e;
  __device__ __forceinline__ float d2(const float (&q)[D], int c) const {
    return dist2<D>(q, e + size_t(c) * D);
  }
  __device__ __forceinline__ void row(int c, float (&q)[D]) const { load_row<D>(e + size_t(c) * D, q); }
};

template <int D>
struct CandNegT {
  const float* t;
  int ns;
  __device__ __forceinline__ float d2(const float (&q)[D], int c) const {
    float s = 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float u = q[d] + t[d * ns + c];
      s = fmaf(u, u, s);
    }
    return s;
  }
  // d^2 of the candidates c and c + 1 (c even), in one lane each
  __device__ __forceinline__ float2 d2_pair(const float (&q)[D], int c) const {
    float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float2 nc = *reinterpret_cast<const float2*>(t + d * ns + c);
      const float2 u = __fadd2_rn(make_float2(q[d], q[d]), nc);
      s = __ffma2_rn(u, u, s);
    }
    return s;
  }
  __device__ __forceinline__ void row(int c, float (&q)[D]) const {
#pragma unroll
    for (int d = 0; d < D; ++d) q[d] = -t[d * ns + c];
  }
};

// number of candidates [c0, c0 + nc) inside the radius whose key (d^2 as
// ordered bits) is < bound (<= bound when inclusive)
template <int D, class Cand>
__device__ int count_below(const Cand& cd, const float (&q)[D], int c0, int nc, float r2,
                           unsigned bound, bool inclusive) {
  const int lane = threadIdx.x & 31;
  int n = 0;
  for (int base = 0; base < nc; base += 32) {
    const int c = base + lane;
    bool ok = false;
    if (c < nc) {
      const float s = cd.d2(q, c0 + c);
      const unsigned key = __float_as_uint(s);
      ok = s < r2 && (inclusive ? key <= bound : key < bound);
    }
    n += __popc(__ballot_sync(kFull, ok));
  }
  return n;
}

// The edges of one hit with more than k_max candidates inside the radius,
// written by its warp: the k_max smallest keys (d^2 as ordered bits), ties
// broken by candidate position, in ascending candidate order. T is the
// k_max-th smallest key (bisection over the key bits); keys < T are kept,
// then the first keys == T. Candidates are [c0, c0 + nc), event-local;
// positions are written as pos0 + local index.
template <int D, class Cand>
__device__ void fill_capped(const Ws& w, const Cand& cd, const float (&qe)[D], int c0, int nc,
                            float r2, int k_max, int64_t out0, int src_pos, int pos0) {
  const int lane = threadIdx.x & 31;
  unsigned lo = 0, hi = __float_as_uint(r2);
  for (int it = 0; it < 40 && lo < hi; ++it) {
    const unsigned mid = lo + (hi - lo) / 2;
    if (count_below<D>(cd, qe, c0, nc, r2, mid, true) >= k_max)
      hi = mid;
    else
      lo = mid + 1;
  }
  const unsigned T = lo;
  const int need_eq = k_max - count_below<D>(cd, qe, c0, nc, r2, T, false);
  int written = 0, eq_seen = 0;
  for (int base = 0; base < nc; base += 32) {
    const int c = base + lane;
    bool ok = false, eq = false;
    float s = 0.0f;
    if (c < nc) {
      s = cd.d2(qe, c0 + c);
      if (s < r2) {
        const unsigned key = __float_as_uint(s);
        eq = key == T;
        ok = key < T;
      }
    }
    const unsigned eqm = __ballot_sync(kFull, eq);
    const int eq_rank = eq_seen + __popc(eqm & ((1u << lane) - 1u));
    if (eq && eq_rank < need_eq) ok = true;
    eq_seen += __popc(eqm);
    const unsigned m = __ballot_sync(kFull, ok);
    if (ok) {
      const int64_t e = out0 + written + __popc(m & ((1u << lane) - 1u));
      if (e < w.e_cap) {
        w.col[e] = pos0 + c0 + c;
        w.src[e] = src_pos;
        w.d2[e] = s;
      }
    }
    written += __popc(m);
  }
}

// The k_max edges of a hit over k_max as its mask (the same selection as
// fill_capped), rewritten by its warp: mrow[k] bit b is candidate
// cA + 32 k + b, candidates [c0, c1).
template <int D, class Cand>
__device__ void select_capped(const Cand& cd, const float (&qe)[D], int c0, int c1, int cA,
                              float r2, int k_max, uint32_t* mrow) {
  const int lane = threadIdx.x & 31;
  const int nc = c1 - c0;
  unsigned lo = 0, hi = __float_as_uint(r2);
  for (int it = 0; it < 40 && lo < hi; ++it) {
    const unsigned mid = lo + (hi - lo) / 2;
    if (count_below<D>(cd, qe, c0, nc, r2, mid, true) >= k_max)
      hi = mid;
    else
      lo = mid + 1;
  }
  const unsigned T = lo;
  const int need_eq = k_max - count_below<D>(cd, qe, c0, nc, r2, T, false);
  int eq_seen = 0;
  for (int k = 0; cA + 32 * k < c1; ++k) {
    const int c = cA + 32 * k + lane;
    bool keep = false, eq = false;
    if (c >= c0 && c < c1) {
      const float s = cd.d2(qe, c);
      if (s < r2) {
        const unsigned key = __float_as_uint(s);
        eq = key == T;
        keep = key < T;
      }
    }
    const unsigned eqm = __ballot_sync(kFull, eq);
    if (eq && eq_seen + __popc(eqm & ((1u << lane) - 1u)) < need_eq) keep = true;
    eq_seen += __popc(eqm);
    const unsigned m = __ballot_sync(kFull, keep);
    if (lane == 0) mrow[k] = m;
  }
}

// ---------------------------------------------------------------------------
// rough graph and in-edge index, one block per event
// ---------------------------------------------------------------------------
// Rough graph of Sec. "Hit Embedding and Rough Graph Construction": hit i on
// plane p joins hit j on plane p+1 or p+2 when d^2(i, j) = |e_i - e_j|^2 <
// d^2_max, keeping at most k_max per i (the k_max smallest by (d^2, sorted
// position)); the edges of a hit are stored in ascending target order, the
// hits in sorted order (CSR). Then the in-edge index: each hit's in-edges in
// ascending edge id, so that message sums run in a fixed order.
//
// Events go to blocks in index order by a ticket (counters[C_GRAPH_TICKET]),
// and each event takes its global edge offset (the edges of all earlier
// events) from a look-back over the totals its predecessors publish: an event
// publishes its own edge count as soon as its degrees are known and its
// inclusive prefix after its look-back, so a block only waits for blocks that
// took their tickets before it and are therefore running. Per event:
//   1. degrees: one thread per query hit, the 32 lanes of a warp on 32 hits
//      of one plane, so that they read the same candidate rows (broadcast);
//      the event's embeddings are staged in shared memory when they fit, and
//      then each hit's in-radius candidates are kept as a bit mask (a hit
//      over k_max keeps its k_max selected ones);
//   2. CSR offsets: block scan of min(deg, k_max), look-back, row pointers;
//   3. fill: one thread per query hit walking its mask bits in ascending
//      order (or, without masks, its candidates; a hit over k_max is then
//      filled by its warp, fill_capped);
//   4. in-edge index: in-degrees by shared-memory atomics, a block scan,
//      placement by cursors, then each target's list put in ascending edge
//      id.
constexpr int kGraphThreads = 512;
constexpr int kGraphWarps = kGraphThreads / 32;
constexpr int kGraphBlocksPerSm = 2;            // 16 warps each: 54-62 registers per thread
constexpr int kGraphSmemBytes = 110 * 1024;  // an event of up to about 4600 hits staged
constexpr int kGraphSmemInts = kGraphSmemBytes / 4;
constexpr unsigned long long kDescAgg = 1ull << 62;  // the event's own edge count
constexpr unsigned long long kDescInc = 2ull << 62;  // edges up to and including the event
constexpr unsigned long long kDescVal = (1ull << 62) - 1;
constexpr int kLookbackSpins = 1 << 22;  // x >= 100 ns sleeps: a bound of about half a second

// The look-back walks back over windows of 32 predecessors until one has
// published its inclusive prefix, summing the counts of the others. A wait
// that runs out sets ST_TIMEOUT and returns what was summed (the event then
// publishes no inclusive prefix; later events sum its count instead).

// (lane 0) publishes the event's edge count: event 0's is its inclusive prefix
__device__ __forceinline__ void graph_publish(unsigned long long* desc, int ev, long long agg) {
  atomicExch(desc + ev, (ev == 0 ? +kDescInc : +kDescAgg) | static_cast<unsigned long long>(agg));
}

// Warp 0, after graph_publish: the edges of all earlier events, then the
// event's inclusive prefix published.
__device__ long long graph_wait(unsigned long long* desc, int ev, long long agg,
                                int32_t* counters) {
  const int lane = threadIdx.x & 31;
  long long excl = 0;
  int spins = 0;
  for (int top = ev - 1; top >= 0; top -= 32) {
    const int i = top - lane;
    unsigned long long d = i >= 0 ? *reinterpret_cast<volatile unsigned long long*>(desc + i)
                                  : +kDescInc;  // before event 0: an inclusive prefix of 0
    while (__any_sync(kFull, (d >> 62) == 0)) {
      if (++spins > kLookbackSpins) {
        if (lane == 0) set_status(counters, ST_TIMEOUT);
        return excl;
      }
      __nanosleep(100);
      if ((d >> 62) == 0) d = *reinterpret_cast<volatile unsigned long long*>(desc + i);
    }
    const unsigned inc = __ballot_sync(kFull, (d >> 62) == 2);
    const int stop = inc ? __ffs(inc) - 1 : 31;  // the nearest inclusive prefix
    long long v = lane <= stop ? static_cast<long long>(d & kDescVal) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    excl += v;
    if (inc) break;
  }
  if (lane == 0 && ev > 0)
    atomicExch(desc + ev, kDescInc | static_cast<unsigned long long>(excl + agg));
  return excl;
}

// warp 0: publish, then wait
__device__ __forceinline__ long long graph_lookback(unsigned long long* desc, int ev, long long agg,
                                                    int32_t* counters) {
  if ((threadIdx.x & 31) == 0) graph_publish(desc, ev, agg);
  __syncwarp();
  return graph_wait(desc, ev, agg, counters);
}

// exclusive scan of min(in[i], clamp) over i < n into out (both may be
// shared or global memory); every thread gets the total
__device__ int block_scan(const int32_t* in, int32_t* out, int n, int clamp, int* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kGraphThreads - 1) / kGraphThreads;
  const int a = min(n, tid * per), z = min(n, a + per);
  int sum = 0;
  for (int i = a; i < z; ++i) sum += min(in[i], clamp);
  int x = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int k = 0; k < kGraphWarps; ++k) {
    const int t = wsum[k];
    if (k < warp) before += t;
    total += t;
  }
  int run = before + x - sum;
  for (int i = a; i < z; ++i) {
    const int c = min(in[i], clamp);
    out[i] = run;
    run += c;
  }
  __syncthreads();  // out complete, wsum free
  return total;
}

__device__ __forceinline__ int clamp31(long long v) {
  return int(v > 0x7fffffffLL ? 0x7fffffffLL : v);
}

// The query hits of an event are processed in items of up to 32 hits of one
// plane (a lane per hit), so that the lanes of a warp read the same
// candidate rows; item t is on plane p with chunk_s[p] <= t < chunk_s[p + 1].
struct GraphItem {
  int q0, q1, c0, c1;  // its hits [q0, q1) and their candidates [c0, c1), event-local
};

__device__ __forceinline__ GraphItem graph_item(const int* po_s, const int* chunk_s, int P, int t) {
  int p = 0;
  while (chunk_s[p + 1] <= t) ++p;
  return GraphItem{po_s[p] + (t - chunk_s[p]) * 32, po_s[p + 1], po_s[p + 1], po_s[min(p + 3, P)]};
}

// 1. degrees (uncapped) of the event's query hits. With PAIR (the staged,
// transposed rows) two candidates per step from an even start cA = c0 & ~1,
// and, when mw > 0, the in-radius candidates of hit q as bit masks:
// mask[q * mw + k] bit b is candidate cA + 32 k + b.
template <int D, bool PAIR, class Cand>
__device__ void graph_degrees(const Cand& cd, const int* po_s, const int* chunk_s, int P,
                              int n_items, float r2, int32_t* deg, uint32_t* mask, int mw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < n_items; t += kGraphWarps) {
    const GraphItem it = graph_item(po_s, chunk_s, P, t);
    const int q = it.q0 + lane;
    const bool valid = q < it.q1;
    float qe[D];
    cd.row(valid ? q : it.q0, qe);
    int cnt = 0;
    if constexpr (PAIR) {
      const int cA = it.c0 & ~1;
      for (int wb = cA; wb < it.c1; wb += 32) {
        const int we = min(it.c1, wb + 32);
        unsigned m = 0;
#pragma unroll 4
        for (int c = wb; c < we; c += 2) {
          const float2 s = cd.d2_pair(qe, c);
          m |= ((s.x < r2 ? 1u : 0u) | (s.y < r2 ? 2u : 0u)) << (c - wb);
        }
        if (wb == cA && it.c0 != cA) m &= ~1u;       // c0 - 1 is not a candidate
        if (we - wb < 32) m &= (1u << (we - wb)) - 1u;  // nor c1 (odd end)
        cnt += __popc(m);
        if (mw > 0 && valid) mask[q * mw + (wb - cA) / 32] = m;
      }
    } else {
      for (int c = it.c0; c < it.c1; ++c) cnt += cd.d2(qe, c) < r2;
    }
    if (valid) deg[q] = cnt;
  }
}

// 3. fill from the candidate masks (which hold exactly each hit's edges,
// capped hits reduced to their selection): one lane per query hit walks the
// set bits of its mask in ascending order, recomputes d^2 there from the
// staged rows and writes its edges at base + off[q].
template <int D>
__device__ void graph_fill_masks(const Ws& w, const CandNegT<D>& cd, const int* po_s,
                                 const int* chunk_s, int P, int n_items, const int32_t* off,
                                 const uint32_t* mask, int mw, long long base, int v0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < n_items; t += kGraphWarps) {
    const GraphItem it = graph_item(po_s, chunk_s, P, t);
    const int q = it.q0 + lane;
    if (q >= it.q1) continue;
    float qe[D];
    cd.row(q, qe);
    int64_t e = base + off[q];
    const int cA = it.c0 & ~1;
    const int nw = (it.c1 - cA + 31) / 32;
    for (int k = 0; k < nw; ++k) {
      unsigned m = mask[q * mw + k];
      while (m) {
        const int c = cA + 32 * k + __ffs(m) - 1;
        m &= m - 1;
        if (e < w.e_cap) {
          w.col[e] = v0 + c;
          w.src[e] = v0 + q;
          w.d2[e] = cd.d2(qe, c);
        }
        ++e;
      }
    }
  }
}

// 3. fill without masks: one lane per query hit tests its candidates again in
// ascending order and writes its edges at base + off[q]; a hit over k_max is
// filled by its warp (fill_capped).
template <int D, class Cand>
__device__ void graph_fill(const Ws& w, const Cand& cd, const int* po_s, const int* chunk_s, int P,
                           int n_items, float r2, int k_max, const int32_t* deg,
                           const int32_t* off, long long base, int v0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < n_items; t += kGraphWarps) {
    const GraphItem it = graph_item(po_s, chunk_s, P, t);
    const int q = it.q0 + lane;
    const bool valid = q < it.q1;
    const int cnt = valid ? deg[q] : 0;
    if (valid && cnt > 0 && cnt <= k_max) {
      float qe[D];
      cd.row(q, qe);
      int64_t e = base + off[q];
      for (int c = it.c0; c < it.c1; ++c) {
        const float s = cd.d2(qe, c);
        if (s < r2) {
          if (e < w.e_cap) {
            w.col[e] = v0 + c;
            w.src[e] = v0 + q;
            w.d2[e] = s;
          }
          ++e;
        }
      }
    }
    unsigned capped = __ballot_sync(kFull, cnt > k_max);
    while (capped) {
      const int qq = it.q0 + __ffs(capped) - 1;
      capped &= capped - 1;
      float qe[D];
      cd.row(qq, qe);
      fill_capped<D>(w, cd, qe, it.c0, it.c1 - it.c0, r2, k_max, base + off[qq], v0 + qq, v0);
    }
  }
}

// In-edge index of the event's stored edges [e0, e1) (read back from col):
// in-degrees by shared-memory atomics, a block scan, placement by cursors,
// then each target's list in ascending edge id. When the counts, list starts,
// lists and list targets all fit in shared memory, each list is ranked into
// in_edge (an entry's place is the number of smaller entries in its list);
// else the lists are placed in the event's slice of in_edge and sorted there
// (counts in in_cnt for events of more hits than fit).
__device__ void csc_general(const Ws& w, int n, int v0, int v1, int e0, int e1, int32_t* sm_i,
                            int* wsum) {
  const int tid = threadIdx.x;
  const int ne = e1 - e0;
  const bool full = 2 * int64_t(n) + 2 * int64_t(ne) <= kGraphSmemInts;
  const bool c_smem = n <= kGraphSmemInts;
  int32_t* C = c_smem ? sm_i : w.in_cnt + v0;
  int32_t* St = sm_i + n;               // (full only) list starts, event-local
  int32_t* L = full ? sm_i + 2 * n : w.in_edge + e0;
  int32_t* Tg = sm_i + 2 * n + ne;      // (full only) target of each list entry
  for (int i = tid; i < n; i += kGraphThreads) C[i] = 0;
  __syncthreads();
  for (int e = e0 + tid; e < e1; e += kGraphThreads) atomicAdd(&C[w.col[e] - v0], 1);
  __syncthreads();
  if (full) {
    block_scan(C, St, n, 0x7fffffff, wsum);
    for (int i = tid; i < n; i += kGraphThreads) {
      C[i] = St[i];  // cursor
      w.in_ptr[v0 + i] = e0 + St[i];
    }
  } else {
    // in place: C becomes the cursors, in_ptr the starts
    const int lane = tid & 31, warp = tid >> 5;
    const int per = (n + kGraphThreads - 1) / kGraphThreads;
    const int a = min(n, tid * per), z = min(n, a + per);
    int sum = 0;
    for (int i = a; i < z; ++i) sum += C[i];
    int x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(kFull, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < warp; ++k) before += wsum[k];
    int run = before + x - sum;
    for (int i = a; i < z; ++i) {
      const int c = C[i];
      C[i] = run;
      w.in_ptr[v0 + i] = e0 + run;
      run += c;
    }
  }
  if (tid == 0) w.in_ptr[v1] = e1;  // the next event writes the same value
  __syncthreads();
  for (int e = e0 + tid; e < e1; e += kGraphThreads) {
    const int t = w.col[e] - v0;
    const int k = atomicAdd(&C[t], 1);
    L[k] = e;
    if (full) Tg[k] = t;
  }
  __syncthreads();
  // C[i] is now the end of target i's list (event-local position)
  if (full) {
    for (int k = tid; k < ne; k += kGraphThreads) {
      const int e = L[k], t = Tg[k];
      const int lo = St[t], hi = C[t];
      int rank = 0;
      for (int m = lo; m < hi; ++m) rank += L[m] < e;
      w.in_edge[e0 + lo + rank] = e;
    }
  } else {
    for (int i = tid; i < n; i += kGraphThreads) {
      const int lo = w.in_ptr[v0 + i] - e0, hi = C[i];
      for (int j = lo + 1; j < hi; ++j) {
        const int key = L[j];
        int k = j - 1;
        while (k >= lo && L[k] > key) {
          L[k + 1] = L[k];
          --k;
        }
        L[k + 1] = key;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kGraphThreads, kGraphBlocksPerSm) k_graph_event(Batch b, Ws w, GraphParams g) {
  extern __shared__ __align__(16) float sm_graph[];
  __shared__ int po_s[kMaxPlanes + 1];     // event-local plane offsets
  __shared__ int chunk_s[kMaxPlanes + 1];  // 32-hit chunks of the query planes before p
  __shared__ int wsum[kGraphWarps];
  __shared__ int ticket_s, mw_s;
  __shared__ long long base_s;
  if (input_bad(w)) return;
  const int P = g.n_planes;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float r2 = g.radius2;
  const int k_max = g.k_max;
  int32_t* sm_i = reinterpret_cast<int32_t*>(sm_graph);
  for (;;) {
    if (tid == 0) ticket_s = atomicAdd(&w.counters[C_GRAPH_TICKET], 1);
    __syncthreads();
    const int ev = ticket_s;
    if (ev >= b.n_events) return;
    const int v0 = int(w.ev_off[ev]), v1 = int(w.ev_off[ev + 1]);
    const int n = v1 - v0;
    const int32_t* po = w.plane_off + size_t(ev) * (P + 1);
    for (int i = tid; i <= P; i += kGraphThreads) po_s[i] = po[i] - v0;
    __syncthreads();
    if (tid == 0) {
      int run = 0, words = 0;
      for (int p = 0; p + 1 < P; ++p) {
        chunk_s[p] = run;
        run += (po_s[p + 1] - po_s[p] + 31) / 32;
        if (po_s[p + 1] > po_s[p])
          words = max(words, (po_s[min(p + 3, P)] - (po_s[p + 1] & ~1) + 31) / 32);
      }
      chunk_s[P > 1 ? P - 1 : 0] = run;
      mw_s = words;
    }
    __syncthreads();  // chunk_s and mw_s (which sets the layout below) visible
    // rows of this event, event-local index, in shared memory when they fit:
    //   [off n][mask n*mw][deg n][t D*ns]
    // off: CSR offsets; mask: in-radius candidates per hit (when they fit too);
    // t: the embeddings transposed and negated, t[d * ns + i] = -e_i[d]
    // (8-byte aligned, for the candidate pairs). Else global scratch.
    const int ns = (n + 2) & ~1;  // even, with a pad column read by the last pair
    const int64_t rows_ints = int64_t(D) * ns + 3;
    const bool staged = rows_ints + 2 * int64_t(n) <= kGraphSmemInts;
    const int mw = staged && rows_ints + int64_t(n) * (2 + mw_s) <= kGraphSmemInts ? mw_s : 0;
    int32_t* off = staged ? sm_i : w.in_cnt + v0;
    uint32_t* mask = reinterpret_cast<uint32_t*>(sm_i + n);
    int32_t* deg = staged ? sm_i + n * (1 + mw) : w.deg + v0;
    float* tT = sm_graph + ((n * (2 + mw) + 3) & ~3);
    if (staged) {
      for (int k = tid; k < n * D; k += kGraphThreads) {
        const int i = k / D, d = k - i * D;
        tT[d * ns + i] = -w.emb[size_t(v0) * D + k];
      }
      for (int k = tid; k < D * (ns - n); k += kGraphThreads) {
        const int d = k / (ns - n);
        tT[d * ns + n + (k - d * (ns - n))] = 0.0f;
      }
    }
    __syncthreads();
    const int n_items = chunk_s[P > 1 ? P - 1 : 0];
    const CandNegT<D> cst{tT, ns};
    const CandRows<D> cgl{w.emb + size_t(v0) * D};

    // 1. degrees (uncapped); with masks, a hit over k_max keeps only its
    //    k_max selected candidates in its mask (the masks then hold exactly
    //    the edges)
    if (staged)
      graph_degrees<D, true>(cst, po_s, chunk_s, P, n_items, r2, deg, mask, mw);
    else
      graph_degrees<D, false>(cgl, po_s, chunk_s, P, n_items, r2, deg, nullptr, 0);
    if (P >= 1)
      for (int q = po_s[P - 1] + tid; q < n; q += kGraphThreads) deg[q] = 0;  // no candidates
    __syncthreads();
    if (mw > 0) {
      for (int t = warp; t < n_items; t += kGraphWarps) {
        const GraphItem it = graph_item(po_s, chunk_s, P, t);
        unsigned capped = __ballot_sync(kFull, it.q0 + lane < it.q1 && deg[it.q0 + lane] > k_max);
        while (capped) {
          const int qq = it.q0 + __ffs(capped) - 1;
          capped &= capped - 1;
          float qe[D];
          cst.row(qq, qe);
          select_capped<D>(cst, qe, it.c0, it.c1, it.c0 & ~1, r2, k_max, mask + qq * mw);
        }
      }
      __syncthreads();
    }

    // 2. offsets: event-local exclusive scan of min(deg, k_max), then the
    //    event's base by the look-back
    const int total = block_scan(deg, off, n, k_max, wsum);
    if (warp == 0) {
      const long long ex = graph_lookback(w.graph_desc, ev, total, w.counters);
      if (lane == 0) base_s = ex;
    }
    __syncthreads();
    const long long base = base_s;
    for (int i = tid; i < n; i += kGraphThreads) w.row_ptr[v0 + i] = clamp31(base + off[i]);
    if (ev == b.n_events - 1 && tid == 0) {
      const long long all = base + total;
      w.row_ptr[v1] = clamp31(all);
      w.counters[C_EDGES] = clamp31(all);
      if (all > w.e_cap || all > 0x7fffffffLL) set_status(w.counters, ST_CAPACITY);
    }

    // 3. fill
    if (mw > 0)
      graph_fill_masks<D>(w, cst, po_s, chunk_s, P, n_items, off, mask, mw, base, v0);
    else if (staged)
      graph_fill<D>(w, cst, po_s, chunk_s, P, n_items, r2, k_max, deg, off, base, v0);
    else
      graph_fill<D>(w, cgl, po_s, chunk_s, P, n_items, r2, k_max, deg, off, base, v0);
    __syncthreads();  // edges written; shared memory free

    // 4. in-edge index of the event's edges [e0, e1)
    const int e0 = int(base < w.e_cap ? base : w.e_cap);
    const int e1 = int(base + total < w.e_cap ? base + total : w.e_cap);
    csc_general(w, n, v0, v1, e0, e1, sm_i, wsum);
    __syncthreads();  // shared memory and ticket_s are reused by the next event
  }
}

template <int D>
void graph_d(const Batch& b, const Ws& w, const GraphParams& g, int grid, cudaStream_t s) {
  // set once per instantiation (thread-safe initialisation of a local static)
  static const bool attr = [] {
    cudaFuncSetAttribute(k_graph_event<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kGraphSmemBytes);
    return true;
  }();
  (void)attr;
  k_graph_event<D><<<grid, kGraphThreads, kGraphSmemBytes, s>>>(b, w, g);
}

// ---------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_s, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_s[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int t = lane < nw ? warp_s[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_s[lane] = t;
  }
  __syncthreads();
  total = warp_s[(blockDim.x >> 5) - 1];
  const int r = x - v + (warp > 0 ? warp_s[warp - 1] : 0);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* in, int n,
                                                              int clamp_max, int32_t* blocks,
                                                              int32_t* counters, int total_slot,
                                                              int64_t cap) {
  __shared__ int warp_s[32];
  __shared__ int is_last;
  if ((*(volatile int32_t*)&counters[C_STATUS]) & ST_INPUT) return;
  const int base = blockIdx.x * kScanChunk;
  int v = 0;
  for (int k = 0; k < kScanPer; ++k) {
    const int i = base + k * kScanThreads + threadIdx.x;
    if (i < n) v += min(in[i], clamp_max);
  }
  int total;
  block_exclusive_scan(v, warp_s, total);
  if (threadIdx.x == 0) {
    blocks[blockIdx.x] = total;
    __threadfence();
    const int t = atomicAdd(&counters[C_TICKET], 1);
    is_last = t == int(gridDim.x) - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the last block scans the block sums
  long long run = 0;
  for (int c = 0; c < int(gridDim.x); c += kScanThreads) {
    const int i = c + threadIdx.x;
    const int x = i < int(gridDim.x) ? ((volatile int32_t*)blocks)[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(x, warp_s, tot);
    if (i < int(gridDim.x)) blocks[i] = int(run + ex);
    run += tot;
  }
  if (threadIdx.x == 0) {
    if (run > cap || run > 0x7fffffffLL) set_status(counters, ST_CAPACITY);
    counters[total_slot] = int(run > 0x7fffffffLL ? 0x7fffffffLL : run);
    counters[C_TICKET] = 0;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t* in, int32_t* out,
                                                             int n, int clamp_max,
                                                             const int32_t* blocks,
                                                             const int32_t* counters,
                                                             int total_slot) {
  __shared__ int warp_s[32];
  if ((*(volatile const int32_t*)&counters[C_STATUS]) & ST_INPUT) return;
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int v[kScanPer];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int i = base + k;
    v[k] = i < n ? min(in[i], clamp_max) : 0;
    sum += v[k];
  }
  int total;
  int run = block_exclusive_scan(sum, warp_s, total) + blocks[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = counters[total_slot];
}

int num_sms() {
  // queried once per process (thread-safe initialisation of a local static)
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

}  // namespace

void launch_sort(const Batch& b, const Ws& w, int n_planes, cudaStream_t s) {
  if (b.n_events <= 0) return;
  k_sort<<<b.n_events, kSortThreads, 0, s>>>(b, w, n_planes);
}

void launch_scan(const int32_t* in, int32_t* out, int n, int clamp_max, int32_t* counters,
                 int total_slot, int64_t cap, int32_t* blocks, cudaStream_t s) {
  const int nb = div_up(n > 0 ? n : 1, kScanChunk);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, clamp_max, blocks, counters, total_slot, cap);
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, clamp_max, blocks, counters, total_slot);
}

void launch_graph(const Batch& b, const Ws& w, const GraphParams& g, int D, cudaStream_t s) {
  if (b.n_events <= 0) return;
  cudaMemsetAsync(w.graph_desc, 0, sizeof(unsigned long long) * b.n_events, s);
  const int grid = std::min(b.n_events, num_sms() * kGraphBlocksPerSm);
  switch (D) {
    case 1: graph_d<1>(b, w, g, grid, s); break;
    case 2: graph_d<2>(b, w, g, grid, s); break;
    case 3: graph_d<3>(b, w, g, grid, s); break;
    case 4: graph_d<4>(b, w, g, grid, s); break;
    case 5: graph_d<5>(b, w, g, grid, s); break;
    case 6: graph_d<6>(b, w, g, grid, s); break;
    case 7: graph_d<7>(b, w, g, grid, s); break;
    case 8: graph_d<8>(b, w, g, grid, s); break;
    case 16: graph_d<16>(b, w, g, grid, s); break;
    default: break;
  }
}

int device_sms() { return num_sms(); }

}  // namespace gnntrk
