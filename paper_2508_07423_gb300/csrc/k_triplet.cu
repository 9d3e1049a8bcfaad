// Triplet stage: triplet building, the two triplet classifiers and track
// building from the purified edge graph (Secs. "Triplet Building" and "Track
// Building").
//
// A triplet is a pair of kept edges sharing one hit C: an articulation
// (A -> C, C -> B), a left elbow (C -> A, C -> B) or a right elbow (A -> C,
// B -> C). An elbow's edges are ordered by the sorted position of their far
// hit, which orders them by (plane, input index). Articulations and elbows go
// to two lists (they take different classifiers); within a list the triplets
// of hit C are contiguous and C ascends, so each event owns one range of each.
//
// The triplet classifiers run on the tensor cores (k_tc, triplet mode) or, on
// the FP32 path, on the warp-tile FP32 kernels (k_gnn_f32, triplet mode).
//
// Track building, per event (one block):
//   1. kept elbows join their edges into groups (union-find over edge ids);
//   2. kept articulations link groups; a link g1 -> g2 is shared when g1 links
//      to two different groups or g2 is linked from two different groups
//      (detected with a first-partner compare-and-swap per group); components
//      of the groups over the links that are not shared (second union-find);
//   3. tracks: each component touching no shared link, and each distinct
//      component pair (X, Y) joined by a shared link (the shared component is
//      duplicated into each branch);
//   4. a track's hits are the endpoints of its edges.
// Every union hooks the larger root under the smaller one, so each root is the
// smallest edge id of its set and the result does not depend on the order of
// the unions. Track hits are written in sorted-position order (plane, then
// input index) as event-local input indices; an event's tracks are its plain
// components by ascending root, then its component pairs in ascending order.
#include <algorithm>

#include "../../include/gnntrk.h"
#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kTbThreads = 256;
constexpr int kUnionRetries = 1 << 20;
constexpr int kPairSort = 1024;  // pairs sorted in shared memory (else in place, O(n^2))

__device__ __forceinline__ int tb_find(volatile int32_t* P, int x) {
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

__device__ __forceinline__ void tb_union(volatile int32_t* P, int a, int b, int32_t* counters) {
  int ra = tb_find(P, a), rb = tb_find(P, b);
  for (int it = 0; it < kUnionRetries; ++it) {
    if (ra == rb) return;
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    const int old = atomicCAS((int32_t*)&P[rb], rb, ra);
    if (old == rb) return;
    rb = tb_find(P, old);
    ra = tb_find(P, ra);
  }
  set_status(counters, ST_TIMEOUT);
}

// Inclusive scan of one int per thread over a kTbThreads block (warp shuffles,
// then the warp totals); `sw` holds kTbThreads / 32 ints of shared scratch.
// Returns the thread's inclusive sum, the block total in `total`. Every thread
// must call it (two barriers inside).
__device__ __forceinline__ int block_scan(int v, int* sw, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  if (lane == 31) sw[wid] = v;
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < kTbThreads / 32; ++k) {
    const int t = sw[k];
    off += k < wid ? t : 0;
    tot += t;
  }
  __syncthreads();
  total = tot;
  return v + off;
}

// ---- 1. triplet counts per hit ----------------------------------------------
__global__ void k_trip_count(Batch b, Ws w) {
  if (*(volatile int32_t*)&w.counters[C_STATUS] & (ST_INPUT | ST_CAPACITY)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b.n_hits; c += gridDim.x * blockDim.x) {
    int kout = 0, kin = 0;
    for (int e = w.row_ptr[c]; e < w.row_ptr[c + 1]; ++e) kout += w.keep[e];
    for (int j = w.in_ptr[c]; j < w.in_ptr[c + 1]; ++j) kin += w.keep[w.in_edge[j]];
    w.trip_cnt_a[c] = kin * kout;
    w.trip_cnt_e[c] = kout * (kout - 1) / 2 + kin * (kin - 1) / 2;
  }
}

// ---- 2. triplet lists ----------------------------------------------------------
__global__ void k_trip_fill(Batch b, Ws w) {
  if (*(volatile int32_t*)&w.counters[C_STATUS] & (ST_INPUT | ST_CAPACITY)) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b.n_hits; c += gridDim.x * blockDim.x) {
    const int o0 = w.row_ptr[c], o1 = w.row_ptr[c + 1];
    const int i0 = w.in_ptr[c], i1 = w.in_ptr[c + 1];
    int ta = w.trip_off_a[c], te = w.trip_off_e[c];
    // articulations: in-edges in edge-id order (their sources ascend), then
    // out-edges in list order
    for (int j = i0; j < i1; ++j) {
      const int a = w.in_edge[j];
      if (!w.keep[a]) continue;
      for (int e = o0; e < o1; ++e)
        if (w.keep[e]) {
          w.trip_a1[ta] = a;
          w.trip_a2[ta] = e;
          ++ta;
        }
    }
    // left elbows: pairs of kept out-edges, the nearer far hit first
    for (int e = o0; e < o1; ++e) {
      if (!w.keep[e]) continue;
      for (int f = o0; f < o1; ++f)
        if (w.keep[f] && w.col[f] > w.col[e]) {
          w.trip_e1[te] = e;
          w.trip_e2[te] = f;
          w.trip_et[te] = 1;
          ++te;
        }
    }
    // right elbows: pairs of kept in-edges (sources ascend with the edge id)
    for (int j = i0; j < i1; ++j) {
      const int a = w.in_edge[j];
      if (!w.keep[a]) continue;
      for (int k = j + 1; k < i1; ++k) {
        const int f = w.in_edge[k];
        if (!w.keep[f]) continue;
        w.trip_e1[te] = a;
        w.trip_e2[te] = f;
        w.trip_et[te] = 2;
        ++te;
      }
    }
  }
}

// Call f(X) once for every distinct component X among the kept edges of hit v
// (CE[e] = component of edge e, -1 if the edge is not kept). The components
// of up to 16 incident kept edges are kept in registers; beyond that the
// earlier edges are re-read.
template <class F>
__device__ __forceinline__ void for_hit_components(const Ws& w, const int32_t* CE, int v, F&& f) {
  constexpr int kReg = 16;
  const int o0 = w.row_ptr[v], o1 = w.row_ptr[v + 1];
  const int i0 = w.in_ptr[v], i1 = w.in_ptr[v + 1];
  const int dout = o1 - o0, deg = dout + (i1 - i0);
  auto edge = [&](int q) { return q < dout ? o0 + q : w.in_edge[i0 + q - dout]; };
  int cs[kReg];
  int nc = 0;
  for (int q = 0; q < deg; ++q) {
    const int X = CE[edge(q)];
    if (X < 0) continue;
    bool seen = false;
    if (q <= kReg) {
      // every earlier distinct component is in cs (fewer than kReg edges before q)
#pragma unroll
      for (int r = 0; r < kReg; ++r) seen |= r < nc && cs[r] == X;
    } else {
      for (int r = 0; r < q && !seen; ++r) seen = CE[edge(r)] == X;
    }
    if (seen) continue;
    if (nc < kReg) cs[nc++] = X;
    f(X);
  }
}

// ---- 4. track building, per event ------------------------------------------------
// Phase 1: groups, links, components, component hit lists, pair list; counts
// of tracks and track hits per event.
__global__ void __launch_bounds__(kTbThreads) k_tb_event(Batch b, Ws w) {
  __shared__ int s_np, s_nuniq, s_tracks, s_hits;
  __shared__ unsigned long long s_last;
  __shared__ unsigned long long s_pairs[kPairSort];
  __shared__ int s_w[kTbThreads / 32];
  if (*(volatile int32_t*)&w.counters[C_STATUS] & (ST_INPUT | ST_CAPACITY)) return;
  const int tid = threadIdx.x;
  for (int ev = blockIdx.x; ev < b.n_events; ev += gridDim.x) {
    const int h0 = int(w.ev_off[ev]), h1 = int(w.ev_off[ev + 1]);
    const int E0 = w.row_ptr[h0], E1 = w.row_ptr[h1];
    const int A0 = w.trip_off_a[h0], A1 = w.trip_off_a[h1];
    const int L0 = w.trip_off_e[h0], L1 = w.trip_off_e[h1];
    int32_t* P = w.tb_par;
    int32_t* P2 = w.tb_par2;
    if (tid == 0) {
      s_np = 0;
      s_tracks = 0;
      s_hits = 0;
    }
    for (int e = E0 + tid; e < E1; e += kTbThreads) {
      P[e] = e;
      P2[e] = e;
      w.tb_out[e] = -1;
      w.tb_in[e] = -1;
      w.tb_flag[e] = 0;
      w.tb_cnt[e] = 0;
    }
    __syncthreads();
    // 1. kept elbows join their two edges
    for (int t = L0 + tid; t < L1; t += kTbThreads)
      if (w.trip_ekeep[t]) tb_union(P, w.trip_e1[t], w.trip_e2[t], w.counters);
    __syncthreads();
    // compress in two passes: a find's path halving may still move a pointer
    // that another thread has just set to its root, so the roots are found
    // first (into tb_cur) and stored after every find has finished
    for (int e = E0 + tid; e < E1; e += kTbThreads)
      if (w.keep[e]) w.tb_cur[e] = tb_find(P, e);
    __syncthreads();
    for (int e = E0 + tid; e < E1; e += kTbThreads)
      if (w.keep[e]) P[e] = w.tb_cur[e];
    __syncthreads();
    // 2. articulation links: first partner per group and direction; a second,
    //    different partner marks the group (bit 0 onwards, bit 1 backwards)
    for (int t = A0 + tid; t < A1; t += kTbThreads) {
      if (!w.trip_akeep[t]) continue;
      const int ga = P[w.trip_a1[t]], gb = P[w.trip_a2[t]];
      if (ga == gb) continue;
      const int o = atomicCAS(&w.tb_out[ga], -1, gb);
      if (o != -1 && o != gb) atomicOr(&w.tb_flag[ga], 1);
      const int i = atomicCAS(&w.tb_in[gb], -1, ga);
      if (i != -1 && i != ga) atomicOr(&w.tb_flag[gb], 2);
    }
    __syncthreads();
    for (int t = A0 + tid; t < A1; t += kTbThreads) {
      if (!w.trip_akeep[t]) continue;
      const int ga = P[w.trip_a1[t]], gb = P[w.trip_a2[t]];
      if (ga == gb) continue;
      if (!(w.tb_flag[ga] & 1) && !(w.tb_flag[gb] & 2)) tb_union(P2, ga, gb, w.counters);
    }
    __syncthreads();
    // component of every group root (two passes, as above)
    for (int e = E0 + tid; e < E1; e += kTbThreads)
      if (w.keep[e] && P[e] == e) w.tb_off[e] = tb_find(P2, e);
    __syncthreads();
    for (int e = E0 + tid; e < E1; e += kTbThreads)
      if (w.keep[e] && P[e] == e) P2[e] = w.tb_off[e];
    __syncthreads();
    // 3. shared links -> component pairs (X << 32 | Y), X != Y
    for (int t = A0 + tid; t < A1; t += kTbThreads) {
      if (!w.trip_akeep[t]) continue;
      const int ga = P[w.trip_a1[t]], gb = P[w.trip_a2[t]];
      if (ga == gb || (!(w.tb_flag[ga] & 1) && !(w.tb_flag[gb] & 2))) continue;
      const int X = P2[ga], Y = P2[gb];
      if (X == Y) continue;
      const int k = atomicAdd(&s_np, 1);
      w.tb_pairs[A0 + k] = (static_cast<unsigned long long>(X) << 32) | unsigned(Y);
      atomicOr(&w.tb_flag[X], 4);
      atomicOr(&w.tb_flag[Y], 4);
    }
    __syncthreads();
    const int np = s_np;
    unsigned long long* pairs = w.tb_pairs + A0;
    if (np <= kPairSort) {
      // bitonic sort in shared memory (padded with the maximum key)
      int m = 1;
      while (m < np) m <<= 1;
      for (int i = tid; i < m; i += kTbThreads) s_pairs[i] = i < np ? pairs[i] : ~0ull;
      __syncthreads();
      for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = tid; i < m; i += kTbThreads) {
            const int l = i ^ j;
            if (l > i) {
              const unsigned long long a = s_pairs[i], c = s_pairs[l];
              const bool up = (i & k) == 0;
              if ((a > c) == up) {
                s_pairs[i] = c;
                s_pairs[l] = a;
              }
            }
          }
          __syncthreads();
        }
      for (int i = tid; i < np; i += kTbThreads) pairs[i] = s_pairs[i];
      __syncthreads();
    } else if (tid == 0) {
      // rare: more shared links than the shared-memory sort holds
      for (int i = 1; i < np; ++i) {
        const unsigned long long v = pairs[i];
        int j = i - 1;
        while (j >= 0 && pairs[j] > v) {
          pairs[j + 1] = pairs[j];
          --j;
        }
        pairs[j + 1] = v;
      }
    }
    __syncthreads();
    // compact the distinct pairs to the front (block scan of first-occurrence flags)
    {
      int nu = 0;
      for (int base = 0; base < np; base += kTbThreads) {
        const int i = base + tid;
        const unsigned long long v = i < np ? pairs[i] : 0ull;
        // the previous entry as it was before this pass compacted anything:
        // inside the chunk a neighbour's value, across chunks the saved one
        const unsigned long long prev =
            tid > 0 ? (i < np ? pairs[i - 1] : 0ull) : (base > 0 ? s_last : ~v);
        const bool f = i < np && (i == 0 || v != prev);
        int tot;
        const int inc = block_scan(f ? 1 : 0, s_w, tot);
        if (tid == kTbThreads - 1 || i == np - 1) s_last = v;
        // every thread read its entries before the scan's barriers; a write
        // goes to slot nu + inc - 1 <= i
        if (f) pairs[nu + inc - 1] = v;
        nu += tot;
        __syncthreads();
      }
      if (tid == 0) s_nuniq = nu;
    }
    __syncthreads();
    // 4. hits per component: every hit with a kept edge counts once per
    //    distinct component among its kept edges. The component of every
    //    edge first (-1 if not kept; tb_in is free again), so a hit reads
    //    one value per incident edge.
    int32_t* CE = w.tb_in;
    for (int e = E0 + tid; e < E1; e += kTbThreads) CE[e] = w.keep[e] ? P2[P[e]] : -1;
    __syncthreads();
    for (int v = h0 + tid; v < h1; v += kTbThreads)
      for_hit_components(w, CE, v, [&](int X) { atomicAdd(&w.tb_cnt[X], 1); });
    __syncthreads();
    // offsets of the component hit lists (block scan over the event's edges),
    // and counts of the plain tracks
    {
      int run = 0;
      for (int base = E0; base < E1; base += kTbThreads) {
        const int e = base + tid;
        const int c = (e < E1 && w.keep[e] && P[e] == e && P2[e] == e) ? w.tb_cnt[e] : 0;
        int tot;
        const int inc = block_scan(c, s_w, tot);
        if (c > 0) {
          w.tb_off[e] = 2 * E0 + run + inc - c;
          w.tb_cur[e] = 0;
          if (!(w.tb_flag[e] & 4)) {
            atomicAdd(&s_tracks, 1);
            atomicAdd(&s_hits, c);
          }
        }
        run += tot;
      }
    }
    __syncthreads();
    // place the hits (sorted positions), then sort each list
    for (int v = h0 + tid; v < h1; v += kTbThreads)
      for_hit_components(w, CE, v, [&](int X) {
        w.tb_hits[w.tb_off[X] + atomicAdd(&w.tb_cur[X], 1)] = v;
      });
    __syncthreads();
    for (int e = E0 + tid; e < E1; e += kTbThreads) {
      if (!(w.keep[e] && P[e] == e && P2[e] == e)) continue;
      int32_t* L = w.tb_hits + w.tb_off[e];
      const int n = w.tb_cnt[e];
      for (int i = 1; i < n; ++i) {
        const int v = L[i];
        int j = i - 1;
        while (j >= 0 && L[j] > v) {
          L[j + 1] = L[j];
          --j;
        }
        L[j + 1] = v;
      }
    }
    __syncthreads();
    // pair tracks: size of the union of the two sorted lists
    for (int k = tid; k < s_nuniq; k += kTbThreads) {
      const int X = int(pairs[k] >> 32), Y = int(pairs[k] & 0xffffffffu);
      const int32_t *a = w.tb_hits + w.tb_off[X], *c = w.tb_hits + w.tb_off[Y];
      const int na = w.tb_cnt[X], nc = w.tb_cnt[Y];
      int i = 0, j = 0, u = 0;
      while (i < na || j < nc) {
        if (j >= nc || (i < na && a[i] < c[j])) ++i;
        else if (i >= na || c[j] < a[i]) ++j;
        else ++i, ++j;
        ++u;
      }
      atomicAdd(&s_tracks, 1);
      atomicAdd(&s_hits, u);
    }
    __syncthreads();
    if (tid == 0) {
      w.tb_ev_tracks[ev] = s_tracks;
      w.tb_ev_hits[ev] = s_hits;
      w.tb_ev_pairs[ev] = s_nuniq;
    }
    __syncthreads();
  }
}

// Phase 2: write the tracks at the scanned offsets (capacity-checked).
__global__ void __launch_bounds__(kTbThreads) k_tb_write(Batch b, Ws w, const int32_t* ev_tracks,
                                                          int64_t* track_off, int32_t* track_hits,
                                                          int64_t max_tracks, int64_t max_hits) {
  __shared__ int s_w[kTbThreads / 32];
  __shared__ int s_t, s_h;
  if (*(volatile int32_t*)&w.counters[C_STATUS] & (ST_INPUT | ST_CAPACITY)) return;
  const int tid = threadIdx.x;
  const int64_t total_tracks = ev_tracks[b.n_events];
  const int64_t total_hits = w.tb_ev_hit_off[b.n_events];
  if (total_tracks > max_tracks || total_hits > max_hits) {
    if (blockIdx.x == 0 && tid == 0) set_status(w.counters, ST_CAPACITY);
    return;
  }
  if (blockIdx.x == 0 && tid == 0) track_off[total_tracks] = total_hits;
  for (int ev = blockIdx.x; ev < b.n_events; ev += gridDim.x) {
    const int h0 = int(w.ev_off[ev]), h1 = int(w.ev_off[ev + 1]);
    const int E0 = w.row_ptr[h0], E1 = w.row_ptr[h1];
    const int A0 = w.trip_off_a[h0];
    const int32_t* P = w.tb_par;
    const int32_t* P2 = w.tb_par2;
    const unsigned long long* pairs = w.tb_pairs + A0;
    const int base_ev = int(w.ev_off[ev]);
    if (tid == 0) {
      s_t = ev_tracks[ev];
      s_h = w.tb_ev_hit_off[ev];
    }
    __syncthreads();
    // plain components in ascending root order: ranks by a block scan
    for (int base = E0; base < E1; base += kTbThreads) {
      const int e = base + tid;
      const bool f = e < E1 && w.keep[e] && P[e] == e && P2[e] == e && !(w.tb_flag[e] & 4);
      const int c = f ? w.tb_cnt[e] : 0;
      int last, last2;
      const int inc = block_scan(f ? 1 : 0, s_w, last);
      const int inc2 = block_scan(c, s_w, last2);
      if (f) {
        const int t = s_t + inc - 1;
        const int64_t o = s_h + inc2 - c;
        track_off[t] = o;
        const int32_t* L = w.tb_hits + w.tb_off[e];
        for (int i = 0; i < c; ++i) track_hits[o + i] = w.perm[L[i]] - base_ev;
      }
      __syncthreads();
      if (tid == 0) {
        s_t += last;
        s_h += last2;
      }
      __syncthreads();
    }
    // component pairs: sizes again (union of two sorted lists), then a scan
    const int nu = w.tb_ev_pairs[ev];
    for (int base = 0; base < nu; base += kTbThreads) {
      const int k = base + tid;
      int u = 0, X = 0, Y = 0;
      if (k < nu) {
        X = int(pairs[k] >> 32);
        Y = int(pairs[k] & 0xffffffffu);
        const int32_t *a = w.tb_hits + w.tb_off[X], *c = w.tb_hits + w.tb_off[Y];
        const int na = w.tb_cnt[X], nc = w.tb_cnt[Y];
        int i = 0, j = 0;
        while (i < na || j < nc) {
          if (j >= nc || (i < na && a[i] < c[j])) ++i;
          else if (i >= na || c[j] < a[i]) ++j;
          else ++i, ++j;
          ++u;
        }
      }
      int last;
      const int inc = block_scan(u, s_w, last);
      if (k < nu) {
        const int t = s_t + k - base;
        const int64_t o = s_h + inc - u;
        track_off[t] = o;
        const int32_t *a = w.tb_hits + w.tb_off[X], *c = w.tb_hits + w.tb_off[Y];
        const int na = w.tb_cnt[X], nc = w.tb_cnt[Y];
        int i = 0, j = 0, m = 0;
        while (i < na || j < nc) {
          int v;
          if (j >= nc || (i < na && a[i] < c[j])) v = a[i++];
          else if (i >= na || c[j] < a[i]) v = c[j++];
          else v = a[i++], ++j;
          track_hits[o + m++] = w.perm[v] - base_ev;
        }
      }
      __syncthreads();
      if (tid == 0) {
        s_t += min(kTbThreads, nu - base);
        s_h += last;
      }
      __syncthreads();
    }
  }
}

// totals: kept triplets
__global__ void k_trip_kept(const uint8_t* ka, const int32_t* na, const uint8_t* ke,
                            const int32_t* ne, int32_t* counters) {
  if (*(volatile int32_t*)&counters[C_STATUS] & (ST_INPUT | ST_CAPACITY)) return;
  const int a = *na, e = *ne;
  int k = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a + e; t += gridDim.x * blockDim.x)
    k += t < a ? ka[t] : ke[t - a];
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(&counters[C_TRIP_KEPT], k);
}

}  // namespace

void launch_triplets(const Batch& b, const Ws& w, int h, cudaStream_t s) {
  const int grid = std::max(1, std::min(div_up(b.n_hits, 256), device_sms() * 8));
  k_trip_count<<<grid, 256, 0, s>>>(b, w);
  launch_scan(w.trip_cnt_a, w.trip_off_a, b.n_hits, 1 << 30, w.counters, C_TRIP_A, w.t_cap,
              w.scan_blocks, s);
  launch_scan(w.trip_cnt_e, w.trip_off_e, b.n_hits, 1 << 30, w.counters, C_TRIP_E, w.t_cap,
              w.scan_blocks, s);
  k_trip_fill<<<grid, 256, 0, s>>>(b, w);
  (void)h;
}

void launch_triplet_kept(const Ws& w, cudaStream_t s) {
  k_trip_kept<<<device_sms() * 4, 256, 0, s>>>(w.trip_akeep, w.counters + C_TRIP_A, w.trip_ekeep,
                                               w.counters + C_TRIP_E, w.counters);
}

void launch_track_build(const Batch& b, const Ws& w, const TrackOut& out, cudaStream_t s) {
  if (b.n_events <= 0) return;
  const int grid = std::min(b.n_events, device_sms() * 8);
  k_tb_event<<<grid, kTbThreads, 0, s>>>(b, w);
  launch_scan(w.tb_ev_tracks, out.ev_tracks, b.n_events, 1 << 30, w.counters, C_TRACKS,
              int64_t(1) << 40, w.scan_blocks, s);
  launch_scan(w.tb_ev_hits, w.tb_ev_hit_off, b.n_events, 1 << 30, w.counters, C_TRACK_HITS,
              int64_t(1) << 40, w.scan_blocks, s);
  k_tb_write<<<grid, kTbThreads, 0, s>>>(b, w, out.ev_tracks, out.track_off, out.track_hits,
                                         out.max_tracks, out.max_hits);
}

}  // namespace gnntrk
