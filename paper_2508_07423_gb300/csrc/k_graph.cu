// Input staging and rough-graph construction.
//
//  k_sort      per event, a stable counting sort of the hits by plane: the
//              sorted order is (event, plane, input index), so the candidates of
//              a hit on plane p (planes p+1 and p+2) form one contiguous range.
//  k_radius    rough graph of Sec. "Hit Embedding and Rough Graph Construction":
//              hit i on plane p joins hit j on plane p+1 or p+2 when
//              d^2(i, j) = |e_i - e_j|^2 < d^2_max, keeping at most k_max per i
//              (the k_max smallest by (d^2, sorted position)). One block per
//              (event, plane p) stages the candidate embeddings in shared
//              memory; one warp per query hit tests 32 candidates at a time and
//              compacts the passing ones with a ballot. A count pass fills the
//              per-hit candidate count, a scan turns it into CSR row pointers
//              and a fill pass writes the edges in ascending target order.
//  k_scan_*    exclusive scan in two kernels (block sums, with the last block
//              scanning them; then block scans plus the block offset).
//  k_csc_*     in-edge index: edges grouped by target, ascending edge id, so
//              that message sums run in a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace gnntrk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kRadiusThreads = 256;
constexpr int kRadiusCountThreads = 64;  // count pass: one thread per query (about 65 per plane)
constexpr int kCandSmemBytes = 12 * 1024;  // staged candidates (about 2-6 KB needed); 8 blocks per SM
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
// radius search
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

// number of candidates with key < bound (strict) among those inside the radius
template <int D>
__device__ int count_below(const float (&q)[D], const float* ce, int nc, float r2,
                           unsigned bound, bool inclusive) {
  const int lane = threadIdx.x & 31;
  int n = 0;
  for (int base = 0; base < nc; base += 32) {
    const int c = base + lane;
    bool ok = false;
    if (c < nc) {
      const float s = dist2<D>(q, ce + size_t(c) * D);
      const unsigned key = __float_as_uint(s);
      ok = s < r2 && (inclusive ? key <= bound : key < bound);
    }
    n += __popc(__ballot_sync(kFull, ok));
  }
  return n;
}

template <int D, bool FILL>
__global__ void __launch_bounds__(kRadiusThreads) k_radius(Batch b, Ws w, GraphParams g) {
  extern __shared__ float cand_s[];
  if (input_bad(w)) return;
  const int P = g.n_planes;
  const int ev = blockIdx.x / (P - 1), p = blockIdx.x % (P - 1);
  const int32_t* po = w.plane_off + size_t(ev) * (P + 1);
  const int q0 = po[p], q1 = po[p + 1];
  if (q0 == q1) return;
  const int c0 = po[p + 1], c1 = po[min(p + 3, P)];
  const int nc = c1 - c0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const bool staged = size_t(nc) * D * sizeof(float) <= size_t(kCandSmemBytes);
  const float* ce = staged ? cand_s : w.emb + size_t(c0) * D;
  if (staged) {
    if constexpr (D % 4 == 0) {
      const float4* g4 = reinterpret_cast<const float4*>(w.emb + size_t(c0) * D);
      float4* s4 = reinterpret_cast<float4*>(cand_s);
      for (int k = tid; k < nc * D / 4; k += blockDim.x) s4[k] = g4[k];
    } else {
      for (int k = tid; k < nc * D; k += blockDim.x) cand_s[k] = w.emb[size_t(c0) * D + k];
    }
    __syncthreads();
  }
  const float r2 = g.radius2;
  if constexpr (!FILL) {
    // count: one thread per query, all threads stepping through the same
    // candidates (shared-memory broadcasts); the candidates inside the radius
    // go to the query's mask words for the fill pass
    for (int q = q0 + tid; q < q1; q += blockDim.x) {
      float qe[D];
#pragma unroll
      for (int d = 0; d < D; ++d) qe[d] = w.emb[size_t(q) * D + d];
      int cnt = 0;
      for (int base = 0; base < nc; base += 32) {
        const int m_end = min(32, nc - base);
        unsigned m = 0;
        for (int j = 0; j < m_end; ++j)
          if (dist2<D>(qe, ce + size_t(base + j) * D) < r2) m |= 1u << j;
        cnt += __popc(m);
        if (nc <= kMaskCands) w.rmask[size_t(q) * kMaskWords + base / 32] = m;
      }
      w.deg[q] = cnt;
    }
    return;
  }
  if (FILL && nc <= kMaskCands) {
    // one thread per query: walk the set bits of its masks (ascending
    // candidate index, the order of the warp path), recompute d^2 only there
    const int nwords = (nc + 31) / 32;
    for (int q = q0 + tid; q < q1; q += blockDim.x) {
      const int cnt = w.deg[q];
      if (cnt > g.k_max) continue;  // capped: the warp path below selects
      float qe[D];
#pragma unroll
      for (int d = 0; d < D; ++d) qe[d] = w.emb[size_t(q) * D + d];
      int64_t e = w.row_ptr[q];
      for (int k = 0; k < nwords; ++k) {
        unsigned m = w.rmask[size_t(q) * kMaskWords + k];
        while (m) {
          const int c = k * 32 + __ffs(m) - 1;
          m &= m - 1;
          if (e < w.e_cap) {
            w.col[e] = c0 + c;
            w.src[e] = q;
            w.d2[e] = dist2<D>(qe, ce + size_t(c) * D);
          }
          ++e;
        }
      }
    }
  }
  for (int q = q0 + warp; q < q1; q += nwarps) {
    float qe[D];
    if constexpr (D % 4 == 0) {
#pragma unroll
      for (int d = 0; d < D; d += 4) {
        const float4 v = *reinterpret_cast<const float4*>(w.emb + size_t(q) * D + d);
        qe[d] = v.x;
        qe[d + 1] = v.y;
        qe[d + 2] = v.z;
        qe[d + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d) qe[d] = w.emb[size_t(q) * D + d];
    }
    const int cnt = w.deg[q];
    // queries within k_max with stored masks were written lane-per-query above
    if (nc <= kMaskCands && cnt <= g.k_max) continue;
    const int64_t out0 = w.row_ptr[q];
    // selection threshold when more than k_max candidates pass: T is the
    // k_max-th smallest key; keys < T are kept, then the first keys == T
    unsigned T = 0xffffffffu;
    int need_eq = 0;
    const bool capped = cnt > g.k_max;
    if (capped) {
      unsigned lo = 0, hi = __float_as_uint(r2);
      for (int it = 0; it < 40 && lo < hi; ++it) {
        const unsigned mid = lo + (hi - lo) / 2;
        if (count_below<D>(qe, ce, nc, r2, mid, true) >= g.k_max)
          hi = mid;
        else
          lo = mid + 1;
      }
      T = lo;
      need_eq = g.k_max - count_below<D>(qe, ce, nc, r2, T, false);
    }
    int written = 0, eq_seen = 0;
    for (int base = 0; base < nc; base += 32) {
      const int c = base + lane;
      bool ok = false, eq = false;
      float s = 0.0f;
      if (c < nc) {
        s = dist2<D>(qe, ce + size_t(c) * D);
        ok = s < r2;
        if (capped && ok) {
          const unsigned key = __float_as_uint(s);
          eq = key == T;
          ok = key < T;
        }
      }
      if (capped) {
        const unsigned eqm = __ballot_sync(kFull, eq);
        const int eq_rank = eq_seen + __popc(eqm & ((1u << lane) - 1u));
        if (eq && eq_rank < need_eq) ok = true;
        eq_seen += __popc(eqm);
      }
      const unsigned m = __ballot_sync(kFull, ok);
      if (ok) {
        const int64_t e = out0 + written + __popc(m & ((1u << lane) - 1u));
        if (e < w.e_cap) {
          const int t = c0 + c;
          w.col[e] = t;
          w.src[e] = q;
          w.d2[e] = s;
        }
      }
      written += __popc(m);
    }
  }
}

template <int D>
void radius_d(const Batch& b, const Ws& w, const GraphParams& g, bool fill, cudaStream_t s) {
  const int grid = b.n_events * (g.n_planes - 1);
  if (grid <= 0) return;
  // set once per instantiation (thread-safe initialisation of a local static)
  static const bool attr = [] {
    cudaFuncSetAttribute(k_radius<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kCandSmemBytes);
    cudaFuncSetAttribute(k_radius<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kCandSmemBytes);
    return true;
  }();
  (void)attr;
  if (fill)
    k_radius<D, true><<<grid, kRadiusThreads, kCandSmemBytes, s>>>(b, w, g);
  else
    k_radius<D, false><<<grid, kRadiusCountThreads, kCandSmemBytes, s>>>(b, w, g);
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

// ---------------------------------------------------------------------------
// in-edge index
// ---------------------------------------------------------------------------
// In-edge index, one block per event: an event's edges are the contiguous
// range [row_ptr[v0], row_ptr[v1]) and its in-edges are among them, so its
// in_ptr / in_edge slice is built locally: in-degrees by shared-memory atomics,
// a block-wide exclusive scan, placement by cursors, then each target's list
// sorted by edge id (ascending, so the message sums have a fixed order). An
// event with more than kCscSmemHits hits counts in its slice of in_cnt.
constexpr int kCscThreads = 512;
constexpr int kCscSmemHits = 8192;
constexpr int kCscSmemEdges = 12288;  // an event's in-edge list staged in shared memory

__global__ void __launch_bounds__(kCscThreads) k_csc_event(Batch b, Ws w) {
  extern __shared__ int32_t sm_csc[];
  __shared__ int wsum[kCscThreads / 32];
  if (input_bad(w)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int ev = blockIdx.x; ev < b.n_events; ev += gridDim.x) {
    const int v0 = int(w.ev_off[ev]), v1 = int(w.ev_off[ev + 1]);
    const int n = v1 - v0;
    const int e0 = min(w.row_ptr[v0], E), e1 = min(w.row_ptr[v1], E);
    int32_t* C = n <= kCscSmemHits ? sm_csc : w.in_cnt + v0;
    for (int i = tid; i < n; i += kCscThreads) C[i] = 0;
    __syncthreads();
    for (int e = e0 + tid; e < e1; e += kCscThreads) atomicAdd(&C[w.col[e] - v0], 1);
    __syncthreads();
    // exclusive scan: thread t owns the consecutive counts [t*per, (t+1)*per)
    const int per = (n + kCscThreads - 1) / kCscThreads;
    const int a = min(n, tid * per), z = min(n, a + per);
    int sum = 0;
    for (int i = a; i < z; ++i) sum += C[i];
    int x = sum;
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
      C[i] = run;  // cursor
      w.in_ptr[v0 + i] = e0 + run;
      run += c;
    }
    if (tid == 0) w.in_ptr[v1] = e1;  // the next event writes the same value
    __syncthreads();
    // placement and per-target sort in shared memory when the event's list
    // fits (copied out coalesced), else in its slice of in_edge
    const bool staged = n <= kCscSmemHits && e1 - e0 <= kCscSmemEdges;
    int32_t* L = staged ? sm_csc + kCscSmemHits : w.in_edge + e0;  // L[k]: list position e0 + k
    for (int e = e0 + tid; e < e1; e += kCscThreads) {
      const int k = atomicAdd(&C[w.col[e] - v0], 1);
      L[k] = e;
    }
    __syncthreads();
    // C[i] is now the end of target i's list (event-local position)
    for (int i = tid; i < n; i += kCscThreads) {
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
    __syncthreads();
    if (staged)
      for (int k = tid; k < e1 - e0; k += kCscThreads) w.in_edge[e0 + k] = L[k];
    __syncthreads();  // C and the staged list are reused by the next event
  }
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

void launch_radius(const Batch& b, const Ws& w, const GraphParams& g, int D, bool fill,
                   cudaStream_t s) {
  switch (D) {
    case 1: radius_d<1>(b, w, g, fill, s); break;
    case 2: radius_d<2>(b, w, g, fill, s); break;
    case 3: radius_d<3>(b, w, g, fill, s); break;
    case 4: radius_d<4>(b, w, g, fill, s); break;
    case 5: radius_d<5>(b, w, g, fill, s); break;
    case 6: radius_d<6>(b, w, g, fill, s); break;
    case 7: radius_d<7>(b, w, g, fill, s); break;
    case 8: radius_d<8>(b, w, g, fill, s); break;
    case 16: radius_d<16>(b, w, g, fill, s); break;
    default: break;
  }
}

void launch_scan(const int32_t* in, int32_t* out, int n, int clamp_max, int32_t* counters,
                 int total_slot, int64_t cap, int32_t* blocks, cudaStream_t s) {
  const int nb = div_up(n > 0 ? n : 1, kScanChunk);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, clamp_max, blocks, counters, total_slot, cap);
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, clamp_max, blocks, counters, total_slot);
}

void launch_csc(const Batch& b, const Ws& w, cudaStream_t s) {
  if (b.n_events <= 0) return;
  static const bool attr_set = [] {
    cudaFuncSetAttribute(k_csc_event, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (kCscSmemHits + kCscSmemEdges) * int(sizeof(int32_t)));
    return true;
  }();
  (void)attr_set;
  k_csc_event<<<std::min(b.n_events, num_sms() * 16), kCscThreads,
                (kCscSmemHits + kCscSmemEdges) * sizeof(int32_t), s>>>(b, w);
}

int device_sms() { return num_sms(); }

}  // namespace gnntrk
