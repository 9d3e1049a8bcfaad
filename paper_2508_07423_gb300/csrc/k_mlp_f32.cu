// FP32 SIMT kernels of the embedding MLP and the interaction network.
//
// Work is cut into tiles of TM rows (hits or edges). A block of 256 threads
// stages the tile's input rows TRANSPOSED in shared memory (As[k][row], so a
// warp reading one k for 32 row groups touches consecutive words) and computes
// each layer as a register-tiled product: thread (lane, warp) owns RM rows x CW
// columns of the output, reads RM inputs per k with one vector shared-memory
// load and CW weights with CW/4 warp-uniform float4 loads through the
// read-only cache, and keeps RM x CW FP32 accumulators in registers (inputs are
// added in increasing k order). A hidden layer is written back transposed; one
// thread per row then applies LayerNorm + ReLU over it in place.
//
//  k_embed_f32     embedding MLP (Sec. "Hit Embedding and Rough Graph
//                  Construction") on (r/s0, phi/s1, z/s2), ReLU between layers
//  k_gnn_f32<MODE> node encoder on (x/s3, y/s4, z/s5); edge encoder on
//                  [h_src, h_dst]; node step: m = [sum_out e, sum_in e]
//                  (Eq. of m^k_l), h <- h + N_k([h, m]); edge step:
//                  e <- e + E_k([e, h_src, h_dst]) with the updated h, and at
//                  the last step the classifier and the cut (Sec. "Graph Neural
//                  Network and Classifiers"). Sub-networks are
//                  Linear -> LayerNorm -> ReLU -> Linear.
#include <algorithm>

#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kThreads = 256;                      // embedding kernel
constexpr int kRowGroups = 32;                     // lanes of a warp
constexpr int kColGroups = kThreads / kRowGroups;  // warps of the embedding block

// Interaction-network tile shape per hidden width: NT threads in NCG column
// groups (warps w with the same w % NCG share columns), TM rows. Per k a warp
// reads RM rows of A (RM wavefronts) and CW weights (CW/4 uniform loads) for
// RM x CW FMAs per lane, so RM * CW / 4 FMA cycles per RM + CW / 4 wavefronts.
// Two variants per width; the autotuner picks one per kernel family.
template <int H, int V>
struct Shape;
template <>
struct Shape<32, 0> {
  static constexpr int NT = 256, NCG = 8, TM = 128;  // RM 4, CW 4
};
template <>
struct Shape<32, 1> {
  static constexpr int NT = 256, NCG = 4, TM = 128;  // RM 2, CW 8
};
template <>
struct Shape<64, 0> {
  static constexpr int NT = 256, NCG = 8, TM = 64;   // RM 2, CW 8
};
template <>
struct Shape<64, 1> {
  static constexpr int NT = 128, NCG = 4, TM = 64;   // RM 2, CW 16
};
template <>
struct Shape<128, 0> {
  static constexpr int NT = 256, NCG = 8, TM = 64;   // RM 2, CW 16
};
template <>
struct Shape<128, 1> {
  static constexpr int NT = 128, NCG = 4, TM = 64;   // RM 2, CW 32
};

// Variant chosen per (hidden index, kernel family: 0 encoders, 1 node step,
// 2 edge step and classifier); set by the autotuner, process wide.
int g_f32_variant[3][3] = {};

enum GMode : int { G_NODE_ENC = 0, G_EDGE_ENC = 1, G_NODE_UPD = 2, G_EDGE_UPD = 3,
                   G_EDGE_UPD_CLS = 4, G_CLS = 5 };

__device__ __forceinline__ bool input_bad(const Ws& w) {
  return (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) != 0;
}

// acc[i][j] = b[c0 + j] + sum_k A[k][r0 + i] * W[k][c0 + j]
// A: shared [K][TM]; W: global [K][ldo] (transposed weights)
template <int RM, int CW, int TM>
__device__ __forceinline__ void tile_layer(const float* As, int K, const LayerF32& L, int r0,
                                           int c0, float (&acc)[RM][CW]) {
  static_assert(CW % 4 == 0 && (RM == 2 || RM == 4), "tile shape");
#pragma unroll
  for (int j = 0; j < CW; j += 4) {
    const float4 bb = __ldg(reinterpret_cast<const float4*>(L.b + c0 + j));
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      acc[i][j] = bb.x;
      acc[i][j + 1] = bb.y;
      acc[i][j + 2] = bb.z;
      acc[i][j + 3] = bb.w;
    }
  }
  const float* wp = L.WT + c0;
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    float a[RM];
    if constexpr (RM == 4) {
      const float4 v = *reinterpret_cast<const float4*>(As + k * TM + r0);
      a[0] = v.x;
      a[1] = v.y;
      a[2] = v.z;
      a[3] = v.w;
    } else {
      const float2 v = *reinterpret_cast<const float2*>(As + k * TM + r0);
      a[0] = v.x;
      a[1] = v.y;
    }
    const float4* w4 = reinterpret_cast<const float4*>(wp + size_t(k) * L.ldo);
#pragma unroll
    for (int j = 0; j < CW; j += 4) {
      const float4 q = __ldg(w4 + j / 4);
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        acc[i][j] = fmaf(a[i], q.x, acc[i][j]);
        acc[i][j + 1] = fmaf(a[i], q.y, acc[i][j + 1]);
        acc[i][j + 2] = fmaf(a[i], q.z, acc[i][j + 2]);
        acc[i][j + 3] = fmaf(a[i], q.w, acc[i][j + 3]);
      }
    }
  }
}

// store acc transposed into S[c][row] (one vector store per column)
template <int RM, int CW, int TM>
__device__ __forceinline__ void tile_store_t(float* S, int r0, int c0, const float (&acc)[RM][CW],
                                             bool relu) {
#pragma unroll
  for (int j = 0; j < CW; ++j) {
    float v[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) v[i] = relu ? fmaxf(acc[i][j], 0.f) : acc[i][j];
    if constexpr (RM == 4)
      *reinterpret_cast<float4*>(S + (c0 + j) * TM + r0) = make_float4(v[0], v[1], v[2], v[3]);
    else
      *reinterpret_cast<float2*>(S + (c0 + j) * TM + r0) = make_float2(v[0], v[1]);
  }
}

// in place over column r of S[n][TM]: ReLU((v - mean) / sqrt(var + eps))
template <int TM>
__device__ __forceinline__ void col_ln_relu(float* S, int n, int r) {
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += S[i * TM + r];
  const float mean = s / float(n);
  float q = 0.f;
  for (int i = 0; i < n; ++i) {
    const float t = S[i * TM + r] - mean;
    q = fmaf(t, t, q);
  }
  const float inv = 1.0f / sqrtf(q / float(n) + kLnEps);
  for (int i = 0; i < n; ++i) S[i * TM + r] = fmaxf((S[i * TM + r] - mean) * inv, 0.f);
}

// copy an h-float global row into column `row` of S[k0 .. k0+h)[TM]
template <int TM>
__device__ __forceinline__ void put_col(float* S, int k0, int row, const float* src, int h) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (int c = 0; c < h / 4; ++c) {
    const float4 v = s4[c];
    S[(k0 + 4 * c) * TM + row] = v.x;
    S[(k0 + 4 * c + 1) * TM + row] = v.y;
    S[(k0 + 4 * c + 2) * TM + row] = v.z;
    S[(k0 + 4 * c + 3) * TM + row] = v.w;
  }
}

template <int TM>
__device__ __forceinline__ void add_col(float* S, int k0, int row, const float* src, int h) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (int c = 0; c < h / 4; ++c) {
    const float4 v = s4[c];
    S[(k0 + 4 * c) * TM + row] += v.x;
    S[(k0 + 4 * c + 1) * TM + row] += v.y;
    S[(k0 + 4 * c + 2) * TM + row] += v.z;
    S[(k0 + 4 * c + 3) * TM + row] += v.w;
  }
}

// ---------------------------------------------------------------------------
// interaction network, one kernel per mode
// ---------------------------------------------------------------------------
struct GnnArgs {
  Batch b;
  Ws w;
  EdgeProj proj;  // node kernels: projections for the next edge layer
  Mlp2F32 m;    // the sub-network of this kernel
  Mlp2F32 cls;  // classifier (G_EDGE_UPD_CLS, G_CLS)
  float fs[6];
  float cut;
  int rescore_only;
  float band_lo, band_hi;
  Sel sel;
};

__host__ __device__ constexpr int g_nseg(int mode) {
  return mode == G_NODE_ENC ? 0 : (mode == G_EDGE_ENC ? 2 : (mode == G_CLS ? 1 : 3));
}

template <int H, int MODE, int V>
__global__ void __launch_bounds__(Shape<H, V>::NT) k_gnn_f32(const GnnArgs p) {
  constexpr int NT = Shape<H, V>::NT, NCG = Shape<H, V>::NCG, TM = Shape<H, V>::TM;
  constexpr int RM = TM / (NT / NCG);
  constexpr int CW = H / NCG;
  constexpr int NSEG = g_nseg(MODE);
  constexpr int K1 = MODE == G_NODE_ENC ? 3 : NSEG * H;
  constexpr int KA = K1 > 4 ? K1 : 4;
  extern __shared__ __align__(16) float sm[];
  float* As = sm;            // [KA][TM] input rows, transposed
  float* Hs = sm + KA * TM;  // [H][TM] hidden rows, transposed
  const Ws& w = p.w;
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(p.b, w, p.sel, MODE != G_NODE_ENC && MODE != G_NODE_UPD, lo, hi)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = ((warp / NCG) * 32 + lane) * RM;
  const int c0 = (warp % NCG) * CW;
  const int E = clamp_edges(w.counters, w.e_cap);

  for (int base = lo + blockIdx.x * TM; base < hi; base += gridDim.x * TM) {
    // ---- gather: task t = (segment t / TM, row t % TM) --------------------
    if constexpr (MODE == G_NODE_ENC) {
      for (int r = tid; r < TM; r += NT) {
        const int pos = base + r;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        if (pos < hi) {
          const float4 q = w.pos[sel_row(p.sel, pos)];
          f0 = q.x / p.fs[3];
          f1 = q.y / p.fs[4];
          f2 = q.z / p.fs[5];
        }
        As[r] = f0;
        As[TM + r] = f1;
        As[2 * TM + r] = f2;
      }
    } else {
      for (int t = tid; t < NSEG * TM; t += NT) {
        const int seg = t / TM, r = t % TM, pos = base + r;
        const int k0 = seg * H;
        if (pos >= hi) {
          for (int k = 0; k < H; ++k) As[(k0 + k) * TM + r] = 0.f;
          continue;
        }
        const int row = sel_row(p.sel, pos);
        if constexpr (MODE == G_NODE_UPD) {
          if (seg == 0) {
            put_col<TM>(As, k0, r, w.hstate + size_t(row) * H, H);
          } else {
            for (int k = 0; k < H; ++k) As[(k0 + k) * TM + r] = 0.f;
            if (seg == 1) {
              const int a = min(w.row_ptr[row], E), z = min(w.row_ptr[row + 1], E);
              for (int e = a; e < z; ++e) add_col<TM>(As, k0, r, w.estate + size_t(e) * H, H);
            } else {
              const int a = w.in_ptr[row], z = w.in_ptr[row + 1];
              for (int q = a; q < z; ++q)
                add_col<TM>(As, k0, r, w.estate + size_t(w.in_edge[q]) * H, H);
            }
          }
        } else if constexpr (MODE == G_EDGE_ENC) {
          // projections: W_src h_src (first half of P[src]), W_dst h_dst (second half of P[dst])
          put_col<TM>(As, k0, r,
                      w.pstate + size_t(seg == 0 ? w.src[row] : w.col[row]) * 2 * H + seg * H, H);
        } else if constexpr (MODE == G_CLS) {
          put_col<TM>(As, k0, r, w.estate + size_t(row) * H, H);
        } else {  // edge step: [e, W_src h_src, W_dst h_dst]
          const float* src =
              seg == 0 ? w.estate + size_t(row) * H
                       : w.pstate + size_t(seg == 1 ? w.src[row] : w.col[row]) * 2 * H + (seg - 1) * H;
          put_col<TM>(As, k0, r, src, H);
        }
      }
    }
    __syncthreads();

    float acc[RM][CW];
    if constexpr (MODE != G_CLS) {
      // ---- layer 1 -> LayerNorm -> ReLU -------------------------------------
      if constexpr (MODE == G_EDGE_ENC) {
        // b + W_src h_src + W_dst h_dst: the products come projected
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const float bj = p.m.l1.b[c0 + j];
#pragma unroll
          for (int i = 0; i < RM; ++i)
            acc[i][j] = bj + As[(c0 + j) * TM + r0 + i] + As[(H + c0 + j) * TM + r0 + i];
        }
      } else if constexpr (MODE == G_EDGE_UPD || MODE == G_EDGE_UPD_CLS) {
        // b + W_e e over the e block, plus the gathered projections
        LayerF32 le = p.m.l1;
        le.in = H;
        tile_layer<RM, CW, TM>(As, H, le, r0, c0, acc);
#pragma unroll
        for (int j = 0; j < CW; ++j)
#pragma unroll
          for (int i = 0; i < RM; ++i)
            acc[i][j] += As[(H + c0 + j) * TM + r0 + i] + As[(2 * H + c0 + j) * TM + r0 + i];
      } else {
        tile_layer<RM, CW, TM>(As, K1, p.m.l1, r0, c0, acc);
      }
      tile_store_t<RM, CW, TM>(Hs, r0, c0, acc, false);
      __syncthreads();
      for (int r = tid; r < TM; r += NT) col_ln_relu<TM>(Hs, H, r);
      __syncthreads();
      // ---- layer 2 + residual ---------------------------------------------
      tile_layer<RM, CW, TM>(Hs, H, p.m.l2, r0, c0, acc);
      if constexpr (MODE == G_NODE_UPD || MODE == G_EDGE_UPD || MODE == G_EDGE_UPD_CLS) {
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < CW; ++j) acc[i][j] += As[(c0 + j) * TM + r0 + i];
      }
    }
    if constexpr (MODE == G_EDGE_UPD_CLS || MODE == G_CLS) {
      // ---- classifier: Linear -> LayerNorm -> ReLU -> dot, then the cut ------
      if constexpr (MODE == G_EDGE_UPD_CLS) {
        // the new edge state becomes segment 0 of As (each element is read and
        // written by the same thread)
        tile_store_t<RM, CW, TM>(As, r0, c0, acc, false);
        __syncthreads();
      }
      tile_layer<RM, CW, TM>(As, H, p.cls.l1, r0, c0, acc);
      __syncthreads();  // everyone is done reading Hs (layer 2 above)
      tile_store_t<RM, CW, TM>(Hs, r0, c0, acc, false);
      __syncthreads();
      for (int r = tid; r < TM; r += NT) {
        col_ln_relu<TM>(Hs, H, r);
        if (base + r < hi) {
          const int row = sel_row(p.sel, base + r);
          float lg = p.cls.l2.b[0];
          for (int k = 0; k < H; ++k) lg = fmaf(Hs[k * TM + r], p.cls.l2.WT[k * p.cls.l2.ldo], lg);
          bool write = true;
          if (p.rescore_only) {
            const float old = w.logit[row];
            write = old > p.band_lo && old < p.band_hi;
          }
          if (write) {
            w.logit[row] = lg;
            w.keep[row] = lg >= p.cut ? 1 : 0;
          }
        }
      }
    } else {
      // ---- store the new state ---------------------------------------------
      float* dst = (MODE == G_NODE_ENC || MODE == G_NODE_UPD) ? w.hstate : w.estate;
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        if (base + r0 + i < hi) {
          const int row = sel_row(p.sel, base + r0 + i);
          float4* d4 = reinterpret_cast<float4*>(dst + size_t(row) * H + c0);
#pragma unroll
          for (int j = 0; j < CW; j += 4)
            d4[j / 4] = make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
        }
      }
      if constexpr (MODE == G_NODE_ENC || MODE == G_NODE_UPD) {
        // ---- projections of the new node state for the next edge layer -----
        __syncthreads();  // everyone is done reading Hs (layer 2 above)
        tile_store_t<RM, CW, TM>(Hs, r0, c0, acc, false);
        __syncthreads();
        for (int half = 0; half < 2; ++half) {
          tile_layer<RM, CW, TM>(Hs, H, half == 0 ? p.proj.src : p.proj.dst, r0, c0, acc);
#pragma unroll
          for (int i = 0; i < RM; ++i) {
            if (base + r0 + i < hi) {
              const int row = sel_row(p.sel, base + r0 + i);
              float4* d4 = reinterpret_cast<float4*>(w.pstate + size_t(row) * 2 * H + half * H + c0);
#pragma unroll
              for (int j = 0; j < CW; j += 4)
                d4[j / 4] = make_float4(acc[i][j], acc[i][j + 1], acc[i][j + 2], acc[i][j + 3]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// embedding MLP
// ---------------------------------------------------------------------------
struct EmbedLayers {
  LayerF32 l[kMaxEmbedLayers];
};

constexpr int kEmbedTM = 128;

template <int CW>
__device__ __forceinline__ void embed_layer_tiled(const float* X, float* Y, const LayerF32& L,
                                                  int tid, bool relu) {
  float acc[4][CW];
  const int r0 = (tid % kRowGroups) * 4, c0 = (tid / kRowGroups) * CW;
  tile_layer<4, CW, kEmbedTM>(X, L.in, L, r0, c0, acc);
  tile_store_t<4, CW, kEmbedTM>(Y, r0, c0, acc, relu);
}

__global__ void __launch_bounds__(kThreads) k_embed_f32(Batch b, Ws w, EmbedLayers em,
                                                        int n_embed, int D, GraphParams g,
                                                        int maxw) {
  extern __shared__ __align__(16) float sm[];
  if (input_bad(w)) return;
  const int tid = threadIdx.x;
  for (int base = blockIdx.x * kEmbedTM; base < b.n_hits; base += gridDim.x * kEmbedTM) {
    float* X = sm;
    float* Y = sm + maxw * kEmbedTM;
    for (int r = tid; r < kEmbedTM; r += kThreads) {
      const int v = base + r;
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (v < b.n_hits) {
        const float4 p = w.pos[v];
        f0 = sqrtf(p.x * p.x + p.y * p.y) / g.fs[0];
        f1 = atan2f(p.y, p.x) / g.fs[1];
        f2 = p.z / g.fs[2];
      }
      X[r] = f0;
      X[kEmbedTM + r] = f1;
      X[2 * kEmbedTM + r] = f2;
    }
    __syncthreads();
    for (int l = 0; l < n_embed; ++l) {
      const LayerF32& L = em.l[l];
      const bool relu = l + 1 < n_embed;
      const int cw = L.ldo / kColGroups;
      if (L.ldo % 32 == 0 && (cw == 4 || cw == 8 || cw == 16)) {
        // register-tiled: 32 row groups x 8 column groups of ldo/8 columns
        if (cw == 4)
          embed_layer_tiled<4>(X, Y, L, tid, relu);
        else if (cw == 8)
          embed_layer_tiled<8>(X, Y, L, tid, relu);
        else
          embed_layer_tiled<16>(X, Y, L, tid, relu);
      } else {
        // any other width (the D-wide output): one thread per (row, output)
        for (int t = tid; t < kEmbedTM * L.out; t += kThreads) {
          const int r = t % kEmbedTM, o = t / kEmbedTM;
          float a = L.b[o];
          for (int k = 0; k < L.in; ++k) a = fmaf(X[k * kEmbedTM + r], L.WT[k * L.ldo + o], a);
          Y[o * kEmbedTM + r] = relu ? fmaxf(a, 0.f) : a;
        }
      }
      __syncthreads();
      float* t = X;
      X = Y;
      Y = t;
    }
    for (int t = tid; t < kEmbedTM * D; t += kThreads) {
      const int r = t / D, d = t % D, v = base + r;
      if (v < b.n_hits) w.emb[size_t(v) * D + d] = X[d * kEmbedTM + r];
    }
    __syncthreads();
  }
}

// occupancy of (kernel, block size, shared memory), queried once and cached
int blocks_per_sm(const void* fn, int threads, size_t smem) {
  struct Entry {
    const void* fn;
    int threads;
    size_t smem;
    int n;
  };
  static Entry cache[64];
  static int used = 0;
  for (int i = 0; i < used; ++i)
    if (cache[i].fn == fn && cache[i].threads == threads && cache[i].smem == smem) return cache[i].n;
  int n = 0;
  // the attribute is an upper bound: set it once to the device maximum, so a
  // later configuration with less shared memory never lowers it
  bool seen = false;
  for (int i = 0; i < used; ++i) seen = seen || cache[i].fn == fn;
  if (!seen) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
  n = n > 0 ? n : 1;
  if (used < 64) cache[used++] = Entry{fn, threads, smem, n};
  return n;
}

template <int H, int MODE, int V>
size_t gnn_smem() {
  constexpr int TM = Shape<H, V>::TM;
  constexpr int NSEG = g_nseg(MODE);
  constexpr int K1 = MODE == G_NODE_ENC ? 3 : NSEG * H;
  return size_t((K1 > 4 ? K1 : 4) + H) * TM * sizeof(float);
}

template <int H, int MODE, int V>
void launch_gnn_v(const GnnArgs& a, int64_t rows_hint, cudaStream_t s) {
  constexpr int TM = Shape<H, V>::TM, NT = Shape<H, V>::NT;
  const size_t smem = gnn_smem<H, MODE, V>();
  const void* fn = (const void*)k_gnn_f32<H, MODE, V>;
  const int full = device_sms() * blocks_per_sm(fn, NT, smem);
  dim3 grid(full, 1);
  if (a.sel.rows == nullptr && rows_hint >= 0)
    grid.x = rows_hint == 0 ? 1 : unsigned(std::min<int64_t>(full, div_up(rows_hint, TM)));
  k_gnn_f32<H, MODE, V><<<grid, NT, smem, s>>>(a);
}

constexpr int f32_family(int mode) {
  return (mode == G_NODE_ENC || mode == G_EDGE_ENC) ? 0 : (mode == G_NODE_UPD ? 1 : 2);
}

template <int H, int MODE>
void launch_gnn(const GnnArgs& a, int64_t rows_hint, cudaStream_t s) {
  const int v = g_f32_variant[H == 32 ? 0 : (H == 64 ? 1 : 2)][f32_family(MODE)];
  if (v == 1)
    launch_gnn_v<H, MODE, 1>(a, rows_hint, s);
  else
    launch_gnn_v<H, MODE, 0>(a, rows_hint, s);
}

void launch_gnn_any(int h, int mode, const GnnArgs& a, int64_t rows_hint, cudaStream_t s) {
#define GNNTRK_M(HH)                                                                \
  switch (mode) {                                                                   \
    case G_NODE_ENC: launch_gnn<HH, G_NODE_ENC>(a, rows_hint, s); break;            \
    case G_EDGE_ENC: launch_gnn<HH, G_EDGE_ENC>(a, rows_hint, s); break;            \
    case G_NODE_UPD: launch_gnn<HH, G_NODE_UPD>(a, rows_hint, s); break;            \
    case G_EDGE_UPD: launch_gnn<HH, G_EDGE_UPD>(a, rows_hint, s); break;            \
    case G_EDGE_UPD_CLS: launch_gnn<HH, G_EDGE_UPD_CLS>(a, rows_hint, s); break;    \
    case G_CLS: launch_gnn<HH, G_CLS>(a, rows_hint, s); break;                      \
  }
  if (h == 32) {
    GNNTRK_M(32)
  } else if (h == 64) {
    GNNTRK_M(64)
  } else {
    GNNTRK_M(128)
  }
#undef GNNTRK_M
}

GnnArgs gnn_args(const Batch& b, const Ws& w, Sel sel) {
  GnnArgs a{};
  a.b = b;
  a.w = w;
  a.sel = sel;
  return a;
}

}  // namespace

void f32_set_variant(int h, int family, int v) {
  if ((h != 32 && h != 64 && h != 128) || family < 0 || family > 2) return;
  g_f32_variant[h == 32 ? 0 : (h == 64 ? 1 : 2)][family] = (v == 1) ? 1 : 0;
}

int f32_get_variant(int h, int family) {
  if ((h != 32 && h != 64 && h != 128) || family < 0 || family > 2) return 0;
  return g_f32_variant[h == 32 ? 0 : (h == 64 ? 1 : 2)][family];
}

void launch_node_prep_f32(const Batch& b, const Ws& w, const LayerF32* embed, int n_embed,
                          const Mlp2F32& node_enc, const EdgeProj& proj, int D, int h,
                          const GraphParams& g, bool do_embed, bool do_node_enc, Sel sel,
                          cudaStream_t s) {
  if (b.n_hits <= 0) return;
  if (do_embed) {
    EmbedLayers em{};
    int maxw = 4;
    for (int l = 0; l < n_embed; ++l) {
      em.l[l] = embed[l];
      maxw = std::max(maxw, embed[l].ldo);
    }
    const size_t smem = size_t(2) * maxw * kEmbedTM * sizeof(float);
    const int full = device_sms() * blocks_per_sm((const void*)k_embed_f32, kThreads, smem);
    const int grid = std::max(1, std::min(full, div_up(b.n_hits, kEmbedTM)));
    k_embed_f32<<<grid, kThreads, smem, s>>>(b, w, em, n_embed, D, g, maxw);
  }
  if (do_node_enc) {
    GnnArgs a = gnn_args(b, w, sel);
    a.m = node_enc;
    a.proj = proj;
    for (int i = 0; i < 6; ++i) a.fs[i] = g.fs[i];
    launch_gnn_any(h, G_NODE_ENC, a, b.n_hits, s);
  }
}

void launch_edge_enc_f32(const Batch& b, const Ws& w, const Mlp2F32& m, int h, Sel sel,
                         cudaStream_t s) {
  GnnArgs a = gnn_args(b, w, sel);
  a.m = m;
  launch_gnn_any(h, G_EDGE_ENC, a, -1, s);
}

void launch_node_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, const EdgeProj& proj,
                            int h, Sel sel, cudaStream_t s) {
  if (b.n_hits <= 0) return;
  GnnArgs a = gnn_args(b, w, sel);
  a.m = m;
  a.proj = proj;
  launch_gnn_any(h, G_NODE_UPD, a, b.n_hits, s);
}

void launch_edge_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, const Mlp2F32* cls,
                            int h, float cut_logit, bool rescore_only, float band_lo,
                            float band_hi, Sel sel, cudaStream_t s) {
  GnnArgs a = gnn_args(b, w, sel);
  a.m = m;
  if (cls) a.cls = *cls;
  a.cut = cut_logit;
  a.rescore_only = rescore_only;
  a.band_lo = band_lo;
  a.band_hi = band_hi;
  const int mode = cls == nullptr ? G_EDGE_UPD : (m.l1.WT == nullptr ? G_CLS : G_EDGE_UPD_CLS);
  launch_gnn_any(h, mode, a, -1, s);
}

}  // namespace gnntrk
