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
#include <atomic>
#include <mutex>

#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kThreads = 256;                      // embedding kernel
constexpr int kRowGroups = 32;                     // lanes of a warp
constexpr int kColGroups = kThreads / kRowGroups;  // warps of the embedding block

// Interaction network: every warp owns whole rows. Lane (rg = lane / 8,
// cg = lane % 8) holds RM rows (rg + 4 i) x CW columns (32 j + 4 cg + u) of a
// layer's output in registers (RM x CW = 32 accumulators); a warp covers
// WR = 4 RM rows and all H columns, so a row's LayerNorm is a reduction over
// the 8 lanes of its row group and no block-wide barrier is needed. Inputs are
// staged row-major in the warp's own shared-memory slice with a row stride of
// H + 4 floats: the four rows a warp reads at one k fall in distinct bank
// quads, and the eight lanes of a row group read the same address (broadcast).
template <int H>
struct WarpTile {
  static constexpr int CW = H / 8;    // columns per lane
  static constexpr int RM = 256 / H;  // rows per lane
  static constexpr int WR = 4 * RM;   // rows per warp
  static constexpr int NJ = CW / 4;   // float4 column chunks per lane
  static constexpr int LDH = H + 4;   // row stride of staged rows (floats)
};

// Warps per block, per variant (the autotuner picks one per kernel family).
template <int V>
struct Warps {
  static constexpr int NW = V == 0 ? 4 : 8;
};

// Variant chosen per (hidden index, kernel family: 0 encoders, 1 node step,
// 2 edge step and classifier); set by the autotuner, process wide. Variants:
// 0 = 4 warps per block, 1 = 8 warps per block, 2 = 4 warps per block with the
// weight matrices of the edge kernels and the node step staged once per block
// in shared memory at hidden 32 (the row gathers evict them from L1; the node
// encoder, and every kernel at hidden 64 and 128, run variant 0 then).
std::atomic<int> g_f32_variant[3][3] = {};

enum GMode : int { G_NODE_ENC = 0, G_EDGE_ENC = 1, G_NODE_UPD = 2, G_EDGE_UPD = 3,
                   G_EDGE_UPD_CLS = 4, G_CLS = 5, G_TRIP = 6 };

__device__ __forceinline__ bool input_bad(const Ws& w) {
  return (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) != 0;
}

// acc[i][4j+u] (+)= sum_{k < KV} A[rg + 4i][k] * WT[(k_off + k) * ldo + 32j + 4cg + u],
// k ascending; A row-major with stride LDA (K a multiple of 4, KV <= K valid)
// (SW: the weights WT are in shared memory, row stride ldo)
template <int H, int K, int KV, int LDA, bool SW = false>
__device__ __forceinline__ void warp_layer(const float* A, const LayerF32& L, int k_off, int rg,
                                           int cg, float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
  constexpr int RM = WarpTile<H>::RM, NJ = WarpTile<H>::NJ;
  const float* wp = L.WT + size_t(k_off) * L.ldo + 4 * cg;
#pragma unroll 2
  for (int k4 = 0; k4 < K; k4 += 4) {
    float4 a[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
      a[i] = *reinterpret_cast<const float4*>(A + (rg + 4 * i) * LDA + k4);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (KV < K && k4 + t >= KV) break;
      float4 q[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        q[j] = SW ? *reinterpret_cast<const float4*>(wp + size_t(k4 + t) * L.ldo + 32 * j)
                  : __ldg(reinterpret_cast<const float4*>(wp + size_t(k4 + t) * L.ldo + 32 * j));
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const float av = t == 0 ? a[i].x : (t == 1 ? a[i].y : (t == 2 ? a[i].z : a[i].w));
        const float2 a2 = make_float2(av, av);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          // two columns per packed FMA (each lane rounds like fmaf)
          float2 c01 = __ffma2_rn(a2, make_float2(q[j].x, q[j].y),
                                  make_float2(acc[i][4 * j], acc[i][4 * j + 1]));
          float2 c23 = __ffma2_rn(a2, make_float2(q[j].z, q[j].w),
                                  make_float2(acc[i][4 * j + 2], acc[i][4 * j + 3]));
          acc[i][4 * j] = c01.x;
          acc[i][4 * j + 1] = c01.y;
          acc[i][4 * j + 2] = c23.x;
          acc[i][4 * j + 3] = c23.y;
        }
      }
    }
  }
}

template <int H>
__device__ __forceinline__ void acc_bias(const float* b, int cg,
                                         float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
#pragma unroll
  for (int j = 0; j < WarpTile<H>::NJ; ++j) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(b + 32 * j + 4 * cg));
#pragma unroll
    for (int i = 0; i < WarpTile<H>::RM; ++i) {
      acc[i][4 * j] = v.x;
      acc[i][4 * j + 1] = v.y;
      acc[i][4 * j + 2] = v.z;
      acc[i][4 * j + 3] = v.w;
    }
  }
}

// acc += S[rg + 4i][32j + 4cg + u] (each lane reads only its own elements)
template <int H>
__device__ __forceinline__ void acc_add_smem(const float* S, int rg, int cg,
                                             float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
  constexpr int LD = WarpTile<H>::LDH;
#pragma unroll
  for (int i = 0; i < WarpTile<H>::RM; ++i)
#pragma unroll
    for (int j = 0; j < WarpTile<H>::NJ; ++j) {
      const float4 v = *reinterpret_cast<const float4*>(S + (rg + 4 * i) * LD + 32 * j + 4 * cg);
      acc[i][4 * j] += v.x;
      acc[i][4 * j + 1] += v.y;
      acc[i][4 * j + 2] += v.z;
      acc[i][4 * j + 3] += v.w;
    }
}

template <int H>
__device__ __forceinline__ void acc_store_smem(float* S, int rg, int cg,
                                               const float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
  constexpr int LD = WarpTile<H>::LDH;
#pragma unroll
  for (int i = 0; i < WarpTile<H>::RM; ++i)
#pragma unroll
    for (int j = 0; j < WarpTile<H>::NJ; ++j)
      *reinterpret_cast<float4*>(S + (rg + 4 * i) * LD + 32 * j + 4 * cg) =
          make_float4(acc[i][4 * j], acc[i][4 * j + 1], acc[i][4 * j + 2], acc[i][4 * j + 3]);
}

// rows of the warp to global: dst[rows[r] * ld + off + col] (rows < 0 skipped)
template <int H>
__device__ __forceinline__ void acc_store_rows(float* dst, int64_t ld, int off, const int* rows,
                                               int rg, int cg,
                                               const float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
#pragma unroll
  for (int i = 0; i < WarpTile<H>::RM; ++i) {
    const int row = rows[rg + 4 * i];
    if (row < 0) continue;
    float* d = dst + size_t(row) * ld + off + 4 * cg;
#pragma unroll
    for (int j = 0; j < WarpTile<H>::NJ; ++j)
      *reinterpret_cast<float4*>(d + 32 * j) =
          make_float4(acc[i][4 * j], acc[i][4 * j + 1], acc[i][4 * j + 2], acc[i][4 * j + 3]);
  }
}

// sum over the 8 lanes of a row group (lane bits 0..2)
__device__ __forceinline__ float row_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// per row: ReLU((v - mean) / sqrt(var + eps)) over the H columns
template <int H>
__device__ __forceinline__ void acc_ln_relu(float (&acc)[WarpTile<H>::RM][WarpTile<H>::CW]) {
  constexpr int CW = WarpTile<H>::CW;
#pragma unroll
  for (int i = 0; i < WarpTile<H>::RM; ++i) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CW; ++c) s += acc[i][c];
    const float mean = row_sum(s) / float(H);
    float q = 0.f;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const float t = acc[i][c] - mean;
      q = fmaf(t, t, q);
    }
    const float inv = 1.0f / sqrtf(row_sum(q) / float(H) + kLnEps);
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[i][c] = fmaxf((acc[i][c] - mean) * inv, 0.f);
  }
}

// S[r][col] = X[rows[r]][off + col] (+ Y[rows2[r]][off2 + col]), zero for rows < 0;
// 8 lanes per row, one float4 column chunk each, four rows per instruction.
// Loads are unconditional (row 0 stands in for a missing row, its value is
// then dropped) so that all of a lane's loads are in flight together.
template <int H, bool TWO>
__device__ __forceinline__ void stage_rows(float* S, const int* rows, const float* X, int64_t ldx,
                                           int offx, const int* rows2, const float* Y,
                                           int64_t ldy, int offy, int lane) {
  constexpr int RM = WarpTile<H>::RM, NJ = WarpTile<H>::NJ, LD = WarpTile<H>::LDH;
  const int gr = lane >> 3, q = lane & 7;
  float4 v[RM][NJ];
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int row = rows[gr + 4 * i];
    const int rx = max(row, 0);
    const int ry = TWO ? (row >= 0 ? rows2[gr + 4 * i] : 0) : 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      v[i][j] = __ldcg(reinterpret_cast<const float4*>(X + size_t(rx) * ldx + offx + 32 * j + 4 * q));
      if (TWO) {
        const float4 y =
            __ldcg(reinterpret_cast<const float4*>(Y + size_t(ry) * ldy + offy + 32 * j + 4 * q));
        v[i][j].x += y.x;
        v[i][j].y += y.y;
        v[i][j].z += y.z;
        v[i][j].w += y.w;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const bool ok = rows[gr + 4 * i] >= 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j)
      *reinterpret_cast<float4*>(S + (gr + 4 * i) * LD + 32 * j + 4 * q) =
          ok ? v[i][j] : make_float4(0.f, 0.f, 0.f, 0.f);
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
  // G_TRIP: one triplet list (its two edges, count on the device) and outputs
  const int32_t* t1;
  const int32_t* t2;
  const int32_t* tn;
  float* tlogit;
  uint8_t* tkeep;
};

template <int H, int MODE>
__host__ __device__ constexpr int g_lda() {
  return MODE == G_NODE_ENC ? 8 : WarpTile<H>::LDH;
}

// shared memory of one warp (floats): staged input A, hidden Hs, row ids and,
// for the node step, a third row buffer Bs
template <int H, int MODE>
__host__ __device__ constexpr int g_warp_floats() {
  return WarpTile<H>::WR * (g_lda<H, MODE>() + WarpTile<H>::LDH) + 4 * WarpTile<H>::WR +
         (MODE == G_NODE_UPD ? WarpTile<H>::WR * WarpTile<H>::LDH : 0);
}

// Resident blocks per SM the register budget is sized for: at h = 32 the
// 4-warp edge kernels fit 5 blocks of shared memory per SM, so their
// registers are capped to let 5 blocks (20 warps) reside; elsewhere the
// compiler's choice stands.
template <int H, int MODE, int NW, bool SW>
__host__ __device__ constexpr int g_min_blocks() {
  return (H == 32 && NW == 4 && MODE != G_NODE_ENC && MODE != G_NODE_UPD) ? (SW ? 4 : 5) : 1;
}

// Weight matrices a kernel keeps in shared memory (variant 2), in units of
// H x H floats: edge steps the e block of the first layer, the second layer
// and (last step) the classifier's first layer; the edge encoder its second
// layer; the node step its first layer (3 blocks: h, m_out, m_in) and its
// second layer, which leaves the node kernel at the 3 blocks per SM its
// registers allow. (Staging only one matrix in the edge steps, so that a
// fifth block fits an SM, measured slower: 2.14 against 2.06 ms per step of
// the headline's re-score edge steps.)
template <int MODE>
__host__ __device__ constexpr int g_sw_mats() {
  return MODE == G_EDGE_ENC ? 1
         : MODE == G_EDGE_UPD ? 2
         : MODE == G_EDGE_UPD_CLS ? 3
         : MODE == G_NODE_UPD ? 4 : 0;
}

// copy rows [0, R) of a transposed layer (row stride ldo) into S (row stride H)
template <int H, int NT, int R = H>
__device__ __forceinline__ void stage_weights(float* S, const LayerF32& L) {
  for (int i = threadIdx.x; i < R * H / 4; i += NT) {
    const int k = i / (H / 4), c = 4 * (i % (H / 4));
    *reinterpret_cast<float4*>(S + k * H + c) =
        __ldg(reinterpret_cast<const float4*>(L.WT + size_t(k) * L.ldo + c));
  }
}

template <int H, int MODE, int NW, bool SW = false>
__global__ void __launch_bounds__(NW * 32, (g_min_blocks<H, MODE, NW, SW>())) k_gnn_f32(const GnnArgs p) {
  using T = WarpTile<H>;
  constexpr int RM = T::RM, CW = T::CW, WR = T::WR;
  constexpr int LDA = g_lda<H, MODE>();
  constexpr bool EDGE_ROWS = MODE != G_NODE_ENC && MODE != G_NODE_UPD;
  static_assert(!SW || g_sw_mats<MODE>() > 0, "weights in shared memory: edge and node-step kernels");
  extern __shared__ __align__(16) float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* As = sm + warp * g_warp_floats<H, MODE>();  // [WR][LDA]
  float* Hs = As + WR * LDA;                          // [WR][H + 4]
  int* rows = reinterpret_cast<int*>(Hs + WR * T::LDH);
  int* srcs = rows + WR;
  int* dsts = srcs + WR;
  const Ws& w = p.w;
  if (input_bad(w)) return;
  int lo, hi;
  if constexpr (MODE == G_TRIP) {
    if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_CAPACITY) return;
    lo = 0;
    hi = min(*p.tn, int(w.t_cap));
    if (hi <= 0) return;
  } else {
    if (!sel_rows(p.b, w, p.sel, EDGE_ROWS, lo, hi)) return;
  }
  const int rg = lane >> 3, cg = lane & 7;
  const int E = clamp_edges(w.counters, w.e_cap);
  // the layers this kernel multiplies by: global memory, or (SW) copies in
  // shared memory after the warps' slices (row stride H)
  LayerF32 l1 = p.m.l1, l2 = p.m.l2, c1 = p.cls.l1;
  if constexpr (SW && MODE == G_NODE_UPD) {
    float* S = sm + NW * g_warp_floats<H, MODE>();
    stage_weights<H, NW * 32, 3 * H>(S, p.m.l1);  // [h, m_out, m_in] -> H
    l1 = LayerF32{S, p.m.l1.b, 3 * H, H, H};
    S += 3 * H * H;
    stage_weights<H, NW * 32>(S, p.m.l2);
    l2 = LayerF32{S, p.m.l2.b, H, H, H};
    __syncthreads();
  } else if constexpr (SW) {
    float* S = sm + NW * g_warp_floats<H, MODE>();
    if constexpr (MODE != G_EDGE_ENC) {
      stage_weights<H, NW * 32>(S, p.m.l1);  // rows [0, H): the e block
      l1 = LayerF32{S, p.m.l1.b, H, H, H};
      S += H * H;
    }
    stage_weights<H, NW * 32>(S, p.m.l2);
    l2 = LayerF32{S, p.m.l2.b, H, H, H};
    S += H * H;
    if constexpr (MODE == G_EDGE_UPD_CLS) {
      stage_weights<H, NW * 32>(S, p.cls.l1);
      c1 = LayerF32{S, p.cls.l1.b, H, H, H};
    }
    __syncthreads();
  }
  (void)l1;
  (void)l2;
  (void)c1;

  // Edge rows: the index chain (row id from the list, then its source and
  // target) is loaded ahead in registers, lane r holding row r of a tile: the
  // row ids two tiles ahead and the source / target one tile ahead are loaded
  // during a tile and first used in the next one, so a tile's row gathers
  // start without waiting for its indices.
  // (variant 2 only: the index registers push the 5-block register budget of
  // the other variants into spills)
  constexpr bool AHEAD = SW && EDGE_ROWS && MODE != G_TRIP;
  const int tstride = gridDim.x * NW * WR;
  const int base0 = lo + (blockIdx.x * NW + warp) * WR;
  auto row_at = [&](int b) {
    const int pos = b + lane;
    return (lane < WR && pos < hi) ? sel_row(p.sel, pos) : -1;
  };
  int r_cur = -1, s_cur = 0, d_cur = 0, r_next = -1;
  if constexpr (AHEAD) {
    r_cur = row_at(base0);
    s_cur = r_cur >= 0 ? w.src[r_cur] : 0;
    d_cur = r_cur >= 0 ? w.col[r_cur] : 0;
    r_next = row_at(base0 + tstride);
  }
  for (int base = base0; base < hi; base += tstride) {
    // ---- rows of this warp -----------------------------------------------
    if constexpr (AHEAD) {
      if (lane < WR) {
        rows[lane] = r_cur;
        srcs[lane] = s_cur;
        dsts[lane] = d_cur;
      }
      s_cur = r_next >= 0 ? w.src[r_next] : 0;
      d_cur = r_next >= 0 ? w.col[r_next] : 0;
      r_cur = r_next;
      r_next = row_at(base + 2 * tstride);
    } else if (lane < WR) {
      const int pos = base + lane;
      int row = -1, a = 0, c = 0;
      if (pos < hi) {
        row = MODE == G_TRIP ? pos : sel_row(p.sel, pos);
        if (MODE == G_TRIP) {
          a = p.t1[row];
          c = p.t2[row];
        } else if (EDGE_ROWS) {
          a = w.src[row];
          c = w.col[row];
        }
      }
      rows[lane] = row;
      srcs[lane] = a;
      dsts[lane] = c;
    }
    __syncwarp();
    float acc[RM][CW];

    if constexpr (MODE == G_NODE_ENC || MODE == G_NODE_UPD) {
      if constexpr (MODE == G_NODE_ENC) {
        // features (x/s3, y/s4, z/s5) of each hit, column 3 zero
        if (lane < WR) {
          const int row = rows[lane];
          float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row >= 0) {
            const float4 q = w.pos[row];
            f = make_float4(q.x / p.fs[3], q.y / p.fs[4], q.z / p.fs[5], 0.f);
          }
          *reinterpret_cast<float4*>(As + lane * LDA) = f;
        }
        __syncwarp();
        acc_bias<H>(p.m.l1.b, cg, acc);
        warp_layer<H, 4, 3, LDA>(As, p.m.l1, 0, rg, cg, acc);
        acc_ln_relu<H>(acc);
        acc_store_smem<H>(Hs, rg, cg, acc);
        __syncwarp();
        acc_bias<H>(p.m.l2.b, cg, acc);
        warp_layer<H, H, H, T::LDH>(Hs, p.m.l2, 0, rg, cg, acc);
        __syncwarp();  // all lanes are done reading Hs
      } else {
        // [h, sum_out e, sum_in e]: h in Hs, the two sums (written into the
        // node's projection row by k_msg_f32) in As and Bs
        float* Bs = Hs + WR * T::LDH + 4 * WR;
        stage_rows<H, false>(Hs, rows, w.hstate, H, 0, nullptr, nullptr, 0, 0, lane);
        stage_rows<H, false>(As, rows, w.pstate, 2 * H, 0, nullptr, nullptr, 0, 0, lane);
        stage_rows<H, false>(Bs, rows, w.pstate, 2 * H, H, nullptr, nullptr, 0, 0, lane);
        __syncwarp();
        acc_bias<H>(p.m.l1.b, cg, acc);
        warp_layer<H, H, H, T::LDH, SW>(Hs, l1, 0, rg, cg, acc);
        warp_layer<H, H, H, LDA, SW>(As, l1, H, rg, cg, acc);
        warp_layer<H, H, H, T::LDH, SW>(Bs, l1, 2 * H, rg, cg, acc);
        acc_ln_relu<H>(acc);
        __syncwarp();  // all lanes are done reading As
        acc_store_smem<H>(As, rg, cg, acc);
        __syncwarp();
        acc_bias<H>(p.m.l2.b, cg, acc);
        warp_layer<H, H, H, LDA, SW>(As, l2, 0, rg, cg, acc);
        acc_add_smem<H>(Hs, rg, cg, acc);  // residual h
      }
      acc_store_rows<H>(w.hstate, H, 0, rows, rg, cg, acc);
      // ---- projections of the new node state for the next edge layer -------
      acc_store_smem<H>(Hs, rg, cg, acc);
      __syncwarp();
      acc_bias<H>(p.proj.src.b, cg, acc);
      warp_layer<H, H, H, T::LDH>(Hs, p.proj.src, 0, rg, cg, acc);
      acc_store_rows<H>(w.pstate, 2 * H, 0, rows, rg, cg, acc);
      acc_bias<H>(p.proj.dst.b, cg, acc);
      warp_layer<H, H, H, T::LDH>(Hs, p.proj.dst, 0, rg, cg, acc);
      acc_store_rows<H>(w.pstate, 2 * H, H, rows, rg, cg, acc);
    } else if constexpr (MODE == G_TRIP) {
      // ---- triplet classifier: [e^K(first), e^K(second)] -> Linear ->
      //      LayerNorm -> ReLU -> dot, then the triplet cut -----------------
      stage_rows<H, false>(As, srcs, w.estate, H, 0, nullptr, nullptr, 0, 0, lane);
      stage_rows<H, false>(Hs, dsts, w.estate, H, 0, nullptr, nullptr, 0, 0, lane);
      __syncwarp();
      acc_bias<H>(p.m.l1.b, cg, acc);
      warp_layer<H, H, H, LDA>(As, p.m.l1, 0, rg, cg, acc);
      warp_layer<H, H, H, T::LDH>(Hs, p.m.l1, H, rg, cg, acc);
      acc_ln_relu<H>(acc);
      const LayerF32& tl2 = p.m.l2;
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < T::NJ; ++j)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            part = fmaf(acc[i][4 * j + u], __ldg(tl2.WT + size_t(32 * j + 4 * cg + u) * tl2.ldo), part);
        const float lg = tl2.b[0] + row_sum(part);
        const int row = rows[rg + 4 * i];
        if (cg == 0 && row >= 0) {
          p.tlogit[row] = lg;
          p.tkeep[row] = lg >= p.cut ? 1 : 0;
        }
      }
    } else {
      if constexpr (MODE != G_CLS) {
        // ---- layer 1: b + W_e e + (W_src h_src + W_dst h_dst, projected) ----
        stage_rows<H, true>(Hs, srcs, w.pstate, 2 * H, 0, dsts, w.pstate, 2 * H, H, lane);
        if constexpr (MODE != G_EDGE_ENC)
          stage_rows<H, false>(As, rows, w.estate, H, 0, nullptr, nullptr, 0, 0, lane);
        __syncwarp();
        acc_bias<H>(p.m.l1.b, cg, acc);
        if constexpr (MODE != G_EDGE_ENC) warp_layer<H, H, H, LDA, SW>(As, l1, 0, rg, cg, acc);
        acc_add_smem<H>(Hs, rg, cg, acc);
        acc_ln_relu<H>(acc);
        acc_store_smem<H>(Hs, rg, cg, acc);  // own elements only
        __syncwarp();
        // ---- layer 2 (+ residual e) -----------------------------------------
        acc_bias<H>(p.m.l2.b, cg, acc);
        warp_layer<H, H, H, T::LDH, SW>(Hs, l2, 0, rg, cg, acc);
        if constexpr (MODE != G_EDGE_ENC) acc_add_smem<H>(As, rg, cg, acc);
        if constexpr (MODE != G_EDGE_UPD_CLS) acc_store_rows<H>(w.estate, H, 0, rows, rg, cg, acc);
        if constexpr (MODE == G_EDGE_UPD_CLS) {
          acc_store_smem<H>(As, rg, cg, acc);  // own elements only
        }
      } else {
        stage_rows<H, false>(As, rows, w.estate, H, 0, nullptr, nullptr, 0, 0, lane);
      }
      if constexpr (MODE == G_EDGE_UPD_CLS || MODE == G_CLS) {
        // ---- classifier: Linear -> LayerNorm -> ReLU -> dot, then the cut ----
        __syncwarp();
        acc_bias<H>(p.cls.l1.b, cg, acc);
        warp_layer<H, H, H, LDA, SW && MODE == G_EDGE_UPD_CLS>(As, c1, 0, rg, cg, acc);
        acc_ln_relu<H>(acc);
        const LayerF32& cl2 = p.cls.l2;
#pragma unroll
        for (int i = 0; i < RM; ++i) {
          float part = 0.f;
#pragma unroll
          for (int j = 0; j < T::NJ; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u)
              part = fmaf(acc[i][4 * j + u], __ldg(cl2.WT + size_t(32 * j + 4 * cg + u) * cl2.ldo), part);
          const float lg = cl2.b[0] + row_sum(part);
          const int row = rows[rg + 4 * i];
          if (cg == 0 && row >= 0) {
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
      }
    }
    __syncwarp();  // the next tile overwrites this warp's shared memory
  }
}

// ---------------------------------------------------------------------------
// messages of the node step: m_v = [sum of e over v's out edges, sum over its
// in edges], each sum in increasing list order starting from zero, written to
// the node's projection row P[v] = [m_out | m_in] (the node step reads it
// there and then overwrites the row with the new projections). One group of
// 8 lanes per node, one float4 column chunk per lane; U list entries per
// round are loaded together (entries past the end reload a valid row and are
// dropped), so each lane keeps U loads in flight.
// ---------------------------------------------------------------------------
template <int H>
__global__ void __launch_bounds__(256) k_msg_f32(Batch b, Ws w, Sel sel) {
  constexpr int NJ = H / 32, U = 8 / NJ;
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(b, w, sel, false, lo, hi)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int q = threadIdx.x & 7;
  const int groups = gridDim.x * (blockDim.x >> 3);
  for (int pos = lo + blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3); pos < hi; pos += groups) {
    const int row = sel_row(sel, pos);
    float* out = w.pstate + size_t(row) * 2 * H + 4 * q;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      int a, n;
      if (side == 0) {
        a = min(w.row_ptr[row], E);
        n = min(w.row_ptr[row + 1], E) - a;
      } else {
        a = w.in_ptr[row];
        n = w.in_ptr[row + 1] - a;
      }
      float4 s[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) s[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int t0 = 0; t0 < n; t0 += U) {
        float4 v[U][NJ];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int at = a + min(t0 + u, n - 1);
          const int e = side == 0 ? at : __ldg(w.in_edge + at);
#pragma unroll
          for (int j = 0; j < NJ; ++j)
            v[u][j] = __ldg(reinterpret_cast<const float4*>(w.estate + size_t(e) * H + 32 * j + 4 * q));
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t0 + u < n) {
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              const float2 lo = __fadd2_rn(make_float2(s[j].x, s[j].y), make_float2(v[u][j].x, v[u][j].y));
              const float2 hi = __fadd2_rn(make_float2(s[j].z, s[j].w), make_float2(v[u][j].z, v[u][j].w));
              s[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
          }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        *reinterpret_cast<float4*>(out + side * H + 32 * j) = s[j];
    }
  }
}

// ---- transposed register tiles of the embedding MLP -------------------------
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
        // two columns per packed FMA (each lane rounds like fmaf)
        const float2 a2 = make_float2(a[i], a[i]);
        const float2 c01 = __ffma2_rn(a2, make_float2(q.x, q.y), make_float2(acc[i][j], acc[i][j + 1]));
        const float2 c23 = __ffma2_rn(a2, make_float2(q.z, q.w), make_float2(acc[i][j + 2], acc[i][j + 3]));
        acc[i][j] = c01.x;
        acc[i][j + 1] = c01.y;
        acc[i][j + 2] = c23.x;
        acc[i][j + 3] = c23.y;
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

__global__ void __launch_bounds__(kThreads, 3) k_embed_f32(Batch b, Ws w, EmbedLayers em,
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
  static std::mutex mu;  // handles may launch from several host threads
  std::lock_guard<std::mutex> lock(mu);
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
void launch_gnn_v(const GnnArgs& a, int64_t rows_hint, cudaStream_t s) {
  // (at hidden 64 and 128 the matrices would cost most of the shared memory
  // the warps' slices need, so variant 2 is variant 0 there)
  constexpr bool SW = V == 2 && H == 32 && g_sw_mats<MODE>() > 0;
  constexpr int NW = Warps<V == 1 ? 1 : 0>::NW, WR = WarpTile<H>::WR;
  const size_t smem =
      (size_t(NW) * g_warp_floats<H, MODE>() + (SW ? size_t(g_sw_mats<MODE>()) * H * H : 0)) *
      sizeof(float);
  const void* fn = (const void*)k_gnn_f32<H, MODE, NW, SW>;
  const int full = device_sms() * blocks_per_sm(fn, NW * 32, smem);
  dim3 grid(full, 1);
  if (a.sel.rows == nullptr && rows_hint >= 0)
    grid.x = rows_hint == 0 ? 1 : unsigned(std::min<int64_t>(full, div_up(rows_hint, NW * WR)));
  k_gnn_f32<H, MODE, NW, SW><<<grid, NW * 32, smem, s>>>(a);
}

constexpr int f32_family(int mode) {
  return (mode == G_NODE_ENC || mode == G_EDGE_ENC) ? 0 : (mode == G_NODE_UPD ? 1 : 2);
}

template <int H, int MODE>
void launch_gnn(const GnnArgs& a, int64_t rows_hint, cudaStream_t s) {
  const int v =
      g_f32_variant[H == 32 ? 0 : (H == 64 ? 1 : 2)][f32_family(MODE)].load(std::memory_order_relaxed);
  if (v == 2)
    launch_gnn_v<H, MODE, 2>(a, rows_hint, s);
  else if (v == 1)
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
    case G_TRIP: launch_gnn<HH, G_TRIP>(a, rows_hint, s); break;                    \
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

void launch_triplet_scores_f32(const Batch& b, const Ws& w, const TripletHeads& t, int h,
                               float cut_logit, cudaStream_t s) {
  GnnArgs a{};
  a.b = b;
  a.w = w;
  a.cut = cut_logit;
  a.sel = Sel{nullptr, nullptr};
  a.m = t.art;
  a.t1 = w.trip_a1;
  a.t2 = w.trip_a2;
  a.tn = w.counters + C_TRIP_A;
  a.tlogit = w.trip_alogit;
  a.tkeep = w.trip_akeep;
  launch_gnn_any(h, G_TRIP, a, -1, s);
  a.m = t.elb;
  a.t1 = w.trip_e1;
  a.t2 = w.trip_e2;
  a.tn = w.counters + C_TRIP_E;
  a.tlogit = w.trip_elogit;
  a.tkeep = w.trip_ekeep;
  launch_gnn_any(h, G_TRIP, a, -1, s);
}

void f32_set_variant(int h, int family, int v) {
  if ((h != 32 && h != 64 && h != 128) || family < 0 || family > 2) return;
  g_f32_variant[h == 32 ? 0 : (h == 64 ? 1 : 2)][family].store((v >= 0 && v <= 2) ? v : 0,
                                                                std::memory_order_relaxed);
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

void launch_messages_f32(const Batch& b, const Ws& w, int h, Sel sel, cudaStream_t s) {
  if (b.n_hits <= 0) return;
  const int full = device_sms() * 8;
  const int grid = sel.rows ? full : std::max(1, std::min(full, div_up(b.n_hits, 32)));
  if (h == 32)
    k_msg_f32<32><<<grid, 256, 0, s>>>(b, w, sel);
  else if (h == 64)
    k_msg_f32<64><<<grid, 256, 0, s>>>(b, w, sel);
  else
    k_msg_f32<128><<<grid, 256, 0, s>>>(b, w, sel);
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
