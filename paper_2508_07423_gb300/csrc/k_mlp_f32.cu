// FP32 SIMT kernels of the embedding MLP and the interaction network.
//
// One thread owns one row (a hit or an edge). Its input row, hidden row and
// output live in thread-private rows of shared memory (odd strides, so the 32
// rows a warp touches at one column fall in 32 different banks); the weights
// are read through the read-only cache as float4 (every thread of a warp reads
// the same address, one transaction). Each layer accumulates 32 outputs at a
// time in registers, adding inputs in increasing index order.
//
//  k_node_prep_f32   embedding MLP (Sec. "Hit Embedding and Rough Graph
//                    Construction") on (r/s0, phi/s1, z/s2) and the node encoder
//                    on (x/s3, y/s4, z/s5) (Sec. "Graph Neural Network and
//                    Classifiers").
//  k_edge_enc_f32    edge encoder on [h_src, h_dst].
//  k_node_upd_f32    message m_l = [sum of outgoing e, sum of incoming e]
//                    (Eq. of m^k_l) and h_l <- h_l + N_k([h_l, m_l]).
//  k_edge_upd_f32    e_ij <- e_ij + E_k([e_ij, h_i, h_j]) with the updated h;
//                    at the last step also the edge classifier and the cut.
// Sub-networks are Linear -> LayerNorm -> ReLU -> Linear.
#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kPrepThreads = 64;

__device__ __forceinline__ bool input_bad(const Ws& w) {
  return (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) != 0;
}

// out[o] = b[o] + sum_i in[i] * W[o][i] for o < ldo (padding columns give 0)
__device__ __forceinline__ void row_linear(const float* in, const LayerF32& L, float* out,
                                           bool relu) {
  for (int o0 = 0; o0 < L.ldo; o0 += 32) {
    const int nv = min(8, (L.ldo - o0) >> 2);
    float acc[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < nv) bb = __ldg(reinterpret_cast<const float4*>(L.b + o0) + j);
      acc[4 * j] = bb.x;
      acc[4 * j + 1] = bb.y;
      acc[4 * j + 2] = bb.z;
      acc[4 * j + 3] = bb.w;
    }
    const float* wrow = L.WT + o0;
    for (int i = 0; i < L.in; ++i) {
      const float a = in[i];
      const float4* wv = reinterpret_cast<const float4*>(wrow + size_t(i) * L.ldo);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < nv) {
          const float4 q = __ldg(wv + j);
          acc[4 * j] = fmaf(a, q.x, acc[4 * j]);
          acc[4 * j + 1] = fmaf(a, q.y, acc[4 * j + 1]);
          acc[4 * j + 2] = fmaf(a, q.z, acc[4 * j + 2]);
          acc[4 * j + 3] = fmaf(a, q.w, acc[4 * j + 3]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if ((j >> 2) < nv) out[o0 + j] = relu ? fmaxf(acc[j], 0.f) : acc[j];
  }
}

// in place: v <- ReLU((v - mean) / sqrt(var + eps)), biased variance
__device__ __forceinline__ void row_ln_relu(float* v, int n) {
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += v[i];
  const float mean = s / float(n);
  float q = 0.f;
  for (int i = 0; i < n; ++i) {
    const float t = v[i] - mean;
    q = fmaf(t, t, q);
  }
  const float inv = 1.0f / sqrtf(q / float(n) + kLnEps);
  for (int i = 0; i < n; ++i) v[i] = fmaxf((v[i] - mean) * inv, 0.f);
}

// Linear -> LayerNorm -> ReLU -> Linear
__device__ __forceinline__ void row_mlp2(const float* in, const Mlp2F32& m, float* hid,
                                         float* out) {
  row_linear(in, m.l1, hid, false);
  row_ln_relu(hid, m.l1.out);
  row_linear(hid, m.l2, out, false);
}

__device__ __forceinline__ void load_row(float* dst, const float* src, int h) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (int c = 0; c < (h >> 2); ++c) {
    const float4 v = s4[c];
    dst[4 * c] = v.x;
    dst[4 * c + 1] = v.y;
    dst[4 * c + 2] = v.z;
    dst[4 * c + 3] = v.w;
  }
}

__device__ __forceinline__ void add_row(float* dst, const float* src, int h) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (int c = 0; c < (h >> 2); ++c) {
    const float4 v = s4[c];
    dst[4 * c] += v.x;
    dst[4 * c + 1] += v.y;
    dst[4 * c + 2] += v.z;
    dst[4 * c + 3] += v.w;
  }
}

// ---------------------------------------------------------------------------
// embedding and node encoder
// ---------------------------------------------------------------------------
struct EmbedLayers {
  LayerF32 l[kMaxEmbedLayers];
};

__global__ void __launch_bounds__(kPrepThreads) k_node_prep_f32(Batch b, Ws w, EmbedLayers em,
                                                                int n_embed, Mlp2F32 ne, int D,
                                                                int h, GraphParams g,
                                                                int stride, int do_embed,
                                                                int do_node_enc, Sel sel) {
  extern __shared__ float smem[];
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(b, w, sel, false, lo, hi)) return;
  float* A = smem + threadIdx.x * stride;
  float* B = smem + (blockDim.x + threadIdx.x) * stride;
  for (int v = lo + blockIdx.x * blockDim.x + threadIdx.x; v < hi;
       v += gridDim.x * blockDim.x) {
    const float4 p = w.pos[v];
    if (do_embed) {
      A[0] = sqrtf(p.x * p.x + p.y * p.y) / g.fs[0];
      A[1] = atan2f(p.y, p.x) / g.fs[1];
      A[2] = p.z / g.fs[2];
      float* in = A;
      float* out = B;
      for (int l = 0; l < n_embed; ++l) {
        row_linear(in, em.l[l], out, l + 1 < n_embed);
        float* t = in;
        in = out;
        out = t;
      }
      for (int d = 0; d < D; ++d) w.emb[size_t(v) * D + d] = in[d];
    }
    if (do_node_enc) {
      A[0] = p.x / g.fs[3];
      A[1] = p.y / g.fs[4];
      A[2] = p.z / g.fs[5];
      row_mlp2(A, ne, B, A);
      float4* dst = reinterpret_cast<float4*>(w.hstate + size_t(v) * h);
      for (int c = 0; c < (h >> 2); ++c)
        dst[c] = make_float4(A[4 * c], A[4 * c + 1], A[4 * c + 2], A[4 * c + 3]);
    }
  }
}

// ---------------------------------------------------------------------------
// edge encoder: e0 = EE([h_src, h_dst])
// ---------------------------------------------------------------------------
__global__ void k_edge_enc_f32(Batch b, Ws w, Mlp2F32 m, int h, int stride, Sel sel) {
  extern __shared__ float smem[];
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(b, w, sel, true, lo, hi)) return;
  float* R = smem + threadIdx.x * stride;  // [2h] input, then output
  float* H = R + 2 * h + 1;                // [h] hidden (stride includes it)
  for (int e = lo + blockIdx.x * blockDim.x + threadIdx.x; e < hi;
       e += gridDim.x * blockDim.x) {
    load_row(R, w.hstate + size_t(w.src[e]) * h, h);
    load_row(R + h, w.hstate + size_t(w.col[e]) * h, h);
    row_mlp2(R, m, H, R);
    float4* dst = reinterpret_cast<float4*>(w.estate + size_t(e) * h);
    for (int c = 0; c < (h >> 2); ++c)
      dst[c] = make_float4(R[4 * c], R[4 * c + 1], R[4 * c + 2], R[4 * c + 3]);
  }
}

// ---------------------------------------------------------------------------
// node update: h <- h + N_k([h, sum_out e, sum_in e])
// ---------------------------------------------------------------------------
__global__ void k_node_upd_f32(Batch b, Ws w, Mlp2F32 m, int h, int stride, Sel sel) {
  extern __shared__ float smem[];
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(b, w, sel, false, lo, hi)) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  float* R = smem + threadIdx.x * stride;  // [3h] input
  float* H = R + 3 * h + 1;                // [h] hidden
  for (int v = lo + blockIdx.x * blockDim.x + threadIdx.x; v < hi;
       v += gridDim.x * blockDim.x) {
    load_row(R, w.hstate + size_t(v) * h, h);
    for (int c = 0; c < 2 * h; ++c) R[h + c] = 0.f;
    const int a = min(w.row_ptr[v], E), z = min(w.row_ptr[v + 1], E);
    for (int e = a; e < z; ++e) add_row(R + h, w.estate + size_t(e) * h, h);
    const int ia = w.in_ptr[v], iz = w.in_ptr[v + 1];
    for (int k = ia; k < iz; ++k) add_row(R + 2 * h, w.estate + size_t(w.in_edge[k]) * h, h);
    row_mlp2(R, m, H, R + h);
    float4* dst = reinterpret_cast<float4*>(w.hstate + size_t(v) * h);
    for (int c = 0; c < (h >> 2); ++c)
      dst[c] = make_float4(R[4 * c] + R[h + 4 * c], R[4 * c + 1] + R[h + 4 * c + 1],
                           R[4 * c + 2] + R[h + 4 * c + 2], R[4 * c + 3] + R[h + 4 * c + 3]);
  }
}

// ---------------------------------------------------------------------------
// edge update: e <- e + E_k([e, h_src, h_dst]); last step: classifier + cut
// ---------------------------------------------------------------------------
__global__ void k_edge_upd_f32(Batch b, Ws w, Mlp2F32 m, Mlp2F32 cls, int has_cls, int h,
                               int stride, float cut, int rescore_only, float band_lo,
                               float band_hi, Sel sel) {
  extern __shared__ float smem[];
  if (input_bad(w)) return;
  int lo, hi;
  if (!sel_rows(b, w, sel, true, lo, hi)) return;
  float* R = smem + threadIdx.x * stride;  // [3h] input
  float* H = R + 3 * h + 1;                // [h] hidden
  for (int e = lo + blockIdx.x * blockDim.x + threadIdx.x; e < hi;
       e += gridDim.x * blockDim.x) {
    load_row(R, w.estate + size_t(e) * h, h);
    if (m.l1.WT != nullptr) {
      load_row(R + h, w.hstate + size_t(w.src[e]) * h, h);
      load_row(R + 2 * h, w.hstate + size_t(w.col[e]) * h, h);
      row_mlp2(R, m, H, R + h);
      for (int c = 0; c < h; ++c) R[c] += R[h + c];
    }
    if (!has_cls) {
      float4* dst = reinterpret_cast<float4*>(w.estate + size_t(e) * h);
      for (int c = 0; c < (h >> 2); ++c)
        dst[c] = make_float4(R[4 * c], R[4 * c + 1], R[4 * c + 2], R[4 * c + 3]);
      continue;
    }
    row_mlp2(R, cls, H, R + h);
    const float lg = R[h];
    if (rescore_only) {
      const float old = w.logit[e];
      if (!(old > band_lo && old < band_hi)) continue;
    }
    w.logit[e] = lg;
    w.keep[e] = lg >= cut ? 1 : 0;
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
  static Entry cache[32];
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
  if (used < 32) cache[used++] = Entry{fn, threads, smem, n};
  return n;
}

// rows per block and shared memory of the interaction-network kernels
int gnn_threads(int h) { return h <= 32 ? 128 : (h <= 64 ? 64 : 32); }

dim3 grid_for(const void* fn, int threads, size_t smem, Sel sel, int64_t rows_hint) {
  const int full = device_sms() * blocks_per_sm(fn, threads, smem);
  if (sel.list != nullptr) return dim3(4, sel.max_list > 0 ? sel.max_list : 1);
  int g = full;
  if (rows_hint >= 0) g = max(1, min(full, div_up(rows_hint, threads)));
  return dim3(g, 1);
}

}  // namespace

void launch_node_prep_f32(const Batch& b, const Ws& w, const LayerF32* embed, int n_embed,
                          const Mlp2F32& node_enc, int D, int h, const GraphParams& g,
                          bool do_embed, bool do_node_enc, Sel sel, cudaStream_t s) {
  if (b.n_hits <= 0) return;
  EmbedLayers em{};
  int width = 3;
  for (int l = 0; l < n_embed; ++l) {
    em.l[l] = embed[l];
    width = max(width, embed[l].ldo);
  }
  width = max(width, h);
  const int stride = width | 1;
  const size_t smem = size_t(2) * kPrepThreads * stride * sizeof(float);
  const dim3 grid = grid_for((const void*)k_node_prep_f32, kPrepThreads, smem, sel, b.n_hits);
  k_node_prep_f32<<<grid, kPrepThreads, smem, s>>>(b, w, em, n_embed, node_enc, D, h, g, stride,
                                                   do_embed, do_node_enc, sel);
}

void launch_edge_enc_f32(const Batch& b, const Ws& w, const Mlp2F32& m, int h, Sel sel,
                         cudaStream_t s) {
  const int T = gnn_threads(h);
  const int stride = (3 * h + 2) | 1;
  const size_t smem = size_t(T) * stride * sizeof(float);
  const dim3 grid = grid_for((const void*)k_edge_enc_f32, T, smem, sel, -1);
  k_edge_enc_f32<<<grid, T, smem, s>>>(b, w, m, h, stride, sel);
}

void launch_node_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, int h, Sel sel,
                            cudaStream_t s) {
  if (b.n_hits <= 0) return;
  const int T = gnn_threads(h);
  const int stride = (4 * h + 2) | 1;
  const size_t smem = size_t(T) * stride * sizeof(float);
  const dim3 grid = grid_for((const void*)k_node_upd_f32, T, smem, sel, b.n_hits);
  k_node_upd_f32<<<grid, T, smem, s>>>(b, w, m, h, stride, sel);
}

void launch_edge_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, const Mlp2F32* cls,
                            int h, float cut_logit, bool rescore_only, float band_lo,
                            float band_hi, Sel sel, cudaStream_t s) {
  const int T = gnn_threads(h);
  const int stride = (4 * h + 2) | 1;
  const size_t smem = size_t(T) * stride * sizeof(float);
  const dim3 grid = grid_for((const void*)k_edge_upd_f32, T, smem, sel, -1);
  Mlp2F32 c{};
  if (cls) c = *cls;
  k_edge_upd_f32<<<grid, T, smem, s>>>(b, w, m, c, cls != nullptr, h, stride, cut_logit,
                                       rescore_only, band_lo, band_hi, sel);
}

}  // namespace gnntrk
