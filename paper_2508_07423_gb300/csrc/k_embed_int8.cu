// INT8 embedding MLP: the thesis's post-training quantisation of the
// embedding (Sec. on MLP quantisation), in the symmetric scheme of its
// quantisation section: x = S x_q, x_q = clip(round(x / S), -127, 127).
//   * every layer's input: one static scale S_a = alpha / 127 per layer, alpha
//     set by calibration (gnntrk_embed_amax gives the max calibration) or left
//     at 1 (uncalibrated);
//   * weights: one scale per output channel, S_w = max |W_row| / 127;
//   * y = (S_a S_w) acc + b with acc the exact INT32 dot product of the codes
//     (dp4a: four INT8 products per instruction), ReLU between layers, the last
//     layer's y (FP32) the embedding coordinate.
// One thread per hit; the thread's input codes stay in registers (4 per
// 32-bit word), the packed weights in shared memory are read as 16-byte
// broadcasts. The max calibration runs the FP32 embedding over a batch and
// keeps the largest |input| of every layer.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/gnntrk.h"
#include "internal.cuh"

namespace gnntrk {

int device_sms();

namespace {

constexpr int kI8Threads = 128;

__device__ __forceinline__ int q8(float v, float inv) {
  const int q = __float2int_rn(v * inv);
  return max(-127, min(127, q));
}

__device__ __forceinline__ uint32_t pack4(int a, int b, int c, int d) {
  return (uint32_t(a) & 0xffu) | ((uint32_t(b) & 0xffu) << 8) | ((uint32_t(c) & 0xffu) << 16) |
         ((uint32_t(d) & 0xffu) << 24);
}

// One layer for this thread's row: x[IN4] packed input codes; writes the
// next layer's packed codes into act (shared, [out4][kI8Threads]) or, for the
// last layer, the FP32 outputs into y_out.
template <int IN4>
__device__ __forceinline__ void i8_layer(const uint32_t (&x)[IN4], const int4* W, const float* s,
                                         const float* b, int out, bool last, float inv_next,
                                         uint32_t* act, float* y_out, int tid) {
  for (int o4 = 0; o4 < out; o4 += 4) {
    int acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (o4 + u >= out) break;
      const int4* wr = W + size_t(o4 + u) * ((IN4 + 3) / 4);
#pragma unroll
      for (int k = 0; k < IN4; k += 4) {
        const int4 w4 = wr[k / 4];
        acc[u] = __dp4a(int(x[k]), w4.x, acc[u]);
        if (k + 1 < IN4) acc[u] = __dp4a(int(x[k + 1]), w4.y, acc[u]);
        if (k + 2 < IN4) acc[u] = __dp4a(int(x[k + 2]), w4.z, acc[u]);
        if (k + 3 < IN4) acc[u] = __dp4a(int(x[k + 3]), w4.w, acc[u]);
      }
    }
    float y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = min(o4 + u, out - 1);
      y[u] = fmaf(float(acc[u]), s[o], b[o]);
    }
    if (last) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (o4 + u < out) y_out[o4 + u] = y[u];
    } else {
      int q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = o4 + u < out ? q8(fmaxf(y[u], 0.f), inv_next) : 0;
      act[(o4 / 4) * kI8Threads + tid] = pack4(q[0], q[1], q[2], q[3]);
    }
  }
}

template <int IN4>
__device__ __forceinline__ void i8_layer_from(const uint32_t* act_in, const int4* W, const float* s,
                                              const float* b, int out, bool last, float inv_next,
                                              uint32_t* act_out, float* y_out, int tid) {
  uint32_t x[IN4];
#pragma unroll
  for (int k = 0; k < IN4; ++k) x[k] = act_in[k * kI8Threads + tid];
  i8_layer<IN4>(x, W, s, b, out, last, inv_next, act_out, y_out, tid);
}

__global__ void __launch_bounds__(kI8Threads) k_embed_int8(Batch b, Ws w, Int8Embed m, int D,
                                                           GraphParams g) {
  extern __shared__ __align__(16) uint8_t smem_i8[];
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;
  const int tid = threadIdx.x;
  // stage weights (int4 rows), scales, biases and activation buffers
  int4* sW[kMaxEmbedLayers];
  float* sS[kMaxEmbedLayers];
  float* sB[kMaxEmbedLayers];
  uint8_t* p = smem_i8;
  for (int l = 0; l < m.n; ++l) {
    const int words = m.l[l].out * m.l[l].in16 * 4;
    sW[l] = reinterpret_cast<int4*>(p);
    for (int i = tid; i < words; i += kI8Threads)
      reinterpret_cast<uint32_t*>(p)[i] = m.l[l].Wq[i];
    p += words * 4;
    sS[l] = reinterpret_cast<float*>(p);
    sB[l] = sS[l] + m.l[l].out;
    for (int i = tid; i < m.l[l].out; i += kI8Threads) {
      sS[l][i] = m.l[l].s[i];
      sB[l][i] = m.l[l].b[i];
    }
    p += ((8 * m.l[l].out + 15) / 16) * 16;
  }
  uint32_t* act0 = reinterpret_cast<uint32_t*>(p);
  uint32_t* act1 = act0 + m.max_in4 * kI8Threads;
  float* inv = reinterpret_cast<float*>(act1 + m.max_in4 * kI8Threads);
  for (int i = tid; i < m.n; i += kI8Threads) inv[i] = m.inv[i];
  __syncthreads();
  for (int base = blockIdx.x * kI8Threads; base < b.n_hits; base += gridDim.x * kI8Threads) {
    const int v = base + tid;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    if (v < b.n_hits) {
      const float4 q = w.pos[v];
      f0 = sqrtf(q.x * q.x + q.y * q.y) / g.fs[0];
      f1 = atan2f(q.y, q.x) / g.fs[1];
      f2 = q.z / g.fs[2];
    }
    float out[16];
    uint32_t x0[1] = {pack4(q8(f0, inv[0]), q8(f1, inv[0]), q8(f2, inv[0]), 0)};
    uint32_t* a_in = act0;
    uint32_t* a_out = act1;
    i8_layer<1>(x0, sW[0], sS[0], sB[0], m.l[0].out, m.n == 1, m.n > 1 ? inv[1] : 1.f, a_in,
                out, tid);
    for (int l = 1; l < m.n; ++l) {
      const bool last = l + 1 == m.n;
      const float inv_next = last ? 1.f : inv[l + 1];
      switch (m.l[l].in4) {
        case 1: i8_layer_from<1>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        case 2: i8_layer_from<2>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        case 4: i8_layer_from<4>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        case 8: i8_layer_from<8>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        case 16: i8_layer_from<16>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        case 32: i8_layer_from<32>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
        default: i8_layer_from<64>(a_in, sW[l], sS[l], sB[l], m.l[l].out, last, inv_next, a_out, out, tid); break;
      }
      uint32_t* t = a_in;
      a_in = a_out;
      a_out = t;
    }
    if (v < b.n_hits)
      for (int d = 0; d < D; ++d) w.emb[size_t(v) * D + d] = out[d];
  }
}

// Max calibration: the FP32 embedding of every input hit, the largest |input|
// of each layer kept as float bits (non-negative floats order like integers).
__global__ void __launch_bounds__(128) k_embed_amax(const float* xyz, int n_hits, EmbedAmax m,
                                                    GraphParams g, int32_t* amax_bits) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  float a[256], c[256];
  float mx[kMaxEmbedLayers];
  for (int l = 0; l < kMaxEmbedLayers; ++l) mx[l] = 0.f;
  if (v < n_hits) {
    const float x = xyz[v], y = xyz[n_hits + v], z = xyz[2 * size_t(n_hits) + v];
    a[0] = sqrtf(x * x + y * y) / g.fs[0];
    a[1] = atan2f(y, x) / g.fs[1];
    a[2] = z / g.fs[2];
    int width = 3;
    for (int l = 0; l < m.n; ++l) {
      const LayerF32& L = m.l[l];
      float t = 0.f;
      for (int k = 0; k < width; ++k) t = fmaxf(t, fabsf(a[k]));
      mx[l] = t;
      for (int o = 0; o < L.out; ++o) {
        float s = L.b[o];
        for (int k = 0; k < L.in; ++k) s = fmaf(a[k], L.WT[size_t(k) * L.ldo + o], s);
        c[o] = l + 1 < m.n ? fmaxf(s, 0.f) : s;
      }
      width = L.out;
      for (int o = 0; o < width; ++o) a[o] = c[o];
    }
  }
  for (int l = 0; l < m.n; ++l) {
    float t = mx[l];
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&amax_bits[l], __float_as_int(t));
  }
}

}  // namespace

size_t embed_int8_smem(const Int8Embed& m) {
  size_t bytes = 0;
  for (int l = 0; l < m.n; ++l)
    bytes += size_t(m.l[l].out) * m.l[l].in16 * 16 + ((8 * m.l[l].out + 15) / 16) * 16;
  bytes += 2 * size_t(m.max_in4) * kI8Threads * 4 + 4 * kMaxEmbedLayers;
  return bytes;
}

void launch_embed_int8(const Batch& b, const Ws& w, const Int8Embed& m, int D,
                       const GraphParams& g, cudaStream_t s) {
  const size_t smem = embed_int8_smem(m);
  {
    // the attribute only grows; handles may launch from several host threads
    static size_t attr = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > attr) {
      cudaFuncSetAttribute(k_embed_int8, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      attr = smem;
    }
  }
  const int grid = std::max(1, std::min(div_up(b.n_hits, kI8Threads), device_sms() * 8));
  k_embed_int8<<<grid, kI8Threads, smem, s>>>(b, w, m, D, g);
}

void launch_embed_amax(const float* xyz, int n_hits, const EmbedAmax& m, const GraphParams& g,
                       int32_t* amax_bits, cudaStream_t s) {
  cudaMemsetAsync(amax_bits, 0, sizeof(int32_t) * kMaxEmbedLayers, s);
  if (n_hits > 0) k_embed_amax<<<div_up(n_hits, 128), 128, 0, s>>>(xyz, n_hits, m, g, amax_bits);
}

}  // namespace gnntrk
