// Tensor-core (tcgen05) kernels of the interaction network: BF16 or FP8-E4M3
// operands, FP32 accumulation in tensor memory.
//
// One CTA of 128 threads works on tiles of 128 rows (edges or hits); thread t
// owns row t of the tile and TMEM lane t (warp w reads lanes 32w..32w+31). Per
// tile:
//   1. gather: each thread copies the pieces of its input row ([e, h_src,
//      h_dst], [h, sum_out e, sum_in e], ...) from global memory into the A
//      tile in shared memory, laid out as 8-row x 16-byte core matrices
//      (K-major, no swizzle: row r, 16-byte chunk c at
//      ((r/8) * (K/epc) + c) * 128 + (r%8) * 16);
//   2. one thread issues the layer-1 MMAs (weights resident in shared memory,
//      loaded once per CTA by cp.async.bulk) and commits them to an mbarrier;
//   3. every thread reads its row of the accumulator back with tcgen05.ld,
//      adds the bias, applies LayerNorm and ReLU and writes the hidden row as
//      the next A tile; layer 2 follows the same way;
//   4. the epilogue adds the residual and stores the new state (BF16); at the
//      last step the edge classifier (a third MMA, LayerNorm, ReLU and a dot
//      product) and the cut run instead of the store.
// FP8: each input segment of layer 1 (e.g. e, h_src, h_dst) is quantised with
// its own per-row scale amax/448 and accumulated in its own TMEM block, so the
// epilogue can apply the scales (the edge steps at hidden 128: h_src and h_dst
// under one scale in one block, layer 1 in three passes, see Layout::P3);
// weights carry per-output-channel scales amax/448. Hidden rows are quantised per row as well. The K = 3 first layer of
// the node encoder and the 1-unit last layer of the classifier stay FP32.
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../include/gnntrk.h"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace gnntrk {

int device_sms();

namespace {

using namespace tc;

constexpr int kRows = 128;       // rows per tile = threads per CTA = TMEM lanes
constexpr long long kWaitCycles = 4000000000LL;  // bounded waits: about 2 s

enum Mode : int { M_NODE_ENC = 0, M_EDGE_ENC = 1, M_NODE_UPD = 2, M_EDGE_UPD = 3,
                  M_EDGE_UPD_CLS = 4, M_CLS = 5, M_TRIP = 6 };

struct TcArgs {
  Batch b;
  Ws w;
  const uint8_t* W1;  // layer-1 operand image (classifier layer 1 in M_CLS)
  const uint8_t* W2;  // layer-2 operand image
  const uint8_t* Wc;  // classifier layer-1 image (M_EDGE_UPD_CLS)
  const float* b1;
  const float* b2;
  const float* bc1;
  const float* s1;    // FP8 per-output-channel weight scales
  const float* s2;
  const float* sc;
  LayerF32 ne1;       // node encoder layer 1 (FP32, M_NODE_ENC)
  LayerF32 c2;        // classifier layer 2 (FP32, h -> 1)
  // M_TRIP: one triplet list (edge pairs, count on the device) and its outputs
  const int32_t* t1;
  const int32_t* t2;
  const int32_t* tn;
  float* tlogit;
  uint8_t* tkeep;
  float fs[6];
  float cut;
};

__host__ __device__ constexpr int n_seg(int mode) {
  return (mode == M_EDGE_ENC || mode == M_TRIP)
             ? 2
             : ((mode == M_NODE_UPD || mode == M_EDGE_UPD || mode == M_EDGE_UPD_CLS) ? 3 : 1);
}
__host__ __device__ constexpr int align1k(int x) { return (x + 1023) & ~1023; }
__host__ __device__ constexpr int pow2_cols(int x) {
  return x <= 32 ? 32 : (x <= 64 ? 64 : (x <= 128 ? 128 : (x <= 256 ? 256 : 512)));
}

// Shared-memory layout of one CTA (byte offsets).
template <int H, bool FP8, int MODE>
struct Layout {
  static constexpr int ESZ = FP8 ? 1 : 2;
  static constexpr int NSEG = n_seg(MODE);
  // BF16 encoders carry the node encoding at about 16 significant bits: an
  // operand x enters the MMA as hi = bf16(x) and lo = bf16(x - hi) over a K
  // twice as long, against the weight image repeated along K (node encoder
  // layer 2: its hidden row; edge encoder layer 1: the FP32 rows h_src, h_dst).
  // The encoders see hit coordinates, whose useful precision (a 12 um
  // resolution over a 45 mm radius) is finer than BF16's 8-bit mantissa.
  static constexpr bool SPLIT = !FP8 && (MODE == M_NODE_ENC || MODE == M_EDGE_ENC);
  // at hidden 128 the split edge encoder runs layer 1 in two passes over one
  // [h_src, h_dst] tile (hi parts, then lo parts accumulated into the same
  // tensor memory) against the plain weight image, so it fits shared memory
  static constexpr bool SPLIT2 = SPLIT && MODE == M_EDGE_ENC && H > 64;
  // FP8 edge steps at hidden 128 run layer 1 in three passes of K = H over a
  // one-segment tile (e, then h_src, then h_dst) against the K chunks of the
  // weight image; h_src and h_dst share one per-row scale and accumulate into
  // one tensor-memory block (e into the other), so that the tiles (86 KB)
  // and the accumulators (256 columns) of two CTAs fit an SM
  static constexpr bool P3 = FP8 && H == 128 && (MODE == M_EDGE_UPD || MODE == M_EDGE_UPD_CLS);
  static constexpr int K1 = (MODE == M_NODE_ENC) ? H : (SPLIT && !SPLIT2 ? 2 : 1) * NSEG * H;
  static constexpr int K2 = (SPLIT && MODE == M_NODE_ENC) ? 2 * H : H;
  static constexpr bool HAS_W1 = MODE != M_NODE_ENC;
  static constexpr bool HAS_W2 = MODE != M_CLS && MODE != M_TRIP;
  static constexpr bool HAS_WC = MODE == M_EDGE_UPD_CLS;
  static constexpr int W1 = 0;
  static constexpr int W1_BYTES = HAS_W1 ? H * K1 * ESZ : 0;
  static constexpr int W2 = align1k(W1 + W1_BYTES);
  static constexpr int W2_BYTES = HAS_W2 ? H * K2 * ESZ : 0;
  static constexpr int WC = align1k(W2 + W2_BYTES);
  static constexpr int WC_BYTES = HAS_WC ? H * H * ESZ : 0;
  // BF16 node-step tiles ([h, m_out, m_in], contiguous rows) are gathered by
  // coalesced cp.async copies; with PREFETCH into two alternating layer-1
  // input buffers (tile t + 1 loads while tile t computes). Edge tiles keep
  // the per-row copies: on the 1000-event batch they measured faster than
  // cp.async (single or double buffered) and than conflict-free coalesced
  // copies through registers (2.27 ms against 2.59-3.12 ms per 4 launches).
  static constexpr bool PIPE = !FP8 && MODE == M_NODE_UPD;
  static constexpr bool PREFETCH = false;
  static constexpr int A = align1k(WC + WC_BYTES);
  static constexpr int A_BYTES = MODE == M_NODE_ENC ? 0 : kRows * (P3 ? H : K1) * ESZ;
  static constexpr int NBUF = PIPE && PREFETCH ? 2 : 1;
  // hidden / classifier input: its own tile with two input buffers, else it
  // overwrites the layer-1 input once the layer-1 MMAs are done
  static constexpr int HA = NBUF == 2 || MODE == M_NODE_ENC ? align1k(A + NBUF * A_BYTES) : A;
  static constexpr int HA_BYTES = NBUF == 2 || MODE == M_NODE_ENC ? kRows * K2 * ESZ : 0;
  static constexpr int PAR = align1k(HA_BYTES > 0 ? HA + HA_BYTES : A + NBUF * A_BYTES);
  // fp32 parameters: b1, b2, bc1, s1, s2, sc, c2 weights, ne1 (3 x H + H)
  static constexpr int PAR_FLOATS = 7 * H + 4 * H + 8;
  static constexpr int BAR = PAR + PAR_FLOATS * 4;
  static constexpr int TOTAL = BAR + 64;
  // FP8: one accumulator block per layer-1 segment scale
  static constexpr int TSEG = P3 ? 2 : (FP8 ? NSEG : 1);
  static constexpr int TMEM_COLS = pow2_cols(TSEG * H);
};

__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

// byte offset of (row, 16-byte chunk) in a canonical tile with `kchunks`
// chunks per row
__device__ __forceinline__ uint32_t tile_off(int row, int chunk, int kchunks) {
  return uint32_t(((row >> 3) * kchunks + chunk) * 128 + (row & 7) * 16);
}

// Write `n` (multiple of 16 for FP8, of 8 for BF16) FP32 values of this
// thread's row into the A tile starting at element k0, scaled by `inv` for FP8.
template <bool FP8>
__device__ __forceinline__ void put_row_f32(uint8_t* tile, int row, int kchunks, int k0,
                                            const float* v, int n, float inv) {
  if constexpr (FP8) {
    for (int c = 0; c < n / 16; ++c) {
      const float* q = v + 16 * c;
      uint4 u;
      u.x = pack_e4m3x4(q[0] * inv, q[1] * inv, q[2] * inv, q[3] * inv);
      u.y = pack_e4m3x4(q[4] * inv, q[5] * inv, q[6] * inv, q[7] * inv);
      u.z = pack_e4m3x4(q[8] * inv, q[9] * inv, q[10] * inv, q[11] * inv);
      u.w = pack_e4m3x4(q[12] * inv, q[13] * inv, q[14] * inv, q[15] * inv);
      *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 4) + c, kchunks)) = u;
    }
  } else {
    for (int c = 0; c < n / 8; ++c) {
      const float* q = v + 8 * c;
      uint4 u;
      u.x = pack_bf16(q[0], q[1]);
      u.y = pack_bf16(q[2], q[3]);
      u.z = pack_bf16(q[4], q[5]);
      u.w = pack_bf16(q[6], q[7]);
      *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 3) + c, kchunks)) = u;
    }
  }
}

// Copy one BF16 row of H values from global memory into the A tile (BF16) or
// quantise it (FP8, per-row scale returned). `keep` receives the raw row when
// not null.
template <int H, bool FP8>
__device__ __forceinline__ float put_row_bf16(uint8_t* tile, int row, int kchunks, int k0,
                                              const __nv_bfloat16* src, uint4* keep) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  if constexpr (!FP8) {
#pragma unroll
    for (int c = 0; c < H / 8; ++c) {
      const uint4 u = s4[c];
      if (keep) keep[c] = u;
      *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 3) + c, kchunks)) = u;
    }
    return 1.0f;
  } else {
    uint4 r[H / 8];
    float amax = 0.f;
#pragma unroll
    for (int c = 0; c < H / 8; ++c) {
      r[c] = s4[c];
      if (keep) keep[c] = r[c];
      const uint32_t q[4] = {r[c].x, r[c].y, r[c].z, r[c].w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        amax = fmaxf(amax, fmaxf(fabsf(bf16_lo(q[j])), fabsf(bf16_hi(q[j]))));
    }
    const float scale = amax > 0.f ? amax / 448.f : 1.f;
    const float inv = amax > 0.f ? 448.f / amax : 1.f;
#pragma unroll
    for (int c = 0; c < H / 16; ++c) {
      const uint4 a = r[2 * c], b = r[2 * c + 1];
      uint4 u;
      u.x = pack_e4m3x4(bf16_lo(a.x) * inv, bf16_hi(a.x) * inv, bf16_lo(a.y) * inv, bf16_hi(a.y) * inv);
      u.y = pack_e4m3x4(bf16_lo(a.z) * inv, bf16_hi(a.z) * inv, bf16_lo(a.w) * inv, bf16_hi(a.w) * inv);
      u.z = pack_e4m3x4(bf16_lo(b.x) * inv, bf16_hi(b.x) * inv, bf16_lo(b.y) * inv, bf16_hi(b.y) * inv);
      u.w = pack_e4m3x4(bf16_lo(b.z) * inv, bf16_hi(b.z) * inv, bf16_lo(b.w) * inv, bf16_hi(b.w) * inv);
      *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 4) + c, kchunks)) = u;
    }
    return scale;
  }
}

// One BF16 row of H values from global memory into an E4M3 tile at element
// k0, each value multiplied by `inv` (the caller's per-row scale).
template <int H>
__device__ __forceinline__ void put_row_bf16_e4m3(uint8_t* tile, int row, int kchunks, int k0,
                                                  const __nv_bfloat16* src, float inv) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int c = 0; c < H / 16; ++c) {
    const uint4 a = s4[2 * c], b = s4[2 * c + 1];
    uint4 u;
    u.x = pack_e4m3x4(bf16_lo(a.x) * inv, bf16_hi(a.x) * inv, bf16_lo(a.y) * inv, bf16_hi(a.y) * inv);
    u.y = pack_e4m3x4(bf16_lo(a.z) * inv, bf16_hi(a.z) * inv, bf16_lo(a.w) * inv, bf16_hi(a.w) * inv);
    u.z = pack_e4m3x4(bf16_lo(b.x) * inv, bf16_hi(b.x) * inv, bf16_lo(b.y) * inv, bf16_hi(b.y) * inv);
    u.w = pack_e4m3x4(bf16_lo(b.z) * inv, bf16_hi(b.z) * inv, bf16_lo(b.w) * inv, bf16_hi(b.w) * inv);
    *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 4) + c, kchunks)) = u;
  }
}

// Write n FP32 values (a multiple of 8) into a BF16 tile as two parts, hi =
// bf16(v) at element k_hi and lo = bf16(v - hi) at element k_lo.
__device__ __forceinline__ void put_row_split(uint8_t* tile, int row, int kchunks, int k_hi,
                                              int k_lo, const float* v, int n) {
  for (int c = 0; c < n / 8; ++c) {
    const float* q = v + 8 * c;
    float r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = q[j] - __bfloat162float(__float2bfloat16_rn(q[j]));
    *reinterpret_cast<uint4*>(tile + tile_off(row, (k_hi >> 3) + c, kchunks)) =
        make_uint4(pack_bf16(q[0], q[1]), pack_bf16(q[2], q[3]), pack_bf16(q[4], q[5]),
                   pack_bf16(q[6], q[7]));
    *reinterpret_cast<uint4*>(tile + tile_off(row, (k_lo >> 3) + c, kchunks)) =
        make_uint4(pack_bf16(r[0], r[1]), pack_bf16(r[2], r[3]), pack_bf16(r[4], r[5]),
                   pack_bf16(r[6], r[7]));
  }
}

// One FP32 row of H values from global memory into a BF16 tile, split as above.
template <int H>
__device__ __forceinline__ void put_row_f32_split(uint8_t* tile, int row, int kchunks, int k_hi,
                                                  int k_lo, const float* src) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int c = 0; c < H / 8; ++c) {
    const float4 a = s4[2 * c], b = s4[2 * c + 1];
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    put_row_split(tile, row, kchunks, k_hi + 8 * c, k_lo + 8 * c, v, 8);
  }
}

// One FP32 row of H values into a BF16 tile at element k0: its hi parts
// bf16(v) (lo = false) or its lo parts bf16(v - bf16(v)) (lo = true).
template <int H>
__device__ __forceinline__ void put_row_f32_part(uint8_t* tile, int row, int kchunks, int k0,
                                                 const float* src, bool lo) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int c = 0; c < H / 8; ++c) {
    const float4 a = s4[2 * c], b = s4[2 * c + 1];
    float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    if (lo) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] -= __bfloat162float(__float2bfloat16_rn(v[j]));
    }
    *reinterpret_cast<uint4*>(tile + tile_off(row, (k0 >> 3) + c, kchunks)) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                   pack_bf16(v[6], v[7]));
  }
}

template <int H>
__device__ __forceinline__ void add_bf16_row(float* acc, const __nv_bfloat16* src) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int c = 0; c < H / 8; ++c) {
    const uint4 u = s4[c];
    acc[8 * c + 0] += bf16_lo(u.x);
    acc[8 * c + 1] += bf16_hi(u.x);
    acc[8 * c + 2] += bf16_lo(u.y);
    acc[8 * c + 3] += bf16_hi(u.y);
    acc[8 * c + 4] += bf16_lo(u.z);
    acc[8 * c + 5] += bf16_hi(u.z);
    acc[8 * c + 6] += bf16_lo(u.w);
    acc[8 * c + 7] += bf16_hi(u.w);
  }
}

// x[j] = v[j] + b[j] (BF16) or fma(v[j], sc[j], b[j]) (FP8) for 32 columns,
// the parameters read as 16-byte broadcasts from shared memory
template <bool FP8>
__device__ __forceinline__ void add_params(const float (&v)[32], const float* b, const float* sc,
                                           float (&x)[32]) {
  const float4* b4 = reinterpret_cast<const float4*>(b);
  const float4* s4 = reinterpret_cast<const float4*>(sc);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 bb = b4[q];
    if constexpr (FP8) {
      const float4 ss = s4[q];
      x[4 * q] = fmaf(v[4 * q], ss.x, bb.x);
      x[4 * q + 1] = fmaf(v[4 * q + 1], ss.y, bb.y);
      x[4 * q + 2] = fmaf(v[4 * q + 2], ss.z, bb.z);
      x[4 * q + 3] = fmaf(v[4 * q + 3], ss.w, bb.w);
    } else {
      x[4 * q] = v[4 * q] + bb.x;
      x[4 * q + 1] = v[4 * q + 1] + bb.y;
      x[4 * q + 2] = v[4 * q + 2] + bb.z;
      x[4 * q + 3] = v[4 * q + 3] + bb.w;
    }
  }
}

// Issue the MMAs of one layer: A tile (kchunks 16-byte chunks per row) times
// the weight image (H rows) over K elements. FP8 with segments: segment s
// (H columns of K) accumulates into TMEM columns [s*H, (s+1)*H).
template <int H, bool FP8>
__device__ __forceinline__ void issue_layer(uint32_t tmem, const uint8_t* A, const uint8_t* W,
                                            int K, int nseg_sep, bool accumulate = false) {
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int KSTEP = FP8 ? 32 : 16;
  constexpr uint32_t IDESC = FP8 ? idesc_e4m3(kRows, H) : idesc_bf16(kRows, H);
  const int kchunks = K * ESZ / 16;
  const uint32_t sbo = uint32_t(kchunks) * 128;
  const uint32_t a0 = smem_u32(A), w0 = smem_u32(W);
  const int seg_len = nseg_sep > 1 ? K / nseg_sep : K;
  for (int k = 0; k < K; k += KSTEP) {
    const int seg = k / seg_len;
    const uint32_t byte_k = uint32_t(k * ESZ / 16) * 128;  // chunk index * 128
    const uint64_t ad = smem_desc(a0 + byte_k, 128, sbo);
    const uint64_t bd = smem_desc(w0 + byte_k, 128, sbo);
    const uint32_t d = tmem + uint32_t(nseg_sep > 1 ? seg * H : 0);
    const uint32_t acc = accumulate || (k % seg_len) != 0;
    if constexpr (FP8)
      mma_e4m3(d, ad, bd, IDESC, acc);
    else
      mma_bf16(d, ad, bd, IDESC, acc);
  }
}

// One pass of a three-pass FP8 layer 1 (K = 3H): the one-segment A tile
// (E4M3, H per row) times K chunk `pass` of the weight image (E4M3, 3H per
// row); pass 0 starts its accumulator, pass 1 starts the other, pass 2 adds
// to it.
template <int H>
__device__ __forceinline__ void issue_pass_e4m3(uint32_t tmem, const uint8_t* A, const uint8_t* W,
                                                int pass) {
  constexpr uint32_t IDESC = idesc_e4m3(kRows, H);
  constexpr uint32_t SBO_A = uint32_t(H / 16) * 128;
  constexpr uint32_t SBO_W = uint32_t(3 * H / 16) * 128;
  const uint32_t a0 = smem_u32(A), w0 = smem_u32(W) + uint32_t(pass * (H / 16)) * 128;
#pragma unroll
  for (int k = 0; k < H; k += 32) {
    const uint32_t byte_k = uint32_t(k / 16) * 128;
    mma_e4m3(tmem, smem_desc(a0 + byte_k, 128, SBO_A), smem_desc(w0 + byte_k, 128, SBO_W), IDESC,
             (pass == 2 || k > 0) ? 1u : 0u);
  }
}

// Copy slot l (0 .. H/8 - 1) of thread tid in a tile copy: warp w covers rows
// 32w .. 32w+31; a quarter-warp (8 lanes) takes one 16-byte chunk of 8
// consecutive rows, a contiguous 128-byte run of the canonical tile, so the
// shared-memory stores are conflict-free, and a warp instruction reads 8 rows
// x 4 chunks.
template <int CH>
__device__ __forceinline__ void copy_slot(int tid, int l, int& rr, int& c) {
  const int warp = tid >> 5, lane = tid & 31;
  const int g = l % 4, cq = l / 4;  // row group of 8, chunk quad
  rr = warp * 32 + g * 8 + (lane & 7);
  c = cq * 4 + (lane >> 3);
}

// Issue the cp.async copies of one BF16 tile's layer-1 input (rows row0 ..
// row0 + 127; rows at or past `hi` are zero-filled): segment s of row r, chunk
// c (16 bytes) lands at tile_off(r, s * H/8 + c). Consecutive threads take the
// chunks of one row, so a warp reads 8 rows x H*2 bytes per segment.
template <int H, int MODE>
__device__ __forceinline__ void gather_async(uint8_t* dst, const TcArgs& p, int row0, int hi,
                                             int tid) {
  constexpr int CH = H / 8;
  constexpr int NSEG = n_seg(MODE);
  constexpr int KCH = NSEG * CH;
  const Ws& w = p.w;
  const __nv_bfloat16* msg16 = reinterpret_cast<const __nv_bfloat16*>(w.pstate);
#pragma unroll
  for (int l = 0; l < CH; ++l) {
    int rr, c;
    copy_slot<CH>(tid, l, rr, c);
    const int r = row0 + rr;
    const uint32_t n = r < hi ? 16u : 0u;
    const int rs = r < hi ? r : 0;
    const __nv_bfloat16* src[3];
    if constexpr (MODE == M_NODE_UPD) {
      src[0] = w.hstate16 + size_t(rs) * H;
      src[1] = msg16 + size_t(rs) * 2 * H;
      src[2] = src[1] + H;
    } else if constexpr (MODE == M_EDGE_ENC) {
      src[0] = w.hstate16 + size_t(w.src[rs]) * H;
      src[1] = w.hstate16 + size_t(w.col[rs]) * H;
    } else if constexpr (MODE == M_CLS) {
      src[0] = w.estate16 + size_t(rs) * H;
    } else {
      src[0] = w.estate16 + size_t(rs) * H;
      src[1] = w.hstate16 + size_t(w.src[rs]) * H;
      src[2] = w.hstate16 + size_t(w.col[rs]) * H;
    }
#pragma unroll
    for (int sg = 0; sg < NSEG; ++sg) cp_async16(dst + tile_off(rr, sg * CH + c, KCH), src[sg] + 8 * c, n);
  }
}

template <int H, bool FP8, int MODE>
__global__ void __launch_bounds__(kRows, 1) k_tc(const TcArgs p) {
  using L = Layout<H, FP8, MODE>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sW1 = smem + L::W1;
  uint8_t* sW2 = smem + L::W2;
  uint8_t* sWC = smem + L::WC;
  float* par = reinterpret_cast<float*>(smem + L::PAR);
  float* pb1 = par;
  float* pb2 = par + H;
  float* pbc = par + 2 * H;
  float* ps1 = par + 3 * H;
  float* ps2 = par + 4 * H;
  float* psc = par + 5 * H;
  float* pc2 = par + 6 * H;      // classifier layer 2 weights [H] + bias
  float* pne = par + 7 * H + 4;  // node encoder layer 1: W[3][H], b[H]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);  // [0] weights, [1] mma
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::BAR + 16);

  const int tid = threadIdx.x, warp = tid >> 5;
  const Ws& w = p.w;
  // (the triplet lists are only valid when the triplet workspace held them)
  if (*(volatile int32_t*)&w.counters[C_STATUS] & (MODE == M_TRIP ? (ST_INPUT | ST_CAPACITY) : ST_INPUT))
    return;

  // ---- set-up: barriers, TMEM, weights --------------------------------------
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, L::TMEM_COLS);
    tmem_relinquish();
  }
  for (int i = tid; i < H; i += kRows) {
    pb1[i] = MODE == M_NODE_ENC ? p.ne1.b[i] : (MODE == M_CLS ? p.bc1[i] : p.b1[i]);
    pb2[i] = (MODE == M_CLS || MODE == M_TRIP) ? 0.f : p.b2[i];
    pbc[i] = (MODE == M_EDGE_UPD_CLS) ? p.bc1[i] : 0.f;
    if constexpr (FP8) {
      ps1[i] = MODE == M_NODE_ENC ? 1.f : (MODE == M_CLS ? p.sc[i] : p.s1[i]);
      ps2[i] = (MODE == M_CLS || MODE == M_TRIP) ? 1.f : p.s2[i];
      psc[i] = (MODE == M_EDGE_UPD_CLS) ? p.sc[i] : 1.f;
    }
    if (MODE == M_EDGE_UPD_CLS || MODE == M_CLS || MODE == M_TRIP) pc2[i] = p.c2.WT[i * p.c2.ldo];
    if (MODE == M_NODE_ENC) {
      for (int j = 0; j < 3; ++j) pne[j * H + i] = p.ne1.WT[j * p.ne1.ldo + i];
      pne[3 * H + i] = p.ne1.b[i];
    }
  }
  if (tid == 0 && (MODE == M_EDGE_UPD_CLS || MODE == M_CLS || MODE == M_TRIP)) pc2[H] = p.c2.b[0];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const uint32_t tmem_lane = tmem_base + (uint32_t(warp * 32) << 16);

  if (tid == 0) {
    uint32_t bytes = uint32_t(L::W1_BYTES + L::W2_BYTES + L::WC_BYTES);
    mbar_expect_tx(&bar[0], bytes);
    if (L::HAS_W1) bulk_g2s(sW1, MODE == M_CLS ? p.Wc : p.W1, L::W1_BYTES, &bar[0]);
    if (L::HAS_W2) bulk_g2s(sW2, p.W2, L::W2_BYTES, &bar[0]);
    if (L::HAS_WC) bulk_g2s(sWC, p.Wc, L::WC_BYTES, &bar[0]);
  }
  bool ok = mbar_wait_bounded(&bar[0], 0, kWaitCycles);
  uint32_t mma_phase = 0;
  bool mma_pending = false;  // an MMA commit not yet waited for
  const bool weights_late = __syncthreads_or(!ok);
  bool aborted = weights_late;

  const bool edge_rows = MODE != M_NODE_ENC && MODE != M_NODE_UPD;
  int lo = 0, hi = 0;
  {
    const Batch& b = p.b;
    hi = edge_rows ? clamp_edges(w.counters, w.e_cap) : b.n_hits;
    if constexpr (MODE == M_TRIP) hi = min(*p.tn, int(w.t_cap));
  }
  const int n_tiles = (hi - lo + kRows - 1) / kRows;
  constexpr int K1 = L::K1;
  constexpr int KCH1 = K1 * L::ESZ / 16;  // 16-byte chunks per A row, layer 1
  constexpr int KCHA = L::P3 ? H * L::ESZ / 16 : KCH1;  // per row of the A tile
  constexpr int KCHH = H * L::ESZ / 16;   // 16-byte chunks per A row, K = H
  constexpr int KCH2 = L::K2 * L::ESZ / 16;  // 16-byte chunks per A row, layer 2

  // wait for the MMAs committed so far; false on timeout (uniform across CTA)
  auto wait_mma = [&]() -> bool {
    mma_pending = true;
    bool good = mbar_wait_bounded(&bar[1], mma_phase, kWaitCycles);
    tc_fence_after();
    if (__syncthreads_or(!good)) return false;
    mma_phase ^= 1;
    mma_pending = false;
    return true;
  };

  if constexpr (L::PIPE && L::PREFETCH) {
    if (int(blockIdx.x) < n_tiles && !aborted)
      gather_async<H, MODE>(smem + L::A, p, lo + int(blockIdx.x) * kRows, hi, tid);
    cp_async_commit();
  }
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles && !aborted; t += gridDim.x, ++it) {
    const int r = lo + t * kRows + tid;
    const bool valid = r < hi;
    uint8_t* sA = smem + L::A + (L::NBUF == 2 ? (it & 1) * L::A_BYTES : 0);
    uint8_t* sHA = L::HA == L::A ? sA : smem + L::HA;  // layer-2 input and classifier input
    float sa[3] = {1.f, 1.f, 1.f};  // FP8 per-row scales of the layer-1 segments
    uint4 keep_row[(H <= 64) ? H / 8 : 1];
    (void)keep_row;

    // ---- 1. gather ---------------------------------------------------------
    if constexpr (L::PIPE && L::PREFETCH) {
      // every thread is done with the other buffer (tile it - 1): fill it with
      // the next tile, then wait for this tile's copies
      __syncthreads();
      const int tn = t + int(gridDim.x);
      if (tn < n_tiles)
        gather_async<H, MODE>(smem + L::A + ((it + 1) & 1) * L::A_BYTES, p, lo + tn * kRows, hi, tid);
      cp_async_commit();
      cp_async_wait<1>();
    } else if constexpr (L::PIPE) {
      __syncthreads();  // every thread is done with the buffer (tile it - 1)
      gather_async<H, MODE>(sA, p, lo + t * kRows, hi, tid);
      cp_async_commit();
      cp_async_wait<0>();
    } else if constexpr (MODE == M_NODE_ENC) {
      // FP32 first layer (K = 3) in registers, then LayerNorm + ReLU into A
      float hid[H];
      if (valid) {
        const float4 q = w.pos[r];
        const float f0 = q.x / p.fs[3], f1 = q.y / p.fs[4], f2 = q.z / p.fs[5];
#pragma unroll
        for (int i = 0; i < H; ++i) {
          float a = pne[3 * H + i];
          a = fmaf(f0, pne[i], a);
          a = fmaf(f1, pne[H + i], a);
          a = fmaf(f2, pne[2 * H + i], a);
          hid[i] = a;
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) s += hid[i];
        const float mean = s / float(H);
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) {
          const float d = hid[i] - mean;
          v = fmaf(d, d, v);
        }
        const float inv = 1.0f / sqrtf(v / float(H) + kLnEps);
        float amax = 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) {
          hid[i] = fmaxf((hid[i] - mean) * inv, 0.f);
          amax = fmaxf(amax, hid[i]);
        }
        sa[0] = FP8 ? (amax > 0.f ? amax / 448.f : 1.f) : 1.f;
        if constexpr (L::SPLIT)
          put_row_split(sHA, tid, KCH2, 0, H, hid, H);
        else
          put_row_f32<FP8>(sHA, tid, KCHH, 0, hid, H, FP8 ? (amax > 0.f ? 448.f / amax : 1.f) : 1.f);
      } else {
#pragma unroll
        for (int i = 0; i < H; ++i) hid[i] = 0.f;
        for (int k = 0; k < L::K2; k += H) put_row_f32<FP8>(sHA, tid, KCH2, k, hid, H, 1.f);
      }
    } else if constexpr (MODE == M_NODE_UPD) {
      if (valid) {
        sa[0] = put_row_bf16<H, FP8>(sA, tid, KCH1, 0, w.hstate16 + size_t(r) * H,
                                     H <= 64 ? keep_row : nullptr);
        // the message sums [sum_out e, sum_in e] (FP32, written by k_msg_bf16
        // into the node's projection row)
        const float4* m4 = reinterpret_cast<const float4*>(w.pstate + size_t(r) * 2 * H);
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          float acc[H];
#pragma unroll
          for (int i = 0; i < H / 4; ++i) {
            const float4 v = m4[side * (H / 4) + i];
            acc[4 * i] = v.x;
            acc[4 * i + 1] = v.y;
            acc[4 * i + 2] = v.z;
            acc[4 * i + 3] = v.w;
          }
          float amax = 0.f;
          if constexpr (FP8) {
#pragma unroll
            for (int i = 0; i < H; ++i) amax = fmaxf(amax, fabsf(acc[i]));
          }
          sa[1 + side] = FP8 ? (amax > 0.f ? amax / 448.f : 1.f) : 1.f;
          put_row_f32<FP8>(sA, tid, KCH1, (1 + side) * H, acc, H,
                           FP8 ? (amax > 0.f ? 448.f / amax : 1.f) : 1.f);
        }
      } else {
        float z[16] = {};
        for (int k = 0; k < K1; k += 16) put_row_f32<FP8>(sA, tid, KCH1, k, z, 16, 1.f);
      }
    } else {
      // edge rows: [e], [h_src, h_dst], [e, h_src, h_dst]
      if (valid) {
        int seg = 0;
        if constexpr (MODE == M_TRIP) {
          // [e^K(first edge), e^K(second edge)]
          sa[0] = put_row_bf16<H, FP8>(sA, tid, KCH1, 0, w.estate16 + size_t(p.t1[r]) * H, nullptr);
          sa[1] = put_row_bf16<H, FP8>(sA, tid, KCH1, H, w.estate16 + size_t(p.t2[r]) * H, nullptr);
          seg = 2;
        } else if constexpr (MODE == M_EDGE_UPD || MODE == M_EDGE_UPD_CLS || MODE == M_CLS) {
          sa[0] = put_row_bf16<H, FP8>(sA, tid, KCHA, 0, w.estate16 + size_t(r) * H,
                                       (H <= 64 && MODE != M_CLS) ? keep_row : nullptr);
          seg = 1;
        }
        if constexpr (L::P3) {
          // pass 0 holds e alone; h_src and h_dst follow in passes 1 and 2
          // with one scale, the larger of their two row maxima
          // (the node kernels store each row's maximum as they write it)
          const float amax = fmaxf(w.hamax[w.src[r]], w.hamax[w.col[r]]);
          sa[1] = amax > 0.f ? amax / 448.f : 1.f;
        } else if constexpr (L::SPLIT2) {
          // pass 1: [hi(h_src), hi(h_dst)] (the lo parts follow after the MMA)
          put_row_f32_part<H>(sA, tid, KCH1, 0, w.hstate + size_t(w.src[r]) * H, false);
          put_row_f32_part<H>(sA, tid, KCH1, H, w.hstate + size_t(w.col[r]) * H, false);
        } else if constexpr (L::SPLIT) {
          // [hi(h_src), hi(h_dst), lo(h_src), lo(h_dst)] from the FP32 encodings
          put_row_f32_split<H>(sA, tid, KCH1, 0, 2 * H, w.hstate + size_t(w.src[r]) * H);
          put_row_f32_split<H>(sA, tid, KCH1, H, 3 * H, w.hstate + size_t(w.col[r]) * H);
        } else if constexpr (MODE != M_CLS && MODE != M_TRIP) {
          sa[seg] = put_row_bf16<H, FP8>(sA, tid, KCH1, seg * H, w.hstate16 + size_t(w.src[r]) * H,
                                         nullptr);
          sa[seg + 1] = put_row_bf16<H, FP8>(sA, tid, KCH1, (seg + 1) * H,
                                             w.hstate16 + size_t(w.col[r]) * H, nullptr);
        }
      } else {
        float z[16] = {};
        for (int k = 0; k < (L::P3 ? H : K1); k += 16) put_row_f32<FP8>(sA, tid, KCHA, k, z, 16, 1.f);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();

    float hid_scale = 1.f;  // FP8 per-row scale of the layer-2 input
    if constexpr (MODE != M_NODE_ENC) {
      // ---- 2. layer 1 ------------------------------------------------------
      if (tid == 0) {
        tc_fence_after();
        if constexpr (L::P3)
          issue_pass_e4m3<H>(tmem_base, sA, sW1, 0);
        else
          issue_layer<H, FP8>(tmem_base, sA, sW1, K1, FP8 ? L::NSEG : 1);
        mma_commit(&bar[1]);
      }
      if (!wait_mma()) {
        aborted = true;
        break;
      }
      if constexpr (L::P3) {
        // passes 1 and 2: h_src, then h_dst, into the same tile (the MMAs of
        // the pass before have read it); invalid rows keep pass 0's zeros
        const float hinv = 1.f / sa[1];
        for (int pass = 1; pass <= 2 && !aborted; ++pass) {
          if (valid)
            put_row_bf16_e4m3<H>(sA, tid, KCHA, 0,
                                 w.hstate16 + size_t(pass == 1 ? w.src[r] : w.col[r]) * H, hinv);
          fence_proxy_async();
          tc_fence_before();
          __syncthreads();
          if (tid == 0) {
            tc_fence_after();
            issue_pass_e4m3<H>(tmem_base + uint32_t(H), sA, sW1, pass);
            mma_commit(&bar[1]);
          }
          if (!wait_mma()) aborted = true;
        }
        if (aborted) break;
      }
      if constexpr (L::SPLIT2) {
        // pass 2: [lo(h_src), lo(h_dst)] into the same tile, accumulated
        if (valid) {
          put_row_f32_part<H>(sA, tid, KCH1, 0, w.hstate + size_t(w.src[r]) * H, true);
          put_row_f32_part<H>(sA, tid, KCH1, H, w.hstate + size_t(w.col[r]) * H, true);
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc_fence_after();
          issue_layer<H, FP8>(tmem_base, sA, sW1, K1, 1, true);
          mma_commit(&bar[1]);
        }
        if (!wait_mma()) {
          aborted = true;
          break;
        }
      }
      if constexpr (L::PIPE && L::HA == L::A) {
        // the hidden tile overwrites the layer-1 input: keep this row's
        // residual segment in registers first
        if constexpr (MODE == M_NODE_UPD || MODE == M_EDGE_UPD || MODE == M_EDGE_UPD_CLS) {
#pragma unroll
          for (int c = 0; c < H / 8; ++c)
            keep_row[c] = *reinterpret_cast<const uint4*>(sA + tile_off(tid, c, KCH1));
        }
        __syncthreads();
      }
      // ---- 3. bias + LayerNorm + ReLU (-> A as the next operand, or the
      //         classifier output for M_CLS) -------------------------------
      // x[n] = s_w[n] * sum_seg s_a[seg] * acc_seg[n] + b[n]  (FP8)
      //      = acc[n] + b[n]                                   (BF16)
      auto xval_ld = [&](int c, float (&x)[32]) {
        float v[32];
        tmem_ld32(tmem_lane + uint32_t(c * 32), v);
        if constexpr (FP8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] *= sa[0];
#pragma unroll
          for (int s = 1; s < L::TSEG; ++s) {
            float u[32];
            tmem_ld32(tmem_lane + uint32_t(s * H + c * 32), u);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fmaf(u[j], sa[s], v[j]);
          }
        }
        tmem_wait_ld();
        add_params<FP8>(v, pb1 + c * 32, ps1 + c * 32, x);
      };
      // h = 32: one chunk, read from tensor memory once and kept in registers
      float xc[H == 32 ? 32 : 1];
      if constexpr (H == 32) xval_ld(0, xc);
      auto xval = [&](int c, float (&x)[32]) {
        if constexpr (H == 32) {
#pragma unroll
          for (int j = 0; j < 32; ++j) x[j] = xc[j];
        } else {
          xval_ld(c, x);
        }
      };
      float sum = 0.f, xmax = -INFINITY;
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        xval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          sum += x[j];
          xmax = fmaxf(xmax, x[j]);
        }
      }
      const float mean = sum / float(H);
      float var = 0.f;
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        xval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float d = x[j] - mean;
          var = fmaf(d, d, var);
        }
      }
      const float inv = 1.0f / sqrtf(var / float(H) + kLnEps);
      if constexpr (MODE == M_CLS || MODE == M_TRIP) {
        float logit = pc2[H];
#pragma unroll
        for (int c = 0; c < H / 32; ++c) {
          float x[32];
          xval(c, x);
#pragma unroll
          for (int j = 0; j < 32; ++j) logit = fmaf(fmaxf((x[j] - mean) * inv, 0.f), pc2[c * 32 + j], logit);
        }
        if (valid) {
          if constexpr (MODE == M_TRIP) {
            p.tlogit[r] = logit;
            p.tkeep[r] = logit >= p.cut ? 1 : 0;
          } else {
            w.logit[r] = logit;
            w.keep[r] = logit >= p.cut ? 1 : 0;
          }
        }
        tc_fence_before();
        continue;
      }
      const float hmax = fmaxf((xmax - mean) * inv, 0.f);
      hid_scale = FP8 ? (hmax > 0.f ? hmax / 448.f : 1.f) : 1.f;
      const float hinv = FP8 ? (hmax > 0.f ? 448.f / hmax : 1.f) : 1.f;
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        xval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = fmaxf((x[j] - mean) * inv, 0.f);
        put_row_f32<FP8>(sHA, tid, KCHH, c * 32, x, 32, hinv);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
    } else {
      hid_scale = sa[0];
    }

    // ---- 4. layer 2 ----------------------------------------------------------
    if (tid == 0) {
      tc_fence_after();
      issue_layer<H, FP8>(tmem_base, sHA, sW2, L::K2, 1);
      mma_commit(&bar[1]);
    }
    if (!wait_mma()) {
      aborted = true;
      break;
    }
    // z[n] = s_w2[n] * s_h * acc[n] + b2[n] (FP8) or acc[n] + b2[n]
    auto zval = [&](int c, float (&z)[32]) {
      float v[32];
      tmem_ld32(tmem_lane + uint32_t(c * 32), v);
      tmem_wait_ld();
      if constexpr (FP8) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= hid_scale;
      }
      add_params<FP8>(v, pb2 + c * 32, ps2 + c * 32, z);
    };
    // residual input row (BF16) for the update modes
    auto resid = [&](int c, float (&z)[32]) {
      if constexpr (MODE == M_NODE_UPD || MODE == M_EDGE_UPD || MODE == M_EDGE_UPD_CLS) {
        const __nv_bfloat16* rowp = (MODE == M_NODE_UPD ? w.hstate16 : w.estate16) + size_t(r) * H;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 u = (L::PIPE && L::HA != L::A)
                              ? *reinterpret_cast<const uint4*>(sA + tile_off(tid, c * 4 + q, KCH1))
                          : (H <= 64) ? keep_row[c * 4 + q]
                                      : reinterpret_cast<const uint4*>(rowp)[c * 4 + q];
          z[8 * q + 0] += bf16_lo(u.x);
          z[8 * q + 1] += bf16_hi(u.x);
          z[8 * q + 2] += bf16_lo(u.y);
          z[8 * q + 3] += bf16_hi(u.y);
          z[8 * q + 4] += bf16_lo(u.z);
          z[8 * q + 5] += bf16_hi(u.z);
          z[8 * q + 6] += bf16_lo(u.w);
          z[8 * q + 7] += bf16_hi(u.w);
        }
      }
    };

    if constexpr (MODE != M_EDGE_UPD_CLS) {
      // ---- 5. store the new state (BF16) -----------------------------------
      constexpr bool NODE_ROWS = MODE == M_NODE_ENC || MODE == M_NODE_UPD;
      __nv_bfloat16* dst = (NODE_ROWS ? w.hstate16 : w.estate16) + size_t(r) * H;
      float row_max = 0.f;  // largest |stored value| of a node row
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float z[32];
        zval(c, z);
        if (valid) {
          resid(c, z);
          if constexpr (L::SPLIT && MODE == M_NODE_ENC) {
            // the FP32 encoding, read by the edge encoder
            float4* f4 = reinterpret_cast<float4*>(w.hstate + size_t(r) * H) + c * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) f4[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
          }
          uint4* d4 = reinterpret_cast<uint4*>(dst) + c * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 u = make_uint4(pack_bf16(z[8 * q], z[8 * q + 1]), pack_bf16(z[8 * q + 2], z[8 * q + 3]),
                                       pack_bf16(z[8 * q + 4], z[8 * q + 5]), pack_bf16(z[8 * q + 6], z[8 * q + 7]));
            d4[q] = u;
            if constexpr (NODE_ROWS && H == 128) {
              const uint32_t pk[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
              for (int j = 0; j < 4; ++j)
                row_max = fmaxf(row_max, fmaxf(fabsf(bf16_lo(pk[j])), fabsf(bf16_hi(pk[j]))));
            }
          }
        }
      }
      // (read by the FP8 edge steps at hidden 128 for their shared h scale)
      if constexpr (NODE_ROWS && H == 128)
        if (valid && w.hamax != nullptr) w.hamax[r] = row_max;
      tc_fence_before();
    } else {
      // ---- 5'. classifier on the new edge state, then the cut ---------------
      float emax = 0.f;
      if constexpr (FP8) {
#pragma unroll
        for (int c = 0; c < H / 32; ++c) {
          float z[32];
          zval(c, z);
          resid(c, z);
#pragma unroll
          for (int j = 0; j < 32; ++j) emax = fmaxf(emax, fabsf(z[j]));
        }
      }
      const float es = FP8 ? (emax > 0.f ? emax / 448.f : 1.f) : 1.f;
      const float einv = FP8 ? (emax > 0.f ? 448.f / emax : 1.f) : 1.f;
      // the new state is rounded to BF16 as it would be stored, then fed on
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float z[32];
        zval(c, z);
        resid(c, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = __bfloat162float(__float2bfloat16_rn(z[j]));
        put_row_f32<FP8>(sHA, tid, KCHH, c * 32, z, 32, einv);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_layer<H, FP8>(tmem_base, sHA, sWC, H, 1);
        mma_commit(&bar[1]);
      }
      if (!wait_mma()) {
        aborted = true;
        break;
      }
      auto cval_ld = [&](int c, float (&x)[32]) {
        float v[32];
        tmem_ld32(tmem_lane + uint32_t(c * 32), v);
        tmem_wait_ld();
        if constexpr (FP8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] *= es;
        }
        add_params<FP8>(v, pbc + c * 32, psc + c * 32, x);
      };
      float cc[H == 32 ? 32 : 1];
      if constexpr (H == 32) cval_ld(0, cc);
      auto cval = [&](int c, float (&x)[32]) {
        if constexpr (H == 32) {
#pragma unroll
          for (int j = 0; j < 32; ++j) x[j] = cc[j];
        } else {
          cval_ld(c, x);
        }
      };
      float sum = 0.f;
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        cval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) sum += x[j];
      }
      const float mean = sum / float(H);
      float var = 0.f;
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        cval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float d = x[j] - mean;
          var = fmaf(d, d, var);
        }
      }
      const float inv = 1.0f / sqrtf(var / float(H) + kLnEps);
      float logit = pc2[H];
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        float x[32];
        cval(c, x);
#pragma unroll
        for (int j = 0; j < 32; ++j) logit = fmaf(fmaxf((x[j] - mean) * inv, 0.f), pc2[c * 32 + j], logit);
      }
      if (valid) {
        w.logit[r] = logit;
        w.keep[r] = logit >= p.cut ? 1 : 0;
      }
      tc_fence_before();
    }
  }

  // ---- clean-up: on a timeout, give the outstanding MMAs one more bounded
  //      wait, then free the tensor memory -----------------------------------
  if constexpr (L::PIPE) cp_async_wait<0>();  // no copy may land after the exit
  if (aborted) {
    if (tid == 0) set_status(w.counters, ST_TIMEOUT);
    if (weights_late) mbar_wait_bounded(&bar[0], 0, kWaitCycles);
    if (mma_pending) mbar_wait_bounded(&bar[1], mma_phase, kWaitCycles);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// BF16 edge step with TMA-staged tiles (hidden 32). Same arithmetic as
// k_tc<32, BF16, M_EDGE_UPD / M_EDGE_UPD_CLS> (the MMAs see the same operand
// values in the same K order), but the layer-1 input [e, h_src, h_dst] of a
// tile is never touched by the threads:
//   * segment 0 (e rows, contiguous edges) is one 2-D TMA box of 128 rows;
//   * segments 1 and 2 (h_src, h_dst rows) are TMA row gathers, four rows per
//     instruction, one instruction per lane of warp 0 and segment;
// each segment lands as 128 rows x 64 bytes in the 64-byte swizzle layout
// (8 KB, 1024-byte aligned), which the MMA reads through swizzled
// descriptors. One tile buffer: once layer 1 has read it and every thread has
// taken its residual row into registers, the next tile's rows load while
// layer 2 and the epilogue run. The hidden row and the classifier input are
// written by the threads into a no-swizzle tile as in k_tc.
// ---------------------------------------------------------------------------
template <int H, bool CLS>
struct TmaLayout {
  static constexpr int SEG = kRows * H * 2;  // one segment: 128 rows x 64 bytes
  static constexpr int K1 = 3 * H;
  static constexpr int W1 = 0;
  static constexpr int W1_BYTES = H * K1 * 2;
  static constexpr int W2 = align1k(W1 + W1_BYTES);
  static constexpr int W2_BYTES = H * H * 2;
  static constexpr int WC = align1k(W2 + W2_BYTES);
  static constexpr int WC_BYTES = CLS ? H * H * 2 : 0;
  static constexpr int A = align1k(WC + WC_BYTES);
  static constexpr int ABUF = 3 * SEG;
  static constexpr int HA = align1k(A + ABUF);
  static constexpr int HA_BYTES = kRows * H * 2;
  static constexpr int PAR = HA + HA_BYTES;
  static constexpr int PAR_FLOATS = 4 * H + 4;  // b1, b2, bc1, c2 weights + bias
  static constexpr int BAR = PAR + PAR_FLOATS * 4;  // [0] weights [1] mma [2] tile
  static constexpr int TOTAL = BAR + 64;
  static constexpr int ALLOC = TOTAL + 1024;  // room to align the base to 1024 bytes
};

// (registers capped so that five CTAs fit an SM, as their shared memory does)
template <int H, bool CLS>
__global__ void __launch_bounds__(kRows, 5)
    k_tc_edge_tma(const TcArgs p, const __grid_constant__ CUtensorMap map_e,
                  const __grid_constant__ CUtensorMap map_h) {
  static_assert(H == 32, "one BF16 row segment of 32 elements is one 64-byte swizzle row");
  using L = TmaLayout<H, CLS>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sW1 = smem + L::W1;
  uint8_t* sW2 = smem + L::W2;
  uint8_t* sWC = smem + L::WC;
  uint8_t* sHA = smem + L::HA;
  float* par = reinterpret_cast<float*>(smem + L::PAR);
  float* pb1 = par;
  float* pb2 = par + H;
  float* pbc = par + 2 * H;
  float* pc2 = par + 3 * H;  // classifier layer 2: H weights, then the bias
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::BAR + 32);
  constexpr int KCHH = H * 2 / 16;  // 16-byte chunks per row of the hidden tile
  constexpr int MODE = CLS ? M_EDGE_UPD_CLS : M_EDGE_UPD;
  (void)MODE;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Ws& w = p.w;
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 32);
    tmem_relinquish();
  }
  for (int i = tid; i < H; i += kRows) {
    pb1[i] = p.b1[i];
    pb2[i] = p.b2[i];
    pbc[i] = CLS ? p.bc1[i] : 0.f;
    pc2[i] = CLS ? p.c2.WT[i * p.c2.ldo] : 0.f;
  }
  if (tid == 0) pc2[H] = CLS ? p.c2.b[0] : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const uint32_t tmem_lane = tmem_base + (uint32_t(warp * 32) << 16);

  if (tid == 0) {
    mbar_expect_tx(&bar[0], uint32_t(L::W1_BYTES + L::W2_BYTES + L::WC_BYTES));
    bulk_g2s(sW1, p.W1, L::W1_BYTES, &bar[0]);
    bulk_g2s(sW2, p.W2, L::W2_BYTES, &bar[0]);
    if (CLS) bulk_g2s(sWC, p.Wc, L::WC_BYTES, &bar[0]);
  }
  const bool wok = mbar_wait_bounded(&bar[0], 0, kWaitCycles);
  const bool weights_late = __syncthreads_or(!wok);
  bool aborted = weights_late;
  uint32_t mma_phase = 0, a_phase = 0;
  bool mma_pending = false, a_pending = false;

  const int hi = clamp_edges(w.counters, w.e_cap);
  const int n_tiles = (hi + kRows - 1) / kRows;
  uint8_t* A = smem + L::A;

  // warp 0: the node indices of the four rows 4 lane .. 4 lane + 3 of tile t
  // (rows past the last edge gather node 0 and are never stored), loaded a
  // phase ahead of their use
  int sv[4] = {0, 0, 0, 0}, dv[4] = {0, 0, 0, 0};
  auto load_idx = [&](int t) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = t * kRows + 4 * lane + i;
      sv[i] = r < hi ? w.src[r] : 0;
      dv[i] = r < hi ? w.col[r] : 0;
    }
  };
  // warp 0: the loads of tile t (expect-tx first, then the box of e rows and
  // each lane's two four-row gathers)
  auto issue = [&](int t) {
    if (lane == 0) {
      mbar_expect_tx(&bar[2], uint32_t(3 * L::SEG));
      tma_load_2d(A, &map_e, 0, t * kRows, &bar[2]);
    }
    __syncwarp();
    tma_gather4(A + L::SEG + 4 * lane * (H * 2), &map_h, 0, sv[0], sv[1], sv[2], sv[3], &bar[2]);
    tma_gather4(A + 2 * L::SEG + 4 * lane * (H * 2), &map_h, 0, dv[0], dv[1], dv[2], dv[3],
                &bar[2]);
  };
  auto wait_mma = [&]() -> bool {
    mma_pending = true;
    const bool good = mbar_wait_bounded(&bar[1], mma_phase, kWaitCycles);
    tc_fence_after();
    if (__syncthreads_or(!good)) return false;
    mma_phase ^= 1;
    mma_pending = false;
    return true;
  };

  if (!aborted && int(blockIdx.x) < n_tiles) {
    if (warp == 0) {
      load_idx(blockIdx.x);
      issue(blockIdx.x);
    }
    a_pending = true;
  }
  for (int t = blockIdx.x; t < n_tiles && !aborted; t += gridDim.x) {
    const int tn = t + int(gridDim.x);
    if (warp == 0 && tn < n_tiles) load_idx(tn);  // used after layer 1
    const bool got = mbar_wait_bounded(&bar[2], a_phase, kWaitCycles);
    if (__syncthreads_or(!got)) {
      aborted = true;
      break;
    }
    a_phase ^= 1;
    a_pending = false;
    const int r = t * kRows + tid;
    const bool valid = r < hi;

    // ---- layer 1: [e, h_src, h_dst] x W1 (K = 3H, 16 per instruction) --------
    if (tid == 0) {
      tc_fence_after();
      constexpr uint32_t IDESC = idesc_bf16(kRows, H);
      constexpr uint32_t SBO_W = uint32_t(L::K1 * 2 / 16) * 128;
      const uint32_t a0 = smem_u32(A), w0 = smem_u32(sW1);
#pragma unroll
      for (int k = 0; k < L::K1; k += 16) {
        const int seg = k / H, j = (k % H) / 16;
        const uint64_t ad = smem_desc_sw64(a0 + uint32_t(seg * L::SEG + j * 32));
        const uint64_t bd = smem_desc(w0 + uint32_t(k * 2 / 16) * 128, 128, SBO_W);
        mma_bf16(tmem_base, ad, bd, IDESC, k > 0 ? 1u : 0u);
      }
      mma_commit(&bar[1]);
    }
    if (!wait_mma()) {
      aborted = true;
      break;
    }
    // the residual: this row's e from segment 0 (64-byte swizzle), kept in
    // registers so that the buffer is free once the barrier below is passed
    uint4 e_row[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      e_row[q] = *reinterpret_cast<const uint4*>(A + tid * (H * 2) + ((q ^ ((tid >> 1) & 3)) << 4));
    // ---- bias + LayerNorm + ReLU -> hidden tile --------------------------------
    float x[32];
    {
      float v[32];
      tmem_ld32(tmem_lane, v);
      tmem_wait_ld();
      add_params<false>(v, pb1, pb1, x);
    }
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) sum += x[j];
    const float mean = sum / float(H);
    float var = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float d = x[j] - mean;
      var = fmaf(d, d, var);
    }
    const float inv = 1.0f / sqrtf(var / float(H) + kLnEps);
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = fmaxf((x[j] - mean) * inv, 0.f);
    put_row_f32<false>(sHA, tid, KCHH, 0, x, 32, 1.f);
    fence_proxy_async();  // hidden tile (MMA operand) and the reads of A done
    tc_fence_before();
    __syncthreads();
    // the tile buffer is free: the next tile's rows load during layer 2
    if (tn < n_tiles) {
      if (warp == 0) issue(tn);
      a_pending = true;
    }

    // ---- layer 2 ----------------------------------------------------------------
    if (tid == 0) {
      tc_fence_after();
      issue_layer<H, false>(tmem_base, sHA, sW2, H, 1);
      mma_commit(&bar[1]);
    }
    if (!wait_mma()) {
      aborted = true;
      break;
    }
    float z[32];
    {
      float v[32];
      tmem_ld32(tmem_lane, v);
      tmem_wait_ld();
      add_params<false>(v, pb2, pb2, z);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 u = e_row[q];
      z[8 * q + 0] += bf16_lo(u.x);
      z[8 * q + 1] += bf16_hi(u.x);
      z[8 * q + 2] += bf16_lo(u.y);
      z[8 * q + 3] += bf16_hi(u.y);
      z[8 * q + 4] += bf16_lo(u.z);
      z[8 * q + 5] += bf16_hi(u.z);
      z[8 * q + 6] += bf16_lo(u.w);
      z[8 * q + 7] += bf16_hi(u.w);
    }
    if constexpr (!CLS) {
      if (valid) {
        uint4* d4 = reinterpret_cast<uint4*>(w.estate16 + size_t(r) * H);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          d4[q] = make_uint4(pack_bf16(z[8 * q], z[8 * q + 1]), pack_bf16(z[8 * q + 2], z[8 * q + 3]),
                             pack_bf16(z[8 * q + 4], z[8 * q + 5]), pack_bf16(z[8 * q + 6], z[8 * q + 7]));
      }
      tc_fence_before();
      __syncthreads();  // every thread has read the tensor memory of this tile
    } else {
      // ---- classifier on the new edge state (rounded to BF16 as stored) -------
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = __bfloat162float(__float2bfloat16_rn(z[j]));
      put_row_f32<false>(sHA, tid, KCHH, 0, z, 32, 1.f);
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_layer<H, false>(tmem_base, sHA, sWC, H, 1);
        mma_commit(&bar[1]);
      }
      if (!wait_mma()) {
        aborted = true;
        break;
      }
      float c[32];
      {
        float v[32];
        tmem_ld32(tmem_lane, v);
        tmem_wait_ld();
        add_params<false>(v, pbc, pbc, c);
      }
      float cs = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) cs += c[j];
      const float cmean = cs / float(H);
      float cvar = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float d = c[j] - cmean;
        cvar = fmaf(d, d, cvar);
      }
      const float cinv = 1.0f / sqrtf(cvar / float(H) + kLnEps);
      float logit = pc2[H];
#pragma unroll
      for (int j = 0; j < 32; ++j) logit = fmaf(fmaxf((c[j] - cmean) * cinv, 0.f), pc2[j], logit);
      if (valid) {
        w.logit[r] = logit;
        w.keep[r] = logit >= p.cut ? 1 : 0;
      }
      tc_fence_before();
      __syncthreads();  // the hidden tile and the tensor memory are reused
    }
  }

  // ---- clean-up: on a timeout, give what is still in flight one more bounded
  //      wait, then free the tensor memory ---------------------------------------
  if (aborted) {
    if (tid == 0) set_status(w.counters, ST_TIMEOUT);
    if (weights_late) mbar_wait_bounded(&bar[0], 0, kWaitCycles);
    if (a_pending) mbar_wait_bounded(&bar[2], a_phase, kWaitCycles);
    if (mma_pending) mbar_wait_bounded(&bar[1], mma_phase, kWaitCycles);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 32);
  }
}

// ---------------------------------------------------------------------------
// BF16 edge step at hidden 32, warp-specialised (tuning form 2): same
// operands, K order and epilogue arithmetic as k_tc<32, BF16, M_EDGE_UPD /
// M_EDGE_UPD_CLS>, with several tiles in flight per CTA:
//   * warp 0 (producer) fills a ring of kWsStages tile buffers by TMA (box of
//     128 e rows, row gathers of h_src and h_dst, as in k_tc_edge_tma);
//   * warp 1 (one lane issues) runs the MMAs: layer 1 of tile i + 1 into one
//     of two tensor-memory accumulators while the epilogue works on tile i in
//     the other, then layer 2 (and the classifier) of tile i once its hidden
//     tile is written;
//   * two epilogue warpgroups (warps 2-5 and 6-9) take alternate tiles:
//     bias, LayerNorm, ReLU, the hidden tile, the residual e read from the
//     tile buffer (which then goes back to the producer), the new state or
//     the classifier and the cut.
// Hand-offs are mbarriers (full / empty per tile buffer; accumulator, hidden
// tile and accumulator-free per accumulator). Every wait is bounded; a wait
// that runs out raises a shared abort flag on which every other wait gives
// up too, and the kernel latches ST_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr int kWsStages = 3;
constexpr int kWsThreads = 320;  // producer, MMA, two epilogue warpgroups

template <bool CLS>
struct WsLayout {
  static constexpr int H = 32;
  static constexpr int SEG = kRows * H * 2;
  static constexpr int K1 = 3 * H;
  static constexpr int W1 = 0;
  static constexpr int W1_BYTES = H * K1 * 2;
  static constexpr int W2 = align1k(W1 + W1_BYTES);
  static constexpr int W2_BYTES = H * H * 2;
  static constexpr int WC = align1k(W2 + W2_BYTES);
  static constexpr int WC_BYTES = CLS ? H * H * 2 : 0;
  static constexpr int A = align1k(WC + WC_BYTES);
  static constexpr int ABUF = 3 * SEG;
  static constexpr int HA = A + kWsStages * ABUF;  // two hidden tiles
  static constexpr int HA_BYTES = kRows * H * 2;
  static constexpr int PAR = HA + 2 * HA_BYTES;
  static constexpr int PAR_FLOATS = 4 * H + 4;
  // barriers: full[S], empty[S], then per accumulator acc1, hid, acc2, cin,
  // acc3, free (2 each)
  static constexpr int BAR = PAR + PAR_FLOATS * 4;
  static constexpr int NBAR = 2 * kWsStages + 12;
  static constexpr int FLAG = BAR + NBAR * 8;  // abort flag, TMEM address
  static constexpr int TOTAL = FLAG + 16;
  static constexpr int ALLOC = TOTAL + 1024;
};

// Bounded wait that also gives up when another role has raised the abort flag.
__device__ __forceinline__ bool ws_wait(uint64_t* m, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(m, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(m, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(m)) : "memory");
}

template <bool CLS>
__global__ void __launch_bounds__(kWsThreads, 2)
    k_tc_edge_ws(const TcArgs p, const __grid_constant__ CUtensorMap map_e,
                 const __grid_constant__ CUtensorMap map_h) {
  constexpr int H = 32;
  using L = WsLayout<CLS>;
  constexpr int S = kWsStages;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sW1 = smem + L::W1;
  uint8_t* sW2 = smem + L::W2;
  uint8_t* sWC = smem + L::WC;
  float* par = reinterpret_cast<float*>(smem + L::PAR);
  float* pb1 = par;
  float* pb2 = par + H;
  float* pbc = par + 2 * H;
  float* pc2 = par + 3 * H;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::BAR);
  uint64_t* full = bar;            // [S] tile loaded
  uint64_t* empty = bar + S;       // [S] tile buffer free (128 arrivals)
  uint64_t* acc1 = bar + 2 * S;    // [2] layer-1 accumulator ready
  uint64_t* hid = acc1 + 2;        // [2] hidden tile written (128)
  uint64_t* acc2 = acc1 + 4;       // [2] layer-2 accumulator ready
  uint64_t* cin = acc1 + 6;        // [2] classifier input written (128)
  uint64_t* acc3 = acc1 + 8;       // [2] classifier accumulator ready
  uint64_t* tfree = acc1 + 10;     // [2] accumulator read out (128)
  volatile int* abort = reinterpret_cast<volatile int*>(smem + L::FLAG);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L::FLAG + 4);
  constexpr int KCHH = H * 2 / 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Ws& w = p.w;
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;

  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kRows);
    }
    for (int d = 0; d < 2; ++d) {
      mbar_init(&acc1[d], 1);
      mbar_init(&hid[d], kRows);
      mbar_init(&acc2[d], 1);
      mbar_init(&cin[d], kRows);
      mbar_init(&acc3[d], 1);
      mbar_init(&tfree[d], kRows);
    }
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, 64);  // two accumulators of 32 columns
    tmem_relinquish();
  }
  for (int i = tid; i < H; i += kWsThreads) {
    pb1[i] = p.b1[i];
    pb2[i] = p.b2[i];
    pbc[i] = CLS ? p.bc1[i] : 0.f;
    pc2[i] = CLS ? p.c2.WT[i * p.c2.ldo] : 0.f;
  }
  if (tid == 0) pc2[H] = CLS ? p.c2.b[0] : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tslot;

  // the weights come with the first tile: their bytes are counted on the
  // first full barrier, which the MMA warp waits for before its first MMA
  const int hi = clamp_edges(w.counters, w.e_cap);
  const int n_tiles = (hi + kRows - 1) / kRows;
  const int n_local = int(blockIdx.x) < n_tiles ? (n_tiles - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x) : 0;
  // a whole warp waits; it goes on only if every lane saw the phase complete
  // (so that the warp-collective instructions after it never diverge)
  auto wait_warp = [&](uint64_t* m, uint32_t parity) -> bool {
    const bool ok = ws_wait(m, parity, abort);
    return __all_sync(0xffffffffu, ok);
  };

  if (warp == 0) {
    // ---- producer ----------------------------------------------------------
    for (int i = 0; i < n_local; ++i) {
      const int t = int(blockIdx.x) + i * int(gridDim.x);
      const int s = i % S, u = i / S;
      if (u > 0 && !wait_warp(&empty[s], uint32_t((u - 1) & 1))) break;
      int sv[4], dv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = t * kRows + 4 * lane + q;
        sv[q] = r < hi ? w.src[r] : 0;
        dv[q] = r < hi ? w.col[r] : 0;
      }
      uint8_t* A = smem + L::A + s * L::ABUF;
      if (lane == 0) {
        const uint32_t wbytes = i == 0 ? uint32_t(L::W1_BYTES + L::W2_BYTES + L::WC_BYTES) : 0u;
        mbar_expect_tx(&full[s], uint32_t(3 * L::SEG) + wbytes);
        if (i == 0) {
          bulk_g2s(sW1, p.W1, L::W1_BYTES, &full[s]);
          bulk_g2s(sW2, p.W2, L::W2_BYTES, &full[s]);
          if (CLS) bulk_g2s(sWC, p.Wc, L::WC_BYTES, &full[s]);
        }
        tma_load_2d(A, &map_e, 0, t * kRows, &full[s]);
      }
      __syncwarp();
      tma_gather4(A + L::SEG + 4 * lane * (H * 2), &map_h, 0, sv[0], sv[1], sv[2], sv[3], &full[s]);
      tma_gather4(A + 2 * L::SEG + 4 * lane * (H * 2), &map_h, 0, dv[0], dv[1], dv[2], dv[3],
                  &full[s]);
    }
  } else if (warp == 1) {
    // ---- MMA issuer (lane 0; the other lanes wait for it at the warp barrier)
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16(kRows, H);
      constexpr uint32_t SBO_W = uint32_t(L::K1 * 2 / 16) * 128;
      auto layer1 = [&](int i) -> bool {
        const int s = i % S, d = i & 1;
        if (!ws_wait(&full[s], uint32_t((i / S) & 1), abort)) return false;
        if (i >= 2 && !ws_wait(&tfree[d], uint32_t(((i >> 1) - 1) & 1), abort)) return false;
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + L::A + s * L::ABUF), w0 = smem_u32(sW1);
#pragma unroll
        for (int k = 0; k < L::K1; k += 16) {
          const int seg = k / H, j = (k % H) / 16;
          const uint64_t ad = smem_desc_sw64(a0 + uint32_t(seg * L::SEG + j * 32));
          const uint64_t bd = smem_desc(w0 + uint32_t(k * 2 / 16) * 128, 128, SBO_W);
          mma_bf16(tmem_base + uint32_t(32 * d), ad, bd, IDESC, k > 0 ? 1u : 0u);
        }
        mma_commit(&acc1[d]);
        return true;
      };
      bool ok = n_local == 0 || layer1(0);
      for (int i = 0; i < n_local && ok; ++i) {
        const int d = i & 1;
        const uint32_t ph = uint32_t((i >> 1) & 1);
        if (i + 1 < n_local && !layer1(i + 1)) break;
        uint8_t* HA = smem + L::HA + d * L::HA_BYTES;
        if (!ws_wait(&hid[d], ph, abort)) break;
        tc_fence_after();
        issue_layer<H, false>(tmem_base + uint32_t(32 * d), HA, sW2, H, 1);
        mma_commit(&acc2[d]);
        if constexpr (CLS) {
          if (!ws_wait(&cin[d], ph, abort)) break;
          tc_fence_after();
          issue_layer<H, false>(tmem_base + uint32_t(32 * d), HA, sWC, H, 1);
          mma_commit(&acc3[d]);
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warpgroups: g takes tiles i = g, g + 2, ... ---------------
    const int g = (warp - 2) >> 2;
    const int row = 32 * (warp & 3) + lane;  // TMEM lane of this thread
    const uint32_t tmem_row = tmem_base + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(32 * g);
    uint8_t* HA = smem + L::HA + g * L::HA_BYTES;
    for (int i = g; i < n_local; i += 2) {
      const int t = int(blockIdx.x) + i * int(gridDim.x);
      const int s = i % S;
      const uint32_t ph = uint32_t((i >> 1) & 1);
      const int r = t * kRows + row;
      const bool valid = r < hi;
      const uint8_t* A = smem + L::A + s * L::ABUF;
      if (!wait_warp(&acc1[g], ph)) break;
      tc_fence_after();
      float x[32];
      {
        float v[32];
        tmem_ld32(tmem_row, v);
        tmem_wait_ld();
        add_params<false>(v, pb1, pb1, x);
      }
      float sum = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) sum += x[j];
      const float mean = sum / float(H);
      float var = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float dd = x[j] - mean;
        var = fmaf(dd, dd, var);
      }
      const float inv = 1.0f / sqrtf(var / float(H) + kLnEps);
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = fmaxf((x[j] - mean) * inv, 0.f);
      put_row_f32<false>(HA, row, KCHH, 0, x, 32, 1.f);
      uint4 e_row[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        e_row[q] = *reinterpret_cast<const uint4*>(A + row * (H * 2) + ((q ^ ((row >> 1) & 3)) << 4));
      fence_proxy_async();  // hidden tile to the MMA; the reads of A before its refill
      mbar_arrive(&hid[g]);
      mbar_arrive(&empty[s]);
      if (!wait_warp(&acc2[g], ph)) break;
      tc_fence_after();
      float z[32];
      {
        float v[32];
        tmem_ld32(tmem_row, v);
        tmem_wait_ld();
        add_params<false>(v, pb2, pb2, z);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 u = e_row[q];
        z[8 * q + 0] += bf16_lo(u.x);
        z[8 * q + 1] += bf16_hi(u.x);
        z[8 * q + 2] += bf16_lo(u.y);
        z[8 * q + 3] += bf16_hi(u.y);
        z[8 * q + 4] += bf16_lo(u.z);
        z[8 * q + 5] += bf16_hi(u.z);
        z[8 * q + 6] += bf16_lo(u.w);
        z[8 * q + 7] += bf16_hi(u.w);
      }
      if constexpr (!CLS) {
        if (valid) {
          uint4* d4 = reinterpret_cast<uint4*>(w.estate16 + size_t(r) * H);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            d4[q] = make_uint4(pack_bf16(z[8 * q], z[8 * q + 1]), pack_bf16(z[8 * q + 2], z[8 * q + 3]),
                               pack_bf16(z[8 * q + 4], z[8 * q + 5]),
                               pack_bf16(z[8 * q + 6], z[8 * q + 7]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = __bfloat162float(__float2bfloat16_rn(z[j]));
        put_row_f32<false>(HA, row, KCHH, 0, z, 32, 1.f);  // layer 2 has read HA
        fence_proxy_async();
        mbar_arrive(&cin[g]);
        if (!wait_warp(&acc3[g], ph)) break;
        tc_fence_after();
        float c[32];
        {
          float v[32];
          tmem_ld32(tmem_row, v);
          tmem_wait_ld();
          add_params<false>(v, pbc, pbc, c);
        }
        float cs = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) cs += c[j];
        const float cmean = cs / float(H);
        float cvar = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float dd = c[j] - cmean;
          cvar = fmaf(dd, dd, cvar);
        }
        const float cinv = 1.0f / sqrtf(cvar / float(H) + kLnEps);
        float logit = pc2[H];
#pragma unroll
        for (int j = 0; j < 32; ++j) logit = fmaf(fmaxf((c[j] - cmean) * cinv, 0.f), pc2[j], logit);
        if (valid) {
          w.logit[r] = logit;
          w.keep[r] = logit >= p.cut ? 1 : 0;
        }
      }
      tc_fence_before();
      mbar_arrive(&tfree[g]);  // this accumulator's tensor memory is read out
    }
  }

  // ---- end: after an abort, let copies and MMAs in flight drain (bounded
  //      sleep), then free the tensor memory -------------------------------------
  __syncthreads();
  if (*abort) {
    if (tid == 0) set_status(w.counters, ST_TIMEOUT);
    const long long t0 = clock64();
    while (clock64() - t0 < 20000000LL) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 64);
  }
}

// ---------------------------------------------------------------------------
// messages of the node step from the BF16 edge states: P[v] = [sum of e over
// v's out edges | sum over its in edges], FP32 sums in increasing list order
// starting from zero, stored as FP32 (FP8 path: the node step quantises them
// with a per-row scale) or rounded to BF16 (BF16 path: the layer-1 operand
// as the node step would round it). One group of 8 lanes per node, H/8
// columns per lane; U list entries per round are loaded together (entries
// past the end reload a valid row and are dropped).
// ---------------------------------------------------------------------------
template <int H, bool OUT16>
__global__ void __launch_bounds__(256) k_msg_bf16(Batch b, Ws w) {
  constexpr int LPN = H / 8;    // lanes per hit: 8 columns (16 bytes) each
  constexpr int NPW = 32 / LPN; // hits per warp
  constexpr int U = 8;
  if (*(volatile int32_t*)&w.counters[C_STATUS] & ST_INPUT) return;
  const int E = clamp_edges(w.counters, w.e_cap);
  const int q = threadIdx.x % LPN;
  const int groups = gridDim.x * (blockDim.x / LPN);
  (void)NPW;
  for (int row = blockIdx.x * (blockDim.x / LPN) + threadIdx.x / LPN; row < b.n_hits; row += groups) {
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
      float2 s[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 < n; t0 += U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int at = a + min(t0 + u, n - 1);
          const int e = side == 0 ? at : __ldg(w.in_edge + at);
          v[u] = __ldg(reinterpret_cast<const uint4*>(w.estate16 + size_t(e) * H) + q);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (t0 + u < n) {
            s[0] = __fadd2_rn(s[0], make_float2(bf16_lo(v[u].x), bf16_hi(v[u].x)));
            s[1] = __fadd2_rn(s[1], make_float2(bf16_lo(v[u].y), bf16_hi(v[u].y)));
            s[2] = __fadd2_rn(s[2], make_float2(bf16_lo(v[u].z), bf16_hi(v[u].z)));
            s[3] = __fadd2_rn(s[3], make_float2(bf16_lo(v[u].w), bf16_hi(v[u].w)));
          }
      }
      if constexpr (OUT16) {
        uint4* o16 = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(w.pstate) +
                                              size_t(row) * 2 * H + side * H) + q;
        *o16 = make_uint4(pack_bf16(s[0].x, s[0].y), pack_bf16(s[1].x, s[1].y),
                          pack_bf16(s[2].x, s[2].y), pack_bf16(s[3].x, s[3].y));
      } else {
        float4* o = reinterpret_cast<float4*>(w.pstate + size_t(row) * 2 * H + side * H + 8 * q);
        o[0] = make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
        o[1] = make_float4(s[2].x, s[2].y, s[3].x, s[3].y);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
// CTAs per SM of one kernel: the occupancy query, capped so that the CTAs of an
// SM fit in its 512 tensor-memory columns; computed once per instantiation.
template <int H, bool FP8, int MODE>
int tc_blocks_per_sm() {
  using L = Layout<H, FP8, MODE>;
  // computed once per instantiation (thread-safe initialisation of a local static)
  static const int per_sm = [] {
    cudaError_t e = cudaFuncSetAttribute(k_tc<H, FP8, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc<H, FP8, MODE>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int n = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tc<H, FP8, MODE>, kRows, L::TOTAL);
    // the same bound from the kernel's resources: registers (allocated per warp
    // in units of 256), shared memory (228 KB per SM, 1 KB reserved per CTA),
    // 2048 threads per SM. CTAs never wait on one another, so a bound above
    // what fits only queues CTAs.
    cudaFuncAttributes fa{};
    int est = 16;
    if (cudaFuncGetAttributes(&fa, k_tc<H, FP8, MODE>) == cudaSuccess && fa.numRegs > 0) {
      const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
      est = std::min(est, 65536 / (regs_warp * (kRows / 32)));
    }
    est = std::min(est, 233472 / (L::TOTAL + 1024));
    if (e != cudaSuccess) cudaGetLastError();
    if (getenv("GNNTRK_VERBOSE"))
      fprintf(stderr, "gnntrk: k_tc<%d,%d,%d> occupancy query %d (%s), resource bound %d\n", H,
              int(FP8), MODE, n, cudaGetErrorString(e), est);
    n = std::max(n, est);
    n = n < 1 ? 1 : n;
    while (n > 1 && n * L::TMEM_COLS > 512) --n;
    if (getenv("GNNTRK_VERBOSE"))
      fprintf(stderr, "gnntrk: k_tc<%d,%d,%d> smem %d B, %d CTAs/SM\n", H, int(FP8), MODE,
              L::TOTAL, n);
    return n;
  }();
  return per_sm;
}

// Resident CTAs per SM chosen by the autotuner, per (FP8, hidden, kernel
// family); 0 = the resource bound. Families: 0 node encoder, 1 edge encoder,
// 2 node step, 3 edge step and classifier.
std::atomic<int> g_tuned[2][3][4] = {};

constexpr int family_of(int mode) {
  return mode == M_NODE_ENC ? 0 : mode == M_EDGE_ENC ? 1 : mode == M_NODE_UPD ? 2 : 3;
}
static_assert(family_of(M_TRIP) == 3, "triplet classifier tunes with the edge family");
constexpr int hidx(int h) { return h == 32 ? 0 : (h == 64 ? 1 : 2); }

// BF16 edge step at hidden 32: 0 per-thread copies, 1 TMA-staged tiles, 2
// warp-specialised with TMA-staged tiles
std::atomic<int> g_edge_form{0};

// CTAs per SM of the TMA edge step: shared memory and tensor memory bound
template <bool CLS>
int tma_blocks_per_sm() {
  using L = TmaLayout<32, CLS>;
  static const int per_sm = [] {
    cudaError_t e = cudaFuncSetAttribute(k_tc_edge_tma<32, CLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_edge_tma<32, CLS>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) cudaGetLastError();
    int n = 233472 / (L::ALLOC + 1024);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_tc_edge_tma<32, CLS>) == cudaSuccess && fa.numRegs > 0) {
      const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
      n = std::min(n, 65536 / (regs_warp * (kRows / 32)));
    }
    n = std::max(1, std::min(n, 512 / 32));
    if (getenv("GNNTRK_VERBOSE"))
      fprintf(stderr, "gnntrk: k_tc_edge_tma<32,%d> smem %d B, %d CTAs/SM\n", int(CLS), L::ALLOC, n);
    return n;
  }();
  return per_sm;
}

template <bool CLS>
void launch_edge_tma(const TcArgs& a, const TcModel& m, cudaStream_t s) {
  using L = TmaLayout<32, CLS>;
  const int grid = device_sms() * tma_blocks_per_sm<CLS>();
  k_tc_edge_tma<32, CLS><<<grid, kRows, L::ALLOC, s>>>(a, m.map_e, m.map_h);
}

// CTAs per SM of the warp-specialised edge step (shared memory bound)
template <bool CLS>
int ws_blocks_per_sm() {
  using L = WsLayout<CLS>;
  static const int per_sm = [] {
    cudaError_t e = cudaFuncSetAttribute(k_tc_edge_ws<CLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_edge_ws<CLS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               100);
    if (e != cudaSuccess) cudaGetLastError();
    int n = std::max(1, std::min(2, 233472 / (L::ALLOC + 1024)));
    if (getenv("GNNTRK_VERBOSE"))
      fprintf(stderr, "gnntrk: k_tc_edge_ws<%d> smem %d B, %d CTAs/SM\n", int(CLS), L::ALLOC, n);
    return n;
  }();
  return per_sm;
}

template <bool CLS>
void launch_edge_ws(const TcArgs& a, const TcModel& m, cudaStream_t s) {
  using L = WsLayout<CLS>;
  const int grid = device_sms() * ws_blocks_per_sm<CLS>();
  k_tc_edge_ws<CLS><<<grid, kWsThreads, L::ALLOC, s>>>(a, m.map_e, m.map_h);
}

template <int H, bool FP8, int MODE>
void launch_mode(const TcArgs& a, cudaStream_t s, int rows_hint) {
  using L = Layout<H, FP8, MODE>;
  int per_sm = tc_blocks_per_sm<H, FP8, MODE>();
  const int tuned = g_tuned[FP8 ? 1 : 0][hidx(H)][family_of(MODE)].load(std::memory_order_relaxed);
  if (tuned > 0 && tuned < per_sm) per_sm = tuned;
  int grid = device_sms() * per_sm;
  if (rows_hint >= 0) grid = rows_hint == 0 ? 1 : min(grid, div_up(rows_hint, kRows));
  k_tc<H, FP8, MODE><<<grid, kRows, L::TOTAL, s>>>(a);
}

template <int H, bool FP8>
void launch_h(int mode, const TcArgs& a, cudaStream_t s, int rows_hint) {
  switch (mode) {
    case M_NODE_ENC: launch_mode<H, FP8, M_NODE_ENC>(a, s, rows_hint); break;
    case M_EDGE_ENC: launch_mode<H, FP8, M_EDGE_ENC>(a, s, rows_hint); break;
    case M_NODE_UPD: launch_mode<H, FP8, M_NODE_UPD>(a, s, rows_hint); break;
    case M_EDGE_UPD: launch_mode<H, FP8, M_EDGE_UPD>(a, s, rows_hint); break;
    case M_EDGE_UPD_CLS: launch_mode<H, FP8, M_EDGE_UPD_CLS>(a, s, rows_hint); break;
    case M_CLS: launch_mode<H, FP8, M_CLS>(a, s, rows_hint); break;
    case M_TRIP:
      if constexpr (!FP8) launch_mode<H, false, M_TRIP>(a, s, rows_hint);
      break;
  }
}

template <bool FP8>
constexpr int smem_total(int H, int mode) {
#define GNNTRK_LT(HH)                                                                 \
  (mode == M_NODE_ENC ? Layout<HH, FP8, M_NODE_ENC>::TOTAL                            \
   : mode == M_EDGE_ENC ? Layout<HH, FP8, M_EDGE_ENC>::TOTAL                          \
   : mode == M_NODE_UPD ? Layout<HH, FP8, M_NODE_UPD>::TOTAL                          \
   : mode == M_EDGE_UPD ? Layout<HH, FP8, M_EDGE_UPD>::TOTAL                          \
   : mode == M_EDGE_UPD_CLS ? Layout<HH, FP8, M_EDGE_UPD_CLS>::TOTAL                  \
   : mode == M_TRIP ? Layout<HH, FP8, M_TRIP>::TOTAL                                  \
                            : Layout<HH, FP8, M_CLS>::TOTAL)
  return H == 32 ? GNNTRK_LT(32) : (H == 64 ? GNNTRK_LT(64) : GNNTRK_LT(128));
#undef GNNTRK_LT
}

void launch_any(int H, bool fp8, int mode, const TcArgs& a, cudaStream_t s, int rows_hint) {
  if (fp8) {
    if (H == 32) launch_h<32, true>(mode, a, s, rows_hint);
    else if (H == 64) launch_h<64, true>(mode, a, s, rows_hint);
    else launch_h<128, true>(mode, a, s, rows_hint);
  } else {
    if (H == 32) launch_h<32, false>(mode, a, s, rows_hint);
    else if (H == 64) launch_h<64, false>(mode, a, s, rows_hint);
    else launch_h<128, false>(mode, a, s, rows_hint);
  }
}

constexpr int kMaxSmem = 232448;  // 227 KB of dynamic shared memory per CTA

// ---------------------------------------------------------------------------
// host: weight packing
// ---------------------------------------------------------------------------
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return uint16_t((u >> 16) | 0x40);  // quiet NaN
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
  return uint16_t(u >> 16);
}

}  // namespace

// E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, no infinities,
// largest finite 448) of a float, rounding to nearest even and saturating to
// +-448; NaN maps to 0x7F.
uint8_t e4m3_from_float(float f) {
  if (std::isnan(f)) return 0x7f;
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  double a = std::fabs(double(f));
  if (a >= 448.0) return sign | 0x7e;
  // candidates: subnormals k * 2^-9 (k = 0..7), normals (1 + m/8) * 2^(e-7)
  int e = 0;
  if (a < std::ldexp(1.0, -6)) {
    double k = a / std::ldexp(1.0, -9);
    double fl = std::floor(k), r = k - fl;
    int q = int(fl);
    if (r > 0.5 || (r == 0.5 && (q & 1))) ++q;
    return sign | uint8_t(q);  // q == 8 is the smallest normal (0x08)
  }
  std::frexp(a, &e);  // a = f * 2^e, f in [0.5, 1)
  int E = e - 1;      // a in [2^E, 2^(E+1))
  double m = a / std::ldexp(1.0, E) - 1.0;  // [0, 1)
  double k = m * 8.0;
  double fl = std::floor(k), r = k - fl;
  int q = int(fl);
  if (r > 0.5 || (r == 0.5 && (q & 1))) ++q;
  if (q == 8) {
    q = 0;
    ++E;
  }
  int be = E + 7;
  uint8_t code = uint8_t((be << 3) | q);
  if (code > 0x7e) code = 0x7e;
  return sign | code;
}

float e4m3_to_float(uint8_t c) {
  const float s = (c & 0x80) ? -1.f : 1.f;
  const int be = (c >> 3) & 0xf, m = c & 7;
  if (be == 0xf && m == 7) return NAN;
  if (be == 0) return s * std::ldexp(float(m), -9);
  return s * std::ldexp(1.f + float(m) / 8.f, be - 7);
}

namespace {

// Operand image of W[out][in] for the tensor cores: K-major rows of `out`,
// core matrices of 8 rows x 16 bytes, chunks of a row contiguous per 8-row
// group. FP8: per-output-channel scale amax/448 applied before encoding.
void pack_layer(const HostLayer& l, bool fp8, std::vector<uint8_t>& img, std::vector<float>& scale) {
  const int N = l.out, K = l.in;
  const int esz = fp8 ? 1 : 2, epc = 16 / esz;
  const int kch = K / epc;
  img.assign(size_t(N) * K * esz, 0);
  scale.assign(N, 1.f);
  for (int n = 0; n < N; ++n) {
    float amax = 0.f;
    for (int k = 0; k < K; ++k) amax = std::max(amax, std::fabs(l.W[size_t(n) * K + k]));
    if (fp8) scale[n] = amax > 0.f ? amax / 448.f : 1.f;
    for (int k = 0; k < K; ++k) {
      const size_t off = size_t((n / 8) * kch + k / epc) * 128 + (n % 8) * 16 + (k % epc) * esz;
      const float v = l.W[size_t(n) * K + k];
      if (fp8) {
        img[off] = e4m3_from_float(v / scale[n]);
      } else {
        const uint16_t b = bf16_bits(v);
        img[off] = uint8_t(b & 0xff);
        img[off + 1] = uint8_t(b >> 8);
      }
    }
  }
}

}  // namespace

int tc_upload(TcModel& m, const HostLayer* L, int n_layers, int n_embed, int h, int K,
              int precision, void** dmem, std::string& err) {
  const bool fp8 = precision == GNNTRK_FP8_E4M3;
  // which layers: node enc l2, edge enc l1/l2, per step node l1/l2 edge l1/l2, cls l1
  // (BF16: the node encoder's layer 2 and the edge encoder's layer 1 take
  // split operands, so their images repeat W along K)
  // (FP8: the encoders run as the BF16 split-operand kernels, whose images
  // are packed in BF16 as well; E4M3 cannot carry the node encoding the
  // encoders consume)
  struct Item {
    int layer;
    LayerTC* dst;
    bool repeat_k = false;
    bool bf16 = false;  // a BF16 image on an FP8 handle
  };
  std::vector<Item> items;
  int c = n_embed;
  items.push_back({c + 1, &m.node_enc.l2, !fp8});
  items.push_back({c + 2, &m.edge_enc.l1, !fp8});
  items.push_back({c + 3, &m.edge_enc.l2});
  m.enc16 = fp8;
  if (m.enc16) {
    items.push_back({c + 1, &m.node_enc16.l2, true, true});
    items.push_back({c + 2, &m.edge_enc16.l1, h <= 64, true});  // h 128: two passes, plain image
    items.push_back({c + 3, &m.edge_enc16.l2, false, true});
  }
  c += 4;
  for (int k = 0; k < K; ++k) {
    items.push_back({c, &m.node[k].l1});
    items.push_back({c + 1, &m.node[k].l2});
    items.push_back({c + 2, &m.edge[k].l1});
    items.push_back({c + 3, &m.edge[k].l2});
    c += 4;
  }
  items.push_back({c, &m.cls.l1});
  if (c + 2 != n_layers) {
    err = "tensor-core packing: unexpected layer count";
    return GNNTRK_ERR_WEIGHTS;
  }
  // shared-memory budget of the largest kernel (FP8: its encoders are BF16)
  for (int mode : {M_EDGE_UPD, M_NODE_UPD, M_EDGE_ENC, M_NODE_ENC}) {
    const bool enc = mode == M_EDGE_ENC || mode == M_NODE_ENC;
    const bool as_fp8 = fp8 && !(enc && m.enc16);
    if ((as_fp8 ? smem_total<true>(h, mode) : smem_total<false>(h, mode)) > kMaxSmem) {
      err = "tensor-core kernels do not fit shared memory at this hidden size";
      return GNNTRK_ERR_UNSUPPORTED;
    }
  }
  std::vector<uint8_t> blob;
  std::vector<size_t> off_img(items.size()), off_b(items.size()), off_s(items.size());
  auto align = [&](size_t a) { blob.resize((blob.size() + a - 1) / a * a, 0); };
  for (size_t i = 0; i < items.size(); ++i) {
    std::vector<uint8_t> img;
    std::vector<float> sc;
    if (items[i].repeat_k) {
      const HostLayer& l = L[items[i].layer];
      HostLayer r2;
      r2.in = 2 * l.in;
      r2.out = l.out;
      r2.b = l.b;
      r2.W.resize(size_t(r2.out) * r2.in);
      for (int n = 0; n < l.out; ++n)
        for (int k = 0; k < r2.in; ++k) r2.W[size_t(n) * r2.in + k] = l.W[size_t(n) * l.in + k % l.in];
      pack_layer(r2, fp8 && !items[i].bf16, img, sc);
    } else {
      pack_layer(L[items[i].layer], fp8 && !items[i].bf16, img, sc);
    }
    align(1024);
    off_img[i] = blob.size();
    blob.insert(blob.end(), img.begin(), img.end());
    align(16);
    off_b[i] = blob.size();
    const auto& bb = L[items[i].layer].b;
    blob.resize(blob.size() + 4 * bb.size());
    std::memcpy(blob.data() + off_b[i], bb.data(), 4 * bb.size());
    align(16);
    off_s[i] = blob.size();
    blob.resize(blob.size() + 4 * sc.size());
    std::memcpy(blob.data() + off_s[i], sc.data(), 4 * sc.size());
  }
  void* d = nullptr;
  if (cudaMalloc(&d, blob.size()) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc of the tensor-core weights failed";
    return GNNTRK_ERR_OOM;
  }
  if (cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    err = "tensor-core weight upload failed";
    return GNNTRK_ERR_CUDA;
  }
  *dmem = d;
  const uint8_t* base = static_cast<const uint8_t*>(d);
  for (size_t i = 0; i < items.size(); ++i) {
    const HostLayer& l = L[items[i].layer];
    *items[i].dst = LayerTC{base + off_img[i], reinterpret_cast<const float*>(base + off_b[i]),
                            reinterpret_cast<const float*>(base + off_s[i]),
                            items[i].repeat_k ? 2 * l.in : l.in, l.out};
  }
  m.precision = precision;
  m.h = h;
  m.K = K;
  m.n_embed = n_embed;
  return GNNTRK_OK;
}

int tc_upload_triplets(TcModel& m, const HostLayer& art1, const HostLayer& elb1, void** dmem,
                       std::string& err) {
  std::vector<uint8_t> ia, ie;
  std::vector<float> sa, se;
  pack_layer(art1, false, ia, sa);
  pack_layer(elb1, false, ie, se);
  const size_t off_e = (ia.size() + 1023) / 1024 * 1024;
  std::vector<uint8_t> blob(off_e + ie.size());
  std::memcpy(blob.data(), ia.data(), ia.size());
  std::memcpy(blob.data() + off_e, ie.data(), ie.size());
  void* d = nullptr;
  if (cudaMalloc(&d, blob.size()) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc of the triplet-classifier weights failed";
    return GNNTRK_ERR_OOM;
  }
  if (cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    err = "triplet-classifier weight upload failed";
    return GNNTRK_ERR_CUDA;
  }
  *dmem = d;
  const uint8_t* base = static_cast<const uint8_t*>(d);
  m.art1 = LayerTC{base, nullptr, nullptr, art1.in, art1.out};
  m.elb1 = LayerTC{base + off_e, nullptr, nullptr, elb1.in, elb1.out};
  m.has_trip = true;
  return GNNTRK_OK;
}

namespace {
TcArgs base_args(const Batch& b, const Ws& w, const GraphParams& g) {
  TcArgs a{};
  a.b = b;
  a.w = w;
  for (int i = 0; i < 6; ++i) a.fs[i] = g.fs[i];
  a.cut = g.cut_logit;
  return a;
}
}  // namespace

void tc_node_prep(const Batch& b, const Ws& w, const TcModel& m, const LayerF32* embed_f32,
                  int n_embed, int D, int h, const GraphParams& g, const LayerF32& ne1_f32,
                  cudaStream_t s, bool do_embed) {
  // embedding in FP32: its output feeds the threshold d^2 < r^2
  const Sel all{nullptr, nullptr};
  if (do_embed)
    launch_node_prep_f32(b, w, embed_f32, n_embed, Mlp2F32{}, EdgeProj{}, D, h, g, true, false,
                         all, s);
  TcArgs a = base_args(b, w, g);
  a.ne1 = ne1_f32;
  const Mlp2TC& ne = m.enc16 ? m.node_enc16 : m.node_enc;
  a.W2 = static_cast<const uint8_t*>(ne.l2.B);
  a.b2 = ne.l2.b;
  a.s2 = ne.l2.scale;
  launch_any(h, m.precision == GNNTRK_FP8_E4M3 && !m.enc16, M_NODE_ENC, a, s, b.n_hits);
}

void tc_messages(const Batch& b, const Ws& w, int h, bool fp8, cudaStream_t s) {
  const int grid = std::max(1, std::min(device_sms() * 8, div_up(b.n_hits, 256 / (h / 8))));
  if (h == 32)
    fp8 ? k_msg_bf16<32, false><<<grid, 256, 0, s>>>(b, w) : k_msg_bf16<32, true><<<grid, 256, 0, s>>>(b, w);
  else if (h == 64)
    fp8 ? k_msg_bf16<64, false><<<grid, 256, 0, s>>>(b, w) : k_msg_bf16<64, true><<<grid, 256, 0, s>>>(b, w);
  else
    fp8 ? k_msg_bf16<128, false><<<grid, 256, 0, s>>>(b, w) : k_msg_bf16<128, true><<<grid, 256, 0, s>>>(b, w);
}

void tc_gnn(const Batch& b, const Ws& w, const TcModel& m, int h, int K, const GraphParams& g,
            const LayerF32& cls2_f32, cudaStream_t s, int stage, bool store_final) {
  const bool fp8 = m.precision == GNNTRK_FP8_E4M3;
  TcArgs a = base_args(b, w, g);
  a.c2 = cls2_f32;
  a.Wc = static_cast<const uint8_t*>(m.cls.l1.B);
  a.bc1 = m.cls.l1.b;
  a.sc = m.cls.l1.scale;
  const bool fuse = !store_final &&
                    (fp8 ? smem_total<true>(h, M_EDGE_UPD_CLS) : smem_total<false>(h, M_EDGE_UPD_CLS)) <= kMaxSmem;
  auto set = [&](const Mlp2TC& mm) {
    a.W1 = static_cast<const uint8_t*>(mm.l1.B);
    a.b1 = mm.l1.b;
    a.s1 = mm.l1.scale;
    a.W2 = static_cast<const uint8_t*>(mm.l2.B);
    a.b2 = mm.l2.b;
    a.s2 = mm.l2.scale;
  };
  // stage < 0: everything; otherwise 0 = edge encoder, 1 + 2k = node step k,
  // 2 + 2k = edge step k (with the classifier at the last step)
  if (stage < 0 || stage == 0) {
    if (m.enc16) {
      set(m.edge_enc16);
      launch_any(h, false, M_EDGE_ENC, a, s, -1);
    } else {
      set(m.edge_enc);
      launch_any(h, fp8, M_EDGE_ENC, a, s, -1);
    }
  }
  for (int k = 0; k < K; ++k) {
    if (stage < 0) tc_messages(b, w, h, fp8, s);
    if (stage < 0 || stage == 1 + 2 * k) {
      set(m.node[k]);
      launch_any(h, fp8, M_NODE_UPD, a, s, b.n_hits);
    }
    if (stage < 0 || stage == 2 + 2 * k) {
      set(m.edge[k]);
      const bool last = k + 1 == K;
      const int form = (!fp8 && h == 32 && m.maps) ? g_edge_form.load(std::memory_order_relaxed) : 0;
      if (form == 1 && last && fuse)
        launch_edge_tma<true>(a, m, s);
      else if (form == 1)
        launch_edge_tma<false>(a, m, s);
      else if (form == 2 && last && fuse)
        launch_edge_ws<true>(a, m, s);
      else if (form == 2)
        launch_edge_ws<false>(a, m, s);
      else
        launch_any(h, fp8, last && fuse ? M_EDGE_UPD_CLS : M_EDGE_UPD, a, s, -1);
      if (last && !fuse) launch_any(h, fp8, M_CLS, a, s, -1);
    }
  }
  if (K == 0 && (stage < 0 || stage == 1)) launch_any(h, fp8, M_CLS, a, s, -1);
}

void tc_set_edge_form(int form) {
  g_edge_form.store(form >= 0 && form <= 2 ? form : 0, std::memory_order_relaxed);
}
int tc_get_edge_form() { return g_edge_form.load(std::memory_order_relaxed); }

void tc_make_maps(TcModel& m, const Ws& w, int h) {
  m.maps = false;
  if (h != 32 || w.estate16 == nullptr || w.hstate16 == nullptr) return;
  // the CUDA driver API encoder, looked up through the runtime (the library does not
  // link libcuda, so it loads on machines without a GPU driver)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      fn = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (encode == nullptr) return;
  const cuuint32_t es[2] = {1, 1};
  const cuuint64_t dim_e[2] = {cuuint64_t(h), cuuint64_t(w.e_cap)};
  const cuuint64_t dim_h[2] = {cuuint64_t(h), cuuint64_t(w.h_cap)};
  const cuuint64_t stride[1] = {cuuint64_t(h) * 2};  // bytes between rows
  const cuuint32_t box_e[2] = {cuuint32_t(h), cuuint32_t(kRows)};
  const cuuint32_t box_h[2] = {cuuint32_t(h), 1};  // one row high: row gathers
  CUresult r1 = encode(&m.map_e, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                       static_cast<void*>(w.estate16), dim_e, stride, box_e, es,
                                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = encode(&m.map_h, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                       static_cast<void*>(w.hstate16), dim_h, stride, box_h, es,
                                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  m.maps = r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

void tc_set_ctas(int precision, int h, int family, int n) {
  if (family < 0 || family > 3 || (h != 32 && h != 64 && h != 128)) return;
  g_tuned[precision == GNNTRK_FP8_E4M3 ? 1 : 0][hidx(h)][family].store(n < 0 ? 0 : n,
                                                                       std::memory_order_relaxed);
}

int tc_get_ctas(int precision, int h, int family) {
  if (family < 0 || family > 3 || (h != 32 && h != 64 && h != 128)) return 0;
  return g_tuned[precision == GNNTRK_FP8_E4M3 ? 1 : 0][hidx(h)][family].load(
      std::memory_order_relaxed);
}

void tc_triplet_scores(const Batch& b, const Ws& w, const TcModel& m, int h, const LayerF32& art2,
                       const LayerF32& elb2, const float* art_b1, const float* elb_b1,
                       float cut_logit, cudaStream_t s) {
  GraphParams g{};
  g.cut_logit = cut_logit;
  TcArgs a = base_args(b, w, g);
  // articulations
  a.W1 = static_cast<const uint8_t*>(m.art1.B);
  a.b1 = art_b1;
  a.c2 = art2;
  a.t1 = w.trip_a1;
  a.t2 = w.trip_a2;
  a.tn = w.counters + C_TRIP_A;
  a.tlogit = w.trip_alogit;
  a.tkeep = w.trip_akeep;
  launch_any(h, false, M_TRIP, a, s, -1);
  // elbows
  a.W1 = static_cast<const uint8_t*>(m.elb1.B);
  a.b1 = elb_b1;
  a.c2 = elb2;
  a.t1 = w.trip_e1;
  a.t2 = w.trip_e2;
  a.tn = w.counters + C_TRIP_E;
  a.tlogit = w.trip_elogit;
  a.tkeep = w.trip_ekeep;
  launch_any(h, false, M_TRIP, a, s, -1);
}

bool tc_cls_fused(int h, int precision) {
  const bool fp8 = precision == GNNTRK_FP8_E4M3;
  return (fp8 ? smem_total<true>(h, M_EDGE_UPD_CLS) : smem_total<false>(h, M_EDGE_UPD_CLS)) <= kMaxSmem;
}


namespace {
// Tensor-core throughput probe: one CTA per SM, one thread issuing BF16 MMAs
// M = 128, N = NN, K = 64 (four K = 16 instructions) back to back from shared
// memory (zeros, no-swizzle layout) into one tensor-memory accumulator, one
// commit at the end (bounded wait). Measures what the tensor pipe sustains at
// the narrow N of the interaction-network layers.
template <int NN>
__global__ void __launch_bounds__(32, 1) k_tc_probe(int64_t iters, int32_t* flag) {
  constexpr int K = 64;
  __shared__ __align__(1024) uint8_t sA[kRows * K * 2];
  __shared__ __align__(1024) uint8_t sB[NN * K * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  for (int i = threadIdx.x * 16; i < kRows * K * 2; i += 32 * 16)
    *reinterpret_cast<uint4*>(sA + i) = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x * 16; i < NN * K * 2; i += 32 * 16)
    *reinterpret_cast<uint4*>(sB + i) = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  tmem_alloc(&tslot, NN < 32 ? 32 : NN);
  tmem_relinquish();
  fence_proxy_async();
  tc_fence_before();
  __syncwarp();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    constexpr uint32_t IDESC = idesc_bf16(kRows, NN);
    constexpr uint32_t SBO = uint32_t(K * 2 / 16) * 128;
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < K; k += 16) {
        const uint32_t off = uint32_t(k * 2 / 16) * 128;
        mma_bf16(tmem, smem_desc(a0 + off, 128, SBO), smem_desc(b0 + off, 128, SBO), IDESC,
                 (it > 0 || k > 0) ? 1u : 0u);
      }
    }
    mma_commit(&bar);
    if (!mbar_wait_bounded(&bar, 0, kWaitCycles)) atomicExch(flag, 1);
  }
  tc_fence_before();
  __syncwarp();
  tc_fence_after();
  tmem_dealloc(tmem, NN < 32 ? 32 : NN);
}
}  // namespace

int tc_probe(int n, int64_t iters, double* ms) {
  int32_t* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int32_t)) != cudaSuccess) return GNNTRK_ERR_OOM;
  cudaMemset(flag, 0, sizeof(int32_t));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int grid = device_sms();
  auto go = [&](int64_t its) {
    if (n == 32) k_tc_probe<32><<<grid, 32>>>(its, flag);
    else if (n == 64) k_tc_probe<64><<<grid, 32>>>(its, flag);
    else if (n == 128) k_tc_probe<128><<<grid, 32>>>(its, flag);
    else k_tc_probe<256><<<grid, 32>>>(its, flag);
  };
  go(16);  // warm-up
  cudaEventRecord(a);
  go(iters);
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  int32_t hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(flag);
  if (e != cudaSuccess) return GNNTRK_ERR_CUDA;
  if (hflag) return GNNTRK_ERR_TIMEOUT;
  *ms = double(t);
  return GNNTRK_OK;
}

namespace {
// Self-test of the bounded waits: one thread waits on an mbarrier that no
// thread ever arrives on, through the same bounded wait the tensor-core
// kernels use, and latches ST_TIMEOUT when it runs out, as they do.
__global__ void k_wait_selftest(int32_t* counters, long long max_cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0, max_cycles)) set_status(counters, ST_TIMEOUT);
}
}  // namespace

void tc_wait_selftest(int32_t* counters, long long max_cycles, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(counters, max_cycles);
}

}  // namespace gnntrk

// ---------------------------------------------------------------------------
// E4M3 conversion entry points (host packing routine, device activation
// conversion), for checks of both against an independent codec
// ---------------------------------------------------------------------------
namespace gnntrk {
namespace {
__global__ void k_e4m3_encode(const float* in, uint8_t* out, int64_t n) {
  const int64_t pairs = (n + 1) / 2;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < pairs;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float a = in[2 * i];
    const float b = 2 * i + 1 < n ? in[2 * i + 1] : 0.f;
    const uint32_t c = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    out[2 * i] = uint8_t(c & 0xff);
    if (2 * i + 1 < n) out[2 * i + 1] = uint8_t(c >> 8);
  }
}
}  // namespace
void set_global_error(const std::string& msg);
}  // namespace gnntrk

extern "C" gnntrk_status gnntrk_e4m3_encode(const float* in, uint8_t* out, int64_t n,
                                            int32_t on_device, void* stream) {
  using namespace gnntrk;
  if (n < 0 || (n > 0 && (in == nullptr || out == nullptr))) {
    set_global_error("gnntrk_e4m3_encode: bad arguments");
    return GNNTRK_ERR_INVALID_ARG;
  }
  if (n == 0) return GNNTRK_OK;
  if (!on_device) {
    for (int64_t i = 0; i < n; ++i) out[i] = e4m3_from_float(in[i]);
    return GNNTRK_OK;
  }
  const int64_t pairs = (n + 1) / 2;
  const int grid = int(std::min<int64_t>(int64_t(device_sms()) * 8, (pairs + 255) / 256));
  k_e4m3_encode<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("gnntrk_e4m3_encode: ") + cudaGetErrorString(e));
    return GNNTRK_ERR_CUDA;
  }
  return GNNTRK_OK;
}

extern "C" gnntrk_status gnntrk_tc_throughput(int32_t n, int64_t iters, double* ms) {
  using namespace gnntrk;
  if (!ms || (n != 32 && n != 64 && n != 128 && n != 256) || iters < 1 || iters > (int64_t(1) << 30)) {
    set_global_error("gnntrk_tc_throughput: n must be 32, 64, 128 or 256, iters 1..2^30, ms not NULL");
    return GNNTRK_ERR_INVALID_ARG;
  }
  const int st = tc_probe(n, iters, ms);
  if (st != GNNTRK_OK) set_global_error("gnntrk_tc_throughput: the probe failed or timed out");
  return gnntrk_status(st);
}

extern "C" gnntrk_status gnntrk_e4m3_decode(const uint8_t* in, float* out, int64_t n) {
  using namespace gnntrk;
  if (n < 0 || (n > 0 && (in == nullptr || out == nullptr))) {
    set_global_error("gnntrk_e4m3_decode: bad arguments");
    return GNNTRK_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < n; ++i) out[i] = e4m3_to_float(in[i]);
  return GNNTRK_OK;
}
