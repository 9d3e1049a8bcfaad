// Internal declarations shared by the CUDA translation units of libgnntrk.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace gnntrk {

constexpr int kMaxPlanes = 64;
constexpr int kMaxEmbedLayers = 8;
constexpr int kMaxIters = 16;
constexpr float kLnEps = 1e-5f;

// Bits of the device status word (counters[C_STATUS]).
enum StatusBits : int {
  ST_INPUT = 1,     // an input value out of range (plane id, offsets)
  ST_CAPACITY = 2,  // more edges than the edge workspace
  ST_TIMEOUT = 4,   // a bounded wait ran out
  ST_INTERNAL = 8,  // an internal consistency check failed
};

// Slots of the device counter array.
enum Counter : int {
  C_EDGES = 0,     // total edges of the last call (may exceed capacity)
  C_STATUS = 1,    // status bits
  C_TICKET = 2,    // last-block ticket of the two-kernel scan
  C_KEPT = 3,      // kept edges
  C_BAND = 4,      // edges in the re-score band
  C_RERUN = 5,     // events holding a band edge
  C_RERUN_EDGES = 7,  // edges the FP32 re-score recomputes (receptive field)
  C_RERUN_HITS = 8,   // hits the FP32 re-score recomputes
  C_TRIP_A = 9,       // articulations of the last call
  C_TRIP_E = 10,      // elbows of the last call
  C_TRACKS = 11,      // tracks built from triplets
  C_TRACK_HITS = 12,  // hits over all those tracks
  C_TRIP_KEPT = 13,   // triplets above the triplet cut
  C_GRAPH_TICKET = 14,  // next event of the graph kernel
  C_RS_TICKET = 15,     // next event of the re-score receptive-field kernel
  C_COUNT = 16
};

// A layer as parsed from the weight blob (host memory).
struct HostLayer {
  int in = 0, out = 0;
  std::vector<float> W;  // [out][in]
  std::vector<float> b;  // [out]
};

// One FP32 linear layer in the SIMT layout: WT[in][ldo] (transposed, output
// dimension padded to a multiple of 4 with zeros) and b[ldo].
struct LayerF32 {
  const float* WT;
  const float* b;
  int in, out, ldo;
};

struct Mlp2F32 {
  LayerF32 l1, l2;
};

// One layer packed for tcgen05: B operand (W[out][in], K-major) in the
// no-swizzle canonical layout of 8x16-byte core matrices, the FP32 bias and,
// for FP8, the per-output-channel dequantisation scale.
struct LayerTC {
  const void* B;       // packed operand image, bytes = out * in * elem_size
  const float* b;      // [out]
  const float* scale;  // [out], FP8 only (else nullptr)
  int in, out;
};

struct Mlp2TC {
  LayerTC l1, l2;
};

// Device workspace of a handle.
struct Ws {
  int32_t* perm;        // [H] sorted position -> global input index
  int32_t* node_event;  // [H] sorted position -> event
  float4* pos;          // [H] sorted (x, y, z, 0)
  int32_t* plane_off;   // [max_events][n_planes + 1] sorted offsets (global)
  float* emb;           // [H][D]
  int32_t* deg;         // [H] candidates inside the radius (uncapped), large events
  unsigned long long* graph_desc;  // [max_events] look-back words of the graph kernel
  int32_t* row_ptr;     // [H + 1]
  int32_t* col;         // [Ecap] target (sorted position)
  int32_t* src;         // [Ecap] source (sorted position)
  float* d2;            // [Ecap]
  int32_t* in_cnt;      // [H] CSR offsets, then in-degrees (large events)
  int32_t* in_ptr;      // [H + 1]
  int32_t* in_edge;     // [Ecap] edge ids grouped by target, ascending
  float* hstate;        // [H][h]   FP32 node state (FP32 path and re-score)
  float* estate;        // [Ecap][h] FP32 edge state
  float* pstate;        // [H][2h]  FP32 node projections for the next edge layer
  __nv_bfloat16* hstate16;  // [H][h]   BF16 node state (tensor-core paths)
  __nv_bfloat16* estate16;  // [Ecap][h] BF16 edge state
  float* hamax;         // [H] largest |BF16 node state| per hit (FP8 handles at h = 128)
  float* logit;         // [Ecap]
  uint8_t* keep;        // [Ecap]
  int32_t* parent;      // [H] union-find parent over global input indices
  int32_t* counters;    // [C_COUNT]
  int32_t* scan_blocks; // block partials of the scan
  int8_t* rs_elev;      // [Ecap] re-score level of each edge + 2 (0 none)
  int8_t* rs_nlev;      // [H]    re-score level of each hit + 2 (0 none)
  int32_t* rs_elist;    // [K + 1][Ecap] rows of each re-score step, index order
  int32_t* rs_nlist;    // [K + 1][H]    hits of each re-score step, index order
  int32_t* rs_counts;   // [6][kMaxIters + 2]: [2] and [5] rows with level >= k (edges, hits)
  int32_t* rs_desc;     // [max_events][1 + 4 (kMaxIters + 1)] look-back flags and counts of the lists
  int64_t* ev_off;      // [max_events + 1] copy of the call's offsets
  // triplet stage (allocated when the handle builds tracks from triplets)
  int32_t* trip_cnt_a;  // [H] articulations per hit
  int32_t* trip_cnt_e;  // [H] elbows per hit
  int32_t* trip_off_a;  // [H + 1]
  int32_t* trip_off_e;  // [H + 1]
  int32_t* trip_a1;     // [Tcap] articulation: edge A -> C
  int32_t* trip_a2;     // [Tcap]               edge C -> B
  float* trip_alogit;   // [Tcap]
  uint8_t* trip_akeep;  // [Tcap]
  int32_t* trip_e1;     // [Tcap] elbow: edge to / from the nearer far hit
  int32_t* trip_e2;     // [Tcap]        the other edge
  uint8_t* trip_et;     // [Tcap] 1 left elbow, 2 right elbow
  float* trip_elogit;   // [Tcap]
  uint8_t* trip_ekeep;  // [Tcap]
  int32_t* tb_par;      // [Ecap] edge groups (union-find)
  int32_t* tb_par2;     // [Ecap] components of groups (union-find)
  int32_t* tb_out;      // [Ecap] first group linked onwards
  int32_t* tb_in;       // [Ecap] first group linked from
  int32_t* tb_flag;     // [Ecap] 1 several onwards, 2 several from, 4 in a shared pair
  int32_t* tb_cnt;      // [Ecap] hits of a component
  int32_t* tb_off;      // [Ecap] its hit list in tb_hits
  int32_t* tb_cur;      // [Ecap] placement cursor
  int32_t* tb_hits;     // [2 Ecap] component hit lists (sorted positions)
  unsigned long long* tb_pairs;  // [Tcap] component pairs of shared links
  int32_t* tb_ev_tracks;   // [max_events]
  int32_t* tb_ev_hits;     // [max_events]
  int32_t* tb_ev_pairs;    // [max_events]
  int32_t* tb_ev_hit_off;  // [max_events + 1]
  int64_t h_cap, e_cap, t_cap;
};

// The current call.
struct Batch {
  int n_events;
  int n_hits;
  const float* x;
  const float* y;
  const float* z;
  const uint8_t* plane;
  const int64_t* offsets;
  int32_t* labels;
};

struct GraphParams {
  int n_planes;
  int k_max;
  float radius2;
  float cut_logit;
  float fs[6];
};

// Row selection of a row-parallel kernel: all rows of the batch (rows ==
// nullptr), or the rows rows[0 .. *n_rows) (device memory).
struct Sel {
  const int32_t* rows;
  const int32_t* n_rows;
};

// Levels of the FP32 re-score (exact receptive field of the edges whose logit
// lies in (band_lo, band_hi)): a row of level >= k is recomputed at step k
// (k = -1: the encoders); one block per event. Also the row lists of every
// step: list k + 1 of w.rs_elist ([K + 1][e_cap]) and w.rs_nlist ([K + 1][h_cap])
// holds the rows of step k in index order, their counts at
// rs_counts[2 (kMaxIters + 2) + k + 1] (edges) and rs_counts[5 (kMaxIters + 2) +
// k + 1] (hits). Counts the band edges (counters[C_BAND]), the events holding
// one (counters[C_RERUN]) and the encoder rows (C_RERUN_EDGES, C_RERUN_HITS).
// Returns the number of kernels launched.
int launch_rescore_sets(const Batch& b, const Ws& w, float band_lo, float band_hi, int K,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// launchers (host functions), one per kernel family
// ---------------------------------------------------------------------------
void launch_sort(const Batch& b, const Ws& w, int n_planes, cudaStream_t s);
// Column blocks of an edge layer's first Linear for the inputs h_src and
// h_dst (views into its transposed weights, zero bias): the node kernels
// project each node once, P[v] = [W_src h_v, W_dst h_v], and the edge kernels
// gather P[src] and P[dst] instead of multiplying h_src and h_dst per edge.
struct EdgeProj {
  LayerF32 src, dst;
};

// embedding (when do_embed) and FP32 node encoder (when do_node_enc), the
// encoder also writing the projections for the edge encoder
void launch_node_prep_f32(const Batch& b, const Ws& w, const LayerF32* embed, int n_embed,
                          const Mlp2F32& node_enc, const EdgeProj& proj, int D, int h,
                          const GraphParams& g, bool do_embed, bool do_node_enc, Sel sel,
                          cudaStream_t s);
// rough graph (CSR: row_ptr, col, src, d2; counters[C_EDGES]) and the in-edge
// index (in_ptr, in_edge), one kernel
void launch_graph(const Batch& b, const Ws& w, const GraphParams& g, int D, cudaStream_t s);
// exclusive scan of n entries of `in` (each clamped to clamp_max) into out[0..n],
// out[n] = total; the total also goes to counters[total_slot] and is checked
// against `cap` (ST_CAPACITY when above).
void launch_scan(const int32_t* in, int32_t* out, int n, int clamp_max, int32_t* counters,
                 int total_slot, int64_t cap, int32_t* blocks, cudaStream_t s);

// FP32 SIMT interaction network
void launch_edge_enc_f32(const Batch& b, const Ws& w, const Mlp2F32& m, int h, Sel sel,
                         cudaStream_t s);
// messages of a node step, m_v = [sum of e over out edges, sum over in edges]
// (FP32, into the node's projection row), for the selected hits
void launch_messages_f32(const Batch& b, const Ws& w, int h, Sel sel, cudaStream_t s);
// node step (after launch_messages_f32), also writing the projections for the
// edge step that follows
void launch_node_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, const EdgeProj& proj,
                            int h, Sel sel, cudaStream_t s);
// last step (cls != nullptr): also runs the classifier and writes logit/keep;
// with rescore_only, only edges whose current logit lies in (band_lo, band_hi)
// take the new FP32 logit and decision.
void launch_edge_update_f32(const Batch& b, const Ws& w, const Mlp2F32& m, const Mlp2F32* cls,
                            int h, float cut_logit, bool rescore_only, float band_lo,
                            float band_hi, Sel sel, cudaStream_t s);

// FP32 tile-shape variant (0 or 1) per kernel family (0 encoders, 1 node step,
// 2 edge step + classifier), process wide; chosen by the autotuner.
void f32_set_variant(int h, int family, int v);

// connected components
void launch_cc(const Batch& b, const Ws& w, cudaStream_t s);

// INT8 embedding (post-training quantisation)
struct Int8Layer {
  const uint32_t* Wq;  // [out][in16 * 4] weight codes, 4 per word along K, zero padded
  const float* s;      // [out] dequantisation scale (alpha / 127) S_w
  const float* b;      // [out] bias
  int in4, in16, out;  // input words (padded to 1, 2, 4, ..., 64), int4 per row, outputs
};
struct Int8Embed {
  Int8Layer l[kMaxEmbedLayers];
  const float* inv;  // [n] 127 / alpha of every layer's input
  int n, max_in4;
};
struct EmbedAmax {
  LayerF32 l[kMaxEmbedLayers];
  int n;
};
void launch_embed_int8(const Batch& b, const Ws& w, const Int8Embed& m, int D,
                       const GraphParams& g, cudaStream_t s);
// max calibration over n_hits input hits (device xyz [3][n_hits]); the largest
// |input| of each embedding layer as float bits in amax_bits[layer]
void launch_embed_amax(const float* xyz, int n_hits, const EmbedAmax& m, const GraphParams& g,
                       int32_t* amax_bits, cudaStream_t s);

// triplet stage
struct TripletHeads {
  Mlp2F32 art, elb;  // articulation and elbow classifiers (2h -> h -> 1)
};
struct TrackOut {
  int32_t* ev_tracks;   // [n_events + 1] tracks of event e: [ev_tracks[e], ev_tracks[e+1])
  int64_t* track_off;   // [max_tracks + 1] hits of track t: [track_off[t], track_off[t+1])
  int32_t* track_hits;  // [max_hits] event-local input indices
  int64_t max_tracks, max_hits;
};
// triplet lists of the kept edges
void launch_triplets(const Batch& b, const Ws& w, int h, cudaStream_t s);
// triplet classifiers on the FP32 path (FP32 final edge encodings; the
// warp-tile FP32 kernels in triplet mode)
void launch_triplet_scores_f32(const Batch& b, const Ws& w, const TripletHeads& t, int h,
                               float cut_logit, cudaStream_t s);
// count of the triplets above the cut (after either classifier path)
void launch_triplet_kept(const Ws& w, cudaStream_t s);
// track building into `out`
void launch_track_build(const Batch& b, const Ws& w, const TrackOut& out, cudaStream_t s);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* counters, int bits) {
  atomicOr(&counters[C_STATUS], bits);
}

__device__ __forceinline__ int clamp_edges(const int32_t* counters, int64_t cap) {
  int e = counters[C_EDGES];
  return e < cap ? e : int(cap);
}

inline int div_up(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// Positions [lo, hi) this kernel works on under `sel` (false: nothing to do);
// position i is row sel_row(sel, i).
__device__ __forceinline__ bool sel_rows(const Batch& b, const Ws& w, Sel sel, bool edges,
                                         int& lo, int& hi) {
  lo = 0;
  hi = edges ? clamp_edges(w.counters, w.e_cap) : b.n_hits;
  if (sel.rows != nullptr) hi = min(hi, *sel.n_rows);
  return hi > 0;
}

__device__ __forceinline__ int sel_row(Sel sel, int pos) {
  return sel.rows != nullptr ? sel.rows[pos] : pos;
}

}  // namespace gnntrk
