// Tensor-core (tcgen05) path: BF16 and FP8-E4M3 operands, FP32 accumulation
// in tensor memory. Interface used by the C ABI.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace gnntrk {

// Packed weights of the whole model for the tensor-core kernels.
struct TcModel {
  int precision = 0;  // GNNTRK_BF16 or GNNTRK_FP8_E4M3
  int h = 0, K = 0, n_embed = 0;
  LayerTC embed[kMaxEmbedLayers]{};
  Mlp2TC node_enc{}, edge_enc{}, cls{}, node[kMaxIters]{}, edge[kMaxIters]{};
  // FP8: BF16 split-operand encoders (node_enc16.l2, edge_enc16.l1 and .l2
  // hold BF16 images; edge_enc16.l1 repeated along K up to hidden 64, plain at
  // 128 where the edge encoder runs its layer 1 in two passes)
  Mlp2TC node_enc16{}, edge_enc16{};
  bool enc16 = false;
  // first layers of the triplet classifiers (BF16 images in every precision)
  LayerTC art1{}, elb1{};
  bool has_trip = false;
  // TMA tensor maps of the handle's BF16 states at hidden 32: the edge states
  // (boxes of 128 rows) and the node states (one-row boxes for row gathers),
  // both in the 64-byte swizzle layout; valid when `maps` is set
  CUtensorMap map_e{}, map_h{};
  bool maps = false;
};

// Encode the tensor maps of a BF16 handle's workspace (hidden 32); on failure
// the TMA edge step stays unavailable and the per-thread copies run.
void tc_make_maps(TcModel& m, const Ws& w, int h);

// BF16 edge-step form at hidden 32, process wide: 0 per-thread row copies, 1
// TMA tile load and row gathers, 2 the same loads in a ring with producer,
// MMA and epilogue warps (1 and 2 only where the handle has tensor maps).
void tc_set_edge_form(int form);
int tc_get_edge_form();

// Pack the layers (blob order) for the tensor cores and upload them to one
// device allocation (*dmem, freed by the caller). Returns a gnntrk_status.
int tc_upload(TcModel& m, const HostLayer* L, int n_layers, int n_embed, int h, int K,
              int precision, void** dmem, std::string& err);

// Pack the first layers of the triplet classifiers (BF16) into their own
// device allocation (*dmem, freed by the caller). Returns a gnntrk_status.
int tc_upload_triplets(TcModel& m, const HostLayer& art1, const HostLayer& elb1, void** dmem,
                       std::string& err);

// Triplet classifiers on the tensor cores: [e^K(e1), e^K(e2)] (BF16) times
// the first layer, LayerNorm and ReLU in the epilogue, the 1-unit second
// layer (FP32) as a dot product; writes the logits and keep flags of both
// triplet lists.
void tc_triplet_scores(const Batch& b, const Ws& w, const TcModel& m, int h, const LayerF32& art2,
                       const LayerF32& elb2, const float* art_b1, const float* elb_b1,
                       float cut_logit, cudaStream_t s);

// FP32 embedding (its output feeds the radius test) and the node encoder
// (FP32 K = 3 first layer, tensor-core second layer); writes w.emb and
// w.hstate16.
void tc_node_prep(const Batch& b, const Ws& w, const TcModel& m, const LayerF32* embed_f32,
                  int n_embed, int D, int h, const GraphParams& g, const LayerF32& ne1_f32,
                  cudaStream_t s, bool do_embed = true);

// Messages of a node step from the BF16 edge states (FP32 sums, stored
// rounded to BF16 for BF16 handles and in FP32 for FP8 handles), for every hit.
void tc_messages(const Batch& b, const Ws& w, int h, bool fp8, cudaStream_t s);

// Edge encoder, K message-passing steps and the classifier with the cut;
// writes w.logit and w.keep. stage < 0 runs everything (messages included);
// otherwise only stage 0 (edge encoder), 1 + 2k (node step k, after
// tc_messages) or 2 + 2k (edge step k, with the classifier at the last step;
// stage 1 is the classifier when K = 0).
// With store_final the last edge step stores e^K (BF16) and the classifier
// runs as its own kernel (the triplet classifiers read e^K).
void tc_gnn(const Batch& b, const Ws& w, const TcModel& m, int h, int K, const GraphParams& g,
            const LayerF32& cls2_f32, cudaStream_t s, int stage, bool store_final = false);

// Autotuner hooks: resident CTAs per SM for a tensor-core kernel family
// (0 node encoder, 1 edge encoder, 2 node step, 3 edge step + classifier) at a
// precision and hidden width, shared by every handle of the process; n = 0
// restores the resource bound.
void tc_set_ctas(int precision, int h, int family, int n);
int tc_get_ctas(int precision, int h, int family);

// Whether the classifier runs inside the last edge step (shared memory fits).
bool tc_cls_fused(int h, int precision);

// Host reference codec of E4M3 (used to pack weights).
uint8_t e4m3_from_float(float f);
float e4m3_to_float(uint8_t c);


// Tensor-core throughput probe (gnntrk_tc_throughput): device ms of SMs x
// iters x 4 BF16 MMAs of M = 128, N = n, K = 16; returns a gnntrk_status.
int tc_probe(int n, int64_t iters, double* ms);

// Launch the bounded-wait self-test: a wait on an mbarrier nothing arrives on,
// for at most max_cycles SM cycles, then ST_TIMEOUT in counters.
void tc_wait_selftest(int32_t* counters, long long max_cycles, cudaStream_t s);

}  // namespace gnntrk
