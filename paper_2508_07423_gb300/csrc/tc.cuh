// Tensor-core (tcgen05) path: BF16 and FP8-E4M3 operands, FP32 accumulation
// in tensor memory. Interface used by the C ABI.
#pragma once

#include "internal.cuh"

namespace gnntrk {

// Packed weights of the whole model for the tensor-core kernels.
struct TcModel {
  int precision = 0;  // GNNTRK_BF16 or GNNTRK_FP8_E4M3
  int h = 0, K = 0, n_embed = 0;
  LayerTC embed[kMaxEmbedLayers]{};
  Mlp2TC node_enc{}, edge_enc{}, cls{}, node[kMaxIters]{}, edge[kMaxIters]{};
};

// Pack the layers (blob order) for the tensor cores and upload them to one
// device allocation (*dmem, freed by the caller). Returns a gnntrk_status.
int tc_upload(TcModel& m, const HostLayer* L, int n_layers, int n_embed, int h, int K,
              int precision, void** dmem, std::string& err);

// Embedding (FP32 first layer, tensor-core hidden layers) and node encoder;
// writes w.emb (FP32) and w.hstate16.
void tc_node_prep(const Batch& b, const Ws& w, const TcModel& m, const LayerF32* embed_f32,
                  int n_embed, int D, int h, const GraphParams& g, cudaStream_t s);

// Edge encoder, K message-passing steps and the classifier with the cut;
// writes w.logit and w.keep.
void tc_gnn(const Batch& b, const Ws& w, const TcModel& m, int h, int K, const GraphParams& g,
            cudaStream_t s);

// Count the edges whose logit lies in (band_lo, band_hi) and list the events
// holding one (w.rerun_list, count in counters[C_RERUN]).
void tc_mark_band(const Batch& b, const Ws& w, float band_lo, float band_hi, cudaStream_t s);

}  // namespace gnntrk
