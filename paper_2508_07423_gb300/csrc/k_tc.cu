// Tensor-core path (placeholder until the tcgen05 kernels land).
#include "../../include/gnntrk.h"
#include "tc.cuh"

namespace gnntrk {

int tc_upload(TcModel&, const HostLayer*, int, int, int, int, int, void**, std::string& err) {
  err = "BF16/FP8 tensor-core path not built yet";
  return GNNTRK_ERR_UNSUPPORTED;
}
void tc_node_prep(const Batch&, const Ws&, const TcModel&, const LayerF32*, int, int, int,
                  const GraphParams&, cudaStream_t) {}
void tc_gnn(const Batch&, const Ws&, const TcModel&, int, int, const GraphParams&, cudaStream_t) {}
void tc_mark_band(const Batch&, const Ws&, float, float, cudaStream_t) {}

}  // namespace gnntrk
