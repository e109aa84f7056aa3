// Block-row products with float blocks (instantiations of k_blockrow.cuh).
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_f32(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) { dispatch_R<float>(d, cfg, s); }
}  // namespace hdg
