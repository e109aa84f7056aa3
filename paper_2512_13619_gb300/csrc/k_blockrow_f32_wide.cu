// Block-row products with float blocks and four or eight right-hand sides
// (instantiations of k_blockrow.cuh).
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_f32_wide(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) { dispatch_R_wide<float>(d, cfg, s); }
}  // namespace hdg
