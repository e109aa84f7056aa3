// Block-row products with float blocks (instantiations of k_blockrow.cuh);
// four or eight right-hand sides are in k_blockrow_f32_wide.cu.
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_f32_wide(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);
void blockrow_f32(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  if (d.R <= 2) dispatch_R_narrow<float>(d, cfg, s);
  else blockrow_f32_wide(d, cfg, s);
}
}  // namespace hdg
