// Block-row products with bf16 blocks (instantiations of k_blockrow.cuh);
// four or eight right-hand sides are in k_blockrow_bf16_wide.cu.
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_bf16_wide(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);
void blockrow_bf16(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  if (d.R <= 2) dispatch_R_narrow<__nv_bfloat16>(d, cfg, s);
  else blockrow_bf16_wide(d, cfg, s);
}
}  // namespace hdg
