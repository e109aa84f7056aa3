// Block-row products with bf16 blocks and four or eight right-hand sides
// (instantiations of k_blockrow.cuh).
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_bf16_wide(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) { dispatch_R_wide<__nv_bfloat16>(d, cfg, s); }
}  // namespace hdg
