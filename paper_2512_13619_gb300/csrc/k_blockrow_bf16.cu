// Block-row products with BF16 blocks (instantiations of k_blockrow.cuh).
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_bf16(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) { dispatch_R<__nv_bfloat16>(d, cfg, s); }
}  // namespace hdg
