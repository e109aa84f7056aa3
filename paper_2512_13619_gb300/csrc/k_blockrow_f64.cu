// Block-row products with double blocks (instantiations of k_blockrow.cuh).
#include "k_blockrow.cuh"

namespace hdg {
void blockrow_f64(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) { dispatch_R<double>(d, cfg, s); }
}  // namespace hdg
