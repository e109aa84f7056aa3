// Entry points of the block-row products (face-block matvec, block-Jacobi
// apply, additive-Schwarz element solves): dispatch by block precision to the
// per-precision units, the FP32 copy of x, and the candidate launch
// configurations the autotuner times.  The kernels are in k_blockrow.cuh.
#include "k_blockrow.cuh"

namespace hdg {

void blockrow_f64(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);
void blockrow_f32(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);
void blockrow_bf16(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);

namespace {
__global__ void to_f32_kernel(const double* x, float* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
}  // namespace

int blockrow_candidates(const BlockRowDesc& d, BrCfg* out, int cap) {
  if (d.prec == HDG_FP64) return candidates_T<double>(d, out, cap);
  if (d.prec == HDG_FP32) return candidates_T<float>(d, out, cap);
  return candidates_T<__nv_bfloat16>(d, out, cap);
}

int blockrow_variants() { return 2; }

void to_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  count_launch(); to_f32_kernel<<<(unsigned)g, 256, 0, s>>>(x, y, n);
}

void blockrow(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  if (d.n_units <= 0) return;
  if (d.prec == HDG_FP64) blockrow_f64(d, cfg, s);
  else if (d.prec == HDG_FP32) blockrow_f32(d, cfg, s);
  else blockrow_bf16(d, cfg, s);
}

}  // namespace hdg
