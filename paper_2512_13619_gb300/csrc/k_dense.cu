// Dense FP64 building blocks of the batched static condensation (Sec. 4.1,
// Eqs. w16-w22) and of the block-Jacobi / ASM factorizations (Sec. 4.5, 4.6):
// a batched GEMM and a batched Gauss-Jordan inverse with partial pivoting.
//
// FP64 on this GPU runs on the CUDA-core FP64 pipes (about 1.2 TFLOP/s
// measured), so both kernels are ALU-bound; they keep operands in shared
// memory and each thread owns a register tile sized to the product.
#include "hdg_common.cuh"
#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int BK = 16;

// Tile of (16*TM) x (16*TN) outputs per 256-thread CTA, each thread a TM x TN
// register block; the tile shape is picked per product so that the 64-, 96-,
// 135- or 162-wide operands of the condensation waste little work.
template <int TM, int TN>
__global__ void __launch_bounds__(256) gemm_f64_kernel(GemmDesc d) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int b0 = blockIdx.z / d.nb1, b1 = blockIdx.z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  double* C = d.C + b0 * d.sC0 + b1 * d.sC1;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < d.K; k0 += BK) {
#pragma unroll
    for (int t = 0; t < TM; ++t) {
      const int idx = threadIdx.x + t * 256;
      const int r = idx / BK, c = idx % BK;
      const int gr = row0 + r, gc = k0 + c;
      As[c][r] = (gr < d.M && gc < d.K) ? A[(int64_t)gr * d.lda + gc] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const int idx = threadIdx.x + t * 256;
      const int br = idx / BN, bcol = idx % BN;
      const int gbr = k0 + br, gbc = col0 + bcol;
      Bs[br][bcol] = (gbr < d.K && gbc < d.N) ? B[(int64_t)gbr * d.ldb + gbc] : 0.0;
    }
    __syncthreads();
    auto step = [&](int kk) {
      double a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    };
    // the last tile runs over its real depth only (the FP64 pipe is the bound)
    const int kc = d.K - k0 < BK ? d.K - k0 : BK;
    if (kc == BK) {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) step(kk);
    } else {
      for (int kk = 0; kk < kc; ++kk) step(kk);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + ty + 16 * i;
    if (gr >= d.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = col0 + tx + 16 * j;
      if (gc >= d.N) continue;
      const int64_t cc = (int64_t)(gc / d.cg) * d.cgs + (gc % d.cg);
      double* p = C + (int64_t)gr * d.ldc + cc;
      *p = (d.beta == 0.0 ? 0.0 : d.beta * *p) + d.alpha * acc[i][j];
    }
  }
}

// Small products (M <= 32, N <= 64, at most 8 outputs per thread): the 256
// threads own outputs o = tid, tid + 256, ... of the exact M x N product (no
// padding rows or columns computed: a partly masked FP64 instruction costs a
// full one), A and B staged through shared memory in K tiles of 32.
constexpr int kFlatK = 32;
template <int NO>
__global__ void __launch_bounds__(256) gemm_f64_flat_kernel(GemmDesc d) {
  __shared__ double As[32][kFlatK + 1];
  __shared__ double Bs[kFlatK][64 + 1];
  const int b0 = blockIdx.z / d.nb1, b1 = blockIdx.z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  double* C = d.C + b0 * d.sC0 + b1 * d.sC1;
  const int MN = d.M * d.N;
  int rr[NO], cc[NO];
  double acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    const int idx = threadIdx.x + 256 * o;
    rr[o] = idx < MN ? idx / d.N : 0;
    cc[o] = idx < MN ? idx - rr[o] * d.N : 0;
    acc[o] = 0.0;
  }
  for (int k0 = 0; k0 < d.K; k0 += kFlatK) {
    const int kc = d.K - k0 < kFlatK ? d.K - k0 : kFlatK;
    for (int t = threadIdx.x; t < d.M * kc; t += 256) {
      const int r = t / kc, c = t - r * kc;
      As[r][c] = A[(int64_t)r * d.lda + k0 + c];
    }
    for (int t = threadIdx.x; t < kc * d.N; t += 256) {
      const int r = t / d.N, c = t - r * d.N;
      Bs[r][c] = B[(int64_t)(k0 + r) * d.ldb + c];
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (threadIdx.x + 256 * o < MN) acc[o] = fma(As[rr[o]][kk], Bs[kk][cc[o]], acc[o]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (threadIdx.x + 256 * o >= MN) continue;
    const int64_t c = (int64_t)(cc[o] / d.cg) * d.cgs + (cc[o] % d.cg);
    double* p = C + (int64_t)rr[o] * d.ldc + c;
    *p = (d.beta == 0.0 ? 0.0 : d.beta * *p) + d.alpha * acc[o];
  }
}

// Products with few columns (N <= 8: the right-hand-side columns of
// Eqs. w19 and w22): one warp per output row, lanes striding over K, the N
// partial sums reduced with shuffles.
template <int NN>
__global__ void __launch_bounds__(256) gemm_f64_smalln_kernel(GemmDesc d) {
  const int z = blockIdx.x;
  const int b0 = z / d.nb1, b1 = z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  double* C = d.C + b0 * d.sC0 + b1 * d.sC1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = blockIdx.y * 8 + warp; r < d.M; r += gridDim.y * 8) {
    double acc[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[j] = 0.0;
    const double* arow = A + (int64_t)r * d.lda;
    for (int k = lane; k < d.K; k += 32) {
      const double a = arow[k];
      const double* brow = B + (int64_t)k * d.ldb;
#pragma unroll
      for (int j = 0; j < NN; ++j)
        if (j < d.N) acc[j] = fma(a, brow[j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[j] = warp_sum(acc[j]);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        if (j >= d.N) continue;
        const int64_t cc = (int64_t)(j / d.cg) * d.cgs + (j % d.cg);
        double* p = C + (int64_t)r * d.ldc + cc;
        *p = (d.beta == 0.0 ? 0.0 : d.beta * *p) + d.alpha * acc[j];
      }
    }
  }
}

template <int NN>
void gemm_smalln_launch(const GemmDesc& d, cudaStream_t s) {
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  const int gy = (d.M + 7) / 8 < 8 ? (d.M + 7) / 8 : 8;
  const int64_t xmax = (2147483647 / d.nb1) * d.nb1;   // launches start at a whole batch row b0
  for (int64_t z0 = 0; z0 < nb; z0 += xmax) {
    GemmDesc e = d;
    const int64_t nz = nb - z0 < xmax ? nb - z0 : xmax;
    if (z0 > 0) {
      e.nb0 = (int)(nz / d.nb1);
      e.A = d.A + (z0 / d.nb1) * d.sA0;
      e.B = d.B + (z0 / d.nb1) * d.sB0;
      e.C = d.C + (z0 / d.nb1) * d.sC0;
    }
    count_launch(); gemm_f64_smalln_kernel<NN><<<dim3((unsigned)nz, (unsigned)gy), 256, 0, s>>>(e);
  }
}

// tile factor (1, 2, 3, 4 or 6) that pads n least, preferring the larger tile on ties
int pick_tile(int n) {
  const int cand[5] = {6, 4, 3, 2, 1};
  int best = 2, bestpad = 1 << 30;
  for (int t : cand) {
    const int b = 16 * t;
    const int pad = (n + b - 1) / b * b - n;
    if (pad < bestpad) { bestpad = pad; best = t; }
  }
  return best;
}

template <int TM, int TN>
void gemm_launch(const GemmDesc& d, cudaStream_t s) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  const int64_t zmax = 65535;
  if (nb <= zmax) {
    dim3 grid((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, (unsigned)nb);
    count_launch(); gemm_f64_kernel<TM, TN><<<grid, 256, 0, s>>>(d);
    return;
  }
  const int per = (int)(zmax / d.nb1);
  for (int b0 = 0; b0 < d.nb0; b0 += per) {
    GemmDesc e = d;
    e.nb0 = (d.nb0 - b0 < per) ? d.nb0 - b0 : per;
    e.A = d.A + b0 * d.sA0;
    e.B = d.B + b0 * d.sB0;
    e.C = d.C + b0 * d.sC0;
    dim3 grid((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, (unsigned)((int64_t)e.nb0 * d.nb1));
    count_launch(); gemm_f64_kernel<TM, TN><<<grid, 256, 0, s>>>(e);
  }
}

template <int NO>
void gemm_flat_launch(const GemmDesc& d, cudaStream_t s) {
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  const int per = (int)(65535 / d.nb1);
  for (int b0 = 0; b0 < d.nb0; b0 += per) {
    GemmDesc e = d;
    e.nb0 = (d.nb0 - b0 < per) ? d.nb0 - b0 : per;
    e.A = d.A + b0 * d.sA0;
    e.B = d.B + b0 * d.sB0;
    e.C = d.C + b0 * d.sC0;
    (void)nb;
    count_launch(); gemm_f64_flat_kernel<NO><<<dim3(1, 1, (unsigned)((int64_t)e.nb0 * d.nb1)), 256, 0, s>>>(e);
  }
}

template <int TM>
void gemm_tn(const GemmDesc& d, int tn, cudaStream_t s) {
  switch (tn) {
    case 1: gemm_launch<TM, 1>(d, s); break;
    case 2: gemm_launch<TM, 2>(d, s); break;
    case 3: gemm_launch<TM, 3>(d, s); break;
    case 4: gemm_launch<TM, 4>(d, s); break;
    default: gemm_launch<TM, 6>(d, s); break;
  }
}

// ----------------------------------------------------------------- inverse
constexpr int kInvThreads = 256;
constexpr size_t kInvSmemMax = 227 * 1024;

__global__ void __launch_bounds__(kInvThreads) inverse_kernel(double* Aall, int n, int64_t stride, unsigned* err) {
  extern __shared__ double sm[];
  double* a = sm;                 // n x n row-major
  double* col = sm + n * n;       // n multipliers
  int* piv = reinterpret_cast<int*>(col + n);
  __shared__ int s_p;
  __shared__ double s_pv;
  double* A = Aall + blockIdx.x * stride;
  const int nn = n * n;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) a[i] = A[i];
  __syncthreads();
  bool singular = false;
  const int step_i = kInvThreads / n, step_j = kInvThreads - step_i * n;   // kInvThreads = step_i n + step_j
  for (int k = 0; k < n; ++k) {
    // pivot search (warp 0): largest |a[i][k]|, i >= k, lowest index on ties
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = n;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        double v = fabs(a[i * n + k]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (threadIdx.x == 0) { s_p = bi; }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double t = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = t;
      }
    }
    if (threadIdx.x == 0) piv[k] = p;
    __syncthreads();
    if (threadIdx.x == 0) s_pv = a[k * n + k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[i * n + k];
    __syncthreads();
    const double pv = s_pv;
    if (pv == 0.0 || !isfinite(pv)) { singular = true; break; }
    const double inv = 1.0 / pv;
    for (int j = threadIdx.x; j < n; j += blockDim.x) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * inv;
    __syncthreads();
    // entries idx = tid, tid + 256, ... of the row-major matrix, so every warp
    // but the last is full (a partly masked FP64 instruction costs a full
    // one); (i, j) advance by the fixed step without a division
    {
      const double* pk = a + k * n;
      int i = threadIdx.x / n, j = threadIdx.x - i * n;
      for (int idx = threadIdx.x; idx < nn; idx += kInvThreads) {
        if (i != k) {
          const double v = (j == k) ? 0.0 : a[idx];
          a[idx] = fma(-col[i], pk[j], v);
        }
        j += step_j;
        i += step_i;
        if (j >= n) {
          j -= n;
          ++i;
        }
      }
    }
    __syncthreads();
  }
  if (singular) {
    if (threadIdx.x == 0) atomicOr(err, ERRBIT_SINGULAR);
    return;
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double t = a[i * n + k];
        a[i * n + k] = a[i * n + p];
        a[i * n + p] = t;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nn; i += blockDim.x) A[i] = a[i];
}

size_t inverse_smem(int n) { return (size_t)n * n * 8 + (size_t)n * 8 + (size_t)n * 4 + 16; }

// dst[c][i][j] = src[c][i][j] for i < rows, j < cols (row-major, leading
// dimensions ldd / lds, batch strides sd / ss).  One CTA per matrix
// (grid-stride), one warp per row, the columns over the lanes: no index
// divisions, coalesced rows; blocks narrower than a warp go flat over the
// matrix instead.
__global__ void copy_block_kernel(double* dst, int64_t ldd, int64_t sd, const double* src, int64_t lds, int64_t ss,
                                  int rows, int cols, int64_t count) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t c = blockIdx.x; c < count; c += gridDim.x) {
    const double* sc = src + c * ss;
    double* dc = dst + c * sd;
    if (cols < 32) {                       // narrow blocks (right-hand-side columns): flat over the matrix
      for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
        const int i = t / cols, j = t - i * cols;
        dc[i * ldd + j] = sc[i * lds + j];
      }
      continue;
    }
    for (int i = warp; i < rows; i += nw) {
      const double* sr = sc + i * lds;
      double* dr = dc + i * ldd;
#pragma unroll 4
      for (int j = lane; j < cols; j += 32) dr[j] = sr[j];
    }
  }
}

}  // namespace

void copy_block_f64(double* dst, int64_t ldd, int64_t sd, const double* src, int64_t lds, int64_t ss, int rows,
                    int cols, int64_t count, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || count <= 0) return;
  const int64_t grid = std::min<int64_t>(count, 4096);   // grid-stride beyond
  count_launch();
  copy_block_kernel<<<(unsigned)grid, 256, 0, s>>>(dst, ldd, sd, src, lds, ss, rows, cols, count);
}

void gemm_f64(const GemmDesc& d, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.nb0 <= 0 || d.nb1 <= 0) return;
  if (d.N <= 2) { gemm_smalln_launch<2>(d, s); return; }
  if (d.N <= 4) { gemm_smalln_launch<4>(d, s); return; }
  if (d.N <= 8) { gemm_smalln_launch<8>(d, s); return; }
  if (d.M <= 32 && d.N <= 64) {
    const int no = (d.M * d.N + 255) / 256;       // <= 8
    switch (no) {
      case 1: gemm_flat_launch<1>(d, s); return;
      case 2: gemm_flat_launch<2>(d, s); return;
      case 3: gemm_flat_launch<3>(d, s); return;
      case 4: gemm_flat_launch<4>(d, s); return;
      case 5: case 6: gemm_flat_launch<6>(d, s); return;
      default: gemm_flat_launch<8>(d, s); return;
    }
  }
  const int tm = pick_tile(d.M), tn = pick_tile(d.N);
  switch (tm) {
    case 1: gemm_tn<1>(d, tn, s); break;
    case 2: gemm_tn<2>(d, tn, s); break;
    case 3: gemm_tn<3>(d, tn, s); break;
    case 4: gemm_tn<4>(d, tn, s); break;
    default: gemm_tn<6>(d, tn, s); break;
  }
}

int inverse_max_n() {
  int n = 1;
  while (inverse_smem(n + 1) <= kInvSmemMax - 1024) ++n;
  return n;
}

bool inverse_f64(double* A, int n, int64_t stride, int64_t count, unsigned* err, cudaStream_t s) {
  if (n <= 0 || count <= 0) return true;
  size_t smem = inverse_smem(n);
  if (smem > kInvSmemMax - 1024) return false;
  cudaFuncSetAttribute(inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kInvSmemMax - 1024));
  const int64_t gmax = 2147483647;
  for (int64_t c0 = 0; c0 < count; c0 += gmax) {
    int64_t c = count - c0 < gmax ? count - c0 : gmax;
    count_launch(); inverse_kernel<<<(unsigned)c, kInvThreads, smem, s>>>(A + c0 * stride, n, stride, err);
  }
  return true;
}

}  // namespace hdg
