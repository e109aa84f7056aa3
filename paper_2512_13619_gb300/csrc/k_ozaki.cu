// FP64-accurate batched GEMM on the BF16 tensor cores (tcgen05.mma with TMEM
// accumulators), for the dense products of the batched static condensation
// (Sec. 4.1, Eqs. w16-w22).
//
// FP64 arithmetic on this GPU runs at about 1.2 TFLOP/s, 1/1800 of the dense
// BF16 tensor rate, so the FP64 products are computed exactly in pieces on
// the tensor cores (error-free operand splitting in the manner of Ozaki et
// al.):
//
//  * every row i of A is written in fixed point relative to a power of two
//    2^{e_i} above its largest entry, with 56 fraction bits, as 8 signed
//    7-bit digits: A_ik = 2^{e_i - 1078} sum_s a^s_ik 2^{7(8-s)}, |a^s| <= 127
//    (the same for every column j of B with 2^{f_j});
//  * a digit is an integer of at most 7 bits, exact in BF16, and the product
//    of two digits (< 2^14) is exact in the FP32 accumulator;
//  * products with the same digit weight s + t = d are summed into one TMEM
//    accumulator D_d, d = 2..9 (36 digit products; pairs with s + t > 9 only
//    carry weight below 2^-56 and are dropped).  For K <= 192 the integer sums
//    of D_2..D_6 stay below 2^24 and are exact; D_7..D_9 carry weight below
//    2^-35 and their FP32 rounding stays below the FP64 rounding of the result;
//  * the epilogue combines the accumulators as integers,
//    H = sum_{d<=5} D_d 2^{7(5-d)} and L = sum_{d>=6} D_d 2^{7(9-d)}, and forms
//    (A B)_ij = (H 2^28 + L) 2^{e_i + f_j - 2107} in FP64.
//
// The truncation to 56 bits and the dropped digit products are bounded by
// 2^-55 K 2^{e_i} 2^{f_j} in absolute value, within a small factor of the
// FP64 rounding of a dot product; the result is rounded once to FP64.
//
// One 256-thread CTA computes a 128 x NT output tile (NT <= 64) of one batch
// item.  K is staged 32 columns at a time through two shared-memory stages:
// all threads load FP64 operands, split them into digits and write the BF16
// digit matrices in the UMMA no-swizzle K-major layout (8 x 16-byte core
// matrices), then one thread issues the 72 MMAs of the stage
// (M = 128, N = NT, K = 16) and commits them to the stage's mbarrier, so the
// split of stage c+1 overlaps the MMAs of stage c.  The 8 accumulators use
// 8 NT TMEM columns.
#include <algorithm>

#include "hdg_common.cuh"
#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kSlices = 8;            // 7-bit digits per operand (56 bits)
constexpr int kAcc = kSlices;         // accumulators D_2 .. D_9
constexpr int kBM = 128;              // UMMA M
constexpr int kMaxNT = 64;
constexpr int kKC = 32;               // K per stage
constexpr int kThreads = 256;
constexpr int kMaxK = 192;            // exactness bound of D_2..D_6 (see above)
constexpr int kSliceA = kBM * kKC * 2;       // bytes of one A digit matrix per stage (8 KB)
constexpr int kSliceB = kMaxNT * kKC * 2;    // bytes of one B digit matrix per stage (4 KB)
constexpr int kStage = kSlices * (kSliceA + kSliceB);
constexpr int kSmem = 2 * kStage + 1024;

// UMMA shared-memory descriptor, no swizzle, K-major: core matrices of
// 8 rows x 16 bytes; LBO = byte distance of core matrices along K, SBO =
// along M/N; bit 46 = descriptor version of this architecture.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive TMEM columns of the warp's 32 lanes -> 8 registers per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// biased exponent field of an FP64 value (0 for zero, 2047 for Inf/NaN)
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// |x| in fixed point with 56 fraction bits relative to 2^(e - 1022), e the
// largest exponent field of its row / column (truncated below 2^-56)
__device__ __forceinline__ uint64_t fixed56(double x, int e) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) return 0;                 // zero / subnormal (below 2^-1022) / Inf, NaN (flagged)
  const uint64_t m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = ex - e + 3;                            // <= 3
  if (sh >= 0) return m << sh;
  if (sh <= -64) return 0;
  return m >> (-sh);
}

// x 2^sc in FP64 for an integer |x| < 2^53, exact, assembled from its bits;
// ok = false when the result would leave the normal range.
__device__ __forceinline__ double i2d_scaled(long long x, int sc, bool& ok) {
  if (x == 0) return 0.0;
  const unsigned long long u = (unsigned long long)(x < 0 ? -x : x);
  const int p = 63 - __clzll((long long)u);
  const int ef = p + 1023 + sc;
  if (ef < 1 || ef > 2046) {
    ok = false;
    return 0.0;
  }
  const unsigned long long bits = ((unsigned long long)(x < 0) << 63) | ((unsigned long long)ef << 52) |
                                  ((u << (52 - p)) & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// digit value +-d (0 <= d <= 127) as BF16 bits
__device__ __forceinline__ uint32_t digit_bf16(uint32_t d, uint32_t neg) {
  const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;   // exactly d
  return (__float_as_uint(f) >> 16) | neg;
}

// Splits 8 values (one core-matrix row of 8 K entries) into the 8 digit
// matrices: 16 bytes per digit at dst + s * slice_bytes.
__device__ __forceinline__ void split8(const double (&v)[8], int e, unsigned char* dst, int slice_bytes,
                                       bool& bad) {
  uint64_t F[8];
  uint32_t neg[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (exp_field(v[j]) == 0x7FF) bad = true;
    F[j] = fixed56(v[j], e);
    neg[j] = (uint32_t)((uint64_t)__double_as_longlong(v[j]) >> 63) << 15;
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const int sh = 7 * (kSlices - 1 - s);
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t d0 = (uint32_t)(F[2 * q] >> sh) & 127u;
      const uint32_t d1 = (uint32_t)(F[2 * q + 1] >> sh) & 127u;
      w[q] = digit_bf16(d0, d0 ? neg[2 * q] : 0u) | (digit_bf16(d1, d1 ? neg[2 * q + 1] : 0u) << 16);
    }
    *reinterpret_cast<uint4*>(dst + (size_t)s * slice_bytes) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// byte offset of (row, k) in a digit matrix with kKC K entries per row:
// core matrix (row/8, k/8) at (row/8)*SBO + (k/8)*LBO, row r%8 at +16 r
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = (kKC / 8) * 128;
__device__ __forceinline__ int core_off(int row, int kgrp) { return (row >> 3) * kSBO + kgrp * kLBO + (row & 7) * 16; }

// Per batch item: the largest exponent field of every row of A and of every
// column of B (over all of K), as 16-bit integers; flags Inf / NaN inputs.
__global__ void __launch_bounds__(256) ozaki_exponents_kernel(GemmDesc d, uint16_t* ea, uint16_t* fb,
                                                              unsigned* err) {
  const int z = blockIdx.x;
  const int b0 = z / d.nb1, b1 = z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad = false;
  for (int r = warp; r < d.M; r += 8) {
    int m = 0;
    const double* row = A + (int64_t)r * d.lda;
#pragma unroll 8
    for (int k = lane; k < d.K; k += 32) m = max(m, exp_field(row[k]));
    bad |= (m == 0x7FF);
    m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
    if (lane == 0) ea[(int64_t)z * d.M + r] = (uint16_t)m;
  }
  for (int n = threadIdx.x; n < d.N; n += 256) {
    int m = 0;
#pragma unroll 8
    for (int k = 0; k < d.K; ++k) m = max(m, exp_field(B[(int64_t)k * d.ldb + n]));
    bad |= (m == 0x7FF);
    fb[(int64_t)z * d.N + n] = (uint16_t)m;
  }
  if (bad) atomicOr(err, ERRBIT_NAN);
}

// FP64 operands of one stage in registers: 2 core rows of A (8 K entries
// each) and 1 core row of B per thread.
struct StageRegs {
  double a[2][8];
  double b[8];
};

__device__ __forceinline__ void load_stage(const GemmDesc& d, const double* A, const double* B, int row0, int col0,
                                           int NT, int k0, int tid, StageRegs& R) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int r = u >> 2, h = u & 3;
    const int gr = row0 + r;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * h + j;
      R.a[i][j] = (gr < d.M && k < d.K) ? __ldg(A + (int64_t)gr * d.lda + k) : 0.0;
    }
  }
  {
    const int n = tid % kMaxNT, h = tid / kMaxNT;
    const int gc = col0 + n;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * h + j;
      R.b[j] = (n < NT && gc < d.N && k < d.K) ? __ldg(B + (int64_t)k * d.ldb + gc) : 0.0;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) gemm_ozaki_kernel(GemmDesc d, int NT, const uint16_t* ea,
                                                                  const uint16_t* fb, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stage_base = smem;
  int* e_row = reinterpret_cast<int*>(smem + 2 * kStage);           // [128]
  int* f_col = e_row + kBM;                                          // [64]
  uint64_t* bar = reinterpret_cast<uint64_t*>(f_col + kMaxNT);       // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z;
  const int b0 = z / d.nb1, b1 = z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  double* C = d.C + b0 * d.sC0 + b1 * d.sC1;
  const int row0 = blockIdx.y * kBM, col0 = blockIdx.x * NT;
  const int ncols_alloc = NT <= 16 ? 128 : NT <= 32 ? 256 : 512;

  // first stage's operands in flight while the CTA sets up
  StageRegs R;
  load_stage(d, A, B, row0, col0, NT, 0, tid, R);

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < kBM) e_row[tid] = (row0 + tid < d.M) ? (int)ea[(int64_t)z * d.M + row0 + tid] : 0;
  else if (tid < kBM + kMaxNT) {
    const int n = tid - kBM;
    f_col[n] = (n < NT && col0 + n < d.N) ? (int)fb[(int64_t)z * d.N + col0 + n] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int nch = (d.K + kKC - 1) / kKC;
  bool bad = false;
  int issued = 0;                       // stages whose MMAs were issued
  for (int c = 0; c < nch; ++c) {
    const int st = c & 1;
    if (c >= 2) {
      if (!mbar_wait_bounded(&bar[st], (unsigned)(((c - 2) >> 1) & 1))) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) break;
    }
    unsigned char* sA = stage_base + (size_t)st * kStage;
    unsigned char* sB = sA + kSlices * kSliceA;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = tid + i * kThreads;
      const int r = u >> 2, h = u & 3;
      split8(R.a[i], e_row[r], sA + core_off(r, h), kSliceA, bad);
    }
    {
      const int n = tid % kMaxNT, h = tid / kMaxNT;
      if (n < NT) split8(R.b, f_col[n], sB + core_off(n, h), kSliceB, bad);
    }
    // next stage's operands in flight during the MMAs of this one
    if (c + 1 < nch) load_stage(d, A, B, row0, col0, NT, (c + 1) * kKC, tid, R);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc = instr_desc(NT);
      const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
#pragma unroll 1
      for (int kk = 0; kk < kKC / 16; ++kk) {
#pragma unroll 1
        for (int s = 0; s < kSlices; ++s) {
          const uint64_t ad = smem_desc(aaddr + s * kSliceA + kk * 2 * kLBO, kLBO, kSBO);
#pragma unroll 1
          for (int t = 0; s + t < kSlices; ++t) {
            const uint64_t bd = smem_desc(baddr + t * kSliceB + kk * 2 * kLBO, kLBO, kSBO);
            const int dg = s + t;                       // digit weight index: D_{s+t+2}
            const uint32_t acc = (c > 0 || kk > 0 || s > 0) ? 1u : 0u;
            umma_bf16(tmem + (uint32_t)(dg * NT), ad, bd, idesc, acc);
          }
        }
      }
      umma_commit(&bar[st]);
    }
    issued = c + 1;
  }
  if (bad) atomicOr(err, ERRBIT_NAN);
  // all MMAs done (the last commit covers every earlier MMA of the thread);
  // after an abort this still waits, bounded, for the MMAs in flight
  if (issued > 0) {
    if (!mbar_wait_bounded(&bar[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1))) *abort_flag = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (*abort_flag) {
    if (tid == 0) atomicOr(err, ERRBIT_TIMEOUT);
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows),
    // columns [half * NT / 2, (half + 1) * NT / 2) in groups of 8
    const int lg = warp & 3, half = warp >> 2;
    const int r = lg * 32 + lane;
    const int gr = row0 + r;
    const int ea = e_row[r];
    // alpha / beta cases: 0: C = AB, 1: C -= AB, 2: general
    const int ab = (d.alpha == 1.0 && d.beta == 0.0) ? 0 : (d.alpha == -1.0 && d.beta == 1.0) ? 1 : 2;
    for (int cb = half * (NT / 2); cb < (half + 1) * (NT / 2); cb += 8) {
      const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)cb;
      long long H[8], L[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) { H[j] = 0; L[j] = 0; }
#pragma unroll
      for (int a = 0; a < kAcc; ++a) {
        float v[8];
        tmem_ld8(tbase + (uint32_t)(a * NT), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long iv = (long long)__float2int_rn(v[j]);     // integral, |v| < 2^31
          if (a < 4) H[j] = (H[j] << 7) + iv;
          else L[j] = (L[j] << 7) + iv;
        }
      }
      if (gr < d.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gc = col0 + cb + j;
          if (cb + j >= NT || gc >= d.N) continue;
          const int fb = f_col[cb + j];
          double val = 0.0;
          if (ea > 0 && fb > 0) {
            // (H 2^28 + L) 2^E: both parts exact in FP64, one rounding in the sum
            const int E = ea + fb - 2107;
            bool ok = true;
            val = i2d_scaled(H[j], E + 28, ok) + i2d_scaled(L[j], E, ok);
            if (!ok) {   // outside the normal range: scale step by step
              const int p1 = ea - 1054, p2 = fb - 1053;
              const double s1 = (p1 >= -1022) ? __longlong_as_double((long long)(p1 + 1023) << 52) : 0.0;
              const double s2 = (p2 >= -1022) ? __longlong_as_double((long long)(p2 + 1023) << 52) : 0.0;
              val = (fma((double)H[j], 268435456.0, (double)L[j]) * s1) * s2;
            }
          }
          const int64_t cc = (int64_t)(gc / d.cg) * d.cgs + (gc % d.cg);
          double* p = C + (int64_t)gr * d.ldc + cc;
          if (ab == 0) *p = val;
          else if (ab == 1) *p = *p - val;
          else *p = (d.beta == 0.0 ? 0.0 : d.beta * *p) + d.alpha * val;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols_alloc) : "memory");
  }
}

}  // namespace

int64_t gemm_ozaki_scratch(const GemmDesc& d) {
  return (int64_t)d.nb0 * d.nb1 * (d.M + d.N);
}

bool gemm_ozaki(const GemmDesc& d, uint16_t* scratch, unsigned* err, cudaStream_t s) {
  if (d.K > kMaxK || d.N < 16 || d.M <= 0 || d.K <= 0 || !scratch) return false;
  static_assert(kSmem <= 227 * 1024, "shared memory");
  cudaFuncSetAttribute(gemm_ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  const int ntile = (d.N + kMaxNT - 1) / kMaxNT;
  int NT = (d.N + ntile - 1) / ntile;
  NT = (NT + 15) / 16 * 16;
  const int mtile = (d.M + kBM - 1) / kBM;
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  const int64_t zmax = 65535;
  const int per = (int)std::max<int64_t>(1, zmax / d.nb1);
  for (int b0 = 0; b0 < d.nb0; b0 += per) {
    GemmDesc e = d;
    e.nb0 = (d.nb0 - b0 < per) ? d.nb0 - b0 : per;
    e.A = d.A + b0 * d.sA0;
    e.B = d.B + b0 * d.sB0;
    e.C = d.C + b0 * d.sC0;
    const unsigned nz = (unsigned)((int64_t)e.nb0 * d.nb1);
    uint16_t* ea = scratch;
    uint16_t* fb = scratch + (int64_t)nz * d.M;
    count_launch(); ozaki_exponents_kernel<<<nz, 256, 0, s>>>(e, ea, fb, err);
    dim3 grid((unsigned)ntile, (unsigned)mtile, nz);
    count_launch(); gemm_ozaki_kernel<<<grid, kThreads, kSmem, s>>>(e, NT, ea, fb, err);
  }
  (void)nb;
  return true;
}

}  // namespace hdg
