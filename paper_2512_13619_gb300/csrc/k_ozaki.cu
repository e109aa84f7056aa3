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
// One CTA computes a 128 x NT output tile (NT <= 64) of one batch item with
// nine warps.  K is staged 32 columns at a time through two shared-memory
// stages.  Warps 0-7 load the FP64 operands (the next stage's loads are in
// flight while the current stage is split), split them into digits and
// write the BF16 digit matrices in the UMMA no-swizzle K-major layout (8 x
// 16-byte core matrices), then arrive on the stage's `full` mbarrier.  Warp 8
// allocates the TMEM accumulators (8 NT columns) and one of its lanes issues
// the stage's 72 MMAs (M = 128, N = NT, K = 16) and commits them to the
// stage's `empty` mbarrier, so splitting and MMAs overlap.  After the last
// stage warps 0-7 read the accumulators and form the FP64 result with
// integer arithmetic (one rounding), so the epilogue spends at most one FP64
// addition per output (for C += alpha A B).
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
constexpr int kSplitThreads = 256;        // warps 0-7: split + epilogue
constexpr int kThreads = kSplitThreads + 32;  // + warp 8: TMEM allocation, MMA issue
constexpr int kMaxK = 192;            // exactness bound of D_2..D_6 (see above)
constexpr int kSliceA = kBM * kKC * 2;       // bytes of one A digit matrix per stage (8 KB)
constexpr int kSliceB = kMaxNT * kKC * 2;    // bytes of one B digit matrix per stage (4 KB)
constexpr int kStage = kSlices * (kSliceA + kSliceB);
constexpr int kSmem = 2 * kStage + 1024;   // stages + barriers

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

// Splits 8 values (one core-matrix row of 8 K entries) into the 8 digit
// matrices: 16 bytes per digit at dst + s * slice_bytes.  A digit d (7 bits)
// becomes the float 2^23 + d (its bits or-ed into 2^23), and one FMA with
// the value's sign gives +-d exactly; the upper halves of two floats are the
// two BF16 values of a 32-bit word.
__device__ __forceinline__ void split8(const double (&v)[8], int e, unsigned char* dst, int slice_bytes) {
  uint32_t lo[8], hi[8];
  float sg[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t F = fixed56(v[j], e);
    lo[j] = (uint32_t)F;
    hi[j] = (uint32_t)(F >> 32);
    sg[j] = (__double_as_longlong(v[j]) < 0) ? -1.0f : 1.0f;
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t f[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = 2 * q + t;
        uint32_t x;    // bits 7 (7 - s) .. + 6 of the 56-bit F in the low bits of x
        if (s == 0) x = hi[j] >> 17;
        else if (s == 1) x = hi[j] >> 10;
        else if (s == 2) x = hi[j] >> 3;
        else if (s == 3) x = __funnelshift_r(lo[j], hi[j], 28);
        else x = lo[j] >> (7 * (7 - s));
        const float big = __uint_as_float((x & 127u) | 0x4B000000u);          // 2^23 + d
        f[t] = __float_as_uint(fmaf(big, sg[j], -8388608.0f * sg[j]));       // +-d
      }
      w[q] = __byte_perm(f[0], f[1], 0x7632);
    }
    *reinterpret_cast<uint4*>(dst + (size_t)s * slice_bytes) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// (H 2^28 + L) 2^sc rounded once to FP64 (nearest, ties to even), from the
// integers alone; ok = false when the result would leave the normal range.
__device__ __forceinline__ double combine_hl(long long H, long long L, int sc, bool& ok) {
  const __int128 X = ((__int128)H << 28) + (__int128)L;      // |X| < 2^76
  if (X == 0) return 0.0;
  const bool neg = X < 0;
  const unsigned __int128 U = (unsigned __int128)(neg ? -X : X);
  const unsigned long long uh = (unsigned long long)(U >> 64), ul = (unsigned long long)U;
  int p = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);
  unsigned long long mant;
  if (p <= 52) {
    mant = ul << (52 - p);
  } else {
    const int sh = p - 52;                                   // 1 .. 23
    mant = (unsigned long long)(U >> sh);
    const unsigned long long rem = ul & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++p;
    }
  }
  const int ef = p + 1023 + sc;
  if (ef < 1 || ef > 2046) {
    ok = false;
    return 0.0;
  }
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)ef << 52) |
                                          (mant & ((1ull << 52) - 1))));
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
// each) and 1 core row of B per splitting thread.
struct StageRegs {
  double a[2][8];
  double b[8];
};

__device__ __forceinline__ void load_stage(const GemmDesc& d, const double* A, const double* B, int row0, int col0,
                                           int NT, int k0, int tid, StageRegs& R) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kSplitThreads;
    const int r = u >> 2, h = u & 3;
    const int gr = row0 + r;
    if (gr >= d.M) continue;                    // padding row: zero digits, never split
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * h + j;
      R.a[i][j] = (k < d.K) ? __ldg(A + (int64_t)gr * d.lda + k) : 0.0;
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

// The 72 MMAs of one stage: K = 32 as two steps of 16; digit pair (s, t)
// into accumulator s + t.  Descriptors differ from the stage's base
// descriptors only in the start-address field.
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int NT,
                                            bool first) {
#pragma unroll
  for (int kk = 0; kk < kKC / 16; ++kk) {
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
#pragma unroll
      for (int t = 0; s + t < kSlices; ++t) {
        const uint64_t ad = adesc + (uint64_t)((s * kSliceA + kk * 2 * (int)kLBO) >> 4);
        const uint64_t bd = bdesc + (uint64_t)((t * kSliceB + kk * 2 * (int)kLBO) >> 4);
        umma_bf16(tmem + (uint32_t)((s + t) * NT), ad, bd, idesc, (first && kk == 0 && s == 0) ? 0u : 1u);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) gemm_ozaki_kernel(GemmDesc d, int NT, const uint16_t* ea,
                                                                  const uint16_t* fb, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stage_base = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * kStage);   // [2] count 256: stage split
  uint64_t* empty = full + 2;                                        // [2] count 1: stage's MMAs done
  uint64_t* done = empty + 2;                                        // [1] count 1: all MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z;
  const int b0 = z / d.nb1, b1 = z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  double* C = d.C + b0 * d.sC0 + b1 * d.sC1;
  const int row0 = blockIdx.y * kBM, col0 = blockIdx.x * NT;
  const int ncols_alloc = NT <= 16 ? 128 : NT <= 32 ? 256 : 512;
  const int nch = (d.K + kKC - 1) / kKC;
  const bool splitter = warp < kSplitThreads / 32;

  StageRegs R;
  int e_a[2] = {0, 0}, e_b = 0;
  if (splitter) {
    // first stage's operands and this thread's exponents in flight during set-up
    load_stage(d, A, B, row0, col0, NT, 0, tid, R);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = (tid + i * kSplitThreads) >> 2;
      e_a[i] = (row0 + r < d.M) ? (int)ea[(int64_t)z * d.M + row0 + r] : 0;
    }
    const int n = tid % kMaxNT;
    e_b = (n < NT && col0 + n < d.N) ? (int)fb[(int64_t)z * d.N + col0 + n] : 0;
  }
  if (tid == 0) {
    mbar_init(&full[0], kSplitThreads);
    mbar_init(&full[1], kSplitThreads);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kSplitThreads / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (splitter) {
    // ---------------------------------------------------------- splitters
    // digits of the padding rows (rows >= M) of both stages: zero, once
    const int mvalid = min(kBM, d.M - row0);
    if (mvalid < kBM) {
      for (int u = tid; u < 2 * kSlices * kBM * (kKC / 8); u += kSplitThreads) {
        const int rh = u % (kBM * (kKC / 8)), ps = u / (kBM * (kKC / 8));
        const int r = rh >> 2, h = rh & 3;
        if (r >= mvalid)
          *reinterpret_cast<uint4*>(stage_base + (size_t)(ps / kSlices) * kStage + (ps % kSlices) * kSliceA +
                                    core_off(r, h)) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    for (int c = 0; c < nch; ++c) {
      const int st = c & 1;
      if (c >= 2 && !mbar_wait_bounded(&empty[st], (unsigned)(((c - 2) >> 1) & 1))) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      unsigned char* sA = stage_base + (size_t)st * kStage;
      unsigned char* sB = sA + kSlices * kSliceA;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int u = tid + i * kSplitThreads;
        if ((u >> 2) < mvalid) split8(R.a[i], e_a[i], sA + core_off(u >> 2, u & 3), kSliceA);
      }
      {
        const int n = tid % kMaxNT, h = tid / kMaxNT;
        if (n < NT) split8(R.b, e_b, sB + core_off(n, h), kSliceB);
      }
      if (c + 1 < nch) load_stage(d, A, B, row0, col0, NT, (c + 1) * kKC, tid, R);   // in flight during the MMAs
      fence_async_smem();
      mbar_arrive(&full[st]);
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------- MMA issue
    const uint32_t idesc = instr_desc(NT);
    for (int c = 0; c < nch; ++c) {
      const int st = c & 1;
      if (!mbar_wait_bounded(&full[st], (unsigned)((c >> 1) & 1))) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      tc_fence_after();
      const uint32_t aaddr = smem_u32(stage_base + (size_t)st * kStage);
      const uint32_t baddr = aaddr + kSlices * kSliceA;
      issue_stage(tmem, smem_desc(aaddr, kLBO, kSBO), smem_desc(baddr, kLBO, kSBO), idesc, NT, c == 0);
      umma_commit(&empty[st]);
    }
    umma_commit(done);   // covers every MMA issued above (also after an abort)
  }
  // all issued MMAs complete before TMEM is read or freed
  if (!mbar_wait_bounded(done, 0u)) *abort_flag = 1;
  tc_fence_after();
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicOr(err, ERRBIT_TIMEOUT);
  } else if (splitter) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows),
    // columns [half * NT / 2, (half + 1) * NT / 2) in groups of 8
    const int lg = warp & 3, half = warp >> 2;
    const int r = lg * 32 + lane;
    const int gr = row0 + r;
    const int ea_r = (gr < d.M) ? (int)ea[(int64_t)z * d.M + gr] : 0;
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
          const int fbj = (int)fb[(int64_t)z * d.N + gc];
          double val = 0.0;
          if (ea_r > 0 && fbj > 0) {
            // (H 2^28 + L) 2^E with E = ea + fb - 2107, one rounding
            bool ok = true;
            val = combine_hl(H[j], L[j], ea_r + fbj - 2107, ok);
            if (!ok) {   // outside the normal range: scale step by step
              const int p1 = ea_r - 1054, p2 = fbj - 1053;
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
  if (warp == kSplitThreads / 32) {
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
