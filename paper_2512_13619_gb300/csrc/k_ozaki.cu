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
// seventeen warps (544 threads).  K is staged 32 columns at a time through
// two shared-memory stages.  Warps 0-15 load the FP64 operands (the next
// stage's loads are in flight while the current stage is split), split them
// into digits and write the BF16 digit matrices in the UMMA no-swizzle
// K-major layout (8 x 16-byte core matrices), then arrive on the stage's
// `full` mbarrier.  Warp 16 allocates the TMEM accumulators (8 NT columns)
// and one of its lanes issues the stage's 72 MMAs (M = 128, N = NT, K = 16)
// and commits them to the stage's `empty` mbarrier, so splitting and MMAs
// overlap.  After the last stage warps 0-15 read the accumulators and form
// the FP64 result with integer arithmetic (one rounding), so the epilogue
// spends at most one FP64 addition per output (for C += alpha A B).
#include <algorithm>

#include "hdg_common.cuh"
#include "hdg_internal.h"
#include "k_umma.cuh"

namespace hdg {

namespace {

constexpr int kSlices = 8;            // 7-bit digits per operand (56 bits)
constexpr int kAcc = kSlices;         // accumulators D_2 .. D_9
constexpr int kBM = 128;              // UMMA M
constexpr int kMaxNT = 64;
constexpr int kKC = 32;               // K per stage
constexpr int kSplitThreads = 512;        // warps 0-15: split + epilogue
constexpr int kThreads = kSplitThreads + 32;  // + warp 16: TMEM allocation, MMA issue
constexpr int kMaxK = 192;            // exactness bound of D_2..D_6 (see above)
constexpr int kSliceA = kBM * kKC * 2;       // bytes of one A digit matrix per stage (8 KB)
constexpr int kSliceB = kMaxNT * kKC * 2;    // bytes of one B digit matrix per stage (4 KB)
constexpr int kStage = kSlices * (kSliceA + kSliceB);
constexpr int kSmem = 2 * kStage + 1024;   // stages + barriers

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
// matrices: 16 bytes per digit at dst + s * slice_bytes.  The digits d0, d1
// (7 bits each) of two neighbouring values are placed in one 32-bit word as
// the BF16 bit patterns of 128 + d (0x4300 | d, exact), and one packed BF16
// FMA with the values' signs, (128 + d) s - 128 s = s d, gives both digits
// exactly.
__device__ __forceinline__ void split8(const double (&v)[8], int e, unsigned char* dst, int slice_bytes) {
  uint32_t lo[8], hi[8];
  __nv_bfloat162 sg[4], off[4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t F = fixed56(v[j], e);
    lo[j] = (uint32_t)F;
    hi[j] = (uint32_t)(F >> 32);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // packed signs (+-1) and offsets (-+128) of values 2q, 2q+1 (bf16 bits)
    const uint32_t s0 = (uint32_t)((unsigned long long)__double_as_longlong(v[2 * q]) >> 63);
    const uint32_t s1 = (uint32_t)((unsigned long long)__double_as_longlong(v[2 * q + 1]) >> 63);
    const uint32_t sb = 0x3F803F80u | (s0 << 15) | (s1 << 31);           // (+-1, +-1)
    const uint32_t ob = 0xC300C300u ^ ((s0 << 15) | (s1 << 31));         // (-+128, -+128)
    sg[q] = *reinterpret_cast<const __nv_bfloat162*>(&sb);
    off[q] = *reinterpret_cast<const __nv_bfloat162*>(&ob);
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t x[2];    // bits 7 (7 - s) .. + 6 of the 56-bit F in the low byte of x
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = 2 * q + t;
        if (s == 0) x[t] = hi[j] >> 17;
        else if (s == 1) x[t] = hi[j] >> 10;
        else if (s == 2) x[t] = hi[j] >> 3;
        else if (s == 3) x[t] = __funnelshift_r(lo[j], hi[j], 28);
        else x[t] = lo[j] >> (7 * (7 - s));
      }
      // low bytes of x[0], x[1] into bytes 0 and 2, 7-bit fields, 128 + d as BF16
      const uint32_t pk = (__byte_perm(x[0], x[1], 0x4400) & 0x007F007Fu) | 0x43004300u;
      const __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162*>(&pk), sg[q], off[q]);
      w[q] = *reinterpret_cast<const uint32_t*>(&r);
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
// Rows of A: one warp per row, lanes along K (coalesced).  Columns of B:
// threads along the columns (coalesced), four K ranges per column merged in
// shared memory.
__global__ void __launch_bounds__(256) ozaki_exponents_kernel(GemmDesc d, uint16_t* ea, uint16_t* fb,
                                                              unsigned* err) {
  __shared__ int colmax[256];
  const int z = blockIdx.x;
  const int b0 = z / d.nb1, b1 = z % d.nb1;
  const double* A = d.A + b0 * d.sA0 + b1 * d.sA1;
  const double* B = d.B + b0 * d.sB0 + b1 * d.sB1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad = false;
  // rows r0, r0 + 8, r0 + 16, r0 + 24 per warp, their loads interleaved so
  // that four rows' loads are in flight together
  const int nk = (d.K + 31) / 32;
  for (int r0 = warp; r0 < d.M; r0 += 32) {
    int m[4] = {0, 0, 0, 0};
    for (int j = 0; j < nk; ++j) {
      const int k = j * 32 + lane;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + 8 * u;
        if (r < d.M && k < d.K) m[u] = max(m[u], exp_field(__ldg(A + (int64_t)r * d.lda + k)));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 8 * u;
      bad |= (m[u] == 0x7FF);
      const int mm = (int)__reduce_max_sync(0xffffffffu, (unsigned)m[u]);
      if (lane == 0 && r < d.M) ea[(int64_t)z * d.M + r] = (uint16_t)mm;
    }
  }
  // columns in blocks of 64: thread (n, q) scans rows k = q, q + 4, ...
  for (int n0 = 0; n0 < d.N; n0 += 64) {
    const int n = n0 + (threadIdx.x & 63), q = threadIdx.x >> 6;
    int m = 0;
    if (n < d.N) {
#pragma unroll 8
      for (int k = q; k < d.K; k += 4) m = max(m, exp_field(__ldg(B + (int64_t)k * d.ldb + n)));
    }
    colmax[threadIdx.x] = m;
    __syncthreads();
    if (q == 0 && n < d.N) {
      const int c = threadIdx.x;
      m = max(max(colmax[c], colmax[c + 64]), max(colmax[c + 128], colmax[c + 192]));
      bad |= (m == 0x7FF);
      fb[(int64_t)z * d.N + n] = (uint16_t)m;
    }
    __syncthreads();
  }
  if (bad) atomicOr(err, ERRBIT_NAN);
}

// FP64 operands of one stage in registers: kAU core rows of A (8 K entries
// each) and at most 1 core row of B per splitting thread.
constexpr int kAU = kBM * (kKC / 8) / kSplitThreads;
struct StageRegs {
  double a[kAU][8];
  double b[8];
};

__device__ __forceinline__ void load_stage(const GemmDesc& d, const double* A, const double* B, int row0, int col0,
                                           int NT, int k0, int tid, StageRegs& R) {
#pragma unroll
  for (int i = 0; i < kAU; ++i) {
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
  if (tid < kMaxNT * (kKC / 8)) {
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
  int e_a[kAU], e_b = 0;
  if (splitter) {
    // first stage's operands and this thread's exponents in flight during set-up
    load_stage(d, A, B, row0, col0, NT, 0, tid, R);
#pragma unroll
    for (int i = 0; i < kAU; ++i) {
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
      for (int i = 0; i < kAU; ++i) {
        const int u = tid + i * kSplitThreads;
        if ((u >> 2) < mvalid) split8(R.a[i], e_a[i], sA + core_off(u >> 2, u & 3), kSliceA);
      }
      if (tid < kMaxNT * (kKC / 8)) {
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
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows) and
    // the column groups of 8 numbered w / 4 modulo the number of warp rows
    constexpr int kWR = kSplitThreads / 128;
    const int lg = warp & 3, part = warp >> 2;
    const int r = lg * 32 + lane;
    const int gr = row0 + r;
    const int ea_r = (gr < d.M) ? (int)ea[(int64_t)z * d.M + gr] : 0;
    // alpha / beta cases: 0: C = AB, 1: C -= AB, 2: general
    const int ab = (d.alpha == 1.0 && d.beta == 0.0) ? 0 : (d.alpha == -1.0 && d.beta == 1.0) ? 1 : 2;
    for (int cb = part * 8; cb < NT; cb += kWR * 8) {
      const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)cb;
      // the block's column exponents and (for C -= AB and the general case)
      // the old C values first, so that their loads overlap the TMEM reads
      int fbv[8];
      double cv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gc = col0 + cb + j;
        const bool in = gr < d.M && cb + j < NT && gc < d.N;
        fbv[j] = in ? (int)fb[(int64_t)z * d.N + gc] : 0;
        cv[j] = 0.0;
        if (in && ab != 0) cv[j] = C[(int64_t)gr * d.ldc + (int64_t)(gc / d.cg) * d.cgs + (gc % d.cg)];
      }
      // the 8 accumulators' columns: all loads issued, one wait
      uint32_t raw[kAcc][8];
#pragma unroll
      for (int a = 0; a < kAcc; ++a) tmem_ld8_nowait(tbase + (uint32_t)(a * NT), raw[a]);
      tmem_wait_ld();
#pragma unroll
      for (int a = 0; a < kAcc; ++a) reg_order8(raw[a]);
      long long H[8], L[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) { H[j] = 0; L[j] = 0; }
#pragma unroll
      for (int a = 0; a < kAcc; ++a) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long iv = (long long)__float2int_rn(__uint_as_float(raw[a][j]));   // integral, |v| < 2^31
          if (a < 4) H[j] = (H[j] << 7) + iv;
          else L[j] = (L[j] << 7) + iv;
        }
      }
      if (gr < d.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gc = col0 + cb + j;
          if (cb + j >= NT || gc >= d.N) continue;
          const int fbj = fbv[j];
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
          else if (ab == 1) *p = cv[j] - val;
          else *p = (d.beta == 0.0 ? 0.0 : d.beta * cv[j]) + d.alpha * val;
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

// ================================================= persistent per-tile path
// One CTA per SM walks the output tiles (128 x NT, NT in {32, 48, 64}) of
// the whole batch.  Warps 0-7 split the FP64 operands of each stage into
// digits (as above), warp 8 issues the MMAs, warps 9-12 drain the
// accumulators.  The stage ring runs on across tiles.  With NT = 32 the
// accumulators are double-buffered in TMEM (2 x 8 x 32 columns), so the
// epilogue of tile i overlaps the MMAs of tile i+1; with 48 or 64 one buffer
// fills TMEM and only the digit split of the next tile overlaps the
// epilogue.
template <int NT> struct QCfg {
  static constexpr int kSliceB = NT * kKC * 2;
  static constexpr int kStage = kSlices * (kSliceA + kSliceB);
  static constexpr int kSmem = 2 * kStage + 1024;
  static constexpr int kBuf = (NT == 32) ? 2 : 1;            // TMEM accumulator buffers
};
constexpr int kQSplit = 256;
constexpr int kQThreads = kQSplit + 32 + 128;             // splitters, MMA warp, 4 epilogue warps

struct QTile {
  int nt, mt;
  int64_t z, b0, b1;
};
__device__ __forceinline__ QTile qtile(int64_t q, int ntile, int mtile, int nb1) {  // q -> (nt, mt, z)
  QTile t;
  t.nt = (int)(q % ntile);
  t.mt = (int)((q / ntile) % mtile);
  t.z = q / ((int64_t)ntile * mtile);
  t.b0 = t.z / nb1;
  t.b1 = t.z % nb1;
  return t;
}

struct QRegs {
  double a[2][8];
  double b[8];
};

template <int NT>
__device__ __forceinline__ void q_load(const GemmDesc& d, const QTile& t, int k0, int tid, QRegs& R) {
  const double* A = d.A + t.b0 * d.sA0 + t.b1 * d.sA1;
  const double* B = d.B + t.b0 * d.sB0 + t.b1 * d.sB1;
  const int row0 = t.mt * kBM, col0 = t.nt * NT;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kQSplit;
    const int r = u >> 2, h = u & 3;
    const int gr = row0 + r;
    if (gr >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * h + j;
      R.a[i][j] = (k < d.K) ? __ldg(A + (int64_t)gr * d.lda + k) : 0.0;
    }
  }
  if (tid < NT * (kKC / 8)) {
    const int n = tid % NT, h = tid / NT;
    const int gc = col0 + n;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * h + j;
      R.b[j] = (gc < d.N && k < d.K) ? __ldg(B + (int64_t)k * d.ldb + gc) : 0.0;
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(kQThreads, 1) gemm_ozaki_persist_kernel(GemmDesc d, const uint16_t* ea,
                                                                          const uint16_t* fb, int ntile, int mtile,
                                                                          int64_t total, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using Q = QCfg<NT>;
  constexpr int NB = Q::kBuf;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * Q::kStage);  // [2] count 256
  uint64_t* empty = full + 2;                                          // [2] MMA commit
  uint64_t* tfull = empty + 2;                                         // [NB] MMA commit: tile accumulated
  uint64_t* tempty = tfull + 2;                                        // [NB] count 4: epilogue warps done
  uint64_t* done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = (d.K + kKC - 1) / kKC;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], kQSplit);
      mbar_init(&empty[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp < 8) {
    // ------------------------------------------------------------ splitters
    QRegs R;
    int64_t q = blockIdx.x;
    QTile t = qtile(q, ntile, mtile, d.nb1);
    if (q < total) q_load<NT>(d, t, 0, tid, R);
    int64_t gs = 0;
    for (; q < total && !*abort_flag; q += gridDim.x) {
      t = qtile(q, ntile, mtile, d.nb1);
      const int row0 = t.mt * kBM, col0 = t.nt * NT;
      const int mvalid = min(kBM, d.M - row0);
      int e_a[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = (tid + i * kQSplit) >> 2;
        e_a[i] = (r < mvalid) ? (int)ea[t.z * d.M + row0 + r] : 0;
      }
      const int nB = tid % NT;
      const int e_b = (tid < NT * (kKC / 8) && col0 + nB < d.N) ? (int)fb[t.z * d.N + col0 + nB] : 0;
      for (int c = 0; c < nch; ++c, ++gs) {
        const int st = (int)(gs & 1);
        if (gs >= 2 && !mbar_wait_bounded(&empty[st], (unsigned)(((gs - 2) >> 1) & 1))) *abort_flag = 1;
        if (*abort_flag) break;
        unsigned char* sA = smem + (size_t)st * Q::kStage;
        unsigned char* sB = sA + kSlices * kSliceA;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int u = tid + i * kQSplit;
          const int r = u >> 2, h = u & 3;
          if (r < mvalid) {
            split8(R.a[i], e_a[i], sA + core_off(r, h), kSliceA);
          } else {
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl)
              *reinterpret_cast<uint4*>(sA + sl * kSliceA + core_off(r, h)) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        if (tid < NT * (kKC / 8)) split8(R.b, e_b, sB + core_off(tid % NT, tid / NT), Q::kSliceB);
        // next stage's operands (this tile's next chunk, or the next tile's first)
        if (c + 1 < nch) {
          q_load<NT>(d, t, (c + 1) * kKC, tid, R);
        } else if (q + gridDim.x < total) {
          q_load<NT>(d, qtile(q + gridDim.x, ntile, mtile, d.nb1), 0, tid, R);
        }
        fence_async_smem();
        mbar_arrive(&full[st]);
      }
    }
  } else if (warp == 8) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = instr_desc(NT);
      int64_t gs = 0;
      int64_t i = 0;
      for (int64_t q = blockIdx.x; q < total && !*abort_flag; q += gridDim.x, ++i) {
        const int buf = (int)(i % NB);
        // the epilogue has read tile i - NB from this buffer
        if (i >= NB && !mbar_wait_bounded(&tempty[buf], (unsigned)((i / NB - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        const uint32_t acc0 = tmem + (uint32_t)(buf * kAcc * NT);
        for (int c = 0; c < nch; ++c, ++gs) {
          const int st = (int)(gs & 1);
          if (!mbar_wait_bounded(&full[st], (unsigned)((gs >> 1) & 1))) *abort_flag = 1;
          if (*abort_flag) break;
          tc_fence_after();
          const uint32_t aaddr = smem_u32(smem + (size_t)st * Q::kStage);
          const uint32_t baddr = aaddr + kSlices * kSliceA;
          const uint64_t ad0 = smem_desc(aaddr, kLBO, kSBO), bd0 = smem_desc(baddr, kLBO, kSBO);
#pragma unroll
          for (int kk = 0; kk < kKC / 16; ++kk) {
#pragma unroll
            for (int sa = 0; sa < kSlices; ++sa) {
#pragma unroll
              for (int sb = 0; sa + sb < kSlices; ++sb) {
                const uint64_t ad = ad0 + (uint64_t)((sa * kSliceA + kk * 2 * (int)kLBO) >> 4);
                const uint64_t bd = bd0 + (uint64_t)((sb * Q::kSliceB + kk * 2 * (int)kLBO) >> 4);
                umma_bf16(acc0 + (uint32_t)((sa + sb) * NT), ad, bd, idesc,
                          (c == 0 && kk == 0 && sa == 0) ? 0u : 1u);
              }
            }
          }
          umma_commit(&empty[st]);
        }
        umma_commit(&tfull[buf]);
      }
      umma_commit(done);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int lg = warp & 3;
    const int ab = (d.alpha == 1.0 && d.beta == 0.0) ? 0 : (d.alpha == -1.0 && d.beta == 1.0) ? 1 : 2;
    int64_t i = 0;
    for (int64_t q = blockIdx.x; q < total; q += gridDim.x, ++i) {
      const int buf = (int)(i % NB);
      if (*abort_flag || !mbar_wait_bounded(&tfull[buf], (unsigned)((i / NB) & 1))) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const QTile t = qtile(q, ntile, mtile, d.nb1);
      const int r = lg * 32 + lane;
      const int gr = t.mt * kBM + r;
      const int col0 = t.nt * NT;
      const int ea_r = (gr < d.M) ? (int)ea[t.z * d.M + gr] : 0;
      double* C = d.C + t.b0 * d.sC0 + t.b1 * d.sC1;
      for (int cb = 0; cb < NT; cb += 8) {
        const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(buf * kAcc * NT + cb);
        long long H[8], L[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { H[j] = 0; L[j] = 0; }
#pragma unroll
        for (int a = 0; a < kAcc; ++a) {
          float v[8];
          tmem_ld8(tbase + (uint32_t)(a * NT), v);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long iv = (long long)__float2int_rn(v[j]);
            if (a < 4) H[j] = (H[j] << 7) + iv;
            else L[j] = (L[j] << 7) + iv;
          }
        }
        if (gr < d.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int gc = col0 + cb + j;
            if (gc >= d.N) continue;
            const int fbj = (int)fb[t.z * d.N + gc];
            double val = 0.0;
            if (ea_r > 0 && fbj > 0) {
              bool ok = true;
              val = combine_hl(H[j], L[j], ea_r + fbj - 2107, ok);
              if (!ok) {
                const int p1 = ea_r - 1054, p2 = fbj - 1053;
                const double s1 = (p1 >= -1022) ? __longlong_as_double((long long)(p1 + 1023) << 52) : 0.0;
                const double s2 = (p2 >= -1022) ? __longlong_as_double((long long)(p2 + 1023) << 52) : 0.0;
                val = (fma((double)H[j], 268435456.0, (double)L[j]) * s1) * s2;
              }
            }
            const int64_t cc = (int64_t)(gc / d.cg) * d.cgs + (gc % d.cg);
            double* pc = C + (int64_t)gr * d.ldc + cc;
            if (ab == 0) *pc = val;
            else if (ab == 1) *pc = *pc - val;
            else *pc = (d.beta == 0.0 ? 0.0 : d.beta * *pc) + d.alpha * val;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  // every issued MMA is complete before TMEM is freed (bounded after an abort)
  if (!mbar_wait_bounded(done, 0u)) *abort_flag = 1;
  tc_fence_after();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(err, ERRBIT_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// =================================================== split once, copy planes
// The digits of an operand can also be computed once per operand by a
// streaming kernel and written to HBM as BF16 planes in the shared-memory
// image the MMAs read; the product kernel then only moves planes with bulk
// copies (cp.async.bulk) and issues MMAs.  An operand (A: its rows, B: its
// columns) is cut into tiles of TR rows (128 for A, NT for B) and K chunks of
// 16.  The image of (tile, chunk) is its 8 digit matrices one after the other,
// each TRp rows x 16 K in the no-swizzle K-major layout (SBO = 256, LBO =
// 128), TRp = the tile's rows rounded up to 8 (A; zero rows above) or NT (B;
// zero columns past N).  Every tile but the last is full.
constexpr int kPC = 16;
constexpr uint32_t kPSBO = (kPC / 8) * 128;
constexpr int kPStages = 4;
constexpr int kPSliceA = kBM * kPC * 2;               // 4 KB: one A digit matrix per stage in shared memory
constexpr int kPStageA = kSlices * kPSliceA;          // 32 KB
constexpr int kPStageB = kSlices * kMaxNT * kPC * 2;  // 16 KB
constexpr int kPStage = kPStageA + kPStageB;
constexpr int kPSmem = kPStages * kPStage + 1024;
constexpr int kPThreads = 192;                        // producer, MMA, 4 epilogue warps

__host__ __device__ inline int plane_rows(int rows, int TR, int t, bool roleB) {
  if (roleB) return TR;
  const int v = rows - t * TR < TR ? rows - t * TR : TR;
  return (v + 7) / 8 * 8;
}
__host__ __device__ inline int64_t plane_tile_off(int TR, int nch, int t) { return (int64_t)t * nch * 8 * TR * (kPC * 2); }
__host__ __device__ inline int64_t plane_chunk_off(int TRp, int c) { return (int64_t)c * 8 * TRp * (kPC * 2); }
__device__ __forceinline__ int core16(int row, int h) { return (row >> 3) * kPSBO + h * 128 + (row & 7) * 16; }

struct SplitDesc {
  const double* X;
  int64_t ld, s0, s1;      // item (i0, i1) at X + i0 s0 + i1 s1; element (r, k) at r ld + k (A) or k ld + r (B)
  int n1;                  // items per i0
  int rows, K, TR, roleB, nch;
  unsigned char* planes;
  int64_t item_bytes;
  uint16_t* ex;            // [item][rows]: largest exponent field of each row (A) / column (B)
  unsigned* err;
};

__global__ void __launch_bounds__(256) ozaki_split_kernel(SplitDesc d) {
  const int64_t item = blockIdx.x;
  const int t = blockIdx.y;
  const double* X = d.X + (item / d.n1) * d.s0 + (item % d.n1) * d.s1;
  const int r0 = t * d.TR;
  const int rv = min(d.TR, d.rows - r0);
  const int TRp = plane_rows(d.rows, d.TR, t, d.roleB);
  __shared__ int e_s[kBM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad = false;
  for (int r = threadIdx.x; r < TRp; r += blockDim.x)
    if (r >= rv) e_s[r] = 0;
  if (!d.roleB) {
    for (int r = warp; r < rv; r += 8) {
      int m = 0;
      const double* row = X + (int64_t)(r0 + r) * d.ld;
#pragma unroll 8
      for (int k = lane; k < d.K; k += 32) m = max(m, exp_field(row[k]));
      m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
      if (lane == 0) {
        e_s[r] = m;
        d.ex[item * d.rows + r0 + r] = (uint16_t)m;
      }
      bad |= (m == 0x7FF);
    }
  } else {
    for (int r = threadIdx.x; r < rv; r += blockDim.x) {
      int m = 0;
#pragma unroll 8
      for (int k = 0; k < d.K; ++k) m = max(m, exp_field(X[(int64_t)k * d.ld + r0 + r]));
      e_s[r] = m;
      d.ex[item * d.rows + r0 + r] = (uint16_t)m;
      bad |= (m == 0x7FF);
    }
  }
  if (bad) atomicOr(d.err, ERRBIT_NAN);
  __syncthreads();
  unsigned char* img = d.planes + item * d.item_bytes + plane_tile_off(d.TR, d.nch, t);
  const int ng = d.nch * 2;                                   // 8-entry K groups
  const int units = TRp * ng;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    int r, g;
    if (!d.roleB) { r = u / ng; g = u - r * ng; }             // consecutive threads along K of a row
    else { g = u / TRp; r = u - g * TRp; }                     // consecutive threads along the columns
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * g + j;
      v[j] = 0.0;
      if (r < rv && k < d.K)
        v[j] = d.roleB ? __ldg(X + (int64_t)k * d.ld + r0 + r) : __ldg(X + (int64_t)(r0 + r) * d.ld + k);
    }
    split8(v, e_s[r], img + plane_chunk_off(TRp, g >> 1) + core16(r, g & 1), TRp * (kPC * 2));
  }
}

struct PlaneGemm {
  int M, N, K, NT, nch, nb1;
  int64_t z0;                          // first batch index of this launch
  const unsigned char* pa; int64_t a_bytes; const uint16_t* ea; int a_b0, a_b1;
  const unsigned char* pb; int64_t b_bytes; const uint16_t* eb; int b_b0, b_b1;
  double* C; int64_t ldc, sC0, sC1; int cg; int64_t cgs;
  double alpha, beta;
};

__global__ void __launch_bounds__(kPThreads, 1) gemm_planes_kernel(PlaneGemm g, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPStages * kPStage);
  uint64_t* empty = full + kPStages;
  uint64_t* done = empty + kPStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t z = g.z0 + blockIdx.z;
  const int64_t b0 = z / g.nb1, b1 = z % g.nb1;
  const int mt = blockIdx.y, nt = blockIdx.x;
  const int row0 = mt * kBM, col0 = nt * g.NT;
  const int NT = g.NT;
  const int TRp = plane_rows(g.M, kBM, mt, false);
  const int64_t ia = (g.a_b0 ? b0 : 0) * (g.a_b1 ? g.nb1 : 1) + (g.a_b1 ? b1 : 0);
  const int64_t ib = (g.b_b0 ? b0 : 0) * (g.b_b1 ? g.nb1 : 1) + (g.b_b1 ? b1 : 0);
  const int ncols_alloc = NT <= 16 ? 128 : NT <= 32 ? 256 : 512;

  if (tid == 0) {
    for (int i = 0; i < kPStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (warp >= 2 && TRp < kBM) {
    // A rows past the tile's image stay zero in every stage
    const int per = (kBM - TRp) * (kPC * 2) / 16;             // 16-byte words per digit matrix
    for (int u = tid - 64; u < kPStages * kSlices * per; u += kPThreads - 64) {
      const int ps = u / per, w = u - ps * per;
      const int r = TRp + w / 2, h = w & 1;
      *reinterpret_cast<uint4*>(smem + (size_t)(ps / kSlices) * kPStage + (ps % kSlices) * kPSliceA + core16(r, h)) =
          make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      const unsigned char* srcA = g.pa + ia * g.a_bytes + plane_tile_off(kBM, g.nch, mt);
      const unsigned char* srcB = g.pb + ib * g.b_bytes + plane_tile_off(NT, g.nch, nt);
      const unsigned bytesA = (unsigned)(kSlices * TRp * (kPC * 2)), bytesB = (unsigned)(kSlices * NT * (kPC * 2));
      for (int c = 0; c < g.nch; ++c) {
        const int st = c % kPStages;
        if (c >= kPStages && !mbar_wait_bounded(&empty[st], (unsigned)((c / kPStages - 1) & 1))) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        unsigned char* sA = smem + (size_t)st * kPStage;
        unsigned char* sB = sA + kPStageA;
        mbar_arrive_expect_tx(&full[st], bytesA + bytesB);
        const unsigned char* a = srcA + plane_chunk_off(TRp, c);
        if (TRp == kBM) {
          bulk_g2s(sA, a, bytesA, &full[st]);
        } else {
          for (int sl = 0; sl < kSlices; ++sl)
            bulk_g2s(sA + sl * kPSliceA, a + (size_t)sl * TRp * (kPC * 2), (unsigned)(TRp * (kPC * 2)), &full[st]);
        }
        bulk_g2s(sB, srcB + plane_chunk_off(NT, c), bytesB, &full[st]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issue
      const uint32_t idesc = instr_desc(NT);
      for (int c = 0; c < g.nch; ++c) {
        const int st = c % kPStages;
        if (!mbar_wait_bounded(&full[st], (unsigned)((c / kPStages) & 1))) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        tc_fence_after();
        const uint32_t aaddr = smem_u32(smem + (size_t)st * kPStage);
        const uint64_t ad0 = smem_desc(aaddr, 128, kPSBO), bd0 = smem_desc(aaddr + kPStageA, 128, kPSBO);
#pragma unroll
        for (int sa = 0; sa < kSlices; ++sa) {
#pragma unroll
          for (int sb = 0; sa + sb < kSlices; ++sb) {
            const uint64_t ad = ad0 + (uint64_t)((sa * kPSliceA) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((sb * NT * (kPC * 2)) >> 4);
            umma_bf16(tmem + (uint32_t)((sa + sb) * NT), ad, bd, idesc, (c == 0 && sa == 0) ? 0u : 1u);
          }
        }
        umma_commit(&empty[st]);
      }
      umma_commit(done);
    }
  }
  if (!mbar_wait_bounded(done, 0u)) *abort_flag = 1;
  tc_fence_after();
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicOr(err, ERRBIT_TIMEOUT);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int lg = warp & 3;
    const int r = lg * 32 + lane;
    const int gr = row0 + r;
    const int ea_r = (gr < g.M) ? (int)g.ea[ia * g.M + gr] : 0;
    double* C = g.C + b0 * g.sC0 + b1 * g.sC1;
    const int ab = (g.alpha == 1.0 && g.beta == 0.0) ? 0 : (g.alpha == -1.0 && g.beta == 1.0) ? 1 : 2;
    for (int cb = 0; cb < NT; cb += 8) {
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
          const long long iv = (long long)__float2int_rn(v[j]);
          if (a < 4) H[j] = (H[j] << 7) + iv;
          else L[j] = (L[j] << 7) + iv;
        }
      }
      if (gr < g.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gc = col0 + cb + j;
          if (gc >= g.N) continue;
          const int fbj = (int)g.eb[ib * g.N + gc];
          double val = 0.0;
          if (ea_r > 0 && fbj > 0) {
            bool ok = true;
            val = combine_hl(H[j], L[j], ea_r + fbj - 2107, ok);
            if (!ok) {
              const int p1 = ea_r - 1054, p2 = fbj - 1053;
              const double s1 = (p1 >= -1022) ? __longlong_as_double((long long)(p1 + 1023) << 52) : 0.0;
              const double s2 = (p2 >= -1022) ? __longlong_as_double((long long)(p2 + 1023) << 52) : 0.0;
              val = (fma((double)H[j], 268435456.0, (double)L[j]) * s1) * s2;
            }
          }
          const int64_t cc = (int64_t)(gc / g.cg) * g.cgs + (gc % g.cg);
          double* pc = C + (int64_t)gr * g.ldc + cc;
          if (ab == 0) *pc = val;
          else if (ab == 1) *pc = *pc - val;
          else *pc = (g.beta == 0.0 ? 0.0 : g.beta * *pc) + g.alpha * val;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols_alloc) : "memory");
  }
}

int pick_nt(int N) {
  const int ntile = (N + kMaxNT - 1) / kMaxNT;
  const int NT = (N + ntile - 1) / ntile;
  return (NT + 15) / 16 * 16;
}

int64_t plane_item_bytes(int rows, int K, int TR, bool roleB) {
  const int ntile = (rows + TR - 1) / TR, nch = (K + kPC - 1) / kPC;
  int64_t by = 0;
  for (int t = 0; t < ntile; ++t) by += (int64_t)nch * 8 * plane_rows(rows, TR, t, roleB) * (kPC * 2);
  return by;
}

}  // namespace

int64_t gemm_ozaki_scratch(const GemmDesc& d) {
  return (int64_t)d.nb0 * d.nb1 * (d.M + d.N);
}

bool gemm_ozaki(const GemmDesc& d, uint16_t* scratch, unsigned* err, cudaStream_t s) {
  if (d.N < 16 || d.M <= 0 || d.K <= 0 || !scratch) return false;
  if (d.K > kMaxK) {
    // K in slices of at most 192 (the exactness bound of the accumulators),
    // each rounded to FP64 and accumulated into C
    for (int k0 = 0; k0 < d.K; k0 += kMaxK) {
      GemmDesc e = d;
      e.K = d.K - k0 < kMaxK ? d.K - k0 : kMaxK;
      e.A = d.A + k0;                      // columns k0.. of A
      e.B = d.B + (int64_t)k0 * d.ldb;     // rows k0.. of B
      if (k0 > 0) e.beta = 1.0;
      gemm_ozaki(e, scratch, err, s);
    }
    return true;
  }
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

// Plane path: split A and B once into digit planes, then the copy-and-MMA
// product.  Scratch: plane bytes and 16-bit exponents; false (nothing
// launched) when the shape is outside K <= 192, N >= 16 or the scratch is
// too small.
int64_t gemm_planes_bytes(const GemmDesc& d, int64_t* ex_words) {
  if (d.K > kMaxK || d.N < 16) return -1;
  const int NT = pick_nt(d.N);
  const bool a_b0 = d.sA0 != 0 && d.nb0 > 1, a_b1 = d.sA1 != 0 && d.nb1 > 1;
  const bool b_b0 = d.sB0 != 0 && d.nb0 > 1, b_b1 = d.sB1 != 0 && d.nb1 > 1;
  const int64_t ia = (int64_t)(a_b0 ? d.nb0 : 1) * (a_b1 ? d.nb1 : 1);
  const int64_t ib = (int64_t)(b_b0 ? d.nb0 : 1) * (b_b1 ? d.nb1 : 1);
  if (ex_words) *ex_words = ia * d.M + ib * d.N;
  return ia * plane_item_bytes(d.M, d.K, kBM, false) + ib * plane_item_bytes(d.N, d.K, NT, true);
}

bool gemm_ozaki_planes(const GemmDesc& d, unsigned char* planes, int64_t planes_cap, uint16_t* ex, int64_t ex_cap,
                       unsigned* err, cudaStream_t s) {
  int64_t exw = 0;
  const int64_t need = gemm_planes_bytes(d, &exw);
  if (need < 0 || need > planes_cap || exw > ex_cap || d.M <= 0 || d.K <= 0) return false;
  static_assert(kPSmem <= 227 * 1024, "shared memory");
  cudaFuncSetAttribute(gemm_planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
  const int NT = pick_nt(d.N);
  const int nch = (d.K + kPC - 1) / kPC;
  const bool a_b0 = d.sA0 != 0 && d.nb0 > 1, a_b1 = d.sA1 != 0 && d.nb1 > 1;
  const bool b_b0 = d.sB0 != 0 && d.nb0 > 1, b_b1 = d.sB1 != 0 && d.nb1 > 1;
  const int64_t ia = (int64_t)(a_b0 ? d.nb0 : 1) * (a_b1 ? d.nb1 : 1);
  const int64_t ib = (int64_t)(b_b0 ? d.nb0 : 1) * (b_b1 ? d.nb1 : 1);
  // A: items (b0, b1) -> rows of A; B: items -> columns of B
  SplitDesc sa{};
  sa.X = d.A; sa.ld = d.lda; sa.s0 = a_b0 ? d.sA0 : 0; sa.s1 = a_b1 ? d.sA1 : 0; sa.n1 = a_b1 ? d.nb1 : 1;
  sa.rows = d.M; sa.K = d.K; sa.TR = kBM; sa.roleB = 0; sa.nch = nch;
  sa.planes = planes; sa.item_bytes = plane_item_bytes(d.M, d.K, kBM, false); sa.ex = ex; sa.err = err;
  SplitDesc sb{};
  sb.X = d.B; sb.ld = d.ldb; sb.s0 = b_b0 ? d.sB0 : 0; sb.s1 = b_b1 ? d.sB1 : 0; sb.n1 = b_b1 ? d.nb1 : 1;
  sb.rows = d.N; sb.K = d.K; sb.TR = NT; sb.roleB = 1; sb.nch = nch;
  sb.planes = planes + ia * sa.item_bytes; sb.item_bytes = plane_item_bytes(d.N, d.K, NT, true);
  sb.ex = ex + ia * d.M; sb.err = err;
  const int mtile = (d.M + kBM - 1) / kBM, ntile = (d.N + NT - 1) / NT;
  count_launch(); ozaki_split_kernel<<<dim3((unsigned)ia, (unsigned)mtile), 256, 0, s>>>(sa);
  count_launch(); ozaki_split_kernel<<<dim3((unsigned)ib, (unsigned)ntile), 256, 0, s>>>(sb);
  PlaneGemm g{};
  g.M = d.M; g.N = d.N; g.K = d.K; g.NT = NT; g.nch = nch; g.nb1 = d.nb1;
  g.pa = planes; g.a_bytes = sa.item_bytes; g.ea = ex; g.a_b0 = a_b0; g.a_b1 = a_b1;
  g.pb = sb.planes; g.b_bytes = sb.item_bytes; g.eb = sb.ex; g.b_b0 = b_b0; g.b_b1 = b_b1;
  g.C = d.C; g.ldc = d.ldc; g.sC0 = d.sC0; g.sC1 = d.sC1; g.cg = d.cg; g.cgs = d.cgs;
  g.alpha = d.alpha; g.beta = d.beta;
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  for (int64_t z0 = 0; z0 < nb; z0 += 65535) {
    g.z0 = z0;
    const unsigned nz = (unsigned)(nb - z0 < 65535 ? nb - z0 : 65535);
    count_launch(); gemm_planes_kernel<<<dim3((unsigned)ntile, (unsigned)mtile, nz), kPThreads, kPSmem, s>>>(g, err);
  }
  return true;
}

template <int NT>
void launch_persist(const GemmDesc& d, const uint16_t* ea, const uint16_t* fb, int64_t nb, unsigned* err,
                    cudaStream_t s) {
  static_assert(QCfg<NT>::kSmem <= 227 * 1024, "shared memory");
  cudaFuncSetAttribute(gemm_ozaki_persist_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, QCfg<NT>::kSmem);
  const int ntile = (d.N + NT - 1) / NT, mtile = (d.M + kBM - 1) / kBM;
  const int64_t total = (int64_t)ntile * mtile * nb;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(total, sms > 0 ? sms : 1);
  count_launch();
  gemm_ozaki_persist_kernel<NT><<<(unsigned)grid, kQThreads, QCfg<NT>::kSmem, s>>>(d, ea, fb, ntile, mtile, total, err);
}

bool gemm_ozaki_persist(const GemmDesc& d, uint16_t* scratch, int64_t scratch_words, unsigned* err,
                        cudaStream_t s) {
  if (d.K > kMaxK || d.N < 16 || d.M <= 0 || d.K <= 0 || !scratch) return false;
  const int64_t nb = (int64_t)d.nb0 * d.nb1;
  if (nb * (d.M + d.N) > scratch_words) return false;
  uint16_t* ea = scratch;
  uint16_t* fb = scratch + nb * d.M;
  count_launch(); ozaki_exponents_kernel<<<(unsigned)nb, 256, 0, s>>>(d, ea, fb, err);
  // tile width: the least of 32, 48, 64 that covers N in as many tiles as 64 would
  const int ntile64 = (d.N + 63) / 64;
  const int need = (d.N + ntile64 - 1) / ntile64;
  if (need <= 32) launch_persist<32>(d, ea, fb, nb, err, s);
  else if (need <= 48) launch_persist<48>(d, ea, fb, nb, err, s);
  else launch_persist<64>(d, ea, fb, nb, err, s);
  return true;
}

}  // namespace hdg
