// FP64-accurate block-row products with several right-hand sides on the BF16
// tensor cores: the face-block matvec y_f = sum_s K_f[s] x_{nbr[f][s]}
// (Sec. 4.3) with R = 4 or 8 right-hand sides, where FP64 arithmetic (two
// FMAs per clock per SM on this GPU) would otherwise bound the product far
// below the bandwidth of HBM.
//
// Exact digits.  Every row i of a unit's concatenated columns j (all slots)
// is written in fixed point relative to a power of two above its largest
// entry, X_ij = trunc(K_ij 2^{54 - e_i}), |X_ij| < 2^54, split into the
// 7-bit fields of its two's complement: X = d_0 128^7 + sum_{s>=1} d_s
// 128^{7-s} with d_0 = X >> 49 in [-32, 31] and d_s in [0, 127].  tc_split
// stores them once per assembly as bytes (d_0 + 64, d_1, ..., d_7): 8 bytes
// per entry, the size of the FP64 block, next to the row exponents.  The
// gathered x of a face row is split the same way per right-hand side r
// (exponent f_r over the row's columns) inside the product kernel.  A digit
// is exact in BF16, a digit product (< 2^14) is exact in FP32 and a sum of
// at most 352 of them (< 2^23) too, so every
//   D_st(i, r) = sum_j d_s(i, j) g_t(j, r)
// comes out of the tensor cores exactly, and
//   (K x)_ir = 2^{e_i + f_r - 108} sum_{s,t} D_st 128^{14 - s - t}.
// Pairs with s + t >= 10 carry weight below 2^-50 of the leading scale and
// are dropped; the rest is combined in 64-bit integers and rounded once to
// FP64.  With the truncation of X and Y the error stays below
// 4 * 2^-53 ncol max_j|K_ij| max_j|x_jr|, the size of FP64 rounding.
//
// Tiles.  The A operand (M = 128) holds the rows (s, i) as s * 32 + i (rows
// of at most 32): tile 0 takes s = 0..3 against t = 0..7 (N = 8 R), tile 1
// s = 4..7 against t = 0..5 (N = 6 R rounded up to 16), the B operand rows
// (t, r) as t * R + r.  One persistent CTA per SM walks the units:
//   warps 0-3   epilogue: tensor-memory loads of both accumulator tiles
//               (lane quadrant = warp), integer recombination, FP64 output;
//   warps 4-7   digits of K: the stored digit bytes of two 16-column steps
//               from the copy ring, converted to BF16 (a byte c as the bits
//               of 128 + c, minus 128 or 192) into a ring of A stages; a
//               thread owns up to two (digit, row) pairs for the whole kernel;
//   warps 8-19  x: per-RHS exponents of the unit's gathered columns, split
//               into the B operand of the whole unit (double-buffered); a
//               thread keeps one RHS;
//   warp 20     tensor-memory allocation and, on one lane, the MMAs (two
//               per 16-column step) with commits to the rings' mbarriers;
//   warp 21     one lane copies each unit's x slots (b x R doubles each,
//               through the neighbour table) into one of two x buffers;
//   warp 22     one lane copies the digit chunks (contiguous, evict-first in
//               L2) into a ring of six stages, independently of the x copies.
// The accumulators (8R + 6R columns) are double-buffered in tensor memory,
// so the epilogue of one unit overlaps the products of the next.  Every wait
// is bounded; on a timeout the kernel sets an error bit, stops, waits
// (bounded) for its issued MMAs and frees its tensor memory.
#include <algorithm>

#include "hdg_common.cuh"
#include "hdg_internal.h"
#include "k_umma.cuh"

namespace hdg {

namespace {

constexpr int kAW = 128;                     // digit converters (warps 4 ..)
constexpr int kBBase = 128 + kAW;            // first thread of the x splitters
constexpr int kBW = 384;                     // x splitters
constexpr int kMmaWarp = (kBBase + kBW) / 32;           // then the MMA warp and two copy warps
constexpr int kTcThreads = kBBase + kBW + 96;           // 23 warps
constexpr int kCK = 2;                       // 16-column steps per A stage
constexpr int kAStages = 2;
constexpr int kARows = 256;                  // (s, i) rows of both tiles
constexpr int kAStageBytes = kARows * kCK * 16 * 2;      // 16 KB
constexpr int kASBO = kCK * 2 * 128;                     // bytes between 8-row groups of an A stage
constexpr int kTmemCols = 256;

struct TcPlan {
  int nks_max;        // 16-column steps of the longest unit
  int b_off;          // byte offsets in shared memory
  int raw_off;
  int x_off;
  int red_off;
  int bar_off;
  int smem;
};

__device__ __forceinline__ int tc_exponent(double m) {
  // smallest e with m < 2^e (m > 0 finite): the exponent field minus 1022
  return (int)((__double_as_longlong(m) >> 52) & 0x7FF) - 1022;
}

// trunc(v 2^{54 - e}) as a signed 64-bit integer, |v| < 2^e
__device__ __forceinline__ long long tc_fixed(double v, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int exf = (int)((bits >> 52) & 0x7FF);
  if (exf == 0 || exf == 0x7FF) return 0;               // zero / subnormal / Inf, NaN (flagged elsewhere)
  const unsigned long long m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = exf - 1021 - e;                        // <= 1
  long long x;
  if (sh >= 0) x = (long long)(m << sh);
  else if (sh <= -63) x = 0;
  else x = (long long)(m >> (-sh));
  return (bits >> 63) ? -x : x;
}

// the 7-bit fields of x (|x| < 2^54) as stored bytes: d_0 + 64 (d_0 = x >> 49,
// signed), then d_1 .. d_7 (unsigned)
__device__ __forceinline__ void tc_digits(long long x, unsigned (&u)[8]) {
  const unsigned lo = (unsigned)x, hi = (unsigned)((unsigned long long)x >> 32);
  u[7] = lo & 127u;
  u[6] = (lo >> 7) & 127u;
  u[5] = (lo >> 14) & 127u;
  u[4] = (lo >> 21) & 127u;
  u[3] = __funnelshift_r(lo, hi, 28) & 127u;
  u[2] = (hi >> 3) & 127u;
  u[1] = (hi >> 10) & 127u;
  u[0] = (unsigned)((int)hi >> 17) + 64u;
}

// ------------------------------------------------------------------ split
// One thread per (unit, row): the row exponent over the unit's columns and
// the digit bytes of every 16-column step.
__global__ void __launch_bounds__(256) tc_split_kernel(BlockRowDesc d, unsigned char* dig, const int64_t* doff,
                                                       int32_t* ex) {
  const double* blk = static_cast<const double*>(d.blk);
  const int b = d.b_rows;
  const int64_t total = d.n_units * b;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / b;
    const int i = (int)(t - u * b);
    const int ncol = d.cnt[u] * d.bc;
    const double* row = blk + d.rowptr[u] * d.blk_stride + i;   // column-major blocks, FP64 ld = b
    auto at = [&](int j) {
      const int sl = j / d.bc, c = j - sl * d.bc;
      return row[(int64_t)sl * d.blk_stride + (int64_t)c * b];
    };
    double m = 0.0;
    bool bad = false;
    for (int j = 0; j < ncol; ++j) {
      const double v = fabs(at(j));
      if (!(v <= 1.7e308)) bad = true;
      m = fmax(m, v);
    }
    if (bad) atomicOr(d.err, ERRBIT_NAN);
    const int e = m > 0.0 ? tc_exponent(m) : 0;
    ex[t] = e;
    const int nk = (ncol + 15) / 16;
    unsigned char* base = dig + doff[u];
    for (int k = 0; k < nk; ++k) {
      unsigned w[8][4];
#pragma unroll
      for (int s = 0; s < 8; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) w[s][q] = 0;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = k * 16 + jj;
        unsigned dg[8];
        tc_digits(j < ncol ? tc_fixed(at(j), e) : 0ll, dg);
#pragma unroll
        for (int s = 0; s < 8; ++s) w[s][jj >> 2] |= dg[s] << (8 * (jj & 3));
      }
#pragma unroll
      for (int s = 0; s < 8; ++s)
        *reinterpret_cast<uint4*>(base + (((int64_t)k * 8 + s) * b + i) * 16) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// byte offset of (row, 8-column group kg) in a no-swizzle K-major operand
__device__ __forceinline__ uint32_t tc_core(int row, int kg, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(row & 7) * 16u;
}

// 8 stored digit bytes -> 8 BF16 digits (exact): a byte c in the low 7
// mantissa bits of 0x4300 gives 128 + c; subtract 128 (digits d_1 .. d_7) or
// 192 (the leading digit, stored as d_0 + 64).
__device__ __forceinline__ uint4 tc_bytes_to_bf16(uint2 raw, bool lead) {
  const float of = lead ? 192.f : 128.f;
  const __nv_bfloat162 off = __floats2bfloat162_rn(of, of);
  uint32_t o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t src = q < 2 ? raw.x : raw.y;
    // result bytes (src byte 2q' , 0x43, src byte 2q' + 1, 0x43), q' = q & 1
    const uint32_t pk = __byte_perm(src, 0x43434343u, (q & 1) ? 0x4342u : 0x4140u);
    const __nv_bfloat162 v = __hsub2(*reinterpret_cast<const __nv_bfloat162*>(&pk), off);
    o[q] = *reinterpret_cast<const uint32_t*>(&v);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// the epilogue modes of the block-row products (EPI_STORE, EPI_RESID, EPI_SCALE)
__device__ __forceinline__ void epi_store_tc(const BlockRowDesc& d, int64_t u, int row, int r, double v) {
  const int64_t o = (u * d.b_rows + row) * d.R + r;
  if (d.epi == EPI_RESID) v = d.rhs[o] - v;
  else if (d.epi == EPI_SCALE) v = d.scale[r] * v;
  if (d.out) d.out[o] = v;
  if (d.out32) d.out32[o] = (float)v;
}

constexpr int kRawStages = 6;                 // raw digit chunks in flight per CTA

struct TcBars {
  uint64_t raw_full[kRawStages], raw_empty[kRawStages];
  uint64_t xs_full[2], xs_empty[2];
  uint64_t a_full[kAStages], a_empty[kAStages];
  uint64_t b_full[2], b_empty[2];
  uint64_t d_full[2], d_empty[2];
  uint64_t f_full[4];
  uint64_t done;
  uint32_t tmem;
  int abort;           // any role gave up (bounded wait): everyone stops
  int bstop, estop;    // the x producers' / the epilogue's own stop flags (set before their named barriers)
  long long issued_raw[kRawStages];   // last use of each copy stage (drained after an abort)
  long long issued_xs[2];
  int fexp[4][8];
};
__device__ __forceinline__ bool tc_aborted(TcBars* b) { return *(volatile int*)&b->abort != 0; }
__device__ __forceinline__ void tc_give_up(TcBars* b, unsigned* err) {
  atomicOr(err, ERRBIT_TIMEOUT);
  *(volatile int*)&b->abort = 1;
}

template <int R>
__global__ void __launch_bounds__(kTcThreads, 1) tc_blockrow_kernel(BlockRowDesc d, const unsigned char* dig,
                                                                    const int64_t* doff, const int32_t* ex,
                                                                    TcPlan pl) {
  constexpr int NA = 8 * R;                          // tile 0: t = 0..7
  constexpr int NB = ((6 * R + 15) / 16) * 16;       // tile 1: t = 0..5 (rounded up to whole 16 columns)
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* astage = smem;                                     // kAStages x 16 KB
  unsigned char* bbuf = smem + pl.b_off;                            // 2 x (64 rows x nks_max*16 columns)
  unsigned char* rawbuf = smem + pl.raw_off;                        // kRawStages x raw chunk
  double* xsbuf = reinterpret_cast<double*>(smem + pl.x_off);      // 2 x (max_slots * b x R)
  long long* red = reinterpret_cast<long long*>(smem + pl.red_off); // 4 x 32 x R x 2
  TcBars* bars = reinterpret_cast<TcBars*>(smem + pl.bar_off);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = d.b_rows, ms = d.max_slots;
  const uint32_t b_sbo = (uint32_t)pl.nks_max * 2u * 128u;
  const int b_bytes = 64 * pl.nks_max * 16 * 2;
  const int raw_bytes = kCK * 8 * b * 16;
  const int xs_elems = ms * b * R;

  if (tid == 0) {
    for (int i = 0; i < kRawStages; ++i) {
      mbar_init(&bars->raw_full[i], 1);
      mbar_init(&bars->raw_empty[i], kAW);
      bars->issued_raw[i] = -1;
    }
    for (int i = 0; i < kAStages; ++i) {
      mbar_init(&bars->a_full[i], kAW);
      mbar_init(&bars->a_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->xs_full[i], 1);
      mbar_init(&bars->xs_empty[i], kBW);
      bars->issued_xs[i] = -1;
      mbar_init(&bars->b_full[i], kBW);
      mbar_init(&bars->b_empty[i], 1);
      mbar_init(&bars->d_full[i], 1);
      mbar_init(&bars->d_empty[i], 4);
    }
    for (int i = 0; i < 4; ++i) mbar_init(&bars->f_full[i], 1);
    mbar_init(&bars->done, 1);
    bars->abort = 0;
    bars->bstop = 0;
    bars->estop = 0;
    fence_mbar_init();
  }
  // A rows past b (i >= b) are never written: zero the whole ring once
  for (int o = tid * 16; o < kAStages * kAStageBytes; o += kTcThreads * 16)
    *reinterpret_cast<uint4*>(astage + o) = make_uint4(0, 0, 0, 0);
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem;
  auto nks_of = [&](int64_t u) { return (d.cnt[u] * d.bc + 15) / 16; };

  if (warp == kMmaWarp + 1) {
    // ------------------------------------------------------- x slots (one lane)
    // per unit: its x slots (contiguous b x R doubles each, through the
    // neighbour table) into one of two x buffers
    if (lane == 0) {
      int64_t n = 0;
      const unsigned xbytes = (unsigned)(b * R * 8);
      for (int64_t u = blockIdx.x; u < d.n_units; u += gridDim.x, ++n) {
        const int xb = (int)(n & 1);
        if (tc_aborted(bars) || !mbar_wait_bounded(&bars->xs_empty[xb], (unsigned)(((n >> 1) & 1) ^ 1))) {
          tc_give_up(bars, d.err);
          break;
        }
        const int cnt = d.cnt[u];
        const int32_t* nbr = d.nbr + u * ms;
        double* xdst = xsbuf + (size_t)xb * xs_elems;
        bars->issued_xs[xb] = n;
        mbar_arrive_expect_tx(&bars->xs_full[xb], xbytes * (unsigned)cnt);
        for (int sl = 0; sl < cnt; ++sl)
          bulk_g2s(xdst + (size_t)sl * b * R, d.in + (int64_t)nbr[sl] * b * R, xbytes, &bars->xs_full[xb]);
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp + 2) {
    // ------------------------------------------------------- digit chunks (one lane)
    // each unit's digits (contiguous), two 16-column steps per copy,
    // evict-first in L2, into a ring of six stages
    if (lane == 0) {
      uint64_t pol;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
      int64_t rseq = 0;
      for (int64_t u = blockIdx.x; u < d.n_units && !tc_aborted(bars); u += gridDim.x) {
        const int nks = nks_of(u);
        const unsigned char* src = dig + doff[u];
        bool ok = true;
        for (int k0 = 0; k0 < nks; k0 += kCK, ++rseq) {
          const int st = (int)(rseq % kRawStages);
          if (tc_aborted(bars) ||
              !mbar_wait_bounded(&bars->raw_empty[st], (unsigned)(((rseq / kRawStages) & 1) ^ 1))) {
            ok = false;
            break;
          }
          const unsigned bytes = (unsigned)(min(kCK, nks - k0) * 8 * b * 16);
          bars->issued_raw[st] = rseq;
          mbar_arrive_expect_tx(&bars->raw_full[st], bytes);
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, "
              "[%3], %4;" ::"r"(smem_u32(rawbuf + (size_t)st * raw_bytes)),
              "l"(src + (int64_t)k0 * 8 * b * 16), "r"(bytes), "r"(smem_u32(&bars->raw_full[st])), "l"(pol)
              : "memory");
        }
        if (!ok) {
          tc_give_up(bars, d.err);
          break;
        }
      }
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 4 + kAW / 32) {
    // ------------------------------------------------------- digits of K: raw ring -> A stages
    // thread tq < 8 b owns digit sd of row i for the whole kernel (raw piece
    // (kk, sd, i) at ((kk * 8 + sd) * b + i) * 16 bytes), so only the column
    // step moves its source and destination
    const int tq = tid - 128;
    int npc = 0;                       // (digit, row) pairs of this thread: tq, tq + kAW
    uint32_t drow[2] = {0u, 0u};
    bool lead[2] = {false, false};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int pr = tq + h * kAW;
      if (pr < 8 * b) {
        const int sd = pr / b, ci = pr - sd * b;
        drow[h] = tc_core(sd * 32 + ci, 0, kASBO);
        lead[h] = sd == 0;
        npc = h + 1;
      }
    }
    const int raw_step = 8 * b * 16;
    int64_t seq = 0;
    for (int64_t u = blockIdx.x; u < d.n_units && !tc_aborted(bars); u += gridDim.x) {
      const int nks = nks_of(u);
      bool ok = true;
      for (int k0 = 0; k0 < nks; k0 += kCK, ++seq) {
        const int rs = (int)(seq % kRawStages), as = (int)(seq % kAStages);
        if (tc_aborted(bars) || !mbar_wait_bounded(&bars->raw_full[rs], (unsigned)((seq / kRawStages) & 1)) ||
            !mbar_wait_bounded(&bars->a_empty[as], (unsigned)(((seq / kAStages) & 1) ^ 1))) {
          ok = false;
          break;
        }
        const int nk = min(kCK, nks - k0);
        // 16 stored bytes = 16 columns of one digit of one row, per 16-column step kk
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h < npc) {
            const unsigned char* raw = rawbuf + (size_t)rs * raw_bytes + (tq + h * kAW) * 16;
            unsigned char* dst = astage + as * kAStageBytes + drow[h];
#pragma unroll
            for (int kk = 0; kk < kCK; ++kk) {
              if (kk < nk) {
                const uint4 q = *reinterpret_cast<const uint4*>(raw + kk * raw_step);
                *reinterpret_cast<uint4*>(dst + kk * 256) = tc_bytes_to_bf16(make_uint2(q.x, q.y), lead[h]);
                *reinterpret_cast<uint4*>(dst + kk * 256 + 128) = tc_bytes_to_bf16(make_uint2(q.z, q.w), lead[h]);
              }
            }
          }
        }
        fence_async_smem();
        mbar_arrive(&bars->a_full[as]);
        mbar_arrive(&bars->raw_empty[rs]);
      }
      if (!ok) {
        tc_give_up(bars, d.err);
        break;
      }
    }
  } else if (warp >= kBBase / 32 && warp < (kBBase + kBW) / 32) {
    // ------------------------------------------------------- x: exponents and split
    const int tq = tid - kBBase;
    __shared__ int s_fmax[kBW / 32][8];
    int64_t n = 0;
    for (int64_t u = blockIdx.x; u < d.n_units; u += gridDim.x, ++n) {
      const int ncol = d.cnt[u] * d.bc;
      const int nks = (ncol + 15) / 16;
      const int kp = nks * 16;
      const int xb = (int)(n & 1), bb = (int)(n & 1);
      const unsigned ph = (unsigned)((n >> 1) & 1);
      if (tc_aborted(bars) || !mbar_wait_bounded(&bars->xs_full[xb], ph)) {
        tc_give_up(bars, d.err);
        bars->bstop = 1;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kBW) : "memory");
      if (*(volatile int*)&bars->bstop) break;
      const double* xs = xsbuf + (size_t)xb * xs_elems;      // (slot, column, r) = x of column j at j * R
      // per-RHS exponent over the columns (integer maximum of |x| as bit
      // patterns): thread (r = tq % R) takes j = tq / R, + kBW / R, ...
      {
        const int r = tq % R;
        unsigned long long m = 0;
        for (int j = tq / R; j < ncol; j += kBW / R)
          m = max(m, (unsigned long long)__double_as_longlong(xs[j * R + r]) & 0x7FFFFFFFFFFFFFFFull);
        for (int o = R; o < 32; o <<= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
        const int ef = (int)(m >> 52);
        if (lane < R) s_fmax[tq >> 5][lane] = m ? ef - 1022 : -100000;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kBW) : "memory");
      // this thread's RHS is tq % R in every work item below (kBW is a multiple of R)
      const int my_r = tq % R;
      int my_f;
      {
        int a = -100000;
        for (int q = 0; q < kBW / 32; ++q) a = max(a, s_fmax[q][my_r]);
        my_f = a < -90000 ? 0 : a;
      }
      if (tc_aborted(bars) || !mbar_wait_bounded(&bars->b_empty[bb], ph ^ 1u)) {
        tc_give_up(bars, d.err);
        bars->bstop = 1;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kBW) : "memory");
      if (*(volatile int*)&bars->bstop) break;
      unsigned char* bdst = bbuf + bb * b_bytes;
      // work item (8-column group jg, r): 8 values -> 8 digit planes t, 16 bytes each
      for (int w = tq; w < (kp / 8) * R; w += kBW) {
        const int jg = w / R, r = my_r;
        unsigned dg[8][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = jg * 8 + q;
          tc_digits(j < ncol ? tc_fixed(xs[j * R + r], my_f) : 0ll, dg[q]);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          uint2 raw;
          raw.x = dg[0][t] | (dg[1][t] << 8) | (dg[2][t] << 16) | (dg[3][t] << 24);
          raw.y = dg[4][t] | (dg[5][t] << 8) | (dg[6][t] << 16) | (dg[7][t] << 24);
          *reinterpret_cast<uint4*>(bdst + tc_core(t * R + r, jg, b_sbo)) = tc_bytes_to_bf16(raw, t == 0);
        }
      }
      if (tq < R) {
        bars->fexp[n & 3][tq] = my_f;
      }
      fence_async_smem();
      mbar_arrive(&bars->b_full[bb]);
      mbar_arrive(&bars->xs_empty[xb]);
      if (tq == 0) mbar_arrive(&bars->f_full[n & 3]);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idA = instr_desc(NA), idB = instr_desc(NB);
      int64_t aseq = 0, n = 0;
      bool issued = false;
      for (int64_t u = blockIdx.x; u < d.n_units; u += gridDim.x, ++n) {
        const int bb = (int)(n & 1);
        const unsigned ph = (unsigned)((n >> 1) & 1);
        if (tc_aborted(bars) || !mbar_wait_bounded(&bars->b_full[bb], ph) ||
            !mbar_wait_bounded(&bars->d_empty[bb], ph ^ 1u)) {
          tc_give_up(bars, d.err);
          break;
        }
        tc_fence_after();
        const int nks = nks_of(u);
        const uint32_t dA = tmem + (uint32_t)(bb * 128), dB = dA + 64u;
        const uint32_t bbase = smem_u32(bbuf + bb * b_bytes);
        bool ok = true;
        for (int k0 = 0; k0 < nks; k0 += kCK, ++aseq) {
          const int st = (int)(aseq % kAStages);
          if (!mbar_wait_bounded(&bars->a_full[st], (unsigned)((aseq / kAStages) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = smem_u32(astage + st * kAStageBytes);
          const int nk = min(kCK, nks - k0);
          for (int kk = 0; kk < nk; ++kk) {
            const uint64_t a0 = smem_desc(abase + (uint32_t)kk * 256u, 128u, kASBO);
            const uint64_t a1 = smem_desc(abase + 16u * kASBO + (uint32_t)kk * 256u, 128u, kASBO);
            const uint64_t bd = smem_desc(bbase + (uint32_t)(k0 + kk) * 256u, 128u, b_sbo);
            const uint32_t acc = (k0 + kk) > 0 ? 1u : 0u;
            umma_bf16(dA, a0, bd, idA, acc);
            umma_bf16(dB, a1, bd, idB, acc);
          }
          umma_commit(&bars->a_empty[st]);
          issued = true;
        }
        if (!ok) {
          tc_give_up(bars, d.err);
          break;
        }
        umma_commit(&bars->b_empty[bb]);
        umma_commit(&bars->d_full[bb]);
      }
      // wait (bounded) for every issued MMA before the tensor memory is freed
      if (issued) {
        umma_commit(&bars->done);
        if (!mbar_wait_bounded(&bars->done, 0)) atomicOr(d.err, ERRBIT_TIMEOUT);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------- epilogue
    const int q = warp;                                  // lane quadrant: rows (s = q | s = 4 + q, i = lane)
    int64_t n = 0;
    for (int64_t u = blockIdx.x; u < d.n_units; u += gridDim.x, ++n) {
      const int bb = (int)(n & 1);
      const unsigned ph = (unsigned)((n >> 1) & 1);
      if (tc_aborted(bars) || !mbar_wait_bounded(&bars->d_full[bb], ph) ||
          !mbar_wait_bounded(&bars->f_full[n & 3], (unsigned)((n >> 2) & 1))) {
        tc_give_up(bars, d.err);
        bars->estop = 1;
      }
      asm volatile("bar.sync 2, 128;" ::: "memory");
      if (*(volatile int*)&bars->estop) break;
      tc_fence_after();
      // H = sum_{w <= 4} D 128^{4 - w}, L = sum_{5 <= w <= 9} D 128^{9 - w}, w = s + t;
      // accumulator columns (t, r) = t R + r, 16 at a time
      long long H[R], L[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        H[r] = 0;
        L[r] = 0;
      }
      const uint32_t tA = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(bb * 128);
#pragma unroll
      for (int c = 0; c < NA + NB; c += 16) {
        uint32_t v16[16];
        const bool tile1 = c >= NA;
        const int c0 = tile1 ? c - NA : c;
        tmem_ld16_nowait(tA + (tile1 ? 64u : 0u) + (uint32_t)c0, v16);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int col = c0 + k;
          const int t = col / R, r = col - t * R;
          const int w = (tile1 ? 4 : 0) + q + t;
          const long long v = (long long)__float2int_rn(__uint_as_float(v16[k]));
          if (w <= 4) H[r] += v << (7 * (4 - w));
          else if (w <= 9) L[r] += v << (7 * (9 - w));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->d_empty[bb]);
      // partials in [quadrant][r][H/L][row]: a warp's 32 lanes write 256
      // contiguous bytes per store
#pragma unroll
      for (int r = 0; r < R; ++r) {
        red[((q * R + r) * 2) * 32 + lane] = H[r];
        red[((q * R + r) * 2 + 1) * 32 + lane] = L[r];
      }
      asm volatile("bar.sync 2, 128;" ::: "memory");
      for (int o = tid; o < b * R; o += 128) {
        const int r = o / b, i = o - r * b;
        long long h = 0, l = 0;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          h += red[((qq * R + r) * 2) * 32 + i];
          l += red[((qq * R + r) * 2 + 1) * 32 + i];
        }
        // (h 2^35 + l) 2^sc with one rounding, the power of two built exactly
        const int sc = ex[u * b + i] + bars->fexp[n & 3][r] - 73;
        const double p2 = (sc >= -1022 && sc <= 1023) ? __longlong_as_double((long long)(sc + 1023) << 52)
                                                      : scalbn(1.0, sc);
        epi_store_tc(d, u, i, r, fma((double)h, 34359738368.0, (double)l) * p2);
      }
      asm volatile("bar.sync 2, 128;" ::: "memory");
    }
  }
  __syncthreads();
  // after an abort, bulk copies may still be in flight: wait (bounded) for
  // them before the CTA's shared memory goes away
  if (tid == 0 && tc_aborted(bars)) {
    for (int i = 0; i < kRawStages; ++i) {
      const long long qn = bars->issued_raw[i];
      if (qn >= 0) mbar_wait_bounded(&bars->raw_full[i], (unsigned)((qn / kRawStages) & 1));
    }
    for (int i = 0; i < 2; ++i) {
      const long long qn = bars->issued_xs[i];
      if (qn >= 0) mbar_wait_bounded(&bars->xs_full[i], (unsigned)((qn >> 1) & 1));
    }
  }
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

TcPlan tc_plan(const BlockRowDesc& d, int R) {
  TcPlan pl{};
  pl.nks_max = (d.max_slots * d.bc + 15) / 16;
  const int b_bytes = 64 * pl.nks_max * 16 * 2;
  pl.b_off = kAStages * kAStageBytes;
  pl.raw_off = pl.b_off + 2 * b_bytes;
  pl.x_off = pl.raw_off + (kRawStages * kCK * 8 * d.b_rows * 16 + 127) / 128 * 128;
  pl.red_off = pl.x_off + (2 * d.max_slots * d.b_rows * R * 8 + 127) / 128 * 128;
  pl.bar_off = pl.red_off + 4 * 32 * R * 2 * 8;
  pl.smem = pl.bar_off + (int)((sizeof(TcBars) + 127) / 128 * 128);
  return pl;
}

}  // namespace

int64_t tc_digit_layout(const int64_t* h_rowptr, int64_t n_units, int b_rows, int bc, int64_t* h_doff) {
  int64_t off = 0;
  for (int64_t u = 0; u < n_units; ++u) {
    h_doff[u] = off;
    const int64_t ncol = (h_rowptr[u + 1] - h_rowptr[u]) * bc;
    off += (ncol + 15) / 16 * 8 * b_rows * 16;
  }
  h_doff[n_units] = off;
  return off;
}

bool tc_supported(const BlockRowDesc& d) {
  if (d.prec != HDG_FP64 || (d.R != 4 && d.R != 8)) return false;
  if (d.b_rows > 32 || d.bc != d.b_rows || d.epi == EPI_POLY) return false;
  // the x slots move by bulk copies: 16-byte aligned source, whole 16-byte rows
  if (((uintptr_t)d.in & 15u) != 0 || (d.b_rows * d.R * 8) % 16 != 0) return false;
  const TcPlan pl = tc_plan(d, d.R);
  return pl.smem <= 226 * 1024;
}

void tc_split(const BlockRowDesc& d, unsigned char* dig, const int64_t* doff, int32_t* ex, cudaStream_t s) {
  const int64_t total = d.n_units * d.b_rows;
  if (total <= 0) return;
  int64_t g = (total + 255) / 256;
  if (g > 8192) g = 8192;
  count_launch(); tc_split_kernel<<<(unsigned)g, 256, 0, s>>>(d, dig, doff, ex);
}

bool tc_blockrow(const BlockRowDesc& d, const unsigned char* dig, const int64_t* doff, const int32_t* ex,
                 cudaStream_t s) {
  if (!tc_supported(d) || d.n_units <= 0) return false;
  const TcPlan pl = tc_plan(d, d.R);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(d.n_units, std::max(nsm, 1));
  if (d.R == 8) {
    cudaFuncSetAttribute(tc_blockrow_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
    count_launch(); tc_blockrow_kernel<8><<<(unsigned)grid, kTcThreads, pl.smem, s>>>(d, dig, doff, ex, pl);
  } else {
    cudaFuncSetAttribute(tc_blockrow_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
    count_launch(); tc_blockrow_kernel<4><<<(unsigned)grid, kTcThreads, pl.smem, s>>>(d, dig, doff, ex, pl);
  }
  return true;
}

}  // namespace hdg
