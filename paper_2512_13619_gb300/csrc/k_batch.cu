// Restarted GMRES for many small trace systems in ONE persistent launch: the
// batching of the serving path (systems of different meshes, polynomial
// orders and block sizes solved together).
//
// One cooperative kernel runs the whole solve of every system in the batch
// (Sec. 3.1 restarted, left-preconditioned GMRES(m) with classical
// Gram-Schmidt, Sec. 4.4, and block-Jacobi, Sec. 4.5): the cycles and
// iterations of all systems advance in lock-step, each phase spread over the
// whole grid through ragged work lists (all systems' trace rows, vector
// entries, and fixed 4096-entry reduction chunks), and phases are separated
// by a grid barrier.  A system that has converged only skips its work.  The
// host launches once per batch and reads the counts at the end.
//
// Determinism: each row product is summed by one thread in a fixed order,
// each reduction chunk by one warp in a fixed lane order, and the chunk sums
// of a system are added in chunk order, so a system's results do not depend
// on which other systems share the batch (nor on the grid size).
//
// Precision: FP64 blocks throughout, or (restarted mixed mode) FP32 blocks of
// K and of the block-Jacobi inverses inside the cycles with FP32
// accumulation, while the Krylov basis, Gram-Schmidt, Givens rotations and the
// true residual b - K x at every restart stay FP64.
//
// The grid barrier is a counter and a generation word in device memory; every
// wait gives up after a second, sets an error bit and stops the solve.
#include <algorithm>
#include <vector>

#include "hdg_common.cuh"
#include "hdg_gmres.h"
#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kPerThread = 8;                     // vector entries per thread in a chunk
constexpr int kChunk = kBThreads * kPerThread;    // entries per reduction chunk (one CTA)
constexpr int kSlotGroup = 8;                     // Gram-Schmidt slots per dot task

struct GridBar {
  unsigned count, gen;
  int abort;
};

__device__ bool grid_barrier(GridBar* gb, unsigned* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = *(volatile unsigned*)&gb->gen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
      *(volatile unsigned*)&gb->count = 0;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*(volatile unsigned*)&gb->gen == gen) {
        if (*(volatile int*)&gb->abort) break;
        if (global_ns() - t0 > kWaitLimitNs) {
          atomicOr(err, ERRBIT_TIMEOUT);
          *(volatile int*)&gb->abort = 1;
          break;
        }
      }
    }
    __threadfence();
    s_ok = !*(volatile int*)&gb->abort;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int find_item(const int64_t* pre, int n, int64_t g) {
  int lo = 0, hi = n - 1;             // largest p with pre[p] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool any_of(const int* a, int R) {
  for (int r = 0; r < R; ++r)
    if (a[r]) return true;
  return false;
}

// Sum of a system's chunk partials of one slot and RHS, by one warp: lane l
// adds chunks l, l + 32, ... in order, then a fixed butterfly (every lane
// ends with the same value, independent of the batch).
__device__ __forceinline__ double warp_chunk_sum(const BatchItem& it, int slot, int r, int lane) {
  double s = 0.0;
  const double* pp = it.part + (int64_t)slot * it.nchunks * it.R + r;
  for (int64_t c = lane; c < it.nchunks; c += 32) s += pp[c * it.R];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Fixed-order CTA reduction of v (per RHS r = lane % R) into part[slot][c][r].
// sred: kBWarps * kSlotGroup * kMaxR doubles; q indexes the value in a group.
__device__ __forceinline__ void cta_stage(double v, int q, int R, double* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = R; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane < R) sred[(warp * kSlotGroup + q) * kMaxR + lane] = v;
}
__device__ __forceinline__ void cta_finish(const BatchItem& it, int nq, int slot0, int64_t c, const double* sred) {
  const int t = threadIdx.x, R = it.R;
  if (t < nq * R) {
    const int q = t / R, r = t - q * R;
    double s = 0.0;
    for (int w = 0; w < kBWarps; ++w) s += sred[(w * kSlotGroup + q) * kMaxR + r];
    it.part[((int64_t)(slot0 + q) * it.nchunks + c) * R + r] = s;
  }
}

// Row bodies, templated on the RHS count so the accumulators stay in registers.
// y[r] = sum_{s = s0, s0 + ds, ...} sum_c K_f,s(i, c) x_nbr(s)(c, r) with FP64
// blocks (FP64 sums); the column loops are unrolled so their loads overlap.
template <int R>
__device__ __forceinline__ void kprod64(const BatchItem& it, const double* x, int64_t f, int i, int s0, int ds,
                                        double* acc) {
  const int b = it.b;
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  const int n = it.cnt[f];
  const int64_t rp = it.rowptr[f];
  const int32_t* nbr = it.nbr + f * it.ms;
  for (int s = s0; s < n; s += ds) {
    const double* blk = it.K64 + (rp + s) * it.s64 + i;
    const double* xv = x + (int64_t)nbr[s] * b * R;
#pragma unroll 4
    for (int c = 0; c < b; ++c) {
      const double kv = blk[(int64_t)c * b];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(kv, xv[c * R + r], acc[r]);
    }
  }
}
// the same with FP32 blocks, FP32 x and FP32 sums
template <int R>
__device__ __forceinline__ void kprod32(const BatchItem& it, const float* x, int64_t f, int i, int s0, int ds,
                                        float* a32) {
  const int b = it.b;
#pragma unroll
  for (int r = 0; r < R; ++r) a32[r] = 0.f;
  const int n = it.cnt[f];
  const int64_t rp = it.rowptr[f];
  const int32_t* nbr = it.nbr + f * it.ms;
  for (int s = s0; s < n; s += ds) {
    const float* blk = it.K32 + (rp + s) * it.s32 + i;
    const float* xv = x + (int64_t)nbr[s] * b * R;
#pragma unroll 4
    for (int c = 0; c < b; ++c) {
      const float kv = blk[(int64_t)c * it.ld32];
#pragma unroll
      for (int r = 0; r < R; ++r) a32[r] = fmaf(kv, xv[c * R + r], a32[r]);
    }
  }
}
// z = P_f^{-1} y for row i of face f; y(c, r) = y[c * ys + r].  FP64 systems
// apply the FP64 inverse, FP32 systems round y to FP32 and apply the FP32
// inverse with FP32 sums; the identity when there is no preconditioner.
template <int R>
__device__ __forceinline__ void bj_row(const BatchItem& it, const double* y, int ys, int64_t f, int i, double* acc) {
  const int b = it.b;
  const bool f64 = it.kprec == HDG_FP64;
  if (it.pc == HDG_PC_NONE) {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = f64 ? y[i * ys + r] : (double)(float)y[i * ys + r];
  } else if (f64) {
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    const double* blk = it.bj64 + f * it.bs64 + i;
#pragma unroll 4
    for (int c = 0; c < b; ++c) {
      const double kv = blk[(int64_t)c * b];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(kv, y[c * ys + r], acc[r]);
    }
  } else {
    float a32[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a32[r] = 0.f;
    const float* blk = it.bj32 + f * it.bs32 + i;
#pragma unroll 4
    for (int c = 0; c < b; ++c) {
      const float kv = blk[(int64_t)c * it.ld32];
#pragma unroll
      for (int r = 0; r < R; ++r) a32[r] = fmaf(kv, (float)y[c * ys + r], a32[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = a32[r];
  }
}

//   mode 1: res = rhs - K x             (FP64 blocks and x)
//   mode 2: out = P^{-1} in             (in = b into t1, or res into V_0; the
//           FP32 copy of V_0 goes to x32 for FP32 systems)
template <int R>
__device__ __forceinline__ void row_task(const BatchItem& it, int mode, bool to_v0, int64_t f, int i) {
  const int b = it.b;
  double acc[R];
  if (mode == 2) bj_row<R>(it, (to_v0 ? it.res : it.rhs) + f * b * R, R, f, i, acc);
  else kprod64<R>(it, it.x, f, i, 0, 1, acc);
  double* out = mode == 1 ? it.res : to_v0 ? it.V : it.t1;
  const bool o32 = mode == 2 && to_v0 && it.kprec != HDG_FP64;
  const int64_t o = (f * b + i) * R;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double v = acc[r];
    if (mode == 1) v = it.rhs[o + r] - v;
    out[o + r] = v;
    if (o32) it.x32[o + r] = (float)v;
  }
}

// RMAX: the largest RHS count of the batch (the kernel is compiled for 2 and 8)
#define HDG_BY_R(F, ...)                                              \
  switch (it.R) {                                                     \
    case 1: F<1>(__VA_ARGS__); break;                                 \
    case 2: if constexpr (RMAX >= 2) F<2>(__VA_ARGS__); break;        \
    case 4: if constexpr (RMAX >= 4) F<4>(__VA_ARGS__); break;        \
    default: if constexpr (RMAX >= 8) F<8>(__VA_ARGS__); break;       \
  }

// one thread per trace row (f, i) of every system not yet done
template <int RMAX>
__device__ void rows_phase(const BatchDesc& B, int mode, bool to_v0) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < B.rows_total; gi += nthreads) {
    const int p = find_item(B.row_pre, B.n, gi);
    const BatchItem& it = B.items[p];
    if (it.done_all[0]) continue;
    const int64_t lr = gi - B.row_pre[p];
    const int64_t f = lr / it.b;
    const int i = (int)(lr - f * it.b);
    HDG_BY_R(row_task, it, mode, to_v0, f, i)
  }
}

// Layout of the fused step for one system.  FP64 systems: one thread per
// row of a face row (b threads), FP32 systems: one thread per 4 rows (ld32/4
// threads, 16-byte loads of a column).  In a small system (at most 32768
// trace rows) a face row's slots are also split over SP = 4 or 2 threads, so
// that its few faces spread over many CTAs; large systems keep SP = 1.  A CTA
// takes fpc faces (its FP32 partial sums, fpc SP ld32 R floats, fit the
// 16 KB staging area).  The choice depends on the system alone.
struct KbjLayout {
  int sp, fpc;
};
__host__ __device__ __forceinline__ KbjLayout kbj_layout(int64_t nfree, int b, int ld32, int R, bool f32) {
  KbjLayout l;
  const int tpr = f32 ? ld32 / 4 : b;                   // threads per face row and slot part
  l.sp = (nfree * b > 32768) ? 1 : (tpr <= 64 ? 4 : tpr <= 128 ? 2 : 1);
  l.fpc = kBThreads / (tpr * l.sp);
  if (f32) {
    const int cap = (kBThreads * kMaxR * 2) / (l.sp * ld32 * R);
    if (cap < l.fpc) l.fpc = cap;
  }
  if (l.fpc < 1) l.fpc = 1;
  return l;
}

// FP32 systems: 4 rows (rg*4 .. rg*4+3) of face f, slots s0, s0 + ds, ...;
// one 16-byte load per column, FP32 sums.  BC > 0: the column count is BC
// (fully unrolled); BC = 0: it.b columns.  The next slot's neighbour index is
// loaded before the current slot's columns.
template <int R, int BC>
__device__ __forceinline__ void kprod32v_bc(const BatchItem& it, int64_t f, int rg, int s0, int ds, float (&a)[4][R]) {
  const int b = BC > 0 ? BC : it.b, ld = it.ld32;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int r = 0; r < R; ++r) a[v][r] = 0.f;
  const int n = it.cnt[f];
  const int64_t rp = it.rowptr[f];
  const int32_t* nbr = it.nbr + f * it.ms;
  int nb = s0 < n ? nbr[s0] : 0;
  for (int s = s0; s < n; s += ds) {
    const float* blk = it.K32 + (rp + s) * it.s32 + rg * 4;
    const float* xv = it.x32 + (int64_t)nb * b * R;
    nb = s + ds < n ? nbr[s + ds] : 0;
#pragma unroll(BC > 0 ? BC : (R <= 2 ? 8 : 4))
    for (int c = 0; c < b; ++c) {
      const float4 k = __ldg(reinterpret_cast<const float4*>(blk + (int64_t)c * ld));
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float xr = xv[c * R + r];
        a[0][r] = fmaf(k.x, xr, a[0][r]);
        a[1][r] = fmaf(k.y, xr, a[1][r]);
        a[2][r] = fmaf(k.z, xr, a[2][r]);
        a[3][r] = fmaf(k.w, xr, a[3][r]);
      }
    }
  }
}
template <int R>
__device__ __forceinline__ void kprod32v(const BatchItem& it, int64_t f, int rg, int s0, int ds, float (&a)[4][R]) {
  if constexpr (R <= 2) {
    switch (it.b) {
      case 4: kprod32v_bc<R, 4>(it, f, rg, s0, ds, a); return;
      case 9: kprod32v_bc<R, 9>(it, f, rg, s0, ds, a); return;
      case 16: kprod32v_bc<R, 16>(it, f, rg, s0, ds, a); return;
      default: break;
    }
  }
  kprod32v_bc<R, 0>(it, f, rg, s0, ds, a);
}

// FP32 fused step for thread (face lf, part sp, row group rg); sp32 is the
// CTA's FP32 staging area, rows of (face, part) at ((lf SP + sp) ld32 + row) R.
template <int R>
__device__ __forceinline__ void kbj32_k(const BatchItem& it, int64_t f, int lf, int sp, int rg, float* sp32) {
  float a[4][R];
  kprod32v<R>(it, f, rg, sp, it.sp, a);
  float* o = sp32 + ((int64_t)(lf * it.sp + sp) * it.ld32 + rg * 4) * R;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int r = 0; r < R; ++r) o[v * R + r] = a[v][r];
}
// part 0: y = (float)(vscale_j * (sum of the parts in order, in FP32))
template <int R>
__device__ __forceinline__ void kbj32_sum(const BatchItem& it, int j, int lf, int rg, float* sp32) {
  const int SP = it.sp, ld = it.ld32;
  float* o = sp32 + ((int64_t)lf * SP * ld + rg * 4) * R;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float w = o[v * R + r];
      for (int q = 1; q < SP; ++q) w += o[(q * ld + v) * R + r];
      o[v * R + r] = (float)((double)w * it.vscale[(int64_t)j * R + r]);
    }
}
// V_{j+1} rows rg*4.. of face f = P_f^{-1} y (FP32 inverse, FP32 sums), or y
template <int R>
__device__ __forceinline__ void kbj32_bj(const BatchItem& it, int j, int64_t f, int lf, int rg, const float* sp32) {
  const int b = it.b, ld = it.ld32;
  const float* y = sp32 + (int64_t)lf * it.sp * ld * R;     // part 0 of face lf: row c at c R
  float z[4][R];
  if (it.pc == HDG_PC_NONE) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int r = 0; r < R; ++r) z[v][r] = y[(rg * 4 + v) * R + r];
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int r = 0; r < R; ++r) z[v][r] = 0.f;
    const float* blk = it.bj32 + f * it.bs32 + rg * 4;
#pragma unroll(R <= 2 ? 8 : 4)
    for (int c = 0; c < b; ++c) {
      const float4 k = __ldg(reinterpret_cast<const float4*>(blk + (int64_t)c * ld));
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float yr = y[c * R + r];
        z[0][r] = fmaf(k.x, yr, z[0][r]);
        z[1][r] = fmaf(k.y, yr, z[1][r]);
        z[2][r] = fmaf(k.z, yr, z[2][r]);
        z[3][r] = fmaf(k.w, yr, z[3][r]);
      }
    }
  }
  double* out = it.V + (int64_t)(j + 1) * it.len + f * b * R;
#pragma unroll
  for (int v = 0; v < 4; ++v)
    if (rg * 4 + v < b)
#pragma unroll
      for (int r = 0; r < R; ++r) out[(rg * 4 + v) * R + r] = z[v][r];
}

// the three steps of the fused step for row i of face f, slot part sp
template <int R>
__device__ __forceinline__ void kbj_k(const BatchItem& it, int j, int64_t f, int i, int sp, int SP, double* sy_t) {
  double acc[R];
  kprod64<R>(it, it.V + (int64_t)j * it.len, f, i, sp, SP, acc);
#pragma unroll
  for (int r = 0; r < R; ++r) sy_t[r] = acc[r];
}
// part 0 of a row adds the SP parts in order and scales by vscale_j (FP64 systems)
template <int R>
__device__ __forceinline__ void kbj_sum(const BatchItem& it, int j, int SP, int b, double* sy_t) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double v = sy_t[r];
    for (int q = 1; q < SP; ++q) v += sy_t[q * b * kMaxR + r];
    sy_t[r] = v * it.vscale[(int64_t)j * R + r];
  }
}
template <int R>
__device__ __forceinline__ void kbj_bj(const BatchItem& it, int j, int64_t f, int i, const double* sy_face) {
  double acc[R];
  bj_row<R>(it, sy_face, kMaxR, f, i, acc);
  double* out = it.V + (int64_t)(j + 1) * it.len + (f * it.b + i) * R;
#pragma unroll
  for (int r = 0; r < R; ++r) out[r] = acc[r];
}

// V_{j+1} = P^{-1} (vscale_j K V_j) for every running system: one CTA per
// group of whole faces, the K rows of the group go through shared memory into
// the block-Jacobi apply.  FP64 systems: thread (face lf, part sp, row i) sums
// the slots sp, sp + SP, ... in FP64.  FP32 systems: thread (face lf, part sp,
// row group rg) does the same for 4 rows with 16-byte loads, reading the FP32
// copy of V_j and summing in FP32; the product is rounded to FP32 before the
// FP32 block-Jacobi apply.
template <int RMAX>
__device__ void kbj_phase(const BatchDesc& B, int j, double* sy) {
  const int t = threadIdx.x;
  float* sp32 = reinterpret_cast<float*>(sy);
  for (int64_t g = blockIdx.x; g < B.groups_total; g += gridDim.x) {
    const int p = find_item(B.group_pre, B.n, g);
    const BatchItem& it = B.items[p];
    if (!any_of(it.running, it.R)) continue;          // uniform over the CTA
    const int b = it.b, SP = it.sp, fpc = it.fpc;
    if (it.kprec == HDG_FP64) {
      const int lf = t / (b * SP), rem = t - lf * b * SP;
      const int sp = rem / b, i = rem - sp * b;
      const int64_t f = (g - B.group_pre[p]) * fpc + lf;
      const bool act = lf < fpc && f < it.nfree;
      // sy layout: face lf, part sp, row i at ((lf SP + sp) b + i) kMaxR
      double* sy_t = sy + (int64_t)((lf * SP + sp) * b + i) * kMaxR;
      if (act) HDG_BY_R(kbj_k, it, j, f, i, sp, SP, sy_t)
      __syncthreads();
      if (act && sp == 0) HDG_BY_R(kbj_sum, it, j, SP, b, sy_t)
      __syncthreads();
      if (act && sp == 0) HDG_BY_R(kbj_bj, it, j, f, i, sy + (int64_t)(lf * SP * b) * kMaxR)
      __syncthreads();
    } else {
      const int tpr = it.ld32 / 4;
      const int lf = t / (tpr * SP), rem = t - lf * tpr * SP;
      const int sp = rem / tpr, rg = rem - sp * tpr;
      const int64_t f = (g - B.group_pre[p]) * fpc + lf;
      const bool act = lf < fpc && f < it.nfree;
      if (act) HDG_BY_R(kbj32_k, it, f, lf, sp, rg, sp32)
      __syncthreads();
      if (act && sp == 0) HDG_BY_R(kbj32_sum, it, j, lf, rg, sp32)
      __syncthreads();
      if (act && sp == 0) HDG_BY_R(kbj32_bj, it, j, f, lf, rg, sp32)
      __syncthreads();
    }
  }
}

// Chunk partial sums, one CTA per (chunk, group of 8 slots); thread t holds
// entries e0 + t + 256 k (k < 8), whose RHS is t % R = lane % R:
//   kind 0: ||src||^2 into slot `slot` (src: 0 b, 1 t1, 2 res, 3 V_0)
//   kind 1: V_i . V_{j+1} into slots i = 0..j
__device__ void dot_phase(const BatchDesc& B, int kind, int which, int slot, int j, double* sred) {
  const int t = threadIdx.x;
  const int nslots = kind == 0 ? 1 : j + 1;
  const int ngs = (nslots + kSlotGroup - 1) / kSlotGroup;
  const int64_t ntasks = B.chunks_total * ngs;
  for (int64_t task = blockIdx.x; task < ntasks; task += gridDim.x) {
    const int64_t gc = task / ngs;
    const int sg = (int)(task - gc * ngs);
    const int p = find_item(B.chunk_pre, B.n, gc);
    const BatchItem& it = B.items[p];
    const int R = it.R;
    if (kind == 1 ? !any_of(it.running, R) : it.done_all[0] != 0) continue;   // uniform
    const int64_t c = gc - B.chunk_pre[p];
    const int64_t e0 = c * kChunk + t;
    const double* w = kind == 0 ? (which == 0 ? it.rhs : which == 1 ? it.t1 : which == 2 ? it.res : it.V)
                                : it.V + (int64_t)(j + 1) * it.len;
    double wv[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int64_t e = e0 + (int64_t)k * kBThreads;
      wv[k] = e < it.len ? w[e] : 0.0;
    }
    const int q1 = min(kSlotGroup, nslots - sg * kSlotGroup);
    if (kind == 0) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) acc = fma(wv[k], wv[k], acc);
      cta_stage(acc, 0, R, sred);
    } else {
      // four slots per pass: 32 independent loads in flight per thread
      for (int q = 0; q < q1; q += 4) {
        const double* vq = it.V + (int64_t)(sg * kSlotGroup + q) * it.len;
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        double xq[4][kPerThread];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < kPerThread; ++k) {
            const int64_t e = e0 + (int64_t)k * kBThreads;
            xq[u][k] = (q + u < q1 && e < it.len) ? vq[(int64_t)u * it.len + e] : 0.0;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < kPerThread; ++k) a[u] = fma(xq[u][k], wv[k], a[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (q + u < q1) cta_stage(a[u], q + u, R, sred);
      }
    }
    __syncthreads();
    cta_finish(it, q1, kind == 0 ? slot : sg * kSlotGroup, c, sred);
    __syncthreads();
  }
}

// w -= sum_{i <= j} h_i vscale_i V_i (w = V_{j+1}), its FP32 copy for FP32
// systems, and ||w||^2 partials into slot m + 1.  One CTA per chunk; each CTA
// first sums h_i = V_i . w over the chunks (warps over (i, r)), the CTA of
// chunk 0 stores them for the Givens step.
__device__ void update_phase(const BatchDesc& B, int j, double* sred, double* sh) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int m = B.m;
  for (int64_t gc = blockIdx.x; gc < B.chunks_total; gc += gridDim.x) {
    const int p = find_item(B.chunk_pre, B.n, gc);
    const BatchItem& it = B.items[p];
    const int R = it.R;
    if (!any_of(it.running, R)) continue;             // uniform
    const int64_t c = gc - B.chunk_pre[p];
    for (int q = warp; q < (j + 1) * R; q += kBWarps) {
      const int i = q / R, r = q - i * R;
      const double h = warp_chunk_sum(it, i, r, lane);
      if (lane == 0) {
        sh[q] = h;
        if (c == 0) it.htmp[r * (m + 2) + i] = it.vscale[(int64_t)i * R + r] * h;
      }
    }
    __syncthreads();
    const int r = lane % R;
    const bool run = it.running[r] != 0;
    const int64_t e0 = c * kChunk + t;
    double* w = it.V + (int64_t)(j + 1) * it.len;
    double v[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int64_t e = e0 + (int64_t)k * kBThreads;
      v[k] = e < it.len ? w[e] : 0.0;
    }
    if (run) {
#pragma unroll 4
      for (int i = 0; i <= j; ++i) {
        const double vs = it.vscale[(int64_t)i * R + r];
        const double coef = -(vs * sh[i * R + r]) * vs;
        const double* vi = it.V + (int64_t)i * it.len;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
          const int64_t e = e0 + (int64_t)k * kBThreads;
          if (e < it.len) v[k] = fma(coef, vi[e], v[k]);
        }
      }
    }
    double nrm = 0.0;
    const bool f32 = it.kprec != HDG_FP64;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int64_t e = e0 + (int64_t)k * kBThreads;
      if (e < it.len) {
        w[e] = v[k];
        if (f32) it.x32[e] = (float)v[k];
        nrm = fma(v[k], v[k], nrm);
      }
    }
    cta_stage(nrm, 0, R, sred);
    __syncthreads();
    cta_finish(it, 1, m + 1, c, sred);
    __syncthreads();
  }
}

// x += sum_i ycoef_i V_i for the systems still iterating in this cycle
__device__ void xupdate_phase(const BatchDesc& B) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int m = B.m;
  for (int64_t ge = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ge < B.elems_total; ge += nthreads) {
    const int p = find_item(B.elem_pre, B.n, ge);
    const BatchItem& it = B.items[p];
    if (it.done_all[0]) continue;
    const int64_t e = ge - B.elem_pre[p];
    const int r = (int)(e % it.R);
    const int n = it.jend[r];
    double v = it.x[e];
#pragma unroll 4
    for (int i = 0; i < n; ++i) v = fma(it.ycoef[r * (m + 1) + i], it.V[(int64_t)i * it.len + e], v);
    it.x[e] = v;
  }
}

template <int RMAX>
__global__ void __launch_bounds__(kBThreads, RMAX <= 2 ? 3 : 2) batch_gmres_kernel(BatchDesc Bg) {
  // The item descriptors and the four prefix-sum lists are read-only for the
  // whole solve: every CTA keeps a copy in shared memory, so that finding a
  // work unit's system and reading its sizes and pointers costs no global
  // round trip.  (The per-system solver state stays in global memory.)
  extern __shared__ __align__(16) unsigned char dsm[];
  BatchItem* s_items = reinterpret_cast<BatchItem*>(dsm);
  int64_t* s_pre = reinterpret_cast<int64_t*>(dsm + (size_t)Bg.n * sizeof(BatchItem));
  {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(Bg.items);
    uint64_t* dst = reinterpret_cast<uint64_t*>(s_items);
    const int nw = (int)(Bg.n * sizeof(BatchItem) / 8);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
    for (int k = threadIdx.x; k < Bg.n; k += blockDim.x) {
      s_pre[k] = Bg.row_pre[k];
      s_pre[Bg.n + k] = Bg.elem_pre[k];
      s_pre[2 * Bg.n + k] = Bg.chunk_pre[k];
      s_pre[3 * Bg.n + k] = Bg.group_pre[k];
    }
    __syncthreads();
  }
  BatchDesc B = Bg;
  B.items = s_items;
  B.row_pre = s_pre;
  B.elem_pre = s_pre + Bg.n;
  B.chunk_pre = s_pre + 2 * Bg.n;
  B.group_pre = s_pre + 3 * Bg.n;
  // one buffer, viewed per phase: K rows of a face group (kbj), reduction
  // stages (dots, update), h_i of the update's system, and per warp the
  // Hessenberg column and rotations of the Givens step
  __shared__ double sbuf[kBThreads * kMaxR + (kMaxBasis + 1) * kMaxR];
  double* sy = sbuf;                                    // kBThreads * kMaxR
  double* sred = sbuf;                                  // kBWarps * kSlotGroup * kMaxR <= kBThreads * kMaxR
  double* sh = sbuf + kBThreads * kMaxR;                // (kMaxBasis + 1) * kMaxR
  constexpr int kGivW = (kBThreads * kMaxR + (kMaxBasis + 1) * kMaxR) / kBWarps;   // >= 3 m + 2
  static_assert(kGivW >= 3 * (kMaxBasis - 1) + 2, "Givens staging");
  double* sg = sbuf + (threadIdx.x >> 5) * kGivW;       // this warp's Givens area
  const int m = B.m;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = tid >> 5, nwarps = nthreads >> 5;
  GridBar* gb = reinterpret_cast<GridBar*>(B.bar);
#define HDG_SYNC                                 \
  do {                                           \
    if (!grid_barrier(gb, B.err)) return;        \
  } while (0)
  // ---------------------------------------------------------------- start
  // x = 0, res = b; P^{-1} b into t1 (its norm scales the cycle tolerance)
  for (int64_t ge = tid; ge < B.elems_total; ge += nthreads) {
    const int p = find_item(B.elem_pre, B.n, ge);
    const BatchItem& it = B.items[p];
    const int64_t e = ge - B.elem_pre[p];
    it.x[e] = 0.0;
    it.res[e] = it.rhs[e];
  }
  for (int q = (int)tid; q < B.n; q += (int)nthreads) {
    const BatchItem& it = B.items[q];
    it.done_all[0] = 0;
    for (int r = 0; r < it.R; ++r) {
      it.done[r] = 0;
      it.iters[r] = 0;
      it.cfac[r] = 1.0;
      it.on_est[r] = 0;
      it.running[r] = 0;
    }
  }
  HDG_SYNC;
  rows_phase<RMAX>(B, 2, false);                          // t1 = P^{-1} b
  HDG_SYNC;
  dot_phase(B, 0, 0, 0, 0, sred);                   // ||b||^2   -> slot 0
  dot_phase(B, 0, 1, 1, 0, sred);                   // ||t1||^2  -> slot 1
  HDG_SYNC;
  for (int64_t q = gwarp; q < (int64_t)B.n * kMaxR; q += nwarps) {
    const BatchItem& it = B.items[q / kMaxR];
    const int r = (int)(q % kMaxR);
    if (r >= it.R) continue;
    const double b2 = warp_chunk_sum(it, 0, r, lane), z2 = warp_chunk_sum(it, 1, r, lane);
    if (lane == 0) {
      it.bnorm[r] = sqrt(b2);
      it.zb[r] = sqrt(z2);
    }
  }
  HDG_SYNC;
  for (int cycle = 0;; ++cycle) {
    // --------------------------------------------- true residual check
    dot_phase(B, 0, 2, 0, 0, sred);                 // ||res||^2 -> slot 0
    HDG_SYNC;
    for (int64_t q = gwarp; q < (int64_t)B.n * kMaxR; q += nwarps) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R || it.done_all[0]) continue;
      const double r2 = warp_chunk_sum(it, 0, r, lane);
      if (lane != 0) continue;
      const double rel = it.bnorm[r] > 0.0 ? sqrt(r2) / it.bnorm[r] : 0.0;
      if (!isfinite(rel)) atomicOr(B.err, ERRBIT_NAN);
      it.rel[r] = rel;
      if (cycle > 0 && it.on_est[r] && rel > B.rtol) it.cfac[r] *= 0.1;
      it.done[r] = rel <= B.rtol ? 1 : 0;
    }
    HDG_SYNC;
    // a system stops when every RHS is done, or at the iteration cap
    bool any_left = false;
    for (int q = 0; q < B.n; ++q) {
      const BatchItem& it = B.items[q];
      bool all = true;
      int mx = 0;
      for (int r = 0; r < it.R; ++r) {
        all = all && it.done[r];
        mx = max(mx, it.iters[r]);
      }
      const bool stop = all || mx >= B.maxit || !isfinite(it.rel[0]);
      if (tid == 0 && stop) it.done_all[0] = 1;
      if (!stop) any_left = true;
    }
    HDG_SYNC;
    if (!any_left) break;
    // --------------------------------------------- cycle start: V_0 = P^{-1} res
    rows_phase<RMAX>(B, 2, true);                         // V_0 (and its FP32 copy)
    HDG_SYNC;
    dot_phase(B, 0, 3, 1, 0, sred);                 // ||V_0||^2 -> slot 1
    HDG_SYNC;
    for (int64_t q = gwarp; q < (int64_t)B.n * kMaxR; q += nwarps) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R) continue;
      if (it.done_all[0]) {
        if (lane == 0) it.running[r] = 0;
        continue;
      }
      const double nv = sqrt(warp_chunk_sum(it, 1, r, lane));
      if (lane != 0) continue;
      const bool go = !it.done[r] && nv > 0.0 && it.iters[r] < B.maxit;
      it.running[r] = go ? 1 : 0;
      it.jend[r] = 0;
      it.on_est[r] = 0;
      it.vscale[r] = nv > 0.0 ? 1.0 / nv : 0.0;
      double* g = it.g + r * (m + 1);
      for (int i = 0; i <= m; ++i) g[i] = 0.0;
      g[0] = nv;
      it.tolabs[r] = it.cfac[r] * B.rtol * it.zb[r];
    }
    HDG_SYNC;
    // --------------------------------------------- Arnoldi steps
    for (int j = 0; j < m; ++j) {
      bool anyrun = false;
      for (int q = 0; q < B.n && !anyrun; ++q) anyrun = any_of(B.items[q].running, B.items[q].R);
      if (!anyrun) break;
      kbj_phase<RMAX>(B, j, sy);                          // V_{j+1} = P^{-1} vscale_j K V_j
      HDG_SYNC;
      dot_phase(B, 1, 0, 0, j, sred);               // V_i . V_{j+1}
      HDG_SYNC;
      update_phase(B, j, sred, sh);                 // Gram-Schmidt update, ||V_{j+1}||^2
      HDG_SYNC;
      // Givens rotation of the new column, least-squares residual, stop test:
      // the warp stages the column and the earlier rotations in shared memory,
      // lane 0 runs the rotations, the lanes write the column back
      for (int64_t q = gwarp; q < (int64_t)B.n * kMaxR; q += nwarps) {
        const BatchItem& it = B.items[q / kMaxR];
        const int r = (int)(q % kMaxR);
        if (r >= it.R || !it.running[r]) continue;
        const double hn = sqrt(warp_chunk_sum(it, m + 1, r, lane));
        double* h = sg;                 // j + 2
        double* cs = sg + (m + 2);      // j
        double* sn = cs + m;            // j
        for (int i = lane; i <= j; i += 32) h[i] = it.htmp[r * (m + 2) + i];
        for (int i = lane; i < j; i += 32) {
          cs[i] = it.cs[r * m + i];
          sn[i] = it.sn[r * m + i];
        }
        __syncwarp();
        if (lane == 0) {
          h[j + 1] = hn;
          for (int i = 0; i < j; ++i) {
            const double t = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
            h[i] = t;
          }
          double c = 1.0, sv = 0.0;
          if (h[j + 1] != 0.0) {
            const double rr = hypot(h[j], h[j + 1]);
            c = h[j] / rr;
            sv = h[j + 1] / rr;
          }
          it.cs[r * m + j] = c;
          it.sn[r * m + j] = sv;
          h[j] = c * h[j] + sv * h[j + 1];
          h[j + 1] = 0.0;
          double* g = it.g + r * (m + 1);
          const double gj = g[j];
          g[j + 1] = -sv * gj;
          g[j] = c * gj;
          it.vscale[(int64_t)(j + 1) * it.R + r] = hn > 0.0 ? 1.0 / hn : 0.0;
          it.iters[r] += 1;
          const bool bad = !isfinite(hn) || !isfinite(g[j + 1]);
          const bool est = fabs(g[j + 1]) <= it.tolabs[r];
          if (bad) atomicOr(B.err, ERRBIT_NAN);
          if (bad || est || hn == 0.0 || j + 1 >= m || h[j] == 0.0 || it.iters[r] >= B.maxit) {
            it.jend[r] = j + 1;
            it.running[r] = 0;
            it.on_est[r] = est ? 1 : 0;
          }
        }
        __syncwarp();
        double* H = it.H + (int64_t)r * (m + 1) * m;
        for (int i = lane; i <= j; i += 32) H[i * m + j] = h[i];
        __syncwarp();
      }
      HDG_SYNC;
    }
    // --------------------------------------------- cycle end: x update, true residual
    // back substitution H y = g, one warp per (system, RHS): y_i = (g_i -
    // sum_{k > i} H_ik y_k) / H_ii with the sum over the lanes (fixed order)
    for (int64_t q = gwarp; q < (int64_t)B.n * kMaxR; q += nwarps) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R || it.done_all[0]) continue;
      const int n = it.jend[r];
      const double* H = it.H + (int64_t)r * (m + 1) * m;
      const double* g = it.g + r * (m + 1);
      double* y = it.ycoef + r * (m + 1);
      double* ys = sg;                                // the warp's copy of y
      for (int i = lane; i <= m; i += 32) ys[i] = 0.0;
      __syncwarp();
      for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s = fma(-H[i * m + k], ys[k], s);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
          const double d = H[i * m + i];
          ys[i] = d != 0.0 ? (g[i] + s) / d : 0.0;
        }
        __syncwarp();
      }
      for (int i = lane; i <= m; i += 32) y[i] = i < n ? ys[i] * it.vscale[(int64_t)i * it.R + r] : 0.0;
      __syncwarp();
    }
    HDG_SYNC;
    xupdate_phase(B);
    HDG_SYNC;
    rows_phase<RMAX>(B, 1, false);                        // res = b - K x (FP64 blocks)
    HDG_SYNC;
  }
#undef HDG_SYNC
}

}  // namespace

int64_t batch_chunks(int64_t len) { return (len + kChunk - 1) / kChunk; }
int batch_max_b() { return kBThreads; }
int64_t batch_layout(int64_t nfree, int b, int ld32, int R, bool f32, int* sp, int* fpc) {
  const KbjLayout l = kbj_layout(nfree, b, ld32, R, f32);
  *sp = l.sp;
  *fpc = l.fpc;
  return (nfree + l.fpc - 1) / l.fpc;
}

template <int RMAX>
bool launch_batch(const BatchDesc& B, cudaStream_t s) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t dsm = (size_t)B.n * sizeof(BatchItem) + 4 * sizeof(int64_t) * (size_t)B.n;
  if (cudaFuncSetAttribute(batch_gmres_kernel<RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) !=
      cudaSuccess)
    return false;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_gmres_kernel<RMAX>, kBThreads, dsm);
  if (per_sm < 1 || nsm < 1) return false;
  per_sm = std::min(per_sm, 4);
  const int64_t want = std::max((B.rows_total + kBThreads - 1) / kBThreads, B.groups_total);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * per_sm));
  BatchDesc d = B;
  void* args[] = {&d};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)batch_gmres_kernel<RMAX>, dim3(grid), dim3(kBThreads), args, dsm, s) ==
         cudaSuccess;
}

bool batch_gmres(const BatchDesc& B, int rmax, cudaStream_t s) {
  return rmax <= 2 ? launch_batch<2>(B, s) : launch_batch<8>(B, s);
}

}  // namespace hdg
