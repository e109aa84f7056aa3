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
constexpr int kChunk = 4096;          // entries per reduction chunk

struct GridBar {
  unsigned count, gen;
  int abort;
};

__device__ bool grid_barrier(GridBar* gb, unsigned* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
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
    s_ok = ok && !*(volatile int*)&gb->abort;
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

// y_f = K_f x (FP64 or FP32 blocks) or z_f = P_f^{-1} y_f for every row of
// every active system; one thread per trace row, R sums in a fixed order.
//   mode 0: out = scale[r] * K x      (x: FP64 or its FP32 copy)
//   mode 1: out = rhs - K x           (FP64 blocks, FP64 x)
//   mode 2: out = P^{-1} y            (block-Jacobi, or the identity)
// out32 (optional) receives an FP32 copy.
__device__ void rows_phase(const BatchDesc& B, int mode, int which_in, int which_out, int j, bool fp64_blocks,
                           bool only_running) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < B.rows_total; gi += nthreads) {
    const int p = find_item(B.row_pre, B.n, gi);
    const BatchItem& it = B.items[p];
    if (only_running ? !any_of(it.running, it.R) : any_of(it.done_all, 1)) continue;
    const int64_t lr = gi - B.row_pre[p];
    const int b = it.b, R = it.R;
    const int64_t f = lr / b;
    const int i = (int)(lr - f * b);
    const bool f64 = fp64_blocks || it.kprec == HDG_FP64;
    // inputs
    const int64_t len = it.len;
    const double* in64 = which_in == 0 ? it.V + (int64_t)j * len : which_in == 1 ? it.x
                       : which_in == 2 ? it.res : which_in == 3 ? it.t1 : it.rhs;
    const float* in32 = which_in == 3 ? it.t32 : it.x32;
    double acc[kMaxR];
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (mode == 2) {
      if (it.pc == HDG_PC_NONE) {
        for (int r = 0; r < R; ++r) acc[r] = f64 ? in64[(f * b + i) * R + r] : (double)in32[(f * b + i) * R + r];
      } else if (f64) {
        const double* blk = it.bj64 + f * it.bs64 + i;
        for (int c = 0; c < b; ++c) {
          const double kv = blk[(int64_t)c * b];
          for (int r = 0; r < R; ++r) acc[r] = fma(kv, in64[(f * b + c) * R + r], acc[r]);
        }
      } else {
        float a32[kMaxR];
        for (int r = 0; r < R; ++r) a32[r] = 0.f;
        const float* blk = it.bj32 + f * it.bs32 + i;
        for (int c = 0; c < b; ++c) {
          const float kv = blk[(int64_t)c * it.ld32];
          for (int r = 0; r < R; ++r) a32[r] = fmaf(kv, in32[(f * b + c) * R + r], a32[r]);
        }
        for (int r = 0; r < R; ++r) acc[r] = a32[r];
      }
    } else {
      const int n = it.cnt[f];
      const int64_t rp = it.rowptr[f];
      const int32_t* nbr = it.nbr + f * it.ms;
      if (f64) {
        for (int s = 0; s < n; ++s) {
          const double* blk = it.K64 + (rp + s) * it.s64 + i;
          const double* xv = in64 + (int64_t)nbr[s] * b * R;
          for (int c = 0; c < b; ++c) {
            const double kv = blk[(int64_t)c * b];
            for (int r = 0; r < R; ++r) acc[r] = fma(kv, xv[c * R + r], acc[r]);
          }
        }
      } else {
        float a32[kMaxR];
        for (int r = 0; r < R; ++r) a32[r] = 0.f;
        for (int s = 0; s < n; ++s) {
          const float* blk = it.K32 + (rp + s) * it.s32 + i;
          const float* xv = in32 + (int64_t)nbr[s] * b * R;
          for (int c = 0; c < b; ++c) {
            const float kv = blk[(int64_t)c * it.ld32];
            for (int r = 0; r < R; ++r) a32[r] = fmaf(kv, xv[c * R + r], a32[r]);
          }
        }
        for (int r = 0; r < R; ++r) acc[r] = a32[r];
      }
    }
    double* out = which_out == 0 ? it.V + (int64_t)(j + 1) * len : which_out == 1 ? it.t1
                : which_out == 2 ? it.res : it.V;
    float* out32 = which_out == 1 ? it.t32 : nullptr;
    for (int r = 0; r < R; ++r) {
      double v = acc[r];
      if (mode == 0) v *= it.vscale[(int64_t)j * R + r];
      else if (mode == 1) v = it.rhs[(f * b + i) * R + r] - v;
      out[(f * b + i) * R + r] = v;
      if (out32) out32[(f * b + i) * R + r] = (float)v;
    }
  }
}

// FP32 copy of V_j (running systems with FP32 blocks) or of res
__device__ void convert_phase(const BatchDesc& B, int which, int j) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ge = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ge < B.elems_total; ge += nthreads) {
    const int p = find_item(B.elem_pre, B.n, ge);
    const BatchItem& it = B.items[p];
    if (it.kprec == HDG_FP64) continue;
    if (which == 0 ? !any_of(it.running, it.R) : any_of(it.done_all, 1)) continue;
    const int64_t e = ge - B.elem_pre[p];
    const double v = which == 0 ? it.V[(int64_t)j * it.len + e] : it.res[e];
    it.x32[e] = (float)v;
  }
}

// Chunk partial sums, one warp per chunk, lanes over the chunk's entries in a
// fixed order (the RHS of an entry is lane % R, R dividing 32):
//   kind 0: ||src||^2 into slot `slot`
//   kind 1: V_i . V_{j+1} into slots i = 0..j
__device__ void chunk_phase(const BatchDesc& B, int kind, int which, int slot, int j) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t gc = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); gc < B.chunks_total;
       gc += nwarps) {
    const int p = find_item(B.chunk_pre, B.n, gc);
    const BatchItem& it = B.items[p];
    const int R = it.R;
    if (kind == 1 ? !any_of(it.running, R) : any_of(it.done_all, 1)) continue;
    const int64_t c = gc - B.chunk_pre[p];
    const int64_t e0 = c * kChunk, e1 = min(e0 + kChunk, it.len);
    const int nslots = kind == 0 ? 1 : j + 1;
    const double* w = kind == 0 ? (which == 0 ? it.rhs : which == 1 ? it.t1 : which == 2 ? it.res
                                             : it.V)
                                : it.V + (int64_t)(j + 1) * it.len;
    for (int s0 = 0; s0 < nslots; s0 += 8) {
      double acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0;
      for (int64_t e = e0 + lane; e < e1; e += 32) {
        const double we = w[e];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (s0 + q >= nslots) break;
          const double ve = kind == 0 ? we : it.V[(int64_t)(s0 + q) * it.len + e];
          acc[q] = fma(ve, we, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        double v = acc[q];
        for (int o = R; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane < R && s0 + q < nslots)
          it.part[((int64_t)(kind == 0 ? slot : s0 + q) * it.nchunks + c) * R + lane] = v;
      }
    }
  }
}

__device__ __forceinline__ double chunk_sum(const BatchItem& it, int slot, int r) {
  double s = 0.0;
  for (int c = 0; c < it.nchunks; ++c) s += it.part[((int64_t)slot * it.nchunks + c) * it.R + r];
  return s;
}

// w -= sum_{i <= j} h_i vscale_i V_i (w = V_{j+1}), then ||w||^2 partials into slot m + 1
__device__ void update_phase(const BatchDesc& B, int j) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int m = B.m;
  for (int64_t gc = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); gc < B.chunks_total;
       gc += nwarps) {
    const int p = find_item(B.chunk_pre, B.n, gc);
    const BatchItem& it = B.items[p];
    const int R = it.R;
    if (!any_of(it.running, R)) continue;
    const int64_t c = gc - B.chunk_pre[p];
    const int64_t e0 = c * kChunk, e1 = min(e0 + kChunk, it.len);
    double* w = it.V + (int64_t)(j + 1) * it.len;
    const int r = lane % R;
    const bool run = it.running[r] != 0;
    double nrm = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      double v = w[e];
      if (run)
        for (int i = 0; i <= j; ++i)
          v = fma(-it.htmp[r * (m + 2) + i] * it.vscale[(int64_t)i * R + r], it.V[(int64_t)i * it.len + e], v);
      w[e] = v;
      nrm = fma(v, v, nrm);
    }
    for (int o = R; o < 32; o <<= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane < R) it.part[((int64_t)(m + 1) * it.nchunks + c) * R + lane] = nrm;
  }
}

// x += sum_i ycoef_i V_i for the systems still iterating in this cycle
__device__ void xupdate_phase(const BatchDesc& B) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int m = B.m;
  for (int64_t ge = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ge < B.elems_total; ge += nthreads) {
    const int p = find_item(B.elem_pre, B.n, ge);
    const BatchItem& it = B.items[p];
    if (any_of(it.done_all, 1)) continue;
    const int64_t e = ge - B.elem_pre[p];
    const int r = (int)(e % it.R);
    const int n = it.jend[r];
    double v = it.x[e];
    for (int i = 0; i < n; ++i) v = fma(it.ycoef[r * (m + 1) + i], it.V[(int64_t)i * it.len + e], v);
    it.x[e] = v;
  }
}

__global__ void __launch_bounds__(kBThreads) batch_gmres_kernel(BatchDesc B) {
  const int m = B.m;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
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
    if (it.kprec != HDG_FP64) it.x32[e] = (float)it.rhs[e];
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
  rows_phase(B, 2, 4, 1, 0, false, false);          // t1 = P^{-1} b
  HDG_SYNC;
  chunk_phase(B, 0, 0, 0, 0);                       // ||b||^2   -> slot 0
  chunk_phase(B, 0, 1, 1, 0);                       // ||t1||^2  -> slot 1
  HDG_SYNC;
  for (int64_t q = tid; q < (int64_t)B.n * kMaxR; q += nthreads) {
    const BatchItem& it = B.items[q / kMaxR];
    const int r = (int)(q % kMaxR);
    if (r >= it.R) continue;
    it.bnorm[r] = sqrt(chunk_sum(it, 0, r));
    it.zb[r] = sqrt(chunk_sum(it, 1, r));
  }
  HDG_SYNC;
  for (int cycle = 0;; ++cycle) {
    // --------------------------------------------- true residual check
    chunk_phase(B, 0, 2, 0, 0);                     // ||res||^2 -> slot 0
    HDG_SYNC;
    for (int64_t q = tid; q < (int64_t)B.n * kMaxR; q += nthreads) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R || it.done_all[0]) continue;
      const double rel = it.bnorm[r] > 0.0 ? sqrt(chunk_sum(it, 0, r)) / it.bnorm[r] : 0.0;
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
    convert_phase(B, 1, 0);
    HDG_SYNC;
    rows_phase(B, 2, 2, 3, 0, false, false);        // V_0 = P^{-1} res
    HDG_SYNC;
    chunk_phase(B, 0, 3, 1, 0);                     // ||V_0||^2 -> slot 1
    HDG_SYNC;
    for (int64_t q = tid; q < (int64_t)B.n * kMaxR; q += nthreads) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R) continue;
      if (it.done_all[0]) {
        it.running[r] = 0;
        continue;
      }
      const double nv = sqrt(chunk_sum(it, 1, r));
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
      convert_phase(B, 0, j);                       // FP32 copy of V_j
      HDG_SYNC;
      rows_phase(B, 0, 0, 1, j, false, true);       // t1 = vscale_j K V_j
      HDG_SYNC;
      rows_phase(B, 2, 3, 0, j, false, true);       // V_{j+1} = P^{-1} t1
      HDG_SYNC;
      chunk_phase(B, 1, 0, 0, j);                   // V_i . V_{j+1}
      HDG_SYNC;
      for (int64_t q = tid; q < (int64_t)B.n * kMaxR * (m + 1); q += nthreads) {
        const int pi = (int)(q / (kMaxR * (m + 1)));
        const int rem = (int)(q - (int64_t)pi * kMaxR * (m + 1));
        const int r = rem / (m + 1), i = rem - r * (m + 1);
        const BatchItem& it = B.items[pi];
        if (r >= it.R || i > j || !it.running[r]) continue;
        it.htmp[r * (m + 2) + i] = it.vscale[(int64_t)i * it.R + r] * chunk_sum(it, i, r);
      }
      HDG_SYNC;
      update_phase(B, j);
      HDG_SYNC;
      // Givens rotation of the new column, least-squares residual, stop test
      for (int64_t q = tid; q < (int64_t)B.n * kMaxR; q += nthreads) {
        const BatchItem& it = B.items[q / kMaxR];
        const int r = (int)(q % kMaxR);
        if (r >= it.R || !it.running[r]) continue;
        const double hn = sqrt(chunk_sum(it, m + 1, r));
        double* h = it.hcol + r * (m + 2);
        for (int i = 0; i <= j; ++i) h[i] = it.htmp[r * (m + 2) + i];
        h[j + 1] = hn;
        double* cs = it.cs + r * m;
        double* sn = it.sn + r * m;
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
        cs[j] = c;
        sn[j] = sv;
        h[j] = c * h[j] + sv * h[j + 1];
        h[j + 1] = 0.0;
        double* g = it.g + r * (m + 1);
        g[j + 1] = -sv * g[j];
        g[j] = c * g[j];
        double* H = it.H + (int64_t)r * (m + 1) * m;
        for (int i = 0; i <= j; ++i) H[i * m + j] = h[i];
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
      HDG_SYNC;
    }
    // --------------------------------------------- cycle end: x update, true residual
    for (int64_t q = tid; q < (int64_t)B.n * kMaxR; q += nthreads) {
      const BatchItem& it = B.items[q / kMaxR];
      const int r = (int)(q % kMaxR);
      if (r >= it.R || it.done_all[0]) continue;
      const int n = it.jend[r];
      const double* H = it.H + (int64_t)r * (m + 1) * m;
      const double* g = it.g + r * (m + 1);
      double* y = it.ycoef + r * (m + 1);
      for (int i = 0; i <= m; ++i) y[i] = 0.0;
      for (int i = n - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < n; ++k) s = fma(-H[i * m + k], y[k], s);
        y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
      }
      for (int i = 0; i < n; ++i) y[i] *= it.vscale[(int64_t)i * it.R + r];
    }
    HDG_SYNC;
    xupdate_phase(B);
    HDG_SYNC;
    rows_phase(B, 1, 1, 2, 0, true, false);         // res = b - K x (FP64 blocks)
    HDG_SYNC;
  }
#undef HDG_SYNC
}

}  // namespace

int64_t batch_chunks(int64_t len) { return (len + kChunk - 1) / kChunk; }

bool batch_gmres(const BatchDesc& B, cudaStream_t s) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_gmres_kernel, kBThreads, 0);
  if (per_sm < 1 || nsm < 1) return false;
  per_sm = std::min(per_sm, 4);
  const int64_t want = (B.rows_total + kBThreads - 1) / kBThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * per_sm));
  BatchDesc d = B;
  void* args[] = {&d};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)batch_gmres_kernel, dim3(grid), dim3(kBThreads), args, 0, s) ==
         cudaSuccess;
}

}  // namespace hdg
