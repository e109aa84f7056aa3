// GMRES kernels (Sec. 3.1, Sec. 4.4) for R right-hand sides in lock-step:
// fused multi-dot h = V^T w (one pass over the basis), fused w -= V h with
// the norm of the result, the Givens update of the Hessenberg column and the
// convergence test on the device (the paper does this on the CPU), back
// substitution and the solution update x += V y.  Reductions are
// deterministic: every block writes partial sums and the last block to
// finish adds them in block order.
//
// Vectors are n_dof x R doubles with the RHS index fastest; thread e of a
// grid-stride loop owns RHS r = e mod R, which makes the per-RHS warp
// reductions plain shuffles (R is a power of two <= 32).
//
// Also here: the polynomial-preconditioner recurrence steps (Sec. 4.7) and a
// single-thread Hessenberg eigenvalue solver (Francis double-shift QR,
// Golub & Van Loan Sec. 7.5) with the Leja ordering of the Ritz values.
#include "hdg_common.cuh"
#include "hdg_gmres.h"
#include "k_poly.cuh"

namespace hdg {

namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;   // basis vectors per pass of the multi-dot

__device__ __forceinline__ bool any_running(const int* running, int R) {
  for (int r = 0; r < R; ++r)
    if (running[r]) return true;
  return false;
}

// Sum over lanes with the same (lane mod R); result valid in lanes < R.
__device__ __forceinline__ double rhs_warp_sum(double v, int R) {
  for (int o = 16; o >= R; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block-wide sum of v[i*stride], i < n (every thread of the
// block calls it; the result is returned in all threads).  A fixed tree of
// per-thread strided sums, warp shuffles and one shared-memory level: on this
// GPU a long serial chain of dependent FP64 adds costs tens of microseconds.
__device__ double block_sum(const double* v, int n, int stride) {
  __shared__ double ws[32];
  __shared__ double total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[(int64_t)i * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) total = t;
  }
  __syncthreads();
  return total;
}

// Warp-wide deterministic sum of v[i*stride], i < n; result in all lanes.
__device__ __forceinline__ double warp_strided_sum(const double* v, int n, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += v[(int64_t)i * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__device__ __forceinline__ bool last_block_2d(unsigned* counter) {
  __shared__ bool s_last2;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last2 = (prev == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (s_last2) __threadfence();
  return s_last2;
}

__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// --------------------------------------------------------------- dots
// htmp[r][i] = vscale_i[r] * <V_i, w>_r  for i in [i0, i1).
// Grid: x = element chunks, y = groups of kGroup basis vectors.  Each thread
// covers kDotsPerThread elements so the FP64 tree reduction (which costs as
// much as the products on this GPU) is amortised.
constexpr int kDotsThreads = 128;
constexpr int kDotsPerThread = 32;
// elements per block of the multi-dot: >= 32 per thread and <= 1024 blocks
__host__ __device__ __forceinline__ int64_t dots_chunk(int64_t len) {
  int64_t per = (len + 1023) / 1024;
  per = ((per + kDotsThreads - 1) / kDotsThreads) * kDotsThreads;
  const int64_t lo = (int64_t)kDotsThreads * kDotsPerThread;
  return per < lo ? lo : per;
}
// acc[t] += sum over this thread's elements of V_{ig+t}[e] w[e], t < NG (the
// group's basis vectors; predicated-off FMAs would still take the FP64 pipe)
template <int NG>
__device__ __forceinline__ void dots_body(const GmresView& k, const double* w, int ig, int64_t start, int64_t stop,
                                          int64_t len, double (&acc)[kGroup]) {
  // four elements per step: 4 * (NG + 1) independent loads in flight
  int64_t e = start + threadIdx.x;
  for (; e + 3 * kDotsThreads < stop; e += 4 * kDotsThreads) {
    double we[4], vv[4][NG];
#pragma unroll
    for (int q = 0; q < 4; ++q) we[q] = w[e + q * kDotsThreads];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int t = 0; t < NG; ++t) vv[q][t] = k.V[(int64_t)(ig + t) * len + e + q * kDotsThreads];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int t = 0; t < NG; ++t) acc[t] = fma(vv[q][t], we[q], acc[t]);
  }
  for (; e < stop; e += kDotsThreads) {
    const double we1 = w[e];
#pragma unroll
    for (int t = 0; t < NG; ++t) acc[t] = fma(k.V[(int64_t)(ig + t) * len + e], we1, acc[t]);
  }
}

__global__ void __launch_bounds__(kDotsThreads) dots_kernel(GmresView k, const double* w, int i0, int i1) {
  if (!any_running(k.running, k.R)) return;
  const int R = k.R;
  const int64_t len = k.n * R;
  const int64_t chunk = dots_chunk(len);
  const int64_t start = blockIdx.x * chunk;
  const int64_t stop = min(start + chunk, len);
  __shared__ double red[kDotsThreads / 32][kGroup][32];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ig = i0 + blockIdx.y * kGroup;
  const int ng = min(kGroup, i1 - ig);
  double acc[kGroup];
#pragma unroll
  for (int t = 0; t < kGroup; ++t) acc[t] = 0.0;
  switch (ng) {     // uniform over the CTA
    case 1: dots_body<1>(k, w, ig, start, stop, len, acc); break;
    case 2: dots_body<2>(k, w, ig, start, stop, len, acc); break;
    case 3: dots_body<3>(k, w, ig, start, stop, len, acc); break;
    case 4: dots_body<4>(k, w, ig, start, stop, len, acc); break;
    case 5: dots_body<5>(k, w, ig, start, stop, len, acc); break;
    case 6: dots_body<6>(k, w, ig, start, stop, len, acc); break;
    case 7: dots_body<7>(k, w, ig, start, stop, len, acc); break;
    default: dots_body<8>(k, w, ig, start, stop, len, acc); break;
  }
#pragma unroll
  for (int t = 0; t < kGroup; ++t) {
    double v = rhs_warp_sum(acc[t], R);
    if (lane < R) red[warp][t][lane] = v;
  }
  __syncthreads();
  if (threadIdx.x < ng * R) {
    const int t = threadIdx.x / R, r = threadIdx.x % R;
    double sum = 0.0;
    for (int wv = 0; wv < kDotsThreads / 32; ++wv) sum += red[wv][t][r];
    k.partial[((int64_t)(ig + t) * gridDim.x + blockIdx.x) * R + r] = sum;
  }
  if (last_block_2d(k.counter)) {
    // one warp per (vector, RHS): a fixed-order tree over the x-blocks
    for (int idx = warp; idx < (i1 - i0) * R; idx += kDotsThreads / 32) {
      const int i = i0 + idx / R, r = idx % R;
      const double sum = warp_strided_sum(k.partial + ((int64_t)i * gridDim.x) * R + r, gridDim.x, R);
      if (lane == 0) k.htmp[r * (k.m + 2) + i] = k.vscale[i * R + r] * sum;
    }
    if (threadIdx.x == 0) *k.counter = 0;
  }
}

// --------------------------------------------------------------- update
// w -= sum_{i in [i0,i1)} htmp[r][i] vscale_i[r] V_i ; hcol (+)= htmp.
// finalize: ||w|| -> h_{j+1}, Givens rotation of column j, convergence test.
__global__ void __launch_bounds__(kThreads) update_kernel(GmresView k, double* w, int i0, int i1, int j,
                                                          int hmode, int finalize) {
  if (!any_running(k.running, k.R)) return;
  const int R = k.R;
  const int64_t len = k.n * R;
  __shared__ double coef[kMaxBasis * kMaxR];
  for (int idx = threadIdx.x; idx < (i1 - i0) * R; idx += kThreads) {
    const int i = i0 + idx / R, r = idx % R;
    coef[idx] = k.running[r] ? k.htmp[r * (k.m + 2) + i] * k.vscale[i * R + r] : 0.0;
  }
  __syncthreads();
  const int64_t start = blockIdx.x * k.chunk;
  const int64_t stop = min(start + k.chunk, len);
  double nrm = 0.0;
  for (int64_t e = start + threadIdx.x; e < stop; e += kThreads) {
    const int r = (int)e & (R - 1);   // R is a power of two
    double v = w[e];
    int i = i0;
    // eight independent loads in flight per step
    for (; i + 8 <= i1; i += 8) {
      double vv[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) vv[t] = k.V[(int64_t)(i + t) * len + e];
#pragma unroll
      for (int t = 0; t < 8; ++t) v = fma(-coef[(i + t - i0) * R + r], vv[t], v);
    }
    for (; i < i1; ++i) v = fma(-coef[(i - i0) * R + r], k.V[(int64_t)i * len + e], v);
    w[e] = v;
    nrm = fma(v, v, nrm);
  }
  __shared__ double red[kThreads / 32][32];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (finalize) {
    double v = rhs_warp_sum(nrm, R);
    if (lane < R) red[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < R) {
      double s = 0.0;
      for (int wv = 0; wv < kThreads / 32; ++wv) s += red[wv][threadIdx.x];
      k.partial[(int64_t)blockIdx.x * R + threadIdx.x] = s;
    }
  }
  if (last_block(k.counter)) {
    // h column bookkeeping
    for (int idx = threadIdx.x; idx < (i1 - i0) * R; idx += kThreads) {
      const int i = i0 + idx / R, r = idx % R;
      const double h = k.htmp[r * (k.m + 2) + i];
      double* hc = &k.hcol[r * (k.m + 2) + i];
      *hc = hmode ? *hc + h : h;
    }
    __syncthreads();
    __shared__ double s_nrm[kMaxR];
    if (finalize) {
      for (int r = 0; r < R; ++r) {
        const double t = block_sum(k.partial + r, gridDim.x, R);
        if (threadIdx.x == 0) s_nrm[r] = t;
      }
      __syncthreads();
    }
    if (finalize && threadIdx.x < R) {
      const int r = threadIdx.x;
      const double hn = sqrt(s_nrm[r]);
      if (k.running[r] && finalize == 2) {
        // Arnoldi only (polynomial setup): store the column unrotated; stop on
        // breakdown h_{j+1,j} <= 1e-14 |h_{1,1}| or after m steps
        const int m = k.m;
        double* h = &k.hcol[r * (m + 2)];
        h[j + 1] = hn;
        double* H = &k.H[(int64_t)r * (m + 1) * m];
        for (int i = 0; i <= j + 1; ++i) H[i * m + j] = h[i];
        k.vscale[(j + 1) * R + r] = hn > 0.0 ? 1.0 / hn : 0.0;
        k.iters[r] += 1;
        if (!isfinite(hn)) atomicOr(k.err, ERRBIT_NAN);
        if (!isfinite(hn) || hn <= 1e-14 * fabs(H[0]) || j + 1 >= m) {
          k.jend[r] = j + 1;
          k.running[r] = 0;
        }
      } else if (k.running[r]) {
        const int m = k.m;
        double* h = &k.hcol[r * (m + 2)];
        h[j + 1] = hn;
        double* cs = &k.cs[r * m];
        double* sn = &k.sn[r * m];
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
        double* g = &k.g[r * (m + 1)];
        g[j + 1] = -sv * g[j];
        g[j] = c * g[j];
        double* H = &k.H[(int64_t)r * (m + 1) * m];
        for (int i = 0; i <= j; ++i) H[i * m + j] = h[i];
        k.vscale[(j + 1) * R + r] = hn > 0.0 ? 1.0 / hn : 0.0;
        k.iters[r] += 1;
        const bool bad = !isfinite(hn) || !isfinite(g[j + 1]);
        const bool est = fabs(g[j + 1]) <= k.tolabs[r];
        if (bad) atomicOr(k.err, ERRBIT_NAN);
        const int mx = k.dmaxit ? *k.dmaxit : k.maxit;
        if (bad || est || hn == 0.0 || j + 1 >= m || h[j] == 0.0 || k.iters[r] >= mx) {
          k.jend[r] = j + 1;
          k.running[r] = 0;
          k.on_estimate[r] = est ? 1 : 0;
        }
      }
    }
    if (finalize) {
      __syncthreads();
      if (threadIdx.x == 0) {
        int any = 0;
        for (int r = 0; r < R; ++r) any |= k.running[r];
        if (k.hflag) {
          k.hflag[j] = any;
          __threadfence_system();
        }
        // in a captured cycle the next iteration's IF node runs only while
        // some right-hand side is still iterating
        if (k.use_cond) cudaGraphSetConditional(k.cond, any ? 1u : 0u);
      }
    }
    if (threadIdx.x == 0) *k.counter = 0;
  }
}

// --------------------------------------------------------------- norms
// out[r] = ||v||_r ; with `cycle` set also starts a GMRES cycle for the RHS
// that are not done: vscale_0 = 1/beta, g = (beta, 0, ...), running = 1.
__global__ void __launch_bounds__(kThreads) norms_kernel(GmresView k, const double* v, double* out, int cycle,
                                                         const double* denom) {
  const int R = k.R;
  const int64_t len = k.n * R;
  const int64_t start = blockIdx.x * k.chunk;
  const int64_t stop = min(start + k.chunk, len);
  double nrm = 0.0;
  for (int64_t e = start + threadIdx.x; e < stop; e += kThreads) nrm = fma(v[e], v[e], nrm);
  __shared__ double red[kThreads / 32][32];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double s = rhs_warp_sum(nrm, R);
  if (lane < R) red[warp][lane] = s;
  __syncthreads();
  if (threadIdx.x < R) {
    double t = 0.0;
    for (int wv = 0; wv < kThreads / 32; ++wv) t += red[wv][threadIdx.x];
    k.partial[(int64_t)blockIdx.x * R + threadIdx.x] = t;
  }
  if (last_block(k.counter)) {
    __shared__ double s_sq[kMaxR];
    for (int r = 0; r < R; ++r) {
      const double t = block_sum(k.partial + r, gridDim.x, R);
      if (threadIdx.x == 0) s_sq[r] = t;
    }
    __syncthreads();
    if (threadIdx.x < R) {
      const int r = threadIdx.x;
      double nv = sqrt(s_sq[r]);
      if (!isfinite(nv)) atomicOr(k.err, ERRBIT_NAN);
      if (out) out[r] = denom ? (denom[r] > 0.0 ? nv / denom[r] : 0.0) : nv;
      if (cycle) {
        const int m = k.m;
        const bool go = !k.done[r] && nv > 0.0 && k.iters[r] < k.maxit;
        k.running[r] = go ? 1 : 0;
        k.jend[r] = 0;
        k.on_estimate[r] = 0;
        k.vscale[r] = nv > 0.0 ? 1.0 / nv : 0.0;
        double* g = &k.g[r * (m + 1)];
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = nv;
        k.tolabs[r] = k.cfac[r] * k.rtol * k.zb[r];
      }
    }
    if (threadIdx.x == 0) *k.counter = 0;
  }
}

// y = R^{-1} g for each RHS (R = rotated H, jend steps); ycoef_i = y_i vscale_i.
// One warp per RHS: lane l keeps g_i for i = l, l+32, ...; each step divides
// on the owner lane, broadcasts y_i and updates the earlier entries in
// parallel (a serial FP64 chain of O(m^2) dependent operations is slow here).
__global__ void backsolve_kernel(GmresView k) {
  const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= k.R) return;
  const int m = k.m, n = k.jend[r];
  const double* H = &k.H[(int64_t)r * (m + 1) * m];
  const double* g = &k.g[r * (m + 1)];
  double* y = &k.ycoef[r * (m + 1)];
  double gl[kMaxBasis / 32];
#pragma unroll
  for (int q = 0; q < kMaxBasis / 32; ++q) {
    const int i = lane + 32 * q;
    gl[q] = (i < n) ? g[i] : 0.0;
  }
  for (int i = lane; i <= m; i += 32) y[i] = 0.0;
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    const int owner = i & 31, slot = i >> 5;
    double yi = 0.0;
    if (lane == owner) {
      double gi = 0.0;
#pragma unroll
      for (int q = 0; q < kMaxBasis / 32; ++q)
        if (q == slot) gi = gl[q];
      const double d = H[i * m + i];
      yi = (d != 0.0) ? gi / d : 0.0;
    }
    yi = __shfl_sync(0xffffffffu, yi, owner);
#pragma unroll
    for (int q = 0; q < kMaxBasis / 32; ++q) {
      const int kk = lane + 32 * q;
      if (kk < i) gl[q] = fma(-H[kk * m + i], yi, gl[q]);
    }
    if (lane == 0) y[i] = yi * k.vscale[i * k.R + r];
  }
}

// x += sum_i ycoef[r][i] V_i  (i < jend[r])
__global__ void __launch_bounds__(kThreads) xupdate_kernel(GmresView k, double* x) {
  const int R = k.R;
  const int64_t len = k.n * R;
  __shared__ double coef[kMaxBasis * kMaxR];
  __shared__ int s_n;
  if (threadIdx.x == 0) {
    int mx = 0;
    for (int r = 0; r < R; ++r) mx = max(mx, k.jend[r]);
    s_n = mx;
  }
  for (int idx = threadIdx.x; idx < (k.m + 1) * R; idx += kThreads) {
    const int i = idx / R, r = idx % R;
    coef[idx] = (i < k.jend[r]) ? k.ycoef[r * (k.m + 1) + i] : 0.0;
  }
  __syncthreads();
  const int n = s_n;
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < len; e += (int64_t)gridDim.x * kThreads) {
    const int r = (int)e & (R - 1);
    double v = x[e];
    for (int i = 0; i < n; ++i) v = fma(coef[i * R + r], k.V[(int64_t)i * len + e], v);
    x[e] = v;
  }
}

// --------------------------------------------------------------- elementwise
__global__ void axpby_kernel(double* y, const double* x, double a, double b, int64_t len, const int* running, int R) {
  if (running && !any_running(running, R)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

__global__ void pp_real_kernel(double* w, double* q, const double* Aq, double inv_theta, int64_t len, int update_q,
                               const int* running, int R, int first) {
  if (running && !any_running(running, R)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const double qe = q[e];
    w[e] = (first ? 0.0 : w[e]) + inv_theta * qe;
    if (update_q) q[e] = qe - inv_theta * Aq[e];
  }
}

__global__ void pp_pair_t_kernel(double* t, double* w, const double* q, const double* Aq, double two_a,
                                 double inv_mod2, int64_t len, const int* running, int R, int first) {
  if (running && !any_running(running, R)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const double te = two_a * q[e] - Aq[e];
    t[e] = te;
    w[e] = (first ? 0.0 : w[e]) + inv_mod2 * te;
  }
}

__global__ void pp_pair_q_kernel(double* q, const double* At, double inv_mod2, int64_t len, const int* running, int R) {
  if (running && !any_running(running, R)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    q[e] = q[e] - inv_mod2 * At[e];
}

// A polynomial step whose "M^{-1}" is the identity: v is the input vector.
__global__ void poly_epi_kernel(PolyEpi e, const float* v, int64_t len, const int* running, int R) {
  if (running && !any_running(running, R)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    poly_epi(e, i, v[i]);
}

// Chebyshev step: z += d; then (unless last) r -= Ad computed by the caller
// before; d = c1 d + c2 r.  `phase` 0: z = d (first), 1: z += d,
// 2: r -= Ad; d = c1 d + c2 r.
__global__ void cheb_kernel(double* z, double* d, double* r, const double* Ad, double c1, double c2, int64_t len,
                            int phase, const int* running, int R) {
  if (running && !any_running(running, R)) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    if (phase == 0) z[e] = d[e];
    else if (phase == 1) z[e] += d[e];
    else {
      const double re = r[e] - Ad[e];
      r[e] = re;
      d[e] = c1 * d[e] + c2 * re;
    }
  }
}

// --------------------------------------------------------------- eigenvalues
// Eigenvalues of an upper Hessenberg matrix a (n x n, row-major, leading
// dimension n) by the Francis double-shift QR iteration with deflation
// (Golub & Van Loan, Matrix Computations, Sec. 7.5).  Eigenvalues only: the
// transformations touch the active window.  Returns false if it did not
// converge in 60 iterations per eigenvalue.
__device__ bool hessenberg_eigs(double* a, int n, double* wr, double* wi) {
  auto A = [&](int i, int j) -> double& { return a[i * n + j]; };
  int hi = n - 1;
  int its = 0;
  const double eps = 2.220446049250313e-16;
  while (hi >= 0) {
    // find the lowest lo such that a(lo, lo-1) is negligible
    int lo = hi;
    while (lo > 0) {
      double s = fabs(A(lo - 1, lo - 1)) + fabs(A(lo, lo));
      if (s == 0.0) s = 1.0;
      if (fabs(A(lo, lo - 1)) <= eps * s) {
        A(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {                       // 1x1 block
      wr[hi] = A(hi, hi);
      wi[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {                   // 2x2 block
      const double p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), s = A(hi, hi);
      const double tr = 0.5 * (p + s);
      const double det = p * s - q * r;
      const double disc = tr * tr - det;
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        const double l1 = tr + (tr >= 0.0 ? sq : -sq);
        const double l2 = (l1 != 0.0) ? det / l1 : tr - (tr >= 0.0 ? sq : -sq);
        wr[hi - 1] = l1; wi[hi - 1] = 0.0;
        wr[hi] = l2; wi[hi] = 0.0;
      } else {
        const double im = sqrt(-disc);
        wr[hi - 1] = tr; wi[hi - 1] = im;
        wr[hi] = tr; wi[hi] = -im;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++its > 60) return false;
    // double shift from the trailing 2x2 (exceptional shifts every 10 its)
    double sh, tt;
    if (its % 10 == 0) {
      const double x = fabs(A(hi, hi - 1)) + fabs(A(hi - 1, hi - 2));
      sh = 1.5 * x;
      tt = x * x;
    } else {
      sh = A(hi - 1, hi - 1) + A(hi, hi);
      tt = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    }
    double x = A(lo, lo) * A(lo, lo) + A(lo, lo + 1) * A(lo + 1, lo) - sh * A(lo, lo) + tt;
    double y = A(lo + 1, lo) * (A(lo, lo) + A(lo + 1, lo + 1) - sh);
    double z = (lo + 2 <= hi) ? A(lo + 1, lo) * A(lo + 2, lo + 1) : 0.0;
    for (int kk = lo; kk <= hi - 2; ++kk) {
      // Householder reflector P = I - 2 v v^T / v^T v mapping (x, y, z) to (alpha, 0, 0)
      const double nx = sqrt(x * x + y * y + z * z);
      if (nx != 0.0) {
        const double alpha = (x > 0.0) ? -nx : nx;
        double v0 = x - alpha, v1 = y, v2 = z;
        const double vv = v0 * v0 + v1 * v1 + v2 * v2;
        if (vv != 0.0) {
          const double beta = 2.0 / vv;
          const int c0 = (kk > lo) ? kk - 1 : lo;
          for (int c = c0; c <= hi; ++c) {          // rows kk..kk+2 from the left
            const double s = beta * (v0 * A(kk, c) + v1 * A(kk + 1, c) + v2 * A(kk + 2, c));
            A(kk, c) -= s * v0;
            A(kk + 1, c) -= s * v1;
            A(kk + 2, c) -= s * v2;
          }
          const int r1 = min(kk + 3, hi);
          for (int rr = lo; rr <= r1; ++rr) {       // columns kk..kk+2 from the right
            const double s = beta * (v0 * A(rr, kk) + v1 * A(rr, kk + 1) + v2 * A(rr, kk + 2));
            A(rr, kk) -= s * v0;
            A(rr, kk + 1) -= s * v1;
            A(rr, kk + 2) -= s * v2;
          }
        }
      }
      x = A(kk + 1, kk);
      y = A(kk + 2, kk);
      if (kk < hi - 2) z = A(kk + 3, kk);
    }
    // final Givens rotation on rows/columns hi-1, hi
    {
      const int kk = hi - 1;
      const double nx = hypot(x, y);
      if (nx != 0.0) {
        const double c = x / nx, s = y / nx;
        const int c0 = (kk > lo) ? kk - 1 : lo;
        for (int col = c0; col <= hi; ++col) {
          const double t1 = A(kk, col), t2 = A(kk + 1, col);
          A(kk, col) = c * t1 + s * t2;
          A(kk + 1, col) = -s * t1 + c * t2;
        }
        for (int rr = lo; rr <= hi; ++rr) {
          const double t1 = A(rr, kk), t2 = A(rr, kk + 1);
          A(rr, kk) = c * t1 + s * t2;
          A(rr, kk + 1) = -s * t1 + c * t2;
        }
      }
    }
  }
  return true;
}

// harmonic == 1: theta = eig(H_PP + h_{P+1,P}^2 H_PP^{-T} e_P e_P^T), falling
// back to eig(H_PP) when h_{P+1,P} = 0 or H_PP is numerically singular
// (1-norm condition estimate > 1e12).  harmonic == 0: eig(H_PP).
// Output in Leja order (start at the largest modulus; a value with Im > 0
// is followed by its conjugate; greedy max of sum log|theta - chosen|).
__global__ void ritz_leja_kernel(const double* H, int ldh, int P, int harmonic, double* re, double* im, int* nout,
                                 unsigned* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  extern __shared__ double ritz_smem[];
  double* a = ritz_smem;                       // P x P
  double* inv = ritz_smem + kMaxPoly * kMaxPoly;
  double wr[kMaxPoly], wi[kMaxPoly];
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) a[i * P + j] = H[i * ldh + j];
  const double hn = H[P * ldh + (P - 1)];
  if (harmonic && hn != 0.0) {
    // explicit inverse of H_PP by Gauss-Jordan with partial pivoting
    for (int i = 0; i < P * P; ++i) inv[i] = a[i];
    int piv[kMaxPoly];
    bool ok = true;
    for (int kq = 0; kq < P && ok; ++kq) {
      int p = kq;
      for (int i = kq + 1; i < P; ++i)
        if (fabs(inv[i * P + kq]) > fabs(inv[p * P + kq])) p = i;
      piv[kq] = p;
      if (p != kq)
        for (int j = 0; j < P; ++j) { double t = inv[kq * P + j]; inv[kq * P + j] = inv[p * P + j]; inv[p * P + j] = t; }
      const double pv = inv[kq * P + kq];
      if (pv == 0.0) { ok = false; break; }
      const double ip = 1.0 / pv;
      inv[kq * P + kq] = 1.0;
      for (int j = 0; j < P; ++j) inv[kq * P + j] *= ip;
      for (int i = 0; i < P; ++i) {
        if (i == kq) continue;
        const double f = inv[i * P + kq];
        inv[i * P + kq] = 0.0;
        for (int j = 0; j < P; ++j) inv[i * P + j] -= f * inv[kq * P + j];
      }
    }
    if (ok) {
      for (int kq = P - 1; kq >= 0; --kq)
        if (piv[kq] != kq)
          for (int i = 0; i < P; ++i) { double t = inv[i * P + kq]; inv[i * P + kq] = inv[i * P + piv[kq]]; inv[i * P + piv[kq]] = t; }
      double n1 = 0.0, n1i = 0.0;
      for (int j = 0; j < P; ++j) {
        double c = 0.0, ci = 0.0;
        for (int i = 0; i < P; ++i) { c += fabs(a[i * P + j]); ci += fabs(inv[i * P + j]); }
        n1 = fmax(n1, c);
        n1i = fmax(n1i, ci);
      }
      if (n1 * n1i <= 1e12) {
        // f = H_PP^{-T} e_P  ->  f_i = inv[P-1][i]; add h^2 f e_P^T to the last column
        for (int i = 0; i < P; ++i) a[i * P + (P - 1)] += hn * hn * inv[(P - 1) * P + i];
      }
    }
  }
  if (!hessenberg_eigs(a, P, wr, wi)) {
    atomicOr(err, ERRBIT_ARG);
    *nout = 0;
    return;
  }
  // clean: tiny imaginary parts become real
  double scale = 0.0;
  for (int i = 0; i < P; ++i) scale = fmax(scale, hypot(wr[i], wi[i]));
  for (int i = 0; i < P; ++i)
    if (fabs(wi[i]) <= 1e-12 * scale) wi[i] = 0.0;
  // Leja order
  bool used[kMaxPoly];
  for (int i = 0; i < P; ++i) used[i] = false;
  int cnt = 0;
  auto take = [&](int i) {
    re[cnt] = wr[i]; im[cnt] = wi[i]; used[i] = true; ++cnt;
    if (wi[i] > 0.0) {
      int best = -1;
      double bd = 0.0;
      for (int j = 0; j < P; ++j) {
        if (used[j]) continue;
        const double dd = hypot(wr[j] - wr[i], wi[j] + wi[i]);
        if (best < 0 || dd < bd) { best = j; bd = dd; }
      }
      if (best >= 0) { re[cnt] = wr[best]; im[cnt] = wi[best]; used[best] = true; ++cnt; }
    }
  };
  {
    int best = -1;
    for (int i = 0; i < P; ++i) {
      if (wi[i] < 0.0) continue;
      if (best < 0) { best = i; continue; }
      const double mi = hypot(wr[i], wi[i]), mb = hypot(wr[best], wi[best]);
      if (mi > mb || (mi == mb && wi[i] > wi[best])) best = i;
    }
    take(best);
  }
  while (cnt < P) {
    int best = -1;
    double bv = 0.0;
    for (int i = 0; i < P; ++i) {
      if (used[i] || wi[i] < 0.0) continue;
      double v = 0.0;
      for (int c = 0; c < cnt; ++c) v += log(hypot(wr[i] - re[c], wi[i] - im[c]));
      if (best < 0 || v > bv) { best = i; bv = v; }
    }
    if (best < 0) break;
    take(best);
  }
  *nout = cnt;
}

inline unsigned ew_grid(int64_t len) {
  int64_t g = (len + 255) / 256;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int64_t gmres_chunk(int64_t len) {
  // contiguous element range per block of the update / norm kernels: at
  // least 4 elements per thread (the FP64 reduction is amortised), a multiple
  // of kThreads, at most 1024 blocks
  int64_t per = (len + 1023) / 1024;
  per = ((per + kThreads - 1) / kThreads) * kThreads;
  if (per < 4 * kThreads) per = 4 * kThreads;
  return per;
}
int gmres_blocks(int64_t len, int64_t chunk) { return (int)((len + chunk - 1) / chunk); }

void launch_dots(const GmresView& k, const double* w, int i0, int i1, cudaStream_t s) {
  if (i1 <= i0) return;
  dim3 grid(gmres_blocks(k.n * k.R, dots_chunk(k.n * k.R)), (i1 - i0 + kGroup - 1) / kGroup);
  count_launch(); dots_kernel<<<grid, kDotsThreads, 0, s>>>(k, w, i0, i1);
}
void launch_update(const GmresView& k, double* w, int i0, int i1, int j, int hmode, int finalize, cudaStream_t s) {
  count_launch(); update_kernel<<<gmres_blocks(k.n * k.R, k.chunk), kThreads, 0, s>>>(k, w, i0, i1, j, hmode, finalize);
}
void launch_norms(const GmresView& k, const double* v, double* out, int cycle, const double* denom, cudaStream_t s) {
  count_launch(); norms_kernel<<<gmres_blocks(k.n * k.R, k.chunk), kThreads, 0, s>>>(k, v, out, cycle, denom);
}
void launch_backsolve(const GmresView& k, cudaStream_t s) { count_launch(); backsolve_kernel<<<1, 32 * k.R, 0, s>>>(k); }
void launch_xupdate(const GmresView& k, double* x, cudaStream_t s) {
  count_launch(); xupdate_kernel<<<ew_grid(k.n * k.R), kThreads, 0, s>>>(k, x);
}
void launch_axpby(double* y, const double* x, double a, double b, int64_t len, const int* running, int R,
                  cudaStream_t s) {
  count_launch(); axpby_kernel<<<ew_grid(len), 256, 0, s>>>(y, x, a, b, len, running, R);
}
void launch_pp_real(double* w, double* q, const double* Aq, double inv_theta, int64_t len, int update_q,
                    const int* running, int R, int first, cudaStream_t s) {
  count_launch(); pp_real_kernel<<<ew_grid(len), 256, 0, s>>>(w, q, Aq, inv_theta, len, update_q, running, R, first);
}
void launch_pp_pair_t(double* t, double* w, const double* q, const double* Aq, double two_a, double inv_mod2,
                      int64_t len, const int* running, int R, int first, cudaStream_t s) {
  count_launch(); pp_pair_t_kernel<<<ew_grid(len), 256, 0, s>>>(t, w, q, Aq, two_a, inv_mod2, len, running, R, first);
}
void launch_pp_pair_q(double* q, const double* At, double inv_mod2, int64_t len, const int* running, int R,
                      cudaStream_t s) {
  count_launch(); pp_pair_q_kernel<<<ew_grid(len), 256, 0, s>>>(q, At, inv_mod2, len, running, R);
}
void launch_cheb(double* z, double* d, double* r, const double* Ad, double c1, double c2, int64_t len, int phase,
                 const int* running, int R, cudaStream_t s) {
  count_launch(); cheb_kernel<<<ew_grid(len), 256, 0, s>>>(z, d, r, Ad, c1, c2, len, phase, running, R);
}
void poly_epi_apply(const PolyEpi& e, const float* v, int64_t len, const int* active, int R, cudaStream_t s) {
  if (len <= 0) return;
  count_launch(); poly_epi_kernel<<<ew_grid(len), kThreads, 0, s>>>(e, v, len, active, R);
}

void launch_ritz_leja(const double* H, int ldh, int P, int harmonic, double* re, double* im, int* nout,
                      unsigned* err, cudaStream_t s) {
  const size_t smem = sizeof(double) * 2 * kMaxPoly * kMaxPoly;
  cudaFuncSetAttribute(ritz_leja_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch(); ritz_leja_kernel<<<1, 1, smem, s>>>(H, ldh, P, harmonic, re, im, nout, err);
}

}  // namespace hdg
