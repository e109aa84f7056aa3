// Block-row products: the face-block matrix-vector product y_f = K_f x_f
// (Sec. 4.3, each face row couples the face with the faces of its two
// elements), the block-Jacobi apply z_f = P_f^{-1} y_f (Sec. 4.5) and the
// element solves z^e = (Pbar^e)^{-1} y^e of the ASM apply (Sec. 4.6) all have
// the form
//     out[u][row] = sum_{s < cnt[u]} sum_c blk[u][s](row, c) * in[nbr[u][s]][c]
// with dense column-major slot blocks.  Instead of materialising the paper's
// extended x vector, the gather goes through the neighbour table.
//
// Kernel "tma": a persistent CTA streams the slot blocks of a group of units
// through a ring of shared-memory stages with 1D bulk copies
// (cp.async.bulk, completion tracked by mbarrier transaction counts); one
// producer warp issues the copies, the consumer warps read each block with
// one thread per output row (column-major blocks make those reads
// conflict-free) and gather x through L1/L2.  HBM sees each block once.
// Kernel "direct": the same mapping with plain coalesced global loads.
#include <algorithm>
#include "hdg_common.cuh"
#include "hdg_internal.h"

namespace hdg {

namespace {

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <int R, typename A>
__device__ __forceinline__ void epilogue(const BlockRowDesc& d, int64_t u, int row, const A (&acc)[R]) {
  int64_t o = (u * d.b_rows + row) * R;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double v = (double)acc[r];
    if (d.epi == EPI_RESID) v = d.rhs[o + r] - v;
    else if (d.epi == EPI_SCALE) v = d.scale[r] * v;
    d.out[o + r] = v;
  }
}

__device__ __forceinline__ bool any_active(const int* active, int R) {
  if (active == nullptr) return true;
  for (int r = 0; r < R; ++r)
    if (active[r]) return true;
  return false;
}

template <typename T, int R>
__global__ void __launch_bounds__(544) blockrow_tma_kernel(BlockRowDesc d, int S, int nstage, int stage_bytes) {
  using A = typename Acc<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + nstage;
  unsigned char* stages = smem + 128;
  __shared__ volatile int s_abort;

  const int NT = blockDim.x - 32;          // consumer threads
  const int nwc = NT / 32;
  const int tid = threadIdx.x;
  const bool producer = tid >= NT;
  if (!any_active(d.active, R)) return;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < nstage; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], nwc);
    }
    fence_mbar_init();
  }
  __syncthreads();

  const int G = NT / d.b_rows;
  const int64_t ngroups = (d.n_units + G - 1) / G;
  const int nchunks = (d.max_slots + S - 1) / S;
  const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
  const T* blk = static_cast<const T*>(d.blk);
  int64_t issued = 0;

  if (producer) {
    if ((tid & 31) == 0) {
      int64_t it = 0;
      for (int64_t g = blockIdx.x; g < ngroups && !s_abort; g += gridDim.x) {
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int st = (int)(it % nstage);
          const unsigned ph = (unsigned)((it / nstage) & 1);
          if (!mbar_wait_bounded(&empty[st], ph ^ 1u)) {
            atomicOr(d.err, ERRBIT_TIMEOUT);
            s_abort = 1;
            break;
          }
          const int s0 = ch * S;
          unsigned bytes = 0;
          for (int gu = 0; gu < G; ++gu) {
            int64_t u = g * G + gu;
            if (u >= d.n_units) break;
            int ns = min(S, d.cnt[u] - s0);
            if (ns > 0) bytes += (unsigned)(ns * blk_bytes);
          }
          mbar_arrive_expect_tx(&full[st], bytes);
          unsigned char* dst = stages + (size_t)st * stage_bytes;
          for (int gu = 0; gu < G; ++gu) {
            int64_t u = g * G + gu;
            if (u >= d.n_units) break;
            int ns = min(S, d.cnt[u] - s0);
            if (ns > 0)
              bulk_g2s(dst + (size_t)gu * S * blk_bytes, blk + (u * d.max_slots + s0) * d.blk_stride,
                       (unsigned)(ns * blk_bytes), &full[st]);
          }
          issued = it + 1;
        }
      }
      // drain: every issued copy must land before the CTA can exit
      int64_t first = issued > nstage ? issued - nstage : 0;
      for (int64_t t = first; t < issued; ++t)
        if (!mbar_wait_bounded(&full[t % nstage], (unsigned)((t / nstage) & 1))) atomicOr(d.err, ERRBIT_TIMEOUT);
    }
  } else {
    const int gu = tid / d.b_rows;
    const int row = tid - gu * d.b_rows;
    const int lane = tid & 31;
    int64_t it = 0;
    bool abort = false;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
      const int64_t u = g * G + gu;
      const bool act = (gu < G) && (u < d.n_units);
      A acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = (A)0;
      for (int ch = 0; ch < nchunks; ++ch, ++it) {
        const int st = (int)(it % nstage);
        const unsigned ph = (unsigned)((it / nstage) & 1);
        if (!abort && !mbar_wait_bounded(&full[st], ph)) {
          atomicOr(d.err, ERRBIT_TIMEOUT);
          abort = true;
          s_abort = 1;
        }
        if (!abort && act) {
          const int s0 = ch * S;
          const int ns = min(S, d.cnt[u] - s0);
          const T* sb = reinterpret_cast<const T*>(stages + (size_t)st * stage_bytes + (size_t)gu * S * blk_bytes);
          for (int s = 0; s < ns; ++s) {
            const int32_t nb = d.nbr[u * d.max_slots + s0 + s];
            const double* xin = d.in + (int64_t)nb * d.bc * R;
            const T* bs = sb + (size_t)s * d.blk_stride + row;
#pragma unroll 4
            for (int c = 0; c < d.bc; ++c) {
              const A kv = cvt<A>(bs[c * d.b_rows]);
#pragma unroll
              for (int r = 0; r < R; ++r) acc[r] = fma(kv, (A)__ldg(xin + c * R + r), acc[r]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
      }
      if (act && !abort) epilogue<R, A>(d, u, row, acc);
      if (abort) break;
    }
  }
  __syncthreads();
}

template <typename T, int R>
__global__ void __launch_bounds__(512) blockrow_direct_kernel(BlockRowDesc d) {
  using A = typename Acc<T>::type;
  if (!any_active(d.active, R)) return;
  const int G = blockDim.x / d.b_rows;
  const int gu = threadIdx.x / d.b_rows;
  const int row = threadIdx.x - gu * d.b_rows;
  if (gu >= G) return;
  const T* blk = static_cast<const T*>(d.blk);
  const int64_t ngroups = (d.n_units + G - 1) / G;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t u = g * G + gu;
    if (u >= d.n_units) continue;
    A acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = (A)0;
    const int n = d.cnt[u];
    for (int s = 0; s < n; ++s) {
      const int32_t nb = d.nbr[u * d.max_slots + s];
      const double* xin = d.in + (int64_t)nb * d.bc * R;
      const T* bs = blk + (u * d.max_slots + s) * d.blk_stride + row;
#pragma unroll 4
      for (int c = 0; c < d.bc; ++c) {
        const A kv = cvt<A>(__ldg(bs + (size_t)c * d.b_rows));
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fma(kv, (A)__ldg(xin + c * R + r), acc[r]);
      }
    }
    epilogue<R, A>(d, u, row, acc);
  }
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

// consumer thread count giving the best row utilisation (<= 512)
int pick_nt(int b_rows) {
  int best = 32 * ((b_rows + 31) / 32), bestu = -1;
  for (int nt = 32 * ((b_rows + 31) / 32); nt <= 512; nt += 32) {
    int g = nt / b_rows;
    int used = g * b_rows;
    // utilisation in 1/1000, prefer larger CTAs on ties up to 256 threads
    int util = used * 1000 / nt;
    if (util > bestu || (util == bestu && nt <= 256)) { bestu = util; best = nt; }
  }
  return best;
}

template <typename T, int R>
void launch_tma(const BlockRowDesc& d, cudaStream_t s) {
  const int NT = pick_nt(d.b_rows);
  const int G = NT / d.b_rows;
  const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
  const size_t smem_cap = 200 * 1024;
  const size_t stage_target = 32 * 1024;
  int S = (int)std::max<size_t>(1, stage_target / (G * blk_bytes));
  S = std::min(S, d.max_slots);
  size_t stage_bytes = (size_t)G * S * blk_bytes;
  int nstage = (int)std::min<size_t>(8, smem_cap / stage_bytes);
  if (nstage < 2) nstage = 2;
  size_t smem = 128 + (size_t)nstage * stage_bytes;
  auto kern = blockrow_tma_kernel<T, R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT + 32, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t ngroups = (d.n_units + G - 1) / G;
  int64_t grid = std::min<int64_t>(ngroups, (int64_t)num_sms() * per_sm);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT + 32, smem, s>>>(d, S, nstage, (int)stage_bytes);
}

template <typename T, int R>
void launch_direct(const BlockRowDesc& d, cudaStream_t s) {
  const int NT = pick_nt(d.b_rows);
  const int G = NT / d.b_rows;
  int64_t ngroups = (d.n_units + G - 1) / G;
  int64_t grid = std::min<int64_t>(ngroups, (int64_t)num_sms() * 8);
  if (grid < 1) grid = 1;
  blockrow_direct_kernel<T, R><<<(unsigned)grid, NT, 0, s>>>(d);
}

template <typename T>
void dispatch_R(const BlockRowDesc& d, int variant, cudaStream_t s) {
#define HDG_BR_CASE(RR)                              \
  case RR:                                           \
    if (variant == 0) launch_tma<T, RR>(d, s);       \
    else launch_direct<T, RR>(d, s);                 \
    break;
  switch (d.R) {
    HDG_BR_CASE(1)
    HDG_BR_CASE(2)
    HDG_BR_CASE(4)
    HDG_BR_CASE(8)
    default: break;
  }
#undef HDG_BR_CASE
}

}  // namespace

int blockrow_variants() { return 2; }

void blockrow(const BlockRowDesc& d, int variant, cudaStream_t s) {
  if (d.n_units <= 0) return;
  if (d.prec == HDG_FP64) dispatch_R<double>(d, variant, s);
  else if (d.prec == HDG_FP32) dispatch_R<float>(d, variant, s);
  else dispatch_R<__nv_bfloat16>(d, variant, s);
}

}  // namespace hdg
