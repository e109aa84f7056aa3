// Block-row products: the face-block matrix-vector product y_f = K_f x_f
// (Sec. 4.3, each face row couples the face with the faces of its two
// elements), the block-Jacobi apply z_f = P_f^{-1} y_f (Sec. 4.5) and the
// element solves z^e = (Pbar^e)^{-1} y^e of the ASM apply (Sec. 4.6) all have
// the form
//     out[u][row] = sum_{s < cnt[u]} sum_c blk[u][s](row, c) * in[nbr[u][s]][c]
// with dense column-major slot blocks stored compactly (unit u's blocks at
// rowptr[u] .. rowptr[u+1]-1).  Instead of materialising the paper's extended
// x vector, the gather goes through the neighbour table.
//
// Kernel "tma": a persistent CTA takes tasks (a group of G consecutive units,
// or one unit split into slot ranges when a row is long); each task's blocks
// are contiguous in HBM and arrive with ONE 1D bulk copy (cp.async.bulk,
// completion by mbarrier transaction count) into a ring of shared-memory
// stages filled by a producer warp.  Consumer thread (unit g, row, part p)
// accumulates columns c = p, p+P, ... of every slot (column-major blocks make
// the shared-memory reads conflict-free), gathers x through L1/L2, and the P
// partial sums meet in shared memory before the epilogue.
// Kernel "direct": one thread per output row with plain global loads.
// FP32/BF16 blocks multiply an FP32 copy of x (converting each gathered FP64
// value per product would run on the FP64 pipe, 1/57 of the FP32 rate here).
//
// Included by the per-precision translation units (k_blockrow_f64.cu,
// k_blockrow_f32.cu, k_blockrow_bf16.cu) so that their template
// instantiations compile in parallel.
#pragma once
#include <algorithm>
#include <type_traits>
#include "hdg_common.cuh"
#include "hdg_internal.h"
#include "k_poly.cuh"

namespace hdg {

namespace {

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

__device__ __forceinline__ void epi_store(const BlockRowDesc& d, int64_t u, int row, int r, double v) {
  const int64_t o = (u * d.b_rows + row) * d.R + r;
  if (d.epi == EPI_POLY) {
    poly_epi(d.pe, o, (float)v);
    return;
  }
  if (d.epi == EPI_RESID) v = d.rhs[o] - v;
  else if (d.epi == EPI_SCALE) v = d.scale[r] * v;
  if (d.out) d.out[o] = v;
  if (d.out32) d.out32[o] = (float)v;
}

// Four consecutive outputs (u, row, r0 .. r0+3) of a row, r0 a multiple of 4
// (R a multiple of 4): 16-byte state and output accesses.
__device__ __forceinline__ void epi_store4(const BlockRowDesc& d, int64_t u, int row, int r0, float4 v) {
  const int64_t o = (u * d.b_rows + row) * d.R + r0;
  if (d.epi == EPI_POLY) {
    poly_epi4(d.pe, o, v);
    return;
  }
  if (d.epi == EPI_RESID || d.epi == EPI_SCALE) {
    epi_store(d, u, row, r0, (double)v.x);
    epi_store(d, u, row, r0 + 1, (double)v.y);
    epi_store(d, u, row, r0 + 2, (double)v.z);
    epi_store(d, u, row, r0 + 3, (double)v.w);
    return;
  }
  if (d.out) st4d(d.out + o, v);
  if (d.out32) st4(d.out32 + o, v);
}

__device__ __forceinline__ bool any_active(const int* active, int R) {
  if (active == nullptr) return true;
  for (int r = 0; r < R; ++r)
    if (active[r]) return true;
  return false;
}

// x in the accumulation precision: FP64 from `in`, FP32 from the FP32 copy
template <typename A> __device__ __forceinline__ A load_x(const BlockRowDesc& d, int64_t i);
template <> __device__ __forceinline__ double load_x<double>(const BlockRowDesc& d, int64_t i) { return __ldg(d.in + i); }
template <> __device__ __forceinline__ float load_x<float>(const BlockRowDesc& d, int64_t i) { return __ldg(d.in32 + i); }

__device__ __forceinline__ void consumer_bar(int nt) { asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory"); }

struct Plan {
  int G, P, S, nch, nstage, NT, NPW;   // units/task, column parts, slots/chunk, chunks/task, stages, consumers, producer warps
  int stage_bytes;                    // bytes of one stage (blocks + gathered x + metadata)
  int kbytes;                         // block area of a stage
  int xoff, moff;                     // offsets of the x area and the metadata area inside a stage
  int64_t ntasks;
};

// Stage layout: [blocks: kbytes][x: G*S*bc*R doubles][meta: G ints cnt, G ints block offset, G*S ints unused]
template <typename T, int R>
__global__ void __launch_bounds__(640) blockrow_tma_kernel(BlockRowDesc d, Plan pl) {
  using A = typename Acc<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + pl.nstage;
  unsigned char* stages = smem + 256;
  A* red = reinterpret_cast<A*>(stages + (size_t)pl.nstage * pl.stage_bytes);
  __shared__ volatile int s_abort;
  __shared__ long long s_issued[8];   // last iteration issued on each stage (drain after an abort)

  const int NT = pl.NT;
  const int tid = threadIdx.x;
  if (!any_active(d.active, R)) return;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < pl.nstage; ++i) {
      s_issued[i] = -1;
      mbar_init(&full[i], 32);
      mbar_init(&empty[i], NT / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();

  const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
  const T* blk = static_cast<const T*>(d.blk);
  const int G = pl.G, P = pl.P, S = pl.S, bc = d.bc;
  const bool whole = (pl.nch == 1);

  if (tid >= NT) {
    // ------------------------------------------------------------ producers
    // Warp w of NPW takes the CTA's tasks k = w, w+NPW, ...  For each chunk it
    // loads the metadata and gathers x for the chunk into the stage with plain
    // loads, lane 0 issues one bulk copy for the blocks, and all 32 lanes
    // arrive on the stage's full barrier (lane 0 with the byte count).
    const int w = (tid - NT) >> 5, lane = tid & 31;
    bool abort = false;
    for (int64_t k = w, t = blockIdx.x + (int64_t)w * gridDim.x; t < pl.ntasks;
         k += pl.NPW, t += (int64_t)pl.NPW * gridDim.x) {
      const int64_t u0 = t * G;
      const int64_t u1 = min(u0 + G, d.n_units);
      for (int ch = 0; ch < pl.nch; ++ch) {
        const int64_t it = k * pl.nch + ch;
        const int st = (int)(it % pl.nstage);
        const unsigned ph = (unsigned)((it / pl.nstage) & 1);
        if (s_abort || !mbar_wait_bounded(&empty[st], ph ^ 1u)) {
          if (!s_abort) atomicOr(d.err, ERRBIT_TIMEOUT);
          s_abort = 1;
          abort = true;
          break;
        }
        unsigned char* sbase = stages + (size_t)st * pl.stage_bytes;
        A* xs = reinterpret_cast<A*>(sbase + pl.xoff);
        int* meta = reinterpret_cast<int*>(sbase + pl.moff);
        const int s0 = whole ? 0 : ch * S;
        int64_t b0, nb;
        if (whole) {
          b0 = d.rowptr[u0];
          nb = d.rowptr[u1] - b0;
        } else {
          b0 = d.rowptr[u0] + s0;
          nb = max(0, min(S, d.cnt[u0] - s0));
        }
        if (lane == 0) {
          // register the bytes first (no arrival), then start the copy; the
          // 32 arrivals of the warp come after the x stores below
          const unsigned bytes = (unsigned)(nb * blk_bytes);
          s_issued[st] = it;
          if (bytes) {
            mbar_expect_tx(&full[st], bytes);
            bulk_g2s(sbase, blk + b0 * d.blk_stride, bytes, &full[st]);
          }
        }
        // per-unit metadata: number of slots in this chunk and block offset in the stage
        for (int g = lane; g < G; g += 32) {
          const int64_t u = u0 + g;
          int ns = 0, off = 0;
          if (u < d.n_units) {
            ns = whole ? d.cnt[u] : max(0, min(S, d.cnt[u] - s0));
            off = whole ? (int)(d.rowptr[u] - b0) : 0;
          }
          meta[g] = ns;
          meta[G + g] = off;
        }
        // gathered x of every (unit, slot in chunk, column)
        const int per_unit = S * bc * R;
        for (int idx = lane; idx < G * per_unit; idx += 32) {
          const int g = idx / per_unit;
          const int rem = idx - g * per_unit;
          const int sl = rem / (bc * R);
          const int cr = rem - sl * bc * R;
          const int64_t u = u0 + g;
          A v = (A)0;
          if (u < d.n_units) {
            const int ns = whole ? d.cnt[u] : min(S, d.cnt[u] - s0);
            if (sl < ns) v = load_x<A>(d, (int64_t)d.nbr[u * d.max_slots + s0 + sl] * bc * R + cr);
          }
          xs[idx] = v;
        }
        mbar_arrive(&full[st]);  // one arrival per lane (count 32); release orders the x stores
      }
      if (abort) break;
    }
  } else {
  // -------------------------------------------------------------- consumers
  const int rows = G * d.b_rows;
  const int lr = tid % rows;
  const int part = tid / rows;
  const int g = lr / d.b_rows;
  const int row = lr - g * d.b_rows;
  const int lane = tid & 31;
  const bool in_part = part < P;
  bool abort = false;
  int64_t k = 0;
  for (int64_t t = blockIdx.x; t < pl.ntasks; t += gridDim.x, ++k) {
    const int64_t u = t * G + g;
    A acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = (A)0;
    for (int ch = 0; ch < pl.nch; ++ch) {
      const int64_t it = k * pl.nch + ch;
      const int st = (int)(it % pl.nstage);
      const unsigned ph = (unsigned)((it / pl.nstage) & 1);
      if (!abort && !mbar_wait_bounded(&full[st], ph)) {
        atomicOr(d.err, ERRBIT_TIMEOUT);
        abort = true;
        s_abort = 1;
      }
      if (!abort && in_part) {
        const unsigned char* sbase = stages + (size_t)st * pl.stage_bytes;
        const int* meta = reinterpret_cast<const int*>(sbase + pl.moff);
        int ns = meta[g];
        const int off = meta[G + g];
        if (ns < 0 || off < 0 || (int64_t)(off + ns) * blk_bytes > (int64_t)pl.kbytes) {   // never for a sound ring
          atomicOr(d.err, ERRBIT_ARG);
          ns = 0;
        }
        const T* sb = reinterpret_cast<const T*>(sbase) + (int64_t)off * d.blk_stride + row;
        const A* xs = reinterpret_cast<const A*>(sbase + pl.xoff) + (int64_t)g * S * bc * R;
        for (int sl = 0; sl < ns; ++sl) {
          const T* bs = sb + (int64_t)sl * d.blk_stride;
          const A* xv = xs + sl * bc * R;
#pragma unroll 4
          for (int c = part; c < bc; c += P) {
            const A kv = cvt<A>(bs[c * d.ld]);
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(kv, xv[c * R + r], acc[r]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (abort) break;
    // reduce the P column parts of each output row
    if (P == 1) {
      if (in_part && u < d.n_units) {
#pragma unroll
        for (int r = 0; r < R; ++r) epi_store(d, u, row, r, (double)acc[r]);
      }
    } else {
      if (in_part) {
#pragma unroll
        for (int r = 0; r < R; ++r) red[((int64_t)part * rows + lr) * R + r] = acc[r];
      }
      consumer_bar(NT);
      if (part == 0 && u < d.n_units) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          A sum = red[(int64_t)lr * R + r];
          for (int q = 1; q < P; ++q) sum += red[((int64_t)q * rows + lr) * R + r];
          epi_store(d, u, row, r, (double)sum);
        }
      }
      consumer_bar(NT);
    }
  }
  }
  // After an abort, bulk copies may still be in flight on stages nobody
  // consumed: wait (bounded) for them before the CTA's shared memory goes away.
  __syncthreads();
  if (tid == 0 && s_abort) {
    for (int i = 0; i < pl.nstage; ++i) {
      const long long q = s_issued[i];
      if (q >= 0 && !mbar_wait_bounded(&full[i], (unsigned)((q / pl.nstage) & 1))) atomicOr(d.err, ERRBIT_TIMEOUT);
    }
  }
}

// One thread per output row; BC > 0 fixes the column count at compile time so
// the loads of a whole slot block are in flight together.
template <typename T, int R, int BC>
__global__ void __launch_bounds__(512) blockrow_direct_kernel(BlockRowDesc d) {
  using A = typename Acc<T>::type;
  if (!any_active(d.active, R)) return;
  const int bc = BC > 0 ? BC : d.bc;
  // column stride: FP64 blocks are stored unpadded (ld == b_rows)
  const int ldb = std::is_same<T, double>::value ? d.b_rows : d.ld;
  const int G = blockDim.x / d.b_rows;
  const int gu = threadIdx.x / d.b_rows;
  const int row = threadIdx.x - gu * d.b_rows;
  if (gu >= G) return;
  const T* blk = static_cast<const T*>(d.blk);
  const int64_t ngroups = (d.n_units + G - 1) / G;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t u = grp * G + gu;
    if (u >= d.n_units) continue;
    A acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = (A)0;
    const int n = d.cnt[u];
    const int64_t rp = d.rowptr[u];
    const int32_t* nbr = d.nbr + u * d.max_slots;
    for (int s = 0; s < n; ++s) {
      const int64_t xb = (int64_t)nbr[s] * bc * R;
      const T* bs = blk + (rp + s) * d.blk_stride + row;
      if (BC > 0) {
        T kv[BC > 0 ? BC : 1];
#pragma unroll
        for (int c = 0; c < (BC > 0 ? BC : 1); ++c) kv[c] = __ldg(bs + (size_t)c * ldb);
#pragma unroll
        for (int c = 0; c < (BC > 0 ? BC : 1); ++c)
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = fma(cvt<A>(kv[c]), load_x<A>(d, xb + c * R + r), acc[r]);
      } else {
#pragma unroll 4
        for (int c = 0; c < bc; ++c) {
          const A kv = cvt<A>(__ldg(bs + (size_t)c * ldb));
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = fma(kv, load_x<A>(d, xb + c * R + r), acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) epi_store(d, u, row, r, (double)acc[r]);
  }
}

// Rows split over SP slot parts: thread t serves part t % SP of row
// (t / SP) % b_rows of unit t / (SP b_rows) in its group; part p sums slots
// p, p + SP, ...; the SP partial sums of a row sit in SP adjacent lanes of one
// warp and are added by shuffles (every lane takes part, so idle lanes carry
// zeros).  For small meshes, where one thread per row leaves most of the SMs'
// warp slots empty.
template <typename T, int R, int BC, int SP>
__global__ void __launch_bounds__(512) blockrow_split_kernel(BlockRowDesc d) {
  using A = typename Acc<T>::type;
  if (!any_active(d.active, R)) return;
  const int bc = BC > 0 ? BC : d.bc;
  const int ldb = std::is_same<T, double>::value ? d.b_rows : d.ld;
  const int per_unit = d.b_rows * SP;
  const int G = blockDim.x / per_unit;
  const int part = threadIdx.x % SP;
  const int rr = threadIdx.x / SP;
  const int gu = rr / d.b_rows;
  const int row = rr - gu * d.b_rows;
  const T* blk = static_cast<const T*>(d.blk);
  const int64_t ngroups = (d.n_units + G - 1) / G;
  // every CTA runs the same number of group iterations, so the shuffles see full warps
  for (int64_t g0 = 0; g0 < ngroups; g0 += gridDim.x) {
    const int64_t grp = g0 + blockIdx.x;
    const int64_t u = grp * G + gu;
    const bool live = grp < ngroups && gu < G && u < d.n_units;
    A acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = (A)0;
    if (live) {
      const int n = d.cnt[u];
      const int64_t rp = d.rowptr[u];
      const int32_t* nbr = d.nbr + u * d.max_slots;
      for (int s = part; s < n; s += SP) {
        const int64_t xb = (int64_t)nbr[s] * bc * R;
        const T* bs = blk + (rp + s) * d.blk_stride + row;
#pragma unroll 4
        for (int c = 0; c < bc; ++c) {
          const A kv = cvt<A>(__ldg(bs + (size_t)c * ldb));
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] = fma(kv, load_x<A>(d, xb + c * R + r), acc[r]);
        }
      }
    }
#pragma unroll
    for (int o = SP / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (live && part == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) epi_store(d, u, row, r, (double)acc[r]);
    }
  }
}

// FP32/BF16 blocks: each thread owns VR consecutive rows of a unit, so one
// 16-byte load brings VR rows of a column (column-major blocks, rows
// contiguous).  Requires ld % VR == 0 (the FP32/BF16 copies pad every column
// to whole 16-byte vectors; the padding rows are computed and dropped); x
// comes from the FP32 copy, R values of a column in 16-byte loads when R is a
// multiple of 4.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  static constexpr int N = 4;
  __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct Vec16<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};

// Thread (unit, row group rg, slot part sp): rows rg*VR..rg*VR+VR-1, slots
// sp, sp+SP, ...; the SP slot parts of a row group are adjacent lanes and
// combine their sums with shuffles.  SP in {1, 2, 4, 8}; (ld / VR) * SP <= 256.
// MINB > 1 compiles for MINB resident CTAs of 256 threads per SM: 3 (at most
// 80 registers) for more loads in flight at R = 8, 4 (at most 64 registers)
// for small problems at R <= 2, whose few face rows give few threads.
template <typename T, int R, int BC, int SP, int MINB = 1, int RS = 1>
__global__ void __launch_bounds__(MINB > 1 ? 256 : 288, MINB) blockrow_vec_kernel(BlockRowDesc d, int G) {
  constexpr int VR = Vec16<T>::N;
  constexpr int RR = R / RS;                     // right-hand sides of this thread: r0 .. r0 + RR - 1
  if (!any_active(d.active, R)) return;
  const int tpu = (d.ld / VR) * SP * RS;         // threads per unit; G units per CTA,
                                                 // threads past G*tpu only join the shuffles
  const int gu = threadIdx.x / tpu;
  const int q = threadIdx.x - gu * tpu;
  const int sp = q % SP, rg = q / (SP * RS);
  const int r0 = ((q / SP) % RS) * RR;
  const bool valid = gu < G;
  const T* blk = static_cast<const T*>(d.blk);
  const int64_t ngroups = (d.n_units + G - 1) / G;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t u = grp * G + gu;
    const bool act = valid && u < d.n_units;
    float acc[VR][RR];
#pragma unroll
    for (int v = 0; v < VR; ++v)
#pragma unroll
      for (int r = 0; r < RR; ++r) acc[v][r] = 0.f;
    if (act) {
      const int n = d.cnt[u];
      const int64_t rp = d.rowptr[u];
      const int32_t* nbr = d.nbr + u * d.max_slots;
      for (int s = sp; s < n; s += SP) {
        const float* xin = d.in32 + (int64_t)nbr[s] * BC * R + r0;
        const T* bs = blk + (rp + s) * d.blk_stride + rg * VR;
#pragma unroll
        for (int c = 0; c < BC; ++c) {
          float kv[VR];
          Vec16<T>::load(bs + (size_t)c * d.ld, kv);
          float xv[RR];
          if constexpr (RR % 4 == 0) {
#pragma unroll
            for (int r4 = 0; r4 < RR; r4 += 4) {
              const float4 q = __ldg(reinterpret_cast<const float4*>(xin + c * R + r4));
              xv[r4] = q.x; xv[r4 + 1] = q.y; xv[r4 + 2] = q.z; xv[r4 + 3] = q.w;
            }
          } else {
#pragma unroll
            for (int r = 0; r < RR; ++r) xv[r] = __ldg(xin + c * R + r);
          }
#pragma unroll
          for (int r = 0; r < RR; ++r) {
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[v][r] = fmaf(kv[v], xv[r], acc[v][r]);
          }
        }
      }
    }
    if (SP > 1) {
#pragma unroll
      for (int v = 0; v < VR; ++v)
#pragma unroll
        for (int r = 0; r < RR; ++r) {
#pragma unroll
          for (int o = 1; o < SP; o <<= 1) acc[v][r] += __shfl_xor_sync(0xffffffffu, acc[v][r], o);
        }
    }
    if (act && sp == 0) {
#pragma unroll
      for (int v = 0; v < VR; ++v)
        if (rg * VR + v < d.b_rows) {
          if constexpr (RR % 4 == 0) {
#pragma unroll
            for (int r = 0; r < RR; r += 4)
              epi_store4(d, u, rg * VR + v, r0 + r,
                         make_float4(acc[v][r], acc[v][r + 1], acc[v][r + 2], acc[v][r + 3]));
          } else {
#pragma unroll
            for (int r = 0; r < RR; ++r) epi_store(d, u, rg * VR + v, r0 + r, (double)acc[v][r]);
          }
        }
    }
  }
}


// Kernel "bulk": persistent CTAs (one per SM) stream G whole units per stage
// with ONE bulk copy (a unit's blocks are contiguous in HBM; the copy is
// tagged evict-first in L2 so that the gathered x stays resident there) into
// a ring of shared-memory stages that a single producer lane keeps full; the
// same lane copies each unit's x slots (b x R floats each, through the
// neighbour table) into the stage, on the same mbarrier.  Eight consumer
// warps read K and x from shared memory, VR rows of a column per 16-byte
// vector.  Consumer thread (unit g,
// row group rg, column part cp) sums the columns c = cp, cp + NCP, ... of the
// unit's concatenated slot columns; the NSUB parts inside a warp meet by
// shuffles, the WPU warps of a unit in shared memory.  FP32/BF16 blocks.
struct BulkPlan {
  int G, NS, WPU, NSUB, NRG;
  int stage_bytes;     // bytes of one stage (a multiple of 128): blocks, then the x slots
  int x_off;           // offset of the x slots in a stage (G * max_slots slots of b x R floats)
  int red_floats;      // reduction area
  int64_t ntasks;
};
constexpr int kBulkConsumers = 256;
template <typename T, int R, int BC>
__global__ void __launch_bounds__(kBulkConsumers + 32, 1) blockrow_bulk_kernel(BlockRowDesc d, BulkPlan pl) {
  constexpr int VR = Vec16<T>::N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + 8;
  float* red = reinterpret_cast<float*>(smem + 256);
  unsigned char* stages = smem + 256 + ((size_t)pl.red_floats * 4 + 127) / 128 * 128;
  __shared__ volatile int s_abort;
  __shared__ long long s_issued[8];
  const int tid = threadIdx.x;
  if (!any_active(d.active, R)) return;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < pl.NS; ++i) {
      s_issued[i] = -1;
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kBulkConsumers / 32);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
  const T* blk = static_cast<const T*>(d.blk);
  if (tid >= kBulkConsumers) {
    // ------------------------------------------------------------ producer warp
    // Per stage: the lanes load the stage's neighbour indices (before waiting
    // for the stage to be free, so the loads overlap the wait), lane 0 sets the
    // byte count and copies the blocks, and the lanes copy the x slots, pair
    // p = (unit p / max_slots, slot p % max_slots).
    const int lane = tid - kBulkConsumers;
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    const unsigned xbytes = (unsigned)(d.bc * R * sizeof(float));
    const int npairs = pl.G * d.max_slots;
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < pl.ntasks; t += gridDim.x, ++k) {
      const int st = (int)(k % pl.NS);
      const unsigned ph = (unsigned)((k / pl.NS) & 1);
      const int64_t u0 = t * pl.G;
      const int64_t u1 = min(u0 + pl.G, d.n_units);
      const int64_t b0 = d.rowptr[u0], b1 = d.rowptr[u1];
      int32_t src[4];                    // x slot of pair lane + 32 q, or -1
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pr = lane + 32 * q;
        src[q] = -1;
        if (pr < npairs) {
          const int64_t u = u0 + pr / d.max_slots;
          const int sl = pr % d.max_slots;
          if (u < u1 && sl < d.cnt[u]) src[q] = d.nbr[u * d.max_slots + sl];
        }
      }
      bool ok = true;
      if (lane == 0) ok = !s_abort && mbar_wait_bounded(&empty[st], ph ^ 1u);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          if (!s_abort) atomicOr(d.err, ERRBIT_TIMEOUT);
          s_abort = 1;
        }
        break;
      }
      unsigned char* dst = stages + (size_t)st * pl.stage_bytes;
      if (lane == 0) {
        const unsigned bytes = (unsigned)((b1 - b0) * blk_bytes);
        s_issued[st] = k;
        mbar_arrive_expect_tx(&full[st], bytes + xbytes * (unsigned)(b1 - b0));
        if (bytes)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
              "%4;" ::"r"(smem_u32(dst)),
              "l"(blk + b0 * d.blk_stride), "r"(bytes), "r"(smem_u32(&full[st])), "l"(pol)
              : "memory");
      }
      __syncwarp();
      float* xdst = reinterpret_cast<float*>(dst + pl.x_off);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pr = lane + 32 * q;
        if (src[q] >= 0)
          bulk_g2s(xdst + (size_t)pr * d.bc * R, d.in32 + (int64_t)src[q] * d.bc * R, xbytes, &full[st]);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int w = tid >> 5, lane = tid & 31;
    const int g = w / pl.WPU, wu = w - g * pl.WPU;
    const int rg = lane / pl.NSUB, sub = lane - rg * pl.NSUB;
    const bool valid = rg < pl.NRG && g < pl.G;
    const int NCP = pl.WPU * pl.NSUB;
    const int cp = wu * pl.NSUB + sub;
    bool abort = false;
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < pl.ntasks; t += gridDim.x, ++k) {
      const int st = (int)(k % pl.NS);
      const unsigned ph = (unsigned)((k / pl.NS) & 1);
      if (!abort && !mbar_wait_bounded(&full[st], ph)) {
        atomicOr(d.err, ERRBIT_TIMEOUT);
        abort = true;
        s_abort = 1;
      }
      const int64_t u0 = t * pl.G;
      const int64_t u = u0 + g;
      float acc[VR][R];
#pragma unroll
      for (int v = 0; v < VR; ++v)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[v][r] = 0.f;
      if (!abort && valid && u < d.n_units) {
        const int n = d.cnt[u];
        const int64_t off = d.rowptr[u] - d.rowptr[u0];
        const T* sb = reinterpret_cast<const T*>(stages + (size_t)st * pl.stage_bytes) + off * d.blk_stride +
                      rg * VR;
        const float* sx = reinterpret_cast<const float*>(stages + (size_t)st * pl.stage_bytes + pl.x_off) +
                          (size_t)g * d.max_slots * BC * R;
        const int ncol = n * BC;
#pragma unroll 4
        for (int c = cp; c < ncol; c += NCP) {
          const int sl = c / BC;
          const int col = c - sl * BC;
          float kv[VR];
          if constexpr (std::is_same<T, float>::value) {
            const float4 q = *reinterpret_cast<const float4*>(sb + (int64_t)sl * d.blk_stride + col * d.ld);
            kv[0] = q.x; kv[1] = q.y; kv[2] = q.z; kv[3] = q.w;
          } else {
            const uint4 q = *reinterpret_cast<const uint4*>(sb + (int64_t)sl * d.blk_stride + col * d.ld);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
            for (int i = 0; i < VR / 2; ++i) {
              const float2 f = __bfloat1622float2(h[i]);
              kv[2 * i] = f.x;
              kv[2 * i + 1] = f.y;
            }
          }
          const float* xin = sx + c * R;      // slot sl, column col: (sl * BC + col) * R
          float xv[R];
          if constexpr (R % 4 == 0) {
#pragma unroll
            for (int r4 = 0; r4 < R; r4 += 4) {
              const float4 q = *reinterpret_cast<const float4*>(xin + r4);
              xv[r4] = q.x; xv[r4 + 1] = q.y; xv[r4 + 2] = q.z; xv[r4 + 3] = q.w;
            }
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) xv[r] = xin[r];
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < VR; ++v) acc[v][r] = fmaf(kv[v], xv[r], acc[v][r]);
        }
      }
      // the warp is done with the stage's blocks
      __syncwarp();
      if (lane == 0 && !abort) mbar_arrive(&empty[st]);
      // the NSUB column parts of a warp
      for (int o = 1; o < pl.NSUB; o <<= 1)
#pragma unroll
        for (int v = 0; v < VR; ++v)
#pragma unroll
          for (int r = 0; r < R; ++r) acc[v][r] += __shfl_xor_sync(0xffffffffu, acc[v][r], o);
      if (pl.WPU == 1) {
        if (!abort && valid && sub == 0 && u < d.n_units) {
#pragma unroll
          for (int v = 0; v < VR; ++v)
            if (rg * VR + v < d.b_rows) {
              if constexpr (R % 4 == 0) {
#pragma unroll
                for (int r = 0; r < R; r += 4)
                  epi_store4(d, u, rg * VR + v, r,
                             make_float4(acc[v][r], acc[v][r + 1], acc[v][r + 2], acc[v][r + 3]));
              } else {
#pragma unroll
                for (int r = 0; r < R; ++r) epi_store(d, u, rg * VR + v, r, (double)acc[v][r]);
              }
            }
        }
      } else {
        // red[g][wu][row][r], rows rg * VR + v
        const int rows = pl.NRG * VR;
        if (valid && sub == 0) {
#pragma unroll
          for (int v = 0; v < VR; ++v)
#pragma unroll
            for (int r = 0; r < R; ++r) red[(((int64_t)g * pl.WPU + wu) * rows + rg * VR + v) * R + r] = acc[v][r];
        }
        consumer_bar(kBulkConsumers);
        if (!abort) {
          for (int idx = tid; idx < pl.G * d.b_rows * R; idx += kBulkConsumers) {
            const int gg = idx / (d.b_rows * R);
            const int rem = idx - gg * d.b_rows * R;
            const int row = rem / R, r = rem - row * R;
            const int64_t uu = u0 + gg;
            if (uu >= d.n_units) continue;
            float sum = 0.f;
            for (int q = 0; q < pl.WPU; ++q) sum += red[(((int64_t)gg * pl.WPU + q) * rows + row) * R + r];
            epi_store(d, uu, row, r, (double)sum);
          }
        }
        consumer_bar(kBulkConsumers);
      }
      if (abort) break;
    }
  }
  // after an abort, copies may still be in flight: wait (bounded) for them
  // before the CTA's shared memory goes away
  __syncthreads();
  if (tid == 0 && s_abort) {
    for (int i = 0; i < pl.NS; ++i) {
      const long long q = s_issued[i];
      if (q >= 0 && !mbar_wait_bounded(&full[i], (unsigned)((q / pl.NS) & 1))) atomicOr(d.err, ERRBIT_TIMEOUT);
    }
  }
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);  // a cached attribute query
  return n > 0 ? n : 1;
}

constexpr size_t kStageTarget = 40 * 1024;
constexpr size_t kSmemCap = 200 * 1024;

int largest_divisor_leq(int n, int cap) {
  for (int p = std::min(n, cap); p >= 1; --p)
    if (n % p == 0) return p;
  return 1;
}

template <typename T, int R>
Plan make_plan(const BlockRowDesc& d) {
  Plan pl{};
  const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
  const size_t row_bytes = (size_t)d.max_slots * blk_bytes;
  const int nt_max = 512;
  if (row_bytes <= kStageTarget) {
    pl.G = (int)std::max<size_t>(1, std::min<size_t>(kStageTarget / row_bytes, (size_t)(nt_max / d.b_rows)));
    pl.S = d.max_slots;
    pl.nch = 1;
    pl.kbytes = (int)(pl.G * row_bytes);
  } else {
    pl.G = 1;
    pl.S = (int)std::max<size_t>(1, kStageTarget / blk_bytes);
    if (pl.S > d.max_slots) pl.S = d.max_slots;
    pl.nch = (d.max_slots + pl.S - 1) / pl.S;
    pl.kbytes = (int)(pl.S * blk_bytes);
  }
  pl.P = largest_divisor_leq(d.bc, std::max(1, nt_max / (pl.G * d.b_rows)));
  pl.NT = ((pl.G * d.b_rows * pl.P + 31) / 32) * 32;
  const size_t xbytes = (size_t)pl.G * pl.S * d.bc * R * sizeof(typename Acc<T>::type);
  pl.xoff = (pl.kbytes + 15) / 16 * 16;
  pl.moff = (int)((pl.xoff + xbytes + 15) / 16 * 16);
  pl.stage_bytes = (int)((pl.moff + 2 * pl.G * sizeof(int) + 127) / 128 * 128);
  const size_t red = (pl.P > 1) ? (size_t)pl.P * pl.G * d.b_rows * R * sizeof(typename Acc<T>::type) : 0;
  pl.nstage = (int)std::min<size_t>(8, (kSmemCap - red) / pl.stage_bytes);
  if (pl.nstage < 2) pl.nstage = 2;
  // Producer warps fill the stage ring out of order (warp w takes tasks w,
  // w+NPW, ...), and an mbarrier parity wait tells only two generations of a
  // stage apart: the wait for iteration `it` is sound only if iteration
  // it - 2*nstage has been consumed.  A warp's first chunk of a task is
  // covered by its own previous wait iff (NPW-1)*nch + 1 <= nstage (later
  // chunks follow from the one before), hence NPW <= 1 + (nstage-1)/nch.
  pl.NPW = std::max(1, std::min(4, 1 + (pl.nstage - 1) / pl.nch));
  pl.ntasks = (d.n_units + pl.G - 1) / pl.G;
  return pl;
}

// Plan of the bulk kernel; false when a unit's blocks do not fit a stage of
// kBulkStageMax bytes or the rows do not divide into 16-byte vectors.
constexpr size_t kBulkStageMax = 96 * 1024;
template <typename T>
bool bulk_plan(const BlockRowDesc& d, BulkPlan* pl) {
  if constexpr (std::is_same<T, double>::value) {
    return false;
  } else {
    constexpr int VR = Vec16<T>::N;
    if (d.in32 == nullptr || d.ld % VR != 0 || d.ld < d.b_rows) return false;
    const size_t blk_bytes = (size_t)d.blk_stride * sizeof(T);
    const size_t row_bytes = (size_t)d.max_slots * blk_bytes;
    if (blk_bytes == 0 || blk_bytes % 16 != 0 || row_bytes > kBulkStageMax) return false;
    BulkPlan q{};
    q.NRG = d.ld / VR;
    if (q.NRG > 32) return false;
    q.NSUB = 1;
    while (q.NSUB * 2 * q.NRG <= 32) q.NSUB *= 2;
    // units per stage: as many as fit the stage size, with a whole number of
    // consumer warps each (G * WPU = 8)
    // x slots: whole 16-byte rows (b R floats) so that each is one bulk copy;
    // at most 128 (unit, slot) pairs per stage (four per producer lane)
    if ((d.bc * d.R * sizeof(float)) % 16 != 0 || d.max_slots > 128) return false;
    int G = 1;
    while (G * 2 <= 8 && (size_t)G * 2 * row_bytes <= kBulkStageMax && G * 2 * d.max_slots <= 128) G *= 2;
    q.G = G;
    q.WPU = (kBulkConsumers / 32) / G;
    q.x_off = (int)(((size_t)G * row_bytes + 127) / 128 * 128);
    q.stage_bytes = (int)((q.x_off + (size_t)G * d.max_slots * d.bc * d.R * sizeof(float) + 127) / 128 * 128);
    q.red_floats = q.WPU > 1 ? G * q.WPU * q.NRG * VR * d.R : 0;
    const size_t red_bytes = ((size_t)q.red_floats * 4 + 127) / 128 * 128;
    q.NS = (int)std::min<size_t>(8, (kSmemCap - red_bytes) / q.stage_bytes);
    if (q.NS < 2) return false;
    q.ntasks = (d.n_units + G - 1) / G;
    *pl = q;
    return true;
  }
}

template <typename T, int R, int BC>
bool launch_bulk(const BlockRowDesc& d, cudaStream_t s) {
  BulkPlan pl;
  if (!bulk_plan<T>(d, &pl)) return false;
  const size_t smem = 256 + ((size_t)pl.red_floats * 4 + 127) / 128 * 128 + (size_t)pl.NS * pl.stage_bytes;
  auto kern = blockrow_bulk_kernel<T, R, BC>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);  // per context; cheap
  int64_t grid = std::min<int64_t>(pl.ntasks, (int64_t)num_sms());
  if (grid < 1) grid = 1;
  count_launch(); kern<<<(unsigned)grid, kBulkConsumers + 32, smem, s>>>(d, pl);
  return true;
}

template <typename T, int R>
void launch_tma(const BlockRowDesc& d, cudaStream_t s) {
  const Plan pl = make_plan<T, R>(d);
  const size_t red = (pl.P > 1) ? (size_t)pl.P * pl.G * d.b_rows * R * sizeof(typename Acc<T>::type) : 0;
  const size_t smem = 256 + (size_t)pl.nstage * pl.stage_bytes + red;
  auto kern = blockrow_tma_kernel<T, R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);  // per context; cheap
  const int threads = pl.NT + 32 * pl.NPW;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = std::min<int64_t>(pl.ntasks, (int64_t)num_sms() * per_sm);
  if (grid < 1) grid = 1;
  count_launch(); kern<<<(unsigned)grid, threads, smem, s>>>(d, pl);
}

int pick_nt_direct(int b_rows) {
  int best = 32 * ((b_rows + 31) / 32), bestu = -1;
  for (int nt = best; nt <= 512; nt += 32) {
    int util = (nt / b_rows) * b_rows * 1000 / nt;
    if (util > bestu || (util == bestu && nt <= 256)) { bestu = util; best = nt; }
  }
  return best;
}

template <typename T, int R, int BC, int SP, int MINB = 1, int RS = 1>
void launch_vec_sp(const BlockRowDesc& d, int cps, cudaStream_t s) {
  constexpr int VR = Vec16<T>::N;
  const int tpu = (d.ld / VR) * SP * RS;
  const int G = std::max(1, 256 / tpu);
  const int NT = (G * tpu + 31) / 32 * 32;        // whole warps for the full-mask shuffles
  int64_t ngroups = (d.n_units + G - 1) / G;
  int64_t grid = std::min<int64_t>(ngroups, (int64_t)num_sms() * (cps > 0 ? cps : 16));
  if (grid < 1) grid = 1;
  count_launch(); blockrow_vec_kernel<T, R, BC, SP, MINB, RS><<<(unsigned)grid, NT, 0, s>>>(d, G);
}

// A shuffle group is SP adjacent lanes starting at a multiple of SP, so it
// never straddles a warp.  Heuristic: 4 parts for rows of several slots
// (matvec, ASM), 1 for one slot (BJ).
template <typename T, int R, int BC>
void launch_vec(const BlockRowDesc& d, int sp, int cps, bool occ3, cudaStream_t s, bool rsplit = false) {
  if (sp <= 0) sp = d.max_slots >= 4 ? 4 : d.max_slots >= 2 ? 2 : 1;
  while (sp > 1 && (d.ld / Vec16<T>::N) * sp > 256) sp >>= 1;   // threads per unit <= 256
  if constexpr (R == 8) {
    if (rsplit && sp <= 2 && (d.ld / Vec16<T>::N) * sp * 2 <= 256) {
      if (sp == 1) launch_vec_sp<T, R, BC, 1, 3, 2>(d, cps, s);
      else launch_vec_sp<T, R, BC, 2, 3, 2>(d, cps, s);
      return;
    }
  }
  if constexpr (R == 8) {
    if (occ3 && sp <= 2) {
      if (sp == 1) launch_vec_sp<T, R, BC, 1, 3>(d, cps, s);
      else launch_vec_sp<T, R, BC, 2, 3>(d, cps, s);
      return;
    }
  }
  if constexpr (R <= 2 && std::is_same<T, float>::value) {
    if (occ3 && sp <= 4) {
      if (sp == 1) launch_vec_sp<T, R, BC, 1, 4>(d, cps, s);
      else if (sp == 2) launch_vec_sp<T, R, BC, 2, 4>(d, cps, s);
      else launch_vec_sp<T, R, BC, 4, 4>(d, cps, s);
      return;
    }
  }
  switch (sp) {
    case 1: launch_vec_sp<T, R, BC, 1>(d, cps, s); break;
    case 2: launch_vec_sp<T, R, BC, 2>(d, cps, s); break;
    case 4: launch_vec_sp<T, R, BC, 4>(d, cps, s); break;
    default: launch_vec_sp<T, R, BC, 8>(d, cps, s); break;
  }
}

template <typename T>
bool vec_ok(const BlockRowDesc& d) {
  if constexpr (std::is_same<T, double>::value) {
    return false;
  } else {
    return d.ld % Vec16<T>::N == 0 && d.ld / Vec16<T>::N <= 64 && d.ld >= d.b_rows && d.in32 != nullptr;
  }
}

bool bc_compiled(int bc) {
  return bc == 3 || bc == 4 || bc == 9 || bc == 16 || bc == 20 || bc == 27 || bc == 45;
}

// Slot parts for an FP64 product under the heuristic: the largest SP <= 8
// (and <= the slots per unit, SP b_rows <= 512) with at most 2048 threads per
// SM in all; 1 when one thread per row already fills that.
int split_parts(const BlockRowDesc& d) {
  const int64_t threads = d.n_units * (int64_t)d.b_rows;
  int sp = 1;
  while (sp < 8 && 2 * sp <= d.max_slots && 2 * sp * d.b_rows <= 512 &&
         threads * 2 * sp <= (int64_t)num_sms() * 2048)
    sp *= 2;
  return sp;
}

template <typename T, int R, int BC, int SP>
void launch_split_sp(const BlockRowDesc& d, int cps, cudaStream_t s) {
  const int per_unit = d.b_rows * SP;
  const int NT = pick_nt_direct(per_unit);
  const int G = NT / per_unit;
  const int64_t ngroups = (d.n_units + G - 1) / G;
  int64_t grid = std::min<int64_t>(ngroups, (int64_t)num_sms() * (cps > 0 ? cps : 8));
  if (grid < 1) grid = 1;
  count_launch(); blockrow_split_kernel<T, R, BC, SP><<<(unsigned)grid, NT, 0, s>>>(d);
}

template <typename T, int R, int BC>
void launch_split(const BlockRowDesc& d, int sp, int cps, cudaStream_t s) {
  switch (sp) {
    case 2: launch_split_sp<T, R, BC, 2>(d, cps, s); break;
    case 4: launch_split_sp<T, R, BC, 4>(d, cps, s); break;
    default: launch_split_sp<T, R, BC, 8>(d, cps, s); break;
  }
}

template <typename T, int R, int BC>
void launch_direct_bc(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  // the bulk kernel for the shapes whose face rows fit a stage (b = 9, 16,
  // 20, 27) with several right-hand sides
  if constexpr (!std::is_same<T, double>::value && (BC == 9 || BC == 16 || BC == 20 || BC == 27) && R >= 4) {
    if (cfg.kind == BR_BULK && launch_bulk<T, R, BC>(d, s)) return;
  }
  if constexpr (!std::is_same<T, double>::value && BC > 0) {
    if ((cfg.kind == BR_DEFAULT || cfg.kind == BR_VEC || cfg.kind == BR_VEC3 || cfg.kind == BR_VEC3R) &&
        vec_ok<T>(d)) {
      launch_vec<T, R, BC>(d, cfg.sp, cfg.cps, cfg.kind == BR_VEC3 || cfg.kind == BR_VEC3R, s, cfg.kind == BR_VEC3R);
      return;
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    const int sp = cfg.kind == BR_SPLIT ? cfg.sp : (cfg.kind == BR_DEFAULT ? split_parts(d) : 1);
    if (sp > 1 && sp * d.b_rows <= 512) {
      launch_split<T, R, 0>(d, sp, cfg.cps, s);     // the column count stays a run-time value
      return;
    }
  }
  const int NT = pick_nt_direct(d.b_rows);
  const int G = NT / d.b_rows;
  int64_t ngroups = (d.n_units + G - 1) / G;
  int64_t grid = std::min<int64_t>(ngroups, (int64_t)num_sms() * (cfg.cps > 0 ? cfg.cps : 8));
  if (grid < 1) grid = 1;
  count_launch(); blockrow_direct_kernel<T, R, BC><<<(unsigned)grid, NT, 0, s>>>(d);
}

template <typename T, int R>
void launch_direct(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  switch (d.bc) {
    case 3: launch_direct_bc<T, R, 3>(d, cfg, s); break;
    case 4: launch_direct_bc<T, R, 4>(d, cfg, s); break;
    case 9: launch_direct_bc<T, R, 9>(d, cfg, s); break;
    case 16: launch_direct_bc<T, R, 16>(d, cfg, s); break;
    case 20: launch_direct_bc<T, R, 20>(d, cfg, s); break;
    case 27: launch_direct_bc<T, R, 27>(d, cfg, s); break;
    case 45: launch_direct_bc<T, R, 45>(d, cfg, s); break;
    default: launch_direct_bc<T, R, 0>(d, cfg, s); break;
  }
}

#define HDG_BR_CASE(RR)                                  \
  case RR:                                               \
    if (cfg.kind == BR_TMA) launch_tma<T, RR>(d, s);     \
    else launch_direct<T, RR>(d, cfg, s);                \
    break;
// R in {1, 2} and R in {4, 8}: separate translation units compile them in parallel
template <typename T>
void dispatch_R_narrow(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  switch (d.R) {
    HDG_BR_CASE(1)
    HDG_BR_CASE(2)
    default: break;
  }
}
template <typename T>
void dispatch_R_wide(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  switch (d.R) {
    HDG_BR_CASE(4)
    HDG_BR_CASE(8)
    default: break;
  }
}
template <typename T>
void dispatch_R(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s) {
  if (d.R <= 2) dispatch_R_narrow<T>(d, cfg, s);
  else dispatch_R_wide<T>(d, cfg, s);
}
#undef HDG_BR_CASE

template <typename T>
int candidates_T(const BlockRowDesc& d, BrCfg* out, int cap) {
  int n = 0;
  auto add = [&](int kind, int sp, int cps) {
    if (n < cap) {
      out[n].kind = kind; out[n].sp = sp; out[n].cps = cps;
      ++n;
    }
  };
  for (int cps : {4, 8, 16}) add(BR_DIRECT, 0, cps);
  if constexpr (std::is_same<T, double>::value) {
    for (int sp : {2, 4, 8})
      if (sp <= d.max_slots && sp * d.b_rows <= 512)
        for (int cps : {8, 16}) add(BR_SPLIT, sp, cps);
  } else {
    if (vec_ok<T>(d) && bc_compiled(d.bc)) {
      for (int sp : {1, 2, 4, 8})
        if ((sp == 1 || sp <= d.max_slots) && (d.ld / Vec16<T>::N) * sp <= 256)
          for (int cps : {8, 16, 32}) add(BR_VEC, sp, cps);
      if (d.R == 8)
        for (int sp : {1, 2})
          if ((sp == 1 || sp <= d.max_slots) && (d.ld / Vec16<T>::N) * sp <= 256)
            for (int cps : {16, 32}) add(BR_VEC3, sp, cps);
      if (d.R == 8)
        for (int sp : {1, 2})
          if ((sp == 1 || sp <= d.max_slots) && (d.ld / Vec16<T>::N) * sp * 2 <= 256)
            for (int cps : {16, 32}) add(BR_VEC3R, sp, cps);
      if (d.R <= 2 && std::is_same<T, float>::value)
        for (int sp : {1, 2, 4})
          if ((sp == 1 || sp <= d.max_slots) && (d.ld / Vec16<T>::N) * sp <= 256)
            for (int cps : {16, 32}) add(BR_VEC3, sp, cps);
      BulkPlan bp;
      if ((d.bc == 9 || d.bc == 16 || d.bc == 20 || d.bc == 27) && d.R >= 4 && bulk_plan<T>(d, &bp))
        add(BR_BULK, 0, 0);
    }
  }
  add(BR_TMA, 0, 0);
  return n;
}

}  // namespace
}  // namespace hdg
