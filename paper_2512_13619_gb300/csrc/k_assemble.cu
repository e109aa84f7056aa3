// Face-based assembly of the trace matrix (Sec. 4.2), extraction and packing
// of the block-Jacobi diagonal blocks (Sec. 4.5), construction of the ASM
// element matrices (Sec. 4.6), the face-parallel ASM prolongation sum, and
// element recovery (Eq. w19, Eq. w16).
#include "hdg_common.cuh"
#include "hdg_internal.h"
#include "k_poly.cuh"

namespace hdg {

namespace {

// One CTA per free face row: copies the (2N_lfe-1) b x b blocks out of the
// condensed element matrices into column-major padded slot blocks, adds the
// second element's contribution on the diagonal, and forms r_f.
__global__ void assemble_kernel(AssembleDesc d) {
  const int64_t f = blockIdx.x;
  const int b = d.b, bb = b * b, nlb = d.nlb;
  const int64_t r0 = d.rowptr[f];
  const int ns = (int)(d.rowptr[f + 1] - r0);
  for (int s = 0; s < ns; ++s) {
    const int64_t slot = f * d.max_slots + s;
    const int64_t dst = r0 + s;
    const int e = d.slot_e[slot];
    const int lr = d.slot_lr[slot], lc = d.slot_lc[slot];
    const int e2 = (s == 0) ? d.diag2[f * 2] : -1;
    const int l2 = (s == 0) ? d.diag2[f * 2 + 1] : -1;
    for (int idx = threadIdx.x; idx < bb; idx += blockDim.x) {
      const int j = idx / b, i = idx - j * b;      // column-major position (i, j)
      double v = 0.0;
      if (e >= 0) {
        v = d.Kbar[(int64_t)e * nlb * nlb + (int64_t)(lr * b + i) * nlb + lc * b + j];
        if (e2 >= 0) v += d.Kbar[(int64_t)e2 * nlb * nlb + (int64_t)(l2 * b + i) * nlb + l2 * b + j];
      }
      if (d.K64) d.K64[dst * d.s64 + idx] = v;
      if (d.K32) d.K32[dst * d.s32 + (int64_t)j * d.ld32 + i] = (float)v;
      if (d.K16) d.K16[dst * d.s16 + (int64_t)j * d.ld16 + i] = __float2bfloat16_rn((float)v);
    }
  }
  // right-hand side: r_f = sum over the face's elements of rbar^e_l minus the
  // Dirichlet columns of Kbar^e times u_D
  const int R = d.R;
  for (int idx = threadIdx.x; idx < b * R; idx += blockDim.x) {
    const int i = idx / R, r = idx - i * R;
    double acc = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int e = d.rhs_src[f * 4 + 2 * side], l = d.rhs_src[f * 4 + 2 * side + 1];
      if (e < 0) continue;
      const int row = l * b + i;
      acc += d.rbar[((int64_t)e * nlb + row) * R + r];
      for (int lp = 0; lp < d.nl; ++lp) {
        const int fg = d.elem_face[(int64_t)e * d.nl + lp];
        if (!d.face_dir[fg]) continue;
        const double* krow = d.Kbar + (int64_t)e * nlb * nlb + (int64_t)row * nlb + lp * b;
        const double* ud = d.uhatD + (int64_t)fg * b * R;
        for (int j = 0; j < b; ++j) acc -= krow[j] * ud[j * R + r];
      }
    }
    d.r[(f * b + i) * R + r] = acc;
  }
}

__global__ void extract_diag_kernel(const double* K64, int64_t s64, const int64_t* rowptr, int b, int64_t n_free,
                                    double* out) {
  const int64_t f = blockIdx.x;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int j = idx / b, i = idx - j * b;
    out[f * b * b + i * b + j] = K64[rowptr[f] * s64 + idx];
  }
}

__global__ void pack_blocks_kernel(const double* in, int n, double* o64, int64_t s64, float* o32, int64_t s32,
                                   int ld32, __nv_bfloat16* o16, int64_t s16, int ld16) {
  const int64_t m = blockIdx.x;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n, row = idx - c * n;
    const double v = in[m * n * n + (int64_t)row * n + c];
    if (o64) o64[m * s64 + idx] = v;
    if (o32) o32[m * s32 + (int64_t)c * ld32 + row] = (float)v;
    if (o16) o16[m * s16 + (int64_t)c * ld16 + row] = __float2bfloat16_rn((float)v);
  }
}

// P^e (dense row-major nlb x nlb, compacted to the element's free faces):
// off-diagonal blocks from Kbar^e, diagonal blocks = K_ff (both elements),
// padding rows/columns = identity.
__global__ void asm_build_kernel(const double* Kbar, int nlb, int b, int nl, const int32_t* asm_lf,
                                 const int32_t* asm_cnt, const int32_t* asm_face_free, const double* K64,
                                 int64_t s64, const int64_t* rowptr, double* P) {
  const int64_t e = blockIdx.x;
  const int cnt = asm_cnt[e];
  const int n = nlb;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int rr = idx / n, cc = idx - rr * n;
    const int s = rr / b, i = rr - s * b;
    const int t = cc / b, j = cc - t * b;
    double v;
    if (s >= cnt || t >= cnt) {
      v = (rr == cc) ? 1.0 : 0.0;
    } else if (s == t) {
      const int64_t f = asm_face_free[e * nl + s];
      v = K64[rowptr[f] * s64 + (int64_t)j * b + i];
    } else {
      const int ls = asm_lf[e * nl + s], lt = asm_lf[e * nl + t];
      v = Kbar[e * (int64_t)n * n + (int64_t)(ls * b + i) * n + lt * b + j];
    }
    P[e * (int64_t)n * n + idx] = v;
  }
}

__global__ void asm_pack_kernel(const double* Pinv, int nlb, int b, int nl, const int64_t* arowptr, double* o64,
                                int64_t s64, float* o32, int64_t s32, int ld32, __nv_bfloat16* o16, int64_t s16,
                                int ld16) {
  const int64_t e = blockIdx.x;
  const int n = nlb;
  const int ns = (int)(arowptr[e + 1] - arowptr[e]);
  for (int s = 0; s < ns; ++s) {
    const int64_t panel = arowptr[e] + s;
    for (int idx = threadIdx.x; idx < n * b; idx += blockDim.x) {
      const int c = idx / n, row = idx - c * n;
      const double v = Pinv[e * (int64_t)n * n + (int64_t)row * n + s * b + c];
      if (o64) o64[panel * s64 + idx] = v;
      if (o32) o32[panel * s32 + (int64_t)c * ld32 + row] = (float)v;
      if (o16) o16[panel * s16 + (int64_t)c * ld16 + row] = __float2bfloat16_rn((float)v);
    }
  }
}

__global__ void asm_face_sum_kernel(const double* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum,
                                    double* z) {
  const int64_t total = n_free * b * R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = idx / (b * R);
    const int rem = (int)(idx - f * b * R);
    const int e1 = fsum[f * 4], s1 = fsum[f * 4 + 1], e2 = fsum[f * 4 + 2], s2 = fsum[f * 4 + 3];
    double v = ze[((int64_t)e1 * nlb + s1 * b) * R + rem];
    if (e2 >= 0) v += ze[((int64_t)e2 * nlb + s2 * b) * R + rem];
    z[idx] = v;
  }
}

__global__ void asm_face_sum_f32_kernel(const float* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum,
                                        PolyEpi pe, double* z64, float* z32) {
  const int64_t total = n_free * b * R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = idx / (b * R);
    const int rem = (int)(idx - f * b * R);
    const int e1 = fsum[f * 4], s1 = fsum[f * 4 + 1], e2 = fsum[f * 4 + 2], s2 = fsum[f * 4 + 3];
    float v = ze[((int64_t)e1 * nlb + s1 * b) * R + rem];
    if (e2 >= 0) v += ze[((int64_t)e2 * nlb + s2 * b) * R + rem];
    if (pe.op != POLY_OP_NONE) {
      poly_epi(pe, idx, v);
    } else {
      if (z64) z64[idx] = (double)v;
      if (z32) z32[idx] = v;
    }
  }
}

__global__ void expand_trace_kernel(const double* x, const double* uhatD, const int32_t* free_of_face, int64_t n_face,
                                    int b, int R, double* full) {
  const int64_t total = n_face * b * R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = idx / (b * R);
    const int rem = (int)(idx - f * b * R);
    const int32_t ff = free_of_face[f];
    full[idx] = (ff >= 0) ? x[(int64_t)ff * b * R + rem] : uhatD[idx];
  }
}

// One CTA per element: u = Ebar^{-1} r_u - Ebar^{-1} Fbar uhat^e (Eq. w19),
// q_{a,d} = -((M^e)^{-1} B_d u_a + (M^e)^{-1} C_d uhat_a) (Eq. w16).
__global__ void recover_kernel(RecoverDesc d) {
  extern __shared__ double sm[];
  const int b = d.M * d.PF, nlb = d.nl * b, R = d.R, PE = d.PE, MPE = d.M * d.PE, nlPF = d.nl * d.PF;
  double* uh = sm;                  // nlb x R
  double* us = sm + nlb * R;        // MPE x R
  const int64_t e = blockIdx.x;
  for (int idx = threadIdx.x; idx < nlb * R; idx += blockDim.x) {
    const int row = idx / R, r = idx - row * R;
    const int l = row / b, i = row - l * b;
    const int32_t f = d.elem_face[e * d.nl + l];
    uh[idx] = d.uhat_full[((int64_t)f * b + i) * R + r];
  }
  __syncthreads();
  const double* XF = d.XF + e * (int64_t)MPE * nlb;
  const double* Xr = d.Xr + e * (int64_t)MPE * R;
  for (int idx = threadIdx.x; idx < MPE * R; idx += blockDim.x) {
    const int row = idx / R, r = idx - row * R;
    double acc = Xr[idx];
    const double* xr = XF + (int64_t)row * nlb;
    for (int k = 0; k < nlb; ++k) acc -= xr[k] * uh[k * R + r];
    us[idx] = acc;
    d.u[e * (int64_t)MPE * R + idx] = acc;
  }
  __syncthreads();
  const double* MB = d.MinvB + e * (int64_t)d.D * PE * PE;
  const double* MC = d.MinvC + e * (int64_t)d.D * PE * nlPF;
  const int nq = d.M * d.D * PE;
  for (int idx = threadIdx.x; idx < nq * R; idx += blockDim.x) {
    const int row = idx / R, r = idx - row * R;
    const int a = row / (d.D * PE);
    const int rem = row - a * d.D * PE;
    const int dd = rem / PE, i = rem - dd * PE;
    double acc = 0.0;
    const double* mb = MB + ((int64_t)dd * PE + i) * PE;
    for (int k = 0; k < PE; ++k) acc += mb[k] * us[(a * PE + k) * R + r];
    const double* mc = MC + ((int64_t)dd * PE + i) * nlPF;
    for (int l = 0; l < d.nl; ++l)
      for (int j = 0; j < d.PF; ++j) acc += mc[l * d.PF + j] * uh[((l * d.M + a) * d.PF + j) * R + r];
    d.q[e * (int64_t)nq * R + idx] = -acc;
  }
}

__global__ void bcast_copy_kernel(double* dst, const double* src, int64_t n, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i % n];
}

inline unsigned grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 65535 * 16) g = 65535 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void assemble(const AssembleDesc& d, cudaStream_t s) {
  if (d.n_free <= 0) return;
  count_launch(); assemble_kernel<<<(unsigned)d.n_free, 256, 0, s>>>(d);
}

void extract_diag(const double* K64, int64_t s64, const int64_t* rowptr, int b, int64_t n_free, double* out,
                  cudaStream_t s) {
  if (n_free <= 0) return;
  count_launch(); extract_diag_kernel<<<(unsigned)n_free, 256, 0, s>>>(K64, s64, rowptr, b, n_free, out);
}

void pack_blocks(const double* in, int n, int64_t count, double* o64, int64_t s64, float* o32, int64_t s32,
                 int ld32, __nv_bfloat16* o16, int64_t s16, int ld16, cudaStream_t s) {
  if (count <= 0) return;
  count_launch(); pack_blocks_kernel<<<(unsigned)count, 256, 0, s>>>(in, n, o64, s64, o32, s32, ld32, o16, s16, ld16);
}

void asm_build(const double* Kbar, int nlb, int b, int nl, int64_t n_elem, const int32_t* asm_lf,
               const int32_t* asm_cnt, const int32_t* asm_face_free, const double* K64, int64_t s64,
               const int64_t* rowptr, double* P, cudaStream_t s) {
  if (n_elem <= 0) return;
  count_launch(); asm_build_kernel<<<(unsigned)n_elem, 256, 0, s>>>(Kbar, nlb, b, nl, asm_lf, asm_cnt, asm_face_free, K64, s64,
                                                     rowptr, P);
}

void asm_pack(const double* Pinv, int nlb, int b, int nl, int64_t n_elem, const int64_t* arowptr, double* o64,
              int64_t s64, float* o32, int64_t s32, int ld32, __nv_bfloat16* o16, int64_t s16, int ld16,
              cudaStream_t s) {
  if (n_elem <= 0) return;
  count_launch(); asm_pack_kernel<<<(unsigned)n_elem, 256, 0, s>>>(Pinv, nlb, b, nl, arowptr, o64, s64, o32, s32, ld32, o16,
                                                                   s16, ld16);
}

void asm_face_sum(const double* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum, double* z,
                  cudaStream_t s) {
  int64_t total = n_free * b * R;
  if (total <= 0) return;
  count_launch(); asm_face_sum_kernel<<<grid_for(total, 256), 256, 0, s>>>(ze, nlb, b, R, n_free, fsum, z);
}

void asm_face_sum_f32(const float* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum,
                      const PolyEpi* pe, double* z64, float* z32, cudaStream_t s) {
  int64_t total = n_free * b * R;
  if (total <= 0) return;
  PolyEpi e{};
  if (pe) e = *pe;
  count_launch();
  asm_face_sum_f32_kernel<<<grid_for(total, 256), 256, 0, s>>>(ze, nlb, b, R, n_free, fsum, e, z64, z32);
}

void bcast_copy(double* dst, const double* src, int64_t n, int64_t count, cudaStream_t s) {
  const int64_t total = n * count;
  if (total <= 0) return;
  count_launch(); bcast_copy_kernel<<<grid_for(total, 256), 256, 0, s>>>(dst, src, n, total);
}

void expand_trace(const double* x, const double* uhatD, const int32_t* free_of_face, int64_t n_face, int b, int R,
                  double* full, cudaStream_t s) {
  int64_t total = n_face * b * R;
  if (total <= 0) return;
  count_launch(); expand_trace_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, uhatD, free_of_face, n_face, b, R, full);
}

void recover(const RecoverDesc& d, cudaStream_t s) {
  if (d.n_elem <= 0) return;
  const int b = d.M * d.PF;
  size_t smem = (size_t)(d.nl * b + d.M * d.PE) * d.R * sizeof(double);
  cudaFuncSetAttribute(recover_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  count_launch(); recover_kernel<<<(unsigned)d.n_elem, 256, smem, s>>>(d);
}

}  // namespace hdg
