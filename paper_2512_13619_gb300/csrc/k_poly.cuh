// One step of a polynomial preconditioner (Sec. 4.7 recurrence, or the
// Chebyshev iteration) at output index o, fused into the epilogue of the
// kernel that produced v (see PolyEpi in hdg_internal.h).
#pragma once
#include "hdg_common.cuh"
#include "hdg_internal.h"

namespace hdg {
namespace {

__device__ __noinline__ void poly_epi(const PolyEpi& e, int64_t o, float v) {
  switch (e.op) {
    case CHEB_INIT: {
      const float dn = e.c1 * v;
      if (e.last) { e.out64[o] = (double)dn; break; }
      e.p0[o] = v;
      e.p2[o] = dn;
      e.p1[o] = dn;
      break;
    }
    case CHEB_STEP: {
      const float rn = e.p0[o] - v;
      const float dn = fmaf(e.c1, e.p2[o], e.c2 * rn);
      const float zn = e.p1[o] + dn;
      if (e.last) { e.out64[o] = (double)zn; break; }
      e.p0[o] = rn;
      e.p2[o] = dn;
      e.p1[o] = zn;
      break;
    }
    case PP_INIT:
      if (e.fin) e.out64[o] = (double)(e.cfin * v);
      else e.p0[o] = v;
      break;
    case PP_REAL: {
      const float q = e.p0[o];
      const float wn = fmaf(e.c1, q, e.wzero ? 0.f : e.p1[o]);
      const float qn = fmaf(-e.c1, v, q);
      if (e.fin) { e.out64[o] = (double)fmaf(e.cfin, qn, wn); break; }
      e.p0[o] = qn;
      e.p1[o] = wn;
      break;
    }
    case PP_PAIR_T: {
      const float t = fmaf(e.c1, e.p0[o], -v);
      const float wn = fmaf(e.c2, t, e.wzero ? 0.f : e.p1[o]);
      if (e.last) { e.out64[o] = (double)wn; break; }
      e.p2[o] = t;
      e.p1[o] = wn;
      break;
    }
    case PP_PAIR_Q: {
      const float qn = fmaf(-e.c2, v, e.p0[o]);
      if (e.fin) { e.out64[o] = (double)fmaf(e.cfin, qn, e.p1[o]); break; }
      e.p0[o] = qn;
      break;
    }
    default:
      break;
  }
}

// The same step on four consecutive outputs o .. o+3 (o a multiple of 4):
// 16-byte loads and stores of the FP32 state, 2 x 16-byte stores of out64.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4d(double* p, float4 v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
}
#define HDG_F4(expr_x, expr_y, expr_z, expr_w) make_float4(expr_x, expr_y, expr_z, expr_w)
__device__ __noinline__ void poly_epi4(const PolyEpi& e, int64_t o, float4 v) {
  switch (e.op) {
    case CHEB_INIT: {
      const float4 dn = HDG_F4(e.c1 * v.x, e.c1 * v.y, e.c1 * v.z, e.c1 * v.w);
      if (e.last) { st4d(e.out64 + o, dn); break; }
      st4(e.p0 + o, v);
      st4(e.p2 + o, dn);
      st4(e.p1 + o, dn);
      break;
    }
    case CHEB_STEP: {
      const float4 r = ld4(e.p0 + o), d = ld4(e.p2 + o), z = ld4(e.p1 + o);
      const float4 rn = HDG_F4(r.x - v.x, r.y - v.y, r.z - v.z, r.w - v.w);
      const float4 dn = HDG_F4(fmaf(e.c1, d.x, e.c2 * rn.x), fmaf(e.c1, d.y, e.c2 * rn.y),
                               fmaf(e.c1, d.z, e.c2 * rn.z), fmaf(e.c1, d.w, e.c2 * rn.w));
      const float4 zn = HDG_F4(z.x + dn.x, z.y + dn.y, z.z + dn.z, z.w + dn.w);
      if (e.last) { st4d(e.out64 + o, zn); break; }
      st4(e.p0 + o, rn);
      st4(e.p2 + o, dn);
      st4(e.p1 + o, zn);
      break;
    }
    default: {
      // the GMRES-polynomial steps element by element
      poly_epi(e, o, v.x);
      poly_epi(e, o + 1, v.y);
      poly_epi(e, o + 2, v.z);
      poly_epi(e, o + 3, v.w);
      break;
    }
  }
}
#undef HDG_F4

}  // namespace
}  // namespace hdg
