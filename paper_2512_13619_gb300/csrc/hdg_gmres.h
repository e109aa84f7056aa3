// Device-side GMRES state shared by the Krylov kernels and the host driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hdg {

constexpr int kMaxBasis = 128;   // restart length m + 1 <= kMaxBasis
constexpr int kMaxR = 8;         // right-hand sides per problem (1, 2, 4 or 8)
constexpr int kMaxPoly = 48;     // polynomial degree cap

// Plain view of the device arrays (passed by value to kernels).
struct GmresView {
  int64_t n;          // trace unknowns
  int R, m;
  int64_t chunk;      // elements per block in the reductions
  double* V;          // (m+1) x n x R, unnormalised basis
  double* vscale;     // (m+1) x R: V_i / ||V_i|| = vscale_i V_i
  double* H;          // R x (m+1) x m rotated Hessenberg (upper triangular)
  double* g;          // R x (m+1)
  double* cs;         // R x m
  double* sn;         // R x m
  double* hcol;       // R x (m+2) current Hessenberg column
  double* htmp;       // R x (m+2) dot products of the current pass
  double* ycoef;      // R x (m+1)
  double* partial;    // reduction scratch
  double* tolabs;     // R: absolute least-squares tolerance of the cycle
  double* cfac;       // R: tolerance factor (divided by 10 after a false stop)
  double* zb;         // R: ||P^{-1} b||
  double rtol;
  int* running;       // R
  int* jend;          // R
  int* on_estimate;   // R
  int* done;          // R
  int* iters;         // R
  int maxit;
  const int* dmaxit;  // device copy of maxit (read by kernels replayed from cycle graphs); may be NULL
  int* hflag;         // host-mapped: hflag[j] = 1 while any RHS is running after step j
  int use_cond;       // inside a captured cycle: set `cond` after every Givens step
  cudaGraphConditionalHandle cond;
  unsigned* counter;
  unsigned* err;
};

int64_t gmres_chunk(int64_t len);
int gmres_blocks(int64_t len, int64_t chunk);
void launch_dots(const GmresView& k, const double* w, int i0, int i1, cudaStream_t s);
void launch_update(const GmresView& k, double* w, int i0, int i1, int j, int hmode, int finalize, cudaStream_t s);
void launch_norms(const GmresView& k, const double* v, double* out, int cycle, const double* denom, cudaStream_t s);
void launch_backsolve(const GmresView& k, cudaStream_t s);
void launch_xupdate(const GmresView& k, double* x, cudaStream_t s);
void launch_axpby(double* y, const double* x, double a, double b, int64_t len, const int* running, int R,
                  cudaStream_t s);
void launch_pp_real(double* w, double* q, const double* Aq, double inv_theta, int64_t len, int update_q,
                    const int* running, int R, int first, cudaStream_t s);
void launch_pp_pair_t(double* t, double* w, const double* q, const double* Aq, double two_a, double inv_mod2,
                      int64_t len, const int* running, int R, int first, cudaStream_t s);
void launch_pp_pair_q(double* q, const double* At, double inv_mod2, int64_t len, const int* running, int R,
                      cudaStream_t s);
void launch_cheb(double* z, double* d, double* r, const double* Ad, double c1, double c2, int64_t len, int phase,
                 const int* running, int R, cudaStream_t s);
void launch_ritz_leja(const double* H, int ldh, int P, int harmonic, double* re, double* im, int* nout,
                      unsigned* err, cudaStream_t s);

}  // namespace hdg
