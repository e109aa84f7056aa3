// Element matrices of hexahedral Q^k HDG elements on the device: the step
// before the static condensation (Welter & Nguyen, Sec. 4.1 writes the
// element integrals as products of basis tables with quadrature weights,
// M = Phi W, and Eq. matrixform assembles the blocks D..J from them).
//
// Conventions (shared with the host-side input generator, so that both
// produce the same blocks for the same mesh):
//  - reference cube [-1,1]^3; Q^k Lagrange basis on Gauss-Lobatto-Legendre
//    nodes, node (i, j, l) at index i + (k+1) (j + (k+1) l), x fastest;
//  - volume rule: n^3 Gauss-Legendre points, x fastest; face rule: n^2;
//  - local face l = 2 axis + side fixes reference coordinate `axis` at
//    -1 (side 0) or +1 (side 1); its parameters (s, t) are the two other
//    coordinates in increasing axis order; face basis Q^k on GLL nodes in
//    (s, t), node (i, j) at index i + (k+1) j;
//  - trilinear geometry from 8 vertices, vertex v at reference corner
//    ((v & 1 ? 1 : -1), (v & 2 ? 1 : -1), (v & 4 ? 1 : -1));
//  - face_perm[e][l][j] = the local face-node index of element e's face l
//    that carries the face's global node j.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hdg_common.cuh"
#include "hdg_internal.h"

namespace hdg {

// ------------------------------------------------------------ 1D tables
namespace {

// Legendre P_n and P_n' at x by the three-term recurrence.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);     // interior points only
}

// n-point Gauss-Legendre rule: roots of P_n by Newton's method from the
// asymptotic guesses cos(pi (i + 3/4) / (n + 1/2)); w = 2 / ((1 - x^2) P_n'^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &P, &dP);
      const double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(n, t, &P, &dP);
    x[n - 1 - i] = t;                          // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// k+1 Gauss-Lobatto-Legendre nodes: -1, the roots of P_k', +1.  Newton on
// P_k' with P_k'' = (2 x P_k' - k (k+1) P_k) / (1 - x^2), from the
// Chebyshev-Lobatto points.
std::vector<double> gll_nodes(int k) {
  std::vector<double> g(k + 1);
  if (k == 0) {
    g[0] = 0.0;
    return g;
  }
  g[0] = -1.0;
  g[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double t = -std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(k, t, &P, &dP);
      const double d2 = (2.0 * t * dP - k * (k + 1.0) * P) / (1.0 - t * t);
      const double dt = dP / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    g[i] = t;
  }
  return g;
}

// Lagrange polynomials through `nodes` and their derivatives at t (product form).
void lagrange(const std::vector<double>& nodes, double t, double* phi, double* dphi) {
  const int n = (int)nodes.size();
  for (int j = 0; j < n; ++j) {
    double v = 1.0, d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      const double den = nodes[j] - nodes[m];
      d = d * (t - nodes[m]) / den + v / den;    // product rule, one factor at a time
      v *= (t - nodes[m]) / den;
    }
    phi[j] = v;
    dphi[j] = d;
  }
}

// Q^k values and reference gradients at a point of the cube.
void hex_basis_at(const std::vector<double>& g, const double xi[3], double* phi, double* dphi /* PE x 3 */) {
  const int n1 = (int)g.size();
  std::vector<double> p[3], dp[3];
  for (int a = 0; a < 3; ++a) {
    p[a].resize(n1);
    dp[a].resize(n1);
    lagrange(g, xi[a], p[a].data(), dp[a].data());
  }
  for (int l = 0; l < n1; ++l)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        const int idx = (l * n1 + j) * n1 + i;
        phi[idx] = p[0][i] * p[1][j] * p[2][l];
        if (dphi) {
          dphi[idx * 3 + 0] = dp[0][i] * p[1][j] * p[2][l];
          dphi[idx * 3 + 1] = p[0][i] * dp[1][j] * p[2][l];
          dphi[idx * 3 + 2] = p[0][i] * p[1][j] * dp[2][l];
        }
      }
}

// derivatives of the 8 trilinear shape functions at xi: dN[v*3 + b]
void trilinear_dN(const double xi[3], double* dN) {
  for (int v = 0; v < 8; ++v) {
    const double s[3] = {(v & 1) ? 1.0 : -1.0, (v & 2) ? 1.0 : -1.0, (v & 4) ? 1.0 : -1.0};
    for (int b = 0; b < 3; ++b) {
      double f = s[b] / 8.0;
      for (int c = 0; c < 3; ++c)
        if (c != b) f *= 1.0 + xi[c] * s[c];
      dN[v * 3 + b] = f;
    }
  }
}

void face_point(int l, double s, double t, double xi[3]) {
  const int ax = l / 2;
  const int a0 = ax == 0 ? 1 : 0, a1 = ax == 2 ? 1 : 2;
  xi[ax] = (l & 1) ? 1.0 : -1.0;
  xi[a0] = s;
  xi[a1] = t;
}

}  // namespace

HexTables build_hex_tables(int k, int nquad) {
  HexTables T;
  T.k = k;
  T.n1 = k + 1;
  T.PE = T.n1 * T.n1 * T.n1;
  T.PF = T.n1 * T.n1;
  T.nq1 = nquad;
  T.nq = nquad * nquad * nquad;
  T.nfq = nquad * nquad;
  const std::vector<double> g = gll_nodes(k);
  std::vector<double> x, w;
  gauss_legendre(nquad, x, w);
  const int PE = T.PE, PF = T.PF, nq = T.nq, nfq = T.nfq, n = nquad;
  T.phiT.assign((size_t)PE * nq, 0.0);
  T.phi.assign((size_t)nq * PE, 0.0);
  T.dphi.assign((size_t)nq * PE * 3, 0.0);
  T.wq.assign(nq, 0.0);
  T.dN.assign((size_t)nq * 24, 0.0);
  for (int l = 0; l < n; ++l)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int q = (l * n + j) * n + i;
        const double xi[3] = {x[i], x[j], x[l]};
        hex_basis_at(g, xi, &T.phi[(size_t)q * PE], &T.dphi[(size_t)q * PE * 3]);
        T.wq[q] = w[i] * w[j] * w[l];
        trilinear_dN(xi, &T.dN[(size_t)q * 24]);
        for (int a = 0; a < PE; ++a) T.phiT[(size_t)a * nq + q] = T.phi[(size_t)q * PE + a];
      }
  // faces: phi at the face points (PE x 6 nfq, column l nfq + q), trilinear
  // derivatives there, face basis psi (nfq x PF) and face weights
  T.fphiT.assign((size_t)PE * 6 * nfq, 0.0);
  T.fphi.assign((size_t)6 * nfq * PE, 0.0);
  T.fdN.assign((size_t)6 * nfq * 24, 0.0);
  T.psi.assign((size_t)nfq * PF, 0.0);
  T.wf.assign(nfq, 0.0);
  std::vector<double> ps(T.n1), pt(T.n1), dum(T.n1);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const int q = j * n + i;
      T.wf[q] = w[i] * w[j];
      lagrange(g, x[i], ps.data(), dum.data());
      lagrange(g, x[j], pt.data(), dum.data());
      for (int b = 0; b < T.n1; ++b)
        for (int a = 0; a < T.n1; ++a) T.psi[(size_t)q * PF + b * T.n1 + a] = ps[a] * pt[b];
      for (int l = 0; l < 6; ++l) {
        double xi[3];
        face_point(l, x[i], x[j], xi);
        double* ph = &T.fphi[((size_t)l * nfq + q) * PE];
        hex_basis_at(g, xi, ph, nullptr);
        for (int a = 0; a < PE; ++a) T.fphiT[(size_t)a * 6 * nfq + l * nfq + q] = ph[a];
        trilinear_dN(xi, &T.fdN[((size_t)l * nfq + q) * 24]);
      }
    }
  T.b1.assign((size_t)n * T.n1, 0.0);
  T.d1.assign((size_t)n * T.n1, 0.0);
  for (int i = 0; i < n; ++i) lagrange(g, x[i], &T.b1[(size_t)i * T.n1], &T.d1[(size_t)i * T.n1]);
  return T;
}

int64_t hex_gen_scratch(const HexTables& T) {
  const int64_t PE = T.PE, PF = T.PF, nq = T.nq, nfq = T.nfq;
  return nq * PE            // AW: w |det J| phi
         + 3 * PE * nq      // GT: physical gradients, transposed
         + 6 * nfq * 4 * PF // BWN: w psi, w n_d psi per face
         + 6 * nfq * PE     // PW: w phi at face points
         + 6 * PF * nfq     // PsiT: permuted face basis, transposed
         + PE * PE          // Mf
         + 6 * PE * 4 * PF  // EF4: [EF | EFN_0 | EFN_1 | EFN_2] per face
         + 6 * PF * 4 * PF; // FF4: [FF | FFN_0 | FFN_1 | FFN_2] per face
}

namespace {

__device__ __forceinline__ void jac_at(const double* X8, const double* dN, double J[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int v = 0; v < 8; ++v) s += dN[v * 3 + b] * X8[v * 3 + a];
      J[a][b] = s;
    }
}

// adjugate (transpose of the cofactor matrix) and determinant of J
__device__ __forceinline__ double adj3(const double J[3][3], double A[3][3]) {
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
}

// One CTA per element: per volume point q the Jacobian, |det|, J^{-1};
// then AW[q][i] = w_q |det J_q| phi_i(x_q) and GT[d][i][q] = (grad phi_i)_d.
__global__ void hex_vol_geom_kernel(HexGenDesc d) {
  extern __shared__ double sm[];
  double* X8 = sm;                 // 24
  double* geo = sm + 24;           // nq x 10: wJ, Jinv (3 x 3, [b][a] = dxi_b/dx_a)
  const int64_t e = blockIdx.x;
  const int nq = d.nq, PE = d.PE;
  for (int i = threadIdx.x; i < 24; i += blockDim.x) X8[i] = d.verts[e * 24 + i];
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double J[3][3], A[3][3];
    jac_at(X8, d.dN + (int64_t)q * 24, J);
    const double det = adj3(J, A);
    if (!(det != 0.0) || !isfinite(det)) atomicOr(d.err, ERRBIT_SINGULAR);
    const double inv = 1.0 / det;
    double* gq = geo + q * 10;
    gq[0] = d.wq[q] * fabs(det);
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) gq[1 + b * 3 + a] = A[b][a] * inv;
  }
  __syncthreads();
  double* AW = d.AW + e * (int64_t)nq * PE;
  double* GT = d.GT + e * (int64_t)3 * PE * nq;
  for (int idx = threadIdx.x; idx < nq * PE; idx += blockDim.x) {
    const int q = idx / PE, i = idx - q * PE;
    const double* gq = geo + q * 10;
    AW[idx] = gq[0] * d.phi[idx];
    const double* dp = d.dphi + (int64_t)idx * 3;
    for (int a = 0; a < 3; ++a)
      GT[((int64_t)a * PE + i) * nq + q] = dp[0] * gq[1 + a] + dp[1] * gq[4 + a] + dp[2] * gq[7 + a];
  }
}

// Sum factorisation of M^e and B_d over the tensor-product rule, one CTA per
// element.  With phi_i = a_{i1}(x) a_{i2}(y) a_{i3}(z) (i = i1 + n1 (i2 + n1 i3))
// and the points q = q1 + m (q2 + m q3), a weight field W(q) gives (the
// intermediates stored with the pair (i1, j1) fastest, so that neighbouring
// threads touch neighbouring shared-memory words)
//   T1[i1,j1,q2,q3]     = sum_q1 X1[q1,i1] A[q1,j1] W[q1,q2,q3]
//   T2[i1,j1,i2,j2,q3]  = sum_q2 X2[q2,i2] A[q2,j2] T1[i1,j1,q2,q3]
//   O[i,j]              = sum_q3 X3[q3,i3] A[q3,j3] T2[i1,j1,i2,j2,q3]
// (X = A the values, or the derivatives D on one axis).  M^e takes W = w |det J|
// with X = A; B_c[i,j] = int (grad phi_i)_c phi_j sums, over the axis b of the
// derivative, the fields W_bc = w |det J| (J^{-1})_bc with D on axis b.
// The 1D products X[q,i] A[q,j] are tabulated once per CTA, so each term is
// one FP64 FMA (the same rounded product as computed in place).
constexpr int kSfN1 = 5, kSfNQ = 8;
template <int n1, int m>
__global__ void __launch_bounds__(256) hex_mass_grad_sf_kernel(HexGenDesc d, const double* b1g, const double* d1g,
                                                                double* Meo, double* Bdo) {
  extern __shared__ double sm[];
  constexpr int nq = m * m * m, PE = n1 * n1 * n1;
  constexpr int n2 = n1 * n1;
  double* X8 = sm;                          // 24
  double* b1 = X8 + 24;                     // m x n1
  double* d1 = b1 + m * n1;                 // m x n1
  double* Pb = d1 + m * n1;                 // m x n1 x n1: A[q,i] A[q,j]
  double* Pd = Pb + m * n2;                 // m x n1 x n1: D[q,i] A[q,j]
  double* geo = Pd + m * n2;                // nq x 10: w |det J| and w |det J| (J^{-1})_bc ([b][c])
  double* T1 = geo + nq * 10;               // 3 fields x m^2 x n2
  double* T2 = T1 + 3 * n2 * m * m;         // 3 fields x m x n2^2
  const int64_t e = blockIdx.x;
  for (int i = threadIdx.x; i < 24; i += blockDim.x) X8[i] = d.verts[e * 24 + i];
  for (int i = threadIdx.x; i < m * n1; i += blockDim.x) {
    b1[i] = b1g[i];
    d1[i] = d1g[i];
  }
  for (int t = threadIdx.x; t < m * n2; t += blockDim.x) {
    const int q = t / n2, i = (t / n1) % n1, j = t % n1;
    Pb[t] = b1g[q * n1 + i] * b1g[q * n1 + j];
    Pd[t] = d1g[q * n1 + i] * b1g[q * n1 + j];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double J[3][3], A[3][3];
    jac_at(X8, d.dN + (int64_t)q * 24, J);
    const double det = adj3(J, A);
    if (!(det != 0.0) || !isfinite(det)) atomicOr(d.err, ERRBIT_SINGULAR);
    const double wdet = d.wq[q] * fabs(det);
    const double winv = wdet / det;
    double* gq = geo + q * 10;
    gq[0] = wdet;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) gq[1 + b * 3 + c] = A[b][c] * winv;
  }
  __syncthreads();
  // pass 0: M^e (one field); passes 1..3: B_c (three fields, derivative axis b = 0, 1, 2)
  for (int pass = 0; pass < 4; ++pass) {
    const int nf = pass == 0 ? 1 : 3;
    const int c = pass - 1;
    // stage 1: T1[f][q3][q2][i1 j1] (i1 j1 fastest: consecutive lanes, consecutive words)
    for (int t = threadIdx.x; t < nf * n2 * m * m; t += blockDim.x) {
      const int ij1 = t % n2;
      const int r = t / n2;
      const int q2 = r % m, q3 = (r / m) % m, f = r / (m * m);
      const double* P = (pass > 0 && f == 0) ? Pd : Pb;
      const int wf = pass == 0 ? 0 : 1 + f * 3 + c;
      double acc = 0.0;
#pragma unroll
      for (int q1 = 0; q1 < m; ++q1) acc += P[q1 * n2 + ij1] * geo[((q3 * m + q2) * m + q1) * 10 + wf];
      T1[t] = acc;
    }
    __syncthreads();
    // stage 2: T2[f][q3][i2 j2][i1 j1]
    for (int t = threadIdx.x; t < nf * n2 * n2 * m; t += blockDim.x) {
      const int ij1 = t % n2;
      const int r = t / n2;
      const int ij2 = r % n2, q3 = (r / n2) % m, f = r / (n2 * m);
      const double* P = (pass > 0 && f == 1) ? Pd : Pb;
      const double* t1 = T1 + (f * m + q3) * m * n2 + ij1;
      double acc = 0.0;
#pragma unroll
      for (int q2 = 0; q2 < m; ++q2) acc += P[q2 * n2 + ij2] * t1[q2 * n2];
      T2[t] = acc;
    }
    __syncthreads();
    // stage 3: O[i, j], summed over the fields
    double* out = pass == 0 ? Meo + e * (int64_t)PE * PE : Bdo + (e * 3 + c) * (int64_t)PE * PE;
    for (int t = threadIdx.x; t < PE * PE; t += blockDim.x) {
      const int i = t / PE, j = t - i * PE;
      const int i3 = i / n2, i2 = (i / n1) % n1, i1 = i % n1;
      const int j3 = j / n2, j2 = (j / n1) % n1, j1 = j % n1;
      const int ij1 = i1 * n1 + j1, ij2 = i2 * n1 + j2;
      double acc = 0.0;
      const int ij3 = i3 * n1 + j3;
      for (int f = 0; f < nf; ++f) {
        const double* P = (pass > 0 && f == 2) ? Pd : Pb;
        const double* t2 = T2 + (f * m * n2 + ij2) * n2 + ij1;
#pragma unroll
        for (int q3 = 0; q3 < m; ++q3) acc += P[q3 * n2 + ij3] * t2[q3 * n2 * n2];
      }
      out[t] = acc;
    }
    __syncthreads();
  }
}

size_t sf_smem(int n1, int m) {
  const int n2 = n1 * n1;
  return sizeof(double) * (24 + 2 * (size_t)m * n1 + 2 * (size_t)m * n2 + (size_t)m * m * m * 10 +
                           3 * (size_t)n2 * m * m +
                           3 * (size_t)n2 * n2 * m);
}

// One CTA per element: per face point the cofactor normal nv = adj(J)^T e_l,
// dA = |nv|, n = nv / dA, w = w_q dA; then the weighted face tables.
__global__ void hex_face_geom_kernel(HexGenDesc d) {
  extern __shared__ double sm[];
  double* X8 = sm;                 // 24
  double* geo = sm + 24;           // 6 nfq x 4: w, n
  const int64_t e = blockIdx.x;
  const int nfq = d.nfq, PE = d.PE, PF = d.PF, F4 = 4 * PF;
  for (int i = threadIdx.x; i < 24; i += blockDim.x) X8[i] = d.verts[e * 24 + i];
  __syncthreads();
  for (int lq = threadIdx.x; lq < 6 * nfq; lq += blockDim.x) {
    const int l = lq / nfq, q = lq - l * nfq;
    double J[3][3], A[3][3];
    jac_at(X8, d.fdN + (int64_t)lq * 24, J);
    adj3(J, A);
    const int ax = l / 2;
    const double sgn = (l & 1) ? 1.0 : -1.0;
    double nv[3];
    for (int a = 0; a < 3; ++a) nv[a] = sgn * A[ax][a];
    const double dA = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    if (!(dA > 0.0) || !isfinite(dA)) atomicOr(d.err, ERRBIT_SINGULAR);
    double* gq = geo + lq * 4;
    gq[0] = d.wf[q] * dA;
    for (int a = 0; a < 3; ++a) gq[1 + a] = nv[a] / dA;
  }
  __syncthreads();
  const int32_t* perm = d.perm + e * (int64_t)6 * PF;
  double* BWN = d.BWN + e * (int64_t)6 * nfq * F4;
  double* PW = d.PW + e * (int64_t)6 * nfq * PE;
  double* PsiT = d.PsiT + e * (int64_t)6 * PF * nfq;
  for (int idx = threadIdx.x; idx < 6 * nfq * PF; idx += blockDim.x) {
    const int lq = idx / PF, j = idx - lq * PF;
    const int l = lq / nfq, q = lq - l * nfq;
    const int pj = perm[l * PF + j];
    const double ps = (pj >= 0 && pj < PF) ? d.psi[(int64_t)q * PF + pj] : 0.0;
    if (pj < 0 || pj >= PF) atomicOr(d.err, ERRBIT_ARG);
    const double* gq = geo + lq * 4;
    double* row = BWN + (int64_t)lq * F4;
    row[j] = gq[0] * ps;
    row[PF + j] = gq[0] * gq[1] * ps;
    row[2 * PF + j] = gq[0] * gq[2] * ps;
    row[3 * PF + j] = gq[0] * gq[3] * ps;
    PsiT[((int64_t)l * PF + j) * nfq + q] = ps;
  }
  for (int idx = threadIdx.x; idx < 6 * nfq * PE; idx += blockDim.x) {
    const int lq = idx / PE;
    PW[idx] = geo[lq * 4] * d.fphi[idx];
  }
}

// The blocks of Eq. matrixform from the element integrals and the physics
// tensors, written in the row-major per-element layout of the condensation
// inputs:
//   Cd[d][i][l PF + j]   = -EFN[l,d][i,j]
//   D[(a,i),(b,c,k)]     = sum_d Cq[a,d,b,c] Sd[d][k][i]
//   E[(a,i),(b,j)]       = -sum_d Cu[a,d,b] Sd[d][i][j] + tau d_ab Mf[i][j] + Rr[a,b] Me[i][j]
//   F[(a,i),(l,b,j)]     = sum_d Cu[a,d,b] EFN[l,d][i,j] - tau d_ab EF[l][i,j]
//   G[(l,a,j),(b,c,k)]   = sum_d Cq[a,d,b,c] EFN[l,d][k,j]
//   H[(l,a,j),(b,k)]     = tau d_ab EF[l][k,j]
//   J[(l,a,j),(l',b,k)]  = d_ll' (sum_d Cu[a,d,b] FFN[l,d][k,j] - tau d_ab FF[l][k,j])
// EF4 holds EF[l] and EFN[l,d] side by side per row (l, i): columns j, PF + j,
// 2 PF + j, 3 PF + j; FF4 likewise per row (l, k).
// One CTA per element (grid-stride), one warp per output row: the row's
// indices are decoded once per warp, the columns' once per CTA into a
// shared table (two ints per column).  When they fit (kExpandStageMax), the
// element's tables that the block needs are first copied into shared memory
// with odd row strides (EF4/FF4 rows of 4 PF + 1, Sd rows of P_E + 1 for
// even sizes), so that the gathers along the columns are free of bank
// conflicts and no load waits behind a global store.
constexpr int kExpandStageMax = 96 * 1024;

// The nonzero terms of a physics coefficient over d for one (a, column
// group): isotropic elasticity has at most one of the three Cq[a,d,b,c]
// nonzero and Cu = 0, so most FP64 FMAs of the blocks can go.  The kept
// terms run in increasing d, and a skipped term has an exact zero
// coefficient, so the sums are the same as over all three.
struct NzTerms {
  double c[3];
  int n;    // kept terms
  int dd;   // their d, 2 bits each
};
__host__ __device__ inline int expand_groups(int which, int M) {
  return (which == 1 || which == 4) ? 3 * M * M : (which == 2 || which == 3 || which == 6) ? M * M : 0;
}

__host__ __device__ inline int odd_up(int n) { return n | 1; }

// doubles of the staged tables of block WHICH
__host__ __device__ inline int expand_stage_doubles(int which, int M, int PE, int PF) {
  const int fs = odd_up(4 * PF);
  switch (which) {
    case 1: return 3 * PE * odd_up(PE);
    case 2: return 3 * PE * odd_up(PE) + 2 * PE * PE;
    case 6: return 6 * PF * fs;
    default: return 6 * PE * fs;
  }
}

template <int WHICH>
__global__ void __launch_bounds__(256) hex_expand_kernel(HexGenDesc d, int staged) {
  extern __shared__ double smx[];
  const int M = d.M, PE = d.PE, PF = d.PF, F4 = 4 * PF;
  const int MPE = M * PE, MDPE = 3 * MPE, nlb = 6 * M * PF;
  int nrows, ncols;
  double* out;
  switch (WHICH) {
    case 0: nrows = 3 * PE; ncols = 6 * PF; out = d.Cd; break;
    case 1: nrows = MPE; ncols = MDPE; out = d.Dm; break;
    case 2: nrows = MPE; ncols = MPE; out = d.Em; break;
    case 3: nrows = MPE; ncols = nlb; out = d.Fm; break;
    case 4: nrows = nlb; ncols = MDPE; out = d.Gm; break;
    case 5: nrows = nlb; ncols = MPE; out = d.Hm; break;
    default: nrows = nlb; ncols = nlb; out = d.Jm; break;
  }
  int2* ctab = reinterpret_cast<int2*>(smx);
  const int ngr = expand_groups(WHICH, M);
  NzTerms* nz = reinterpret_cast<NzTerms*>(smx + ncols);
  double* stg = smx + ncols + 4 * ngr;       // staged tables after the column and term tables
  for (int g = threadIdx.x; g < ngr; g += blockDim.x) {
    NzTerms z;
    z.n = 0;
    z.dd = 0;
    for (int dd = 0; dd < 3; ++dd) {
      double c;
      if (WHICH == 1 || WHICH == 4) {        // g = a 3M + (b c): Cq[a][d][b c]
        const int a = g / (3 * M), bc = g - a * 3 * M;
        c = d.Cq[a * 9 * M + dd * 3 * M + bc];
      } else {                               // g = a M + b: Cu[a][d][b]
        const int a = g / M, b = g - a * M;
        c = d.Cu[(a * 3 + dd) * M + b];
      }
      if (c != 0.0) {
        z.c[z.n] = c;
        z.dd |= dd << (2 * z.n);
        ++z.n;
      }
    }
    for (int q = z.n; q < 3; ++q) z.c[q] = 0.0;
    nz[g] = z;
  }
  const int fs = staged ? odd_up(F4) : F4;   // row stride of EF4 / FF4
  const int ss = staged ? odd_up(PE) : PE;   // row stride of Sd
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    int2 t;
    if (WHICH == 0) {                     // (l, j): offset of EFN[l,.][., j]
      const int l = c / PF, j = c - l * PF;
      t = make_int2(l * PE * fs + j, 0);
    } else if (WHICH == 1 || WHICH == 4) {   // (b c, k)
      const int bc = c / PE, k = c - bc * PE;
      t = make_int2(bc, WHICH == 1 ? k * ss : k * fs);
    } else if (WHICH == 2 || WHICH == 5) {   // (b, k)
      const int b = c / PE, k = c - b * PE;
      t = make_int2(b, WHICH == 2 ? k : k * fs);
    } else {                              // (l, b, j): l 256 + b and the table offset
      const int lb = c / PF, j = c - lb * PF;
      const int l = lb / M, b = lb - l * M;
      t = make_int2((l << 8) | b, WHICH == 3 ? l * PE * fs + j : j * fs);
    }
    ctab[c] = t;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t per = (int64_t)nrows * ncols;
  const double tau = d.tau;
  for (int64_t e = blockIdx.x; e < d.count; e += gridDim.x) {
    const double* Me = d.Me + e * (int64_t)PE * PE;
    const double* Sd = d.Sd + e * (int64_t)3 * PE * PE;
    const double* Mf = d.Mf + e * (int64_t)PE * PE;
    const double* EF4 = d.EF4 + e * (int64_t)6 * PE * F4;
    const double* FF4 = d.FF4 + e * (int64_t)6 * PF * F4;
    if (staged) {
      __syncthreads();                       // the previous element's reads are done
      if (WHICH == 1 || WHICH == 2) {
        for (int x = threadIdx.x; x < 3 * PE * PE; x += blockDim.x) {
          const int r = x / PE;
          stg[r * ss + (x - r * PE)] = Sd[x];
        }
        if (WHICH == 2) {
          double* sme = stg + 3 * PE * ss;
          for (int x = threadIdx.x; x < PE * PE; x += blockDim.x) {
            sme[x] = Me[x];
            sme[PE * PE + x] = Mf[x];
          }
          Me = sme;
          Mf = sme + PE * PE;
        }
        Sd = stg;
      } else {
        const double* src = (WHICH == 6) ? FF4 : EF4;
        const int rows = (WHICH == 6) ? 6 * PF : 6 * PE;
        for (int x = threadIdx.x; x < rows * F4; x += blockDim.x) {
          const int r = x / F4;
          stg[r * fs + (x - r * F4)] = src[x];
        }
        if (WHICH == 6) FF4 = stg; else EF4 = stg;
      }
    }
    __syncthreads();                         // tables (and, first, the column table) ready
    double* oe = out + e * per;
    for (int r = warp; r < nrows; r += nw) {
      double* orow = oe + (int64_t)r * ncols;
      if (WHICH == 0) {
        const int dd = r / PE, i = r - dd * PE;
        const double* src = EF4 + i * fs + (1 + dd) * PF;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) orow[c] = -src[ctab[c].x];
      } else if (WHICH == 1) {
        const int a = r / PE, i = r - a * PE;
        const NzTerms* za = nz + a * 3 * M;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          const NzTerms& z = za[t.x];
          double v = 0.0;
          for (int q = 0; q < z.n; ++q) v += z.c[q] * Sd[((z.dd >> (2 * q)) & 3) * PE * ss + t.y + i];
          orow[c] = v;
        }
      } else if (WHICH == 2) {
        const int a = r / PE, i = r - a * PE;
        const NzTerms* za = nz + a * M;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          const int b = t.x, j = t.y;
          const NzTerms& z = za[b];
          double v = 0.0;
          for (int q = 0; q < z.n; ++q) v -= z.c[q] * Sd[(((z.dd >> (2 * q)) & 3) * PE + i) * ss + j];
          if (a == b) v += tau * Mf[i * PE + j];
          const double rr = d.Rr[a * M + b];
          if (rr != 0.0) v += rr * Me[i * PE + j];
          orow[c] = v;
        }
      } else if (WHICH == 3) {
        const int a = r / PE, i = r - a * PE;
        const NzTerms* za = nz + a * M;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          const int b = t.x & 255;
          const NzTerms& z = za[b];
          const double* ef = EF4 + t.y + i * fs;
          double v = 0.0;
          for (int q = 0; q < z.n; ++q) v += z.c[q] * ef[(1 + ((z.dd >> (2 * q)) & 3)) * PF];
          if (a == b) v -= tau * ef[0];
          orow[c] = v;
        }
      } else if (WHICH == 4) {
        const int la = r / PF, j = r - la * PF;
        const int l = la / M, a = la - l * M;
        const NzTerms* za = nz + a * 3 * M;
        const double* ef = EF4 + l * PE * fs + j;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          const NzTerms& z = za[t.x];
          double v = 0.0;
          for (int q = 0; q < z.n; ++q) v += z.c[q] * ef[t.y + (1 + ((z.dd >> (2 * q)) & 3)) * PF];
          orow[c] = v;
        }
      } else if (WHICH == 5) {
        const int la = r / PF, j = r - la * PF;
        const int l = la / M, a = la - l * M;
        const double* ef = EF4 + l * PE * fs + j;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          orow[c] = (t.x == a) ? tau * ef[t.y] : 0.0;
        }
      } else {
        const int la = r / PF, j = r - la * PF;
        const int l = la / M, a = la - l * M;
        const NzTerms* za = nz + a * M;
        const double* ff = FF4 + l * PF * fs + j;
#pragma unroll 4
        for (int c = lane; c < ncols; c += 32) {
          const int2 t = ctab[c];
          const int l2 = t.x >> 8, b = t.x & 255;
          double v = 0.0;
          if (l2 == l) {
            const NzTerms& z = za[b];
            const double* f = ff + t.y;
            for (int q = 0; q < z.n; ++q) v += z.c[q] * f[(1 + ((z.dd >> (2 * q)) & 3)) * PF];
            if (a == b) v -= tau * f[0];
          }
          orow[c] = v;
        }
      }
    }
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int W>
void launch_expand(const HexGenDesc& d, cudaStream_t s) {
  const int MPE = d.M * d.PE, nlb = 6 * d.M * d.PF;
  const int ncols = (W == 0) ? 6 * d.PF : (W == 1 || W == 4) ? 3 * MPE : (W == 2 || W == 5) ? MPE : nlb;
  const size_t tab = sizeof(int2) * (size_t)ncols + sizeof(NzTerms) * (size_t)expand_groups(W, d.M);
  const size_t stage = sizeof(double) * (size_t)expand_stage_doubles(W, d.M, d.PE, d.PF);
  const int staged = (tab + stage <= (size_t)kExpandStageMax) ? 1 : 0;
  const size_t smem = tab + (staged ? stage : 0);
  if (smem > 48 * 1024) cudaFuncSetAttribute(hex_expand_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t grid = std::min<int64_t>(d.count, (int64_t)sm_count() * 8);
  count_launch();
  hex_expand_kernel<W><<<(unsigned)grid, 256, smem, s>>>(d, staged);
}

}  // namespace

void hex_geometry(const HexGenDesc& d, cudaStream_t s) {
  if (d.count <= 0) return;
  const size_t sv = sizeof(double) * (24 + (size_t)d.nq * 10);
  cudaFuncSetAttribute(hex_vol_geom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  count_launch();
  hex_vol_geom_kernel<<<(unsigned)d.count, 256, sv, s>>>(d);
  hex_face_geometry(d, s);
}

void hex_face_geometry(const HexGenDesc& d, cudaStream_t s) {
  if (d.count <= 0) return;
  const size_t sf = sizeof(double) * (24 + (size_t)6 * d.nfq * 4);
  cudaFuncSetAttribute(hex_face_geom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  count_launch();
  hex_face_geom_kernel<<<(unsigned)d.count, 256, sf, s>>>(d);
}

template <int n1, int m>
void launch_sf(const HexGenDesc& d, const double* b1, const double* d1, double* Me, double* Bd, size_t smem,
               cudaStream_t s) {
  cudaFuncSetAttribute(hex_mass_grad_sf_kernel<n1, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  count_launch();
  hex_mass_grad_sf_kernel<n1, m><<<(unsigned)d.count, 256, smem, s>>>(d, b1, d1, Me, Bd);
}

template <int n1>
bool launch_sf_m(const HexGenDesc& d, int m, const double* b1, const double* d1, double* Me, double* Bd, size_t smem,
                 cudaStream_t s) {
  switch (m) {
    case 2: launch_sf<n1, 2>(d, b1, d1, Me, Bd, smem, s); return true;
    case 3: launch_sf<n1, 3>(d, b1, d1, Me, Bd, smem, s); return true;
    case 4: launch_sf<n1, 4>(d, b1, d1, Me, Bd, smem, s); return true;
    case 5: launch_sf<n1, 5>(d, b1, d1, Me, Bd, smem, s); return true;
    case 6: launch_sf<n1, 6>(d, b1, d1, Me, Bd, smem, s); return true;
    case 7: launch_sf<n1, 7>(d, b1, d1, Me, Bd, smem, s); return true;
    case 8: launch_sf<n1, 8>(d, b1, d1, Me, Bd, smem, s); return true;
    default: return false;
  }
}

bool hex_mass_grad_sf(const HexGenDesc& d, int n1, int nq1, const double* b1, const double* d1, double* Me,
                      double* Bd, cudaStream_t s) {
  if (n1 < 2 || n1 > kSfN1 || nq1 < 2 || nq1 > kSfNQ) return false;
  if (d.count <= 0) return true;
  const size_t smem = sf_smem(n1, nq1);
  if (smem > 200 * 1024) return false;
  switch (n1) {
    case 2: return launch_sf_m<2>(d, nq1, b1, d1, Me, Bd, smem, s);
    case 3: return launch_sf_m<3>(d, nq1, b1, d1, Me, Bd, smem, s);
    case 4: return launch_sf_m<4>(d, nq1, b1, d1, Me, Bd, smem, s);
    default: return launch_sf_m<5>(d, nq1, b1, d1, Me, Bd, smem, s);
  }
}

void hex_expand(const HexGenDesc& d, cudaStream_t s) {
  if (d.count <= 0) return;
  launch_expand<0>(d, s);
  launch_expand<1>(d, s);
  launch_expand<2>(d, s);
  launch_expand<3>(d, s);
  launch_expand<4>(d, s);
  launch_expand<5>(d, s);
  launch_expand<6>(d, s);
}

}  // namespace hdg
