// C ABI of the HDG trace-solver library: problem state, host-side mesh maps,
// and the orchestration of the device kernels (condensation, assembly,
// preconditioner setup, GMRES, recovery).  Every numerical step runs in the
// library's CUDA kernels; the host only sequences launches and reads small
// status words at synchronisation points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "hdg_common.cuh"
#include "hdg_gmres.h"
#include "hdg_internal.h"

using namespace hdg;

#include <atomic>
#include <map>
#include <mutex>
namespace hdg {
static std::atomic<long long> g_launches{0};
// While this thread captures a stream into a graph, its launches are counted
// here instead of in the process-wide count (captured kernels are counted
// when the graph runs); other threads' launches are unaffected.
static thread_local bool t_capturing = false;
static thread_local long long t_captured = 0;
void count_launch() {
  if (t_capturing) ++t_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
}  // namespace hdg

namespace {

struct CudaError {
  cudaError_t e;
};

// last CUDA failure seen by a library call on this host thread
thread_local char g_last_error[256] = "";

void note_error(cudaError_t e, const char* what, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at %s:%d", cudaGetErrorString(e), cudaGetErrorName(e), what,
           line);
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) {                   \
      note_error(_e, #x, __LINE__);            \
      throw CudaError{_e};                     \
    }                                          \
  } while (0)

template <typename T>
int64_t padded_stride(int64_t elems) {
  int64_t bytes = elems * (int64_t)sizeof(T);
  bytes = (bytes + 15) / 16 * 16;
  return bytes / (int64_t)sizeof(T);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct hdg_problem_s {
  int device = 0;
  int dim = 0, nl = 0, M = 0, PE = 0, PF = 0, D = 0, R = 1, b = 0, nlb = 0, ms = 0, nlPF = 0, MPE = 0, MDPE = 0;
  int64_t NE = 0, NF = 0, nfree = 0, ndof = 0;
  std::vector<int32_t> h_elem_face, h_face_elem, h_free_of_face, h_nbr;
  std::vector<int64_t> h_rowptr;
  int64_t nnzb = 0, asm_nblk = 0;
  std::vector<uint8_t> h_face_dir;
  std::vector<uint8_t> condensed;
  int64_t n_condensed = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;

  // device tables
  int32_t *d_elem_face = nullptr, *d_free_of_face = nullptr;
  uint8_t* d_face_dir = nullptr;
  int32_t *d_nbr = nullptr, *d_cnt = nullptr, *d_slot_e = nullptr, *d_slot_lr = nullptr, *d_slot_lc = nullptr;
  int32_t *d_diag2 = nullptr, *d_rhs_src = nullptr, *d_bj_nbr = nullptr, *d_bj_cnt = nullptr;
  int32_t *d_asm_lf = nullptr, *d_asm_cnt = nullptr, *d_asm_face_free = nullptr, *d_fsum = nullptr;
  int64_t *d_rowptr = nullptr, *d_bj_rowptr = nullptr, *d_asm_rowptr = nullptr;

  // condensation results
  double *d_Kbar = nullptr, *d_rbar = nullptr, *d_MinvB = nullptr, *d_MinvC = nullptr, *d_XF = nullptr,
         *d_Xr = nullptr;
  double* d_uhatD = nullptr;
  // staging / temporaries for condensation
  int64_t chunk = 0;
  int64_t chunk_cap = 0;          // elements the staging and temporaries hold
  double* d_stage = nullptr;
  // second staging buffer, copy stream and events: host blocks of chunk c+1
  // are copied while chunk c is condensed
  double* d_stage2 = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_freed[2] = {nullptr, nullptr}, ev_start = nullptr;
  cudaEvent_t ev_read = nullptr;   // after the last copy from caller memory of a host-input call
  cudaEvent_t ev_uD_used = nullptr;    // after the last stream operation on d_uhatD
  cudaEvent_t ev_uD_copied = nullptr;  // after a host copy into d_uhatD on the copy stream
  cudaEvent_t ev_rec = nullptr;        // recovery pieces handed to the copy stream
  double* d_tmp = nullptr;

  // assembled system
  double* K64 = nullptr;
  float* K32 = nullptr;
  __nv_bfloat16* K16 = nullptr;
  int64_t s64 = 0, s32 = 0, s16 = 0;
  int ld32 = 0, ld16 = 0;          // leading dimensions of the FP32 / BF16 face blocks (K and BJ)
  double* d_r = nullptr;
  bool assembled = false;

  // preconditioners
  double* bj64 = nullptr;
  float* bj32 = nullptr;
  __nv_bfloat16* bj16 = nullptr;
  int64_t bs64 = 0, bs32 = 0, bs16 = 0;
  double* as64 = nullptr;
  float* as32 = nullptr;
  __nv_bfloat16* as16 = nullptr;
  int64_t as_s64 = 0, as_s32 = 0, as_s16 = 0;
  int as_ld32 = 0, as_ld16 = 0;
  int pc_ready = -1;  // which base preconditioner is set up
  int poly_kind = 0, poly_n = 0;
  std::vector<double> th_re, th_im;
  double* d_poly = nullptr;
  double cheb_a = 0.0, cheb_b = 0.0;

  // buffers reused across calls (no per-call cudaMalloc / cudaFree, which
  // would synchronise the device and serialise concurrent problems)
  double *d_full = nullptr, *d_uout = nullptr, *d_qout = nullptr, *d_bjtmp = nullptr, *d_asmP = nullptr;

  // solve workspace
  double* d_x = nullptr;
  int ws_m = -1;
  double *V = nullptr, *vscale = nullptr, *H = nullptr, *g = nullptr, *cs = nullptr, *sn = nullptr, *hcol = nullptr,
         *htmp = nullptr, *ycoef = nullptr, *partial = nullptr, *tolabs = nullptr, *cfac = nullptr, *zb = nullptr,
         *bnorm = nullptr, *rel = nullptr;
  int *running = nullptr, *jend = nullptr, *on_estimate = nullptr, *done = nullptr, *iters = nullptr;
  unsigned* counter = nullptr;
  int* dmaxit = nullptr;           // iteration cap read by the Givens step (cycle graphs replay it)
  int* bdone = nullptr;            // "this system is finished" flag of the batched solve
  unsigned* d_err = nullptr;
  float* x32 = nullptr;
  // FP32 work vectors of the low-precision preconditioner (allocated on first use):
  // polynomial state (lp0, lp1, lp2), K products (ks32), the FP32 copy of the
  // GMRES iteration's K v_j (t1_32), ASM element results (ze32)
  float *lp0 = nullptr, *lp1 = nullptr, *lp2 = nullptr, *ks32 = nullptr, *t1_32 = nullptr, *ze32 = nullptr;
  // K as exact digits for the FP64 products on the tensor cores (R = 4, 8; built by hdg_assemble)
  unsigned char* kdig = nullptr;
  int64_t* d_kdoff = nullptr;
  int32_t* kex = nullptr;
  bool kdig_ready = false;
  double *t1 = nullptr, *res = nullptr, *pq = nullptr, *pw = nullptr, *ptmp = nullptr, *pAq = nullptr,
         *pt = nullptr, *ze = nullptr, *xo = nullptr, *bo = nullptr;
  // pinned host mirrors
  int* h_flag = nullptr;      // host-mapped progress flags of the current cycle
  int* d_flag = nullptr;      // device alias of h_flag
  std::vector<cudaEvent_t> ev_iter;
  double* h_dbl = nullptr;
  int* h_int = nullptr;
  unsigned* h_err = nullptr;

  // captured GMRES cycles (CUDA graphs with one IF node per iteration)
  struct CycleGraph {
    unsigned long long key = 0;
    unsigned poly_gen = 0;         // polynomial coefficients captured by value
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphConditionalHandle> h;
    long long kernels_per_iter = 0;
  };
  std::vector<CycleGraph> graphs;
  bool use_graphs = true;
  unsigned poly_gen = 0;           // bumped by every polynomial set-up
  cudaStream_t cap_stream = nullptr;

  // timing of block-matvec launches
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  // [0..2] matvec per precision, [3] tensor-core GEMMs, [4..5] block-Jacobi
  // applies of the low-precision polynomial with FP32 / BF16 blocks
  double t_mv_ms[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int64_t n_mv[6] = {0, 0, 0, 0, 0, 0};
  std::vector<int> ev_prec;
  int br_variant = 0;              // 1: bulk-copy staging for every block-row product
  int condense_mode = 1;           // condensation GEMMs: 1 tensor cores (digits split per tile), 2 digit
                                   // planes in device memory, 3 persistent CTAs, 0 FP64 cores
  uint16_t* d_oz = nullptr;        // row / column exponents of the tensor-core products
  int64_t oz_cap = 0;
  unsigned char* d_planes = nullptr;   // digit planes of the operands (grown on demand)
  int64_t planes_cap = 0;
  uint16_t* d_pex = nullptr;
  int64_t pex_cap = 0;
  double* d_invs = nullptr;        // scratch of the block inverses of matrices beyond one CTA's shared memory
  int64_t invs_cap = 0;            // (doubles, grown on demand)
  // element-matrix generation of hexahedra: device tables for (hex_k, hex_nq), scratch, inputs
  int hex_k = -1, hex_nq = -1;
  HexTables hex_tab;
  double* d_hextab = nullptr;
  int64_t hextab_cap = 0;
  double* d_gen = nullptr;
  int64_t gen_cap = 0;
  unsigned char* d_genin = nullptr;
  int64_t genin_cap = 0;
  unsigned char* d_hexin[2] = {nullptr, nullptr};   // host inputs of hdg_condense_hex, double-buffered
  int64_t hexin_cap[2] = {0, 0};
  double* d_phys = nullptr;
  int hex_sf = 1;                  // M^e, B_d of generated blocks by sum factorisation (0: dense products)
  // autotuned launch configurations [operation: K, BJ, ASM][precision]
  BrCfg tune[3][3];
  float tune_us[3][3] = {};        // measured time of the chosen configuration
  float tune_us0[3][3] = {};       // measured time of the heuristic default
  unsigned tune_gen = 0;           // changes the cycle-graph key when a tuning changes

  void* dalloc(size_t nbytes) {
    if (nbytes == 0) nbytes = 16;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    allocs.push_back(q);
    bytes += nbytes;
    return q;
  }
  void dfree(void* q, size_t nbytes) {
    if (!q) return;
    auto it = std::find(allocs.begin(), allocs.end(), q);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(q);
    bytes -= std::min(bytes, nbytes);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* q = (T*)dalloc(v.size() * sizeof(T));
    CK(cudaMemcpy(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return q;
  }
};

namespace {

hdg_status to_status(const CudaError& e) {
  (void)e;
  return HDG_ERR_CUDA;
}

// Reads and clears the device error word.
hdg_status check_err(hdg_problem p, cudaStream_t s) {
  CK(cudaMemcpyAsync(p->h_err, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  unsigned e = *p->h_err;
  if (e) {
    CK(cudaMemsetAsync(p->d_err, 0, sizeof(unsigned), s));
    if (e & ERRBIT_TIMEOUT) return HDG_ERR_TIMEOUT;
    if (e & ERRBIT_SINGULAR) return HDG_ERR_SINGULAR;
    if (e & ERRBIT_NAN) return HDG_ERR_NAN;
    if (e & ERRBIT_ARG) return HDG_ERR_ARG;
  }
  return HDG_OK;
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != prev) cudaSetDevice(prev);
  }
};

// ------------------------------------------------------------------ mesh maps
// Face rows (Sec. 2.4, Sec. 4.2): slot 0 is the face itself; then the other
// free faces of e1 in local order, then those of e2.  Dirichlet faces are
// eliminated, so rows near the boundary hold fewer than 2N_lfe-1 blocks;
// the real slots are packed first.
hdg_status build_maps(hdg_problem p) {
  const int nl = p->nl;
  p->h_free_of_face.assign(p->NF, -1);
  int64_t nf = 0;
  for (int64_t f = 0; f < p->NF; ++f)
    if (!p->h_face_dir[f]) p->h_free_of_face[f] = (int32_t)nf++;
  p->nfree = nf;
  p->ndof = nf * p->b;
  const int ms = p->ms;
  std::vector<int32_t> nbr(nf * ms, -1), cnt(nf, 0), se(nf * ms, -1), slr(nf * ms, 0), slc(nf * ms, 0),
      diag2(nf * 2, -1), rsrc(nf * 4, -1);
  for (int64_t f = 0; f < p->NF; ++f) {
    const int32_t ff = p->h_free_of_face[f];
    if (ff < 0) continue;
    const int32_t e1 = p->h_face_elem[f * 4], l1 = p->h_face_elem[f * 4 + 1];
    const int32_t e2 = p->h_face_elem[f * 4 + 2], l2 = p->h_face_elem[f * 4 + 3];
    if (e1 < 0 || e1 >= p->NE || l1 < 0 || l1 >= nl) return HDG_ERR_ARG;
    if (e2 >= p->NE || (e2 >= 0 && (l2 < 0 || l2 >= nl))) return HDG_ERR_ARG;
    if (p->h_elem_face[(int64_t)e1 * nl + l1] != f) return HDG_ERR_ARG;
    if (e2 >= 0 && p->h_elem_face[(int64_t)e2 * nl + l2] != f) return HDG_ERR_ARG;
    int c = 0;
    auto add = [&](int32_t e, int32_t lr, int32_t lc, int32_t g) {
      nbr[ff * ms + c] = g;
      se[ff * ms + c] = e;
      slr[ff * ms + c] = lr;
      slc[ff * ms + c] = lc;
      ++c;
    };
    add(e1, l1, l1, ff);
    diag2[ff * 2] = e2;
    diag2[ff * 2 + 1] = l2;
    for (int l = 0; l < nl; ++l) {
      if (l == l1) continue;
      int32_t g = p->h_elem_face[(int64_t)e1 * nl + l];
      if (g < 0 || g >= p->NF) return HDG_ERR_ARG;
      if (p->h_free_of_face[g] >= 0) add(e1, l1, l, p->h_free_of_face[g]);
    }
    if (e2 >= 0) {
      for (int l = 0; l < nl; ++l) {
        if (l == l2) continue;
        int32_t g = p->h_elem_face[(int64_t)e2 * nl + l];
        if (g < 0 || g >= p->NF) return HDG_ERR_ARG;
        if (p->h_free_of_face[g] >= 0) add(e2, l2, l, p->h_free_of_face[g]);
      }
    }
    cnt[ff] = c;
    rsrc[ff * 4] = e1;
    rsrc[ff * 4 + 1] = l1;
    rsrc[ff * 4 + 2] = e2;
    rsrc[ff * 4 + 3] = l2;
  }
  // ASM: per element, its free local faces (compacted); per free face the
  // positions inside both elements.
  std::vector<int32_t> alf(p->NE * nl, 0), acnt(p->NE, 0), aff(p->NE * nl, 0), fsum(nf * 4, -1);
  std::vector<int32_t> pos(p->NE * nl, -1);
  for (int64_t e = 0; e < p->NE; ++e) {
    int c = 0;
    for (int l = 0; l < nl; ++l) {
      int32_t g = p->h_elem_face[e * nl + l];
      if (g < 0 || g >= p->NF) return HDG_ERR_ARG;
      int32_t ff = p->h_free_of_face[g];
      if (ff >= 0) {
        alf[e * nl + c] = l;
        aff[e * nl + c] = ff;
        pos[e * nl + l] = c;
        ++c;
      }
    }
    for (int s = c; s < nl; ++s) aff[e * nl + s] = 0;
    acnt[e] = c;
  }
  for (int64_t f = 0; f < p->NF; ++f) {
    const int32_t ff = p->h_free_of_face[f];
    if (ff < 0) continue;
    const int32_t e1 = p->h_face_elem[f * 4], l1 = p->h_face_elem[f * 4 + 1];
    const int32_t e2 = p->h_face_elem[f * 4 + 2], l2 = p->h_face_elem[f * 4 + 3];
    fsum[ff * 4] = e1;
    fsum[ff * 4 + 1] = pos[(int64_t)e1 * nl + l1];
    if (e2 >= 0) {
      fsum[ff * 4 + 2] = e2;
      fsum[ff * 4 + 3] = pos[(int64_t)e2 * nl + l2];
    }
  }
  std::vector<int32_t> bjn(nf), bjc(nf, 1);
  for (int64_t f = 0; f < nf; ++f) bjn[f] = (int32_t)f;
  // compact block offsets of the face rows, the BJ blocks and the ASM panels
  std::vector<int64_t> rp(nf + 1, 0), bjrp(nf + 1, 0), arp(p->NE + 1, 0);
  for (int64_t f = 0; f < nf; ++f) {
    rp[f + 1] = rp[f] + cnt[f];
    bjrp[f + 1] = f + 1;
  }
  for (int64_t e = 0; e < p->NE; ++e) arp[e + 1] = arp[e] + acnt[e];
  p->nnzb = rp[nf];
  p->asm_nblk = arp[p->NE];
  p->h_rowptr = rp;
  p->d_rowptr = p->upload(rp);
  p->d_bj_rowptr = p->upload(bjrp);
  p->d_asm_rowptr = p->upload(arp);
  p->h_nbr = nbr;
  p->d_nbr = p->upload(nbr);
  p->d_cnt = p->upload(cnt);
  p->d_slot_e = p->upload(se);
  p->d_slot_lr = p->upload(slr);
  p->d_slot_lc = p->upload(slc);
  p->d_diag2 = p->upload(diag2);
  p->d_rhs_src = p->upload(rsrc);
  p->d_asm_lf = p->upload(alf);
  p->d_asm_cnt = p->upload(acnt);
  p->d_asm_face_free = p->upload(aff);
  p->d_fsum = p->upload(fsum);
  p->d_bj_nbr = p->upload(bjn);
  p->d_bj_cnt = p->upload(bjc);
  p->d_elem_face = p->upload(p->h_elem_face);
  p->d_free_of_face = p->upload(p->h_free_of_face);
  p->d_face_dir = p->upload(p->h_face_dir);
  return HDG_OK;
}

// per-element input sizes (doubles)
struct InSizes {
  int64_t Me, Bd, Cd, D, E, F, G, H, J, ru, ruh, total;
};
InSizes in_sizes(hdg_problem p) {
  InSizes s;
  s.Me = (int64_t)p->PE * p->PE;
  s.Bd = (int64_t)p->D * p->PE * p->PE;
  s.Cd = (int64_t)p->D * p->PE * p->nlPF;
  s.D = (int64_t)p->MPE * p->MDPE;
  s.E = (int64_t)p->MPE * p->MPE;
  s.F = (int64_t)p->MPE * p->nlb;
  s.G = (int64_t)p->nlb * p->MDPE;
  s.H = (int64_t)p->nlb * p->MPE;
  s.J = (int64_t)p->nlb * p->nlb;
  s.ru = (int64_t)p->MPE * p->R;
  s.ruh = (int64_t)p->nlb * p->R;
  s.total = s.Me + s.Bd + s.Cd + s.D + s.E + s.F + s.G + s.H + s.J + s.ru + s.ruh;
  return s;
}
// Condensation scratch per element (doubles): M^{-1}, Ebar, [Fbar | r_u],
// Hbar, [X_F | X_r], [Jbar - Hbar X_F | rbar]  (the last three with nlb + R
// columns, so that the right-hand-side columns ride in the same products).
int64_t tmp_elems(int64_t PE, int64_t MPE, int64_t nlb, int64_t R) {
  return PE * PE + MPE * MPE + MPE * (nlb + R) + nlb * MPE + MPE * (nlb + R) + nlb * (nlb + R);
}
int64_t tmp_per_elem(hdg_problem p) { return tmp_elems(p->PE, p->MPE, p->nlb, p->R); }
// device bytes of one condensation chunk (inputs + scratch)
constexpr int64_t kChunkBudget = 3ll << 29;   // 1.5 GiB
// recovery into host buffers: up to 8 pieces of at least 1024 elements
constexpr int64_t kRecoverPieces = 8, kRecoverPieceMin = 1024;
inline int64_t pieces_run(int64_t n, int64_t per) { return (n + per - 1) / per; }

GemmDesc gd(int M, int N, int K, const double* A, int64_t lda, int64_t sA0, int64_t sA1, const double* B,
            int64_t ldb, int64_t sB0, int64_t sB1, double* C, int64_t ldc, int64_t sC0, int64_t sC1, double alpha,
            double beta, int nb0, int nb1, int cg = 0, int64_t cgs = 0) {
  GemmDesc d;
  d.M = M; d.N = N; d.K = K;
  d.A = A; d.lda = lda; d.sA0 = sA0; d.sA1 = sA1;
  d.B = B; d.ldb = ldb; d.sB0 = sB0; d.sB1 = sB1;
  d.C = C; d.ldc = ldc; d.sC0 = sC0; d.sC1 = sC1;
  d.alpha = alpha; d.beta = beta; d.nb0 = nb0; d.nb1 = nb1;
  d.cg = cg > 0 ? cg : N;
  d.cgs = cg > 0 ? cgs : N;
  return d;
}

// Copy the inputs E, F, H, J or r_uh into the per-element work arrays: one
// contiguous copy, or `count` copies of a block shared by all elements.
void copy_in(double* dst, const double* src, int64_t per, int64_t count, bool shared, cudaStream_t s) {
  if (shared) bcast_copy(dst, src, per, count, s);
  else CK(cudaMemcpyAsync(dst, src, sizeof(double) * per * count, cudaMemcpyDeviceToDevice, s));
}

// Condense elements [e0, e0+ec) whose inputs are device arrays laid out as in
// hdg.h.  sh[i] = true when input i is one block shared by every element
// (batch stride 0 in the products).
// Condensation products: on the BF16 tensor cores with exact operand
// splitting (FP64-accurate) where the shape allows, else on the FP64 cores.
// Event pairs around timed launches (hdg_set_timing): kind 0-2 block-row
// products per precision, 3 tensor-core condensation products.
void timed_begin(hdg_problem p, cudaStream_t s) {
  if (!p->timing) return;
  if (p->ev_used + 2 > p->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      p->ev_pool.push_back(e);
    }
  }
  CK(cudaEventRecord(p->ev_pool[p->ev_used], s));
}
void timed_end(hdg_problem p, cudaStream_t s, int kind) {
  if (!p->timing) return;
  CK(cudaEventRecord(p->ev_pool[p->ev_used + 1], s));
  p->ev_used += 2;
  p->ev_prec.push_back(kind);
}

void gemm_c(hdg_problem p, const GemmDesc& d, cudaStream_t s) {
  if (p->condense_mode == 2) {
    int64_t exw = 0;
    const int64_t need = gemm_planes_bytes(d, &exw);
    if (need >= 0) {
      if (need > p->planes_cap) {
        p->dfree(p->d_planes, (size_t)p->planes_cap);
        p->d_planes = nullptr;
        p->planes_cap = 0;
        p->d_planes = (unsigned char*)p->dalloc((size_t)need);
        p->planes_cap = need;
      }
      if (exw > p->pex_cap) {
        p->dfree(p->d_pex, sizeof(uint16_t) * (size_t)p->pex_cap);
        p->d_pex = nullptr;
        p->pex_cap = 0;
        p->d_pex = (uint16_t*)p->dalloc(sizeof(uint16_t) * (size_t)exw);
        p->pex_cap = exw;
      }
      timed_begin(p, s);
      const bool ok = gemm_ozaki_planes(d, p->d_planes, p->planes_cap, p->d_pex, p->pex_cap, p->d_err, s);
      timed_end(p, s, 3);
      if (ok) return;
    }
  }
  // Products of at most 32 rows fill a quarter or less of the 128-row
  // tensor-core tile; measured on the condensation shapes (M = 9, 27) the FP64
  // pipe is faster for them.
  if (p->condense_mode >= 1 && d.M > 32 && gemm_ozaki_scratch(d) <= p->oz_cap && d.N >= 16 &&
      (d.K <= 192 || p->condense_mode == 1)) {
    timed_begin(p, s);
    if (p->condense_mode == 3) gemm_ozaki_persist(d, p->d_oz, p->oz_cap, p->d_err, s);
    else gemm_ozaki(d, p->d_oz, p->d_err, s);
    timed_end(p, s, 3);
    return;
  }
  gemm_f64(d, s);
}

// Scratch (doubles per matrix) of inverse_any for an n x n matrix.
int64_t inverse_scratch(int n) {
  if (n <= inverse_max_n()) return 0;
  const int n1 = (n + 1) / 2;
  return (int64_t)n * n + inverse_scratch(n1);
}

// Batched in-place inverse of `count` n x n matrices (batch stride `stride`)
// of any size.  Up to one CTA's shared memory: Gauss-Jordan with partial
// pivoting (inverse_f64).  Beyond: the 2 x 2 block form with the leading
// block A11 (n1 = ceil(n/2)) and its Schur complement S = A22 - A21 A11^{-1}
// A12, both inverted recursively,
//   A^{-1} = [A11^{-1} + T S^{-1} U,  -T S^{-1};  -S^{-1} U,  S^{-1}],
//   T = A11^{-1} A12,  U = A21 A11^{-1},
// with the products on the condensation's GEMM path.  Pivoting stays within
// the leaves, so the split needs a nonsingular leading block: true for SPD
// matrices and for matrices whose symmetric part is positive definite, which
// covers the local HDG matrices Ebar (Eq. w19) and the ASM patch matrices
// (Sec. 4.6) of the discretisations here.  A zero leaf pivot sets
// ERRBIT_SINGULAR.
void inverse_any(hdg_problem p, double* A, int n, int64_t stride, int64_t count, cudaStream_t s,
                 int64_t scratch_off = 0) {
  if (n <= 0 || count <= 0) return;
  if (n <= inverse_max_n()) {
    inverse_f64(A, n, stride, count, p->d_err, s);
    return;
  }
  const int64_t need = inverse_scratch(n);
  if (scratch_off == 0) {
    // matrices per pass: scratch of at most 1 GiB (at least one matrix)
    const int64_t per_pass = std::max<int64_t>(1, std::min<int64_t>(count, (1ll << 27) / need));
    if (per_pass * need > p->invs_cap) {
      p->dfree(p->d_invs, sizeof(double) * (size_t)p->invs_cap);
      p->d_invs = nullptr;
      p->invs_cap = 0;
      p->d_invs = (double*)p->dalloc(sizeof(double) * (size_t)(per_pass * need));
      p->invs_cap = per_pass * need;
    }
    if (count > per_pass) {
      for (int64_t c0 = 0; c0 < count; c0 += per_pass)
        inverse_any(p, A + c0 * stride, n, stride, std::min(per_pass, count - c0), s, 0);
      return;
    }
  }
  const int n1 = (n + 1) / 2, n2 = n - n1;
  const int c = (int)count;
  const int64_t nn = (int64_t)n * n;
  double* L = p->d_invs + scratch_off;        // this level: count x n^2
  double* Ai = L;                             // n1 x n1
  double* T = Ai + (int64_t)n1 * n1;          // n1 x n2
  double* U = T + (int64_t)n1 * n2;           // n2 x n1
  double* Sc = U + (int64_t)n2 * n1;          // n2 x n2
  const int64_t deeper = scratch_off + count * nn;
  double* A11 = A;
  double* A12 = A + n1;
  double* A21 = A + (int64_t)n1 * n;
  double* A22 = A21 + n1;
  copy_block_f64(Ai, n1, nn, A11, n, stride, n1, n1, count, s);
  inverse_any(p, Ai, n1, nn, count, s, deeper);
  gemm_c(p, gd(n1, n2, n1, Ai, n1, nn, 0, A12, n, stride, 0, T, n2, nn, 0, 1.0, 0.0, c, 1), s);
  gemm_c(p, gd(n2, n1, n1, A21, n, stride, 0, Ai, n1, nn, 0, U, n1, nn, 0, 1.0, 0.0, c, 1), s);
  gemm_c(p, gd(n2, n2, n1, A21, n, stride, 0, T, n2, nn, 0, A22, n, stride, 0, -1.0, 1.0, c, 1), s);
  copy_block_f64(Sc, n2, nn, A22, n, stride, n2, n2, count, s);
  inverse_any(p, Sc, n2, nn, count, s, deeper);
  gemm_c(p, gd(n1, n2, n2, T, n2, nn, 0, Sc, n2, nn, 0, A12, n, stride, 0, -1.0, 0.0, c, 1), s);
  gemm_c(p, gd(n2, n1, n2, Sc, n2, nn, 0, U, n1, nn, 0, A21, n, stride, 0, -1.0, 0.0, c, 1), s);
  copy_block_f64(A11, n, stride, Ai, n1, nn, n1, n1, count, s);
  gemm_c(p, gd(n1, n1, n2, A12, n, stride, 0, U, n1, nn, 0, A11, n, stride, 0, -1.0, 1.0, c, 1), s);
  copy_block_f64(A22, n, stride, Sc, n2, nn, n2, n2, count, s);
}

void condense_chunk(hdg_problem p, int64_t e0, int64_t ec, const double* Me, const double* Bd, const double* Cd,
                    const double* Dm, const double* Em, const double* Fm, const double* Gm, const double* Hm,
                    const double* Jm, const double* ru, const double* ruh, const bool* sh, cudaStream_t s) {
  const int PE = p->PE, D = p->D, M = p->M, PF = p->PF, MPE = p->MPE, MDPE = p->MDPE, nlb = p->nlb,
            nlPF = p->nlPF, R = p->R;
  const int n = (int)ec;
  const int nlbR = nlb + R;
  double* Minv = p->d_tmp;
  double* Eb = Minv + ec * PE * PE;
  double* Fb = Eb + ec * MPE * MPE;                 // [Fbar | r_u], MPE x nlbR
  double* Hb = Fb + ec * MPE * nlbR;
  double* XFr = Hb + ec * nlb * MPE;                // [X_F | X_r], MPE x nlbR
  double* Kr = XFr + ec * MPE * nlbR;               // [Kbar | rbar], nlb x nlbR
  double* MinvB = p->d_MinvB + e0 * D * PE * PE;
  double* MinvC = p->d_MinvC + e0 * D * PE * nlPF;
  double* XF = p->d_XF + e0 * MPE * nlb;
  double* Xr = p->d_Xr + e0 * MPE * R;
  double* Kb = p->d_Kbar + e0 * nlb * nlb;
  double* rb = p->d_rbar + e0 * nlb * R;
  // batch strides of the inputs (0 = one block shared by every element)
  const int64_t sMe = sh[0] ? 0 : (int64_t)PE * PE, sBd = sh[1] ? 0 : (int64_t)D * PE * PE,
                sCd = sh[2] ? 0 : (int64_t)D * PE * nlPF, sD = sh[3] ? 0 : (int64_t)MPE * MDPE,
                sG = sh[6] ? 0 : (int64_t)nlb * MDPE, sru = sh[9] ? 0 : (int64_t)MPE * R;
  // (M^e)^{-1}  (Eq. w16); a shared mass matrix is inverted once
  const int64_t nM = sh[0] ? 1 : ec;
  CK(cudaMemcpyAsync(Minv, Me, sizeof(double) * nM * PE * PE, cudaMemcpyDeviceToDevice, s));
  inverse_any(p, Minv, PE, (int64_t)PE * PE, nM, s);
  // (M^e)^{-1} B_d, (M^e)^{-1} C_d
  gemm_c(p, gd(PE, PE, PE, Minv, PE, sMe, 0, Bd, PE, sBd, PE * PE, MinvB, PE, (int64_t)D * PE * PE, PE * PE, 1.0, 0.0,
              n, D), s);
  gemm_c(p, gd(PE, nlPF, PE, Minv, PE, sMe, 0, Cd, nlPF, sCd, (int64_t)PE * nlPF, MinvC, nlPF,
              (int64_t)D * PE * nlPF, (int64_t)PE * nlPF, 1.0, 0.0, n, D), s);
  // Ebar = E - D A^{-1} B, per component block b: D[:, (b,.,.)] * stack_d (M^e)^{-1}B_d   (Eq. w19)
  copy_in(Eb, Em, (int64_t)MPE * MPE, ec, sh[4], s);
  gemm_c(p, gd(MPE, PE, D * PE, Dm, MDPE, sD, (int64_t)D * PE, MinvB, PE, (int64_t)D * PE * PE, 0, Eb, MPE,
              (int64_t)MPE * MPE, PE, -1.0, 1.0, n, M), s);
  // Fbar = F - D A^{-1} C, output columns (l, b, j); r_u beside it
  copy_block_f64(Fb, nlbR, (int64_t)MPE * nlbR, Fm, nlb, sh[5] ? 0 : (int64_t)MPE * nlb, MPE, nlb, ec, s);
  copy_block_f64(Fb + nlb, nlbR, (int64_t)MPE * nlbR, ru, R, sru, MPE, R, ec, s);
  gemm_c(p, gd(MPE, nlPF, D * PE, Dm, MDPE, sD, (int64_t)D * PE, MinvC, nlPF, (int64_t)D * PE * nlPF, 0, Fb, nlbR,
              (int64_t)MPE * nlbR, PF, -1.0, 1.0, n, M, PF, (int64_t)M * PF), s);
  // Hbar = H - G A^{-1} B                                       (Eq. w21)
  copy_in(Hb, Hm, (int64_t)nlb * MPE, ec, sh[7], s);
  gemm_c(p, gd(nlb, PE, D * PE, Gm, MDPE, sG, (int64_t)D * PE, MinvB, PE, (int64_t)D * PE * PE, 0, Hb, MPE,
              (int64_t)nlb * MPE, PE, -1.0, 1.0, n, M), s);
  // Jbar = J - G A^{-1} C, r_uh beside it
  copy_block_f64(Kr, nlbR, (int64_t)nlb * nlbR, Jm, nlb, sh[8] ? 0 : (int64_t)nlb * nlb, nlb, nlb, ec, s);
  copy_block_f64(Kr + nlb, nlbR, (int64_t)nlb * nlbR, ruh, R, sh[10] ? 0 : (int64_t)nlb * R, nlb, R, ec, s);
  gemm_c(p, gd(nlb, nlPF, D * PE, Gm, MDPE, sG, (int64_t)D * PE, MinvC, nlPF, (int64_t)D * PE * nlPF, 0, Kr, nlbR,
              (int64_t)nlb * nlbR, PF, -1.0, 1.0, n, M, PF, (int64_t)M * PF), s);
  // Ebar^{-1}; [X_F | X_r] = Ebar^{-1} [Fbar | r_u]
  inverse_any(p, Eb, MPE, (int64_t)MPE * MPE, ec, s);
  gemm_c(p, gd(MPE, nlbR, MPE, Eb, MPE, (int64_t)MPE * MPE, 0, Fb, nlbR, (int64_t)MPE * nlbR, 0, XFr, nlbR,
              (int64_t)MPE * nlbR, 0, 1.0, 0.0, n, 1), s);
  // [Kbar | rbar] = [Jbar | r_uh] - Hbar [X_F | X_r]            (Eq. w22)
  gemm_c(p, gd(nlb, nlbR, MPE, Hb, MPE, (int64_t)nlb * MPE, 0, XFr, nlbR, (int64_t)MPE * nlbR, 0, Kr, nlbR,
              (int64_t)nlb * nlbR, 0, -1.0, 1.0, n, 1), s);
  copy_block_f64(XF, nlb, (int64_t)MPE * nlb, XFr, nlbR, (int64_t)MPE * nlbR, MPE, nlb, ec, s);
  copy_block_f64(Xr, R, (int64_t)MPE * R, XFr + nlb, nlbR, (int64_t)MPE * nlbR, MPE, R, ec, s);
  copy_block_f64(Kb, nlb, (int64_t)nlb * nlb, Kr, nlbR, (int64_t)nlb * nlbR, nlb, nlb, ec, s);
  copy_block_f64(rb, R, (int64_t)nlb * R, Kr + nlb, nlbR, (int64_t)nlb * nlbR, nlb, R, ec, s);
}

// ------------------------------------------------------------------ operators
enum { TUNE_K = 0, TUNE_BJ = 1, TUNE_ASM = 2 };
BrCfg cfg_of(hdg_problem p, int op, int prec) {
  if (p->br_variant == 1) {
    BrCfg c;
    c.kind = BR_TMA;
    return c;
  }
  return p->tune[op][prec];
}

constexpr int kMaxBatch = 256;     // systems per hdg_solve_batch call

// FP32 work vectors of the low-precision preconditioner path
void ensure_low(hdg_problem p) {
  if (p->lp0) return;
  const int64_t len = p->ndof * p->R;
  p->lp0 = (float*)p->dalloc(sizeof(float) * len);
  p->lp1 = (float*)p->dalloc(sizeof(float) * len);
  p->lp2 = (float*)p->dalloc(sizeof(float) * len);
  p->ks32 = (float*)p->dalloc(sizeof(float) * len);
  p->t1_32 = (float*)p->dalloc(sizeof(float) * len);
  p->ze32 = (float*)p->dalloc(sizeof(float) * std::max<int64_t>(p->NE * p->nlb * p->R, 1));
}

struct Ops {
  hdg_problem p;
  cudaStream_t s;
  int R;

  void mv_timed_begin(cudaEvent_t*) { timed_begin(p, s); }
  void mv_timed_end(int prec) { timed_end(p, s, prec); }

  BlockRowDesc kdesc(int prec) const {
    BlockRowDesc d{};
    d.prec = prec;
    d.blk = prec == HDG_FP64 ? (const void*)p->K64 : prec == HDG_FP32 ? (const void*)p->K32 : (const void*)p->K16;
    d.blk_stride = prec == HDG_FP64 ? p->s64 : prec == HDG_FP32 ? p->s32 : p->s16;
    d.rowptr = p->d_rowptr;
    d.nbr = p->d_nbr;
    d.cnt = p->d_cnt;
    d.n_units = p->nfree;
    d.b_rows = p->b;
    d.ld = prec == HDG_FP64 ? p->b : prec == HDG_FP32 ? p->ld32 : p->ld16;
    d.bc = p->b;
    d.max_slots = p->ms;
    d.R = R;
    d.err = p->d_err;
    return d;
  }
  // y32 = K x32 with FP32 / BF16 blocks, FP32 in and out
  void K_low(int prec, const float* x32, float* y32, const int* active) {
    BlockRowDesc d = kdesc(prec);
    d.in32 = x32;
    d.out32 = y32;
    d.epi = EPI_STORE;
    d.active = active;
    cudaEvent_t a;
    mv_timed_begin(&a);
    blockrow(d, cfg_of(p, TUNE_K, prec), s);
    mv_timed_end(prec);
  }
  // M^{-1} v32 (low-precision blocks) followed by the polynomial step e
  void Minv_epi(int pc, int prec, const float* v32, const PolyEpi& e, const int* active) {
    if (pc == HDG_PC_NONE) {
      poly_epi_apply(e, v32, p->ndof * R, active, R, s);
      return;
    }
    BlockRowDesc d{};
    d.prec = prec;
    d.R = R;
    d.in32 = v32;
    d.active = active;
    d.err = p->d_err;
    d.bc = p->b;
    if (pc == HDG_PC_BJ) {
      d.blk = prec == HDG_FP32 ? (const void*)p->bj32 : (const void*)p->bj16;
      d.blk_stride = prec == HDG_FP32 ? p->bs32 : p->bs16;
      d.rowptr = p->d_bj_rowptr;
      d.nbr = p->d_bj_nbr;
      d.cnt = p->d_bj_cnt;
      d.n_units = p->nfree;
      d.b_rows = p->b;
      d.ld = prec == HDG_FP32 ? p->ld32 : p->ld16;
      d.max_slots = 1;
      d.epi = EPI_POLY;
      d.pe = e;
      timed_begin(p, s);
      blockrow(d, cfg_of(p, TUNE_BJ, prec), s);
      timed_end(p, s, prec == HDG_FP32 ? 4 : 5);
    } else {
      d.blk = prec == HDG_FP32 ? (const void*)p->as32 : (const void*)p->as16;
      d.blk_stride = prec == HDG_FP32 ? p->as_s32 : p->as_s16;
      d.rowptr = p->d_asm_rowptr;
      d.nbr = p->d_asm_face_free;
      d.cnt = p->d_asm_cnt;
      d.n_units = p->NE;
      d.b_rows = p->nlb;
      d.ld = prec == HDG_FP32 ? p->as_ld32 : p->as_ld16;
      d.max_slots = p->nl;
      d.epi = EPI_STORE;
      d.out32 = p->ze32;
      blockrow(d, cfg_of(p, TUNE_ASM, prec), s);
      asm_face_sum_f32(p->ze32, p->nlb, p->b, R, p->nfree, p->d_fsum, &e, nullptr, nullptr, s);
    }
  }

  // y = K x (prec storage), epilogue; y32 (optional) receives an FP32 copy of
  // y; x32 (optional) is an FP32 copy of x already at hand
  void K(int prec, const double* x, double* y, int epi, const double* rhs, const double* scale, const int* active,
         float* y32 = nullptr, const float* x32 = nullptr) {
    BlockRowDesc d{};
    d.prec = prec;
    d.blk = prec == HDG_FP64 ? (const void*)p->K64 : prec == HDG_FP32 ? (const void*)p->K32 : (const void*)p->K16;
    d.blk_stride = prec == HDG_FP64 ? p->s64 : prec == HDG_FP32 ? p->s32 : p->s16;
    d.rowptr = p->d_rowptr;
    d.nbr = p->d_nbr;
    d.cnt = p->d_cnt;
    d.n_units = p->nfree;
    d.b_rows = p->b;
    d.ld = prec == HDG_FP64 ? p->b : prec == HDG_FP32 ? p->ld32 : p->ld16;
    d.bc = p->b;
    d.max_slots = p->ms;
    d.R = R;
    d.in = x;
    d.in32 = nullptr;
    if (prec != HDG_FP64) {
      if (x32) {
        d.in32 = x32;
      } else {
        to_f32(x, p->x32, p->ndof * R, s);
        d.in32 = p->x32;
      }
    }
    d.out = y;
    d.out32 = y32;
    d.epi = epi;
    d.rhs = rhs;
    d.scale = scale;
    d.active = active;
    d.err = p->d_err;
    cudaEvent_t a;
    mv_timed_begin(&a);
    const BrCfg cfg = cfg_of(p, TUNE_K, prec);
    const bool tc = prec == HDG_FP64 && p->kdig_ready && (cfg.kind == BR_DEFAULT || cfg.kind == BR_TC) &&
                    tc_blockrow(d, p->kdig, p->d_kdoff, p->kex, s);
    if (!tc) blockrow(d, cfg, s);
    mv_timed_end(prec);
  }
  // y = M^{-1} x for the base preconditioner (x32: optional FP32 copy of x)
  void Minv(int pc, int prec, const double* x, double* y, const int* active, const float* x32 = nullptr) {
    if (pc == HDG_PC_NONE) {
      launch_axpby(y, x, 1.0, 0.0, p->ndof * R, active, R, s);
      return;
    }
    BlockRowDesc d{};
    d.prec = prec;
    d.R = R;
    d.in = x;
    d.in32 = nullptr;
    if (prec != HDG_FP64) {
      if (x32) {
        d.in32 = x32;
      } else {
        to_f32(x, p->x32, p->ndof * R, s);
        d.in32 = p->x32;
      }
    }
    d.epi = EPI_STORE;
    d.active = active;
    d.err = p->d_err;
    d.bc = p->b;
    if (pc == HDG_PC_BJ) {
      d.blk = prec == HDG_FP64 ? (const void*)p->bj64 : prec == HDG_FP32 ? (const void*)p->bj32 : (const void*)p->bj16;
      d.blk_stride = prec == HDG_FP64 ? p->bs64 : prec == HDG_FP32 ? p->bs32 : p->bs16;
      d.rowptr = p->d_bj_rowptr;
      d.nbr = p->d_bj_nbr;
      d.cnt = p->d_bj_cnt;
      d.n_units = p->nfree;
      d.b_rows = p->b;
      d.ld = prec == HDG_FP64 ? p->b : prec == HDG_FP32 ? p->ld32 : p->ld16;
      d.max_slots = 1;
      d.out = y;
      blockrow(d, cfg_of(p, TUNE_BJ, prec), s);
    } else {
      d.blk = prec == HDG_FP64 ? (const void*)p->as64 : prec == HDG_FP32 ? (const void*)p->as32 : (const void*)p->as16;
      d.blk_stride = prec == HDG_FP64 ? p->as_s64 : prec == HDG_FP32 ? p->as_s32 : p->as_s16;
      d.rowptr = p->d_asm_rowptr;
      d.nbr = p->d_asm_face_free;
      d.cnt = p->d_asm_cnt;
      d.n_units = p->NE;
      d.b_rows = p->nlb;
      d.ld = prec == HDG_FP64 ? p->nlb : prec == HDG_FP32 ? p->as_ld32 : p->as_ld16;
      d.max_slots = p->nl;
      if (prec == HDG_FP64) {
        d.out = p->ze;
        blockrow(d, cfg_of(p, TUNE_ASM, prec), s);
        asm_face_sum(p->ze, p->nlb, p->b, R, p->nfree, p->d_fsum, y, s);
      } else {
        // FP32 element results, summed per face in FP32
        ensure_low(p);
        d.out32 = p->ze32;
        blockrow(d, cfg_of(p, TUNE_ASM, prec), s);
        asm_face_sum_f32(p->ze32, p->nlb, p->b, R, p->nfree, p->d_fsum, nullptr, y, nullptr, s);
      }
    }
  }
  // y = A x with A = M^{-1} K
  void A(int pc, int kprec, int mprec, const double* x, double* y, const int* active) {
    if (pc == HDG_PC_NONE) {
      K(kprec, x, y, EPI_STORE, nullptr, nullptr, active);
    } else {
      K(kprec, x, p->ptmp, EPI_STORE, nullptr, nullptr, active);
      Minv(pc, mprec, p->ptmp, y, active);
    }
  }
  // Low-precision polynomial preconditioner: every step is one K product
  // (FP32 in and out) and one M^{-1} apply whose epilogue performs the
  // recurrence on FP32 state vectors; the last step writes y in FP64.
  void Pinv_low(const hdg_solver_opts& o, int mprec, int kpoly, const double* x, const float* x32, double* y,
                const int* active) {
    ensure_low(p);
    const float* xin = x32;
    if (!xin) {
      to_f32(x, p->x32, p->ndof * R, s);
      xin = p->x32;
    }
    PolyEpi e{};
    e.out64 = y;
    e.p0 = p->lp0;
    e.p1 = p->lp1;
    e.p2 = p->lp2;
    if (o.poly == HDG_POLY_CHEBYSHEV) {
      // Chebyshev iteration (Saad, Alg. 12.1), degree+1 terms from z = 0
      const double theta = 0.5 * (p->cheb_b + p->cheb_a), delta = 0.5 * (p->cheb_b - p->cheb_a);
      const double sigma = theta / delta;
      double rho = 1.0 / sigma;
      const int deg = p->poly_n;
      e.op = CHEB_INIT;
      e.c1 = (float)(1.0 / theta);
      e.last = deg == 0 ? 1 : 0;
      Minv_epi(o.pc, mprec, xin, e, active);
      for (int kq = 0; kq < deg; ++kq) {
        K_low(kpoly, p->lp2, p->ks32, active);
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        e.op = CHEB_STEP;
        e.c1 = (float)(rho_new * rho);
        e.c2 = (float)(2.0 * rho_new / delta);
        e.last = kq == deg - 1 ? 1 : 0;
        Minv_epi(o.pc, mprec, p->ks32, e, active);
        rho = rho_new;
      }
      return;
    }
    // GMRES polynomial (Sec. 4.7): q = M^{-1} x; real values and conjugate pairs
    const int P = p->poly_n;
    auto real_at = [&](int i) { return i < P && p->th_im[i] == 0.0; };
    e.op = PP_INIT;
    e.fin = (P == 1 && real_at(0)) ? 1 : 0;
    e.cfin = (float)(1.0 / p->th_re[0]);
    Minv_epi(o.pc, mprec, xin, e, active);
    int i = 0;
    bool first = true;
    while (i < P) {
      const double a = p->th_re[i], bi = p->th_im[i];
      PolyEpi f = e;
      f.wzero = first ? 1 : 0;
      f.fin = 0;
      f.last = 0;
      if (bi == 0.0) {
        if (i == P - 1) break;          // folded into the step that last updated q
        K_low(kpoly, p->lp0, p->ks32, active);
        f.op = PP_REAL;
        f.c1 = (float)(1.0 / a);
        f.fin = (i + 1 == P - 1 && real_at(i + 1)) ? 1 : 0;
        f.cfin = f.fin ? (float)(1.0 / p->th_re[i + 1]) : 0.f;
        Minv_epi(o.pc, mprec, p->ks32, f, active);
        i += 1;
      } else {
        const double mod2 = a * a + bi * bi;
        const bool last = (i + 1 >= P - 1);
        K_low(kpoly, p->lp0, p->ks32, active);
        f.op = PP_PAIR_T;
        f.c1 = (float)(2.0 * a);
        f.c2 = (float)(1.0 / mod2);
        f.last = last ? 1 : 0;
        Minv_epi(o.pc, mprec, p->ks32, f, active);
        if (!last) {
          K_low(kpoly, p->lp2, p->ks32, active);
          PolyEpi g = e;
          g.op = PP_PAIR_Q;
          g.c2 = (float)(1.0 / mod2);
          g.fin = (i + 2 == P - 1 && real_at(i + 2)) ? 1 : 0;
          g.cfin = g.fin ? (float)(1.0 / p->th_re[i + 2]) : 0.f;
          Minv_epi(o.pc, mprec, p->ks32, g, active);
        }
        i += 2;
      }
      first = false;
    }
  }

  // y = P^{-1} x : polynomial p(M^{-1}K) applied to M^{-1} x, or M^{-1} x.
  // x32 (optional): an FP32 copy of x already at hand.
  void Pinv(const hdg_solver_opts& o, int mprec, int kpoly, const double* x, double* y, const int* active,
            const float* x32 = nullptr) {
    const int64_t len = p->ndof * R;
    if (o.poly == HDG_POLY_NONE || p->poly_n == 0) {
      Minv(o.pc, mprec, x, y, active, x32);
      return;
    }
    if (mprec != HDG_FP64 && kpoly != HDG_FP64) {
      Pinv_low(o, mprec, kpoly, x, x32, y, active);
      return;
    }
    double* q = p->pq;
    Minv(o.pc, mprec, x, q, active);
    if (o.poly == HDG_POLY_GMRES) {
      // Sec. 4.7 recurrence, real values and conjugate pairs
      const int P = p->poly_n;
      int i = 0;
      bool first = true;
      while (i < P) {
        const double a = p->th_re[i], bi = p->th_im[i];
        if (bi == 0.0) {
          const bool last = (i == P - 1);
          if (!last) A(o.pc, kpoly, mprec, q, p->pAq, active);
          launch_pp_real(y, q, p->pAq, 1.0 / a, len, last ? 0 : 1, active, R, first ? 1 : 0, s);
          i += 1;
        } else {
          const double mod2 = a * a + bi * bi;
          const bool last = (i + 1 >= P - 1);
          A(o.pc, kpoly, mprec, q, p->pAq, active);
          launch_pp_pair_t(p->pt, y, q, p->pAq, 2.0 * a, 1.0 / mod2, len, active, R, first ? 1 : 0, s);
          if (!last) {
            A(o.pc, kpoly, mprec, p->pt, p->pAq, active);
            launch_pp_pair_q(q, p->pAq, 1.0 / mod2, len, active, R, s);
          }
          i += 2;
        }
        first = false;
      }
    } else {
      // Chebyshev iteration (Saad, Alg. 12.1) with degree+1 steps from z = 0
      const double theta = 0.5 * (p->cheb_b + p->cheb_a), delta = 0.5 * (p->cheb_b - p->cheb_a);
      const double sigma = theta / delta;
      double rho = 1.0 / sigma;
      double* r = q;          // residual, starts at M^{-1} x
      double* d = p->pt;
      launch_axpby(d, r, 1.0 / theta, 0.0, len, active, R, s);
      for (int kq = 0; kq <= p->poly_n; ++kq) {
        launch_cheb(y, d, r, nullptr, 0, 0, len, kq == 0 ? 0 : 1, active, R, s);
        if (kq == p->poly_n) break;
        A(o.pc, kpoly, mprec, d, p->pAq, active);
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        launch_cheb(y, d, r, p->pAq, rho_new * rho, 2.0 * rho_new / delta, len, 2, active, R, s);
        rho = rho_new;
      }
    }
  }
};

// Adds the durations of the recorded block-matvec launches to the per-precision totals.
void collect_timing(hdg_problem p, cudaStream_t s) {
  if (!p->timing || p->ev_used == 0) return;
  CK(cudaStreamSynchronize(s));
  for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->ev_pool[i], p->ev_pool[i + 1]));
    const int pr = p->ev_prec[i / 2];
    p->t_mv_ms[pr] += ms;
    p->n_mv[pr] += 1;
  }
  p->ev_used = 0;
  p->ev_prec.clear();
}

void ensure_workspace(hdg_problem p, int m) {
  if (p->ws_m >= m) return;
  const int64_t len = p->ndof * p->R;
  const int R = p->R;
  auto A = [&](size_t nb) { return p->dalloc(nb); };
  if (p->ws_m < 0) {
    p->d_x = (double*)A(sizeof(double) * len);
    p->t1 = (double*)A(sizeof(double) * len);
    p->res = (double*)A(sizeof(double) * len);
    p->pq = (double*)A(sizeof(double) * len);
    p->pw = (double*)A(sizeof(double) * len);
    p->ptmp = (double*)A(sizeof(double) * len);
    p->pAq = (double*)A(sizeof(double) * len);
    p->pt = (double*)A(sizeof(double) * len);
    p->xo = (double*)A(sizeof(double) * len);
    p->x32 = (float*)A(sizeof(float) * len);
    p->bo = (double*)A(sizeof(double) * len);
    p->ze = (double*)A(sizeof(double) * p->NE * p->nlb * R);
    p->tolabs = (double*)A(sizeof(double) * kMaxR);
    p->cfac = (double*)A(sizeof(double) * kMaxR);
    p->zb = (double*)A(sizeof(double) * kMaxR);
    p->bnorm = (double*)A(sizeof(double) * kMaxR);
    p->rel = (double*)A(sizeof(double) * kMaxR);
    p->running = (int*)A(sizeof(int) * kMaxR);
    p->jend = (int*)A(sizeof(int) * kMaxR);
    p->on_estimate = (int*)A(sizeof(int) * kMaxR);
    p->done = (int*)A(sizeof(int) * kMaxR);
    p->iters = (int*)A(sizeof(int) * kMaxR);
    p->counter = (unsigned*)A(sizeof(unsigned) * 4);
    p->dmaxit = (int*)A(sizeof(int));
    p->bdone = (int*)A(sizeof(int));
    CK(cudaMemset(p->counter, 0, sizeof(unsigned) * 4));
    CK(cudaMemset(p->d_x, 0, sizeof(double) * len));
  } else {
    for (auto& cg : p->graphs) {
      if (cg.exec) cudaGraphExecDestroy(cg.exec);
      if (cg.g) cudaGraphDestroy(cg.g);
    }
    p->graphs.clear();
    p->dfree(p->V, 0);
    p->dfree(p->vscale, 0);
    p->dfree(p->H, 0);
    p->dfree(p->g, 0);
    p->dfree(p->cs, 0);
    p->dfree(p->sn, 0);
    p->dfree(p->hcol, 0);
    p->dfree(p->htmp, 0);
    p->dfree(p->ycoef, 0);
    p->dfree(p->partial, 0);
  }
  p->V = (double*)A(sizeof(double) * (m + 1) * len);
  p->vscale = (double*)A(sizeof(double) * (m + 1) * R);
  p->H = (double*)A(sizeof(double) * R * (m + 1) * m);
  p->g = (double*)A(sizeof(double) * R * (m + 1));
  p->cs = (double*)A(sizeof(double) * R * m);
  p->sn = (double*)A(sizeof(double) * R * m);
  p->hcol = (double*)A(sizeof(double) * R * (m + 2));
  p->htmp = (double*)A(sizeof(double) * R * (m + 2));
  p->ycoef = (double*)A(sizeof(double) * R * (m + 1));
  // reductions use at most 1024 blocks (see gmres_chunk)
  p->partial = (double*)A(sizeof(double) * (int64_t)(m + 2) * 1024 * R);
  p->ws_m = m;
}

GmresView make_view(hdg_problem p, int R, int m, double rtol, int maxit) {
  GmresView k{};
  k.n = p->ndof;
  k.R = R;
  k.m = m;
  k.chunk = gmres_chunk(p->ndof * R);
  k.V = p->V;
  k.vscale = p->vscale;
  k.H = p->H;
  k.g = p->g;
  k.cs = p->cs;
  k.sn = p->sn;
  k.hcol = p->hcol;
  k.htmp = p->htmp;
  k.ycoef = p->ycoef;
  k.partial = p->partial;
  k.tolabs = p->tolabs;
  k.cfac = p->cfac;
  k.zb = p->zb;
  k.rtol = rtol;
  k.running = p->running;
  k.jend = p->jend;
  k.on_estimate = p->on_estimate;
  k.done = p->done;
  k.iters = p->iters;
  k.maxit = maxit;
  k.dmaxit = p->dmaxit;
  k.hflag = p->d_flag;
  k.counter = p->counter;
  k.err = p->d_err;
  return k;
}

// One Arnoldi orthogonalisation of V_{j+1} against V_0..V_j.
void orthogonalize(const GmresView& k, int orth, int j, cudaStream_t s) {
  double* w = k.V + (int64_t)(j + 1) * k.n * k.R;
  if (orth == HDG_ORTH_MGS) {
    for (int i = 0; i <= j; ++i) {
      launch_dots(k, w, i, i + 1, s);
      launch_update(k, w, i, i + 1, j, 0, i == j ? 1 : 0, s);
    }
  } else {
    launch_dots(k, w, 0, j + 1, s);
    launch_update(k, w, 0, j + 1, j, 0, orth == HDG_ORTH_CGS2 ? 0 : 1, s);
    if (orth == HDG_ORTH_CGS2) {
      launch_dots(k, w, 0, j + 1, s);
      launch_update(k, w, 0, j + 1, j, 1, 1, s);
    }
  }
}

void set_ints(hdg_problem p, int* dptr, int v, int R, cudaStream_t s) {
  for (int r = 0; r < R; ++r) p->h_int[r] = v;
  CK(cudaMemcpyAsync(dptr, p->h_int, sizeof(int) * R, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
}
void set_dbls(hdg_problem p, double* dptr, double v, int R, cudaStream_t s) {
  for (int r = 0; r < R; ++r) p->h_dbl[r] = v;
  CK(cudaMemcpyAsync(dptr, p->h_dbl, sizeof(double) * R, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
}

// Captured GMRES cycle: m IF nodes in sequence, node j's body is iteration j
// (matvec, preconditioner, Gram-Schmidt, Givens).  The Givens step of
// iteration j sets node j+1's condition to "some right-hand side still
// running", so the iterations after convergence are skipped on the device.
// Built once per (options, precisions) and replayed per cycle.
struct IterLauncher {
  hdg_problem p;
  const hdg_solver_opts* o;
  int kprec, mprec, kpoly, R;
  void iteration(const GmresView& k, int j, cudaStream_t s) const {
    Ops ops{p, s, R};
    const int64_t len = p->ndof * R;
    double* vj = p->V + (int64_t)j * len;
    double* vn = p->V + (int64_t)(j + 1) * len;
    float* t32 = mprec != HDG_FP64 ? p->t1_32 : nullptr;   // the preconditioner's FP32 input, from the epilogue
    ops.K(kprec, vj, p->t1, EPI_SCALE, nullptr, p->vscale + (int64_t)j * R, p->running, t32);
    ops.Pinv(*o, mprec, kpoly, p->t1, vn, p->running, t32);
    orthogonalize(k, o->orth, j, s);
  }
};

unsigned long long graph_key(const hdg_solver_opts& o, int kprec, int mprec, int kpoly, int variant) {
  unsigned long long k = (unsigned long long)o.restart;
  k = k * 4 + (unsigned)o.orth;
  k = k * 4 + (unsigned)o.pc;
  k = k * 4 + (unsigned)o.poly;
  k = k * 64 + (unsigned)o.poly_degree;
  k = k * 4 + (unsigned)kprec;
  k = k * 4 + (unsigned)mprec;
  k = k * 4 + (unsigned)kpoly;
  k = k * 4096 + (unsigned)variant;
  return k + 1;
}

cudaGraphExec_t cycle_graph(hdg_problem p, const hdg_solver_opts& o, int kprec, int mprec, int kpoly,
                            const GmresView& kin, long long* kernels_per_iter) {
  const unsigned long long key = graph_key(o, kprec, mprec, kpoly, p->br_variant + 2 * (p->tune_gen & 2047));
  const unsigned pgen = (o.poly != HDG_POLY_NONE) ? p->poly_gen : 0u;
  for (auto it = p->graphs.begin(); it != p->graphs.end(); ++it) {
    if (it->key != key) continue;
    if (it->poly_gen == pgen) {
      *kernels_per_iter = it->kernels_per_iter;
      return it->exec;
    }
    // same shape, stale by-value arguments: re-capture
    if (it->exec) cudaGraphExecDestroy(it->exec);
    if (it->g) cudaGraphDestroy(it->g);
    p->graphs.erase(it);
    break;
  }
  if (!p->cap_stream) CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  hdg_problem_s::CycleGraph cg;
  cg.key = key;
  cg.poly_gen = pgen;
  CK(cudaGraphCreate(&cg.g, 0));
  // one handle per IF node: node 0 starts at 1, the others at 0 on every
  // launch; iteration j's Givens step sets node j+1's handle, so a skipped
  // node leaves all later ones switched off
  cg.h.resize(o.restart);
  for (int j = 0; j < o.restart; ++j)
    CK(cudaGraphConditionalHandleCreate(&cg.h[j], cg.g, j == 0 ? 1 : 0, cudaGraphCondAssignDefault));
  GmresView k = kin;
  k.hflag = nullptr;
  IterLauncher it{p, &o, kprec, mprec, kpoly, kin.R};
  const bool timing = p->timing;
  p->timing = false;  // no event records inside a graph
  hdg::t_capturing = true;      // captured kernels are counted when they run
  hdg::t_captured = 0;
  cudaGraphNode_t prev = nullptr;
  for (int j = 0; j < o.restart; ++j) {
    // all bytes of the tagged union past the used member must be zero
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cg.h[j];
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg.g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(p->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    k.use_cond = (j + 1 < o.restart) ? 1 : 0;
    k.cond = (j + 1 < o.restart) ? cg.h[j + 1] : 0;
    try {
      it.iteration(k, j, p->cap_stream);
      CK(cudaGetLastError());
    } catch (...) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(p->cap_stream, &dummy);
      cudaGetLastError();
      p->timing = timing;
      hdg::t_capturing = false;
      cudaGraphDestroy(cg.g);
      throw;
    }
    cudaGraph_t captured = nullptr;
    CK(cudaStreamEndCapture(p->cap_stream, &captured));
    prev = node;
  }
  p->timing = timing;
  hdg::t_capturing = false;
  cg.kernels_per_iter = hdg::t_captured / std::max(o.restart, 1);
  CK(cudaGraphInstantiate(&cg.exec, cg.g, 0));
  p->graphs.push_back(cg);
  *kernels_per_iter = cg.kernels_per_iter;
  return cg.exec;
}

struct GmresResult {
  int iters = 0, restarts = 0;
  bool converged = false;
  double rel = 0.0;
  hdg_status st = HDG_OK;
};

// Restarted left-preconditioned GMRES(m) for the R right-hand sides b
// (device, n x R); x (device) receives the solution, starting from 0.
//  true_check = 1: accept on the true residual ||b - K64 x|| <= rtol ||b||
//                  (FP64), dividing the cycle tolerance by 10 after a false
//                  stop on the least-squares estimate.
//  true_check = 0: (inner solve) stop when a cycle ends on the estimate, when
//                  the true residual with the solve's own matrix is below
//                  rtol, or when three cycles in a row reduced that residual
//                  by less than 10% (an inexact low-precision operator can
//                  hold the estimate above rtol; the outer refinement
//                  corrects what the inner solve leaves).
GmresResult gmres(hdg_problem p, const hdg_solver_opts& o, int kprec, int mprec, int kpoly, const double* b,
                  double* x, double rtol, int maxit, int true_check, cudaStream_t s) {
  GmresResult out;
  const int R = p->R, m = o.restart;
  const int64_t len = p->ndof * R;
  if (mprec != HDG_FP64 || kprec != HDG_FP64 || kpoly != HDG_FP64) ensure_low(p);   // before any capture
  Ops ops{p, s, R};
  GmresView k = make_view(p, R, m, rtol, maxit);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * len, s));
  CK(cudaMemsetAsync(p->iters, 0, sizeof(int) * R, s));
  CK(cudaMemsetAsync(p->done, 0, sizeof(int) * R, s));
  if (p->dmaxit) set_ints(p, p->dmaxit, maxit, 1, s);
  set_ints(p, p->running, 1, R, s);
  set_dbls(p, p->cfac, 1.0, R, s);
  // ||b|| and ||P^{-1} b||
  launch_norms(k, b, p->bnorm, 0, nullptr, s);
  ops.Pinv(o, mprec, kpoly, b, p->t1, p->running);
  launch_norms(k, p->t1, p->zb, 0, nullptr, s);
  CK(cudaMemcpyAsync(p->res, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  std::vector<double> cf(R, 1.0), last(R, 0.0);
  std::vector<int> done(R, 0), slow(R, 0);
  int total_iters = 0;
  while (true) {
    // true relative residual of the current iterate
    launch_norms(k, p->res, p->rel, 0, p->bnorm, s);
    CK(cudaMemcpyAsync(p->h_dbl, p->rel, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(p->h_int, p->on_estimate, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(p->h_int + kMaxR, p->iters, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    hdg_status est = check_err(p, s);
    if (est != HDG_OK) {
      out.st = est;
      break;
    }
    double worst = 0.0;
    bool all_done = true;
    int mx_it = 0;
    for (int r = 0; r < R; ++r) {
      const double rel = p->h_dbl[r];
      worst = std::max(worst, rel);
      mx_it = std::max(mx_it, p->h_int[kMaxR + r]);
      if (true_check) {
        if (out.restarts > 0 && p->h_int[r] && rel > rtol) cf[r] *= 0.1;
        done[r] = rel <= rtol ? 1 : 0;
      } else {
        if (out.restarts > 0) slow[r] = rel > 0.9 * last[r] ? slow[r] + 1 : 0;
        last[r] = rel;
        done[r] = (out.restarts > 0 && p->h_int[r]) || rel <= rtol || slow[r] >= 3 ? 1 : 0;
      }
      if (!done[r]) all_done = false;
    }
    out.rel = worst;
    total_iters = mx_it;
    if (all_done) {
      out.converged = true;
      break;
    }
    if (total_iters >= maxit) break;
    for (int r = 0; r < R; ++r) {
      p->h_int[r] = done[r];
      p->h_dbl[r] = cf[r];
    }
    CK(cudaMemcpyAsync(p->done, p->h_int, sizeof(int) * R, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->cfac, p->h_dbl, sizeof(double) * R, cudaMemcpyHostToDevice, s));
    // start a cycle: V_0 = P^{-1} res, beta = ||V_0||
    set_ints(p, p->running, 1, R, s);
    ops.Pinv(o, mprec, kpoly, p->res, p->V, nullptr);
    launch_norms(k, p->V, nullptr, 1, nullptr, s);
    // Iterations are enqueued at most kLag steps ahead of the device: before
    // step j the host waits for step j-kLag and stops once its flag says that
    // no right-hand side is still running (no empty launches after convergence).
    constexpr int kLag = 2;
    for (int j = 0; j <= m; ++j) p->h_flag[j] = 1;
    const bool graph = p->use_graphs && !p->timing;
    long long kpi = 0;
    if (graph) CK(cudaGraphLaunch(cycle_graph(p, o, kprec, mprec, kpoly, k, &kpi), s));
    for (int j = 0; j < m && !graph; ++j) {
      if (j >= kLag) {
        CK(cudaEventSynchronize(p->ev_iter[j - kLag]));
        if (!((volatile int*)p->h_flag)[j - kLag]) break;
      }
      double* vj = p->V + (int64_t)j * len;
      double* vn = p->V + (int64_t)(j + 1) * len;
      float* t32 = mprec != HDG_FP64 ? p->t1_32 : nullptr;
      ops.K(kprec, vj, p->t1, EPI_SCALE, nullptr, p->vscale + (int64_t)j * R, p->running, t32);
      ops.Pinv(o, mprec, kpoly, p->t1, vn, p->running, t32);
      orthogonalize(k, o.orth, j, s);
      CK(cudaEventRecord(p->ev_iter[j], s));
    }
    launch_backsolve(k, s);
    launch_xupdate(k, x, s);
    // true residual with the FP64 matrix (outer) or the solve's own matrix (inner)
    ops.K(true_check ? HDG_FP64 : kprec, x, p->res, EPI_RESID, b, nullptr, nullptr);
    out.restarts += 1;
    if (graph) {
      // kernels the cycle graph ran: iterations done (max over RHS) x kernels per iteration
      CK(cudaMemcpyAsync(p->h_int + 2 * kMaxR, p->jend, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int mx = 0;
      for (int r = 0; r < R; ++r) mx = std::max(mx, p->h_int[2 * kMaxR + r]);
      hdg::g_launches.fetch_add(kpi * mx);
    }
  }
  out.iters = total_iters;
  return out;
}

// Host inputs: the caller's buffers are not retained after a call returns,
// so the call waits for its last copy from them (not for the work that uses
// the copies): mark_inputs_read after the copies on their stream `cs`,
// wait_inputs_read before returning.
void mark_inputs_read(hdg_problem p, cudaStream_t cs) {
  if (!p->ev_read) CK(cudaEventCreateWithFlags(&p->ev_read, cudaEventDisableTiming));
  CK(cudaEventRecord(p->ev_read, cs));
}
void wait_inputs_read(hdg_problem p) {
  if (p->ev_read) CK(cudaEventSynchronize(p->ev_read));
}

cudaStream_t copy_stream_of(hdg_problem p) {
  if (!p->copy_stream) CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  return p->copy_stream;
}
cudaEvent_t event_of(cudaEvent_t& e) {
  if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return e;
}
// Device address of a caller's host buffer in pinned, mapped memory of the
// problem's device (the kernels then write host outputs directly, their many
// warps taking the translation misses of a buffer not touched for a while in
// parallel, where a copy engine takes them one after another), or nullptr
// for pageable memory and for memory pinned against another device.
double* mapped_host(hdg_problem p, double* ptr) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.device != p->device) return nullptr;
  return static_cast<double*>(a.devicePointer);
}

// Every stream operation that reads or writes the device copy of the
// Dirichlet values records this event after it, so that a host copy into it
// on the copy stream waits for exactly those operations.
void mark_uD_used(hdg_problem p, cudaStream_t s) { CK(cudaEventRecord(event_of(p->ev_uD_used), s)); }

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* hdg_status_str(hdg_status s) {
  switch (s) {
    case HDG_OK: return "ok";
    case HDG_ERR_ARG: return "invalid argument";
    case HDG_ERR_OOM: return "out of device memory";
    case HDG_ERR_BUDGET: return "memory budget exceeded";
    case HDG_ERR_SINGULAR: return "singular block";
    case HDG_ERR_NOT_CONVERGED: return "not converged";
    case HDG_ERR_BREAKDOWN: return "breakdown";
    case HDG_ERR_NAN: return "NaN or Inf";
    case HDG_ERR_TIMEOUT: return "device wait timed out";
    case HDG_ERR_CUDA: return "CUDA error";
    case HDG_ERR_STATE: return "call out of order";
  }
  return "unknown";
}

hdg_status hdg_problem_create(const hdg_mesh* mesh, int nrhs, int device, hdg_problem* out) {
  if (!mesh || !out) return HDG_ERR_ARG;
  *out = nullptr;
  if (mesh->dim < 2 || mesh->dim > 3 || mesh->n_lfe < 3 || mesh->n_lfe > 8 || mesh->M < 1 || mesh->PE < 1 ||
      mesh->PF < 1 || mesh->n_elem < 1 || mesh->n_face < 1 || !mesh->elem_face || !mesh->face_elem ||
      !mesh->face_dirichlet)
    return HDG_ERR_ARG;
  if (!(nrhs == 1 || nrhs == 2 || nrhs == 4 || nrhs == 8)) return HDG_ERR_ARG;
  hdg_problem p = new (std::nothrow) hdg_problem_s();
  if (!p) return HDG_ERR_OOM;
  try {
    DeviceGuard dg(device);
    p->device = device;
    p->dim = mesh->dim;
    p->D = mesh->dim;
    p->nl = mesh->n_lfe;
    p->M = mesh->M;
    p->PE = mesh->PE;
    p->PF = mesh->PF;
    p->NE = mesh->n_elem;
    p->NF = mesh->n_face;
    p->R = nrhs;
    p->b = p->M * p->PF;
    p->nlb = p->nl * p->b;
    p->ms = 2 * p->nl - 1;
    p->nlPF = p->nl * p->PF;
    p->MPE = p->M * p->PE;
    p->MDPE = p->M * p->D * p->PE;
    if (p->b > 512 || p->nlb > 512) {
      delete p;
      return HDG_ERR_ARG;
    }
    p->h_elem_face.assign(mesh->elem_face, mesh->elem_face + p->NE * p->nl);
    p->h_face_elem.assign(mesh->face_elem, mesh->face_elem + p->NF * 4);
    p->h_face_dir.assign(mesh->face_dirichlet, mesh->face_dirichlet + p->NF);
    for (auto& v : p->h_face_dir) v = v ? 1 : 0;
    CK(cudaMallocHost(&p->h_dbl, sizeof(double) * 4 * kMaxR + 64));
    CK(cudaMallocHost(&p->h_int, sizeof(int) * 4 * kMaxR + 64));
    CK(cudaMallocHost(&p->h_err, sizeof(unsigned) * 4));
    CK(cudaHostAlloc(&p->h_flag, sizeof(int) * (kMaxBasis + 8), cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer((void**)&p->d_flag, p->h_flag, 0));
    for (int i = 0; i < kMaxBasis + 8; ++i) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      p->ev_iter.push_back(e);
    }
    p->d_err = (unsigned*)p->dalloc(sizeof(unsigned) * 4);
    CK(cudaMemset(p->d_err, 0, sizeof(unsigned) * 4));
    hdg_status st = build_maps(p);
    if (st != HDG_OK) {
      hdg_problem_destroy(p);
      return st;
    }
    const int R = p->R, D = p->D, PE = p->PE, MPE = p->MPE, nlb = p->nlb, nlPF = p->nlPF;
    p->d_Kbar = (double*)p->dalloc(sizeof(double) * p->NE * nlb * nlb);
    p->d_rbar = (double*)p->dalloc(sizeof(double) * p->NE * nlb * R);
    p->d_MinvB = (double*)p->dalloc(sizeof(double) * p->NE * D * PE * PE);
    p->d_MinvC = (double*)p->dalloc(sizeof(double) * p->NE * D * PE * nlPF);
    p->d_XF = (double*)p->dalloc(sizeof(double) * p->NE * MPE * nlb);
    p->d_Xr = (double*)p->dalloc(sizeof(double) * p->NE * MPE * R);
    p->d_uhatD = (double*)p->dalloc(sizeof(double) * p->NF * p->b * R);
    CK(cudaMemset(p->d_uhatD, 0, sizeof(double) * p->NF * p->b * R));
    p->condensed.assign(p->NE, 0);
    // condensation chunk: inputs + temporaries of ~1 GiB
    const int64_t per = in_sizes(p).total + tmp_per_elem(p);
    int64_t ch = (int64_t)(kChunkBudget / (per * 8));
    ch = std::max<int64_t>(1, std::min<int64_t>(ch, p->NE));
    p->chunk = ch;
    p->chunk_cap = ch;
    p->d_stage = (double*)p->dalloc(sizeof(double) * ch * in_sizes(p).total);
    p->d_tmp = (double*)p->dalloc(sizeof(double) * ch * tmp_per_elem(p));
    // exponents of the largest batched product of a chunk: nb1 <= max(D, M) items
    // per element, M + N <= 2 * max(nlb, MPE, D * PE, nlPF)
    p->oz_cap = ch * std::max(p->D, p->M) * 2 * std::max({p->nlb, p->MPE, p->D * p->PE, p->nlPF});
    p->d_oz = (uint16_t*)p->dalloc(sizeof(uint16_t) * p->oz_cap);
    p->s64 = padded_stride<double>((int64_t)p->b * p->b);
    p->ld32 = ld_f32(p->b);
    p->ld16 = ld_bf16(p->b);
    p->s32 = (int64_t)p->ld32 * p->b;      // whole 16-byte columns: a multiple of 16 bytes
    p->s16 = (int64_t)p->ld16 * p->b;
    *out = p;
    return HDG_OK;
  } catch (const CudaError& e) {
    hdg_problem_destroy(p);
    return to_status(e);
  } catch (const std::bad_alloc&) {
    hdg_problem_destroy(p);
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_problem_destroy(hdg_problem p) {
  if (!p) return HDG_OK;
  DeviceGuard dg(p->device);
  for (void* q : p->allocs) cudaFree(q);
  p->allocs.clear();
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  for (auto e : p->ev_iter) cudaEventDestroy(e);
  for (auto& cg : p->graphs) {
    if (cg.exec) cudaGraphExecDestroy(cg.exec);
    if (cg.g) cudaGraphDestroy(cg.g);
  }
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->ev_read) cudaEventDestroy(p->ev_read);
  if (p->ev_uD_used) cudaEventDestroy(p->ev_uD_used);
  if (p->ev_uD_copied) cudaEventDestroy(p->ev_uD_copied);
  if (p->ev_rec) cudaEventDestroy(p->ev_rec);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
    if (p->ev_freed[i]) cudaEventDestroy(p->ev_freed[i]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  if (p->h_dbl) cudaFreeHost(p->h_dbl);
  if (p->h_int) cudaFreeHost(p->h_int);
  if (p->h_err) cudaFreeHost(p->h_err);
  delete p;
  return HDG_OK;
}

size_t hdg_problem_device_bytes(hdg_problem p) { return p ? p->bytes : 0; }

size_t hdg_workspace_bytes(const hdg_mesh* mesh, int nrhs, const hdg_solver_opts* opts) {
  if (!mesh) return 0;
  const int64_t NE = mesh->n_elem, NF = mesh->n_face;
  const int64_t b = (int64_t)mesh->M * mesh->PF, nl = mesh->n_lfe, nlb = nl * b, PE = mesh->PE,
                D = mesh->dim, MPE = (int64_t)mesh->M * PE, R = nrhs;
  int64_t nfree = 0;
  for (int64_t f = 0; f < NF; ++f) nfree += mesh->face_dirichlet[f] ? 0 : 1;
  const int64_t ms = 2 * nl - 1;
  int64_t by = 0;
  by += NE * (nlb * nlb + nlb * R + D * PE * PE + D * PE * nl * mesh->PF + MPE * nlb + MPE * R) * 8;
  by += NF * b * R * 8;
  {  // condensation staging + temporaries, sized as hdg_problem_create sizes them
    const int64_t MDPE = MPE * D, nlPF = nl * mesh->PF;
    const int64_t in_total = PE * PE + D * PE * PE + D * PE * nlPF + MPE * MDPE + MPE * MPE + MPE * nlb +
                             nlb * MDPE + nlb * MPE + nlb * nlb + MPE * R + nlb * R;
    const int64_t tmp = tmp_elems(PE, MPE, nlb, R);
    const int64_t ch = std::max<int64_t>(1, std::min<int64_t>(kChunkBudget / ((in_total + tmp) * 8), NE));
    by += ch * (in_total + tmp) * 8 + (16ll << 20);               // + small per-call buffers
    if (NE > ch) by += ch * in_total * 8;                          // second staging buffer (host inputs)
    // exponents of the tensor-core products (16-bit, as hdg_problem_create sizes them)
    const int64_t mx = std::max({nlb, MPE, D * PE, nl * (int64_t)mesh->PF});
    by += ch * std::max<int64_t>(D, mesh->M) * 2 * mx * 2;
  }
  by += nfree * ms * b * b * (8 + 4);                             // K in FP64 + FP32
  if (opts && (opts->poly_prec == HDG_BF16 || opts->inner_prec == HDG_BF16)) by += nfree * ms * b * b * 2;
  by += nfree * b * b * (8 + 4 + 8);                              // BJ
  if (opts && opts->pc == HDG_PC_ASM) by += NE * nlb * nlb * (8 + 8 + 4);
  {  // scratch of the block inverses beyond one CTA's shared memory (Ebar, ASM patches)
    const int nbig = (int)std::max<int64_t>(MPE, (opts && opts->pc == HDG_PC_ASM) ? nlb : 0);
    const int64_t need = inverse_scratch(nbig);
    if (need > 0) by += std::max<int64_t>(1, std::min<int64_t>(NE, (1ll << 27) / need)) * need * 8;
  }
  const int m = opts ? opts->restart : 50;
  by += (int64_t)(m + 12) * nfree * b * R * 8;
  by += NE * nlb * R * 8;
  if ((R == 4 || R == 8) && b <= 32) by += nfree * ms * b * b * 8 + nfree * b * 4;   // K as digits (tensor cores)
  if (opts && opts->inner_prec != HDG_FP64)                       // FP32 vectors of the low-precision preconditioner
    by += (5 * nfree * b + NE * nlb) * R * 4;
  return (size_t)by;
}

hdg_status hdg_condense_strided(hdg_problem p, int64_t e0, int64_t count, const double* const* blocks,
                                const int64_t* elem_stride, int on_device, void* stream) {
  if (!p || !blocks) return HDG_ERR_ARG;
  if (e0 < 0 || count < 0 || e0 + count > p->NE) return HDG_ERR_ARG;
  const InSizes z = in_sizes(p);
  const int64_t sz[11] = {z.Me, z.Bd, z.Cd, z.D, z.E, z.F, z.G, z.H, z.J, z.ru, z.ruh};
  bool sh[11];
  for (int i = 0; i < 11; ++i) {
    if (!blocks[i]) return HDG_ERR_ARG;
    const int64_t st = elem_stride ? elem_stride[i] : sz[i];
    if (st != 0 && st != sz[i]) return HDG_ERR_ARG;
    sh[i] = (st == 0);
  }
  cudaStream_t s = (cudaStream_t)stream;
  bool all_shared = true;
  for (int i = 0; i < 11; ++i) all_shared = all_shared && sh[i];
  try {
    DeviceGuard dg(p->device);
    const auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (all_shared && count > 1) {
      // identical elements: condense element e0 once, then copy its results
      // (Kbar, rbar and the recovery data) to the other elements
      hdg_status st = hdg_condense_strided(p, e0, 1, blocks, elem_stride, on_device, stream);
      if (st != HDG_OK) return st;
      const int64_t per[6] = {(int64_t)p->nlb * p->nlb, (int64_t)p->nlb * p->R, (int64_t)p->D * p->PE * p->PE,
                              (int64_t)p->D * p->PE * p->nlPF, (int64_t)p->MPE * p->nlb, (int64_t)p->MPE * p->R};
      double* base[6] = {p->d_Kbar, p->d_rbar, p->d_MinvB, p->d_MinvC, p->d_XF, p->d_Xr};
      for (int i = 0; i < 6; ++i)
        bcast_copy(base[i] + (e0 + 1) * per[i], base[i] + e0 * per[i], per[i], count - 1, s);
      CK(cudaGetLastError());
      for (int64_t e = e0; e < e0 + count; ++e) {
        if (!p->condensed[e]) {
          p->condensed[e] = 1;
          p->n_condensed++;
        }
      }
      p->assembled = false;
      return HDG_OK;
    }
    // host blocks with several chunks: two staging buffers, the copies on a
    // copy stream ordered against the condensation by events
    const bool overlap = !on_device && count > p->chunk;
    if (overlap) {
      if (!p->d_stage2) p->d_stage2 = (double*)p->dalloc(sizeof(double) * p->chunk * in_sizes(p).total);
      if (!p->copy_stream) CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
      for (int i = 0; i < 2; ++i) {
        if (!p->ev_copied[i]) CK(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming));
        if (!p->ev_freed[i]) CK(cudaEventCreateWithFlags(&p->ev_freed[i], cudaEventDisableTiming));
      }
      if (!p->ev_start) CK(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
      CK(cudaEventRecord(p->ev_start, s));                  // earlier work on the staging buffers
      CK(cudaStreamWaitEvent(p->copy_stream, p->ev_start, 0));
    }
    // with overlapped copies the first chunks ramp up (1/8, 1/4, 1/2 of the
    // staging capacity, then full): only the first, small copy is exposed,
    // and each later copy (faster per element than the condensation) hides
    // behind the condensation of the chunk before it
    int64_t ci = 0, ec = 0;
    for (int64_t c0 = 0; c0 < count; c0 += ec, ++ci) {
      const int64_t cap = (overlap && ci < 3) ? std::max<int64_t>(1, p->chunk >> (3 - ci)) : p->chunk;
      ec = std::min<int64_t>(cap, count - c0);
      const int bsel = (int)(ci & 1);
      const double* dev[11];
      double* st = (overlap && bsel) ? p->d_stage2 : p->d_stage;
      cudaStream_t cs = overlap ? p->copy_stream : s;
      if (overlap && ci >= 2) CK(cudaStreamWaitEvent(cs, p->ev_freed[bsel], 0));   // chunk ci-2 is done with it
      for (int i = 0; i < 11; ++i) {
        const double* base = blocks[i] + (sh[i] ? 0 : c0 * sz[i]);
        const int64_t ncopy = sh[i] ? 1 : ec;
        if (on_device) {
          dev[i] = base;
        } else {
          CK(cudaMemcpyAsync(st, base, sizeof(double) * ncopy * sz[i], kind, cs));
          dev[i] = st;
          st += ncopy * sz[i];
        }
      }
      if (overlap) {
        CK(cudaEventRecord(p->ev_copied[bsel], cs));
        CK(cudaStreamWaitEvent(s, p->ev_copied[bsel], 0));
      }
      if (!on_device) mark_inputs_read(p, cs);
      condense_chunk(p, e0 + c0, ec, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], dev[6], dev[7], dev[8], dev[9],
                     dev[10], sh, s);
      if (overlap) CK(cudaEventRecord(p->ev_freed[bsel], s));
      CK(cudaGetLastError());
      for (int64_t e = e0 + c0; e < e0 + c0 + ec; ++e) {
        if (!p->condensed[e]) {
          p->condensed[e] = 1;
          p->n_condensed++;
        }
      }
    }
    if (!on_device) wait_inputs_read(p);
    collect_timing(p, s);
    p->assembled = false;
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_condense(hdg_problem p, int64_t e0, int64_t count, const double* Me, const double* Bd,
                        const double* Cd, const double* Dm, const double* Em, const double* Fm, const double* Gm,
                        const double* Hm, const double* Jm, const double* ru, const double* ruh, int on_device,
                        void* stream) {
  const double* blocks[11] = {Me, Bd, Cd, Dm, Em, Fm, Gm, Hm, Jm, ru, ruh};
  return hdg_condense_strided(p, e0, count, blocks, nullptr, on_device, stream);
}

// ----------------------------------------------- generated hexahedral blocks
}  // extern "C"
namespace {

template <typename T>
T* grow(hdg_problem p, T*& buf, int64_t& cap, int64_t need) {
  if (need > cap) {
    p->dfree(buf, sizeof(T) * (size_t)cap);
    buf = nullptr;
    cap = 0;
    buf = (T*)p->dalloc(sizeof(T) * (size_t)need);
    cap = need;
  }
  return buf;
}

struct HexDev {
  const double *phi, *dphi, *wq, *dN, *fphi, *fdN, *psi, *wf, *phiT, *fphiT, *b1, *d1;
};

// Validates the shapes, builds and uploads the reference tables for
// (k, nquad) when they change, and uploads the physics.
hdg_status hex_prepare(hdg_problem p, int nquad, const hdg_physics* ph, HexDev* dev, cudaStream_t s) {
  if (!ph || !ph->Cq || nquad < 1 || nquad > 12) return HDG_ERR_ARG;
  if (p->D != 3 || p->nl != 6) return HDG_ERR_ARG;
  int n1 = 1;
  while (n1 * n1 * n1 < p->PE) ++n1;
  if (n1 * n1 * n1 != p->PE || n1 * n1 != p->PF || n1 < 2) return HDG_ERR_ARG;
  const int k = n1 - 1;
  if (p->hex_k != k || p->hex_nq != nquad) {
    p->hex_tab = build_hex_tables(k, nquad);
    const HexTables& T = p->hex_tab;
    const std::vector<double>* parts[12] = {&T.phi, &T.dphi, &T.wq, &T.dN, &T.fphi, &T.fdN, &T.psi, &T.wf,
                                            &T.phiT, &T.fphiT, &T.b1, &T.d1};
    int64_t tot = 0;
    for (auto* v : parts) tot += (int64_t)v->size();
    grow(p, p->d_hextab, p->hextab_cap, tot);
    int64_t off = 0;
    for (auto* v : parts) {
      CK(cudaMemcpyAsync(p->d_hextab + off, v->data(), sizeof(double) * v->size(), cudaMemcpyHostToDevice, s));
      off += (int64_t)v->size();
    }
    CK(cudaStreamSynchronize(s));          // the host tables may change with the next call
    p->hex_k = k;
    p->hex_nq = nquad;
  }
  const HexTables& T = p->hex_tab;
  const double* base = p->d_hextab;
  const double** outs[12] = {&dev->phi, &dev->dphi, &dev->wq, &dev->dN, &dev->fphi, &dev->fdN, &dev->psi,
                             &dev->wf, &dev->phiT, &dev->fphiT, &dev->b1, &dev->d1};
  const std::vector<double>* parts[12] = {&T.phi, &T.dphi, &T.wq, &T.dN, &T.fphi, &T.fdN, &T.psi, &T.wf,
                                          &T.phiT, &T.fphiT, &T.b1, &T.d1};
  for (int i = 0; i < 12; ++i) {
    *outs[i] = base;
    base += parts[i]->size();
  }
  // physics: Cq, Cu, Rr
  const int M = p->M;
  std::vector<double> h((size_t)M * 9 * M + (size_t)M * 3 * M + (size_t)M * M, 0.0);
  std::copy(ph->Cq, ph->Cq + (size_t)M * 9 * M, h.begin());
  if (ph->Cu) std::copy(ph->Cu, ph->Cu + (size_t)M * 3 * M, h.begin() + (size_t)M * 9 * M);
  if (ph->Rr) std::copy(ph->Rr, ph->Rr + (size_t)M * M, h.begin() + (size_t)M * 12 * M);
  if (!p->d_phys) p->d_phys = (double*)p->dalloc(sizeof(double) * (size_t)25 * 13);   // M <= 5
  if (M > 5) return HDG_ERR_ARG;
  CK(cudaMemcpyAsync(p->d_phys, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return HDG_OK;
}

// Generates the blocks of `ec` elements into out[0..8] (Me, Bd, Cd, D..J;
// element strides = the condensation input sizes).
void hex_generate_chunk(hdg_problem p, const HexDev& dev, int64_t ec, const double* verts, const int32_t* perm,
                        const hdg_physics* ph, double* const* out, cudaStream_t s) {
  const HexTables& T = p->hex_tab;
  const int PE = T.PE, PF = T.PF, nq = T.nq, nfq = T.nfq, F4 = 4 * PF;
  double* g = grow(p, p->d_gen, p->gen_cap, ec * hex_gen_scratch(T));
  HexGenDesc d;
  d.count = ec;
  d.M = p->M;
  d.PE = PE;
  d.PF = PF;
  d.nq = nq;
  d.nfq = nfq;
  d.verts = verts;
  d.perm = perm;
  d.phi = dev.phi; d.dphi = dev.dphi; d.wq = dev.wq; d.dN = dev.dN;
  d.fphi = dev.fphi; d.fdN = dev.fdN; d.psi = dev.psi; d.wf = dev.wf;
  d.AW = g;                 g += ec * (int64_t)nq * PE;
  d.GT = g;                 g += ec * (int64_t)3 * PE * nq;
  d.BWN = g;                g += ec * (int64_t)6 * nfq * F4;
  d.PW = g;                 g += ec * (int64_t)6 * nfq * PE;
  d.PsiT = g;               g += ec * (int64_t)6 * PF * nfq;
  d.Mf = g;                 g += ec * (int64_t)PE * PE;
  d.EF4 = g;                g += ec * (int64_t)6 * PE * F4;
  d.FF4 = g;
  d.Cq = p->d_phys;
  d.Cu = p->d_phys + (size_t)p->M * 9 * p->M;
  d.Rr = p->d_phys + (size_t)p->M * 12 * p->M;
  d.tau = ph->tau;
  d.Me = out[0];
  d.Sd = out[1];
  d.Cd = out[2]; d.Dm = out[3]; d.Em = out[4]; d.Fm = out[5]; d.Gm = out[6]; d.Hm = out[7]; d.Jm = out[8];
  d.err = p->d_err;
  const int n = (int)ec;
  // M^e and B_d: sum factorisation of the tensor-product rule where its
  // shared memory allows, else M^e = Phi^T (W Phi), B_d = G_d^T (W Phi)
  if (p->hex_sf && hex_mass_grad_sf(d, T.n1, T.nq1, dev.b1, dev.d1, out[0], out[1], s)) {
    hex_face_geometry(d, s);
  } else {
    hex_geometry(d, s);
    gemm_c(p, gd(PE, PE, nq, dev.phiT, nq, 0, 0, d.AW, PE, (int64_t)nq * PE, 0, out[0], PE, (int64_t)PE * PE, 0,
                1.0, 0.0, n, 1), s);
    gemm_c(p, gd(PE, PE, nq, d.GT, nq, (int64_t)3 * PE * nq, (int64_t)PE * nq, d.AW, PE, (int64_t)nq * PE, 0,
                out[1], PE, (int64_t)3 * PE * PE, (int64_t)PE * PE, 1.0, 0.0, n, 3), s);
  }
  // Mf = sum over faces Phi_f^T (W Phi_f)
  gemm_c(p, gd(PE, PE, 6 * nfq, dev.fphiT, 6 * nfq, 0, 0, d.PW, PE, (int64_t)6 * nfq * PE, 0, d.Mf, PE,
              (int64_t)PE * PE, 0, 1.0, 0.0, n, 1), s);
  // per face: [EF | EFN_d] = Phi_f^T [W psi | W n_d psi],  [FF | FFN_d] = psi^T [W psi | W n_d psi]
  gemm_c(p, gd(PE, F4, nfq, dev.fphiT, 6 * nfq, 0, nfq, d.BWN, F4, (int64_t)6 * nfq * F4, (int64_t)nfq * F4, d.EF4,
              F4, (int64_t)6 * PE * F4, (int64_t)PE * F4, 1.0, 0.0, n, 6), s);
  gemm_c(p, gd(PF, F4, nfq, d.PsiT, nfq, (int64_t)6 * PF * nfq, (int64_t)PF * nfq, d.BWN, F4, (int64_t)6 * nfq * F4,
              (int64_t)nfq * F4, d.FF4, F4, (int64_t)6 * PF * F4, (int64_t)PF * F4, 1.0, 0.0, n, 6), s);
  hex_expand(d, s);
}

// device copies of this chunk's vertices and face permutations
void hex_inputs(hdg_problem p, int64_t c0, int64_t ec, const double* verts, const int32_t* perm, int on_device,
                const double** dv, const int32_t** dp, cudaStream_t s) {
  const int64_t nv = ec * 24, np = ec * 6 * (int64_t)p->PF;
  if (on_device) {
    *dv = verts + c0 * 24;
    *dp = perm + c0 * 6 * (int64_t)p->PF;
    return;
  }
  unsigned char* b = grow(p, p->d_genin, p->genin_cap, (int64_t)(sizeof(double) * nv + sizeof(int32_t) * np));
  CK(cudaMemcpyAsync(b, verts + c0 * 24, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b + sizeof(double) * nv, perm + c0 * 6 * (int64_t)p->PF, sizeof(int32_t) * np,
                     cudaMemcpyHostToDevice, s));
  *dv = (const double*)b;
  *dp = (const int32_t*)(b + sizeof(double) * nv);
}


}  // namespace
extern "C" {

hdg_status hdg_condense_hex(hdg_problem p, int64_t e0, int64_t count, int nquad, const double* verts,
                            const int32_t* face_perm, const hdg_physics* phys, const double* ru, const double* ruh,
                            int on_device, void* stream) {
  if (!p || !verts || !face_perm || !ru || !ruh) return HDG_ERR_ARG;
  if (e0 < 0 || count < 0 || e0 + count > p->NE) return HDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    HexDev dev;
    hdg_status st = hex_prepare(p, nquad, phys, &dev, s);
    if (st != HDG_OK) return st;
    const InSizes z = in_sizes(p);
    const int64_t sz[11] = {z.Me, z.Bd, z.Cd, z.D, z.E, z.F, z.G, z.H, z.J, z.ru, z.ruh};
    const bool sh[11] = {false, false, false, false, false, false, false, false, false, false, false};
    // host inputs with several chunks: each chunk's vertices, load vectors and
    // face permutations go to one of two device buffers on the copy stream,
    // ordered against the generation and condensation by events; the first
    // chunks ramp up (1/8, 1/4, 1/2 of a chunk) so that only a small first
    // copy is exposed
    const bool overlap = !on_device && count > p->chunk;
    const int64_t in_per = 24 + sz[9] + sz[10];                 // doubles per element, then the permutation
    if (overlap) {
      for (int i = 0; i < 2; ++i)
        grow(p, p->d_hexin[i], p->hexin_cap[i],
             p->chunk * (int64_t)(sizeof(double) * in_per + sizeof(int32_t) * 6 * p->PF));
      if (!p->copy_stream) CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
      for (int i = 0; i < 2; ++i) {
        if (!p->ev_copied[i]) CK(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming));
        if (!p->ev_freed[i]) CK(cudaEventCreateWithFlags(&p->ev_freed[i], cudaEventDisableTiming));
      }
      if (!p->ev_start) CK(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
      CK(cudaEventRecord(p->ev_start, s));                  // earlier work on the buffers
      CK(cudaStreamWaitEvent(p->copy_stream, p->ev_start, 0));
    }
    int64_t ci = 0, ec = 0;
    for (int64_t c0 = 0; c0 < count; c0 += ec, ++ci) {
      const int64_t cap = (overlap && ci < 3) ? std::max<int64_t>(1, p->chunk >> (3 - ci)) : p->chunk;
      ec = std::min<int64_t>(cap, count - c0);
      double* stg = p->d_stage;
      double* out[11];
      for (int i = 0; i < 11; ++i) {
        out[i] = stg;
        stg += ec * sz[i];
      }
      const double* dv;
      const int32_t* dp;
      const double* dru = ru + c0 * sz[9];
      const double* druh = ruh + c0 * sz[10];
      const int bsel = (int)(ci & 1);
      if (overlap) {
        cudaStream_t cs = p->copy_stream;
        if (ci >= 2) CK(cudaStreamWaitEvent(cs, p->ev_freed[bsel], 0));    // chunk ci-2 is done with it
        double* b = reinterpret_cast<double*>(p->d_hexin[bsel]);
        double* bv = b;
        double* bru = bv + ec * 24;
        double* bruh = bru + ec * sz[9];
        int32_t* bp = reinterpret_cast<int32_t*>(bruh + ec * sz[10]);
        CK(cudaMemcpyAsync(bv, verts + c0 * 24, sizeof(double) * ec * 24, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(bru, dru, sizeof(double) * ec * sz[9], cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(bruh, druh, sizeof(double) * ec * sz[10], cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(bp, face_perm + c0 * 6 * (int64_t)p->PF, sizeof(int32_t) * ec * 6 * p->PF,
                           cudaMemcpyHostToDevice, cs));
        CK(cudaEventRecord(p->ev_copied[bsel], cs));
        CK(cudaStreamWaitEvent(s, p->ev_copied[bsel], 0));
        mark_inputs_read(p, cs);
        dv = bv;
        dp = bp;
        dru = bru;
        druh = bruh;
      } else {
        hex_inputs(p, c0, ec, verts, face_perm, on_device, &dv, &dp, s);
        if (!on_device) {
          CK(cudaMemcpyAsync(out[9], dru, sizeof(double) * ec * sz[9], cudaMemcpyHostToDevice, s));
          CK(cudaMemcpyAsync(out[10], druh, sizeof(double) * ec * sz[10], cudaMemcpyHostToDevice, s));
          dru = out[9];
          druh = out[10];
          mark_inputs_read(p, s);
        }
      }
      hex_generate_chunk(p, dev, ec, dv, dp, phys, out, s);
      condense_chunk(p, e0 + c0, ec, out[0], out[1], out[2], out[3], out[4], out[5], out[6], out[7], out[8], dru,
                     druh, sh, s);
      if (overlap) CK(cudaEventRecord(p->ev_freed[bsel], s));
      CK(cudaGetLastError());
      for (int64_t e = e0 + c0; e < e0 + c0 + ec; ++e) {
        if (!p->condensed[e]) {
          p->condensed[e] = 1;
          p->n_condensed++;
        }
      }
    }
    if (!on_device) wait_inputs_read(p);
    collect_timing(p, s);
    p->assembled = false;
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_hex_blocks(hdg_problem p, int64_t count, int nquad, const double* verts, const int32_t* face_perm,
                          const hdg_physics* phys, double* const* out, int on_device, void* stream) {
  if (!p || !verts || !face_perm || !out || count < 0) return HDG_ERR_ARG;
  for (int i = 0; i < 9; ++i)
    if (!out[i]) return HDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    HexDev dev;
    hdg_status st = hex_prepare(p, nquad, phys, &dev, s);
    if (st != HDG_OK) return st;
    const InSizes z = in_sizes(p);
    const int64_t sz[9] = {z.Me, z.Bd, z.Cd, z.D, z.E, z.F, z.G, z.H, z.J};
    for (int64_t c0 = 0; c0 < count; c0 += p->chunk) {
      const int64_t ec = std::min<int64_t>(p->chunk, count - c0);
      double* o[9];
      for (int i = 0; i < 9; ++i) o[i] = out[i] + c0 * sz[i];
      const double* dv;
      const int32_t* dp;
      hex_inputs(p, c0, ec, verts, face_perm, on_device, &dv, &dp, s);
      hex_generate_chunk(p, dev, ec, dv, dp, phys, o, s);
      CK(cudaGetLastError());
    }
    return check_err(p, s);
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_set_dirichlet(hdg_problem p, const double* uhatD, int on_device, void* stream) {
  if (!p || !uhatD) return HDG_ERR_ARG;
  try {
    DeviceGuard dg(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * p->NF * p->b * p->R;
    if (on_device) {
      CK(cudaMemcpyAsync(p->d_uhatD, uhatD, bytes, cudaMemcpyDeviceToDevice, s));
      mark_uD_used(p, s);
    } else {
      // host values: copied on the copy stream once the earlier operations on
      // the device copy are done, so the copy overlaps whatever else is still
      // queued on `stream` (the end of a condensation); `stream` waits for it,
      // and the call returns once the caller's buffer has been read
      cudaStream_t cs = copy_stream_of(p);
      if (p->ev_uD_used) CK(cudaStreamWaitEvent(cs, p->ev_uD_used, 0));
      CK(cudaMemcpyAsync(p->d_uhatD, uhatD, bytes, cudaMemcpyHostToDevice, cs));
      CK(cudaEventRecord(event_of(p->ev_uD_copied), cs));
      CK(cudaStreamWaitEvent(s, p->ev_uD_copied, 0));
      mark_uD_used(p, s);
      CK(cudaEventSynchronize(p->ev_uD_copied));
    }
    p->assembled = false;
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_assemble(hdg_problem p, const hdg_solver_opts* opts, void* stream) {
  if (!p) return HDG_ERR_ARG;
  if (p->n_condensed != p->NE) return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    const int64_t rows = std::max<int64_t>(p->nnzb, 1);
    if (!p->K64) p->K64 = (double*)p->dalloc(sizeof(double) * rows * p->s64);
    if (!p->K32) {
      p->K32 = (float*)p->dalloc(sizeof(float) * rows * p->s32);
      CK(cudaMemsetAsync(p->K32, 0, sizeof(float) * rows * p->s32, s));   // padding rows stay 0
    }
    const bool need16 = opts && (opts->poly_prec == HDG_BF16 || opts->inner_prec == HDG_BF16);
    if (need16 && !p->K16) {
      p->K16 = (__nv_bfloat16*)p->dalloc(sizeof(__nv_bfloat16) * rows * p->s16);
      CK(cudaMemsetAsync(p->K16, 0, sizeof(__nv_bfloat16) * rows * p->s16, s));
    }
    if (!p->d_r) p->d_r = (double*)p->dalloc(sizeof(double) * p->ndof * p->R);
    AssembleDesc d{};
    d.Kbar = p->d_Kbar;
    d.rbar = p->d_rbar;
    d.uhatD = p->d_uhatD;
    d.nlb = p->nlb;
    d.b = p->b;
    d.nl = p->nl;
    d.R = p->R;
    d.max_slots = p->ms;
    d.n_free = p->nfree;
    d.slot_e = p->d_slot_e;
    d.slot_lr = p->d_slot_lr;
    d.slot_lc = p->d_slot_lc;
    d.diag2 = p->d_diag2;
    d.rhs_src = p->d_rhs_src;
    d.elem_face = p->d_elem_face;
    d.face_dir = p->d_face_dir;
    d.rowptr = p->d_rowptr;
    d.K64 = p->K64;
    d.s64 = p->s64;
    d.K32 = p->K32;
    d.s32 = p->s32;
    d.ld32 = p->ld32;
    d.K16 = p->K16;
    d.s16 = p->s16;
    d.ld16 = p->ld16;
    d.r = p->d_r;
    assemble(d, s);
    mark_uD_used(p, s);
    // FP64 products with several right-hand sides run on the tensor cores
    // from the blocks as exact digits (rebuilt with every assembly)
    p->kdig_ready = false;
    {
      BlockRowDesc kd{};
      kd.prec = HDG_FP64;
      kd.R = p->R;
      kd.b_rows = p->b;
      kd.bc = p->b;
      kd.max_slots = p->ms;
      kd.epi = EPI_STORE;
      if (tc_supported(kd) && p->nfree > 0) {
        if (!p->kdig) {
          std::vector<int64_t> doff(p->nfree + 1);
          const int64_t bytes = tc_digit_layout(p->h_rowptr.data(), p->nfree, p->b, p->b, doff.data());
          p->kdig = (unsigned char*)p->dalloc((size_t)std::max<int64_t>(bytes, 16));
          p->kex = (int32_t*)p->dalloc(sizeof(int32_t) * p->nfree * p->b);
          p->d_kdoff = (int64_t*)p->dalloc(sizeof(int64_t) * (p->nfree + 1));
          CK(cudaMemcpyAsync(p->d_kdoff, doff.data(), sizeof(int64_t) * (p->nfree + 1), cudaMemcpyHostToDevice, s));
          CK(cudaStreamSynchronize(s));        // doff is a host temporary
        }
        kd.blk = p->K64;
        kd.blk_stride = p->s64;
        kd.rowptr = p->d_rowptr;
        kd.nbr = p->d_nbr;
        kd.cnt = p->d_cnt;
        kd.n_units = p->nfree;
        kd.ld = p->b;
        kd.err = p->d_err;
        tc_split(kd, p->kdig, p->d_kdoff, p->kex, s);
        p->kdig_ready = true;
      }
    }
    CK(cudaGetLastError());
    hdg_status st = check_err(p, s);
    if (st != HDG_OK) return st;
    p->assembled = true;
    p->pc_ready = -1;
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_setup_precond(hdg_problem p, const hdg_solver_opts* o, const double* v0, void* stream) {
  if (!p || !o) return HDG_ERR_ARG;
  if (!p->assembled) return HDG_ERR_STATE;
  if (o->pc < HDG_PC_NONE || o->pc > HDG_PC_ASM || o->poly < 0 || o->poly > 2) return HDG_ERR_ARG;
  if (o->poly != HDG_POLY_NONE && (o->poly_degree < 1 || o->poly_degree > kMaxPoly || !v0)) return HDG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    const int b = p->b;
    const bool need16 = (o->poly_prec == HDG_BF16 || o->inner_prec == HDG_BF16);
    if (o->pc == HDG_PC_BJ) {
      if (!p->d_bjtmp) p->d_bjtmp = (double*)p->dalloc(sizeof(double) * p->nfree * b * b);
      double* tmp = p->d_bjtmp;
      extract_diag(p->K64, p->s64, p->d_rowptr, b, p->nfree, tmp, s);
      inverse_any(p, tmp, b, (int64_t)b * b, p->nfree, s);
      p->bs64 = padded_stride<double>((int64_t)b * b);
      p->bs32 = (int64_t)p->ld32 * b;
      p->bs16 = (int64_t)p->ld16 * b;
      if (!p->bj64) p->bj64 = (double*)p->dalloc(sizeof(double) * p->nfree * p->bs64);
      if (!p->bj32) {
        p->bj32 = (float*)p->dalloc(sizeof(float) * p->nfree * p->bs32);
        CK(cudaMemsetAsync(p->bj32, 0, sizeof(float) * p->nfree * p->bs32, s));
      }
      if (need16 && !p->bj16) {
        p->bj16 = (__nv_bfloat16*)p->dalloc(sizeof(__nv_bfloat16) * p->nfree * p->bs16);
        CK(cudaMemsetAsync(p->bj16, 0, sizeof(__nv_bfloat16) * p->nfree * p->bs16, s));
      }
      pack_blocks(tmp, b, p->nfree, p->bj64, p->bs64, p->bj32, p->bs32, p->ld32, p->bj16, p->bs16, p->ld16, s);
      hdg_status st = check_err(p, s);
      if (st != HDG_OK) return st;
    } else if (o->pc == HDG_PC_ASM) {
      const int nlb = p->nlb;
      if (!p->d_asmP) p->d_asmP = (double*)p->dalloc(sizeof(double) * p->NE * nlb * nlb);
      double* P = p->d_asmP;
      asm_build(p->d_Kbar, nlb, b, p->nl, p->NE, p->d_asm_lf, p->d_asm_cnt, p->d_asm_face_free, p->K64, p->s64,
                p->d_rowptr, P, s);
      inverse_any(p, P, nlb, (int64_t)nlb * nlb, p->NE, s);
      p->as_s64 = padded_stride<double>((int64_t)nlb * b);
      p->as_ld32 = ld_f32(nlb);
      p->as_ld16 = ld_bf16(nlb);
      p->as_s32 = (int64_t)p->as_ld32 * b;
      p->as_s16 = (int64_t)p->as_ld16 * b;
      const int64_t npan = std::max<int64_t>(p->asm_nblk, 1);
      if (!p->as64) p->as64 = (double*)p->dalloc(sizeof(double) * npan * p->as_s64);
      if (!p->as32) {
        p->as32 = (float*)p->dalloc(sizeof(float) * npan * p->as_s32);
        CK(cudaMemsetAsync(p->as32, 0, sizeof(float) * npan * p->as_s32, s));
      }
      if (need16 && !p->as16) {
        p->as16 = (__nv_bfloat16*)p->dalloc(sizeof(__nv_bfloat16) * npan * p->as_s16);
        CK(cudaMemsetAsync(p->as16, 0, sizeof(__nv_bfloat16) * npan * p->as_s16, s));
      }
      asm_pack(P, nlb, b, p->nl, p->NE, p->d_asm_rowptr, p->as64, p->as_s64, p->as32, p->as_s32, p->as_ld32, p->as16,
               p->as_s16, p->as_ld16, s);
      hdg_status st = check_err(p, s);
      if (st != HDG_OK) return st;
    }
    p->pc_ready = o->pc;
    p->poly_n = 0;
    if (o->poly != HDG_POLY_NONE) p->poly_gen++;    // cycle graphs hold the coefficients by value
    p->poly_kind = o->poly;
    if (o->poly != HDG_POLY_NONE) {
      // one Arnoldi(P) cycle with MGS on A = M^{-1} K (FP64) from v0   (Sec. 4.7)
      const int P = o->poly_degree;
      const int Pa = (o->poly == HDG_POLY_CHEBYSHEV) ? std::max(P, 10) : P;
      ensure_workspace(p, std::max(Pa, o->restart));
      Ops ops{p, s, 1};
      GmresView k = make_view(p, 1, Pa, 0.0, 1 << 30);
      k.chunk = gmres_chunk(p->ndof);
      if (p->dmaxit) set_ints(p, p->dmaxit, 1 << 30, 1, s);
      // Arnoldi variant of the finalize step: the H column is stored unrotated
      CK(cudaMemcpyAsync(p->V, v0, sizeof(double) * p->ndof, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemsetAsync(p->iters, 0, sizeof(int), s));
      CK(cudaMemsetAsync(p->done, 0, sizeof(int), s));
      CK(cudaMemsetAsync(p->H, 0, sizeof(double) * (Pa + 1) * Pa, s));
      set_dbls(p, p->cfac, 1.0, 1, s);
      set_dbls(p, p->zb, 0.0, 1, s);
      launch_norms(k, p->V, nullptr, 1, nullptr, s);   // vscale_0 = 1/||v0||, running = 1
      int Peff = Pa;
      for (int j = 0; j < Pa; ++j) {
        double* vj = p->V + (int64_t)j * p->ndof;
        double* vn = p->V + (int64_t)(j + 1) * p->ndof;
        ops.K(HDG_FP64, vj, p->t1, EPI_SCALE, nullptr, p->vscale + j, nullptr);
        ops.Minv(o->pc, HDG_FP64, p->t1, vn, nullptr);
        for (int i = 0; i <= j; ++i) {
          launch_dots(k, vn, i, i + 1, s);
          launch_update(k, vn, i, i + 1, j, 0, i == j ? 2 : 0, s);
        }
        CK(cudaMemcpyAsync(p->h_int, p->running, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!p->h_int[0]) {
          Peff = j + 1;
          break;
        }
      }
      if (!p->d_poly) p->d_poly = (double*)p->dalloc(sizeof(double) * (2 * kMaxPoly + 2));
      double* d_re = p->d_poly;
      double* d_im = p->d_poly + kMaxPoly;
      int* d_n = (int*)(p->d_poly + 2 * kMaxPoly);
      launch_ritz_leja(p->H, Pa, Peff, o->poly == HDG_POLY_GMRES ? 1 : 0, d_re, d_im, d_n, p->d_err, s);
      std::vector<double> hb(2 * kMaxPoly + 1);
      CK(cudaMemcpyAsync(hb.data(), d_re, sizeof(double) * (2 * kMaxPoly + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      hdg_status st = check_err(p, s);
      if (st != HDG_OK) return st;
      int nth = 0;
      std::memcpy(&nth, &hb[2 * kMaxPoly], sizeof(int));
      if (o->poly == HDG_POLY_GMRES) {
        p->th_re.assign(hb.begin(), hb.begin() + nth);
        p->th_im.assign(hb.begin() + kMaxPoly, hb.begin() + kMaxPoly + nth);
        p->poly_n = nth;
      } else {
        double lo = 1e300, hi = -1e300;
        for (int i = 0; i < nth; ++i) {
          lo = std::min(lo, hb[i]);
          hi = std::max(hi, hb[i]);
        }
        p->cheb_a = 0.9 * lo;
        p->cheb_b = 1.1 * hi;
        p->poly_n = P;
      }
    }
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_solve(hdg_problem p, const hdg_solver_opts* o, void* stream, hdg_solve_info* info) {
  if (!p || !o) return HDG_ERR_ARG;
  if (!p->assembled || p->pc_ready != o->pc) return HDG_ERR_STATE;
  if (o->restart < 1 || o->restart + 1 > kMaxBasis || o->max_iters < 1 || !(o->rtol > 0.0)) return HDG_ERR_ARG;
  if (o->poly != HDG_POLY_NONE && (p->poly_n == 0 || p->poly_kind != o->poly)) return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    ensure_workspace(p, o->restart);
    p->ev_used = 0;
    hdg_solve_info inf{};
    hdg_status st = HDG_OK;
    if (o->inner_prec == HDG_FP64 || o->max_outer == -1 || o->max_outer == -2) {
      // plain FP64 GMRES; or (max_outer = -1) one restarted GMRES whose cycles
      // run on the low-precision blocks and restart from the FP64 residual;
      // or (max_outer = -2) FP64 GMRES with the FP64 operator whose
      // preconditioner alone runs on low-precision blocks
      int kp = o->inner_prec, mp = o->inner_prec;
      int pp = (kp != HDG_FP64 && o->poly_prec == HDG_BF16) ? HDG_BF16 : kp;
      if (o->max_outer == -2) {
        kp = HDG_FP64;
        pp = o->poly_prec;
      }
      GmresResult g = gmres(p, *o, kp, mp, pp, p->d_r, p->d_x, o->rtol, o->max_iters, 1, s);
      inf.iters = g.iters;
      inf.restarts = g.restarts;
      inf.converged = g.converged ? 1 : 0;
      inf.rel_resid = g.rel;
      st = g.st != HDG_OK ? g.st : (g.converged ? HDG_OK : HDG_ERR_NOT_CONVERGED);
    } else {
      // FP64 iterative refinement around a low-precision inner GMRES
      const int64_t len = p->ndof * p->R;
      const int kp = o->inner_prec, pp = (o->poly_prec == HDG_BF16) ? HDG_BF16 : kp;
      Ops ops{p, s, p->R};
      GmresView k = make_view(p, p->R, o->restart, o->rtol, o->max_iters);
      CK(cudaMemsetAsync(p->d_x, 0, sizeof(double) * len, s));
      CK(cudaMemcpyAsync(p->bo, p->d_r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
      double* bnorm0 = p->pw;   // keep ||b|| of the original system
      launch_norms(k, p->d_r, bnorm0, 0, nullptr, s);
      int total = 0, outer = 0;
      double rel = 1.0;
      bool conv = false;
      const int max_outer = o->max_outer > 0 ? o->max_outer : 20;
      while (outer < max_outer) {
        launch_norms(k, p->bo, p->rel, 0, bnorm0, s);
        CK(cudaMemcpyAsync(p->h_dbl, p->rel, sizeof(double) * p->R, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        rel = 0.0;
        for (int r = 0; r < p->R; ++r) rel = std::max(rel, p->h_dbl[r]);
        if (rel <= o->rtol) {
          conv = true;
          break;
        }
        if (total >= o->max_iters) break;
        const double itol = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-4;
        GmresResult g = gmres(p, *o, kp, kp, pp, p->bo, p->xo, itol, o->max_iters - total, 0, s);
        total += g.iters;
        if (g.st != HDG_OK) {
          st = g.st;
          break;
        }
        launch_axpby(p->d_x, p->xo, 1.0, 1.0, len, nullptr, p->R, s);          // x += d
        ops.K(HDG_FP64, p->d_x, p->bo, EPI_RESID, p->d_r, nullptr, nullptr);  // r = b - K x (FP64)
        ++outer;
      }
      inf.iters = total;
      inf.outer = outer;
      inf.converged = conv ? 1 : 0;
      inf.rel_resid = rel;
      if (st == HDG_OK) st = conv ? HDG_OK : HDG_ERR_NOT_CONVERGED;
    }
        collect_timing(p, s);
    if (info) *info = inf;
    return st;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_solve_batch(hdg_problem* probs, int count, const hdg_solver_opts* o, void* stream,
                           hdg_solve_info* infos) {
  if (!probs || !o || count < 1 || count > kMaxBatch) return HDG_ERR_ARG;
  if (o->restart < 1 || o->restart + 1 > kMaxBasis || o->max_iters < 1 || !(o->rtol > 0.0)) return HDG_ERR_ARG;
  if (o->poly != HDG_POLY_NONE || (o->pc != HDG_PC_NONE && o->pc != HDG_PC_BJ) || o->orth != HDG_ORTH_CGS)
    return HDG_ERR_ARG;
  const bool mixed = o->inner_prec != HDG_FP64;
  if (mixed && (o->inner_prec != HDG_FP32 || o->max_outer != -1)) return HDG_ERR_ARG;
  const int dev = probs[0] ? probs[0]->device : -1;
  for (int i = 0; i < count; ++i) {
    hdg_problem p = probs[i];
    if (!p || p->device != dev) return HDG_ERR_ARG;
    if (!p->assembled || p->pc_ready != o->pc) return HDG_ERR_STATE;
    for (int j = 0; j < i; ++j)
      if (probs[j] == p) return HDG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  void* dmem = nullptr;
  try {
    DeviceGuard dg(dev);
    const int m = o->restart;
    std::vector<BatchItem> items(count);
    std::vector<int64_t> pre(4 * count);
    int64_t rows = 0, elems = 0, chunks = 0, groups = 0;
    for (int i = 0; i < count; ++i) {
      hdg_problem p = probs[i];
      ensure_workspace(p, m);
      if (mixed) ensure_low(p);
      BatchItem& it = items[i];
      it.len = p->ndof * p->R;
      it.nchunks = batch_chunks(it.len);
      if (it.nchunks > 1024) return HDG_ERR_ARG;        // the problem's reduction scratch holds 1024 chunks
      if (p->b > batch_max_b()) return HDG_ERR_ARG;     // a face's rows share one CTA
      it.nfree = p->nfree;
      it.b = p->b;
      it.R = p->R;
      it.ms = p->ms;
      it.pc = o->pc;
      it.kprec = mixed ? HDG_FP32 : HDG_FP64;
      it.ld32 = p->ld32;
      it.K64 = p->K64;
      it.s64 = p->s64;
      it.K32 = p->K32;
      it.s32 = p->s32;
      it.rowptr = p->d_rowptr;
      it.nbr = p->d_nbr;
      it.cnt = p->d_cnt;
      it.bj64 = p->bj64;
      it.bs64 = p->bs64;
      it.bj32 = p->bj32;
      it.bs32 = p->bs32;
      it.rhs = p->d_r;
      it.x = p->d_x;
      it.res = p->res;
      it.t1 = p->t1;
      it.x32 = p->x32;
      it.t32 = p->t1_32;
      it.V = p->V;
      it.vscale = p->vscale;
      it.H = p->H;
      it.g = p->g;
      it.cs = p->cs;
      it.sn = p->sn;
      it.hcol = p->hcol;
      it.htmp = p->htmp;
      it.ycoef = p->ycoef;
      it.part = p->partial;
      it.bnorm = p->bnorm;
      it.zb = p->zb;
      it.rel = p->rel;
      it.cfac = p->cfac;
      it.tolabs = p->tolabs;
      it.running = p->running;
      it.done = p->done;
      it.iters = p->iters;
      it.jend = p->jend;
      it.on_est = p->on_estimate;
      it.done_all = p->bdone;
      pre[i] = rows;
      pre[count + i] = elems;
      pre[2 * count + i] = chunks;
      pre[3 * count + i] = groups;
      rows += p->nfree * p->b;
      elems += it.len;
      chunks += it.nchunks;
      groups += batch_layout(p->nfree, p->b, p->ld32, p->R, mixed, &it.sp, &it.fpc);
    }
    // items, prefix sums and the grid-barrier words in one stream-ordered allocation
    const size_t items_bytes = sizeof(BatchItem) * count, pre_bytes = sizeof(int64_t) * 4 * count;
    const size_t bar_off = (items_bytes + pre_bytes + 255) / 256 * 256;
    CK(cudaMallocAsync(&dmem, bar_off + 256, s));
    CK(cudaMemcpyAsync(dmem, items.data(), items_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((char*)dmem + items_bytes, pre.data(), pre_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync((char*)dmem + bar_off, 0, 256, s));
    BatchDesc B{};
    B.items = static_cast<BatchItem*>(dmem);
    B.n = count;
    B.m = m;
    B.maxit = o->max_iters;
    B.rtol = o->rtol;
    B.rows_total = rows;
    B.elems_total = elems;
    B.chunks_total = chunks;
    B.groups_total = groups;
    const int64_t* dpre = reinterpret_cast<const int64_t*>((char*)dmem + items_bytes);
    B.row_pre = dpre;
    B.elem_pre = dpre + count;
    B.chunk_pre = dpre + 2 * count;
    B.group_pre = dpre + 3 * count;
    B.bar = (char*)dmem + bar_off;
    B.err = probs[0]->d_err;
    int rmax = 1;
    for (int i = 0; i < count; ++i) rmax = std::max(rmax, probs[i]->R);
    if (!batch_gmres(B, rmax, s)) {
      cudaGetLastError();
      cudaFreeAsync(dmem, s);
      return HDG_ERR_CUDA;
    }
    CK(cudaFreeAsync(dmem, s));
    dmem = nullptr;
    hdg_status st_all = HDG_OK;
    for (int i = 0; i < count; ++i) {
      hdg_problem p = probs[i];
      const int R = p->R;
      CK(cudaMemcpyAsync(p->h_dbl, p->rel, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(p->h_int, p->iters, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(p->h_int + kMaxR, p->done, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      hdg_solve_info inf{};
      bool conv = true;
      for (int r = 0; r < R; ++r) {
        inf.iters = std::max(inf.iters, p->h_int[r]);
        inf.rel_resid = std::max(inf.rel_resid, p->h_dbl[r]);
        conv = conv && p->h_int[kMaxR + r];
      }
      inf.converged = conv ? 1 : 0;
      if (infos) infos[i] = inf;
      if (i == 0) {
        const hdg_status e = check_err(p, s);
        if (e != HDG_OK) return e;
      }
      if (!conv && st_all == HDG_OK) st_all = HDG_ERR_NOT_CONVERGED;
    }
    return st_all;
  } catch (const CudaError& e) {
    if (dmem) cudaFreeAsync(dmem, s);
    return to_status(e);
  } catch (const std::bad_alloc&) {
    if (dmem) cudaFreeAsync(dmem, s);
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_get_trace(hdg_problem p, double* uhat, int on_device, void* stream) {
  if (!p || !uhat) return HDG_ERR_ARG;
  if (!p->d_x) return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    const int64_t n = p->NF * p->b * p->R;
    double* mapped = on_device ? nullptr : mapped_host(p, uhat);
    if (!on_device && !mapped && !p->d_full) p->d_full = (double*)p->dalloc(sizeof(double) * n);
    double* full = on_device ? uhat : (mapped ? mapped : p->d_full);
    expand_trace(p->d_x, p->d_uhatD, p->d_free_of_face, p->NF, p->b, p->R, full, s);
    mark_uD_used(p, s);
    if (mapped) {
      CK(cudaStreamSynchronize(s));
    } else if (!on_device) {
      CK(cudaMemcpyAsync(uhat, full, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_recover(hdg_problem p, double* u, double* q, int on_device, void* stream) {
  if (!p || !u || !q) return HDG_ERR_ARG;
  if (!p->d_x) return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    const int64_t nu = p->NE * p->MPE * p->R, nq = p->NE * p->MDPE * p->R, nt = p->NF * p->b * p->R;
    // host outputs in pinned, mapped memory are written by the kernel itself
    double* mu = on_device ? nullptr : mapped_host(p, u);
    double* mq = on_device ? nullptr : mapped_host(p, q);
    const bool direct = on_device || (mu && mq);
    if (!p->d_full) p->d_full = (double*)p->dalloc(sizeof(double) * nt);
    if (!direct && !p->d_uout) p->d_uout = (double*)p->dalloc(sizeof(double) * nu);
    if (!direct && !p->d_qout) p->d_qout = (double*)p->dalloc(sizeof(double) * nq);
    double* full = p->d_full;
    double* du = on_device ? u : (direct ? mu : p->d_uout);
    double* dq = on_device ? q : (direct ? mq : p->d_qout);
    expand_trace(p->d_x, p->d_uhatD, p->d_free_of_face, p->NF, p->b, p->R, full, s);
    mark_uD_used(p, s);
    RecoverDesc d{};
    d.XF = p->d_XF;
    d.Xr = p->d_Xr;
    d.MinvB = p->d_MinvB;
    d.MinvC = p->d_MinvC;
    d.uhat_full = full;
    d.elem_face = p->d_elem_face;
    d.M = p->M;
    d.D = p->D;
    d.PE = p->PE;
    d.PF = p->PF;
    d.nl = p->nl;
    d.R = p->R;
    d.n_elem = p->NE;
    d.u = du;
    d.q = dq;
    // host outputs in pageable memory: the elements are recovered in pieces,
    // and the copy stream brings each piece's u and q to the host while the
    // next one is computed
    const int64_t pieces = direct ? 1 : std::min<int64_t>(kRecoverPieces, p->NE / kRecoverPieceMin);
    if (pieces < 2) {
      recover(d, s);
      CK(cudaGetLastError());
      if (!direct) {
        CK(cudaMemcpyAsync(u, du, sizeof(double) * nu, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(q, dq, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
      }
    } else {
      cudaStream_t cs = copy_stream_of(p);
      const int64_t per = (p->NE + pieces - 1) / pieces;
      const int64_t su = (int64_t)p->MPE * p->R, sq = (int64_t)p->MDPE * p->R, nlb = (int64_t)p->nl * p->b;
      const int64_t sB = (int64_t)p->D * p->PE * p->PE, sC = (int64_t)p->D * p->PE * p->nl * p->PF;
      // piece i's copies are issued after piece i+1's launch: a copy to
      // pageable memory returns only when done, and the GPU keeps computing
      auto copy_piece = [&](int64_t e0) {
        const int64_t n = std::min(per, p->NE - e0);
        CK(cudaMemcpyAsync(u + e0 * su, du + e0 * su, sizeof(double) * n * su, cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(q + e0 * sq, dq + e0 * sq, sizeof(double) * n * sq, cudaMemcpyDeviceToHost, cs));
      };
      for (int64_t e0 = 0; e0 < p->NE; e0 += per) {
        RecoverDesc c = d;
        c.XF = d.XF + e0 * p->MPE * nlb;
        c.Xr = d.Xr + e0 * su;
        c.MinvB = d.MinvB + e0 * sB;
        c.MinvC = d.MinvC + e0 * sC;
        c.elem_face = d.elem_face + e0 * p->nl;
        c.u = du + e0 * su;
        c.q = dq + e0 * sq;
        c.n_elem = std::min(per, p->NE - e0);
        recover(c, s);
        CK(cudaGetLastError());
        CK(cudaEventRecord(event_of(p->ev_rec), s));
        if (e0 > 0) copy_piece(e0 - per);
        CK(cudaStreamWaitEvent(cs, p->ev_rec, 0));     // orders the next copy_piece after this piece
      }
      copy_piece((pieces_run(p->NE, per) - 1) * per);
      CK(cudaStreamSynchronize(cs));
    }
    CK(cudaStreamSynchronize(s));
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_apply_K(hdg_problem p, int prec, const double* x, double* y, void* stream) {
  if (!p || !x || !y || prec < 0 || prec > 2) return HDG_ERR_ARG;
  if (!p->assembled) return HDG_ERR_STATE;
  if (prec == HDG_BF16 && !p->K16) return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    ensure_workspace(p, std::max(p->ws_m, 1));
    Ops ops{p, s, p->R};
    ops.K(prec, x, y, EPI_STORE, nullptr, nullptr, nullptr);
    CK(cudaGetLastError());
    collect_timing(p, s);
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_apply_precond(hdg_problem p, const hdg_solver_opts* o, int prec, const double* x, double* y,
                             void* stream) {
  if (!p || !o || !x || !y || prec < 0 || prec > 2) return HDG_ERR_ARG;
  if (!p->assembled || p->pc_ready != o->pc) return HDG_ERR_STATE;
  if (o->poly != HDG_POLY_NONE && (p->poly_n == 0 || p->poly_kind != o->poly)) return HDG_ERR_STATE;
  if (prec == HDG_BF16 && ((o->pc == HDG_PC_BJ && !p->bj16) || (o->pc == HDG_PC_ASM && !p->as16) || !p->K16))
    return HDG_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    ensure_workspace(p, std::max(o->restart, 1));
    Ops ops{p, s, p->R};
    const int pp = (o->poly_prec == HDG_BF16) ? HDG_BF16 : prec;
    ops.Pinv(*o, prec, pp, x, y, nullptr);
    CK(cudaGetLastError());
    return check_err(p, s);
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_get_condensed(hdg_problem p, int64_t e0, int64_t count, double* Kbar, double* rbar) {
  if (!p || e0 < 0 || count < 0 || e0 + count > p->NE) return HDG_ERR_ARG;
  try {
    DeviceGuard dg(p->device);
    CK(cudaDeviceSynchronize());
    if (Kbar)
      CK(cudaMemcpy(Kbar, p->d_Kbar + e0 * p->nlb * p->nlb, sizeof(double) * count * p->nlb * p->nlb,
                    cudaMemcpyDeviceToHost));
    if (rbar)
      CK(cudaMemcpy(rbar, p->d_rbar + e0 * p->nlb * p->R, sizeof(double) * count * p->nlb * p->R,
                    cudaMemcpyDeviceToHost));
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_get_face_rows(hdg_problem p, int64_t f0, int64_t count, double* blocks, int32_t* nbr, double* r) {
  if (!p || f0 < 0 || count < 0 || f0 + count > p->nfree) return HDG_ERR_ARG;
  if (!p->assembled) return HDG_ERR_STATE;
  try {
    DeviceGuard dg(p->device);
    CK(cudaDeviceSynchronize());
    const int b = p->b, ms = p->ms;
    if (blocks) {
      const int64_t b0 = p->h_rowptr[f0], b1 = p->h_rowptr[f0 + count];
      std::vector<double> tmp((size_t)std::max<int64_t>(b1 - b0, 1) * p->s64);
      if (b1 > b0)
        CK(cudaMemcpy(tmp.data(), p->K64 + b0 * p->s64, sizeof(double) * (b1 - b0) * p->s64, cudaMemcpyDeviceToHost));
      std::fill(blocks, blocks + count * ms * b * b, 0.0);
      for (int64_t f = 0; f < count; ++f) {
        const int64_t rb = p->h_rowptr[f0 + f] - b0, ns = p->h_rowptr[f0 + f + 1] - p->h_rowptr[f0 + f];
        for (int64_t s = 0; s < ns; ++s)
          for (int i = 0; i < b; ++i)
            for (int j = 0; j < b; ++j)
              blocks[((f * ms + s) * b + i) * b + j] = tmp[(rb + s) * p->s64 + (int64_t)j * b + i];
      }
    }
    if (nbr) std::memcpy(nbr, p->h_nbr.data() + f0 * ms, sizeof(int32_t) * count * ms);
    if (r) CK(cudaMemcpy(r, p->d_r, sizeof(double) * p->ndof * p->R, cudaMemcpyDeviceToHost));
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_get_poly(hdg_problem p, double* re, double* im, int cap, int* n) {
  if (!p || !n) return HDG_ERR_ARG;
  if (p->poly_kind == HDG_POLY_CHEBYSHEV) {
    if (re && cap >= 2) {
      re[0] = p->cheb_a;
      re[1] = p->cheb_b;
    }
    *n = 2;
    return HDG_OK;
  }
  *n = p->poly_n;
  for (int i = 0; i < p->poly_n && i < cap; ++i) {
    if (re) re[i] = p->th_re[i];
    if (im) im[i] = p->th_im[i];
  }
  return HDG_OK;
}

hdg_status hdg_set_timing(hdg_problem p, int enable) {
  if (!p) return HDG_ERR_ARG;
  p->timing = enable != 0;
  for (int i = 0; i < 6; ++i) {
    p->t_mv_ms[i] = 0.0;
    p->n_mv[i] = 0;
  }
  p->ev_used = 0;
  p->ev_prec.clear();
  return HDG_OK;
}

hdg_status hdg_get_timing(hdg_problem p, int kind, double* total_ms, int64_t* launches) {
  if (!p || kind < 0 || kind > 5) return HDG_ERR_ARG;
  if (total_ms) *total_ms = p->t_mv_ms[kind];
  if (launches) *launches = p->n_mv[kind];
  return HDG_OK;
}

long long hdg_launch_count(void) { return hdg::g_launches.load(); }

}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free matvec.  Some callers cannot call cudaMalloc at the point
// where they need y = K x: code running while a stream is being captured into
// a CUDA graph, hosts whose device memory is owned by their own pool
// allocator and budget, and latency-critical loops where an allocation's
// implicit synchronisation is not acceptable.  For them the FP32 copy of x
// that the FP32/BF16 matvec needs lives in this file-scope device array
// instead of the problem's workspace.  Every GPU that loads the library holds
// the array until the process exits.  Host code must not use the array's name
// as an address: its device address is looked up once per device with
// cudaGetSymbolAddress (device code could name it directly).
namespace {
constexpr int64_t kNoAllocMaxEntries = 8ll * 1024 * 1024;   // n_dof * R <= 8,388,608 (32 MiB)
static __device__ __align__(256) float g_noalloc_x32[kNoAllocMaxEntries];
// error word of the stand-alone GEMM entry point
static __device__ unsigned g_gemm_err;
cudaError_t gemm_err_word(unsigned** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_gemm_err);
  *out = static_cast<unsigned*>(ptr);
  return e;
}
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).
hdg_status noalloc_scratch(int dev, float** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return HDG_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_x32);
    if (e != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return HDG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<float*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return HDG_OK;
}
}  // namespace

extern "C" {

hdg_status hdg_apply_K_noalloc(hdg_problem p, int prec, const double* x, double* y, void* stream) {
  if (!p || !x || !y) return HDG_ERR_ARG;
  if (prec != HDG_FP32 && prec != HDG_BF16) return HDG_ERR_ARG;
  if (!p->assembled) return HDG_ERR_STATE;
  if (prec == HDG_BF16 && !p->K16) return HDG_ERR_STATE;
  if (p->ndof * p->R > kNoAllocMaxEntries) return HDG_ERR_ARG;   // larger than the static scratch
  cudaStream_t s = (cudaStream_t)stream;
  try {
    DeviceGuard dg(p->device);
    float* scratch = nullptr;
    hdg_status st = noalloc_scratch(p->device, &scratch);
    if (st != HDG_OK) return st;
    // the conversion overwrites every entry the matvec reads: nothing to clear
    to_f32(x, scratch, p->ndof * p->R, s);
    BlockRowDesc d{};
    d.prec = prec;
    d.blk = prec == HDG_FP32 ? (const void*)p->K32 : (const void*)p->K16;
    d.blk_stride = prec == HDG_FP32 ? p->s32 : p->s16;
    d.rowptr = p->d_rowptr;
    d.nbr = p->d_nbr;
    d.cnt = p->d_cnt;
    d.n_units = p->nfree;
    d.b_rows = p->b;
    d.ld = prec == HDG_FP32 ? p->ld32 : p->ld16;
    d.bc = p->b;
    d.max_slots = p->ms;
    d.R = p->R;
    d.in = x;
    d.in32 = scratch;
    d.out = y;
    d.epi = EPI_STORE;
    d.err = p->d_err;
    BrCfg direct;
    direct.kind = BR_DIRECT;
    blockrow(d, direct, s);   // the direct kernel: no occupancy queries, no attributes
    CK(cudaGetLastError());
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

const char* hdg_last_error(void) { return g_last_error; }

hdg_status hdg_set_graphs(hdg_problem p, int enable) {
  if (!p) return HDG_ERR_ARG;
  p->use_graphs = enable != 0;
  return HDG_OK;
}

hdg_status hdg_set_condense_chunk(hdg_problem p, int64_t elems) {
  if (!p || elems < 1) return HDG_ERR_ARG;
  if (elems > p->chunk_cap) return HDG_ERR_ARG;
  if (p->d_stage2) {
    p->dfree(p->d_stage2, 0);   // sized for the old chunk
    p->d_stage2 = nullptr;
  }
  p->chunk = elems;
  return HDG_OK;
}

hdg_status hdg_set_hex_generation(hdg_problem p, int sum_factorised) {
  if (!p || sum_factorised < 0 || sum_factorised > 1) return HDG_ERR_ARG;
  p->hex_sf = sum_factorised;
  return HDG_OK;
}

hdg_status hdg_set_condense_mode(hdg_problem p, int mode) {
  if (!p || mode < 0 || mode > 3) return HDG_ERR_ARG;
  p->condense_mode = mode;
  return HDG_OK;
}

hdg_status hdg_gemm_f64(int mode, int M, int N, int K, const double* A, int64_t lda, int64_t sA, const double* B,
                        int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC, double alpha, double beta,
                        int64_t count, void* stream) {
  if (mode < 0 || mode > 3 || M < 1 || N < 1 || K < 1 || count < 0 || !A || !B || !C) return HDG_ERR_ARG;
  if (lda < K || ldb < N || ldc < N || count > (1ll << 31) - 1) return HDG_ERR_ARG;
  if (mode >= 1 && (N < 16 || (mode >= 2 && K > 192))) return HDG_ERR_ARG;
  if (count == 0) return HDG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    unsigned* err = nullptr;
    CK(gemm_err_word(&err));
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    GemmDesc d = gd(M, N, K, A, lda, sA, 0, B, ldb, sB, 0, C, ldc, sC, 0, alpha, beta, (int)count, 1);
    // stream-ordered scratch, released on every path (also when a check throws)
    struct AsyncBuf {
      void* ptr = nullptr;
      cudaStream_t s;
      explicit AsyncBuf(cudaStream_t st) : s(st) {}
      ~AsyncBuf() {
        if (ptr) cudaFreeAsync(ptr, s);
      }
    };
    if (mode == 2) {
      int64_t exw = 0;
      const int64_t need = gemm_planes_bytes(d, &exw);
      AsyncBuf planes(s), exs(s);
      CK(cudaMallocAsync(&planes.ptr, (size_t)need, s));
      CK(cudaMallocAsync(&exs.ptr, sizeof(uint16_t) * (size_t)exw, s));
      gemm_ozaki_planes(d, (unsigned char*)planes.ptr, need, (uint16_t*)exs.ptr, exw, err, s);
    } else if (mode == 1 || mode == 3) {
      AsyncBuf scratch(s);
      const int64_t words = gemm_ozaki_scratch(d);
      CK(cudaMallocAsync(&scratch.ptr, sizeof(uint16_t) * words, s));
      if (mode == 3) gemm_ozaki_persist(d, (uint16_t*)scratch.ptr, words, err, s);
      else gemm_ozaki(d, (uint16_t*)scratch.ptr, err, s);
    } else {
      gemm_f64(d, s);
    }
    CK(cudaGetLastError());
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h & ERRBIT_NAN) return HDG_ERR_NAN;
    if (h & ERRBIT_TIMEOUT) return HDG_ERR_TIMEOUT;
    return HDG_OK;
  } catch (const CudaError& e) {
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

hdg_status hdg_set_kernel_variant(hdg_problem p, int variant) {
  if (!p || variant < 0 || variant >= blockrow_variants()) return HDG_ERR_ARG;
  p->br_variant = variant;
  return HDG_OK;
}

}  // extern "C"

namespace {
// Process-wide tuning cache: problems of the same block shape reuse a choice.
struct TuneKey {
  int op, prec, R, b_rows, max_slots, units_log2;
  bool operator<(const TuneKey& o) const {
    return std::tie(op, prec, R, b_rows, max_slots, units_log2) <
           std::tie(o.op, o.prec, o.R, o.b_rows, o.max_slots, o.units_log2);
  }
};
struct TuneVal {
  BrCfg cfg;
  float us, us0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

int ilog2(int64_t v) {
  int l = 0;
  while (v > 1) { v >>= 1; ++l; }
  return l;
}

// the block-row operations the problem can run now, per precision
bool tune_available(hdg_problem p, int op, int prec) {
  if (op == TUNE_K) return prec == HDG_FP64 ? p->K64 != nullptr : prec == HDG_FP32 ? p->K32 != nullptr : p->K16 != nullptr;
  if (op == TUNE_BJ)
    return p->pc_ready == HDG_PC_BJ &&
           (prec == HDG_FP64 ? p->bj64 != nullptr : prec == HDG_FP32 ? p->bj32 != nullptr : p->bj16 != nullptr);
  return p->pc_ready == HDG_PC_ASM &&
         (prec == HDG_FP64 ? p->as64 != nullptr : prec == HDG_FP32 ? p->as32 != nullptr : p->as16 != nullptr);
}

// elements per stored block (slot) of operation op in precision prec
int64_t stride_of(hdg_problem p, int op, int prec) {
  if (op == TUNE_K) return prec == HDG_FP64 ? p->s64 : prec == HDG_FP32 ? p->s32 : p->s16;
  if (op == TUNE_BJ) return prec == HDG_FP64 ? p->bs64 : prec == HDG_FP32 ? p->bs32 : p->bs16;
  return prec == HDG_FP64 ? p->as_s64 : prec == HDG_FP32 ? p->as_s32 : p->as_s16;
}

int ld_of(hdg_problem p, int op, int prec) {
  if (op == TUNE_ASM) return prec == HDG_FP64 ? p->nlb : prec == HDG_FP32 ? ld_f32(p->nlb) : ld_bf16(p->nlb);
  return prec == HDG_FP64 ? p->b : prec == HDG_FP32 ? p->ld32 : p->ld16;
}

TuneKey tune_key(hdg_problem p, int op, int prec) {
  TuneKey k;
  k.op = op; k.prec = prec; k.R = p->R;
  k.b_rows = op == TUNE_ASM ? p->nlb : p->b;
  k.max_slots = op == TUNE_K ? p->ms : op == TUNE_BJ ? 1 : p->nl;
  k.units_log2 = ilog2(op == TUNE_ASM ? p->NE : p->nfree);
  return k;
}
}  // namespace

extern "C" {

hdg_status hdg_autotune(hdg_problem p, int reps, int force, void* stream) {
  if (!p || reps < 0) return HDG_ERR_ARG;
  if (!p->assembled) return HDG_ERR_STATE;
  if (reps == 0) reps = 10;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    DeviceGuard dg(p->device);
    ensure_workspace(p, std::max(p->ws_m, 1));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double* x = p->pt;
    double* y = p->pAq;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * p->ndof * p->R, s));
    Ops ops{p, s, p->R};
    const bool timing = p->timing;
    p->timing = false;
    for (int op = 0; op < 3; ++op)
      for (int prec = 0; prec < 3; ++prec) {
        if (!tune_available(p, op, prec)) continue;
        const TuneKey key = tune_key(p, op, prec);
        if (!force) {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          auto it = g_tune_cache.find(key);
          if (it != g_tune_cache.end()) {
            p->tune[op][prec] = it->second.cfg;
            p->tune_us[op][prec] = it->second.us;
            p->tune_us0[op][prec] = it->second.us0;
            continue;
          }
        }
        auto run = [&]() {
          if (op == TUNE_K) ops.K(prec, x, y, EPI_STORE, nullptr, nullptr, nullptr);
          else ops.Minv(op == TUNE_BJ ? HDG_PC_BJ : HDG_PC_ASM, prec, x, y, nullptr);
        };
        auto time_cfg = [&](const BrCfg& c) -> float {
          p->tune[op][prec] = c;
          run();
          run();
          CK(cudaEventRecord(e0, s));
          for (int i = 0; i < reps; ++i) run();
          CK(cudaEventRecord(e1, s));
          CK(cudaEventSynchronize(e1));
          CK(cudaGetLastError());
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          return ms * 1000.f / reps;
        };
        BlockRowDesc d{};
        d.prec = prec;
        d.R = p->R;
        d.b_rows = key.b_rows;
        d.ld = ld_of(p, op, prec);
        d.blk_stride = stride_of(p, op, prec);
        d.bc = p->b;
        d.max_slots = key.max_slots;
        d.in32 = p->x32;
        BrCfg cand[32];
        int nc = blockrow_candidates(d, cand, 32);
        if (op == TUNE_K && prec == HDG_FP64 && p->kdig_ready && nc < 32) {
          cand[nc].kind = BR_TC;
          cand[nc].sp = 0;
          cand[nc].cps = 0;
          ++nc;
        }
        BrCfg best;
        const float us0 = time_cfg(best);
        float bus = us0;
        for (int i = 0; i < nc; ++i) {
          const float us = time_cfg(cand[i]);
          if (us < bus) { bus = us; best = cand[i]; }
        }
        p->tune[op][prec] = best;
        p->tune_us[op][prec] = bus;
        p->tune_us0[op][prec] = us0;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneVal{best, bus, us0};
      }
    p->timing = timing;
    p->tune_gen++;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return check_err(p, s);
  } catch (const CudaError& e) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return to_status(e);
  } catch (const std::bad_alloc&) {
    return HDG_ERR_OOM;
  }
}

int hdg_tuning_candidates(hdg_problem p, int op, int prec, int* cfg3, int cap) {
  if (!p || op < 0 || op > 2 || prec < 0 || prec > 2 || cap < 0) return -1;
  BlockRowDesc d{};
  const TuneKey key = tune_key(p, op, prec);
  d.prec = prec;
  d.R = p->R;
  d.b_rows = key.b_rows;
  d.ld = ld_of(p, op, prec);
  d.blk_stride = stride_of(p, op, prec);
  d.bc = p->b;
  d.max_slots = key.max_slots;
  d.in32 = reinterpret_cast<const float*>(16);   // only tested for non-null
  BrCfg cand[32];
  int nc = blockrow_candidates(d, cand, 32);
  if (op == TUNE_K && prec == HDG_FP64 && p->kdig_ready && nc < 32) {
    cand[nc].kind = BR_TC;
    cand[nc].sp = 0;
    cand[nc].cps = 0;
    ++nc;
  }
  for (int i = 0; i < nc && i < cap && cfg3; ++i) {
    cfg3[3 * i] = cand[i].kind; cfg3[3 * i + 1] = cand[i].sp; cfg3[3 * i + 2] = cand[i].cps;
  }
  return nc;
}

hdg_status hdg_set_tuning(hdg_problem p, int op, int prec, const int* cfg3) {
  if (!p || op < 0 || op > 2 || prec < 0 || prec > 2 || !cfg3) return HDG_ERR_ARG;
  if (cfg3[0] < BR_DEFAULT || cfg3[0] > BR_VEC3R || cfg3[1] < 0 || cfg3[1] > 8 || cfg3[2] < 0 || cfg3[2] > 64)
    return HDG_ERR_ARG;
  p->tune[op][prec].kind = cfg3[0];
  p->tune[op][prec].sp = cfg3[1];
  p->tune[op][prec].cps = cfg3[2];
  p->tune_gen++;
  return HDG_OK;
}

hdg_status hdg_get_tuning(hdg_problem p, int op, int prec, int* cfg3, float* us_tuned, float* us_default) {
  if (!p || op < 0 || op > 2 || prec < 0 || prec > 2) return HDG_ERR_ARG;
  const BrCfg c = p->tune[op][prec];
  if (cfg3) { cfg3[0] = c.kind; cfg3[1] = c.sp; cfg3[2] = c.cps; }
  if (us_tuned) *us_tuned = p->tune_us[op][prec];
  if (us_default) *us_default = p->tune_us0[op][prec];
  return HDG_OK;
}

}  // extern "C"
