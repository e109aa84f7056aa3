// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <vector>

#include "../../include/hdg.h"

namespace hdg {

// --------------------------------------------------------------- batched GEMM
// C[b] = beta*C[b] + alpha*A[b]*B[b] for a two-level batch (b0 < nb0, b1 < nb1),
// row-major FP64.  The output column c is stored at (c / cg)*cgs + (c % cg),
// which lets one product write a strided set of column groups.
struct GemmDesc {
  int M, N, K;
  const double* A; int64_t lda, sA0, sA1;
  const double* B; int64_t ldb, sB0, sB1;
  double* C; int64_t ldc, sC0, sC1;
  int cg; int64_t cgs;
  double alpha, beta;
  int nb0, nb1;
};
void gemm_f64(const GemmDesc& d, cudaStream_t s);
// The same product on the BF16 tensor cores by exact operand splitting
// (FP64-accurate); K > 192 runs in slices of at most 192 accumulated into C.
// Returns false (nothing launched) when N < 16.
// scratch: gemm_ozaki_scratch(d) 16-bit words of device memory (the row and
// column exponents), reused after the launches complete.
int64_t gemm_ozaki_scratch(const GemmDesc& d);
bool gemm_ozaki(const GemmDesc& d, uint16_t* scratch, unsigned* err, cudaStream_t s);
// The same product with each operand split once into BF16 digit planes in
// device memory (gemm_planes_bytes(d, &ex_words) plane bytes and ex_words
// 16-bit words of scratch; -1 outside K <= 192, N >= 16), then bulk-copied
// into the tensor-core product kernel.  False when the scratch is too small.
int64_t gemm_planes_bytes(const GemmDesc& d, int64_t* ex_words);
// Persistent variant of gemm_ozaki (one CTA per SM over all 128 x 32 tiles,
// accumulators double-buffered in TMEM); scratch as gemm_ozaki_scratch.
bool gemm_ozaki_persist(const GemmDesc& d, uint16_t* scratch, int64_t scratch_words, unsigned* err,
                        cudaStream_t s);
bool gemm_ozaki_planes(const GemmDesc& d, unsigned char* planes, int64_t planes_cap, uint16_t* ex, int64_t ex_cap,
                       unsigned* err, cudaStream_t s);

// Batched in-place inverse (Gauss-Jordan, partial pivoting) of `count`
// n x n FP64 matrices with batch stride `stride`.  Sets ERRBIT_SINGULAR in
// *err on a zero pivot.  Returns false if n is too large for one CTA.
bool inverse_f64(double* A, int n, int64_t stride, int64_t count, unsigned* err, cudaStream_t s);
int inverse_max_n();
// ------------------------------------------- hexahedral element matrices
// Reference tables of Q^k on the cube with an n^3 / n^2 Gauss rule (host).
struct HexTables {
  int k = 0, n1 = 0, PE = 0, PF = 0, nq1 = 0, nq = 0, nfq = 0;
  std::vector<double> phiT;    // PE x nq
  std::vector<double> phi;     // nq x PE
  std::vector<double> dphi;    // nq x PE x 3 (reference gradients)
  std::vector<double> wq;      // nq
  std::vector<double> dN;      // nq x 8 x 3 trilinear shape derivatives
  std::vector<double> fphiT;   // PE x (6 nfq): phi at face points, column l nfq + q
  std::vector<double> fphi;    // (6 nfq) x PE
  std::vector<double> fdN;     // (6 nfq) x 8 x 3
  std::vector<double> psi;     // nfq x PF face basis
  std::vector<double> wf;      // nfq face weights
  std::vector<double> b1, d1;  // nq1 x (k+1): 1D Lagrange values and derivatives at the 1D Gauss points
};
HexTables build_hex_tables(int k, int nquad);
// per-element scratch (doubles) of the generation steps
int64_t hex_gen_scratch(const HexTables& T);
// device pointers of one generation chunk (count elements)
struct HexGenDesc {
  int64_t count;
  int M, PE, PF, nq, nfq;
  const double* verts;         // count x 8 x 3
  const int32_t* perm;         // count x 6 x PF
  // device copies of the tables
  const double *phi, *dphi, *wq, *dN, *fphi, *fdN, *psi, *wf;
  // scratch (per element, see hex_gen_scratch)
  double *AW, *GT, *BWN, *PW, *PsiT, *Mf, *EF4, *FF4;
  // physics (device): Cq M x 3 x M x 3, Cu M x 3 x M, Rr M x M
  const double *Cq, *Cu, *Rr;
  double tau;
  // outputs (row-major per element, the condensation's input layout)
  const double* Me;            // written by the mass product
  const double* Sd;            // = Bd, written by the gradient products
  double *Cd, *Dm, *Em, *Fm, *Gm, *Hm, *Jm;
  unsigned* err;
};
// AW, GT (volume) and BWN, PW, PsiT (faces) from the vertices
void hex_geometry(const HexGenDesc& d, cudaStream_t s);
void hex_face_geometry(const HexGenDesc& d, cudaStream_t s);
// M^e and B_d by sum factorisation of the tensor-product rule (FP64, one CTA
// per element): per weight field three 1D contractions.  b1, d1: device 1D
// tables (nq1 x n1).  Returns false (nothing launched) beyond n1 <= 5, nq1 <= 8.
bool hex_mass_grad_sf(const HexGenDesc& d, int n1, int nq1, const double* b1, const double* d1, double* Me,
                      double* Bd, cudaStream_t s);
// Cd, D, E, F, G, H, J from Me, Sd, Mf, EF4, FF4 and the physics (seven kernels)
void hex_expand(const HexGenDesc& d, cudaStream_t s);

// Batched copy of a rows x cols submatrix between row-major FP64 arrays.
void copy_block_f64(double* dst, int64_t ldd, int64_t sd, const double* src, int64_t lds, int64_t ss, int rows,
                    int cols, int64_t count, cudaStream_t s);

// --------------------------------------------------------------- block rows
// out[u][row][r] = epilogue( sum_{s < cnt[u]} sum_{c < bc}
//                   blk[u][s](row, c) * in[(nbr[u][s]*bc + c)*R + r] )
// blk[u][s] is a column-major b_rows x bc block at blk + (rowptr[u] + s)*
// blk_stride elements (compact storage: cnt[u] = rowptr[u+1] - rowptr[u]).
enum Epi { EPI_STORE = 0, EPI_RESID = 1, EPI_SCALE = 2, EPI_POLY = 3 };

// One step of a polynomial preconditioner fused into the epilogue of the
// block-Jacobi apply (or of the ASM face sum), on FP32 state vectors: v is the
// freshly computed (M^{-1} K s)[o] (or (M^{-1} x)[o] for the INIT steps).
//   CHEB_INIT  r = v; d = c1 v; z = d                       (c1 = 1 / theta)
//   CHEB_STEP  r -= v; d = c1 d + c2 r; z += d               (Chebyshev iteration)
//   PP_INIT    q = v
//   PP_REAL    w += c1 q; q -= c1 v                          (c1 = 1 / theta_i)
//   PP_PAIR_T  t = c1 q - v; w += c2 t                       (c1 = 2a, c2 = 1 / (a^2 + b^2))
//   PP_PAIR_Q  q -= c2 v                                     (c2 = 1 / (a^2 + b^2))
// p0, p1, p2 hold (r, z, d) for Chebyshev and (q, w, t) for the GMRES
// polynomial.  wzero: w reads as 0 (first term).  fin: the step is followed
// by the final real value theta_P, so out64 = w + cfin q_new (PP_INIT:
// cfin v).  last: the step completes the polynomial, out64 = z (Chebyshev) or
// w (PP_PAIR_T); the state is then not written back.
enum PolyOp { POLY_OP_NONE = 0, CHEB_INIT = 1, CHEB_STEP = 2, PP_INIT = 3, PP_REAL = 4, PP_PAIR_T = 5,
              PP_PAIR_Q = 6 };
struct PolyEpi {
  int op;
  int wzero, fin, last;
  float c1, c2, cfin;
  float *p0, *p1, *p2;
  double* out64;
};
// out64 / FP32 state update of one polynomial step on `len` values of v
// (FP32), for the preconditioner without a base (M = I).
void poly_epi_apply(const PolyEpi& e, const float* v, int64_t len, const int* active, int R, cudaStream_t s);

struct BlockRowDesc {
  int prec;               // HDG_FP64 / HDG_FP32 / HDG_BF16 storage of blk
  const void* blk;
  int64_t blk_stride;     // elements per slot block (padded to 16 bytes)
  const int64_t* rowptr;  // n_units + 1 block offsets
  const int32_t* nbr;     // n_units * max_slots
  const int32_t* cnt;     // n_units
  int64_t n_units;
  int b_rows, bc, max_slots, R;
  int ld;                 // stored rows per block column (>= b_rows; rows past b_rows are padding)
  const double* in;
  const float* in32;      // FP32 copy of `in` (required for FP32/BF16 blocks)
  double* out;            // FP64 output (may be NULL when out32 is set)
  float* out32;           // optional FP32 copy of the output
  PolyEpi pe;             // EPI_POLY: the polynomial step applied to the output
  int epi;
  const double* rhs;      // EPI_RESID: out = rhs - acc
  const double* scale;    // EPI_SCALE: out = scale[r] * acc (per RHS)
  const int* active;      // optional: skip the launch work when all R entries are 0
  unsigned* err;
};
// Launch configuration of a block-row product.  kind: BR_DEFAULT (heuristic:
// vectorised loads for FP32/BF16 where the rows allow, else one thread per
// row; FP64 rows split over slot parts when one thread per row would leave
// the SMs mostly idle), BR_TMA (bulk-copy staging), BR_DIRECT (one thread per
// row), BR_VEC (VR rows per thread, 16-byte loads, sp slot parts), BR_SPLIT
// (sp threads per row, each summing every sp-th slot, shuffle reduction).
// cps: CTAs per SM of the grid-stride launch (0 = heuristic).
enum { BR_DEFAULT = 0, BR_TMA = 1, BR_DIRECT = 2, BR_VEC = 3, BR_SPLIT = 4, BR_BULK = 5, BR_TC = 6, BR_VEC3 = 7,
       BR_VEC3R = 8 };
struct BrCfg {
  int kind = BR_DEFAULT, sp = 0, cps = 0;
};
void blockrow(const BlockRowDesc& d, BrCfg cfg, cudaStream_t s);
// Leading dimension of FP32 / BF16 block copies: the column length rounded up
// to a whole 16-byte vector, so that every column starts 16-byte aligned.
inline int ld_f32(int rows) { return (rows + 3) / 4 * 4; }
inline int ld_bf16(int rows) { return (rows + 7) / 8 * 8; }
// valid configurations for d (at most cap); returns their number
int blockrow_candidates(const BlockRowDesc& d, BrCfg* out, int cap);
int blockrow_variants();
// FP64 -> FP32 copy of a vector (rounding to nearest)
void to_f32(const double* x, float* y, int64_t n, cudaStream_t s);

// ------------------------------------- FP64 block rows on the tensor cores
// FP64-accurate products of FP64 blocks with R = 4 or 8 right-hand sides on
// the BF16 tensor cores (k_tcmv.cu), from the blocks stored as exact digits:
// per unit u and row i an exponent ex[u * b_rows + i] and, at byte offset
// doff[u], 8 digit bytes per entry ((k * 8 + s) * b_rows + i) * 16 + jj for
// column 16 k + jj.  tc_digit_layout fills the host offsets (n_units + 1)
// from the host block offsets and returns the bytes; tc_split writes the
// digits of d's FP64 blocks; tc_blockrow runs the product (false, nothing
// launched, when tc_supported(d) is not: FP64 blocks, R in {4, 8}, square
// blocks of at most 32 rows, no polynomial epilogue).
int64_t tc_digit_layout(const int64_t* h_rowptr, int64_t n_units, int b_rows, int bc, int64_t* h_doff);
bool tc_supported(const BlockRowDesc& d);
void tc_split(const BlockRowDesc& d, unsigned char* dig, const int64_t* doff, int32_t* ex, cudaStream_t s);
bool tc_blockrow(const BlockRowDesc& d, const unsigned char* dig, const int64_t* doff, const int32_t* ex,
                 cudaStream_t s);

// ------------------------------------------------ batched persistent GMRES
// One system of a batch solved by batch_gmres (k_batch.cu): its blocks,
// preconditioner, vectors and GMRES workspace (the problem's own buffers).
struct BatchItem {
  int64_t len;                  // n_dof * R
  int64_t nchunks;              // reduction chunks of len entries
  int64_t nfree;                // trace face rows
  int b, R, ms, pc, kprec, ld32;
  int sp, fpc;                  // fused K / block-Jacobi step: slot parts of a face row, faces per CTA
  const double* K64; int64_t s64;
  const float* K32; int64_t s32;
  const int64_t* rowptr; const int32_t* nbr; const int32_t* cnt;
  const double* bj64; int64_t bs64;
  const float* bj32; int64_t bs32;
  const double* rhs; double* x; double* res; double* t1;
  float* x32; float* t32;
  double *V, *vscale, *H, *g, *cs, *sn, *hcol, *htmp, *ycoef, *part;
  double *bnorm, *zb, *rel, *cfac, *tolabs;
  int *running, *done, *iters, *jend, *on_est, *done_all;
};
struct BatchDesc {
  BatchItem* items;             // device, n
  int n, m, maxit;
  double rtol;
  int64_t rows_total, elems_total, chunks_total, groups_total;   // groups: whole faces per CTA
  const int64_t *row_pre, *elem_pre, *chunk_pre, *group_pre;     // device prefix sums (n entries)
  void* bar;                    // device grid-barrier words (zeroed before the launch)
  unsigned* err;
};
int64_t batch_chunks(int64_t len);
// fused-step layout of one system (b <= batch_max_b()): slot parts and faces
// per CTA; returns the number of face groups
int64_t batch_layout(int64_t nfree, int b, int ld32, int R, bool f32, int* sp, int* fpc);
int batch_max_b();
// one cooperative launch; false if it could not be launched
bool batch_gmres(const BatchDesc& B, int rmax, cudaStream_t s);   // rmax: the largest R of the batch

// --------------------------------------------------------------- assembly etc.
struct AssembleDesc {
  const double* Kbar; const double* rbar; const double* uhatD;
  int nlb;                       // n_lfe*b: side of Kbar
  int b, nl, R, max_slots;
  int64_t n_free;
  const int32_t* slot_e;         // n_free*max_slots element of the block (-1 pad)
  const int32_t* slot_lr;        // row local face
  const int32_t* slot_lc;        // column local face
  const int32_t* diag2;          // n_free*2: (e2, l2) second element of the diagonal (-1)
  const int32_t* rhs_src;        // n_free*4: (e1,l1,e2,l2)
  const int32_t* elem_face;      // n_elem*nl
  const uint8_t* face_dir;       // n_face
  const int64_t* rowptr;         // n_free + 1 compact block offsets of the face rows
  double* K64; int64_t s64;
  float* K32; int64_t s32; int ld32;
  __nv_bfloat16* K16; int64_t s16; int ld16;
  double* r;
};
void assemble(const AssembleDesc& d, cudaStream_t s);

// copy diagonal blocks (slot 0, column-major) into dense row-major blocks
void extract_diag(const double* K64, int64_t s64, const int64_t* rowptr, int b, int64_t n_free, double* out,
                  cudaStream_t s);
// dense row-major FP64 n x n blocks -> column-major padded blocks in the three precisions
void pack_blocks(const double* in, int n, int64_t count, double* o64, int64_t s64, float* o32, int64_t s32,
                 int ld32, __nv_bfloat16* o16, int64_t s16, int ld16, cudaStream_t s);
// ASM element matrices from Kbar: rows/cols restricted to free faces in local order
// (compacted), diagonal blocks of interior faces replaced by K_ff, padding = identity.
void asm_build(const double* Kbar, int nlb, int b, int nl, int64_t n_elem, const int32_t* asm_lf,
               const int32_t* asm_cnt, const int32_t* asm_face_free, const double* K64, int64_t s64,
               const int64_t* rowptr, double* P, cudaStream_t s);
// ASM panels: column-major (nl*b) x b panels for the free local faces of each element
void asm_pack(const double* Pinv, int nlb, int b, int nl, int64_t n_elem, const int64_t* arowptr, double* o64,
              int64_t s64, float* o32, int64_t s32, int ld32, __nv_bfloat16* o16, int64_t s16, int ld16,
              cudaStream_t s);
// z_f = z^{e1}[slot s1] + z^{e2}[slot s2] (face-parallel, no atomics)
void asm_face_sum(const double* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum, double* z,
                  cudaStream_t s);
// the same sum from FP32 element results, followed by a polynomial step (or,
// with pe->op == POLY_OP_NONE, stored to z64 and/or z32)
void asm_face_sum_f32(const float* ze, int nlb, int b, int R, int64_t n_free, const int32_t* fsum,
                      const PolyEpi* pe, double* z64, float* z32, cudaStream_t s);

// --------------------------------------------------------------- recovery
struct RecoverDesc {
  const double* XF; const double* Xr; const double* MinvB; const double* MinvC;
  const double* uhat_full;   // n_face*b*R
  const int32_t* elem_face;
  int M, D, PE, PF, nl, R;
  int64_t n_elem;
  double* u; double* q;
  double* uhe;               // scratch n_elem * nl*b * R
};
void recover(const RecoverDesc& d, cudaStream_t s);
// count copies of the n-element block src into dst
void bcast_copy(double* dst, const double* src, int64_t n, int64_t count, cudaStream_t s);
// free-vector -> full trace (Dirichlet faces from uhatD)
void expand_trace(const double* x, const double* uhatD, const int32_t* free_of_face, int64_t n_face, int b, int R,
                  double* full, cudaStream_t s);

}  // namespace hdg
