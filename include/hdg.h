/*
 * hdg.h -- C ABI of the GB300 HDG trace-solver library (libhdg.so).
 *
 * The library implements the data-parallel hot path of the HDG solver of
 * Welter & Nguyen, "Preconditioning Techniques for Hybridizable Discontinuous
 * Galerkin Discretizations on GPU Architectures" (arXiv 2512.13619):
 * batched static condensation of element blocks, face-based assembly of the
 * trace matrix K in face-block format, and restarted left-preconditioned
 * GMRES on K with block-Jacobi, additive-Schwarz and polynomial
 * preconditioners, followed by element-wise recovery.
 *
 * Conventions shared by every entry point
 *  - Plain pointers and sizes only.  A pointer argument documented as
 *    "host or device" is a device pointer when the call's `on_device` flag is
 *    non-zero, otherwise a host pointer.  Arguments documented as "device"
 *    are always device pointers on the problem's device.
 *  - The library owns every buffer it allocates and frees them in
 *    hdg_problem_destroy.  Caller buffers are never retained after a call
 *    returns (except the stream handle, which is only used during the call).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  All device work is stream-ordered on it.  Calls that
 *    return values computed on the device (iteration counts, residuals)
 *    synchronise that stream before returning; no call synchronises the whole
 *    device.
 *  - Every call returns an hdg_status.  No C++ exception crosses the ABI.  On
 *    an error the problem stays valid (it can be destroyed) unless the status
 *    is HDG_ERR_CUDA, after which only hdg_problem_destroy is allowed.
 *  - All matrices are row-major, element-contiguous (strided batches).
 *
 * Unknown ordering (M components, D dimensions, P_E element and P_F face
 * basis functions, N_lfe local faces per element, R right-hand sides):
 *    element u   : (a, i)     -> a*P_E + i
 *    element q   : (a, c, i)  -> (a*D + c)*P_E + i
 *    element uhat: (l, a, j)  -> (l*M + a)*P_F + j
 *    face trace  : (a, j)     -> a*P_F + j            (b = M*P_F per face)
 * Face basis functions of every element are ordered as the global face's
 * nodes, so both elements of a face address the same face unknowns.
 * Vectors with R right-hand sides keep the RHS index fastest:
 *    v[dof*R + r].
 * The trace unknowns of the linear solver are the "free" faces (faces not
 * marked Dirichlet), numbered in increasing global face id; n_dof = n_free*b.
 */
#ifndef HDG_H
#define HDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_problem_s* hdg_problem;

typedef enum {
  HDG_OK = 0,
  HDG_ERR_ARG = 1,           /* invalid argument or size                            */
  HDG_ERR_OOM = 2,           /* device allocation failed                             */
  HDG_ERR_BUDGET = 3,        /* request exceeds the configured memory budget         */
  HDG_ERR_SINGULAR = 4,      /* zero pivot in a batched inverse (M^e, Ebar, BJ, ASM) */
  HDG_ERR_NOT_CONVERGED = 5, /* max iterations reached above the tolerance           */
  HDG_ERR_BREAKDOWN = 6,     /* GMRES / Arnoldi breakdown that is not a lucky one     */
  HDG_ERR_NAN = 7,           /* NaN or Inf met in a norm                              */
  HDG_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up                   */
  HDG_ERR_CUDA = 9,          /* CUDA runtime error                                    */
  HDG_ERR_STATE = 10         /* call out of order (e.g. solve before assemble)        */
} hdg_status;

typedef enum { HDG_FP64 = 0, HDG_FP32 = 1, HDG_BF16 = 2 } hdg_prec;
typedef enum { HDG_PC_NONE = 0, HDG_PC_BJ = 1, HDG_PC_ASM = 2 } hdg_pc;
typedef enum { HDG_POLY_NONE = 0, HDG_POLY_GMRES = 1, HDG_POLY_CHEBYSHEV = 2 } hdg_poly;
typedef enum { HDG_ORTH_CGS = 0, HDG_ORTH_MGS = 1, HDG_ORTH_CGS2 = 2 } hdg_orth;

/* Mesh connectivity (Sec. 4.2 face-based assembly, Sec. 4.6 ASM update).
 *  elem_face      host, n_elem*n_lfe int32: global face id f(e, l)
 *  face_elem      host, n_face*4 int32: (e1, l1, e2, l2); e2 = l2 = -1 for a
 *                 face with one element
 *  face_dirichlet host, n_face uint8: 1 = Dirichlet face (trace known,
 *                 eliminated from K), 0 = free face
 * Copied by hdg_problem_create. */
typedef struct {
  int dim, n_lfe, M, PE, PF;
  int64_t n_elem, n_face;
  const int32_t* elem_face;
  const int32_t* face_elem;
  const uint8_t* face_dirichlet;
} hdg_mesh;

/* Solver options (Sec. 3.1-3.4 and Sec. 5 solver parameters: restart 50,
 * CGS, max 1000 iterations).
 *  restart      GMRES restart length m (1..200)
 *  max_iters    total iteration cap (inner iterations in mixed mode)
 *  rtol         accepted when ||b - K x||_2 / ||b||_2 <= rtol, computed in
 *               FP64 per right-hand side
 *  orth         Gram-Schmidt variant
 *  pc           base preconditioner M^{-1} (none, block-Jacobi, ASM)
 *  poly         polynomial preconditioner p(M^{-1} K) composed with pc
 *  poly_degree  number of Ritz values P (GMRES polynomial) or polynomial
 *               degree (Chebyshev)
 *  inner_prec   HDG_FP64: plain FP64 GMRES.  HDG_FP32 / HDG_BF16: FP64
 *               iterative refinement around an inner GMRES whose matrix and
 *               preconditioner blocks are stored in FP32 (the polynomial
 *               smoother's matrix in poly_prec) and accumulated in FP32; the
 *               Krylov basis, Gram-Schmidt and Givens stay in FP64
 *  poly_prec    storage precision of K inside the polynomial smoother
 *  inner_rtol   relative tolerance of each inner solve in mixed mode
 *  max_outer    refinement-step cap in mixed mode; -1 selects the restarted
 *               mixed mode instead: one restarted GMRES whose cycles (matvecs
 *               and preconditioner) run on the inner_prec blocks while every
 *               restart recomputes the true residual with the FP64 blocks,
 *               so convergence is judged in FP64 and no inner solves are
 *               nested; -2 selects the preconditioner-only mixed mode: FP64
 *               GMRES on the FP64 operator (matvecs, Krylov basis, Givens,
 *               residuals in FP64) whose preconditioner M^{-1} runs on
 *               inner_prec blocks (BJ inverses, ASM inverses) and whose
 *               polynomial smoother multiplies by K stored in poly_prec
 *               (FP64, FP32 or BF16), accumulated in FP32 for low-precision
 *               blocks.  The preconditioner stays a fixed linear operator,
 *               so left-preconditioned GMRES applies unchanged */
typedef struct {
  int restart;
  int max_iters;
  double rtol;
  int orth;
  int pc;
  int poly;
  int poly_degree;
  int inner_prec;
  int poly_prec;
  double inner_rtol;
  int max_outer;
} hdg_solver_opts;

typedef struct {
  int iters;          /* GMRES iterations (max over right-hand sides)        */
  int restarts;       /* restart cycles                                       */
  int outer;          /* refinement steps (mixed mode), 0 otherwise           */
  int converged;      /* 1 if every right-hand side met rtol                  */
  double rel_resid;   /* max over RHS of ||b - K x|| / ||b|| (FP64)           */
} hdg_solve_info;

/* Human-readable name of a status. */
const char* hdg_status_str(hdg_status s);

/* Text of the last CUDA failure a library call met on this host thread
 * (runtime error name and the failing call), "" if none. */
const char* hdg_last_error(void);

/* Create a problem on CUDA device `device` for `nrhs` right-hand sides.
 * Builds the face-row neighbour tables (free-face numbering, 2N_lfe-1 slots
 * per face row, Sec. 2.4) on the host and uploads them.  *out owns all device
 * memory of the problem.  Errors: HDG_ERR_ARG (bad sizes, inconsistent maps),
 * HDG_ERR_OOM. */
hdg_status hdg_problem_create(const hdg_mesh* mesh, int nrhs, int device, hdg_problem* out);

/* Release every buffer of the problem.  NULL is accepted. */
hdg_status hdg_problem_destroy(hdg_problem p);

/* Device bytes the problem currently holds (for admission by budget). */
size_t hdg_problem_device_bytes(hdg_problem p);

/* Device bytes a problem of this mesh would hold after create, condense,
 * assemble and setup with `opts` (an estimate used for admission control). */
size_t hdg_workspace_bytes(const hdg_mesh* mesh, int nrhs, const hdg_solver_opts* opts);

/* Batched static condensation of elements [e0, e0+count) (Eq. 13; Sec. 4.1
 * Eqs. w15-w19, Sec. 4.2 Eqs. w21-w22), FP64:
 *   A^{-1} from (M^e)^{-1}; Ebar = E - D A^{-1} B; Fbar = F - D A^{-1} C;
 *   Hbar = H - G A^{-1} B; Jbar = J - G A^{-1} C;
 *   Kbar^e = Jbar - Hbar Ebar^{-1} Fbar;  rbar^e = r_uh - Hbar Ebar^{-1} r_u.
 * Inputs (host or device per on_device), `count` elements each, row-major:
 *   Me  P_E x P_E           mass matrix M^e of Eq. w16
 *   Bd  D x P_E x P_E       B_d of Eq. w16 (matrix of (u, div r) of Eq. HDGa)
 *   Cd  D x P_E x N_lfe*P_F C_d of Eq. w16
 *   D   M*P_E x M*D*P_E     E   M*P_E x M*P_E     F  M*P_E x N_lfe*M*P_F
 *   G   N_lfe*M*P_F x M*D*P_E  H  N_lfe*M*P_F x M*P_E
 *   J   N_lfe*M*P_F x N_lfe*M*P_F
 *   ru  M*P_E x R           ruh N_lfe*M*P_F x R
 * r_q = 0 as in Sec. 4.1.  Results stay on the device (Kbar^e, rbar^e and the
 * recovery data (M^e)^{-1}B_d, (M^e)^{-1}C_d, Ebar^{-1}Fbar, Ebar^{-1}r_u).
 * Elements may be condensed in any number of calls, in any order; assembly
 * requires all of them.  Errors: HDG_ERR_ARG, HDG_ERR_SINGULAR (zero pivot in
 * M^e or Ebar; reported at the next synchronising call), HDG_ERR_CUDA. */
hdg_status hdg_condense(hdg_problem p, int64_t e0, int64_t count,
                        const double* Me, const double* Bd, const double* Cd,
                        const double* D, const double* E, const double* F,
                        const double* G, const double* H, const double* J,
                        const double* ru, const double* ruh, int on_device, void* stream);

/* Physics of a linear HDG system (Eq. HDG): flux F_{a,d} = sum_{b,c}
 * Cq[a][d][b][c] q_{b,c} + sum_b Cu[a][d][b] u_b, source -sum_b Rr[a][b] u_b,
 * stabilisation S = tau I; q = grad u.  Host arrays, M components, D = 3:
 * Cq M*3*M*3, Cu M*3*M (NULL: zero), Rr M*M (NULL: zero). */
typedef struct {
  const double* Cq;
  const double* Cu;
  const double* Rr;
  double tau;
} hdg_physics;

/* Static condensation of hexahedral Q^k elements whose blocks are generated
 * on the device (the element integrals of Sec. 4.1 as batched products of
 * basis tables with quadrature weights, M = Phi W, then the blocks of
 * Eq. matrixform), chunk by chunk, without the blocks ever leaving the GPU.
 * Requires dim 3, N_lfe 6, P_E = (k+1)^3, P_F = (k+1)^2, M <= 5.  Reference element:
 * Q^k on Gauss-Lobatto-Legendre nodes (x fastest), an nquad^3 Gauss rule
 * (nquad^2 on faces), local face l fixing reference coordinate l/2 at -1
 * (l even) or +1 (l odd) with parameters the other two coordinates in
 * increasing order; trilinear geometry.
 *   verts      count x 8 x 3: vertex v at reference corner (+-1 by bits 0,1,2 of v)
 *   face_perm  count x 6 x P_F int32: the local face-node index of face l
 *              that carries the face's global node j
 *   ru, ruh    as hdg_condense (load vectors; count x M*P_E x R and
 *              count x N_lfe*M*P_F x R)
 * verts, face_perm, ru, ruh are host or device per on_device.  The
 * generation's scratch (per element of a condensation chunk: about
 * P_E (4 nq + P_E) + 6 nq_f (5 P_F + P_E) + 24 P_F (P_E + P_F) doubles, nq and
 * nq_f the volume and face quadrature points) and the reference tables are
 * allocated on first use and are not part of hdg_workspace_bytes.  Errors:
 * HDG_ERR_ARG (shapes, nquad outside 1..12, a face_perm entry outside
 * 0..P_F-1), HDG_ERR_SINGULAR (a degenerate element), as hdg_condense. */
hdg_status hdg_condense_hex(hdg_problem p, int64_t e0, int64_t count, int nquad, const double* verts,
                            const int32_t* face_perm, const hdg_physics* phys, const double* ru,
                            const double* ruh, int on_device, void* stream);

/* How hdg_condense_hex / hdg_hex_blocks form M^e and B_d: 1 (default) by sum
 * factorisation of the tensor-product rule (three 1D contractions per
 * weight field, FP64; used for k <= 4 and 2 <= nquad <= 8), 0 by dense products
 * of the weighted basis tables on the condensation's GEMM path.  Both give
 * the same integrals up to rounding.  Errors: HDG_ERR_ARG. */
hdg_status hdg_set_hex_generation(hdg_problem p, int sum_factorised);

/* The generated blocks themselves (tests, callers that keep them): out[9]
 * are device buffers for Me, Bd, Cd, D, E, F, G, H, J of `count` elements in
 * hdg_condense's layout.  Inputs as hdg_condense_hex. */
hdg_status hdg_hex_blocks(hdg_problem p, int64_t count, int nquad, const double* verts, const int32_t* face_perm,
                          const hdg_physics* phys, double* const* out, int on_device, void* stream);

/* hdg_condense with per-input element strides.  blocks[11] are the inputs in
 * the order Me, Bd, Cd, D, E, F, G, H, J, ru, ruh; elem_stride[i] (doubles)
 * is either the input's size per element (one block per element, as in
 * hdg_condense) or 0: one block shared by all `count` elements (identical
 * elements of a structured mesh with constant coefficients).  A shared M^e is
 * inverted once; when all eleven inputs are shared, one element is condensed
 * and its results are copied to the others.  elem_stride may be NULL (all
 * per element).  Errors as hdg_condense; HDG_ERR_ARG for any other stride. */
hdg_status hdg_condense_strided(hdg_problem p, int64_t e0, int64_t count, const double* const* blocks,
                                const int64_t* elem_stride, int on_device, void* stream);

/* Dirichlet trace values u_D (b_hat = uhat - u_D on Dirichlet faces, Sec.
 * 2.1): host or device, n_face x b x R; rows of free faces are ignored.
 * Defaults to zero.  Must be set before hdg_assemble.  From host memory the
 * copy runs on the problem's copy stream as soon as the earlier operations
 * on the stored values are done, overlapping other work still queued on
 * `stream`; the call returns once the caller's buffer has been read, and
 * later work on `stream` sees the new values. */
hdg_status hdg_set_dirichlet(hdg_problem p, const double* uhat_dirichlet, int on_device, void* stream);

/* Face-based assembly (Sec. 4.2): for every free face f the face row of K,
 * (2N_lfe-1) blocks of b x b (diagonal K_ff = Kbar^{e1}_{l1l1} +
 * Kbar^{e2}_{l2l2}, off-diagonal K_fg = Kbar^e_{l(f)l(g)}), stored in FP64 and,
 * when `opts` needs them, FP32/BF16 copies; r_f = sum_e rbar^e_l minus the
 * Dirichlet columns times u_D.  Errors: HDG_ERR_STATE if not every element
 * was condensed. */
hdg_status hdg_assemble(hdg_problem p, const hdg_solver_opts* opts, void* stream);

/* Preconditioner setup: block-Jacobi inverses of K_ff (Sec. 4.5, FP64 with
 * partial pivoting), ASM element matrices and inverses (Sec. 4.6), and for a
 * polynomial preconditioner one Arnoldi(P) cycle (MGS) with A = M^{-1} K from
 * the start vector `v0` (device, n_dof doubles), harmonic Ritz values and
 * Leja order (Sec. 4.7) or Chebyshev bounds.  v0 may be NULL when
 * opts->poly == HDG_POLY_NONE.  Errors: HDG_ERR_SINGULAR, HDG_ERR_ARG.
 * Inverses (BJ blocks, ASM patches, and Ebar and M^e in the condensation)
 * of order <= 169 run as Gauss-Jordan with partial pivoting in one CTA's
 * shared memory; larger ones split into 2 x 2 blocks (leading block and its
 * Schur complement, recursively), which needs a nonsingular leading block
 * (SPD matrices, or a positive definite symmetric part, as for the HDG
 * local and patch matrices). */
hdg_status hdg_setup_precond(hdg_problem p, const hdg_solver_opts* opts, const double* v0, void* stream);

/* Restarted left-preconditioned GMRES(m) on K x = r for all R right-hand
 * sides (Sec. 3.1, Sec. 4.4), x0 = 0.  The solution stays on the device; read
 * it with hdg_get_trace.  `info` (host, may be NULL) receives the counts.
 * Returns HDG_OK when every RHS met rtol, HDG_ERR_NOT_CONVERGED otherwise. */
hdg_status hdg_solve(hdg_problem p, const hdg_solver_opts* opts, void* stream, hdg_solve_info* info);

/* Restarted GMRES(m) for several problems at once (Sec. 3.1, Sec. 4.4), the
 * batching of many small systems: ONE persistent cooperative launch runs the
 * cycles and iterations of all `count` problems in lock-step, each phase
 * (block-row products, block-Jacobi applies, Gram-Schmidt reductions, Givens
 * steps, restarts with the FP64 true residual) spread over the whole GPU
 * through ragged work lists over the problems' rows and vector entries, so
 * systems of different meshes, orders and block sizes share every launch
 * and no per-iteration launches remain.  Each problem's result does not
 * depend on the others in the batch (fixed summation orders); it can differ
 * from hdg_solve's in the last bits.  The paper solves one system at a time;
 * this entry point has no counterpart there.
 * Requirements: every problem assembled on the same device with
 * hdg_setup_precond(opts) done (pc HDG_PC_NONE or HDG_PC_BJ, no
 * polynomial), orth HDG_ORTH_CGS, and inner_prec HDG_FP64 (plain FP64) or
 * HDG_FP32 with max_outer = -1 (the restarted mixed mode: FP32 blocks and
 * block-Jacobi inverses in the cycles, FP64 true residual at every
 * restart); at most 256 problems of at most 2,097,152 entries (n_dof x R)
 * and block size b <= 256 each.  The solutions stay on the device (hdg_get_trace per problem);
 * infos (host, may be NULL) receives one hdg_solve_info per problem.
 * Allocates a few KB of stream-ordered device memory for the work lists.
 * Returns HDG_OK when every problem converged, HDG_ERR_NOT_CONVERGED
 * otherwise, HDG_ERR_ARG / HDG_ERR_STATE for unsupported options or a
 * problem not ready. */
hdg_status hdg_solve_batch(hdg_problem* problems, int count, const hdg_solver_opts* opts, void* stream,
                           hdg_solve_info* infos);

/* Full trace uhat (host or device): n_face x b x R, Dirichlet faces filled
 * with u_D.  A host buffer in pinned, mapped memory is written by the kernel
 * directly; a pageable one through a device buffer and a copy. */
hdg_status hdg_get_trace(hdg_problem p, double* uhat, int on_device, void* stream);

/* Element recovery (Eq. w19, Eq. w16): u^e = Ebar^{-1}(r_u - Fbar uhat^e),
 * q^e_{a,d} = -(M^e)^{-1}(B_d u^e_a + C_d uhat^e_a).  Outputs host or device:
 * u  n_elem x M*P_E x R,  q  n_elem x M*D*P_E x R.  Host outputs in
 * pinned, mapped memory are written by the kernel directly.  Pageable host
 * outputs of at least 2048 elements are recovered in up to 8 pieces, each
 * piece's copy to the host overlapping the next piece's computation.  Every
 * way gives the same values. */
hdg_status hdg_recover(hdg_problem p, double* u, double* q, int on_device, void* stream);

/* y = K x with K stored in `prec` (FP64, FP32 or BF16 blocks; products
 * accumulated in FP64 for FP64 blocks -- with R = 4 or 8 on the tensor cores
 * through exact digit expansions, see the autotuner's configuration 6 --,
 * FP32 otherwise) (Sec. 4.3).  x, y: device, n_dof x R doubles.  For tests
 * and benchmarks. */
hdg_status hdg_apply_K(hdg_problem p, int prec, const double* x, double* y, void* stream);

/* y = P^{-1} x for the preconditioner of the last hdg_setup_precond call,
 * blocks in `prec` (Sec. 4.5-4.7).  x, y: device, n_dof x R doubles. */
hdg_status hdg_apply_precond(hdg_problem p, const hdg_solver_opts* opts, int prec,
                             const double* x, double* y, void* stream);

/* Copy condensed element data to the host: Kbar (count x n x n, n =
 * N_lfe*M*P_F) and rbar (count x n x R); either may be NULL. */
hdg_status hdg_get_condensed(hdg_problem p, int64_t e0, int64_t count, double* Kbar, double* rbar);

/* Copy the assembled right-hand side r (host, n_dof x R) and the FP64 face
 * row blocks of free faces [f0, f0+count) (host, count x (2N_lfe-1) x b x b,
 * slot s of face row f couples f with free face nbr[f][s]; zero blocks where
 * nbr = -1) together with nbr (host, count x (2N_lfe-1) int32).  Any pointer
 * may be NULL. */
hdg_status hdg_get_face_rows(hdg_problem p, int64_t f0, int64_t count, double* blocks,
                             int32_t* nbr, double* r);

/* Polynomial coefficients of the last setup: theta (Leja order) as real and
 * imaginary parts (host, capacity `cap`), or for Chebyshev (alpha, beta) in
 * re[0], re[1].  *n receives the count. */
hdg_status hdg_get_poly(hdg_problem p, double* re, double* im, int cap, int* n);

/* Event timing while enabled: hdg_set_timing(p, 1) clears and enables,
 * hdg_get_timing returns the summed device time (ms) and launch count of
 *   kind 0-2: the block-row matvec launches (hdg_solve, hdg_apply_K and the
 *             polynomial steps) with blocks in precision HDG_FP64, HDG_FP32,
 *             HDG_BF16 (the block-row kernel only, not the FP32 copy of x);
 *   kind 3:   the tensor-core condensation products of hdg_condense (each
 *             the exponent pass plus the product kernel);
 *   kind 4-5: the block-Jacobi applies of the low-precision polynomial
 *             preconditioner (each with the recurrence step in its
 *             epilogue) with blocks in FP32, BF16.
 * The events are recorded on the caller's stream around each launch;
 * hdg_condense then synchronizes the stream to read them. */
hdg_status hdg_set_timing(hdg_problem p, int enable);
hdg_status hdg_get_timing(hdg_problem p, int kind, double* total_ms, int64_t* launches);

/* y = K x with FP32 or BF16 blocks (prec = HDG_FP32 / HDG_BF16), like
 * hdg_apply_K, but without allocating device memory.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc
 * when they need the product (code inside a stream capture, hosts whose
 * device memory belongs to their own pool allocator, latency-critical loops).
 * The FP32 copy of x that the product needs goes to a static device array of
 * 8,388,608 floats (32 MiB) that every GPU loading the library holds until
 * the process exits; n_dof * R above that limit returns HDG_ERR_ARG, as does
 * prec = HDG_FP64.  The problem must be assembled (HDG_ERR_STATE otherwise).
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other problems on the same device) race and must be ordered by the
 * caller.  Nothing in the array needs to start at zero.  The looked-up
 * address is kept for the life of the process, so a device reset
 * (cudaDeviceReset) after the first call on that device is not supported.
 * x, y: device, n_dof x R doubles. */
hdg_status hdg_apply_K_noalloc(hdg_problem p, int prec, const double* x, double* y, void* stream);

/* GMRES cycles as CUDA graphs (default on): each cycle of hdg_solve is
 * captured once per option set as m conditional (IF) nodes, one per
 * iteration, and replayed; the device-side Givens step switches the
 * remaining iterations off after convergence.  enable = 0 launches the
 * iterations one by one instead (the host then polls a progress flag two
 * iterations behind).  Event timing (hdg_set_timing) also uses the one-by-one
 * launches.  Results are identical either way. */
hdg_status hdg_set_graphs(hdg_problem p, int enable);

/* Number of CUDA kernels the library has launched in this process. */
long long hdg_launch_count(void);

/* Kernel variant of the block-row products (matvec, BJ and ASM applies):
 * 0 = one thread per output row with direct global loads (default),
 * 1 = shared-memory staging with bulk copies.  Used by the autotuner;
 * results agree to rounding. */
hdg_status hdg_set_kernel_variant(hdg_problem p, int variant);

/* ---------------------------------------------------------- dense products
 * Batched FP64 GEMM, the building block of the static condensation
 * (Sec. 4.1, Eqs. w16-w22): C_b = alpha A_b B_b + beta C_b for
 * b = 0..count-1, row-major M x K, K x N and M x N matrices (device
 * pointers; leading dimensions and batch strides in elements).
 *   mode 0: FP64 CUDA cores.
 *   mode 1: BF16 tensor cores (tcgen05) with exact operand splitting: each
 *           row of A and column of B in 56-bit fixed point relative to its
 *           largest entry, as 8 digits of 7 bits; digit products summed
 *           exactly in FP32 per digit weight; the result rounded once to FP64.
 *           The error is within a small factor of FP64 rounding,
 *           |err_ij| <= 2^-54 K max_k|A_ik| max_k|B_kj| for K <= 192 (the
 *           exactness bound of the accumulators); larger K runs in slices of
 *           at most 192, each rounded to FP64 and accumulated into C.  Needs
 *           N >= 16 (HDG_ERR_ARG otherwise); HDG_ERR_NAN if an input is Inf
 *           or NaN (the result is then not defined).  The digits are
 *           computed inside the product kernel for every output tile from the
 *           FP64 operands ((M + N) * count 16-bit words of stream-ordered
 *           scratch from cudaMallocAsync).
 *   mode 2: as mode 1 (K <= 192), with each operand split once into BF16 digit planes
 *           in device memory (16 bytes per entry, twice the FP64 operand)
 *           that the product kernel moves with bulk copies; the same
 *           results, slower at the condensation shapes (the plane traffic
 *           bounds it).
 *   mode 3: as mode 1 (K <= 192) with one persistent CTA per SM walking all output
 *           tiles (accumulators double-buffered in TMEM for 32-column
 *           tiles); the same results, slower at the condensation shapes.  Synchronizes `stream` to read the error word it shares
 * with other calls of this function in the process (do not call it
 * concurrently).  The paper
 * condenses on the GPU with batched vendor BLAS (cuBLAS/hipBLAS GEMMs and
 * inverses, Sec. 4.1); this entry point, the library's own tensor-core
 * product, has no counterpart there. */
hdg_status hdg_gemm_f64(int mode, int M, int N, int K, const double* A, int64_t lda, int64_t sA, const double* B,
                        int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC, double alpha, double beta,
                        int64_t count, void* stream);

/* Elements per condensation chunk (default: as many as ~1 GiB of staging and
 * temporaries hold, the most allowed).  With host inputs and several chunks
 * the copies of chunk c+1 overlap the condensation of chunk c (two staging
 * buffers, a copy stream ordered by events).  HDG_ERR_ARG for elems < 1 or
 * above the default. */
hdg_status hdg_set_condense_chunk(hdg_problem p, int64_t elems);

/* Condensation products of this problem on the tensor cores (mode 1, the
 * default, 2 or 3, as hdg_gemm_f64 modes 1-3, where K <= 192 and N >= 16)
 * or on the FP64 cores (mode 0).  Mode 2 keeps a digit-plane buffer of the
 * largest product of a condensation chunk (grown on first use).
 * HDG_ERR_ARG for another mode. */
hdg_status hdg_set_condense_mode(hdg_problem p, int mode);

/* ---------------------------------------------------------------- autotuner
 * Launch configurations of the block-row products (the face-block matvec of
 * Sec. 4.2, the block-Jacobi apply of Sec. 4.3 and the additive-Schwarz
 * element solves of Sec. 4.3), chosen by measurement.  The paper fixes one
 * mapping per kernel; this tuning has no counterpart there.
 *
 * op: 0 = K (matvec), 1 = block-Jacobi apply, 2 = additive-Schwarz apply.
 * prec: HDG_FP64 / HDG_FP32 / HDG_BF16 block storage.
 * A configuration is three ints {kind, sp, cps}: kind 0 = heuristic default
 * (vectorised 16-byte loads for FP32/BF16 blocks whose rows divide into
 * 16-byte groups; FP64 rows split over slot parts when one thread per row
 * would fill less than 2048 threads per SM; else one thread per row), 1 =
 * shared-memory staging with bulk copies, 2 = one thread per output row, 3 =
 * 16-byte loads of 4 (FP32) or 8 (BF16) rows per thread with the slots of a
 * row split over sp adjacent lanes (sp in {1,2,4,8}), 4 = FP64 rows with the
 * slots split over sp adjacent lanes (sp in {2,4,8}) and a shuffle
 * reduction, 5 = FP32/BF16 blocks of whole face rows streamed by one bulk
 * copy each (evict-first in L2) into a shared-memory ring of one persistent
 * CTA per SM, 16-byte vectors of 4 (FP32) or 8 (BF16) rows per thread, the
 * columns split over the CTA's warps (units whose blocks exceed 48 KB fall
 * back to the default), 6 = FP64 blocks with R = 4 or 8 right-hand sides
 * (square blocks of at most 32 rows) on the BF16 tensor cores: K kept as
 * exact 8-digit expansions of 54-bit fixed point per row (rebuilt by every
 * hdg_assemble, 8 bytes per entry next to the FP64 blocks), the gathered x
 * split the same way per face row and RHS, the digit products summed exactly
 * and the result rounded once to FP64 (error below 4 * 2^-53 * ncol *
 * max_j |K_ij| * max_j |x_jr| over the row's ncol columns); the default for
 * those shapes, 7 = kind 3 compiled for more resident 256-thread CTAs per
 * SM: three (at most 80 registers per thread) at R = 8 with sp in {1,2}, four
 * (at most 64) for FP32 blocks at R <= 2 with sp in {1,2,4}; otherwise as
 * kind 3; 8 = kind 7 at R = 8 with the right-hand sides split over two
 * threads (4 each), sp in {1,2}; cps = CTAs per SM of the grid-stride launch
 * (0 = heuristic).  Every other configuration computes the same sums; they differ
 * in summation order only. */

/* Time every candidate configuration of every operation the problem can run
 * now (K at each stored precision; BJ or ASM when set up) with `reps`
 * back-to-back launches (0 = 10) after two warm-up launches, on `stream`, and
 * keep the fastest.  Choices are cached per block shape for the process:
 * unless `force`, a problem whose shapes were tuned before adopts the cached
 * choice without timing.  Synchronizes `stream`.  Requires hdg_assemble
 * (HDG_ERR_STATE otherwise).  Overwrites the problem's GMRES scratch
 * vectors (not the solution). */
hdg_status hdg_autotune(hdg_problem p, int reps, int force, void* stream);

/* The configuration in use for (op, prec) -> cfg3[3], with the measured
 * microseconds per launch of it and of the heuristic default (0 when not
 * tuned). */
hdg_status hdg_get_tuning(hdg_problem p, int op, int prec, int* cfg3, float* us_tuned, float* us_default);

/* Candidate configurations for (op, prec): writes min(n, cap) triples to
 * cfg3 (may be NULL) and returns n; -1 on bad arguments. */
int hdg_tuning_candidates(hdg_problem p, int op, int prec, int* cfg3, int cap);

/* Use configuration cfg3 for (op, prec) (e.g. one from
 * hdg_tuning_candidates).  HDG_ERR_ARG for values outside the ranges above. */
hdg_status hdg_set_tuning(hdg_problem p, int op, int prec, const int* cfg3);

#ifdef __cplusplus
}
#endif

#endif /* HDG_H */
