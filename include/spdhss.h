/*
 * spdhss.h - C ABI of the GB300 implementation of the SPD HSS preconditioner for
 * SPD H^2 kernel matrices (Xing, Huang, Chow: "Efficient construction of an HSS
 * preconditioner for symmetric positive definite H^2 matrices").
 *
 * Pipeline (problem statement of Sec. 5.2 and Sec. 6):
 *   points + kernel + diagonal shift
 *     -> h2_build      cluster tree, admissibility lists, proxy-point H^2 (Sec. 5.1, Sec. 6)
 *     -> spdhss_build  SPD HSS by accelerated scaling-and-compression (Alg. 5.3)
 *     -> ulv_factor    ULV factorization of the SPD HSS matrix (Sec. 1, Sec. 6)
 *     -> pcg_solve     PCG with the H^2 matvec and the ULV preconditioner (Sec. 6.2)
 *
 * Conventions shared by every call:
 *  - All floating point data is IEEE binary64 (double).
 *  - Points are row-major n x dim (point p at points[p*dim .. p*dim+dim-1]).
 *  - Block vectors (right-hand sides, products, sketches) are column-major n x ncol with
 *    leading dimension ld >= n, and are in the ORIGINAL point order; the library applies
 *    the tree permutation internally.
 *  - Unless a call says otherwise, array arguments are device pointers (memory the caller
 *    allocated with cudaMalloc or a PyTorch CUDA tensor); the caller owns them.  Handles
 *    own their device memory and release it in the matching *_destroy call.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *    Calls enqueue their kernels on it.  Calls that must size allocations or return
 *    host results synchronize that stream before returning.
 *  - Every call returns a status and never exits or traps.  On failure a message is
 *    available from spdhss_last_error() (thread-local, valid until the next call).
 *  - Handles are not thread-safe: one handle must not be used by two threads at once.
 */
#ifndef SPDHSS_H
#define SPDHSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPDHSS_OK = 0,
  SPDHSS_EINVAL = 1,          /* invalid argument (size, pointer, layout) */
  SPDHSS_ENOMEM = 2,          /* device or host allocation failed */
  SPDHSS_NOT_SPD = 3,         /* a Cholesky factorization met a non-positive pivot */
  SPDHSS_NO_CONVERGENCE = 4,  /* PCG reached maxit before the tolerance */
  SPDHSS_NUMERIC = 5,         /* NaN or Inf met */
  SPDHSS_TIMEOUT = 6,         /* a bounded device-side wait gave up */
  SPDHSS_ECUDA = 7            /* a CUDA runtime call failed */
} spdhss_status;

/* Kernel functions of Sec. 6, with a length scale ell that divides the distance r:
 * EXP exp(-r/ell); GAUSS exp(-r^2/ell^2); MATERN32 (1+sqrt3 r/ell) exp(-sqrt3 r/ell);
 * IMQ 1/sqrt(1 + r^2/ell^2).  K(x,x) = 1.  The matrix is A = shift*I + K(X,X).
 * RPY is the Rotne-Prager-Yamakawa tensor of Sec. 6 for 3D points, ell = the particle
 * radius a (r = x - y):
 *   r = 0: (1/a) I;   |r| >= 2a: 3/(4|r|)(I + rr^T/|r|^2) + 3a^2/(2|r|^3)(I/3 - rr^T/|r|^2);
 *   |r| < 2a: (1/a)[(1 - 9|r|/(32a)) I + 3|r|/(32a) rr^T/|r|^2]
 * (the overlap branch read with 1/a on both terms, the form continuous at |r| = 2a).  Its
 * matrix has THREE unknowns per point: with n points it is 3n x 3n, row 3p + c being
 * component c of point p, and every "n" below (block vector rows, h2_info[0], the
 * exported permutation and index ranges, skeleton indices) counts unknowns, 3n. */
typedef enum {
  SPDHSS_K_EXP = 0,
  SPDHSS_K_GAUSS = 1,
  SPDHSS_K_MATERN32 = 2,
  SPDHSS_K_IMQ = 3,
  SPDHSS_K_RPY = 4
} spdhss_kernel_kind;

typedef struct {
  int kind;       /* spdhss_kernel_kind */
  double ell;     /* length scale (RPY: particle radius a), > 0 */
  double shift;   /* diagonal shift sigma >= 0 (Sec. 6.2) */
} spdhss_kernel_desc;

typedef struct spdhss_h2_s* h2_handle;
typedef struct spdhss_hss_s* hss_handle;
typedef struct spdhss_ulv_s* ulv_handle;

/* ---- H^2 representation (Sec. 5.1; proxy point construction of Sec. 6) -------------
 * h2_build: cluster tree (2^dim-ary box bisection until a box holds <= leaf_size points,
 * shallow leaves padded to the deepest level), admissibility lists (Type-1 near pairs,
 * Type-3 far pairs of Sec. 5.2.2) and a proxy-point H^2 representation whose
 * interpolative decompositions stop at relative pivot size `tol` (the paper uses 1e-8).
 *   points   n x dim row-major, HOST or DEVICE pointer (detected), read only.
 *   n >= 1 points, dim in {2, 3} (3 for RPY), leaf_size >= 1 points, tol >= 0 (0 keeps
 *   full rank: exact H^2).  For RPY every proxy point carries the three components.
 *   out      receives a new handle; destroy with h2_destroy.
 * Errors: EINVAL for bad sizes, ENOMEM, ECUDA. */
spdhss_status h2_build(const double* points, int64_t n, int dim, spdhss_kernel_desc kernel,
                       int leaf_size, double tol, void* stream, h2_handle* out);

/* Values of a scalar kernel function of Sec. 6 (EXP, GAUSS, MATERN32, IMQ; not RPY) at n
 * squared distances, computed on the device by the same code that fills every kernel
 * tile, proxy matrix and near-field block of the path (the diagonal shift is not added):
 *   out[i] = K(sqrt(r2[i])) with the descriptor's length scale.
 *   r2, out  DEVICE arrays of n doubles (n >= 0) that do not overlap.
 * The exponential of the EXP, GAUSS and MATERN32 kernels is a table-driven method (Tang
 * 1989, 64 entries): within two units in the last place of the exact value.
 * Errors: EINVAL for the RPY kind, a length scale <= 0, host pointers; ECUDA. */
spdhss_status spdhss_kernel_eval(spdhss_kernel_desc kernel, const double* r2, double* out,
                                 int64_t n, void* stream);

/* Y = A X with the H^2 matrix A (Sec. 5.1): upward pass, Type-3 couplings, downward pass,
 * and near-field kernel tiles evaluated on the fly (shift included).
 *   X, Y  device, n x nrhs column-major, leading dimension ld >= n, original point order.
 *   X and Y must not overlap.  nrhs >= 1. */
spdhss_status h2_matmul(h2_handle h2, const double* X, double* Y, int nrhs, int64_t ld,
                        void* stream);

/* Sizes of the tree and the H^2 data, written to the HOST array info[16]:
 *  [0] n (unknowns: 3 x points for RPY)  [1] dim  [2] number of tree nodes  [3] D (depth
 *  of the leaf level; HSS levels
 *  L = D + 1)  [4] entries of all near lists  [5] entries of all far lists
 *  [6] total skeleton size (sum of H^2 ranks)  [7] bytes of stored H^2 generators
 *  (bases, transfers, couplings)  [8] near-field kernel entries per matvec
 *  [9] coupling entries per matvec  [10] basis/transfer entries per matvec
 *  [11] largest H^2 rank  [12..15] reserved (0). */
spdhss_status h2_info(h2_handle h2, int64_t* info);

/* Export of the cluster tree for parity checks; every pointer is a HOST array sized from
 * h2_info (nn = info[2], nnear = info[4], nfar = info[5]); any pointer may be NULL.
 *   perm[n]           sorted position -> original index (of the unknown, for RPY)
 *   depth_off[D+2]    nodes of depth t are [depth_off[t], depth_off[t+1])
 *   begin[nn], end[nn]  range of sorted positions (unknowns for RPY: 3 x the points')
 *   parent[nn]        -1 for the root
 *   cell_lo[nn*dim], cell_hi[nn*dim]  integer cell on the finest grid, row-major
 *   near_off[nn+1], near_idx[nnear], far_off[nn+1], far_idx[nfar]  CSR lists */
spdhss_status h2_export_tree(h2_handle h2, int64_t* perm, int64_t* depth_off, int64_t* begin,
                             int64_t* end, int64_t* parent, int64_t* cell_lo, int64_t* cell_hi,
                             int64_t* near_off, int64_t* near_idx, int64_t* far_off,
                             int64_t* far_idx);

/* Export of the H^2 skeletons (HOST arrays): skel_off[nn+1] (node i owns
 * skel_idx[skel_off[i] .. skel_off[i+1]-1]), skel_idx[info[6]] = sorted-order point
 * (for RPY: unknown) indices in pivot order.  Either pointer may be NULL. */
spdhss_status h2_export_skeletons(h2_handle h2, int64_t* skel_off, int64_t* skel_idx);

spdhss_status h2_destroy(h2_handle h2);

/* ---- SPD HSS construction (Alg. 5.3 with Alg. 5.1 and Alg. 5.2) ----------------------
 * Builds the SPD HSS approximation {A_ii, U_i, R_i, B_ij} of the H^2 matrix with rank cap
 * `rank` (r) and oversampling `oversample` (p, the paper uses 10); rank 0 gives the block
 * diagonal of the leaf blocks (the block-Jacobi preconditioner).  The Gaussian sketch
 * Omega is n x (r+p):
 *   omega   DEVICE pointer, column-major, leading dimension n, original point order; or
 *           NULL, in which case Omega is drawn on the device from `seed`.
 * (I + bold B_ii) is factored by Cholesky (equivalent to the symmetric square root of
 * Eq. Si0 up to an orthogonal factor that the pivoted QR absorbs).
 * Errors: NOT_SPD (message names the node) when a Cholesky factorization fails, EINVAL,
 * ENOMEM, ECUDA. */
spdhss_status spdhss_build(h2_handle h2, int rank, int oversample, const double* omega,
                           uint64_t seed, void* stream, hss_handle* out);

/* Tolerance-driven variant of spdhss_build: every basis is truncated at the relative
 * tolerance `tol` (the column-pivoted QR of the scaled sample stops when the largest
 * remaining column norm is <= tol times the first), `rank` being the largest rank allowed;
 * tol = 0 is spdhss_build.  The sketch grows: an attempt with rank cap r uses the first
 * r + oversample sketch columns (of omega, which then holds rank + oversample columns, or
 * of the device sketch, whose columns do not depend on its width); starting from
 * r = min(rank, 64), r doubles until every rank is below r or r reaches `rank` (each
 * attempt is a full construction).  The result is SPD for every tol (Sec. 3.2).  EINVAL
 * unless 0 <= tol < 1. */
spdhss_status spdhss_build_tol(h2_handle h2, int rank, double tol, int oversample,
                               const double* omega, uint64_t seed, void* stream,
                               hss_handle* out);

/* spdhss_build_tol with a precision mode for the sampling product Y^(k) = (A - blkdiag_k A)
 * Omega, the construction's dominant cost (Sec. 6.1):
 *   precision 0: FP64 throughout (= spdhss_build_tol);
 *   precision 1: the H^2 product run in FP32 (FP32 copies of the bases and couplings made
 *                on first use and kept in the H^2 handle, near-field kernel entries
 *                evaluated in FP32, FP32 accumulation), its basis and coupling GEMMs on
 *                the tensor cores with split operands (3xTF32: FP32-accurate products);
 *   precision 2: the same with plain TF32 products (about 1e-3 relative error per product).
 * Everything after the sampling stays FP64: the diagonal-block Cholesky factorizations,
 * the triangular solves, the column-pivoted QR that compresses the scaled samples into
 * orthonormal bases, and the formation of B_ij, U_i and R_i, so that the result keeps the
 * SPD guarantee of Sec. 3.2 (the bases are orthonormal to FP64 rounding).  Errors as
 * spdhss_build_tol, and EINVAL for another precision, TIMEOUT if a bounded wait in a
 * tensor-core kernel gave up. */
spdhss_status spdhss_build_precision(h2_handle h2, int rank, double tol, int oversample,
                                     const double* omega, uint64_t seed, int precision,
                                     void* stream, hss_handle* out);

/* Y = H X with the HSS approximation H (same layout rules as h2_matmul). */
spdhss_status hss_matmul(hss_handle hss, const double* X, double* Y, int nrhs, int64_t ld,
                         void* stream);

/* HOST info[8]: [0] number of HSS levels L  [1] largest rank r_i  [2] bytes of stored HSS
 * generators  [3] number of nodes  [4..7] reserved. */
spdhss_status hss_info(hss_handle hss, int64_t* info);

spdhss_status hss_destroy(hss_handle hss);

/* ---- ULV factorization and solve (Sec. 1 and Sec. 6) -----------------------------------
 * The paper factors the SPD HSS matrix with the ULV factorization it cites (Sec. 1; the
 * reported construction times include it, Sec. 6) and applies the factors as the PCG
 * preconditioner; it does not spell out the steps.
 * ulv_factor: symmetric ULV of the SPD HSS matrix (orthogonal compression of every
 * basis, Cholesky elimination of the complement, Schur update, dense Cholesky at the
 * root).  Every Cholesky exists in exact arithmetic because the SPD HSS matrix is SPD
 * (Sec. 3.2).  Errors: NOT_SPD if a pivot is not positive, ENOMEM, ECUDA. */
spdhss_status ulv_factor(hss_handle hss, void* stream, ulv_handle* out);

/* X = H^{-1} B: the forward and backward sweeps of the ULV factors (the preconditioner
 * apply of Sec. 6).  B, X device, n x nrhs column-major, leading dimension ld, original
 * order; B and X may be the same array.  Errors: EINVAL, ENOMEM, ECUDA. */
spdhss_status ulv_solve(ulv_handle ulv, const double* B, double* X, int nrhs, int64_t ld,
                        void* stream);

spdhss_status ulv_destroy(ulv_handle ulv);

/* X = H^{-1} B like ulv_solve, for callers that cannot allocate device memory (an
 * application whose device memory is all reserved by its own allocator, or a latency-
 * critical path that cannot accept the device-wide synchronization of cudaMalloc and
 * cudaFree).  The paper has no counterpart: this is a property of the library, not of the
 * method.  The call allocates no device memory: it works in two fixed device arrays that
 * are part of the library image (48 MiB of level buffers, 8 MiB of launch descriptors),
 * held by every GPU that loads them until the process exits.
 *   B, X     DEVICE pointers, n x nrhs column-major, leading dimension ld >= n, original
 *            point order; B and X may be the same array.
 *   Limit:   the level buffers need about (n + sum of the block sizes above the leaves) x
 *            nrhs doubles (roughly 2 to 3 x n x nrhs); a call that needs more than 6 Mi
 *            doubles, or more than 8 MiB of descriptors, returns EINVAL and does nothing.
 *   Loading: the library's device code is loaded lazily, and loading the two arrays takes
 *            their 56 MiB from the device.  ulv_factor, which allocates anyway, loads them
 *            on its device and looks up their addresses (once per device, with that device
 *            current), so that this call allocates nothing.  Only a call on a device where
 *            no ulv_factor has run loads them itself; make that first call before any
 *            stream capture.
 *   Descriptors: built on the host once per (handle, nrhs) and kept, unchanged, by the
 *            handle until ulv_destroy; every call copies them into the descriptor array
 *            (a host-to-device copy of a few KB to a few MB on `stream`).
 *   Every call shares the two arrays and leaves its data there; nothing needs to start at
 *   zero.  Calls whose work overlaps on the GPU (different streams) race on the arrays:
 *   serialize them, e.g. on one stream.
 * Errors: EINVAL (NULL pointer, nrhs < 1, ld < n, sizes over the arrays), ECUDA. */
spdhss_status ulv_solve_noalloc(ulv_handle ulv, const double* B, double* X, int nrhs,
                                int64_t ld, void* stream);

/* ---- PCG (Sec. 6.2) ------------------------------------------------------------------
 * Solves A X = B with the H^2 matrix A and the ULV-factored SPD HSS preconditioner, from
 * X_0 = 0, every column independently, until the relative residual of every column is
 * <= relres_tol (recursive residual, confirmed by a recomputed true residual) or maxit
 * iterations.  ulv = NULL runs unpreconditioned CG (the baseline of the paper's
 * iteration tables); so does pcg_solve_mixed.
 *   B, X          n x nrhs column-major, leading dimension ld, original order; HOST or
 *                 DEVICE pointers (detected; host data is staged through the device).
 *   iters_out     HOST int[nrhs] or NULL: iterations taken per column.
 *   relres_out    HOST double[nrhs] or NULL: final true relative residual per column.
 * Returns NO_CONVERGENCE if some column missed the tolerance (X holds the last iterate). */
spdhss_status pcg_solve(h2_handle h2, ulv_handle ulv, const double* B, double* X, int nrhs,
                        int64_t ld, double relres_tol, int maxit, int* iters_out,
                        double* relres_out, void* stream);

/* ---- mixed precision (FP32 products, FP64 factorizations and residuals) ---------------
 * h2_matmul_mixed: Y = A X like h2_matmul, computed with an FP32 copy of the H^2 generators
 * (made on the first mixed call and kept in the handle), FP32 near-field kernel entries and
 * FP32 accumulation; X and Y are FP64.  Relative error ~1e-6.  nrhs in [1, 16].
 * pcg_solve_mixed: pcg_solve whose products with A inside the iteration are the FP32
 * product; the ULV preconditioner, the recurrences and the residuals stay FP64, and
 * convergence is declared on the FP64 true residual.  Every 50 iterations the recursive
 * residual is replaced by the FP64 true residual; a column whose true residual is above
 * twice its recursive one also restarts its direction (the solve then proceeds as
 * iterative refinement with FP32 inner iterations), and when a block of 50 iterations has
 * lowered some column's true residual by less than 10% the remaining iterations use the
 * FP64 product (all columns restarting): kernel systems whose solution is dominated by
 * the smallest eigenvalues put the FP32 product's error close to the residual itself.
 * Arguments as pcg_solve, nrhs in [1, 16]. */
spdhss_status h2_matmul_mixed(h2_handle h2, const double* X, double* Y, int nrhs, int64_t ld,
                              void* stream);
spdhss_status pcg_solve_mixed(h2_handle h2, ulv_handle ulv, const double* B, double* X,
                              int nrhs, int64_t ld, double relres_tol, int maxit, int* iters_out,
                              double* relres_out, void* stream);

/* ---- FP32 grouped GEMM (test and benchmark hook) -------------------------------------
 * C = alpha op(A) op(B) + beta C for one M x N x K product of FP32 column-major DEVICE
 * matrices (op = transpose when tA / tB is 1), through the library's grouped GEMM:
 * mode 0 on the CUDA cores (FP32 FMA), mode 1 on the tensor cores in TF32 (tcgen05.mma
 * kind::tf32, FP32 accumulation), mode 2 on the tensor cores with every operand split into
 * two TF32 parts (3xTF32: FP32-accurate products); mode 3 is a test of the tensor-core
 * kernel's bounded waits (it issues no MMA, its waits give up after about a second and the
 * call returns TIMEOUT).  The FP32 H^2 products of the precision mode use modes 1 and 2.  The paper has no counterpart: the operation is the
 * dense GEMM the H^2 products consist of.  Synchronizes `stream`.  Errors: EINVAL,
 * TIMEOUT (a bounded wait in the tensor-core kernel gave up), ECUDA. */
spdhss_status spdhss_gemm_f32(int M, int N, int K, const float* A, int64_t lda, int tA,
                              const float* B, int64_t ldb, int tB, float* C, int64_t ldc,
                              float alpha, float beta, int mode, void* stream);

/* ---- batched level sweep over independent instances -----------------------------------
 * The construction of Alg. 5.3 (with the H^2 build before it and the ULV factorization
 * after it) proceeds level by level with the same steps for every matrix; for many
 * independent matrices these calls run them together: one host thread per instance
 * prepares that instance's descriptors, and every batched kernel launch (grouped GEMM,
 * kernel tiles, proxy matrices, near field, Cholesky, TRSM, pivoted QR, reflectors,
 * copies) takes the nodes of all instances at the same step, so the GPU sees one launch
 * per step instead of one per step and instance.  Instances at different steps (other
 * depths, other iteration counts) form separate launches; an instance that fails leaves
 * the sweep without stopping the others.  Every instance's results are bit-identical to
 * those of the one-instance calls: each kernel's per-problem arithmetic (variant, split of
 * a sum over CTAs, lanes per column) is fixed by that problem and its own instance, never
 * by the other instances sharing a launch.
 * All work runs on `stream`.  Arrays are HOST arrays of `count` entries.
 *
 * spdhss_build_batched: for instance i, h2_build(points[i], n[i], dim[i], kernel[i],
 *   leaf_size[i], tol[i]) -> spdhss_build_precision(rank[i], 0, oversample[i], omega[i],
 *   seed[i], precision[i]) ->
 *   ulv_factor.  points[i]: n[i] x dim[i] column-major, HOST or DEVICE.  omega: NULL, or a
 *   HOST array of `count` entries, each NULL (the sketch drawn from seed[i]) or a DEVICE
 *   n[i] x (rank[i] + oversample[i]) column-major sketch as spdhss_build's.  precision: NULL
 *   (all 0) or a HOST array of `count` modes as spdhss_build_precision's.  Outputs: HOST
 *   arrays of handles (NULL entry where that instance failed) and status[i] per instance
 *   (may be NULL).  Returns OK when every instance succeeded, else the first failing
 *   instance's status (spdhss_last_error names it).  The caller destroys the handles.
 * pcg_solve_batched: pcg_solve for every instance (B[i], X[i]: n_i x nrhs[i], ld[i];
 *   iters_out[i] / relres_out[i]: HOST arrays of nrhs[i] entries or NULL), the iterations
 *   of all instances in lockstep from one host thread: every stage of an iteration is one
 *   launch over all instances still iterating (an instance leaves when it has converged).
 *   status[i] per instance (NO_CONVERGENCE for one that missed the tolerance).
 * pcg_solve_batched_mixed: pcg_solve_mixed for every instance in the same lockstep (the
 *   precision mode's solve, Sec. 6.2 with FP32 products): the FP32 H^2 products of all
 *   instances still iterating run as merged launches of their once-read plans, the ULV
 *   solves, recurrences, FP64 true residuals (every 50 iterations and at convergence) and
 *   the convergence test are those of pcg_solve_mixed.  Arguments as pcg_solve_batched,
 *   nrhs[i] in [1, 16]; every instance's X, iterations and residuals are bit-identical to
 *   its pcg_solve_mixed call.
 * pcg_solve_batched_ex: pcg_solve_batched (precision 0) or pcg_solve_batched_mixed
 *   (precision 1) that reports every instance as soon as it has finished, for callers that
 *   return results one by one (a serving loop): when instance i stops iterating (every
 *   column converged), its X[i], iters_out[i], relres_out[i] and status[i] are written,
 *   `stream` is synchronized, and on_done(user, i, status of i) is called on the calling
 *   thread, before the other instances continue; instances that run out of iterations are
 *   reported at the end.  Results are bit-identical to the calls without the callback.  The
 *   callback must not destroy any handle of the call (the remaining iterations may still
 *   launch kernels over a finished instance's data) and must not call into the library on
 *   `stream`.  on_done may be NULL. */
spdhss_status spdhss_build_batched(int count, const double* const* points, const int64_t* n,
                                   const int* dim, const spdhss_kernel_desc* kernel,
                                   const int* leaf_size, const double* tol, const int* rank,
                                   const int* oversample, const uint64_t* seed,
                                   const double* const* omega, const int* precision,
                                   void* stream,
                                   h2_handle* h2_out, hss_handle* hss_out, ulv_handle* ulv_out,
                                   spdhss_status* status);
spdhss_status pcg_solve_batched(int count, const h2_handle* h2, const ulv_handle* ulv,
                                const double* const* B, double* const* X, const int* nrhs,
                                const int64_t* ld, double relres_tol, int maxit,
                                int* const* iters_out, double* const* relres_out, void* stream,
                                spdhss_status* status);
spdhss_status pcg_solve_batched_mixed(int count, const h2_handle* h2, const ulv_handle* ulv,
                                      const double* const* B, double* const* X,
                                      const int* nrhs, const int64_t* ld, double relres_tol,
                                      int maxit, int* const* iters_out,
                                      double* const* relres_out, void* stream,
                                      spdhss_status* status);
typedef void (*spdhss_done_fn)(void* user, int instance, spdhss_status status);
spdhss_status pcg_solve_batched_ex(int count, const h2_handle* h2, const ulv_handle* ulv,
                                   const double* const* B, double* const* X, const int* nrhs,
                                   const int64_t* ld, double relres_tol, int maxit,
                                   int* const* iters_out, double* const* relres_out,
                                   void* stream, spdhss_status* status, int precision,
                                   spdhss_done_fn on_done, void* user);
/* Launches issued by the last batched call of the calling thread: merged[0] = launches of
 * the batched kernels after merging, merged[1] = the hand-overs they replaced. */
void spdhss_batched_stats(int64_t* merged);

/* ---- diagnostics ---------------------------------------------------------------------- */
const char* spdhss_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded. */
int64_t spdhss_launch_count(void);

/* Library version string. */
const char* spdhss_version(void);

/* Kernel timing for diagnostics.  spdhss_profile(1) clears the counters and brackets every
 * later launch with CUDA events on its stream (adds a small host cost per launch);
 * spdhss_profile(0) stops.  spdhss_profile_report writes a NUL-terminated JSON object
 * {"family": {"launches", "ms", "flops", "bytes"}, ...} into the HOST buffer buf of len
 * bytes (truncated if short) and returns the length the full report needs.  flops and
 * bytes are the algorithmic FP64 operations and operand bytes of the timed launches. */
void spdhss_profile(int enable);
int64_t spdhss_profile_report(char* buf, int64_t len);

/* Launch-variant autotuning (no counterpart in the paper: a GPU launch detail).  The first
 * launch of a tuned kind for a new shape bucket times each candidate variant once on a
 * synthetic problem set of that shape (private stream) and keeps the fastest for the
 * process, per device; only variants that leave the arithmetic unchanged are tuned (today
 * the columns per CTA of the blocked triangular solve), so results never depend on the
 * choice.  SPDHSS_TUNE=0 in the environment keeps the fixed launch rules.
 * spdhss_tuning_report writes the choices, one line per key ("dev0 trsm_blk n64 c8 p256 ->
 * 4  (1:ms 2:ms ...)"), NUL-terminated into the HOST buffer buf of len bytes (truncated if
 * short) and returns the length the full report needs. */
int64_t spdhss_tuning_report(char* buf, int64_t len);

#ifdef __cplusplus
}
#endif

#endif /* SPDHSS_H */
