// Batched FP64 dense kernels over per-node matrices of uneven sizes.  All matrices are
// column-major with an explicit leading dimension; every batch entry carries its own
// pointers and sizes, so one launch covers all nodes of a tree level.
#pragma once

#include "common.cuh"
#include "merge.cuh"

namespace spd {

// ---- grouped, segmented GEMM:  C = alpha * sum_s op(A_s) op(B_s) + beta * C -----------
// T = double (the FP64 path) or float (the mixed-precision H^2 products).
template <class T>
struct GemmSegT {
  const T* A;
  const T* B;
  int64_t lda, ldb;
  int K;
  int tA, tB;   // 1: use the transpose
};
template <class T>
struct GemmProbT {
  T* C;
  int64_t ldc;
  int M, N;
  int seg0, seg1;
  double alpha, beta;
  int tC = 0;   // 1: the product is stored transposed, (m, n) at C[n + m * ldc]
};
using GemmSeg = GemmSegT<double>;
using GemmProb = GemmProbT<double>;

// Host-side builder of one grouped GEMM launch.
template <class T>
struct GemmBatchT {
  std::vector<GemmSegT<T>> segs;
  std::vector<GemmProbT<T>> probs;
  // Start a problem; add its segments with seg(); beta applies once.
  void prob(T* C, int64_t ldc, int M, int N, double alpha, double beta) {
    GemmProbT<T> p;
    p.C = C; p.ldc = ldc; p.M = M; p.N = N; p.alpha = alpha; p.beta = beta;
    p.seg0 = p.seg1 = (int)segs.size();
    probs.push_back(p);
  }
  void seg(const T* A, int64_t lda, int tA, const T* B, int64_t ldb, int tB, int K) {
    GemmSegT<T> s;
    s.A = A; s.B = B; s.lda = lda; s.ldb = ldb; s.K = K; s.tA = tA; s.tB = tB;
    segs.push_back(s);
    probs.back().seg1 = (int)segs.size();
  }
  // single-segment convenience
  void add(T* C, int64_t ldc, int M, int N, const T* A, int64_t lda, int tA,
           const T* B, int64_t ldb, int tB, int K, double alpha, double beta) {
    prob(C, ldc, M, N, alpha, beta);
    seg(A, lda, tA, B, ldb, tB, K);
  }
  bool empty() const { return probs.empty(); }
  // upload() copies the descriptors to the device once; launch() may then be repeated.
  void upload(cudaStream_t s);
  void launch(cudaStream_t s) const;
  void run(cudaStream_t s) { upload(s); launch(s); }
  void clear() { segs.clear(); probs.clear(); tiles.clear(); kparts.clear(); reds.clear(); rednp.clear(); }
  std::vector<int4> tiles;   // (prob, m0, n0, K part + 1 or 0), grouped by kernel variant
  const char* tag = "gemm";
  // FP32 batches only: 0 CUDA cores; 1 tensor cores in TF32 (tcgen05, FP32 accumulation);
  // 2 tensor cores with split operands (3xTF32, FP32-accurate products)
  int tc = 0;
  int tc_nt = 0;             // tensor cores: tiles [0, tc_nt) are 128 x 64, the rest 128 x 128
  int tc_stall = 0;          // test of the bounded waits: issue nothing, let the waits expire
  int nb = 0;                        // 1/2/4: K-split kernel; 8/16/32: skinny kernel; 0: 64x64 tiles
  // launched problems: every problem in the orientation (C or C^T = B^T A^T) that wastes
  // the fewest padded FMAs, grouped by the kernel variant of its column count; one launch
  // per variant over the tile range [vbeg[v], vbeg[v + 1])
  std::vector<GemmProbT<T>> lprobs;
  std::vector<GemmSegT<T>> lsegs;
  std::vector<int> vnb;
  std::vector<int64_t> vbeg;
  double flops = 0.0, bytes = 0.0;   // algorithmic work of one launch
  DevBuf<GemmSegT<T>> d_segs;
  DevBuf<GemmProbT<T>> d_probs;
  DevBuf<int4> d_tiles;
  // K-split tiles of the few-column kernel: (k_lo, k_hi, slot) per split tile, and per
  // split output tile (problem, m0, n0, first slot) with its number of parts
  std::vector<int4> kparts, reds;
  std::vector<int> rednp;
  DevBuf<int4> d_kparts, d_reds;
  DevBuf<int> d_rednp;
  DevBuf<T> d_partial;
};
using GemmBatch = GemmBatchT<double>;
using SGemmBatch = GemmBatchT<float>;

// Tensor-core grouped FP32 GEMM (tc_gemm.cu): 128 x 64 tiles for problems of at most 64
// columns (the first n64 tiles), 128 x 128 for the others; split = 3xTF32.  A bounded wait that gives up sets the device error word,
// which tc_check() reads (and clears), throwing SPDHSS_TIMEOUT.
std::vector<int4> tc_gemm_tiles(const std::vector<GemmProbT<float>>& probs, int* n64_out);
void tc_gemm_launch(const GemmProbT<float>* d_probs, const GemmSegT<float>* d_segs,
                    const int4* d_tiles, int64_t ntiles, int n64, bool split, int* d_err,
                    cudaStream_t s, int stall = 0);
int* tc_error_word();
void tc_check(cudaStream_t s);

// A batch of descriptors of one kind with its device copy.
template <class P>
struct Batch {
  std::vector<P> h;
  DevBuf<P> d;
  // optional prepared (problem, column) work list of the column-parallel kernels
  DevBuf<int2> work;
  int64_t nwork = -1;
  const char* tag = nullptr;   // profiler label of the call site
  int variant = 0;        // kernel variant chosen when the work list was prepared
  size_t smem = 0;        // dynamic shared memory of that variant
  int64_t nfirst = 0;     // work items [0, nfirst) go to the first of two kernels
  void upload(cudaStream_t s) { d.upload(h, s); }
  size_t size() const { return h.size(); }
  bool empty() const { return h.empty(); }
  void push(const P& p) { h.push_back(p); }
};

// ---- batched Cholesky, in place (lower), upper triangle zeroed --------------------------
struct PotrfProb {
  double* A;
  int64_t lda;
  int n;
  int tag;   // reported in the failure record
  int* info = nullptr;   // failure record of this matrix (null: the launch's d_info)
  int col0 = 0;          // added to the failing column in the record (a diagonal block)
};
// info[0] receives tag+1 of a failing matrix (0 if all succeed); info[1] the failing column.
void potrf_launch(const Batch<PotrfProb>& b, int* d_info, cudaStream_t s);

// ---- batched triangular solves, in place on B (n x ncol): op(T) X = B -------------------
// lower=1: T lower triangular; trans=1: solve with T^T.
struct TrsmProb {
  const double* T;
  int64_t ldt;
  double* B;
  int64_t ldb;
  int n, ncol;
  int lower, trans;
};
void trsm_launch(const Batch<TrsmProb>& b, cudaStream_t s);
// builds the (problem, column) work list once so that later launches need no allocation
void trsm_prepare(Batch<TrsmProb>& b, cudaStream_t s);

// ---- batched Householder QR with optional column pivoting -----------------------------
// On exit A holds R in its upper triangle (first `rank` rows, all columns in pivot order)
// and the reflectors v (v_0 = 1 implicit) below the diagonal of its first `rank` columns.
// piv[0..n) receives the column order (indices of the input columns).  The factorization
// stops after kmax steps, or before step j when the largest remaining column norm is
// <= rtol * (first pivot norm).  pivot=0 disables pivoting (plain QR of kmax columns).
struct QrProb {
  double* A;
  int64_t lda;
  int m, n, kmax;
  double rtol;
  int* piv;       // n entries (may be null when pivot == 0)
  double* tau;    // kmax entries
  int* rank;      // 1 entry
  double* norms;  // 2n entries of scratch (downdated norms, norms at the last recompute)
  int downdate = 1;   // 0: recompute every remaining norm at every step (nearly full-rank
                      //    matrices, where downdates would be recomputed anyway)
};
// returns the profiler record of the launch (-1 when profiling is off); the caller adds
// the flops with prof_add_flops once the ranks are known
int geqp3_launch(const Batch<QrProb>& b, int pivot, int cluster, int max_m, cudaStream_t s);

// Apply the k reflectors stored in (V, ldv, tau) to B (m x ncol) in place:
// trans=1: B <- Q^T B;  trans=0: B <- Q B.   Q = H_0 H_1 ... H_{k-1}.
// ---- shared-memory factorizations with one lane group per column ----------------------
// A CTA of 256 threads gives each of the m columns of a matrix a group of `lanes` lanes
// (a power of two <= 32, all threads busy when m <= 256); the lanes of a group take the
// rows of their column round robin and add their partial sums by shuffles.  The column
// stride ld of the shared-memory copy is padded to ld = lanes (mod 16) (any value for
// lanes >= 16), so that the groups of a warp read disjoint banks.
__host__ __device__ inline int col_group_lanes(int m) {
  return m <= 8 ? 32 : (m <= 16 ? 16 : (m <= 32 ? 8 : (m <= 64 ? 4 : (m <= 128 ? 2 : 1))));
}
__host__ __device__ inline int col_group_ld(int rows, int lanes) {
  if (lanes >= 16) return rows;
  return rows + (((lanes - rows) % 16) + 16) % 16;
}
#ifdef __CUDACC__
// sum over the `lanes` lanes of a group (every lane of the warp must call it)
__device__ __forceinline__ double group_sum_n(double x, int lanes) {
  for (int o = lanes >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// Householder scalars of x (x_0 = *x0, |x|^2 = n2), the reflector left unnormalized:
// u = x - beta e_1, H = I - c u u^T.  Writes u_0 over x_0, stores beta, returns c
// (c = 0 for x = 0: the identity).
// A column whose norm is at most 2^-480 is left alone (no reflector, beta = alpha): below
// that, beta * u0 can leave the normal range and c = -1 / (beta u0) overflow, and the sum
// of squares it came from has already lost its precision to underflow.
constexpr double kHhMinNorm = 0x1p-480;
__device__ __forceinline__ double hh_scalars(double* x0, double n2, double* beta_out) {
  const double alpha = *x0;
  const double normx = sqrt(n2);
  double beta = alpha, c = 0.0;
  if (normx > kHhMinNorm) {
    beta = alpha >= 0.0 ? -normx : normx;
    const double u0 = alpha - beta;
    *x0 = u0;
    c = -1.0 / (beta * u0);
  }
  *beta_out = beta;
  return c;
}
#endif

// Column-pivoted QR of small square (or short) matrices, one CTA each (H^2 ID on the
// TSQR triangle): the pivot is the column of largest downdated norm (LAPACK's downdate
// with its recomputation safeguard, qr_downdate), ties to the lowest position; the
// factorization stops before step k when the exact norm |R_kk| of the pivot column is
// <= rtol |R_00| (or 0).  On return A holds the columns in pivot order with R in their
// upper k rows (below the diagonal: unspecified), piv[p] = original column at position
// p, *rank = k.  m <= 160 (rows and columns).  Uses A, lda, m, n, rtol, piv, rank.
int geqp3_small_launch(const Batch<QrProb>& b, const char* tag, cudaStream_t s);

// ---- R factor of two stacked upper triangles: R1 <- R of QR([R1; R2]) ----------------
// R1, R2: m x m upper triangular, column-major, leading dimension m (entries below the
// diagonal are ignored on input; R1's are written as zeros).  The reduction step of a
// blocked (TSQR) QR: merging the R factors of two row blocks gives the R factor of both.
struct TriMergeProb {
  double* R1;
  const double* R2;
  int m;
};
void tri_merge_launch(const Batch<TriMergeProb>& b, const char* tag, cudaStream_t s);

struct HhApplyProb {
  const double* V;
  int64_t ldv;
  const double* tau;
  const int* k;     // device pointer to the reflector count (rank of the QR)
  double* B;
  int64_t ldb;
  int m, ncol;
};
void householder_launch(const Batch<HhApplyProb>& b, int trans, cudaStream_t s);
void householder_prepare(Batch<HhApplyProb>& b, cudaStream_t s);

// Q(:, 0:k) explicitly into Q (m x kcols, only columns < *k written; others zeroed).
struct FormQProb {
  const double* V;
  int64_t ldv;
  const double* tau;
  const int* k;
  double* Q;
  int64_t ldq;
  int m, kcols;
};
void form_q_launch(const Batch<FormQProb>& b, cudaStream_t s);

// ---- batched strided 2-D copies: dst(i,j) = alpha*src(i,j) (+ dst if accumulate) --------
struct CopyProb {
  const double* src;
  int64_t lds;
  double* dst;
  int64_t ldd;
  int m, n;
  int trans;        // 1: dst(i,j) = src(j,i)   (src null: zeros)
  int accumulate;   // 1: dst += ...
  double alpha;
};
void copy_launch(const Batch<CopyProb>& b, cudaStream_t s);
// dst(0:m, 0:m) = I for every entry (src unused)
void identity_launch(const Batch<CopyProb>& b, cudaStream_t s);
// dst[0:count) = src[0:count) (src null: zeros), device vectors; merged like the batched
// copies when the calling thread runs an instance of a batched sweep
void copy_vec(double* dst, const double* src, int64_t count, cudaStream_t s);

// one-shot helpers: upload and launch (descriptors freed when the call returns)
template <class P, class F>
void run_once(std::vector<P> h, cudaStream_t s, F launch) {
  if (h.empty()) return;
  Batch<P> b;
  b.h = std::move(h);
  b.upload(s);
  launch(b);
}

}  // namespace spd

namespace spd {
// Launchers over descriptor arrays that already sit in device memory: they neither
// allocate nor upload anything.
std::vector<int4> gemm_tiles(const std::vector<GemmProb>& probs, int* nb_out);
void gemm_launch_raw(const GemmProb* d_probs, const GemmSeg* d_segs, const int4* d_tiles,
                     int64_t ntiles, int nb, cudaStream_t s);
void trsm_launch_raw(const TrsmProb* d_probs, const int2* d_work, int64_t nwork, cudaStream_t s);
void householder_launch_raw(const HhApplyProb* d_probs, const int2* d_work, int64_t nwork,
                            int trans, cudaStream_t s);
void copy_launch_raw(const CopyProb* d_probs, int64_t nprob, int64_t max_elems, cudaStream_t s);
}  // namespace spd
