// H^2 representation (Sec. 5.1) built by the proxy point method (Sec. 6), and its
// products.  Node numbering, lists and the permutation come from the cluster tree.
#pragma once

#include <map>
#include <memory>

#include "keval.cuh"
#include "tree.cuh"

namespace spd {

// Couplings in destination-major form (FP32 copies for the mixed-precision products, FP64
// copies for products with at most 4 columns): node i owns one column-major
// k_i x (sum of its far partners' ranks) matrix [B_ij1 B_ij2 ...], so the coupling step
// streams every entry exactly once and coalesced.  The columns are cut into chunks of at
// most 64 that stay within one partner; the CTA of a node stages the x^_j pieces of a few
// chunks in shared memory and each thread accumulates one row over its chunks.
constexpr int kRowChunk = 64;   // columns per chunk

template <class T>
struct RowCoupProbT {
  T* C;              // y^_i (k_i x ncol, ld ldc)
  int64_t ldc;
  int M;             // k_i
  int ncol;
  const T* A;        // k_i x (sum k_j), ld k_i
  int ch0, ch1;      // chunk range
  int beta = 0;      // 1: add to C instead of overwriting it
  // coupling entries per CTA chosen when the problem's own batch was first uploaded (0:
  // not yet); kept so that the problem is summed the same way in merged launches
  int64_t item = 0;
};
template <class T>
struct RowCoupChunkT {
  const T* x;        // x^_j rows [kk0, kk0 + K) (ld ldx)
  int64_t ldx;
  int64_t col;       // first column of the chunk in A
  int K;             // <= 64
};
// one CTA: rows [r0, r0 + 256) of problem p over chunks [ch0, ch1); part >= 0 writes a
// partial tile (summed later in part order) instead of the output
struct RowCoupWork {
  int p, r0, ch0, ch1;
  int64_t part;
};
struct RowCoupRed {
  int p, r0;
  int64_t part0;
  int nparts;
};
template <class T>
struct RowCoupBatchT {
  std::vector<RowCoupProbT<T>> probs;
  std::vector<RowCoupChunkT<T>> chunks;
  std::vector<RowCoupWork> work;
  std::vector<RowCoupRed> red;
  DevBuf<RowCoupProbT<T>> d_probs;
  DevBuf<RowCoupChunkT<T>> d_chunks;
  DevBuf<RowCoupWork> d_work;
  DevBuf<RowCoupRed> d_red;
  DevBuf<T> partial;          // nparts x NC x 256
  int ncol = 1;
  const char* tag = "h2_coupling";
  double flops = 0.0, bytes = 0.0;
  void upload(cudaStream_t s);
  void launch(cudaStream_t s) const;
};

// The FP32 product that reads every stored generator once (couplings once per unordered
// pair, both directions from the same tile).  Skeleton-space vectors (x^, y^, per-pair
// pieces, partial tiles) are row-interleaved: entry (row r, right-hand side c) at
// [r * nc + c], nc = the launch width (1, 2, 4, 8 or 16), right-hand sides >= ncol zero.
// A job is rows [r0, r0 + R) (R <= 512, r0 % 4 == 0) and columns [c0, c1) of an FP32
// column-major matrix A whose leading dimension is a multiple of 4 (zero rows below the
// matrix) on a 16-byte boundary:
//   direction 1 (y1 != null): y1[r * y1rs + c * y1cs] (mode1: += / =)
//                             sum_col A[r0 + r, col] x1[idx(col) * nc + c],
//                             idx(col) = cmap ? cmap[col] : col  (x1 row-interleaved);
//   direction 2 (z != null):  z[(col - c0) * zcs + c * zrs] (mode2)
//                             sum_r A[r0 + r, col] x2[r * x2rs + c * x2cs].
struct SymJob {
  const float* A;
  int64_t lda;
  int r0, R, c0, c1;
  int S;                       // columns per pipeline stage (chosen from R and the width)
  int ncol;                    // right-hand sides (<= the launch width)
  float* y1;
  int64_t y1rs, y1cs;
  int mode1;
  const float* x1;
  const int* cmap;
  float* z;
  int64_t zcs, zrs;
  int mode2;
  const float* x2;
  int64_t x2rs, x2cs;
};
// y (rows x ncol, row-interleaved with stride nc) (mode: += / =) the sum of the
// row-interleaved sources [s0, s1) (same stride) in that order
struct SymSrc {
  const float* p;
};
struct SymSum {
  float* y;
  int rows, ncol, nc, mode, s0, s1;
};
struct SymBatch {
  std::vector<SymJob> jobs;
  DevBuf<SymJob> d_jobs;
  int nc = 8, ncol = 1;
  const char* tag = "h2_coupling_f32";
  double flops = 0.0, bytes = 0.0;
  void upload(cudaStream_t s);
  void launch(cudaStream_t s) const;
};
struct SymSumBatch {
  std::vector<SymSum> jobs;
  std::vector<SymSrc> srcs;
  DevBuf<SymSum> d_jobs;
  DevBuf<SymSrc> d_srcs;
  int ncol = 1;
  const char* tag = "h2_coupling_f32";
  double bytes = 0.0;
  void upload(cudaStream_t s);
  void launch(cudaStream_t s) const;
};
struct PlanStep {
  std::unique_ptr<SymBatch> sym;
  std::unique_ptr<SymSumBatch> sum;
};
// upward levels (each with its partial sums), couplings, their sums, downward levels
struct SymPlan {
  int nc = 0;
  std::vector<PlanStep> steps;
  DevBuf<float> xh, yh;  // x^ and y^ (K x nc, row-interleaved)
  DevBuf<float> part;    // partial tiles and the per-pair pieces of the couplings
};

// One H^2 product plan for a fixed number of columns: upward pass, Type-3 couplings,
// downward pass, leaf bases and near field.  With nslot > 1 the product is split by the
// HSS level of the lowest common ancestor of every block (slot l - 2 for level l), which
// the SPD-HSS sampling uses to form all Y^(k) of Eq. Yk in one pass.
// T = double, or float for the mixed-precision product (FP32 copies of the generators,
// FP32 kernel entries, FP32 accumulation).
template <class T>
struct H2PlanT {
  RowCoupBatchT<T> rowcoup;   // destination-major coupling step (replaces `coupling`)
  bool use_rowcoup = false;
  int ncol = 0;      // columns per slot
  int nslot = 1;
  DevBuf<T> xs, ys, xhat, yhat;   // sorted-order input/output, skeleton-space vectors
  GemmBatchT<T> up_leaf;
  std::vector<GemmBatchT<T>> up;       // per depth D-1 .. 1
  GemmBatchT<T> coupling;
  std::vector<GemmBatchT<T>> down;     // per depth 1 .. D-1
  GemmBatchT<T> leaf_out;
  NearBatchT<T> near;
  GemmBatchT<T> near_g;     // the near field from the stored blocks (replaces `near`)
  RowCoupBatchT<T> near_r;  // ... streamed row by row for at most 4 columns
  bool near_stored = false, near_rows = false;
  DevBuf<T> coup_src;       // couplings in this plan's type when it owns a copy of them
  std::shared_ptr<SymPlan> sym;   // FP32: the once-read product (replaces the GEMM steps)
};
using H2Plan = H2PlanT<double>;
using H2PlanF = H2PlanT<float>;

}  // namespace spd

struct spdhss_h2_s {
  spd::KernelFn kfn{};
  double tol = 0;
  spd::TreeHost th;
  spd::TreeDev td;
  // skeletons (sorted-order unknown indices, pivot order), node-major
  std::vector<int64_t> skel_off, skel_idx;
  int64_t Ktot = 0;
  spd::DevBuf<double> skel_x;        // (dim + component row if vector-valued) x Ktot, SoA
  // bases: leaf U_i (|I_i| x k_i) or transfer R_i (sum k_c x k_i), column-major
  std::vector<int64_t> U_off;
  std::vector<int> U_rows;
  spd::DevBuf<double> basis;
  // couplings B_ij = K(skel_i, skel_j) for far pairs, stored once per unordered pair
  std::vector<int64_t> far_boff;     // per far-list entry: offset into coup
  std::vector<int> far_trans;        // 1: the entry uses the stored transpose
  spd::DevBuf<double> coup;
  int max_rank = 0;
  std::map<int, std::unique_ptr<spd::H2Plan>> plans;   // by nrhs
  // near-field blocks K(X_i, X_j) (+ shift on the diagonal) of every leaf near pair, stored
  // on the first FP64 product when they fit kNearStoreBytes: per near-list entry the
  // offset of its |I_i| x |I_j| block; the blocks of leaf i are consecutive (one
  // |I_i| x sum |I_j| column-major row block)
  std::vector<int64_t> near_boff;
  spd::DevBuf<double> near_blk;
  int near_state = 0;   // 0: not decided, 1: stored, 2: evaluated on the fly
  // FP32 copies of the generators for the mixed-precision products (made on first use)
  spd::DevBuf<float> basis_f;
  // destination-major FP64 couplings (made on first use for products of at most 4
  // columns), and per node the offset of its coupling matrix in them
  spd::DevBuf<double> coup_dd;
  std::vector<int64_t> coup_dm_off;
  std::map<int, std::unique_ptr<spd::H2PlanF>> plans_f;
  // the FP32 once-read layout (made on first FP32 product): padded copies of the bases
  // (offset per node) and of every owner's coupling region M_i = [B_ij ...] over its
  // partners j > i (offset and columns per node), the x^ row of every region column, and
  // per far-list entry the first column of its pair's block in the owner's region
  spd::DevBuf<float> sym_f;
  std::vector<int64_t> sym_U_off, sym_M_off, sym_Kc, sym_cmap_off, sym_colstart;
  spd::DevBuf<int> sym_cmap;

  int rank(int64_t i) const { return (int)(skel_off[i + 1] - skel_off[i]); }
};

namespace spd {
void h2_build_impl(spdhss_h2_s* h, const double* d_points, int64_t n, int dim, int leaf_size,
                   cudaStream_t s);
// Y = A X on sorted-order data owned by the plan (plan.xs -> plan.ys)
void h2_plan_build(const spdhss_h2_s* h, H2Plan& p, int ncol, int nslot, cudaStream_t s);
void h2_plan_run(const spdhss_h2_s* h, const H2Plan& p, cudaStream_t s);
// the FP32 plan for ncol columns (generators converted on first use), cached in the handle
H2PlanF& h2_plan_f(spdhss_h2_s* h, int ncol, cudaStream_t s);
// the precision mode's sampling plan: FP32, LCA slots, GEMMs on the tensor cores
// (tc = 1 TF32, 2 3xTF32), near field in FP32 on the fly
void h2_plan_sample_f(spdhss_h2_s* h, H2PlanF& p, int ncol, int nslot, int tc, cudaStream_t s);
void h2_plan_run(const spdhss_h2_s* h, const H2PlanF& p, cudaStream_t s);
// the once-read FP32 layout of the handle: whether it fits, building it, a plan's steps
bool sym_layout_fits(const spdhss_h2_s* h, cudaStream_t s);
void sym_layout(spdhss_h2_s* h, cudaStream_t s);
void sym_plan_build(const spdhss_h2_s* h, H2PlanF& p, int ncol, cudaStream_t s);
void sym_plan_run(const SymPlan& P, cudaStream_t s);
// element-wise conversions of n x ncol column-major blocks between FP64 and FP32
void convert_d2f(const double* x, float* y, int64_t count, cudaStream_t s);
void convert_f2d(const float* x, double* y, int64_t count, cudaStream_t s);
// permutations between original and sorted order (ld of the original-order data given)
void permute_to_sorted(const double* X, int64_t ldx, double* Xs, int64_t n, int ncol,
                       const int64_t* perm, cudaStream_t s);
void permute_from_sorted(const double* Xs, double* Y, int64_t ldy, int64_t n, int ncol,
                         const int64_t* perm, cudaStream_t s);
}  // namespace spd
