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
  // destination-major couplings (made on first use): FP32 and FP64 copies, and per node the
  // offset of its coupling matrix in them
  spd::DevBuf<float> coup_fd;
  spd::DevBuf<double> coup_dd;
  std::vector<int64_t> coup_dm_off;
  std::map<int, std::unique_ptr<spd::H2PlanF>> plans_f;

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
// element-wise conversions of n x ncol column-major blocks between FP64 and FP32
void convert_d2f(const double* x, float* y, int64_t count, cudaStream_t s);
void convert_f2d(const float* x, double* y, int64_t count, cudaStream_t s);
// permutations between original and sorted order (ld of the original-order data given)
void permute_to_sorted(const double* X, int64_t ldx, double* Xs, int64_t n, int ncol,
                       const int64_t* perm, cudaStream_t s);
void permute_from_sorted(const double* Xs, double* Y, int64_t ldy, int64_t n, int ncol,
                         const int64_t* perm, cudaStream_t s);
}  // namespace spd
