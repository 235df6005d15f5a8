// H^2 representation (Sec. 5.1) built by the proxy point method (Sec. 6), and its
// products.  Node numbering, lists and the permutation come from the cluster tree.
#pragma once

#include <map>
#include <memory>

#include "keval.cuh"
#include "tree.cuh"

namespace spd {

// One H^2 product plan for a fixed number of columns: upward pass, Type-3 couplings,
// downward pass, leaf bases and near field.  With nslot > 1 the product is split by the
// HSS level of the lowest common ancestor of every block (slot l - 2 for level l), which
// the SPD-HSS sampling uses to form all Y^(k) of Eq. Yk in one pass.
struct H2Plan {
  int ncol = 0;      // columns per slot
  int nslot = 1;
  DevBuf<double> xs, ys, xhat, yhat;   // sorted-order input/output, skeleton-space vectors
  GemmBatch up_leaf;
  std::vector<GemmBatch> up;       // per depth D-1 .. 1
  GemmBatch coupling;
  std::vector<GemmBatch> down;     // per depth 1 .. D-1
  GemmBatch leaf_out;
  NearBatch near;
};

}  // namespace spd

struct spdhss_h2_s {
  spd::KernelFn kfn{};
  double tol = 0;
  spd::TreeHost th;
  spd::TreeDev td;
  // skeletons (sorted-order point indices, pivot order), node-major
  std::vector<int64_t> skel_off, skel_idx;
  int64_t Ktot = 0;
  spd::DevBuf<double> skel_x;        // dim x Ktot, structure of arrays
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

  int rank(int64_t i) const { return (int)(skel_off[i + 1] - skel_off[i]); }
};

namespace spd {
void h2_build_impl(spdhss_h2_s* h, const double* d_points, int64_t n, int dim, int leaf_size,
                   cudaStream_t s);
// Y = A X on sorted-order data owned by the plan (plan.xs -> plan.ys)
void h2_plan_build(const spdhss_h2_s* h, H2Plan& p, int ncol, int nslot, cudaStream_t s);
void h2_plan_run(const spdhss_h2_s* h, const H2Plan& p, cudaStream_t s);
// permutations between original and sorted order (ld of the original-order data given)
void permute_to_sorted(const double* X, int64_t ldx, double* Xs, int64_t n, int ncol,
                       const int64_t* perm, cudaStream_t s);
void permute_from_sorted(const double* Xs, double* Y, int64_t ldy, int64_t n, int ncol,
                         const int64_t* perm, cudaStream_t s);
}  // namespace spd
