// Cluster tree and admissibility lists (Sec. 2, Sec. 5.1, Sec. 6), built on the device.
#pragma once

#include "common.cuh"

namespace spd {

// Host mirror of the tree (small: O(number of nodes + list entries)).
struct TreeHost {
  int64_t n = 0;                    // unknowns (points x dofs)
  int dim = 0;
  int dofs = 1;                     // unknowns per point (3 for a vector-valued kernel)
  int leaf_size = 0;
  int B = 0;                        // bits per dimension of the finest grid
  int D = 0;                        // depth of the leaf level
  double lo[3] = {0, 0, 0};         // lower corner of the enclosing cube
  double w = 0;                     // side of the enclosing cube
  std::vector<int64_t> depth_off;   // D + 2 entries
  std::vector<int64_t> begin, end, parent, child_begin, child_end;
  std::vector<int64_t> cell_lo;     // nn * dim
  std::vector<int64_t> width;       // nn
  std::vector<int64_t> near_off, near_idx, far_off, far_idx;
  int64_t nn() const { return (int64_t)begin.size(); }
  int depth_of(int64_t i) const {
    int t = 0;
    while (depth_off[t + 1] <= i) ++t;
    return t;
  }
  int level_of_depth(int t) const { return D + 1 - t; }
  int64_t size(int64_t i) const { return end[i] - begin[i]; }
};

// Device-resident tree data used by kernels.
struct TreeDev {
  DevBuf<double> xs;          // sorted coordinates, structure of arrays: xs[a * n + p]
  DevBuf<int64_t> perm;       // sorted position -> original index
  DevBuf<int64_t> begin, end; // per node
  DevBuf<int64_t> near_off, near_idx, far_off, far_idx;
};

// Builds the tree from device points (row-major n x dim).
void build_tree(const double* d_points, int64_t n, int dim, int leaf_size, cudaStream_t s,
                TreeHost& th, TreeDev& td);

// Turns a point tree into a tree of k unknowns per point (k > 1): n, the permutation and
// every index range count unknowns, unknown k*p + c being component c of point p; the
// sorted coordinates gain a row (index dim) holding c.  No-op for k = 1.
void expand_dofs(int k, cudaStream_t s, TreeHost& th, TreeDev& td);

// Device exclusive scan of int64 values (in place); returns the total.
int64_t exclusive_scan_i64(int64_t* d, int64_t n, cudaStream_t s);

}  // namespace spd
