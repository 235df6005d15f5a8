// Kernel-matrix evaluation on the device: dense tiles K(X_r, X_c) (+ shift on the
// diagonal), proxy-point matrices K(P_i, X_cand) of the H^2 construction, and the
// near-field product Y_i += sum_j K(X_i, X_j) X_j with tiles evaluated on the fly.
#pragma once

#include <algorithm>

#include "dense.cuh"
#include "merge.cuh"

namespace spd {

// Points are structure-of-arrays: coordinate a of point p at x[a * ldx + p].
struct TileProb {
  const double* xr;
  int64_t ldxr, r0;
  int rows;
  const double* xc;
  int64_t ldxc, c0;
  int cols;
  double* out;
  int64_t ldo;
  double diag_add;   // added where r0 + i == c0 + j and xr == xc (self block)
  KernelFn kf{};     // kernel and dimension of this problem (dim 0: the launch's)
  int dim = 0;
};
void tile_launch(const Batch<TileProb>& b, const KernelFn& k, int dim, cudaStream_t s);
// out[i] = K(r) for r2[i] = r^2, the scalar kernel function exactly as the tiles evaluate
// it (no shift); device arrays of n entries
void kernel_eval_launch(const KernelFn& k, const double* r2, double* out, int64_t n,
                        cudaStream_t s);

// Proxy points of one node (reading of the proxy point method): 6 cube surfaces of
// half-width h_t = 3h + (H - 3h) (t/5)^2 around the cell centre c, each face carrying a
// q x q cell-centred grid (q = 8 in 3D, 32 points per edge in 2D).
constexpr int PROXY_SHELLS = 6;
__host__ __device__ inline int proxy_grid(int dim) { return dim == 3 ? 8 : 32; }
__host__ __device__ inline int proxy_count(int dim) {
  const int q = proxy_grid(dim);
  return PROXY_SHELLS * 2 * dim * (dim == 3 ? q * q : q);
}
struct ProxyProb {
  double c[3];
  double h, H;
  const double* xc;
  int64_t ldxc, c0;
  int cols;
  double* out;     // proxy_count(dim) * kernel_dofs(kind) x cols, column-major (row i:
                   // component i % kernel_dofs of proxy point i / kernel_dofs)
  int64_t ldo;
  KernelFn kf{};   // kernel and dimension of this problem (dim 0: the launch's)
  int dim = 0;
  double scale = 1.0;   // power of two multiplying every entry (proxy_scale)
};
void proxy_launch(const Batch<ProxyProb>& b, const KernelFn& k, int dim, cudaStream_t s);
// The power of two that brings the entries of a node's proxy matrix near 1 when they are
// tiny, so that the sums of squares of the ID's Householder steps stay clear of underflow:
// every entry is K(r) at a distance r >= 2h (the inner proxy surface lies 3h from the
// centre of the cell of half-width h that holds the candidates) and the scalar kernels
// decrease in r, so K(2h) bounds them.  Multiplying by 2^s is exact, and the ID (pivot
// order, the relative rank test, R11^-1 R12) does not change under it.  1 unless
// 0 < K(2h) < 2^-200 (and for the RPY tensor).
double proxy_scale(const KernelFn& k, double h);

// One row block of a proxy matrix, evaluated and factored in shared memory: rows
// [r0, r0 + rows) of K(P_i, X_cand) (p.cols = m candidate columns) are reduced by an
// unpivoted Householder QR to their upper-triangular factor R_b, written as a dense
// m x m matrix (zeros below the diagonal) at p.out, leading dimension p.ldo (= m).
struct ProxyQrProb {
  ProxyProb p;
  int r0, rows;
};
// Largest candidate count of the blocked ID and the shared-memory budget of one block:
// a node with m <= kIdTsqrMaxM candidates is factored in row blocks of
// id_tsqr_rows(m, np) rows (at least m, about kIdTsqrBlockEntries / m).
constexpr int kIdTsqrMaxM = 160;
constexpr int kIdTsqrBlockEntries = 12800;
inline int id_tsqr_rows(int m, int np) {
  return std::min(np, std::max(m, kIdTsqrBlockEntries / std::max(m, 1)));
}
void proxy_qr_launch(const Batch<ProxyQrProb>& b, const KernelFn& k, int dim, const char* tag,
                     cudaStream_t s);

// Near-field product.  Problem: rows [row0, row0 + rows) of the sorted points; output
// out (rows x ncol, ld ldo), accumulated (beta = 1) or overwritten (beta = 0).
// Segment: columns [col0, col0 + cols) of the sorted points with their input block x
// (cols x ncol, ld ldx); self = 1 adds shift * x on the diagonal.
// T = double, or float for the mixed-precision products (kernel entries evaluated and
// accumulated in FP32, few columns only).
template <class T>
struct NearProbT {
  int64_t row0;
  int rows;
  T* out;
  int64_t ldo;
  int ncol;
  int seg0, seg1;
  int beta;
  // points, dimension and kernel parameters of this problem (xs null: the launch's); set
  // when the problems of several instances share one launch
  const double* xs = nullptr;
  int64_t ldx = 0;
  int dim = 0;
  double inv_ell = 0.0, shift = 0.0;
  // launch choices made when the problem's own batch was first uploaded (0: not yet): the
  // column block cb and the segment parts, kept so that the problem is computed the same
  // way (same bits) when it is later launched together with other instances' problems
  int cb = 0, parts = 0;
};
template <class T>
struct NearSegT {
  int64_t col0;
  int cols;
  const T* x;
  int64_t ldx;
  int self;
};
using NearProb = NearProbT<double>;
using NearSeg = NearSegT<double>;

template <class T>
struct NearBatchT {
  std::vector<NearProbT<T>> probs;
  std::vector<NearSegT<T>> segs;
  std::vector<int2> work;   // (prob, first column) over the launched problems
  std::vector<NearProbT<T>> exec_probs;   // the problems as launched (d_probs)
  DevBuf<NearProbT<T>> d_probs;
  DevBuf<NearSegT<T>> d_segs;
  DevBuf<int2> d_work;
  int cb = 8;               // column block per CTA: 64 pair-tile kernel, -NC few-column kernel
  double flops = 0.0;       // 2 * (kernel entries) * columns: the block product
  double evals = 0.0;       // kernel entries of one launch
  const char* tag = "near";
  // few-column products over too few problems to fill the GPU: every problem's segments
  // are split into parts written as partial sums, then added in a fixed order
  int parts = 1;
  std::vector<NearProbT<T>> part_probs;   // one per (problem, part), output into the scratch
  std::vector<int4> red;                  // (problem, scratch offset, parts, 0)
  DevBuf<NearProbT<T>> d_part_probs;
  DevBuf<int4> d_red;
  DevBuf<T> scratch;
  void prob(int64_t row0, int rows, T* out, int64_t ldo, int ncol, int beta) {
    NearProbT<T> p;
    p.row0 = row0; p.rows = rows; p.out = out; p.ldo = ldo; p.ncol = ncol; p.beta = beta;
    p.seg0 = p.seg1 = (int)segs.size();
    probs.push_back(p);
  }
  void seg(int64_t col0, int cols, const T* x, int64_t ldx, int self) {
    NearSegT<T> g;
    g.col0 = col0; g.cols = cols; g.x = x; g.ldx = ldx; g.self = self;
    segs.push_back(g);
    probs.back().seg1 = (int)segs.size();
  }
  bool empty() const { return probs.empty(); }
  void upload(cudaStream_t s);
  void launch(const KernelFn& k, const double* xs, int64_t ldx, int dim, cudaStream_t s) const;
  void run(const KernelFn& k, const double* xs, int64_t ldx, int dim, cudaStream_t s) {
    upload(s);
    launch(k, xs, ldx, dim, s);
  }
};
using NearBatch = NearBatchT<double>;
using NearBatchF = NearBatchT<float>;

}  // namespace spd
