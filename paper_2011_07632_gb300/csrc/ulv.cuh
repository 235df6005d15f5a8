// Symmetric ULV factorization of an SPD HSS matrix and its solve.
#pragma once

#include "spdhss.cuh"

namespace spd {

// Solve plan for a fixed number of right-hand sides; works in place on bw[0] (the leaf
// level buffer, sorted order, ld n).  Every node's forward step (Q_i^T, the complement
// solve, the update of the kept rows) is one explicit m_i x m_i matrix F_i, and its
// backward step (the update from the parent's solution, the transposed complement solve,
// Q_i) another, B_i (both made once per factorization by running those steps on the
// identity); the root's solves are the explicit inverses of its Cholesky factor and of
// its transpose.  A solve is then two grouped GEMMs and two copies per level, spread over
// the whole GPU, instead of dependent chains of reflectors and substitutions.
struct UlvPlan {
  int ncol = 0;
  std::vector<DevBuf<double>> bw, tw;        // per level 1..L-1 (index k-1), plus the root
  std::vector<int64_t> ldk;                  // leading dimension per level buffer
  std::vector<GemmBatch> fwd, bwd;           // per level: t = F_i b ; b = B_i t
  std::vector<Batch<CopyProb>> up, down;     // per level: kept rows to / from the parent
  GemmBatch root_f, root_b;                  // t = L^{-1} b ; b = L^{-T} t
};

// State of the allocation-free solve for one column count (ulv_noalloc.cu).
struct NoallocPlan;
// Looks up the allocation-free solve's device arrays on the current device (once per
// device); loading them is the one allocation they need, so ulv_factor makes it.
void ulv_noalloc_prepare_device();

}  // namespace spd

struct spdhss_ulv_s {
  const spdhss_hss_s* hs = nullptr;
  int L = 1, D = 0;
  std::vector<int> m, r;                     // per node: block size and reduced size
  std::vector<int64_t> Doff, Woff, toff, Uoff;
  spd::DevBuf<double> Dbuf, Wbuf, taub, Ubuf;
  spd::DevBuf<int> rdev;                     // per node reflector counts (device)
  int mroot = 0;
  spd::DevBuf<double> root;                  // Cholesky factor of the root block
  // explicit per-node solve matrices (see UlvPlan), made on the first solve plan
  std::vector<int64_t> Foff;
  spd::DevBuf<double> Fbuf, Bbuf, rootF, rootB;
  std::map<int, std::unique_ptr<spd::UlvPlan>> plans;
  std::map<int, std::shared_ptr<spd::NoallocPlan>> noalloc_plans;   // ulv_solve_noalloc
  size_t stored_bytes() const { return Dbuf.bytes() + Wbuf.bytes() + taub.bytes() + Ubuf.bytes() + root.bytes(); }
};

namespace spd {
void ulv_factor_impl(spdhss_ulv_s* u, const spdhss_hss_s* hs, cudaStream_t s);
UlvPlan& ulv_plan(spdhss_ulv_s* u, int ncol, cudaStream_t s);
// in place on plan.bw[0] (sorted order, n x ncol, ld n)
void ulv_solve_sorted(const spdhss_ulv_s* u, const UlvPlan& p, cudaStream_t s);
void ulv_solve_noalloc_impl(spdhss_ulv_s* u, const double* B, double* X, int ncol, int64_t ld,
                            cudaStream_t s);
}  // namespace spd
