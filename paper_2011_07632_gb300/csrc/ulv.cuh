// Symmetric ULV factorization of an SPD HSS matrix and its solve.
#pragma once

#include "spdhss.cuh"

namespace spd {

// Solve plan for a fixed number of right-hand sides; works in place on bw[0] (the leaf
// level buffer, sorted order, ld n).
struct UlvPlan {
  int ncol = 0;
  std::vector<DevBuf<double>> bw;            // per level 1..L-1 (index k-1), plus the root
  std::vector<int64_t> ldk;                  // leading dimension per level buffer
  std::vector<Batch<HhApplyProb>> qt, q;     // per level: Q^T / Q on every node block
  std::vector<Batch<TrsmProb>> fw, bk;       // per level: L_q^{-1}, L_q^{-T}
  std::vector<GemmBatch> upd_f, upd_b;       // per level: b_p -= X^T y_q ; y_q -= X x_p
  std::vector<Batch<CopyProb>> up, down;     // per level: reduced parts to / from the parent
  Batch<TrsmProb> root_f, root_b;
};

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
  std::map<int, std::unique_ptr<spd::UlvPlan>> plans;
  size_t stored_bytes() const { return Dbuf.bytes() + Wbuf.bytes() + taub.bytes() + Ubuf.bytes() + root.bytes(); }
};

namespace spd {
void ulv_factor_impl(spdhss_ulv_s* u, const spdhss_hss_s* hs, cudaStream_t s);
UlvPlan& ulv_plan(spdhss_ulv_s* u, int ncol, cudaStream_t s);
// in place on plan.bw[0] (sorted order, n x ncol, ld n)
void ulv_solve_sorted(const spdhss_ulv_s* u, const UlvPlan& p, cudaStream_t s);
}  // namespace spd
