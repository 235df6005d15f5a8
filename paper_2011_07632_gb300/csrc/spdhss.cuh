// SPD HSS construction from an H^2 matrix (Alg. 5.3) and the HSS product.
#pragma once

#include "h2.cuh"

struct spdhss_hss_s {
  const spdhss_h2_s* h2 = nullptr;
  int r = 0, p = 0, s = 0;
  int L = 1;                              // HSS levels (root = level L)
  std::vector<int> rk;                    // r_i per node (0 at the root)
  std::vector<int> mrow;                  // leaf: |I_i|; above: M_i = sum of children's r
  std::vector<int64_t> hoff;              // node-major offsets of r_i (skeleton space)
  int64_t Rtot = 0;
  // generators: leaf U_i (|I_i| x r_i), nonleaf R_i (M_i x r_i)
  std::vector<int64_t> gen_off;
  spd::DevBuf<double> gen;
  // sibling couplings B_ab for every ordered sibling pair (a != b), r_a x r_b, ld r_a
  std::vector<int64_t> sib_off;           // per node a: first entry in sib_list
  std::vector<int64_t> sib_node;          // partner b of each entry
  std::vector<int64_t> sib_boff;          // offset of B_ab in sib
  spd::DevBuf<double> sib;
  std::map<int, std::unique_ptr<spd::GemmBatch>> dummy;
  struct Plan;
  std::map<int, std::shared_ptr<void>> plans;   // hss_matmul plans by nrhs
  size_t stored_bytes() const { return gen.bytes() + sib.bytes(); }
};

namespace spd {
// precision: 0 FP64 throughout; 1 the sampling product in FP32 with its GEMMs on the
// tensor cores in 3xTF32; 2 the same in plain TF32.  Everything after the sampling is FP64.
void spdhss_build_impl(spdhss_hss_s* hs, const spdhss_h2_s* h2, int r, int p,
                       const double* omega, uint64_t seed, cudaStream_t s, double rtol = 0.0,
                       int precision = 0);
void hss_matmul_impl(spdhss_hss_s* hs, const double* X, double* Y, int nrhs, int64_t ld,
                     cudaStream_t s);
// Philox4x32-10 standard normals: out[i + j*ld] for i < n, j < ncol, counter (i, j)
void philox_normal(double* out, int64_t n, int ncol, int64_t ld, uint64_t seed, cudaStream_t s);
}  // namespace spd
