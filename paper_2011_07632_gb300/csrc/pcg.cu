// Preconditioned conjugate gradients (Sec. 6.2) with the H^2 product and the ULV solve of
// the SPD HSS approximation.  Every right-hand side column runs its own recurrence; a
// column stops when its recursive relative residual and then its recomputed true residual
// b - A x are both <= tol (otherwise the true residual replaces the recursive one).  All
// vectors stay on the device in tree order; the host reads one residual norm per column
// per iteration to decide.
#include <algorithm>
#include <cmath>

#include "ulv.cuh"

namespace spd {

// per-column dot products, deterministic two-pass reduction
constexpr int DOT_BLOCKS = 64;

__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ a,
                                                     const double* __restrict__ b, int64_t n,
                                                     double* __restrict__ part) {
  const int c = blockIdx.y;
  const double* x = a + (int64_t)c * n;
  const double* y = b + (int64_t)c * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    part[c * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* __restrict__ part, int nb, double* __restrict__ out,
                            int ncol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[c * nb + b];
  out[c] = t;
}

static void dots(const double* a, const double* b, int64_t n, int ncol, double* part, double* out,
                 cudaStream_t s) {
  k_dot_partial<<<dim3(DOT_BLOCKS, ncol), 256, 0, s>>>(a, b, n, part);
  SPD_LAUNCHED();
  k_dot_final<<<ceil_div(ncol, 128), 128, 0, s>>>(part, DOT_BLOCKS, out, ncol);
  SPD_LAUNCHED();
}

// x += alpha p, r -= alpha q with alpha = rz / pq (active columns)
__global__ void k_axpy_xr(double* __restrict__ x, double* __restrict__ r,
                          const double* __restrict__ p, const double* __restrict__ q, int64_t n,
                          int ncol, const double* __restrict__ rz, const double* __restrict__ pq,
                          const int* __restrict__ done) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncol) return;
  const int c = (int)(e / n);
  if (done[c] == 1) return;
  const double alpha = pq[c] != 0.0 ? rz[c] / pq[c] : 0.0;
  x[e] += alpha * p[e];
  r[e] -= alpha * q[e];
}

// p = z + beta p with beta = rz_new / rz (active columns; beta = 0 right after a residual
// replacement, done[c] == 2); then rz = rz_new
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                           int ncol, const double* __restrict__ rzn, const double* __restrict__ rz,
                           const int* __restrict__ done) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncol) return;
  const int c = (int)(e / n);
  if (done[c] == 1) return;
  const double beta = (done[c] == 0 && rz[c] != 0.0) ? rzn[c] / rz[c] : 0.0;
  p[e] = z[e] + beta * p[e];
}

__global__ void k_sub(const double* __restrict__ b, const double* __restrict__ ax,
                      double* __restrict__ out, int64_t count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = b[e] - ax[e];
}

// precision = 0: FP64 throughout.  precision = 1: the product with A inside the iteration
// uses the FP32 copy of the H^2 matrix (FP32 kernel entries and accumulation); the ULV
// preconditioner, the recurrences and every residual check stay FP64, and every
// `refresh` iterations the recursive residual is replaced by the FP64 true residual.
void pcg_impl(const spdhss_h2_s* h2c, spdhss_ulv_s* u, const double* B, double* X, int nrhs,
              int64_t ld, double tol, int maxit, int* iters_out, double* relres_out,
              bool& converged, cudaStream_t s, int precision = 0, int refresh = 50) {
  spdhss_h2_s* h2 = const_cast<spdhss_h2_s*>(h2c);
  const int64_t n = h2->th.n;
  const int64_t nc = n * nrhs;
  const int64_t* perm = h2->td.perm.p;
  // plans: H^2 product for the search direction (p lives in its xs, q in its ys), a second
  // H^2 product for true residuals, and the ULV solve (z lives in its leaf buffer)
  auto get_plan = [&](int key) -> H2Plan& {
    auto it = h2->plans.find(key);
    if (it == h2->plans.end()) {
      std::unique_ptr<H2Plan> p(new H2Plan());
      h2_plan_build(h2, *p, nrhs, 1, s);
      it = h2->plans.emplace(key, std::move(p)).first;
    }
    return *it->second;
  };
  H2Plan& PA = get_plan(nrhs);
  H2Plan& PR = get_plan(-nrhs);   // second plan (negative key) for residual checks
  UlvPlan& PU = ulv_plan(u, nrhs, s);
  double* p = PA.xs.p;
  double* q = PA.ys.p;
  H2PlanF* PF = precision ? &h2_plan_f(h2, nrhs, s) : nullptr;
  double* z = PU.bw[0].p;
  DevBuf<double> bs(nc), x(nc), r(nc), part((size_t)DOT_BLOCKS * nrhs), sc((size_t)4 * nrhs);
  DevBuf<int> done(nrhs);
  double* rz = sc.p;
  double* pq = sc.p + nrhs;
  double* rzn = sc.p + 2 * nrhs;
  double* rr = sc.p + 3 * nrhs;
  const bool host_b = !is_device_pointer(B);
  const bool host_x = !is_device_pointer(X);
  if (host_b) {
    DevBuf<double> tmp((size_t)ld * nrhs);
    SPD_CUDA(cudaMemcpyAsync(tmp.p, B, (size_t)ld * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    permute_to_sorted(tmp.p, ld, bs.p, n, nrhs, perm, s);
    SPD_CUDA(cudaStreamSynchronize(s));
  } else {
    permute_to_sorted(B, ld, bs.p, n, nrhs, perm, s);
  }
  const unsigned gb = (unsigned)ceil_div(nc, 256);
  x.zero(s);
  done.zero(s);
  SPD_CUDA(cudaMemcpyAsync(r.p, bs.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<double> bn(nrhs);
  dots(bs.p, bs.p, n, nrhs, part.p, rr, s);
  {
    std::vector<double> h(nrhs);
    SPD_CUDA(cudaMemcpyAsync(h.data(), rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < nrhs; ++c) bn[c] = h[c] > 0.0 ? std::sqrt(h[c]) : 1.0;
  }
  std::vector<int> hdone(nrhs, 0), hit(nrhs, 0);
  for (int c = 0; c < nrhs; ++c) hdone[c] = 0;
  // z = M^{-1} r, p = z, rz = r.z
  SPD_CUDA(cudaMemcpyAsync(z, r.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ulv_solve_sorted(u, PU, s);
  SPD_CUDA(cudaMemcpyAsync(p, z, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  dots(r.p, z, n, nrhs, part.p, rz, s);
  std::vector<double> hrr(nrhs);
  auto true_residual = [&](std::vector<double>& rel, bool replace_active) {
    SPD_CUDA(cudaMemcpyAsync(PR.xs.p, x.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    h2_plan_run(h2, PR, s);
    k_sub<<<gb, 256, 0, s>>>(bs.p, PR.ys.p, PR.ys.p, nc);
    SPD_LAUNCHED();
    dots(PR.ys.p, PR.ys.p, n, nrhs, part.p, rr, s);
    std::vector<double> h(nrhs);
    SPD_CUDA(cudaMemcpyAsync(h.data(), rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    rel.resize(nrhs);
    for (int c = 0; c < nrhs; ++c) rel[c] = std::sqrt(std::max(h[c], 0.0)) / bn[c];
    (void)replace_active;
  };
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    if (PF) {                                     // q = A p in FP32
      convert_d2f(p, PF->xs.p, nc, s);
      h2_plan_run(h2, *PF, s);
      convert_f2d(PF->ys.p, q, nc, s);
    } else {
      h2_plan_run(h2, PA, s);                     // q = A p
    }
    dots(p, q, n, nrhs, part.p, pq, s);
    k_axpy_xr<<<gb, 256, 0, s>>>(x.p, r.p, p, q, n, nrhs, rz, pq, done.p);
    SPD_LAUNCHED();
    dots(r.p, r.p, n, nrhs, part.p, rr, s);
    SPD_CUDA(cudaMemcpyAsync(hrr.data(), rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    bool any_pass = false;
    for (int c = 0; c < nrhs; ++c) {
      if (hdone[c] == 1) continue;
      hit[c] = it;
      if (!std::isfinite(hrr[c])) throw Error(SPDHSS_NUMERIC, "pcg_solve: residual is not finite");
      if (std::sqrt(std::max(hrr[c], 0.0)) / bn[c] <= tol) any_pass = true;
    }
    if (any_pass) {
      std::vector<double> trel;
      true_residual(trel, true);
      bool changed = false;
      for (int c = 0; c < nrhs; ++c) {
        if (hdone[c] == 1) continue;
        if (std::sqrt(std::max(hrr[c], 0.0)) / bn[c] > tol) continue;
        if (trel[c] <= tol) { hdone[c] = 1; changed = true; }
        else {
          // residual replacement: r = b - A x, and the next direction restarts (beta = 0)
          SPD_CUDA(cudaMemcpyAsync(r.p + (int64_t)c * n, PR.ys.p + (int64_t)c * n, n * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
          hdone[c] = 2;
          changed = true;
        }
      }
      if (changed)
        SPD_CUDA(cudaMemcpyAsync(done.p, hdone.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    bool all = true;
    for (int c = 0; c < nrhs; ++c) all = all && hdone[c] == 1;
    if (all) break;
    if (PF && refresh > 0 && it % refresh == 0) {
      // refine: the recursive residual of the FP32 product drifts; replace it by b - A x
      std::vector<double> trel;
      true_residual(trel, false);
      SPD_CUDA(cudaMemcpyAsync(r.p, PR.ys.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    SPD_CUDA(cudaMemcpyAsync(z, r.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ulv_solve_sorted(u, PU, s);                   // z = M^{-1} r
    dots(r.p, z, n, nrhs, part.p, rzn, s);
    k_update_p<<<gb, 256, 0, s>>>(p, z, n, nrhs, rzn, rz, done.p);
    SPD_LAUNCHED();
    SPD_CUDA(cudaMemcpyAsync(rz, rzn, nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    bool restarted = false;
    for (int c = 0; c < nrhs; ++c)
      if (hdone[c] == 2) { hdone[c] = 0; restarted = true; }
    if (restarted)
      SPD_CUDA(cudaMemcpyAsync(done.p, hdone.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  std::vector<double> trel;
  true_residual(trel, false);
  converged = true;
  for (int c = 0; c < nrhs; ++c) {
    if (iters_out) iters_out[c] = hit[c];
    if (relres_out) relres_out[c] = trel[c];
    converged = converged && trel[c] <= tol;
  }
  if (host_x) {
    DevBuf<double> tmp((size_t)ld * nrhs);
    if (ld > n) SPD_CUDA(cudaMemcpyAsync(tmp.p, X, (size_t)ld * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    permute_from_sorted(x.p, tmp.p, ld, n, nrhs, perm, s);
    SPD_CUDA(cudaMemcpyAsync(X, tmp.p, (size_t)ld * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
  } else {
    permute_from_sorted(x.p, X, ld, n, nrhs, perm, s);
    SPD_CUDA(cudaStreamSynchronize(s));
  }
}

void h2_matmul_mixed_impl(spdhss_h2_s* h2, const double* X, double* Y, int nrhs, int64_t ld,
                          cudaStream_t s) {
  const int64_t n = h2->th.n;
  H2PlanF& PF = h2_plan_f(h2, nrhs, s);
  DevBuf<double> tmp((size_t)n * nrhs);
  permute_to_sorted(X, ld, tmp.p, n, nrhs, h2->td.perm.p, s);
  convert_d2f(tmp.p, PF.xs.p, n * nrhs, s);
  h2_plan_run(h2, PF, s);
  convert_f2d(PF.ys.p, tmp.p, n * nrhs, s);
  permute_from_sorted(tmp.p, Y, ld, n, nrhs, h2->td.perm.p, s);
}

}  // namespace spd
