// Preconditioned conjugate gradients (Sec. 6.2) with the H^2 product and the ULV solve of
// the SPD HSS approximation.  Every right-hand side column runs its own recurrence; a
// column stops when its recursive relative residual and then its recomputed true residual
// b - A x are both <= tol (otherwise the true residual replaces the recursive one).  All
// vectors stay on the device in tree order; the host reads one residual norm per column
// per iteration to decide.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <memory>
#include <utility>

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

// the same dot products for the vectors of several instances in one launch: work item =
// (problem, column); the partition of every column and the summation order are those of
// k_dot_partial / k_dot_final
struct DotProb {
  const double* a;
  const double* b;
  int64_t n;
  int ncol;
  double* part;
  double* out;
};

__global__ void __launch_bounds__(256) k_dot_partial_b(const DotProb* __restrict__ probs,
                                                       const int2* __restrict__ work) {
  const int2 w = work[blockIdx.y];
  const DotProb P = probs[w.x];
  const int c = w.y;
  const double* x = P.a + (int64_t)c * P.n;
  const double* y = P.b + (int64_t)c * P.n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < 8; ++w2) t += ws[w2];
    P.part[c * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_dot_final_b(const DotProb* __restrict__ probs, const int2* __restrict__ work,
                              int nwork) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nwork) return;
  const int2 w = work[k];
  const DotProb P = probs[w.x];
  double t = 0.0;
  for (int b = 0; b < DOT_BLOCKS; ++b) t += P.part[w.y * DOT_BLOCKS + b];
  P.out[w.y] = t;
}

static void dots_merged(std::vector<DotProb>& all, cudaStream_t s) {
  std::vector<int2> work;
  for (int p = 0; p < (int)all.size(); ++p)
    for (int c = 0; c < all[p].ncol; ++c) work.push_back(make_int2(p, c));
  if (work.empty()) return;
  DevBuf<DotProb> dp;
  DevBuf<int2> dw;
  dp.upload(all, s);
  dw.upload(work, s);
  for (size_t w0 = 0; w0 < work.size(); w0 += 65535) {
    const unsigned gy = (unsigned)std::min<size_t>(65535, work.size() - w0);
    k_dot_partial_b<<<dim3(DOT_BLOCKS, gy), 256, 0, s>>>(dp.p, dw.p + w0);
    SPD_LAUNCHED();
  }
  k_dot_final_b<<<ceil_div((int64_t)work.size(), 128), 128, 0, s>>>(dp.p, dw.p, (int)work.size());
  SPD_LAUNCHED();
}

static void dots(const double* a, const double* b, int64_t n, int ncol, double* part, double* out,
                 cudaStream_t s) {
  if (defer_launch("dots", std::vector<DotProb>{DotProb{a, b, n, ncol, part, out}}, dots_merged))
    return;
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

// The vector updates of several instances in one launch (blockIdx.y = instance).
struct VecProb {
  int op;                // 0: x, r update (k_axpy_xr); 1: p update (k_update_p); 2: out = b - ax
  double* x;             // x | p | out
  double* r;             // r | - | -
  const double* p;       // p | z | b
  const double* q;       // q | - | ax
  int64_t n;
  int ncol;
  const double* s1;      // rz | rzn
  const double* s2;      // pq | rz
  const int* done;
};

__global__ void __launch_bounds__(256) k_vec_b(const VecProb* __restrict__ probs) {
  const VecProb P = probs[blockIdx.y];
  const int64_t tot = P.n * P.ncol;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (P.op == 2) {
      P.x[e] = P.p[e] - P.q[e];
      continue;
    }
    const int c = (int)(e / P.n);
    if (P.done[c] == 1) continue;
    if (P.op == 0) {
      const double alpha = P.s2[c] != 0.0 ? P.s1[c] / P.s2[c] : 0.0;
      P.x[e] += alpha * P.p[e];
      P.r[e] -= alpha * P.q[e];
    } else {
      const double beta = (P.done[c] == 0 && P.s2[c] != 0.0) ? P.s1[c] / P.s2[c] : 0.0;
      P.x[e] = P.p[e] + beta * P.x[e];
    }
  }
}

static void vec_merged(std::vector<VecProb>& all, cudaStream_t s) {
  int64_t mx = 1;
  for (const auto& p : all) mx = std::max<int64_t>(mx, p.n * p.ncol);
  DevBuf<VecProb> dp;
  dp.upload(all, s);
  const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(mx, 256), 128);
  for (size_t y0 = 0; y0 < all.size(); y0 += 65535) {
    const unsigned gy = (unsigned)std::min<size_t>(65535, all.size() - y0);
    k_vec_b<<<dim3(gx, gy), 256, 0, s>>>(dp.p + y0);
    SPD_LAUNCHED();
  }
}

static void axpy_xr(double* x, double* r, const double* p, const double* q, int64_t n, int ncol,
                    const double* rz, const double* pq, const int* done, cudaStream_t s) {
  if (defer_launch("vec_axpy", std::vector<VecProb>{VecProb{0, x, r, p, q, n, ncol, rz, pq, done}},
                   vec_merged))
    return;
  k_axpy_xr<<<ceil_div(n * ncol, 256), 256, 0, s>>>(x, r, p, q, n, ncol, rz, pq, done);
  SPD_LAUNCHED();
}

static void update_p(double* p, const double* z, int64_t n, int ncol, const double* rzn,
                     const double* rz, const int* done, cudaStream_t s) {
  if (defer_launch("vec_update",
                   std::vector<VecProb>{VecProb{1, p, nullptr, z, nullptr, n, ncol, rzn, rz, done}},
                   vec_merged))
    return;
  k_update_p<<<ceil_div(n * ncol, 256), 256, 0, s>>>(p, z, n, ncol, rzn, rz, done);
  SPD_LAUNCHED();
}

static void sub(const double* b, const double* ax, double* out, int64_t count, cudaStream_t s) {
  if (defer_launch("vec_sub",
                   std::vector<VecProb>{VecProb{2, out, nullptr, b, ax, count, 1, nullptr, nullptr,
                                                nullptr}},
                   vec_merged))
    return;
  k_sub<<<ceil_div(count, 256), 256, 0, s>>>(b, ax, out, count);
  SPD_LAUNCHED();
}

// Pinned host landing place of the per-iteration residual norms (a device-to-host copy
// that a captured graph can hold).
struct PinnedScalars {
  double* p = nullptr;
  explicit PinnedScalars(int n) { SPD_CUDA(cudaHostAlloc((void**)&p, sizeof(double) * std::max(n, 1), cudaHostAllocDefault)); }
  ~PinnedScalars() { if (p) cudaFreeHost(p); }
  PinnedScalars(const PinnedScalars&) = delete;
  PinnedScalars& operator=(const PinnedScalars&) = delete;
};

// SPDHSS_PCG_GRAPHS=0 launches every iteration directly (the graphs replay the same
// launches in the same order, so results do not depend on the setting).
static bool pcg_graphs_enabled() {
  const char* e = std::getenv("SPDHSS_PCG_GRAPHS");
  return !(e && e[0] == '0');
}

// A CUDA graph of a fixed launch sequence, captured once on the solve's stream (relaxed
// mode: the launchers' attribute calls are allowed) and replayed; if the capture fails the
// solve keeps launching directly.
struct PcgGraph {
  bool enabled;
  bool tried = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  int64_t launches = 0;   // kernels per replay (added to the launch count)
  explicit PcgGraph(bool on) : enabled(on) {}
  ~PcgGraph() {
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
  }
  bool ready() const { return ex != nullptr; }
  // forget the captured iteration (its launches changed); the next steady one re-captures
  void reset() {
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    ex = nullptr;
    g = nullptr;
    tried = false;
  }
  template <class F>
  void capture(cudaStream_t s, F&& body) {
    if (tried) return;
    tried = true;
    const int64_t before = spdhss_launch_count();
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    bool ok = true;
    try {
      body();
    } catch (...) {
      ok = false;
    }
    cudaGraph_t cg = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &cg);
    launches = spdhss_launch_count() - before;
    count_launches(-launches);   // captured, not executed
    if (!ok || e != cudaSuccess || !cg) {
      if (cg) cudaGraphDestroy(cg);
      cudaGetLastError();
      return;
    }
    if (cudaGraphInstantiate(&ex, cg, 0) != cudaSuccess) {
      cudaGraphDestroy(cg);
      ex = nullptr;
      cudaGetLastError();
      return;
    }
    g = cg;
  }
  void launch(cudaStream_t s) {
    SPD_CUDA(cudaGraphLaunch(ex, s));
    count_launches(launches);
  }
};

// At a residual refresh of the mixed-precision solve: a column still iterating whose FP64
// true residual is more than twice its recursive one (the FP32 recursion no longer describes
// the FP64 residual: the FP32 product's error, relative to the residual, has become
// comparable to the residual itself, as for kernel matrices of large condition number)
// also restarts its direction (beta = 0, flag 2).  Its iteration then proceeds as
// iterative refinement: every block of iterations is an inner PCG for A d = r with the
// FP32 product, started from the FP64 residual.  Columns whose recursion still holds keep
// their direction (plain residual replacement).  Returns whether a flag changed.
static bool refresh_restarts(const std::vector<double>& trel, const std::vector<double>& rr,
                             const std::vector<double>& bn, std::vector<int>& hdone) {
  bool any = false;
  for (size_t c = 0; c < hdone.size(); ++c) {
    if (hdone[c] != 0) continue;
    if (trel[c] > 2.0 * std::sqrt(std::max(rr[c], 0.0)) / bn[c]) {
      hdone[c] = 2;
      any = true;
    }
  }
  return any;
}

// At a residual refresh of the mixed-precision solve: whether a column still iterating has
// a true residual above 0.9 of its value at the previous refresh (a whole block of
// iterations without progress: the FP32 product's error relative to the residual is too
// large for the refinement to contract).  The solve then takes FP64 products from here on,
// every column restarting its direction.  tprev is updated to trel.
static bool refresh_stalled(const std::vector<double>& trel, std::vector<double>& tprev,
                            const std::vector<int>& hdone) {
  bool stalled = false;
  for (size_t c = 0; c < hdone.size(); ++c) {
    if (hdone[c] == 0 && trel[c] > 0.9 * tprev[c]) stalled = true;
    tprev[c] = trel[c];
  }
  return stalled;
}

// precision = 0: FP64 throughout.  precision = 1: the product with A inside the iteration
// uses the FP32 copy of the H^2 matrix (FP32 kernel entries and accumulation); the ULV
// preconditioner, the recurrences and every residual check stay FP64, and every
// `refresh` iterations the recursive residual is replaced by the FP64 true residual
// (restarting the columns whose recursion has drifted, refresh_restarts; switching to FP64
// products when a block of iterations made no progress, refresh_stalled).
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
  // no factorization: plain CG (z = r)
  UlvPlan* PU = u ? &ulv_plan(u, nrhs, s) : nullptr;
  double* p = PA.xs.p;
  double* q = PA.ys.p;
  H2PlanF* PF = precision ? &h2_plan_f(h2, nrhs, s) : nullptr;
  DevBuf<double> zown;
  if (!PU) zown.alloc(nc);
  double* z = PU ? PU->bw[0].p : zown.p;
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
  x.zero(s);
  done.zero(s);
  merge_stage(10, 0);
  copy_vec(r.p, bs.p, nc, s);
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
  std::vector<double> tprev(nrhs, INFINITY);   // true residuals at the previous refresh
  // z = M^{-1} r, p = z, rz = r.z
  copy_vec(z, r.p, nc, s);
  if (PU) ulv_solve_sorted(u, *PU, s);
  copy_vec(p, z, nc, s);
  dots(r.p, z, n, nrhs, part.p, rz, s);
  std::vector<double> hrr(nrhs);
  auto true_residual = [&](std::vector<double>& rel, bool replace_active) {
    copy_vec(PR.xs.p, x.p, nc, s);
    h2_plan_run(h2, PR, s);
    sub(bs.p, PR.ys.p, PR.ys.p, nc, s);
    dots(PR.ys.p, PR.ys.p, n, nrhs, part.p, rr, s);
    std::vector<double> h(nrhs);
    SPD_CUDA(cudaMemcpyAsync(h.data(), rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    rel.resize(nrhs);
    for (int c = 0; c < nrhs; ++c) rel[c] = std::sqrt(std::max(h[c], 0.0)) / bn[c];
    (void)replace_active;
  };
  // One iteration's launches between its two host decisions: s1 (q = A p, the step, the
  // residual norms, landing in pinned host memory) and s2 (z = M^-1 r, the new direction).
  PinnedScalars prr(nrhs);
  auto s1 = [&]() {
    if (PF) {                                     // q = A p in FP32
      convert_d2f(p, PF->xs.p, nc, s);
      h2_plan_run(h2, *PF, s);
      convert_f2d(PF->ys.p, q, nc, s);
    } else {
      h2_plan_run(h2, PA, s);                     // q = A p
    }
    dots(p, q, n, nrhs, part.p, pq, s);
    axpy_xr(x.p, r.p, p, q, n, nrhs, rz, pq, done.p, s);
    dots(r.p, r.p, n, nrhs, part.p, rr, s);
    SPD_CUDA(cudaMemcpyAsync(prr.p, rr, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  };
  auto s2 = [&]() {
    copy_vec(z, r.p, nc, s);
    if (PU) ulv_solve_sorted(u, *PU, s);          // z = M^{-1} r
    dots(r.p, z, n, nrhs, part.p, rzn, s);
    update_p(p, z, n, nrhs, rzn, rz, done.p, s);
    copy_vec(rz, rzn, nrhs, s);
  };
  // Steady iterations (no host intervention) replay s2 of one iteration and s1 of the next
  // as one captured CUDA graph: the launches and their order are those of the direct path,
  // so the results are identical.  Captured from the third iteration on, once per solve.
  PcgGraph graph(pcg_graphs_enabled() && !merging() && !prof_enabled() && s != nullptr &&
                 s != cudaStreamLegacy && s != cudaStreamPerThread);
  bool fused = false;   // s1 of this iteration was launched inside the graph
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    merge_stage(10, it);
    if (!fused) s1();
    fused = false;
    SPD_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < nrhs; ++c) hrr[c] = prr.p[c];
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
          copy_vec(r.p + (int64_t)c * n, PR.ys.p + (int64_t)c * n, n, s);
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
      copy_vec(r.p, PR.ys.p, nc, s);
      bool flags = false;
      if (refresh_stalled(trel, tprev, hdone)) {
        PF = nullptr;                               // FP64 products from here on
        for (int c = 0; c < nrhs; ++c)
          if (hdone[c] == 0) hdone[c] = 2;
        graph.reset();
        flags = true;
      } else {
        flags = refresh_restarts(trel, hrr, bn, hdone);
      }
      if (flags)
        SPD_CUDA(cudaMemcpyAsync(done.p, hdone.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    bool restart = false;
    for (int c = 0; c < nrhs; ++c) restart = restart || hdone[c] == 2;
    // a restart changes the device flags between s2 and the next s1: launched directly
    if (graph.enabled && !restart && it >= 2 && it < maxit) {
      if (!graph.ready()) graph.capture(s, [&]() { s2(); s1(); });
      if (graph.ready()) {
        graph.launch(s);
        fused = true;
        continue;
      }
    }
    s2();
    if (restart) {
      for (int c = 0; c < nrhs; ++c)
        if (hdone[c] == 2) hdone[c] = 0;
      SPD_CUDA(cudaMemcpyAsync(done.p, hdone.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
  }
  std::vector<double> trel;
  merge_stage(11, 0);
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

// ---------------------------------------------------------------------------------------
// PCG for many independent instances in lockstep, driven by one host thread: every stage
// of an iteration (each level of the H^2 passes, the coupling and near-field steps, each
// level of the ULV solve, the dots and vector updates) is one launch over the problems of
// all active instances, concatenated from the instances' own plans whenever the active
// set changes.  The recurrences, the true-residual confirmation and the residual
// replacement are those of pcg_impl, per instance and per column.
// ---------------------------------------------------------------------------------------
namespace spd {
namespace {

void gemm_cat(GemmBatch& out, const GemmBatch& in) {
  const int off = (int)out.segs.size();
  out.segs.insert(out.segs.end(), in.segs.begin(), in.segs.end());
  for (GemmProb p : in.probs) {
    p.seg0 += off;
    p.seg1 += off;
    out.probs.push_back(p);
  }
}

void rowcoup_cat(RowCoupBatchT<double>& out, const RowCoupBatchT<double>& in) {
  const int off = (int)out.chunks.size();
  out.chunks.insert(out.chunks.end(), in.chunks.begin(), in.chunks.end());
  for (RowCoupProbT<double> p : in.probs) {
    p.ch0 += off;
    p.ch1 += off;
    out.probs.push_back(p);
  }
  out.ncol = std::max(out.ncol, in.ncol);
}

struct Inst {
  spdhss_h2_s* h2 = nullptr;
  spdhss_ulv_s* u = nullptr;
  H2Plan* PA = nullptr;
  H2Plan* PR = nullptr;
  UlvPlan* PU = nullptr;
  H2PlanF* PF = nullptr;      // mixed precision: the FP32 plan of q = A p
  bool fp64 = false;          // mixed precision: switched to FP64 products (refresh_stalled)
  std::vector<double> tprev;  // mixed precision: true residuals at the previous refresh
  int64_t n = 0, ld = 0;
  int nrhs = 0, D = 0, nlev = 0;
  const double* B = nullptr;
  double* X = nullptr;
  DevBuf<double> bs, x, r, part;
  int64_t so = 0;             // offset of this instance's columns in the scalar pools
  std::vector<double> bn;
  std::vector<int> hdone, hit;
  bool active = true;
};

// scalar pools: rz | pq | rzn | rr, NC entries each (NC = all columns of all instances)
struct Pools {
  int64_t NC = 0;
  DevBuf<double> sc;
  DevBuf<int> done;
  double* rz(const Inst& a) const { return sc.p + a.so; }
  double* pq(const Inst& a) const { return sc.p + NC + a.so; }
  double* rzn(const Inst& a) const { return sc.p + 2 * NC + a.so; }
  double* rr(const Inst& a) const { return sc.p + 3 * NC + a.so; }
  int* dn(const Inst& a) const { return done.p + a.so; }
};

struct Merged {
  GemmBatch up_leaf, leaf_out, near_g, coupling, root_f, root_b;
  std::vector<GemmBatch> up, down, fwd, bwd;
  RowCoupBatchT<double> rowcoup, near_r;
  Batch<CopyProb> zero_yhat, z_from_r, rz_from_rzn;
  std::vector<Batch<CopyProb>> uup, udown;
  std::vector<DotProb> d_pq, d_rr, d_rz;
  std::vector<VecProb> v_axpy, v_upd;
  std::vector<int> near_direct;   // instances whose near field is evaluated on the fly
};

CopyProb vcopy(double* dst, const double* src, int64_t count) {
  CopyProb c{};
  c.src = src; c.lds = count; c.dst = dst; c.ldd = count; c.m = (int)count; c.n = 1;
  c.alpha = 1.0;
  return c;
}

// mixed: the FP64 product steps only of the instances switched to FP64 products (the
// others take q = A p from MergedF)
void build_merged(std::vector<Inst>& I, const Pools& pl, Merged& M, cudaStream_t s,
                  bool mixed = false) {
  M = Merged();
  int maxD = 0, maxlev = 0;
  for (auto& a : I)
    if (a.active) { maxD = std::max(maxD, a.D); maxlev = std::max(maxlev, a.nlev); }
  M.up.resize(std::max(maxD - 1, 0));
  M.down.resize(std::max(maxD - 1, 0));
  M.fwd.resize(maxlev);
  M.bwd.resize(maxlev);
  M.uup.resize(maxlev);
  M.udown.resize(maxlev);
  for (int k = 0; k < (int)I.size(); ++k) {
    Inst& a = I[k];
    if (!a.active) continue;
    const H2Plan& P = *a.PA;
    const int64_t nc = a.n * a.nrhs;
    if (!mixed || a.fp64) {
      gemm_cat(M.up_leaf, P.up_leaf);
      for (size_t h = 0; h < P.up.size(); ++h) gemm_cat(M.up[h], P.up[h]);
      // down[t] is depth t + 1, at height nd - t above the leaves; merged top first
      const int nd = (int)P.down.size();
      for (int t = 0; t < nd; ++t) gemm_cat(M.down[(maxD - 1) - (nd - t)], P.down[t]);
      gemm_cat(M.leaf_out, P.leaf_out);
      if (P.use_rowcoup) rowcoup_cat(M.rowcoup, P.rowcoup);
      else gemm_cat(M.coupling, P.coupling);
      if (P.near_rows) rowcoup_cat(M.near_r, P.near_r);
      else if (P.near_stored) gemm_cat(M.near_g, P.near_g);
      else M.near_direct.push_back(k);
      if (P.yhat.n > 0) M.zero_yhat.push(vcopy(P.yhat.p, nullptr, (int64_t)P.yhat.n));
    }
    // ULV solve by level from the leaves; every root after every forward level
    const UlvPlan& U = *a.PU;
    for (int l = 0; l < a.nlev; ++l) {
      gemm_cat(M.fwd[l], U.fwd[l]);
      gemm_cat(M.bwd[l], U.bwd[l]);
      M.uup[l].h.insert(M.uup[l].h.end(), U.up[l].h.begin(), U.up[l].h.end());
      M.udown[l].h.insert(M.udown[l].h.end(), U.down[l].h.begin(), U.down[l].h.end());
    }
    gemm_cat(M.root_f, U.root_f);
    gemm_cat(M.root_b, U.root_b);
    double* p = P.xs.p;
    double* q = P.ys.p;
    double* z = U.bw[0].p;
    M.d_pq.push_back(DotProb{p, q, a.n, a.nrhs, a.part.p, pl.pq(a)});
    M.d_rr.push_back(DotProb{a.r.p, a.r.p, a.n, a.nrhs, a.part.p, pl.rr(a)});
    M.d_rz.push_back(DotProb{a.r.p, z, a.n, a.nrhs, a.part.p, pl.rzn(a)});
    M.v_axpy.push_back(VecProb{0, a.x.p, a.r.p, p, q, a.n, a.nrhs, pl.rz(a), pl.pq(a), pl.dn(a)});
    M.v_upd.push_back(VecProb{1, p, nullptr, z, nullptr, a.n, a.nrhs, pl.rzn(a), pl.rz(a), pl.dn(a)});
    M.z_from_r.push(vcopy(z, a.r.p, nc));
    M.rz_from_rzn.push(vcopy(pl.rz(a), pl.rzn(a), a.nrhs));
  }
  auto up_g = [&](GemmBatch& g, const char* tag) { g.tag = tag; g.upload(s); };
  up_g(M.up_leaf, "h2_basis");
  for (auto& g : M.up) up_g(g, "h2_basis");
  for (auto& g : M.down) up_g(g, "h2_basis");
  up_g(M.leaf_out, "h2_basis");
  up_g(M.coupling, "h2_coupling");
  up_g(M.near_g, "near_h2_stored");
  for (auto& g : M.fwd) up_g(g, "gemm_ulv_solve");
  for (auto& g : M.bwd) up_g(g, "gemm_ulv_solve");
  up_g(M.root_f, "gemm_ulv_root");
  up_g(M.root_b, "gemm_ulv_root");
  M.rowcoup.tag = "h2_coupling";
  M.near_r.tag = "near_h2_stored";
  if (!M.rowcoup.probs.empty()) M.rowcoup.upload(s);
  if (!M.near_r.probs.empty()) M.near_r.upload(s);
  M.zero_yhat.upload(s);
  M.z_from_r.upload(s);
  M.rz_from_rzn.upload(s);
  for (auto& b : M.uup) b.upload(s);
  for (auto& b : M.udown) b.upload(s);
}

void run_h2_merged(const std::vector<Inst>& I, const Merged& M, cudaStream_t s) {
  M.up_leaf.launch(s);
  for (const auto& g : M.up) g.launch(s);
  copy_launch(M.zero_yhat, s);
  if (!M.rowcoup.probs.empty()) M.rowcoup.launch(s);
  M.coupling.launch(s);
  for (const auto& g : M.down) g.launch(s);
  M.leaf_out.launch(s);
  if (!M.near_r.probs.empty()) M.near_r.launch(s);
  M.near_g.launch(s);
  for (int k : M.near_direct) {
    const Inst& a = I[k];
    a.PA->near.launch(a.h2->kfn, a.h2->td.xs.p, a.h2->th.n, a.h2->th.dim, s);
  }
}

void run_ulv_merged(const Merged& M, cudaStream_t s) {
  for (size_t l = 0; l < M.fwd.size(); ++l) {
    M.fwd[l].launch(s);
    copy_launch(M.uup[l], s);
  }
  M.root_f.launch(s);
  M.root_b.launch(s);
  for (int l = (int)M.fwd.size() - 1; l >= 0; --l) {
    copy_launch(M.udown[l], s);
    M.bwd[l].launch(s);
  }
}

// FP64 <-> FP32 copies of several instances' vectors in one launch, element by element
// with the rounding of convert_d2f / convert_f2d
struct ConvProb {
  double* d;
  float* f;
  int64_t count;
};

__global__ void k_convert_b(const ConvProb* __restrict__ probs, int to_float) {
  const ConvProb P = probs[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P.count;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (to_float) P.f[e] = (float)P.d[e];
    else P.d[e] = (double)P.f[e];
  }
}

// q = A p in FP32 for all instances of a mixed solve.  Step t of every instance's once-read
// plan (its upward levels with their partial sums, the couplings and their sums, its
// downward levels) goes into one launch per column count, the near fields into one launch
// per kernel kind and column block.  Every job, sum and near-field problem keeps its own
// arithmetic (the jobs are independent, each output entry is summed by one thread in a
// fixed order, the near-field problems keep the column block and segment split of their
// own plan), so each instance's product is bit-identical to h2_plan_run of its FP32 plan.
// Instances whose FP32 plan has no once-read form run that plan on their own.
struct MergedF {
  std::vector<std::map<int, std::unique_ptr<SymBatch>>> sym;   // per step, by column count
  std::vector<std::unique_ptr<SymSumBatch>> sum;                // per step
  std::map<std::pair<int, int>, std::unique_ptr<NearBatchT<float>>> near;   // (kind, cb)
  std::vector<int> direct;
  std::vector<ConvProb> to_f, to_d;
  DevBuf<ConvProb> d_to_f, d_to_d;
  int64_t max_count = 0;
};

void build_merged_f(const std::vector<Inst>& I, MergedF& F, cudaStream_t s) {
  for (int k = 0; k < (int)I.size(); ++k) {
    const Inst& a = I[k];
    if (!a.active || a.fp64) continue;
    const H2PlanF& P = *a.PF;
    const int64_t nc = a.n * a.nrhs;
    F.to_f.push_back(ConvProb{a.PA->xs.p, P.xs.p, nc});
    F.to_d.push_back(ConvProb{a.PA->ys.p, P.ys.p, nc});
    F.max_count = std::max(F.max_count, nc);
    if (!P.sym) { F.direct.push_back(k); continue; }
    const std::vector<PlanStep>& steps = P.sym->steps;
    if (F.sym.size() < steps.size()) {
      F.sym.resize(steps.size());
      F.sum.resize(steps.size());
    }
    for (size_t t = 0; t < steps.size(); ++t) {
      const SymBatch* b = steps[t].sym.get();
      if (b && !b->jobs.empty()) {
        std::unique_ptr<SymBatch>& m = F.sym[t][b->nc];
        if (!m) {
          m.reset(new SymBatch());
          m->nc = b->nc;
          m->ncol = b->ncol;
          m->tag = b->tag;
        }
        m->jobs.insert(m->jobs.end(), b->jobs.begin(), b->jobs.end());
        m->ncol = std::max(m->ncol, b->ncol);
        m->bytes += b->bytes;
        m->flops += b->flops;
      }
      const SymSumBatch* u = steps[t].sum.get();
      if (u && !u->jobs.empty()) {
        std::unique_ptr<SymSumBatch>& m = F.sum[t];
        if (!m) {
          m.reset(new SymSumBatch());
          m->ncol = u->ncol;
          m->tag = u->tag;
        }
        const int off = (int)m->srcs.size();
        m->srcs.insert(m->srcs.end(), u->srcs.begin(), u->srcs.end());
        for (SymSum j : u->jobs) {
          j.s0 += off;
          j.s1 += off;
          m->jobs.push_back(j);
        }
        m->ncol = std::max(m->ncol, u->ncol);
        m->bytes += u->bytes;
      }
    }
    // the near field as its own launch gets it: the instance's points and kernel parameters
    for (NearProbT<float> p : P.near.probs) {
      SPD_REQUIRE(p.cb != 0, "mixed batched PCG: FP32 near-field plan not uploaded");
      if (!p.xs) {
        p.xs = a.h2->td.xs.p;
        p.ldx = a.h2->th.n;
        p.dim = a.h2->th.dim;
        p.inv_ell = a.h2->kfn.inv_ell;
        p.shift = a.h2->kfn.shift;
      }
      std::unique_ptr<NearBatchT<float>>& m = F.near[std::make_pair(a.h2->kfn.kind, p.cb)];
      if (!m) {
        m.reset(new NearBatchT<float>());
        m->tag = P.near.tag;
      }
      const int so = (int)m->segs.size();
      m->segs.insert(m->segs.end(), P.near.segs.begin() + p.seg0, P.near.segs.begin() + p.seg1);
      p.seg1 = so + (p.seg1 - p.seg0);
      p.seg0 = so;
      m->probs.push_back(p);
    }
  }
  SPD_REQUIRE(F.to_f.size() <= 65535, "mixed batched PCG: at most 65535 instances per call");
  for (auto& st : F.sym)
    for (auto& kv : st) kv.second->upload(s);
  for (auto& u : F.sum)
    if (u) u->upload(s);
  for (auto& kv : F.near) kv.second->upload(s);
  F.d_to_f.upload(F.to_f, s);
  F.d_to_d.upload(F.to_d, s);
}

void convert_merged(const MergedF& F, bool to_float, cudaStream_t s) {
  if (F.to_f.empty()) return;
  const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(F.max_count, 256), 152 * 16);
  k_convert_b<<<dim3(gx, (unsigned)F.to_f.size()), 256, 0, s>>>(
      to_float ? F.d_to_f.p : F.d_to_d.p, to_float ? 1 : 0);
  SPD_LAUNCHED();
}

void run_h2_merged_f(const std::vector<Inst>& I, const MergedF& F, cudaStream_t s) {
  convert_merged(F, true, s);
  for (size_t t = 0; t < F.sym.size(); ++t) {
    for (const auto& kv : F.sym[t]) kv.second->launch(s);
    if (F.sum[t]) F.sum[t]->launch(s);
  }
  for (const auto& kv : F.near) {
    KernelFn k{};
    k.kind = kv.first.first;
    kv.second->launch(k, nullptr, 0, 0, s);
  }
  for (int k : F.direct) h2_plan_run(I[k].h2, *I[k].PF, s);
  convert_merged(F, false, s);
}

}  // namespace

void pcg_batched_impl(int count, spdhss_h2_s* const* h2, spdhss_ulv_s* const* ulv,
                      const double* const* B, double* const* X, const int* nrhs,
                      const int64_t* ld, double tol, int maxit, int* const* iters_out,
                      double* const* relres_out, spdhss_status* status, cudaStream_t s,
                      int precision, spdhss_done_fn on_done, void* user) {
  std::vector<Inst> I(count);
  Pools pl;
  for (int k = 0; k < count; ++k) {
    Inst& a = I[k];
    a.h2 = h2[k];
    a.u = ulv[k];
    a.n = a.h2->th.n;
    a.ld = ld[k];
    a.nrhs = nrhs[k];
    a.D = a.h2->th.D;
    a.nlev = std::max(a.u->L - 1, 0);
    a.B = B[k];
    a.X = X[k];
    a.so = pl.NC;
    pl.NC += a.nrhs;
    auto get_plan = [&](int key) -> H2Plan* {
      auto it = a.h2->plans.find(key);
      if (it == a.h2->plans.end()) {
        std::unique_ptr<H2Plan> p(new H2Plan());
        h2_plan_build(a.h2, *p, a.nrhs, 1, s);
        it = a.h2->plans.emplace(key, std::move(p)).first;
      }
      return it->second.get();
    };
    a.PA = get_plan(a.nrhs);
    a.PR = get_plan(-a.nrhs);
    a.PU = &ulv_plan(a.u, a.nrhs, s);
    if (precision) a.PF = &h2_plan_f(a.h2, a.nrhs, s);
    a.tprev.assign(a.nrhs, INFINITY);
  }
  pl.sc.alloc((size_t)std::max<int64_t>(4 * pl.NC, 1));
  pl.done.alloc((size_t)std::max<int64_t>(pl.NC, 1));
  pl.done.zero(s);
  // start: x = 0, r = b, z = M^{-1} r, p = z, rz = r.z (per instance)
  for (auto& a : I) {
    const int64_t nc = a.n * a.nrhs;
    const int64_t* perm = a.h2->td.perm.p;
    a.bs.alloc(nc);
    a.x.alloc(nc);
    a.r.alloc(nc);
    a.part.alloc((size_t)DOT_BLOCKS * a.nrhs);
    if (!is_device_pointer(a.B)) {
      DevBuf<double> tmp((size_t)a.ld * a.nrhs);
      SPD_CUDA(cudaMemcpyAsync(tmp.p, a.B, (size_t)a.ld * a.nrhs * sizeof(double),
                               cudaMemcpyHostToDevice, s));
      permute_to_sorted(tmp.p, a.ld, a.bs.p, a.n, a.nrhs, perm, s);
      SPD_CUDA(cudaStreamSynchronize(s));
    } else {
      permute_to_sorted(a.B, a.ld, a.bs.p, a.n, a.nrhs, perm, s);
    }
    a.x.zero(s);
    copy_vec(a.r.p, a.bs.p, nc, s);
    dots(a.bs.p, a.bs.p, a.n, a.nrhs, a.part.p, pl.rr(a), s);
    double* z = a.PU->bw[0].p;
    copy_vec(z, a.r.p, nc, s);
    ulv_solve_sorted(a.u, *a.PU, s);
    copy_vec(a.PA->xs.p, z, nc, s);
    dots(a.r.p, z, a.n, a.nrhs, a.part.p, pl.rz(a), s);
    a.hdone.assign(a.nrhs, 0);
    a.hit.assign(a.nrhs, 0);
  }
  std::vector<double> hsc(4 * pl.NC);
  SPD_CUDA(cudaMemcpyAsync(hsc.data(), pl.sc.p, 4 * pl.NC * sizeof(double), cudaMemcpyDeviceToHost, s));
  SPD_CUDA(cudaStreamSynchronize(s));
  for (auto& a : I) {
    a.bn.resize(a.nrhs);
    for (int c = 0; c < a.nrhs; ++c) {
      const double v = hsc[3 * pl.NC + a.so + c];
      a.bn[c] = v > 0.0 ? std::sqrt(v) : 1.0;
    }
  }
  // b - A x of one instance, relative per column (its own plans, direct launches)
  auto true_residual = [&](Inst& a, std::vector<double>& rel) {
    const int64_t nc = a.n * a.nrhs;
    copy_vec(a.PR->xs.p, a.x.p, nc, s);
    h2_plan_run(a.h2, *a.PR, s);
    sub(a.bs.p, a.PR->ys.p, a.PR->ys.p, nc, s);
    dots(a.PR->ys.p, a.PR->ys.p, a.n, a.nrhs, a.part.p, pl.rr(a), s);
    std::vector<double> h(a.nrhs);
    SPD_CUDA(cudaMemcpyAsync(h.data(), pl.rr(a), a.nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    rel.resize(a.nrhs);
    for (int c = 0; c < a.nrhs; ++c) rel[c] = std::sqrt(std::max(h[c], 0.0)) / a.bn[c];
  };
  // the outputs of instance k: its final true residuals, iterations and solution; then, with
  // a callback, the stream is synchronized and the caller told
  std::vector<char> finished(count, 0);
  auto finish = [&](int k) {
    Inst& a = I[k];
    std::vector<double> trel;
    true_residual(a, trel);
    bool conv = true;
    for (int c = 0; c < a.nrhs; ++c) {
      if (iters_out && iters_out[k]) iters_out[k][c] = a.hit[c];
      if (relres_out && relres_out[k]) relres_out[k][c] = trel[c];
      conv = conv && trel[c] <= tol;
    }
    const int64_t* perm = a.h2->td.perm.p;
    if (!is_device_pointer(a.X)) {
      DevBuf<double> tmp((size_t)a.ld * a.nrhs);
      if (a.ld > a.n)
        SPD_CUDA(cudaMemcpyAsync(tmp.p, a.X, (size_t)a.ld * a.nrhs * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
      permute_from_sorted(a.x.p, tmp.p, a.ld, a.n, a.nrhs, perm, s);
      SPD_CUDA(cudaMemcpyAsync(a.X, tmp.p, (size_t)a.ld * a.nrhs * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
      SPD_CUDA(cudaStreamSynchronize(s));
    } else {
      permute_from_sorted(a.x.p, a.X, a.ld, a.n, a.nrhs, perm, s);
    }
    const spdhss_status st = conv ? SPDHSS_OK : SPDHSS_NO_CONVERGENCE;
    if (status) status[k] = st;
    finished[k] = 1;
    if (on_done) {
      SPD_CUDA(cudaStreamSynchronize(s));
      on_done(user, k, st);
    }
  };
  Merged M;
  build_merged(I, pl, M, s, precision != 0);
  std::unique_ptr<MergedF> F;
  if (precision) {
    F.reset(new MergedF());
    build_merged_f(I, *F, s);
  }
  std::vector<double> hrr(pl.NC);
  int nactive = count;
  // Converged instances stay in the merged launches (their updates are masked by the done
  // flags) until the active set has shrunk by a third: re-concatenating the stage batches
  // costs more host time than the masked work of a few instances.
  int merged_active = count;
  for (int it = 1; it <= maxit && nactive > 0; ++it) {
    run_h2_merged(I, M, s);                                   // q = A p
    if (F) run_h2_merged_f(I, *F, s);                         // ... in FP32 where mixed
    { std::vector<DotProb> v = M.d_pq; dots_merged(v, s); }
    { std::vector<VecProb> v = M.v_axpy; vec_merged(v, s); }
    { std::vector<DotProb> v = M.d_rr; dots_merged(v, s); }
    SPD_CUDA(cudaMemcpyAsync(hrr.data(), pl.sc.p + 3 * pl.NC, pl.NC * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    bool changed_set = false;
    for (int k = 0; k < count; ++k) {
      Inst& a = I[k];
      if (!a.active) continue;
      bool any_pass = false;
      for (int c = 0; c < a.nrhs; ++c) {
        if (a.hdone[c] == 1) continue;
        a.hit[c] = it;
        const double v = hrr[a.so + c];
        if (!std::isfinite(v)) throw Error(SPDHSS_NUMERIC, "pcg_solve_batched: residual is not finite");
        if (std::sqrt(std::max(v, 0.0)) / a.bn[c] <= tol) any_pass = true;
      }
      if (any_pass) {
        std::vector<double> trel;
        true_residual(a, trel);
        bool changed = false;
        for (int c = 0; c < a.nrhs; ++c) {
          if (a.hdone[c] == 1) continue;
          if (std::sqrt(std::max(hrr[a.so + c], 0.0)) / a.bn[c] > tol) continue;
          if (trel[c] <= tol) { a.hdone[c] = 1; changed = true; }
          else {
            copy_vec(a.r.p + (int64_t)c * a.n, a.PR->ys.p + (int64_t)c * a.n, a.n, s);
            a.hdone[c] = 2;
            changed = true;
          }
        }
        if (changed)
          SPD_CUDA(cudaMemcpyAsync(pl.dn(a), a.hdone.data(), a.nrhs * sizeof(int),
                                   cudaMemcpyHostToDevice, s));
      }
      bool all = true;
      for (int c = 0; c < a.nrhs; ++c) all = all && a.hdone[c] == 1;
      if (all) {
        a.active = false;
        --nactive;
        changed_set = true;
        if (on_done) finish(k);   // x no longer changes: its outputs now, as at the end
      }
    }
    if (nactive == 0) break;
    // mixed precision: every 50 iterations the recursive residual of each instance still
    // iterating on FP32 products is replaced by its FP64 true residual b - A x, with the
    // restarts and the switch to FP64 products of pcg_impl
    bool switched = false;
    if (F && it % 50 == 0)
      for (auto& a : I) {
        if (!a.active || a.fp64) continue;
        std::vector<double> trel;
        true_residual(a, trel);
        copy_vec(a.r.p, a.PR->ys.p, a.n * a.nrhs, s);
        bool flags = false;
        if (refresh_stalled(trel, a.tprev, a.hdone)) {
          a.fp64 = true;
          switched = true;
          for (int c = 0; c < a.nrhs; ++c)
            if (a.hdone[c] == 0) a.hdone[c] = 2;
          flags = true;
        } else {
          std::vector<double> arr(hrr.begin() + a.so, hrr.begin() + a.so + a.nrhs);
          flags = refresh_restarts(trel, arr, a.bn, a.hdone);
        }
        if (flags)
          SPD_CUDA(cudaMemcpyAsync(pl.dn(a), a.hdone.data(), a.nrhs * sizeof(int),
                                   cudaMemcpyHostToDevice, s));
      }
    if (switched || (changed_set && 3 * nactive <= 2 * merged_active)) {
      build_merged(I, pl, M, s, precision != 0);
      if (F) {
        F.reset(new MergedF());
        build_merged_f(I, *F, s);
      }
      merged_active = nactive;
    }
    copy_launch(M.z_from_r, s);
    run_ulv_merged(M, s);                                     // z = M^{-1} r
    { std::vector<DotProb> v = M.d_rz; dots_merged(v, s); }
    { std::vector<VecProb> v = M.v_upd; vec_merged(v, s); }
    copy_launch(M.rz_from_rzn, s);
    for (auto& a : I) {
      if (!a.active) continue;
      bool restarted = false;
      for (int c = 0; c < a.nrhs; ++c)
        if (a.hdone[c] == 2) { a.hdone[c] = 0; restarted = true; }
      if (restarted)
        SPD_CUDA(cudaMemcpyAsync(pl.dn(a), a.hdone.data(), a.nrhs * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
    }
  }
  // final true residuals, outputs (of the instances not finished early)
  for (int k = 0; k < count; ++k)
    if (!finished[k]) finish(k);
  SPD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace spd
