// C ABI entry points (include/spdhss.h): argument checks, error capture, and the H^2 calls.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_set>

#include "h2.cuh"
#include "tune.cuh"

namespace spd {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_last_error(const std::string& msg) { g_last_error = msg; }

cudaStream_t& current_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}

// One memory pool per device, kept across calls (release threshold: never trim).
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;
static std::unordered_set<void*> g_plain;   // allocations made outside the pool

static cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  SPD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  // the pool may grow to the whole device (its default limit is smaller), so that the
  // largest workloads can hold their generators and factors in it
  size_t free_b = 0, total_b = 0;
  SPD_CUDA(cudaMemGetInfo(&free_b, &total_b));
  props.maxSize = total_b;
  cudaMemPool_t pool;
  SPD_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = UINT64_MAX;
  SPD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  g_pools[dev] = pool;
  return pool;
}

void* pool_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  cudaMemPool_t pool = pool_for_current_device();
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
  if (e == cudaErrorMemoryAllocation) {
    // the pool keeps freed memory for reuse; a large request that its free pieces cannot
    // serve gets the memory back from the pool (after the stream's pending frees) and
    // is tried once more
    cudaGetLastError();
    SPD_CUDA(cudaStreamSynchronize(s));
    SPD_CUDA(cudaMemPoolTrimTo(pool, 0));
    e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    if (e == cudaErrorMemoryAllocation) {
      // the pool's address ranges are fragmented: a plain allocation, which pool_free
      // recognizes and returns with cudaFree
      cudaGetLastError();
      e = cudaMalloc(&p, bytes);
      if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        g_plain.insert(p);
      }
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? SPDHSS_ENOMEM : SPDHSS_ECUDA,
                std::string("device allocation of ") + std::to_string(bytes) + " bytes: " +
                    cudaGetErrorString(e));
  }
  return p;
}

size_t device_free_bytes(cudaStream_t s) {
  (void)s;
  cudaMemPool_t pool = pool_for_current_device();
  uint64_t reserved = 0, used = 0;
  SPD_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  SPD_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  size_t f = 0, t = 0;
  SPD_CUDA(cudaMemGetInfo(&f, &t));
  return f + (size_t)(reserved > used ? reserved - used : 0);
}

void pool_free(void* p, cudaStream_t s) {
  bool plain = false;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    plain = g_plain.erase(p) > 0;
  }
  if (plain) {   // the stream's work on it first, then the plain free
    cudaStreamSynchronize(s);
    cudaFree(p);
    return;
  }
  if (cudaFreeAsync(p, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
  }
}
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---- per-kernel-family timing with CUDA events on the launching stream ------------------
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
};
static std::mutex g_pm;
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
struct ProfAcc { int64_t launches = 0; double ms = 0, flops = 0, bytes = 0; };
static std::map<std::string, ProfAcc> g_acc;

static cudaEvent_t pool_event() {
  if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
  cudaEvent_t e;
  SPD_CUDA(cudaEventCreate(&e));
  return e;
}

static void prof_drain() {
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ProfAcc& a = g_acc[r.name];
      a.launches += 1;
      a.ms += ms;
      a.flops += r.flops;
      a.bytes += r.bytes;
    } else {
      cudaGetLastError();
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

bool prof_enabled() { return g_prof; }

int prof_begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_pm);
  if (g_recs.size() >= 200000) prof_drain();
  ProfRec r{name, pool_event(), pool_event(), 0.0, 0.0};
  SPD_CUDA(cudaEventRecord(r.a, s));
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_add_flops(int slot, double flops) {
  std::lock_guard<std::mutex> lk(g_pm);
  if (slot >= 0 && slot < (int)g_recs.size()) g_recs[slot].flops += flops;
}

void prof_end(int slot, cudaStream_t s, double flops, double bytes) {
  std::lock_guard<std::mutex> lk(g_pm);
  if (slot < 0 || slot >= (int)g_recs.size()) return;
  g_recs[slot].flops = flops;
  g_recs[slot].bytes = bytes;
  cudaEventRecord(g_recs[slot].b, s);
}

template <class F>
spdhss_status guarded(const char* where, F&& f) {
  try {
    f();
    return SPDHSS_OK;
  } catch (const Error& e) {
    set_last_error(std::string(where) + ": " + e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error(std::string(where) + ": host allocation failed");
    return SPDHSS_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(std::string(where) + ": " + e.what());
    return SPDHSS_ECUDA;
  }
}

}  // namespace spd

using namespace spd;

extern "C" {

const char* spdhss_last_error(void) { return g_last_error.c_str(); }
int64_t spdhss_launch_count(void) { return g_launches.load(); }
const char* spdhss_version(void) { return "spdhss-gb300 0.1 (sm_103a, fp64)"; }

void spdhss_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_pm);
  if (enable) {
    prof_drain();
    g_acc.clear();
  }
  g_prof = enable != 0;
}

int64_t spdhss_tuning_report(char* buf, int64_t len) {
  const std::string out = spd::tuning_report();
  if (buf && len > 0) {
    const int64_t k = std::min<int64_t>(len - 1, (int64_t)out.size());
    std::memcpy(buf, out.data(), (size_t)k);
    buf[k] = 0;
  }
  return (int64_t)out.size() + 1;
}

int64_t spdhss_profile_report(char* buf, int64_t len) {
  std::lock_guard<std::mutex> lk(g_pm);
  prof_drain();
  std::string out = "{";
  bool first = true;
  char tmp[256];
  for (const auto& kv : g_acc) {
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
                  first ? "" : ", ", kv.first.c_str(), (long long)kv.second.launches, kv.second.ms,
                  kv.second.flops, kv.second.bytes);
    out += tmp;
    first = false;
  }
  out += "}";
  if (buf && len > 0) {
    const size_t n = std::min<size_t>((size_t)len - 1, out.size());
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return (int64_t)out.size() + 1;
}

}  // extern "C"

namespace spd {
// the body of h2_build (also run per instance by spdhss_build_batched)
static std::unique_ptr<spdhss_h2_s> h2_build_one(const double* points, int64_t n, int dim,
                                                 spdhss_kernel_desc kernel, int leaf_size,
                                                 double tol, cudaStream_t s) {
  SPD_REQUIRE(points != nullptr, "points is NULL");
  SPD_REQUIRE(n >= 1 && n < (1LL << 38), "n out of range");
  SPD_REQUIRE(dim == 2 || dim == 3, "dim must be 2 or 3");
  SPD_REQUIRE(leaf_size >= 1, "leaf_size must be >= 1");
  SPD_REQUIRE(tol >= 0.0 && tol < 1.0, "tol must be in [0, 1)");
  SPD_REQUIRE(kernel.kind >= 0 && kernel.kind <= 4, "unknown kernel kind");
  SPD_REQUIRE(kernel.kind != SPDHSS_K_RPY || dim == 3, "the RPY kernel needs dim 3");
  SPD_REQUIRE(kernel.ell > 0.0, "kernel length scale must be > 0");
  SPD_REQUIRE(kernel.shift >= 0.0, "shift must be >= 0");
  std::unique_ptr<spdhss_h2_s> h(new spdhss_h2_s());
  h->kfn.kind = kernel.kind;
  h->kfn.inv_ell = 1.0 / kernel.ell;
  h->kfn.shift = kernel.shift;
  h->tol = tol;
  const double* dp = points;
  DevBuf<double> staged;
  if (!is_device_pointer(points)) {
    staged.alloc((size_t)n * dim);
    SPD_CUDA(cudaMemcpyAsync(staged.p, points, (size_t)n * dim * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    dp = staged.p;
  }
  h2_build_impl(h.get(), dp, n, dim, leaf_size, s);
  return h;
}
}  // namespace spd

extern "C" {

spdhss_status h2_build(const double* points, int64_t n, int dim, spdhss_kernel_desc kernel,
                       int leaf_size, double tol, void* stream, h2_handle* out) {
  return guarded("h2_build", [&] {
    StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    *out = h2_build_one(points, n, dim, kernel, leaf_size, tol, (cudaStream_t)stream).release();
  });
}

spdhss_status spdhss_kernel_eval(spdhss_kernel_desc kernel, const double* r2, double* out,
                                int64_t n, void* stream) {
  return guarded("spdhss_kernel_eval", [&] {
    SPD_REQUIRE(n >= 0, "n must be >= 0");
    SPD_REQUIRE(n == 0 || (r2 && out), "NULL argument");
    SPD_REQUIRE(kernel.kind >= 0 && kernel.kind <= 3, "scalar kernel kind expected");
    SPD_REQUIRE(kernel.ell > 0.0, "kernel length scale must be > 0");
    SPD_REQUIRE(n == 0 || (is_device_pointer(r2) && is_device_pointer(out)),
                "r2 and out must be device pointers");
    KernelFn k;
    k.kind = kernel.kind;
    k.inv_ell = 1.0 / kernel.ell;
    k.shift = 0.0;
    kernel_eval_launch(k, r2, out, n, (cudaStream_t)stream);
  });
}

spdhss_status h2_matmul(h2_handle h, const double* X, double* Y, int nrhs, int64_t ld,
                        void* stream) {
  return guarded("h2_matmul", [&] {
    StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(h && X && Y, "NULL argument");
    SPD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    SPD_REQUIRE(ld >= h->th.n, "ld must be >= n");
    cudaStream_t s = (cudaStream_t)stream;
    auto it = h->plans.find(nrhs);
    if (it == h->plans.end()) {
      std::unique_ptr<H2Plan> p(new H2Plan());
      h2_plan_build(h, *p, nrhs, 1, s);
      it = h->plans.emplace(nrhs, std::move(p)).first;
    }
    const H2Plan& p = *it->second;
    permute_to_sorted(X, ld, p.xs.p, h->th.n, nrhs, h->td.perm.p, s);
    h2_plan_run(h, p, s);
    permute_from_sorted(p.ys.p, Y, ld, h->th.n, nrhs, h->td.perm.p, s);
  });
}

spdhss_status h2_info(h2_handle h, int64_t* info) {
  return guarded("h2_info", [&] {
    SPD_REQUIRE(h && info, "NULL argument");
    const TreeHost& T = h->th;
    for (int k = 0; k < 16; ++k) info[k] = 0;
    info[0] = T.n;
    info[1] = T.dim;
    info[2] = T.nn();
    info[3] = T.D;
    info[4] = (int64_t)T.near_idx.size();
    info[5] = (int64_t)T.far_idx.size();
    info[6] = h->Ktot;
    info[7] = (int64_t)(h->basis.bytes() + h->coup.bytes());
    int64_t nearE = 0, coupE = 0, basE = 0;
    for (int64_t i = T.depth_off[T.D]; i < T.depth_off[T.D + 1]; ++i)
      for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e)
        nearE += T.size(i) * T.size(T.near_idx[e]);
    for (int64_t i = 0; i < T.nn(); ++i) {
      for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e)
        coupE += (int64_t)h->rank(i) * h->rank(T.far_idx[e]);
      basE += (int64_t)h->U_rows[i] * h->rank(i);
    }
    info[8] = nearE;
    info[9] = coupE;
    info[10] = basE;
    info[11] = h->max_rank;
  });
}

spdhss_status h2_export_tree(h2_handle h, int64_t* perm, int64_t* depth_off, int64_t* begin,
                             int64_t* end, int64_t* parent, int64_t* cell_lo, int64_t* cell_hi,
                             int64_t* near_off, int64_t* near_idx, int64_t* far_off,
                             int64_t* far_idx) {
  return guarded("h2_export_tree", [&] {
    SPD_REQUIRE(h != nullptr, "NULL handle");
    const TreeHost& T = h->th;
    auto cp = [](int64_t* dst, const std::vector<int64_t>& v) {
      if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(int64_t));
    };
    if (perm) {
      std::vector<int64_t> hp = h->td.perm.download(0);
      cp(perm, hp);
    }
    cp(depth_off, T.depth_off);
    cp(begin, T.begin);
    cp(end, T.end);
    cp(parent, T.parent);
    cp(cell_lo, T.cell_lo);
    if (cell_hi) {
      std::vector<int64_t> hi(T.cell_lo.size());
      for (int64_t i = 0; i < T.nn(); ++i)
        for (int a = 0; a < T.dim; ++a) hi[i * T.dim + a] = T.cell_lo[i * T.dim + a] + T.width[i];
      cp(cell_hi, hi);
    }
    cp(near_off, T.near_off);
    cp(near_idx, T.near_idx);
    cp(far_off, T.far_off);
    cp(far_idx, T.far_idx);
  });
}

spdhss_status h2_export_skeletons(h2_handle h, int64_t* skel_off, int64_t* skel_idx) {
  return guarded("h2_export_skeletons", [&] {
    SPD_REQUIRE(h != nullptr, "NULL handle");
    if (skel_off) std::memcpy(skel_off, h->skel_off.data(), h->skel_off.size() * sizeof(int64_t));
    if (skel_idx && !h->skel_idx.empty())
      std::memcpy(skel_idx, h->skel_idx.data(), h->skel_idx.size() * sizeof(int64_t));
  });
}

spdhss_status h2_destroy(h2_handle h) {
  return guarded("h2_destroy", [&] { delete h; });
}

}  // extern "C"

// ---- SPD HSS -------------------------------------------------------------------------
#include "spdhss.cuh"

extern "C" {

spdhss_status spdhss_build_precision(h2_handle h2, int rank, double tol, int oversample,
                                     const double* omega, uint64_t seed, int precision,
                                     void* stream, hss_handle* out) {
  return spd::guarded("spdhss_build", [&] {
    SPD_REQUIRE(tol >= 0.0 && tol < 1.0, "tol must be in [0, 1)");
    SPD_REQUIRE(precision >= 0 && precision <= 2, "precision must be 0, 1 or 2");
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    SPD_REQUIRE(h2 != nullptr, "NULL H2 handle");
    SPD_REQUIRE(rank >= 0, "rank must be >= 0");
    SPD_REQUIRE(oversample >= 0, "oversample must be >= 0");
    SPD_REQUIRE(omega == nullptr || spd::is_device_pointer(omega), "omega must be a device pointer");
    if (tol <= 0.0) {
      std::unique_ptr<spdhss_hss_s> hs(new spdhss_hss_s());
      spd::spdhss_build_impl(hs.get(), h2, rank, oversample, omega, seed, (cudaStream_t)stream, tol,
                             precision);
      *out = hs.release();
      return;
    }
    // growing sketch: an attempt with cap r uses the first r + oversample sketch columns;
    // the cap doubles from 64 until every rank is below it or it reaches `rank`
    int r = std::min(rank, 64);
    while (true) {
      std::unique_ptr<spdhss_hss_s> hs(new spdhss_hss_s());
      spd::spdhss_build_impl(hs.get(), h2, r, oversample, omega, seed, (cudaStream_t)stream, tol,
                             precision);
      int mr = 0;
      for (int v : hs->rk) mr = std::max(mr, v);
      if (mr < r || r >= rank) {
        *out = hs.release();
        return;
      }
      r = std::min(2 * r, rank);
    }
  });
}

spdhss_status spdhss_build_tol(h2_handle h2, int rank, double tol, int oversample,
                               const double* omega, uint64_t seed, void* stream,
                               hss_handle* out) {
  return spdhss_build_precision(h2, rank, tol, oversample, omega, seed, 0, stream, out);
}

spdhss_status spdhss_build(h2_handle h2, int rank, int oversample, const double* omega,
                           uint64_t seed, void* stream, hss_handle* out) {
  return spdhss_build_precision(h2, rank, 0.0, oversample, omega, seed, 0, stream, out);
}

spdhss_status hss_matmul(hss_handle hs, const double* X, double* Y, int nrhs, int64_t ld,
                         void* stream) {
  return spd::guarded("hss_matmul", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(hs && X && Y, "NULL argument");
    SPD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    SPD_REQUIRE(ld >= hs->h2->th.n, "ld must be >= n");
    spd::hss_matmul_impl(hs, X, Y, nrhs, ld, (cudaStream_t)stream);
  });
}

spdhss_status hss_info(hss_handle hs, int64_t* info) {
  return spd::guarded("hss_info", [&] {
    SPD_REQUIRE(hs && info, "NULL argument");
    for (int k = 0; k < 8; ++k) info[k] = 0;
    info[0] = hs->L;
    int mr = 0;
    for (int v : hs->rk) mr = std::max(mr, v);
    info[1] = mr;
    info[2] = (int64_t)hs->stored_bytes();
    info[3] = (int64_t)hs->rk.size();
  });
}

spdhss_status hss_destroy(hss_handle hs) {
  return spd::guarded("hss_destroy", [&] { delete hs; });
}

}  // extern "C"

// ---- ULV and PCG ---------------------------------------------------------------------
#include "ulv.cuh"

namespace spd {
void pcg_impl(const spdhss_h2_s* h2, spdhss_ulv_s* u, const double* B, double* X, int nrhs,
              int64_t ld, double tol, int maxit, int* iters_out, double* relres_out,
              bool& converged, cudaStream_t s, int precision = 0, int refresh = 50);
void h2_matmul_mixed_impl(spdhss_h2_s* h2, const double* X, double* Y, int nrhs, int64_t ld,
                          cudaStream_t s);
void pcg_batched_impl(int count, spdhss_h2_s* const* h2, spdhss_ulv_s* const* ulv,
                      const double* const* B, double* const* X, const int* nrhs,
                      const int64_t* ld, double tol, int maxit, int* const* iters_out,
                      double* const* relres_out, spdhss_status* status, cudaStream_t s,
                      int precision, spdhss_done_fn on_done, void* user);
}

extern "C" {

spdhss_status ulv_factor(hss_handle hs, void* stream, ulv_handle* out) {
  return spd::guarded("ulv_factor", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    SPD_REQUIRE(hs != nullptr, "NULL HSS handle");
    std::unique_ptr<spdhss_ulv_s> u(new spdhss_ulv_s());
    spd::ulv_factor_impl(u.get(), hs, (cudaStream_t)stream);
    *out = u.release();
  });
}

spdhss_status ulv_solve(ulv_handle u, const double* B, double* X, int nrhs, int64_t ld,
                        void* stream) {
  return spd::guarded("ulv_solve", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(u && B && X, "NULL argument");
    SPD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    const int64_t n = u->hs->h2->th.n;
    SPD_REQUIRE(ld >= n, "ld must be >= n");
    cudaStream_t s = (cudaStream_t)stream;
    spd::UlvPlan& P = spd::ulv_plan(u, nrhs, s);
    const int64_t* perm = u->hs->h2->td.perm.p;
    spd::permute_to_sorted(B, ld, P.bw[0].p, n, nrhs, perm, s);
    spd::ulv_solve_sorted(u, P, s);
    spd::permute_from_sorted(P.bw[0].p, X, ld, n, nrhs, perm, s);
  });
}

spdhss_status ulv_destroy(ulv_handle u) {
  return spd::guarded("ulv_destroy", [&] { delete u; });
}

spdhss_status pcg_solve(h2_handle h2, ulv_handle u, const double* B, double* X, int nrhs,
                        int64_t ld, double relres_tol, int maxit, int* iters_out,
                        double* relres_out, void* stream) {
  spdhss_status st = spd::guarded("pcg_solve", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(h2 && B && X, "NULL argument");
    SPD_REQUIRE(!u || u->hs->h2 == h2, "the ULV factorization belongs to another H2 matrix");
    SPD_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    SPD_REQUIRE(ld >= h2->th.n, "ld must be >= n");
    SPD_REQUIRE(relres_tol > 0.0, "relres_tol must be > 0");
    SPD_REQUIRE(maxit >= 1, "maxit must be >= 1");
    bool conv = false;
    spd::pcg_impl(h2, u, B, X, nrhs, ld, relres_tol, maxit, iters_out, relres_out, conv,
                  (cudaStream_t)stream);
    if (!conv) throw spd::Error(SPDHSS_NO_CONVERGENCE, "some column missed the tolerance");
  });
  return st;
}

}  // extern "C"

extern "C" {

spdhss_status h2_matmul_mixed(h2_handle h, const double* X, double* Y, int nrhs, int64_t ld,
                              void* stream) {
  return spd::guarded("h2_matmul_mixed", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(h && X && Y, "NULL argument");
    SPD_REQUIRE(nrhs >= 1 && nrhs <= 16, "nrhs must be in [1, 16]");
    SPD_REQUIRE(ld >= h->th.n, "ld must be >= n");
    spd::h2_matmul_mixed_impl(h, X, Y, nrhs, ld, (cudaStream_t)stream);
  });
}

spdhss_status pcg_solve_mixed(h2_handle h2, ulv_handle u, const double* B, double* X, int nrhs,
                              int64_t ld, double relres_tol, int maxit, int* iters_out,
                              double* relres_out, void* stream) {
  return spd::guarded("pcg_solve_mixed", [&] {
    spd::StreamScope ss((cudaStream_t)stream);
    SPD_REQUIRE(h2 && B && X, "NULL argument");
    SPD_REQUIRE(!u || u->hs->h2 == h2, "the ULV factorization belongs to another H2 matrix");
    SPD_REQUIRE(nrhs >= 1 && nrhs <= 16, "nrhs must be in [1, 16]");
    SPD_REQUIRE(ld >= h2->th.n, "ld must be >= n");
    SPD_REQUIRE(relres_tol > 0.0, "relres_tol must be > 0");
    SPD_REQUIRE(maxit >= 1, "maxit must be >= 1");
    bool conv = false;
    spd::pcg_impl(h2, u, B, X, nrhs, ld, relres_tol, maxit, iters_out, relres_out, conv,
                  (cudaStream_t)stream, 1, 50);
    if (!conv) throw spd::Error(SPDHSS_NO_CONVERGENCE, "some column missed the tolerance");
  });
}

}  // extern "C"

// ---- batched level sweep ---------------------------------------------------------------

namespace spd {

static thread_local int64_t g_batched_stats[2] = {0, 0};

// Runs f(i) for every instance on a host thread of its own, all on stream s, with the
// batched launches of all instances merged (merge.cuh).  Collects each instance's status
// and error message.
template <class F>
static void run_batched(int count, cudaStream_t s, std::vector<spdhss_status>& st,
                        std::vector<std::string>& msg, F f) {
  Merger M(s, count);
  st.assign(count, SPDHSS_OK);
  msg.assign(count, std::string());
  int dev = 0;
  SPD_CUDA(cudaGetDevice(&dev));
  std::vector<std::thread> th;
  th.reserve(count);
  for (int i = 0; i < count; ++i) {
    th.emplace_back([&, i] {
      MergeCtx& c = merge_ctx();
      st[i] = guarded("instance", [&] {
        SPD_CUDA(cudaSetDevice(dev));
        c.m = &M;
        c.instance = i;
        c.bypass = false;
        StreamScope ss(s);
        f(i);
      });
      if (st[i] != SPDHSS_OK) msg[i] = g_last_error;
      c.m = nullptr;
      M.leave();
    });
  }
  for (auto& t : th) t.join();
  g_batched_stats[0] = M.launches();
  g_batched_stats[1] = M.submissions();
}

static spdhss_status batched_result(const char* where, const std::vector<spdhss_status>& st,
                                    const std::vector<std::string>& msg, spdhss_status* status) {
  if (status)
    for (size_t i = 0; i < st.size(); ++i) status[i] = st[i];
  for (size_t i = 0; i < st.size(); ++i)
    if (st[i] != SPDHSS_OK) {
      set_last_error(std::string(where) + ": instance " + std::to_string(i) + ": " + msg[i]);
      return st[i];
    }
  return SPDHSS_OK;
}

}  // namespace spd

extern "C" {

spdhss_status spdhss_build_batched(int count, const double* const* points, const int64_t* n,
                                   const int* dim, const spdhss_kernel_desc* kernel,
                                   const int* leaf_size, const double* tol, const int* rank,
                                   const int* oversample, const uint64_t* seed,
                                   const double* const* omega, const int* precision,
                                   void* stream,
                                   h2_handle* h2_out, hss_handle* hss_out, ulv_handle* ulv_out,
                                   spdhss_status* status) {
  std::vector<spdhss_status> st;
  std::vector<std::string> msg;
  cudaStream_t s = (cudaStream_t)stream;
  const spdhss_status outer = guarded("spdhss_build_batched", [&] {
    SPD_REQUIRE(count >= 1, "count must be >= 1");
    SPD_REQUIRE(points && n && dim && kernel && leaf_size && tol && rank && oversample && seed,
                "NULL argument");
    SPD_REQUIRE(h2_out && hss_out && ulv_out, "NULL output array");
    for (int i = 0; i < count; ++i) {
      h2_out[i] = nullptr;
      hss_out[i] = nullptr;
      ulv_out[i] = nullptr;
    }
    run_batched(count, s, st, msg, [&](int i) {
      SPD_REQUIRE(rank[i] >= 1, "rank must be >= 1");
      SPD_REQUIRE(oversample[i] >= 0, "oversample must be >= 0");
      std::unique_ptr<spdhss_h2_s> h =
          h2_build_one(points[i], n[i], dim[i], kernel[i], leaf_size[i], tol[i], s);
      std::unique_ptr<spdhss_hss_s> hs(new spdhss_hss_s());
      const int prec = precision ? precision[i] : 0;
      SPD_REQUIRE(prec >= 0 && prec <= 2, "precision must be 0, 1 or 2");
      spdhss_build_impl(hs.get(), h.get(), rank[i], oversample[i], omega ? omega[i] : nullptr,
                        seed[i], s, 0.0, prec);
      std::unique_ptr<spdhss_ulv_s> u(new spdhss_ulv_s());
      ulv_factor_impl(u.get(), hs.get(), s);
      ulv_out[i] = u.release();
      hss_out[i] = hs.release();
      h2_out[i] = h.release();
    });
  });
  if (outer != SPDHSS_OK) return outer;
  return batched_result("spdhss_build_batched", st, msg, status);
}

// pcg_solve_batched and pcg_solve_batched_mixed (precision 1: FP32 products)
static spdhss_status pcg_batched_entry(const char* where, int precision, int count,
                                       const h2_handle* h2, const ulv_handle* ulv,
                                       const double* const* B, double* const* X,
                                       const int* nrhs, const int64_t* ld, double relres_tol,
                                       int maxit, int* const* iters_out,
                                       double* const* relres_out, void* stream,
                                       spdhss_status* status, spdhss_done_fn on_done = nullptr,
                                       void* user = nullptr) {
  std::vector<spdhss_status> st;
  std::vector<std::string> msg;
  cudaStream_t s = (cudaStream_t)stream;
  const spdhss_status outer = guarded(where, [&] {
    SPD_REQUIRE(count >= 1, "count must be >= 1");
    SPD_REQUIRE(h2 && ulv && B && X && nrhs && ld, "NULL argument");
    SPD_REQUIRE(relres_tol > 0.0, "relres_tol must be > 0");
    SPD_REQUIRE(maxit >= 1, "maxit must be >= 1");
    StreamScope ss(s);
    st.assign(count, SPDHSS_OK);
    msg.assign(count, std::string());
    for (int i = 0; i < count; ++i) {
      SPD_REQUIRE(h2[i] && ulv[i] && B[i] && X[i], "NULL argument");
      SPD_REQUIRE(ulv[i]->hs->h2 == h2[i], "the ULV factorization belongs to another H2 matrix");
      SPD_REQUIRE(nrhs[i] >= 1, "nrhs must be >= 1");
      SPD_REQUIRE(!precision || nrhs[i] <= 16, "nrhs must be in [1, 16]");
      SPD_REQUIRE(ld[i] >= h2[i]->th.n, "ld must be >= n");
    }
    std::vector<spdhss_h2_s*> hv(h2, h2 + count);
    std::vector<spdhss_ulv_s*> uv(ulv, ulv + count);
    pcg_batched_impl(count, hv.data(), uv.data(), B, X, nrhs, ld, relres_tol, maxit, iters_out,
                     relres_out, st.data(), s, precision, on_done, user);
    for (int i = 0; i < count; ++i)
      if (st[i] == SPDHSS_NO_CONVERGENCE) msg[i] = "some column missed the tolerance";
  });
  if (outer != SPDHSS_OK) return outer;
  return batched_result(where, st, msg, status);
}

spdhss_status pcg_solve_batched(int count, const h2_handle* h2, const ulv_handle* ulv,
                                const double* const* B, double* const* X, const int* nrhs,
                                const int64_t* ld, double relres_tol, int maxit,
                                int* const* iters_out, double* const* relres_out, void* stream,
                                spdhss_status* status) {
  return pcg_batched_entry("pcg_solve_batched", 0, count, h2, ulv, B, X, nrhs, ld, relres_tol,
                           maxit, iters_out, relres_out, stream, status);
}

spdhss_status pcg_solve_batched_mixed(int count, const h2_handle* h2, const ulv_handle* ulv,
                                      const double* const* B, double* const* X,
                                      const int* nrhs, const int64_t* ld, double relres_tol,
                                      int maxit, int* const* iters_out,
                                      double* const* relres_out, void* stream,
                                      spdhss_status* status) {
  return pcg_batched_entry("pcg_solve_batched_mixed", 1, count, h2, ulv, B, X, nrhs, ld,
                           relres_tol, maxit, iters_out, relres_out, stream, status);
}

spdhss_status pcg_solve_batched_ex(int count, const h2_handle* h2, const ulv_handle* ulv,
                                   const double* const* B, double* const* X, const int* nrhs,
                                   const int64_t* ld, double relres_tol, int maxit,
                                   int* const* iters_out, double* const* relres_out,
                                   void* stream, spdhss_status* status, int precision,
                                   spdhss_done_fn on_done, void* user) {
  if (precision != 0 && precision != 1) {
    set_last_error("pcg_solve_batched_ex: precision must be 0 or 1");
    return SPDHSS_EINVAL;
  }
  return pcg_batched_entry("pcg_solve_batched_ex", precision, count, h2, ulv, B, X, nrhs, ld,
                           relres_tol, maxit, iters_out, relres_out, stream, status, on_done,
                           user);
}

void spdhss_batched_stats(int64_t* merged) {
  if (merged) {
    merged[0] = g_batched_stats[0];
    merged[1] = g_batched_stats[1];
  }
}

}  // extern "C"
