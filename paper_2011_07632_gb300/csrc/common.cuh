// Shared host/device helpers of the spdhss library: status errors, device buffers,
// launch accounting, the kernel functions of Sec. 6, and small launch utilities.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/spdhss.h"

namespace spd {

struct Error : std::runtime_error {
  spdhss_status code;
  Error(spdhss_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);
void count_launches(int64_t k = 1);

// Optional per-kernel-family timing: when enabled, every instrumented launch is bracketed
// by CUDA events on its stream; flops are the algorithmic FP64 operations of the launch.
bool prof_enabled();
int prof_begin(const char* name, cudaStream_t s);
void prof_end(int slot, cudaStream_t s, double flops, double bytes);
// add algorithmic flops to a finished record (work known only after the launch, e.g. a rank)
void prof_add_flops(int slot, double flops);
struct ProfScope {
  int slot;
  cudaStream_t s;
  double flops, bytes;
  ProfScope(const char* name, cudaStream_t st, double f = 0.0, double b = 0.0)
      : slot(prof_enabled() ? prof_begin(name, st) : -1), s(st), flops(f), bytes(b) {}
  ~ProfScope() {
    if (slot >= 0) prof_end(slot, s, flops, bytes);
  }
};

// Householder QR flops for k steps on an m x n matrix: per step, every trailing column
// takes a dot product and an update (4 flops per entry) and a recomputed norm (2 flops).
// Householder QR, k steps on m x n: per step the reflector (3 (m - j)) and its application
// to the n - j - 1 trailing columns (4 (m - j) each); column norms are downdated (O(n)).
inline double qr_flops(int64_t m, int64_t n, int64_t k, bool pivot) {
  (void)pivot;
  double f = 0.0;
  for (int64_t j = 0; j < k; ++j) f += (double)(m - j) * (4.0 * (double)(n - j - 1) + 3.0);
  return f;
}

#define SPD_CUDA(x)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      if (e_ == cudaErrorMemoryAllocation)                                                 \
        throw ::spd::Error(SPDHSS_ENOMEM, std::string(#x) + ": " + cudaGetErrorString(e_)); \
      throw ::spd::Error(SPDHSS_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));    \
    }                                                                                      \
  } while (0)

#define SPD_LAUNCHED()                   \
  do {                                   \
    ::spd::count_launches();             \
    SPD_CUDA(cudaGetLastError());        \
  } while (0)

#define SPD_REQUIRE(cond, msg)                                  \
  do {                                                          \
    if (!(cond)) throw ::spd::Error(SPDHSS_EINVAL, (msg));      \
  } while (0)

// The stream of the entry point running on this thread: device buffers are allocated and
// freed in stream order on it (a library memory pool per device), so that freeing a
// buffer neither synchronizes the device nor waits for other streams.
cudaStream_t& current_stream();
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s) : prev(current_stream()) { current_stream() = s; }
  ~StreamScope() { current_stream() = prev; }
};
void* pool_alloc(size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);
// device memory free, counting what the library pool holds unused
size_t device_free_bytes(cudaStream_t s);
// whether an optional copy of `bytes` fits with a margin for the work that follows
inline bool fits_on_device(size_t bytes, cudaStream_t s) {
  return bytes + ((size_t)16 << 30) <= device_free_bytes(s);
}

// Device allocation owned by its object, stream ordered on the stream current at allocation.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), st(o.st) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; st = o.st; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    st = current_stream();
    if (count) p = (T*)pool_alloc(count * sizeof(T), st);
  }
  void release() {
    if (p) pool_free(p, st);
    p = nullptr;
    n = 0;
  }
  void zero(cudaStream_t s) {
    if (n) SPD_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  void upload(const std::vector<T>& h, cudaStream_t s) {
    alloc(h.size());
    if (n) SPD_CUDA(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s) const {
    std::vector<T> h(n);
    if (n) {
      SPD_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
      SPD_CUDA(cudaStreamSynchronize(s));
    }
    return h;
  }
  size_t bytes() const { return n * sizeof(T); }
};

inline bool is_device_pointer(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- kernel functions (Sec. 6), length scale ell divides r ---------------------------
struct KernelFn {
  int kind;
  double inv_ell;   // 1/ell
  double shift;
};

// exp(x) for x <= 0 by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic", ACM TOMS
// 15(2), 1989), here with 64 table entries: x = (64 m + j) ln2/64 + r with |r| <= ln2/128,
// exp(x) = 2^m 2^(j/64) e^r, and e^r - 1 by its Taylor series through r^5 (the first
// omitted term is below 0.16 units in the last place).  ln2/64 is split into a 29-bit head,
// whose product with the integer 64 m + j is exact, and a tail; 2^m is applied to the
// exponent field (the result stays normal for x >= -700).  Arguments below -700 (and NaN)
// take exp().  Each table entry is 2^(j/64) rounded to the nearest double.
// EXP2_TABLE_BEGIN
__device__ const double kExp2By64[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0,
    0x1.0874518759bc8p+0, 0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0,
    0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0, 0x1.172b83c7d517bp+0,
    0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0,
    0x1.2d285a6e4030bp+0, 0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0,
    0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0, 0x1.3dea64c123422p+0,
    0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0,
    0x1.56f4736b527dap+0, 0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0,
    0x1.6247eb03a5585p+0, 0x1.6623882552225p+0, 0x1.6a09e667f3bcdp+0,
    0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0,
    0x1.868d99b4492edp+0, 0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0,
    0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0, 0x1.9c49182a3f090p+0,
    0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0,
    0x1.bcc1e904bc1d2p+0, 0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0,
    0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0, 0x1.d5818dcfba487p+0,
    0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0,
    0x1.fa7c1819e90d8p+0,
};
// EXP2_TABLE_END
__device__ __forceinline__ double exp_neg(double x) {
  if (!(x >= -700.0)) return exp(x);
  const double kInvStep = 0x1.71547652b82fep+6;    // 64 / ln2
  const double kStepHi = 0x1.62e42ff000000p-7;     // ln2/64, head
  const double kStepLo = -0x1.718432a1b0e26p-41;   // ln2/64 - head
  const double kShift = 0x1.8p52;                  // round-to-integer shifter
  const double t = fma(x, kInvStep, kShift);       // 64 m + j in the low word
  const int N = __double2loint(t);
  const double Nd = t - kShift;
  double r = fma(-Nd, kStepHi, x);
  r = fma(-Nd, kStepLo, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r * r, r);                            // e^r - 1
  const double T = __ldg(kExp2By64 + (N & 63));
  const double v = fma(T, p, T);
  return __hiloint2double(__double2hiint(v) + (N >> 6) * (1 << 20), __double2loint(v));
}

__device__ __forceinline__ double kernel_r2(const KernelFn& k, double r2) {
  switch (k.kind) {
    case SPDHSS_K_EXP:
      return exp_neg(-sqrt(r2) * k.inv_ell);
    case SPDHSS_K_GAUSS:
      return exp_neg(-r2 * (k.inv_ell * k.inv_ell));
    case SPDHSS_K_MATERN32: {
      double t = 1.7320508075688772 * sqrt(r2) * k.inv_ell;
      return (1.0 + t) * exp_neg(-t);
    }
    default:
      return 1.0 / sqrt(1.0 + r2 * (k.inv_ell * k.inv_ell));
  }
}

// The same kernel with its kind fixed at compile time (no per-entry branch).
template <int KIND>
__device__ __forceinline__ double kernel_r2_k(double r2, double inv_ell) {
  if (KIND == SPDHSS_K_EXP) return exp_neg(-sqrt(r2) * inv_ell);
  if (KIND == SPDHSS_K_GAUSS) return exp_neg(-r2 * (inv_ell * inv_ell));
  if (KIND == SPDHSS_K_MATERN32) {
    const double t = 1.7320508075688772 * sqrt(r2) * inv_ell;
    return (1.0 + t) * exp_neg(-t);
  }
  return 1.0 / sqrt(1.0 + r2 * (inv_ell * inv_ell));
}

// FP32 evaluation for the mixed-precision products.
template <int KIND>
__device__ __forceinline__ float kernel_r2_k(float r2, float inv_ell) {
  if (KIND == SPDHSS_K_EXP) return expf(-sqrtf(r2) * inv_ell);
  if (KIND == SPDHSS_K_GAUSS) return expf(-r2 * (inv_ell * inv_ell));
  if (KIND == SPDHSS_K_MATERN32) {
    const float t = 1.7320508f * sqrtf(r2) * inv_ell;
    return (1.0f + t) * expf(-t);
  }
  return rsqrtf(1.0f + r2 * (inv_ell * inv_ell));
}

// ---- the Rotne-Prager-Yamakawa tensor (Sec. 6), particle radius a ----------------------
// A vector-valued kernel: the matrix has 3 unknowns per point, and its entry for the
// unknowns (p, ci) and (q, cj) is the (ci, cj) entry of the 3 x 3 tensor K(x_p, x_q),
// r = x_p - x_q:
//   r = 0:        (1/a) I
//   |r| >= 2a:    3/(4|r|) (I + rr^T/|r|^2) + 3a^2/(2|r|^3) (I/3 - rr^T/|r|^2)
//   |r| <  2a:    (1/a) [ (1 - 9|r|/(32a)) I + 3|r|/(32a) rr^T/|r|^2 ]
// (the overlap branch with 1/a on both terms: the form continuous at |r| = 2a).  Such a
// handle stores each point three times in sorted order (unknown 3p + c is component c of
// point p) with one more coordinate row holding the component c.
constexpr int kRpyDofs = 3;
__host__ __device__ inline int kernel_dofs(int kind) { return kind == SPDHSS_K_RPY ? kRpyDofs : 1; }

template <class T>
__device__ __forceinline__ T rpy_entry(T d0, T d1, T d2, int ci, int cj, T inv_a) {
  const T r2 = d0 * d0 + d1 * d1 + d2 * d2;
  const T I = (ci == cj) ? T(1) : T(0);
  if (r2 == T(0)) return I * inv_a;
  const T di = ci == 0 ? d0 : (ci == 1 ? d1 : d2);
  const T dj = cj == 0 ? d0 : (cj == 1 ? d1 : d2);
  const T r = sqrt(r2);
  const T rr = di * dj / r2;
  const T a = T(1) / inv_a;
  if (r >= T(2) * a) {
    const T inv_r = T(1) / r;
    return T(0.75) * inv_r * (I + rr) +
           T(1.5) * a * a * (inv_r * inv_r * inv_r) * (I * T(1.0 / 3.0) - rr);
  }
  const T t = r * inv_a * T(1.0 / 32.0);
  return inv_a * ((T(1) - T(9) * t) * I + T(3) * t * rr);
}

// Points are stored structure-of-arrays: coordinate a of point p at x[a * ldx + p].
__device__ __forceinline__ double sqdist3(const double* __restrict__ x, int64_t ldx, int dim,
                                          int64_t p, double y0, double y1, double y2) {
  double d0 = x[p] - y0;
  double d1 = x[ldx + p] - y1;
  double r2 = d0 * d0 + d1 * d1;
  if (dim == 3) {
    double d2 = x[2 * ldx + p] - y2;
    r2 += d2 * d2;
  }
  return r2;
}

}  // namespace spd
