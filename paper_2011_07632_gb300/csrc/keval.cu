// Kernel-matrix evaluation kernels (see keval.cuh).
#include <algorithm>
#include <mutex>
#include <map>
#include <type_traits>

#include <cmath>

#include "keval.cuh"

namespace spd {

// ---------------------------------------------------------------------------------------
// dense tiles, 32 x 32 per CTA
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tiles(const TileProb* __restrict__ probs,
                                               const int4* __restrict__ work, KernelFn kf_,
                                               int dim_) {
  const int4 w = work[blockIdx.x];
  const TileProb P = probs[w.x];
  const KernelFn kf = P.dim ? P.kf : kf_;
  const int dim = P.dim ? P.dim : dim_;
  const int i0 = w.y, j0 = w.z;
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int i = i0 + (e & 31), j = j0 + (e >> 5);
    if (i >= P.rows || j >= P.cols) continue;
    const int64_t pr = P.r0 + i, pc = P.c0 + j;
    double v;
    if (kf.kind == SPDHSS_K_RPY) {
      // component rows: index dim (= 3) of both point arrays
      v = rpy_entry<double>(P.xr[pr] - P.xc[pc], P.xr[P.ldxr + pr] - P.xc[P.ldxc + pc],
                            P.xr[2 * P.ldxr + pr] - P.xc[2 * P.ldxc + pc],
                            (int)P.xr[3 * P.ldxr + pr], (int)P.xc[3 * P.ldxc + pc], kf.inv_ell);
    } else {
      double r2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double d = P.xr[a * P.ldxr + pr] - P.xc[a * P.ldxc + pc];
        r2 += d * d;
      }
      v = kernel_r2(kf, r2);
    }
    if (P.xr == P.xc && pr == pc) v += P.diag_add;
    P.out[i + (int64_t)j * P.ldo] = v;
  }
}

void tile_launch(const Batch<TileProb>& b, const KernelFn& k, int dim, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    std::vector<TileProb> h = b.h;
    for (auto& p : h)
      if (!p.dim) { p.kf = k; p.dim = dim; }
    defer_launch("tile", h, [](std::vector<TileProb>& all, cudaStream_t st) {
      Batch<TileProb> m;
      m.h = std::move(all);
      m.upload(st);
      tile_launch(m, KernelFn{}, 0, st);
    });
    return;
  }
  std::vector<int4> work;
  for (int p = 0; p < (int)b.size(); ++p)
    for (int i0 = 0; i0 < b.h[p].rows; i0 += 32)
      for (int j0 = 0; j0 < b.h[p].cols; j0 += 32) work.push_back(make_int4(p, i0, j0, 0));
  if (work.empty()) return;
  DevBuf<int4> dw;
  dw.upload(work, s);
  {
    ProfScope ps("tile", s);
    k_tiles<<<(unsigned)work.size(), 256, 0, s>>>(b.d.p, dw.p, k, dim);
    SPD_LAUNCHED();
  }
}

// ---------------------------------------------------------------------------------------
// proxy matrices K(P_i, X_cand): rows are proxy points (generated on the fly)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void proxy_point(const ProxyProb& P, int dim, int r, double* y) {
  const int q = proxy_grid(dim);
  const int per_face = (dim == 3) ? q * q : q;
  const int per_shell = 2 * dim * per_face;
  const int t = r / per_shell;
  int rem = r - t * per_shell;
  const int face = rem / per_face;
  rem -= face * per_face;
  const int a = face >> 1;
  const double sgn = (face & 1) ? 1.0 : -1.0;
  const double f = (double)t / (double)(PROXY_SHELLS - 1);
  const double ht = 3.0 * P.h + (P.H - 3.0 * P.h) * (f * f);
  int o0 = (a == 0) ? 1 : 0;
  int o1 = (a == 2) ? 1 : 2;
  if (dim == 3) {
    const int u = rem / q, v = rem % q;
    const double gu = -1.0 + (2.0 * u + 1.0) / q;
    const double gv = -1.0 + (2.0 * v + 1.0) / q;
    y[o0] = P.c[o0] + gu * ht;
    y[o1] = P.c[o1] + gv * ht;
  } else {
    o0 = 1 - a;
    const double gu = -1.0 + (2.0 * rem + 1.0) / q;
    y[o0] = P.c[o0] + gu * ht;
  }
  y[a] = P.c[a] + sgn * ht;
}

__global__ void __launch_bounds__(256) k_proxy(const ProxyProb* __restrict__ probs,
                                               const int4* __restrict__ work, KernelFn kf_,
                                               int dim_) {
  const int4 w = work[blockIdx.x];
  const ProxyProb P = probs[w.x];
  const KernelFn kf = P.dim ? P.kf : kf_;
  const int dim = P.dim ? P.dim : dim_;
  // a vector-valued kernel: row i is component i % kd of proxy point i / kd
  const int kd = kernel_dofs(kf.kind);
  const int np = proxy_count(dim) * kd;
  const int i0 = w.y, j0 = w.z;
  __shared__ double sy[3][64];
  if (threadIdx.x < 64 && i0 + threadIdx.x < np) {
    double y[3] = {0, 0, 0};
    proxy_point(P, dim, (i0 + threadIdx.x) / kd, y);
    for (int a = 0; a < 3; ++a) sy[a][threadIdx.x] = y[a];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int ii = e & 63, j = j0 + (e >> 6);
    const int i = i0 + ii;
    if (i >= np || j >= P.cols) continue;
    const int64_t pc = P.c0 + j;
    double v;
    if (kd > 1) {
      v = rpy_entry<double>(sy[0][ii] - P.xc[pc], sy[1][ii] - P.xc[P.ldxc + pc],
                            sy[2][ii] - P.xc[2 * P.ldxc + pc], i % kd,
                            (int)P.xc[3 * P.ldxc + pc], kf.inv_ell);
    } else {
      double r2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double d = sy[a][ii] - P.xc[a * P.ldxc + pc];
        r2 += d * d;
      }
      v = kernel_r2(kf, r2) * P.scale;
    }
    P.out[i + (int64_t)j * P.ldo] = v;
  }
}

double proxy_scale(const KernelFn& k, double h) {
  if (k.kind == SPDHSS_K_RPY) return 1.0;
  const double t = 2.0 * h * k.inv_ell;
  double kb;
  switch (k.kind) {
    case SPDHSS_K_EXP: kb = std::exp(-t); break;
    case SPDHSS_K_GAUSS: kb = std::exp(-t * t); break;
    case SPDHSS_K_MATERN32: {
      const double u = 1.7320508075688772 * t;
      kb = (1.0 + u) * std::exp(-u);
      break;
    }
    default: kb = 1.0 / std::sqrt(1.0 + t * t);
  }
  if (!(kb > 0.0) || kb >= 0x1p-200) return 1.0;
  int e = 0;
  std::frexp(kb, &e);   // kb = f 2^e, f in [1/2, 1)
  return std::ldexp(1.0, std::min(-e, 1000));
}

template <int KIND>
__global__ void k_kernel_eval(const double* __restrict__ r2, double* __restrict__ out, int64_t n,
                              double inv_ell) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = kernel_r2_k<KIND>(r2[i], inv_ell);
}

void kernel_eval_launch(const KernelFn& k, const double* r2, double* out, int64_t n,
                        cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16);
  switch (k.kind) {
    case SPDHSS_K_EXP: k_kernel_eval<SPDHSS_K_EXP><<<g, 256, 0, s>>>(r2, out, n, k.inv_ell); break;
    case SPDHSS_K_GAUSS: k_kernel_eval<SPDHSS_K_GAUSS><<<g, 256, 0, s>>>(r2, out, n, k.inv_ell); break;
    case SPDHSS_K_MATERN32:
      k_kernel_eval<SPDHSS_K_MATERN32><<<g, 256, 0, s>>>(r2, out, n, k.inv_ell);
      break;
    default: k_kernel_eval<SPDHSS_K_IMQ><<<g, 256, 0, s>>>(r2, out, n, k.inv_ell); break;
  }
  SPD_LAUNCHED();
}

void proxy_launch(const Batch<ProxyProb>& b, const KernelFn& k, int dim, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    std::vector<ProxyProb> h = b.h;
    for (auto& p : h)
      if (!p.dim) { p.kf = k; p.dim = dim; }
    defer_launch("proxy", h, [](std::vector<ProxyProb>& all, cudaStream_t st) {
      Batch<ProxyProb> m;
      m.h = std::move(all);
      m.upload(st);
      proxy_launch(m, KernelFn{}, 0, st);
    });
    return;
  }
  std::vector<int4> work;
  for (int p = 0; p < (int)b.size(); ++p)
    for (int i0 = 0, np = proxy_count(b.h[p].dim ? b.h[p].dim : dim) *
                          kernel_dofs(b.h[p].dim ? b.h[p].kf.kind : k.kind);
         i0 < np; i0 += 64)
      for (int j0 = 0; j0 < b.h[p].cols; j0 += 32) work.push_back(make_int4(p, i0, j0, 0));
  if (work.empty()) return;
  DevBuf<int4> dw;
  dw.upload(work, s);
  {
    ProfScope ps("proxy", s);
    k_proxy<<<(unsigned)work.size(), 256, 0, s>>>(b.d.p, dw.p, k, dim);
    SPD_LAUNCHED();
  }
}

// ---------------------------------------------------------------------------------------
// Row blocks of the proxy matrices, factored where they are evaluated (the first step of
// the ID's QR).  CTA b evaluates its rows of K(P_i, X_cand) into shared memory (the same
// entries as k_proxy) and reduces them by Householder reflections without pivoting to an
// upper triangle R_b.  Only R is kept: the reflector of column j is u = x - beta e_1 with
// x = A(j:, j), beta = -sign(x_0) |x|, applied as A <- A - c u (u^T A) with
// c = -1 / (beta (x_0 - beta)) (= 2 / u^T u), so the reflectors are never normalized.
// Every column has a group of lanes (col_group_lanes); the group of column j + 1 forms the
// next reflector's scalars right after its own update (look-ahead), so a step costs one
// barrier.  Stacking the R_b of all blocks and reducing them (k_tri_merge) gives the R
// factor of the whole proxy matrix (TSQR), from which the column-pivoted QR chooses the
// ID's skeleton: pivots and |R_kk| depend on the matrix M only through M^T M, which R
// shares.
// ---------------------------------------------------------------------------------------
// one proxy row against the m candidate columns: col[j * ld] = K(y, x_(c0 + j))
template <int KIND>
__device__ __forceinline__ void proxy_row(double* col, int ld, const double* y,
                                          const double* __restrict__ xc, int64_t ldxc,
                                          int64_t c0, int m, int dim, double inv_ell,
                                          double scale) {
  for (int j = 0; j < m; ++j) {
    const int64_t pc = c0 + j;
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double d = y[a] - xc[a * ldxc + pc];
      r2 += d * d;
    }
    col[(int64_t)j * ld] = kernel_r2_k<KIND>(r2, inv_ell) * scale;
  }
}

__global__ void __launch_bounds__(256) k_proxy_qr(const ProxyQrProb* __restrict__ probs,
                                                  KernelFn kf_, int dim_) {
  const ProxyQrProb Q = probs[blockIdx.x];
  const ProxyProb& P = Q.p;
  const KernelFn kf = P.dim ? P.kf : kf_;
  const int dim = P.dim ? P.dim : dim_;
  const int kd = kernel_dofs(kf.kind);
  extern __shared__ double sA[];            // rows x m, column-major, ld col_group_ld
  __shared__ double s_diag[kIdTsqrMaxM];    // R_jj
  __shared__ double s_c[2];                 // reflector coefficient of steps j, j + 1
  const int rows = Q.rows, m = P.cols;
  const int lanes = col_group_lanes(m), ld = col_group_ld(rows, lanes);
  const int tid = threadIdx.x, warp = tid >> 5;
  // evaluation: one proxy point per thread and row, every candidate column (the
  // descriptor's fields in registers, the kernel kind dispatched once per row)
  {
    const double* __restrict__ xc = P.xc;
    const int64_t ldxc = P.ldxc, c0 = P.c0;
    const int r0 = Q.r0;
    for (int i = tid; i < rows; i += blockDim.x) {
      const int r = r0 + i;
      double y[3] = {0, 0, 0};
      proxy_point(P, dim, r / kd, y);
      double* col = sA + i;
      switch (kd > 1 ? -1 : kf.kind) {
        case SPDHSS_K_EXP: proxy_row<SPDHSS_K_EXP>(col, ld, y, xc, ldxc, c0, m, dim, kf.inv_ell, P.scale); break;
        case SPDHSS_K_GAUSS: proxy_row<SPDHSS_K_GAUSS>(col, ld, y, xc, ldxc, c0, m, dim, kf.inv_ell, P.scale); break;
        case SPDHSS_K_MATERN32:
          proxy_row<SPDHSS_K_MATERN32>(col, ld, y, xc, ldxc, c0, m, dim, kf.inv_ell, P.scale);
          break;
        case SPDHSS_K_IMQ: proxy_row<SPDHSS_K_IMQ>(col, ld, y, xc, ldxc, c0, m, dim, kf.inv_ell, P.scale); break;
        default:
          for (int j = 0; j < m; ++j) {
            const int64_t pc = c0 + j;
            col[(int64_t)j * ld] =
                rpy_entry<double>(y[0] - xc[pc], y[1] - xc[ldxc + pc], y[2] - xc[2 * ldxc + pc],
                                  r % kd, (int)xc[3 * ldxc + pc], kf.inv_ell);
          }
      }
    }
  }
  __syncthreads();
  const int g = tid / lanes, sl = tid % lanes;     // column g, lane sl of its group
  const int gpw = 32 / lanes;                      // groups per warp
  const int g_lo = warp * gpw, g_hi = g_lo + gpw - 1;
  // the first reflector, by the warp of column 0
  if (warp == 0) {
    double sq = 0.0;
    if (g == 0)
      for (int i = sl; i < rows; i += lanes) sq += sA[i] * sA[i];
    sq = group_sum_n(sq, lanes);
    if (tid == 0) s_c[0] = hh_scalars(&sA[0], sq, &s_diag[0]);
  }
  __syncthreads();
  const int steps = min(rows, m);
  for (int j = 0; j < steps; ++j) {
    // warps without a column > j skip the step (warp-uniform)
    if (g_hi > j && g_lo < m) {
      const double c = s_c[j & 1];
      const double* u = sA + (int64_t)j * ld + j;   // u over rows j..rows-1
      const int len = rows - j;
      const bool act = g > j && g < m;
      double* ap = sA + (int64_t)(act ? g : j) * ld + j;
      double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
      if (act && c != 0.0) {
        int i = sl;
        for (; i + 3 * lanes < len; i += 4 * lanes) {   // four independent loads per lane
          w0 = fma(u[i], ap[i], w0);
          w1 = fma(u[i + lanes], ap[i + lanes], w1);
          w2 = fma(u[i + 2 * lanes], ap[i + 2 * lanes], w2);
          w3 = fma(u[i + 3 * lanes], ap[i + 3 * lanes], w3);
        }
        for (; i < len; i += lanes) w0 = fma(u[i], ap[i], w0);
      }
      const double w = group_sum_n((w0 + w1) + (w2 + w3), lanes) * c;
      const bool next = g == j + 1;   // update, and the next reflector's norm
      double sq = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;   // independent partial sums
      if (act && (c != 0.0 || next)) {
        // the column and u are disjoint: loads of four rows before their stores
        int i = sl;
        for (; i + 3 * lanes < len; i += 4 * lanes) {
          const double a0 = ap[i], a1 = ap[i + lanes], a2 = ap[i + 2 * lanes], a3 = ap[i + 3 * lanes];
          const double v0 = u[i], v1 = u[i + lanes], v2 = u[i + 2 * lanes], v3 = u[i + 3 * lanes];
          const double b0 = a0 - w * v0, b1 = a1 - w * v1, b2 = a2 - w * v2, b3 = a3 - w * v3;
          ap[i] = b0; ap[i + lanes] = b1; ap[i + 2 * lanes] = b2; ap[i + 3 * lanes] = b3;
          if (next) {
            q1 = fma(b1, b1, q1);
            q2 = fma(b2, b2, q2);
            q3 = fma(b3, b3, q3);
            if (i > 0) sq = fma(b0, b0, sq);
          }
        }
        for (; i < len; i += lanes) {
          const double b = ap[i] - w * u[i];
          ap[i] = b;
          if (next && i > 0) sq = fma(b, b, sq);
        }
        sq = (sq + q1) + (q2 + q3);
      }
      if (g_lo <= j + 1 && j + 1 <= g_hi && j + 1 < steps) {   // the warp of column j + 1
        sq = group_sum_n(sq, lanes);
        __syncwarp();   // the group's updated rows, visible to its lane 0
        if (g == j + 1 && sl == 0) s_c[(j + 1) & 1] = hh_scalars(ap + 1, sq, &s_diag[j + 1]);
      }
    }
    __syncthreads();
  }
  // R_b, dense m x m with zeros below the diagonal (and in the rows a short block lacks)
  double* R = P.out;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, p = e / m;
    double v = 0.0;
    if (i < steps) v = (i == p) ? s_diag[i] : (i < p ? sA[i + (int64_t)p * ld] : 0.0);
    R[i + (int64_t)p * P.ldo] = v;
  }
}

void proxy_qr_launch(const Batch<ProxyQrProb>& b, const KernelFn& k, int dim, const char* tag,
                     cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    std::vector<ProxyQrProb> h = b.h;
    for (auto& q : h)
      if (!q.p.dim) { q.p.kf = k; q.p.dim = dim; }
    defer_launch("proxy_qr", h, [tag](std::vector<ProxyQrProb>& all, cudaStream_t st) {
      Batch<ProxyQrProb> m;
      m.h = std::move(all);
      m.upload(st);
      proxy_qr_launch(m, KernelFn{}, 0, tag, st);
    });
    return;
  }
  size_t smem = 0;
  double f = 0.0;
  for (const auto& q : b.h) {
    SPD_REQUIRE(q.p.cols <= kIdTsqrMaxM && q.rows >= 1, "proxy_qr: block too large");
    smem = std::max(smem, (size_t)col_group_ld(q.rows, col_group_lanes(q.p.cols)) * q.p.cols *
                              sizeof(double));
    const double mm = q.p.cols, r = q.rows;
    // Householder QR of a rows x m block: 2 m^2 (rows - m/3) flops (rows >= m)
    f += r >= mm ? 2.0 * mm * mm * (r - mm / 3.0) : 2.0 * r * r * (mm - r / 3.0);
  }
  // dynamic shared memory: the 227 KB of a CTA less the kernel's static arrays
  constexpr int kDyn = 227 * 1024 - 4096;
  SPD_REQUIRE(smem <= (size_t)kDyn, "proxy_qr: block exceeds shared memory");
  static std::once_flag once;
  std::call_once(once, [] {
    SPD_CUDA(cudaFuncSetAttribute(k_proxy_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn));
  });
  ProfScope ps(tag ? tag : "proxy_qr", s, f);
  k_proxy_qr<<<(unsigned)b.size(), 256, smem, s>>>(b.d.p, k, dim);
  SPD_LAUNCHED();
}

// ---------------------------------------------------------------------------------------
// near field with few columns (NC <= 16): one thread per target row; when a leaf has fewer
// than 256 points, G = 256 / rows groups of threads split the source points between them
// and a fixed-order sum in shared memory combines the groups.  Every kernel entry is
// evaluated exactly once per column block, and no FMA is spent on padding.
// ---------------------------------------------------------------------------------------
template <class T, int NC, int KIND>
__global__ void __launch_bounds__(256) k_near_small(const NearProbT<T>* __restrict__ probs,
                                                    const NearSegT<T>* __restrict__ segs,
                                                    const int2* __restrict__ work, KernelFn kf_,
                                                    const double* __restrict__ xs_, int64_t ldx_,
                                                    int dim_) {
  // source points staged per chunk; the staging area is reused for the final reduction
  constexpr int CH = NC >= 16 ? 192 : (NC >= 8 ? 256 : 512);
  constexpr bool RPY = KIND == SPDHSS_K_RPY;
  constexpr int NX = RPY ? 4 : 3;   // staged coordinate rows (+ the component row)
  constexpr int STAGE = CH * (NX + NC);
  constexpr int RED = NC * 256;
  __shared__ T smem[STAGE > RED ? STAGE : RED];
  T (*red)[256] = reinterpret_cast<T (*)[256]>(smem);
  T (*sx)[CH] = reinterpret_cast<T (*)[CH]>(smem);
  T (*sv)[CH] = reinterpret_cast<T (*)[CH]>(smem + NX * CH);
  const int2 w = work[blockIdx.x];
  const NearProbT<T> P = probs[w.x];
  const bool own = P.xs != nullptr;
  const double* __restrict__ xs = own ? P.xs : xs_;
  const int64_t ldx = own ? P.ldx : ldx_;
  const int dim = own ? P.dim : dim_;
  KernelFn kf = kf_;
  if (own) { kf.inv_ell = P.inv_ell; kf.shift = P.shift; }
  const int col0 = w.y;
  const int ncb = min(NC, P.ncol - col0);
  const T inv_ell = (T)kf.inv_ell;
  __shared__ int s_seg, s_q;   // chunk start: segment and offset inside it
  const int t = threadIdx.x;
  for (int rb = 0; rb < P.rows; rb += 256) {
    const int m = min(256, P.rows - rb);
    const int G = max(1, 256 / m);
    const int p = t % m, g = t / m;
    const int64_t gp = P.row0 + rb + p;
    T y0 = 0, y1 = 0, y2 = 0;
    int yc = 0;
    if (g < G) {
      y0 = (T)xs[gp];
      y1 = (T)xs[ldx + gp];
      if (dim == 3) y2 = (T)xs[2 * ldx + gp];
      if (RPY) yc = (int)xs[3 * ldx + gp];
    }
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
    if (t == 0) { s_seg = P.seg0; s_q = 0; }
    __syncthreads();
    while (s_seg < P.seg1) {
      int cnt = 0;
      {
        int sg = s_seg, q = s_q;
        while (sg < P.seg1 && cnt < CH) {
          const NearSegT<T> S = segs[sg];
          const int take = min(S.cols - q, CH - cnt);
          const T* xin = S.x + (int64_t)col0 * S.ldx;
          for (int e = t; e < take; e += 256) {
            const int64_t gq = S.col0 + q + e;
            sx[0][cnt + e] = (T)xs[gq];
            sx[1][cnt + e] = (T)xs[ldx + gq];
            sx[2][cnt + e] = (dim == 3) ? (T)xs[2 * ldx + gq] : (T)0;
            if (RPY) sx[NX - 1][cnt + e] = (T)xs[3 * ldx + gq];
#pragma unroll
            for (int c = 0; c < NC; ++c)
              sv[c][cnt + e] = (c < ncb) ? xin[q + e + (int64_t)c * S.ldx] : (T)0;
          }
          cnt += take;
          q += take;
          if (q >= S.cols) { ++sg; q = 0; }
        }
        __syncthreads();
        if (t == 0) { s_seg = sg; s_q = q; }
      }
      if (g < G) {
        if (RPY) {
#pragma unroll 4
          for (int q = g; q < cnt; q += G) {
            const T kv = rpy_entry<T>(y0 - sx[0][q], y1 - sx[1][q], y2 - sx[2][q], yc,
                                      (int)sx[NX - 1][q], inv_ell);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = kv * sv[c][q] + acc[c];
          }
        } else if (dim == 3) {
#pragma unroll 4
          for (int q = g; q < cnt; q += G) {
            const T d0 = y0 - sx[0][q], d1 = y1 - sx[1][q], d2 = y2 - sx[2][q];
            const T kv = kernel_r2_k<KIND>(d0 * d0 + d1 * d1 + d2 * d2, inv_ell);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = kv * sv[c][q] + acc[c];
          }
        } else {
#pragma unroll 4
          for (int q = g; q < cnt; q += G) {
            const T d0 = y0 - sx[0][q], d1 = y1 - sx[1][q];
            const T kv = kernel_r2_k<KIND>(d0 * d0 + d1 * d1, inv_ell);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = kv * sv[c][q] + acc[c];
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) red[c][t] = acc[c];
    __syncthreads();
    if (t < m) {
      // the diagonal shift of a self segment: sigma * x_p
      T shift_x[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) shift_x[c] = 0;
      for (int sg = P.seg0; sg < P.seg1; ++sg) {
        const NearSegT<T> S = segs[sg];
        if (S.self) {
          const int64_t off = P.row0 + rb + t - S.col0;
          if (off >= 0 && off < S.cols) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
              if (c < ncb) shift_x[c] += (T)kf.shift * S.x[off + (int64_t)(col0 + c) * S.ldx];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < ncb) {
          T sum = 0;
          for (int gg = 0; gg < G; ++gg) sum += red[c][t + gg * m];
          sum += shift_x[c];
          T* o = P.out + (rb + t) + (int64_t)(col0 + c) * P.ldo;
          *o = P.beta ? (*o + sum) : sum;
        }
      }
    }
    __syncthreads();
  }
}

// Many columns (17..64): the (row, column) output pairs of 32 rows are spread over the 256
// threads (at most 8 each, a compile-time count), the kernel tile of every 32-point source
// chunk is evaluated once into shared memory, and the source rows of the chunk are staged.
template <int PPT, int KIND>
__device__ __forceinline__ void near_pairs(const NearProb& P, const NearSeg* __restrict__ segs,
                                           int col0, int ncb, int rb, int nr, KernelFn kf,
                                           const double* __restrict__ xs, int64_t ldx, int dim,
                                           double (*Kt)[33], double (*Xt)[65], double (*rx)[32],
                                           double (*cx)[32]) {
  const int t = threadIdx.x;
  const int npair = nr * ncb;
  double acc[PPT];
  int pr[PPT], pc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int e = t + 256 * k;
    acc[k] = 0.0;
    pr[k] = (e < npair) ? e % nr : 0;
    pc[k] = (e < npair) ? e / nr : 0;
  }
  for (int sg = P.seg0; sg < P.seg1; ++sg) {
    const NearSeg S = segs[sg];
    for (int q0 = 0; q0 < S.cols; q0 += 32) {
      const int nq = min(32, S.cols - q0);
      if (t < 32 && t < nq)
        for (int a = 0; a < (KIND == SPDHSS_K_RPY ? 4 : dim); ++a)
          cx[a][t] = xs[a * ldx + S.col0 + q0 + t];
      for (int e = t; e < 32 * 64; e += 256) {
        const int qq = e % 32, cc = e / 32;
        double v = 0.0;
        if (qq < nq && cc < ncb) v = S.x[(q0 + qq) + (int64_t)(col0 + cc) * S.ldx];
        Xt[qq][cc] = v;
      }
      __syncthreads();
      for (int e = t; e < 32 * 32; e += 256) {
        const int rr = e & 31, qq = e >> 5;
        double v = 0.0;
        if (rr < nr && qq < nq) {
          if (KIND == SPDHSS_K_RPY) {
            v = rpy_entry<double>(rx[0][rr] - cx[0][qq], rx[1][rr] - cx[1][qq],
                                  rx[2][rr] - cx[2][qq], (int)rx[3][rr], (int)cx[3][qq],
                                  kf.inv_ell);
          } else {
            double r2 = 0.0;
            for (int a = 0; a < dim; ++a) {
              const double d = rx[a][rr] - cx[a][qq];
              r2 += d * d;
            }
            v = kernel_r2_k<KIND>(r2, kf.inv_ell);
          }
          if (S.self && (P.row0 + rb + rr) == (S.col0 + q0 + qq)) v += kf.shift;
        }
        Kt[qq][rr] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int qq = 0; qq < 32; ++qq) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) acc[k] = fma(Kt[qq][pr[k]], Xt[qq][pc[k]], acc[k]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int e = t + 256 * k;
    if (e < npair) {
      double* o = P.out + (rb + pr[k]) + (int64_t)(col0 + pc[k]) * P.ldo;
      *o = P.beta ? (*o + acc[k]) : acc[k];
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(256) k_near_pairs(const NearProb* __restrict__ probs,
                                                    const NearSeg* __restrict__ segs,
                                                    const int2* __restrict__ work, KernelFn kf_,
                                                    const double* __restrict__ xs_, int64_t ldx_,
                                                    int dim_) {
  __shared__ double Kt[32][33];
  __shared__ double Xt[32][65];
  __shared__ double rx[4][32];   // coordinates (+ the component row of a vector kernel)
  __shared__ double cx[4][32];
  const int2 w = work[blockIdx.x];
  const NearProb P = probs[w.x];
  const bool own = P.xs != nullptr;
  const double* __restrict__ xs = own ? P.xs : xs_;
  const int64_t ldx = own ? P.ldx : ldx_;
  const int dim = own ? P.dim : dim_;
  KernelFn kf = kf_;
  if (own) { kf.inv_ell = P.inv_ell; kf.shift = P.shift; }
  const int col0 = w.y;
  const int ncb = min(64, P.ncol - col0);
  for (int rb = 0; rb < P.rows; rb += 32) {
    const int nr = min(32, P.rows - rb);
    if (threadIdx.x < nr)
      for (int a = 0; a < (KIND == SPDHSS_K_RPY ? 4 : dim); ++a)
        rx[a][threadIdx.x] = xs[a * ldx + P.row0 + rb + threadIdx.x];
    __syncthreads();
    const int ppt = (nr * ncb + 255) / 256;
    if (ppt <= 1) near_pairs<1, KIND>(P, segs, col0, ncb, rb, nr, kf, xs, ldx, dim, Kt, Xt, rx, cx);
    else if (ppt <= 2) near_pairs<2, KIND>(P, segs, col0, ncb, rb, nr, kf, xs, ldx, dim, Kt, Xt, rx, cx);
    else if (ppt <= 4) near_pairs<4, KIND>(P, segs, col0, ncb, rb, nr, kf, xs, ldx, dim, Kt, Xt, rx, cx);
    else near_pairs<8, KIND>(P, segs, col0, ncb, rb, nr, kf, xs, ldx, dim, Kt, Xt, rx, cx);
    __syncthreads();
  }
}

// out = beta * out + sum of the parts (fixed order), one thread per output entry
template <class T>
__global__ void k_near_reduce(const NearProbT<T>* __restrict__ probs, const int4* __restrict__ red,
                              const T* __restrict__ scratch) {
  const int4 r = red[blockIdx.x];
  const NearProbT<T> P = probs[r.x];
  const int64_t tot = (int64_t)P.rows * P.ncol;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int i = (int)(e % P.rows), c = (int)(e / P.rows);
    T sum = 0;
    for (int q = 0; q < r.z; ++q) sum += scratch[(int64_t)r.y + (int64_t)q * tot + e];
    T* o = P.out + i + (int64_t)c * P.ldo;
    *o = P.beta ? (*o + sum) : sum;
  }
}

template <class T>
void NearBatchT<T>::upload(cudaStream_t s) {
  work.clear();
  int mx = 1;
  for (const auto& p : probs) mx = std::max(mx, p.ncol);
  // few columns: thread-per-row kernel (cb = -NC); otherwise shared-memory kernel tiles.
  // Problems that carry the choice of their first upload keep it (all of one launch
  // share it: merged launches are grouped by it).
  if (mx <= 16) cb = -(mx <= 1 ? 1 : (mx <= 2 ? 2 : (mx <= 4 ? 4 : (mx <= 8 ? 8 : 16))));
  else cb = std::is_same<T, double>::value ? 64 : -16;   // FP32: blocks of 16 columns
  for (const auto& p : probs)
    if (p.cb != 0) { cb = p.cb; break; }
  for (auto& p : probs) {
    SPD_REQUIRE(p.cb == 0 || p.cb == cb, "near field: problems of one launch differ in column block");
    p.cb = cb;
  }
  const int step = cb < 0 ? -cb : cb;
  // the problems as launched: the many-column kernel takes 32 rows per CTA, so its
  // problems are cut into 32-row blocks (disjoint output rows)
  exec_probs.clear();
  if (cb > 0) {
    for (const auto& P : probs)
      for (int rb = 0; rb < P.rows; rb += 32) {
        NearProbT<T> q = P;
        q.row0 = P.row0 + rb;
        q.rows = std::min(32, P.rows - rb);
        q.out = P.out + rb;
        exec_probs.push_back(q);
      }
  } else {
    exec_probs = probs;
  }
  // split the segments when there are too few CTAs for the GPU; a problem that carries
  // the split of its first upload keeps it
  parts = 1;
  part_probs.clear();
  red.clear();
  if (!exec_probs.empty()) {
    int64_t ctas = 0, maxseg = 1;
    for (const auto& p : exec_probs) {
      ctas += (p.ncol + step - 1) / step;
      maxseg = std::max<int64_t>(maxseg, p.seg1 - p.seg0);
    }
    const int64_t want = 4 * 152;
    parts = (int)std::min<int64_t>(std::max<int64_t>(1, (want + ctas - 1) / ctas), std::min<int64_t>(8, maxseg));
    for (auto& p : exec_probs)
      if (p.parts == 0) p.parts = parts;
    for (size_t q = 0, e = 0; q < probs.size(); ++q) {   // the choice, back to the originals
      const size_t ne = (cb > 0) ? (size_t)((probs[q].rows + 31) / 32) : 1;
      if (ne > 0) probs[q].parts = exec_probs[e].parts;
      e += ne;
    }
    parts = 1;
    for (const auto& p : exec_probs) parts = std::max(parts, std::min(p.parts, std::max(p.seg1 - p.seg0, 1)));
  }
  if (parts > 1) {
    int64_t off = 0;
    for (int p = 0; p < (int)exec_probs.size(); ++p) {
      const NearProbT<T>& P = exec_probs[p];
      const int ns = P.seg1 - P.seg0;
      const int np = std::min(P.parts, std::max(ns, 1));
      const int64_t tot = (int64_t)P.rows * P.ncol;
      red.push_back(make_int4(p, (int)off, np, 0));
      for (int q = 0; q < np; ++q) {
        NearProbT<T> pp = P;
        pp.seg0 = P.seg0 + (int)((int64_t)ns * q / np);
        pp.seg1 = P.seg0 + (int)((int64_t)ns * (q + 1) / np);
        pp.out = nullptr;          // patched to the scratch below
        pp.ldo = P.rows;
        pp.beta = 0;
        pp.row0 = P.row0;
        part_probs.push_back(pp);
      }
      off += tot * np;
    }
    SPD_REQUIRE(off < (1LL << 31), "near field: partial-sum scratch too large");
    scratch.alloc(std::max<int64_t>(off, 1));
    int64_t o2 = 0;
    size_t k = 0;
    for (size_t r = 0; r < red.size(); ++r) {
      const NearProbT<T>& P = exec_probs[red[r].x];
      const int64_t tot = (int64_t)P.rows * P.ncol;
      for (int q = 0; q < red[r].z; ++q, ++k) part_probs[k].out = scratch.p + o2 + (int64_t)q * tot;
      o2 += tot * red[r].z;
    }
  }
  flops = 0.0;
  evals = 0.0;
  const std::vector<NearProbT<T>>& wp = parts > 1 ? part_probs : exec_probs;
  for (int p = 0; p < (int)wp.size(); ++p)
    for (int c0 = 0; c0 < wp[p].ncol; c0 += step) work.push_back(make_int2(p, c0));
  for (int p = 0; p < (int)probs.size(); ++p) {
    for (int g = probs[p].seg0; g < probs[p].seg1; ++g) {
      const double e = (double)probs[p].rows * segs[g].cols;
      evals += e;
      flops += 2.0 * e * probs[p].ncol;
    }
  }
  d_probs.upload(exec_probs, s);
  d_segs.upload(segs, s);
  d_work.upload(work, s);
  if (parts > 1) {
    d_part_probs.upload(part_probs, s);
    d_red.upload(red, s);
  }
}

// near-field problems of several instances (same kernel kind): every problem carries its
// own points and kernel parameters
template <class T>
struct DeferredNear : Deferred {
  std::vector<NearProbT<T>> probs;
  std::vector<NearSegT<T>> segs;
  const char* tag = "near";
  int kind = 0;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    // one launch per column block chosen by the instances (normally a single one)
    std::map<int, NearBatchT<T>> by_cb;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredNear<T>*>(d);
      for (NearProbT<T> p : x->probs) {
        NearBatchT<T>& m = by_cb[p.cb];
        const int off = (int)m.segs.size();
        m.segs.insert(m.segs.end(), x->segs.begin() + p.seg0, x->segs.begin() + p.seg1);
        p.seg1 = off + (p.seg1 - p.seg0);
        p.seg0 = off;
        m.probs.push_back(p);
      }
    }
    KernelFn k{};
    k.kind = kind;
    for (auto& kv : by_cb) {
      NearBatchT<T>& m = kv.second;
      m.tag = tag;
      m.upload(s);
      m.launch(k, nullptr, 0, 0, s);
    }
  }
};

template <class T>
void NearBatchT<T>::launch(const KernelFn& k, const double* xs, int64_t ldx, int dim,
                           cudaStream_t s) const {
  if (merging()) {
    if (probs.empty()) { merge_skip(); return; }
    std::unique_ptr<DeferredNear<T>> d(new DeferredNear<T>());
    d->probs = probs;
    for (auto& p : d->probs)
      if (!p.xs) { p.xs = xs; p.ldx = ldx; p.dim = dim; p.inv_ell = k.inv_ell; p.shift = k.shift; }
    d->segs = segs;
    d->tag = tag;
    d->kind = k.kind;
    merge_ctx().m->submit(std::string(sizeof(T) == 8 ? "near_f64_" : "near_f32_") +
                              std::to_string(k.kind), std::move(d));
    return;
  }
  if (work.empty()) return;
  ProfScope ps(tag, s, flops, 8.0 * evals);
  const unsigned g = (unsigned)work.size();
  const NearProbT<T>* pr = parts > 1 ? d_part_probs.p : d_probs.p;
  const NearSegT<T>* sg = d_segs.p;
  const int2* wk = d_work.p;
#define SPD_NEAR_SMALL(NC)                                                                  \
  switch (k.kind) {                                                                         \
    case SPDHSS_K_EXP: k_near_small<T, NC, SPDHSS_K_EXP><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break; \
    case SPDHSS_K_GAUSS: k_near_small<T, NC, SPDHSS_K_GAUSS><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break; \
    case SPDHSS_K_MATERN32: k_near_small<T, NC, SPDHSS_K_MATERN32><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break; \
    case SPDHSS_K_RPY: k_near_small<T, NC, SPDHSS_K_RPY><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break; \
    default: k_near_small<T, NC, SPDHSS_K_IMQ><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break; \
  }
  switch (cb) {
    case -1: SPD_NEAR_SMALL(1); break;
    case -2: SPD_NEAR_SMALL(2); break;
    case -4: SPD_NEAR_SMALL(4); break;
    case -8: SPD_NEAR_SMALL(8); break;
    case -16: SPD_NEAR_SMALL(16); break;
    default:
      if constexpr (std::is_same<T, double>::value) {
        switch (k.kind) {
          case SPDHSS_K_EXP: k_near_pairs<SPDHSS_K_EXP><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break;
          case SPDHSS_K_GAUSS: k_near_pairs<SPDHSS_K_GAUSS><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break;
          case SPDHSS_K_MATERN32: k_near_pairs<SPDHSS_K_MATERN32><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break;
          case SPDHSS_K_RPY: k_near_pairs<SPDHSS_K_RPY><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break;
          default: k_near_pairs<SPDHSS_K_IMQ><<<g, 256, 0, s>>>(pr, sg, wk, k, xs, ldx, dim); break;
        }
      } else {
        throw Error(SPDHSS_EINVAL, "mixed-precision near field supports at most 16 columns");
      }
      break;
  }
#undef SPD_NEAR_SMALL
  if (parts > 1) {
    SPD_LAUNCHED();
    k_near_reduce<T><<<(unsigned)red.size(), 128, 0, s>>>(d_probs.p, d_red.p, scratch.p);
  }
  SPD_LAUNCHED();
}

template struct NearBatchT<double>;
template struct NearBatchT<float>;

}  // namespace spd
