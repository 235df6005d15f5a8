// Kernel-matrix evaluation kernels (see keval.cuh).
#include <algorithm>

#include "keval.cuh"

namespace spd {

// ---------------------------------------------------------------------------------------
// dense tiles, 32 x 32 per CTA
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tiles(const TileProb* __restrict__ probs,
                                               const int4* __restrict__ work, KernelFn kf,
                                               int dim) {
  const int4 w = work[blockIdx.x];
  const TileProb P = probs[w.x];
  const int i0 = w.y, j0 = w.z;
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int i = i0 + (e & 31), j = j0 + (e >> 5);
    if (i >= P.rows || j >= P.cols) continue;
    const int64_t pr = P.r0 + i, pc = P.c0 + j;
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double d = P.xr[a * P.ldxr + pr] - P.xc[a * P.ldxc + pc];
      r2 += d * d;
    }
    double v = kernel_r2(kf, r2);
    if (P.xr == P.xc && pr == pc) v += P.diag_add;
    P.out[i + (int64_t)j * P.ldo] = v;
  }
}

void tile_launch(const Batch<TileProb>& b, const KernelFn& k, int dim, cudaStream_t s) {
  if (b.empty()) return;
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
  SPD_CUDA(cudaStreamSynchronize(s));
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
                                               const int4* __restrict__ work, KernelFn kf,
                                               int dim) {
  const int4 w = work[blockIdx.x];
  const ProxyProb P = probs[w.x];
  const int np = proxy_count(dim);
  const int i0 = w.y, j0 = w.z;
  __shared__ double sy[3][64];
  if (threadIdx.x < 64 && i0 + threadIdx.x < np) {
    double y[3] = {0, 0, 0};
    proxy_point(P, dim, i0 + threadIdx.x, y);
    for (int a = 0; a < 3; ++a) sy[a][threadIdx.x] = y[a];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int ii = e & 63, j = j0 + (e >> 6);
    const int i = i0 + ii;
    if (i >= np || j >= P.cols) continue;
    const int64_t pc = P.c0 + j;
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double d = sy[a][ii] - P.xc[a * P.ldxc + pc];
      r2 += d * d;
    }
    P.out[i + (int64_t)j * P.ldo] = kernel_r2(kf, r2);
  }
}

void proxy_launch(const Batch<ProxyProb>& b, const KernelFn& k, int dim, cudaStream_t s) {
  if (b.empty()) return;
  const int np = proxy_count(dim);
  std::vector<int4> work;
  for (int p = 0; p < (int)b.size(); ++p)
    for (int i0 = 0; i0 < np; i0 += 64)
      for (int j0 = 0; j0 < b.h[p].cols; j0 += 32) work.push_back(make_int4(p, i0, j0, 0));
  if (work.empty()) return;
  DevBuf<int4> dw;
  dw.upload(work, s);
  {
    ProfScope ps("proxy", s);
    k_proxy<<<(unsigned)work.size(), 256, 0, s>>>(b.d.p, dw.p, k, dim);
    SPD_LAUNCHED();
  }
  SPD_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------------------
// near field: CTA = (problem, column block of CB); 256 threads = 128 rows x 2 column halves.
// For every segment, 32-point chunks: evaluate the 128 x 32 kernel tile into shared
// memory, stage the 32 x CB input rows, accumulate in registers.
// ---------------------------------------------------------------------------------------
template <int CB>
__global__ void __launch_bounds__(256) k_near(const NearProb* __restrict__ probs,
                                              const NearSeg* __restrict__ segs,
                                              const int2* __restrict__ work, KernelFn kf,
                                              const double* __restrict__ xs, int64_t ldx,
                                              int dim) {
  constexpr int HC = CB / 2;
  const int2 w = work[blockIdx.x];
  const NearProb P = probs[w.x];
  const int col0 = w.y;
  const int ncb = min(CB, P.ncol - col0);
  __shared__ double Kt[32][129];
  __shared__ double Xt[32][CB + 1];
  __shared__ double rx[3][128];
  __shared__ double cx[3][32];
  const int t = threadIdx.x;
  const int row = t & 127, half = t >> 7;
  for (int rb = 0; rb < P.rows; rb += 128) {
    const int nr = min(128, P.rows - rb);
    if (t < 128 && t < nr)
      for (int a = 0; a < dim; ++a) rx[a][t] = xs[a * ldx + P.row0 + rb + t];
    double acc[HC];
#pragma unroll
    for (int c = 0; c < HC; ++c) acc[c] = 0.0;
    __syncthreads();
    for (int sg = P.seg0; sg < P.seg1; ++sg) {
      const NearSeg S = segs[sg];
      for (int q0 = 0; q0 < S.cols; q0 += 32) {
        const int nq = min(32, S.cols - q0);
        if (t < 32 && t < nq)
          for (int a = 0; a < dim; ++a) cx[a][t] = xs[a * ldx + S.col0 + q0 + t];
        for (int e = t; e < 32 * CB; e += 256) {
          const int qq = e % 32, cc = e / 32;
          double v = 0.0;
          if (qq < nq && cc < ncb) v = S.x[(q0 + qq) + (int64_t)(col0 + cc) * S.ldx];
          Xt[qq][cc] = v;
        }
        __syncthreads();
        for (int e = t; e < 32 * 128; e += 256) {
          const int rr = e & 127, qq = e >> 7;
          double v = 0.0;
          if (rr < nr && qq < nq) {
            double r2 = 0.0;
            for (int a = 0; a < dim; ++a) {
              const double d = rx[a][rr] - cx[a][qq];
              r2 += d * d;
            }
            v = kernel_r2(kf, r2);
            if (S.self && (P.row0 + rb + rr) == (S.col0 + q0 + qq)) v += kf.shift;
          }
          Kt[qq][rr] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int qq = 0; qq < 32; ++qq) {
          const double kv = Kt[qq][row];
#pragma unroll
          for (int c = 0; c < HC; ++c) acc[c] = fma(kv, Xt[qq][half * HC + c], acc[c]);
        }
        __syncthreads();
      }
    }
    if (row < nr) {
#pragma unroll
      for (int c = 0; c < HC; ++c) {
        const int cc = half * HC + c;
        if (cc < ncb) {
          double* o = P.out + (rb + row) + (int64_t)(col0 + cc) * P.ldo;
          *o = P.beta ? (*o + acc[c]) : acc[c];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// near field with few columns (NC <= 16): one thread per target row; when a leaf has fewer
// than 256 points, G = 256 / rows groups of threads split the source points between them
// and a fixed-order sum in shared memory combines the groups.  Every kernel entry is
// evaluated exactly once per column block, and no FMA is spent on padding.
// ---------------------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(256) k_near_small(const NearProb* __restrict__ probs,
                                                    const NearSeg* __restrict__ segs,
                                                    const int2* __restrict__ work, KernelFn kf,
                                                    const double* __restrict__ xs, int64_t ldx,
                                                    int dim) {
  // source points staged per chunk; the staging area is reused for the final reduction
  constexpr int CH = NC >= 16 ? 192 : (NC >= 8 ? 256 : 512);
  constexpr int STAGE = CH * (4 + NC);
  constexpr int RED = NC * 256;
  __shared__ double smem[STAGE > RED ? STAGE : RED];
  double (*red)[256] = reinterpret_cast<double (*)[256]>(smem);
  double (*sx)[CH] = reinterpret_cast<double (*)[CH]>(smem);
  double (*sv)[CH] = reinterpret_cast<double (*)[CH]>(smem + 3 * CH);
  int64_t* sg_idx = reinterpret_cast<int64_t*>(smem + (3 + NC) * CH);
  const int2 w = work[blockIdx.x];
  const NearProb P = probs[w.x];
  const int col0 = w.y;
  const int ncb = min(NC, P.ncol - col0);
  __shared__ int s_seg, s_q;   // chunk start: segment and offset inside it
  const int t = threadIdx.x;
  for (int rb = 0; rb < P.rows; rb += 256) {
    const int m = min(256, P.rows - rb);
    const int G = max(1, 256 / m);
    const int p = t % m, g = t / m;
    const int64_t gp = P.row0 + rb + p;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    if (g < G) {
      y0 = xs[gp];
      y1 = xs[ldx + gp];
      if (dim == 3) y2 = xs[2 * ldx + gp];
    }
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    if (t == 0) { s_seg = P.seg0; s_q = 0; }
    __syncthreads();
    while (s_seg < P.seg1) {
      // flatten the next CH source points of the concatenated segments into shared memory
      int cnt = 0;
      {
        int sg = s_seg, q = s_q;
        while (sg < P.seg1 && cnt < CH) {
          const NearSeg S = segs[sg];
          const int take = min(S.cols - q, CH - cnt);
          const double* xin = S.x + (int64_t)col0 * S.ldx;
          for (int e = t; e < take; e += 256) {
            const int64_t gq = S.col0 + q + e;
            sx[0][cnt + e] = xs[gq];
            sx[1][cnt + e] = xs[ldx + gq];
            sx[2][cnt + e] = (dim == 3) ? xs[2 * ldx + gq] : 0.0;
            sg_idx[cnt + e] = S.self ? gq : -1;
#pragma unroll
            for (int c = 0; c < NC; ++c)
              sv[c][cnt + e] = (c < ncb) ? xin[q + e + (int64_t)c * S.ldx] : 0.0;
          }
          cnt += take;
          q += take;
          if (q >= S.cols) { ++sg; q = 0; }
        }
        __syncthreads();
        if (t == 0) { s_seg = sg; s_q = q; }
      }
      if (g < G) {
#pragma unroll 4
        for (int q = g; q < cnt; q += G) {
          const double d0 = y0 - sx[0][q], d1 = y1 - sx[1][q];
          double r2 = d0 * d0 + d1 * d1;
          if (dim == 3) {
            const double d2 = y2 - sx[2][q];
            r2 += d2 * d2;
          }
          double kv = kernel_r2(kf, r2);
          if (sg_idx[q] == gp) kv += kf.shift;
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (c < ncb) acc[c] = fma(kv, sv[c][q], acc[c]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) red[c][t] = acc[c];
    __syncthreads();
    if (t < m) {
      for (int c = 0; c < ncb; ++c) {
        double sum = 0.0;
        for (int gg = 0; gg < G; ++gg) sum += red[c][t + gg * m];
        double* o = P.out + (rb + t) + (int64_t)(col0 + c) * P.ldo;
        *o = P.beta ? (*o + sum) : sum;
      }
    }
    __syncthreads();
  }
}

void NearBatch::upload(cudaStream_t s) {
  work.clear();
  int mx = 1;
  for (const auto& p : probs) mx = std::max(mx, p.ncol);
  // few columns: thread-per-row kernel (cb = -NC); otherwise shared-memory kernel tiles
  if (mx <= 16) cb = -(mx <= 1 ? 1 : (mx <= 2 ? 2 : (mx <= 4 ? 4 : (mx <= 8 ? 8 : 16))));
  else cb = mx <= 32 ? 32 : 64;
  const int step = cb < 0 ? -cb : cb;
  flops = 0.0;
  evals = 0.0;
  for (int p = 0; p < (int)probs.size(); ++p) {
    for (int c0 = 0; c0 < probs[p].ncol; c0 += step) work.push_back(make_int2(p, c0));
    for (int g = probs[p].seg0; g < probs[p].seg1; ++g) {
      const double e = (double)probs[p].rows * segs[g].cols;
      evals += e;
      flops += 2.0 * e * probs[p].ncol;
    }
  }
  d_probs.upload(probs, s);
  d_segs.upload(segs, s);
  d_work.upload(work, s);
}

void NearBatch::launch(const KernelFn& k, const double* xs, int64_t ldx, int dim,
                       cudaStream_t s) const {
  if (work.empty()) return;
  ProfScope ps(tag, s, flops, 8.0 * evals);
  const unsigned g = (unsigned)work.size();
  switch (cb) {
    case -1: k_near_small<1><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case -2: k_near_small<2><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case -4: k_near_small<4><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case -8: k_near_small<8><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case -16: k_near_small<16><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case 8: k_near<8><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case 16: k_near<16><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    case 32: k_near<32><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
    default: k_near<64><<<g, 256, 0, s>>>(d_probs.p, d_segs.p, d_work.p, k, xs, ldx, dim); break;
  }
  SPD_LAUNCHED();
}

}  // namespace spd
