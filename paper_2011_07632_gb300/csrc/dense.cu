// Batched FP64 dense kernels: grouped GEMM, Cholesky, triangular solves, Householder QR
// with column pivoting (thread-block clusters split the columns of a large matrix), and
// reflector application.  One launch covers all nodes of a tree level.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "dense.cuh"
#include "tune.cuh"

namespace cg = cooperative_groups;

namespace spd {

// ---------------------------------------------------------------------------------------
// grouped GEMM: 64x64 tile per CTA, 256 threads, 4x4 register tile per thread, K step 16
// ---------------------------------------------------------------------------------------
constexpr int GM = 64, GN = 64, GK = 16;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// A tile with t.w > 0 covers only the K range kparts[t.w - 1] = (k_lo, k_hi, slot) of the
// problem's concatenated segments and writes its unscaled sums to the partial slots from
// `slot` on (column c, row r at [c * 64 + r]); k_gemm_kreduce adds the parts in order.
template <class T>
__global__ void __launch_bounds__(256) k_gemm(const GemmProbT<T>* __restrict__ probs,
                                              const GemmSegT<T>* __restrict__ segs,
                                              const int4* __restrict__ tiles,
                                              const int4* __restrict__ kparts,
                                              T* __restrict__ partial) {
  const int4 t = tiles[blockIdx.x];
  const GemmProbT<T> P = probs[t.x];
  const int m0 = t.y, n0 = t.z;
  int klo = 0, khi = 0x7fffffff;
  T* pout = nullptr;
  if (t.w > 0) {
    const int4 kp = kparts[t.w - 1];
    klo = kp.x;
    khi = kp.y;
    pout = partial + (int64_t)kp.z * (4 * GM);
  }
  __shared__ T As[GK][GM + 1];
  __shared__ T Bs[GK][GN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  int kbase = 0;   // offset of the segment in the concatenated K range
  for (int s = P.seg0; s < P.seg1; ++s) {
    const GemmSegT<T> S = segs[s];
    const int ks = max(0, klo - kbase), ke = min(S.K, khi - kbase);
    kbase += S.K;
    for (int k0 = ks; k0 < ke; k0 += GK) {
#pragma unroll
      for (int r = 0; r < (GM * GK) / 256; ++r) {
        const int e = tid + 256 * r;
        int mm, kk;
        if (!S.tA) { mm = e % GM; kk = e / GM; } else { kk = e % GK; mm = e / GK; }
        const int gm = m0 + mm, gk = k0 + kk;
        T v = 0;
        if (gm < P.M && gk < ke)
          v = S.tA ? S.A[gk + (int64_t)gm * S.lda] : S.A[gm + (int64_t)gk * S.lda];
        As[kk][mm] = v;
      }
#pragma unroll
      for (int r = 0; r < (GN * GK) / 256; ++r) {
        const int e = tid + 256 * r;
        int nn, kk;
        if (!S.tB) { kk = e % GK; nn = e / GK; } else { nn = e % GN; kk = e / GN; }
        const int gn = n0 + nn, gk = k0 + kk;
        T v = 0;
        if (gn < P.N && gk < ke)
          v = S.tB ? S.B[gn + (int64_t)gk * S.ldb] : S.B[gk + (int64_t)gn * S.ldb];
        Bs[kk][nn] = v;
      }
      __syncthreads();
      const int kc = min(GK, ke - k0);   // no FMA on the padding of a short segment
#pragma unroll 4
      for (int kk = 0; kk < kc; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaT(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  if (pout) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) pout[(tx + 16 * j) * GM + ty + 16 * i] = acc[i][j];
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= P.N) continue;
      T* c = P.tC ? P.C + gn + (int64_t)gm * P.ldc : P.C + gm + (int64_t)gn * P.ldc;
      T v = (T)P.alpha * acc[i][j];
      if (P.beta != 0.0) v += (T)P.beta * (*c);
      *c = v;
    }
  }
}

// Skinny variant for N <= 32 columns: 64-row tiles, 256 threads = 64 rows x 4 column
// groups of NB/4 columns each, K step 32.  No FMA is spent on padding columns.
template <class T, int NB>
__global__ void __launch_bounds__(256) k_gemm_n(const GemmProbT<T>* __restrict__ probs,
                                                const GemmSegT<T>* __restrict__ segs,
                                                const int4* __restrict__ tiles,
                                                const int4* __restrict__ kparts,
                                                T* __restrict__ partial) {
  constexpr int MB = 64, KB = 32, CPT = NB / 4;
  const int4 t = tiles[blockIdx.x];
  const GemmProbT<T> P = probs[t.x];
  const int m0 = t.y, n0 = t.z;
  int klo = 0, khi = 0x7fffffff;
  T* pout = nullptr;
  if (t.w > 0) {   // a K part of a split tile (as in k_gemm)
    const int4 kp = kparts[t.w - 1];
    klo = kp.x;
    khi = kp.y;
    pout = partial + (int64_t)kp.z * (4 * MB);
  }
  __shared__ T As[KB][MB + 1];
  __shared__ T Bs[KB][NB + 1];
  const int tid = threadIdx.x;
  const int row = tid & 63, cg = tid >> 6;
  T acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0;
  int kbase = 0;
  for (int sg = P.seg0; sg < P.seg1; ++sg) {
    const GemmSegT<T> S = segs[sg];
    const int ks = max(0, klo - kbase), ke = min(S.K, khi - kbase);
    kbase += S.K;
    for (int k0 = ks; k0 < ke; k0 += KB) {
#pragma unroll
      for (int r = 0; r < (MB * KB) / 256; ++r) {
        const int e = tid + 256 * r;
        int mm, kk;
        if (!S.tA) { mm = e % MB; kk = e / MB; } else { kk = e % KB; mm = e / KB; }
        const int gm = m0 + mm, gk = k0 + kk;
        T v = 0;
        if (gm < P.M && gk < ke)
          v = S.tA ? S.A[gk + (int64_t)gm * S.lda] : S.A[gm + (int64_t)gk * S.lda];
        As[kk][mm] = v;
      }
      for (int e = tid; e < KB * NB; e += 256) {
        int nn, kk;
        if (!S.tB) { kk = e % KB; nn = e / KB; } else { nn = e % NB; kk = e / NB; }
        const int gn = n0 + nn, gk = k0 + kk;
        T v = 0;
        if (gn < P.N && gk < ke)
          v = S.tB ? S.B[gn + (int64_t)gk * S.ldb] : S.B[gk + (int64_t)gn * S.ldb];
        Bs[kk][nn] = v;
      }
      __syncthreads();
      const int kc = min(KB, ke - k0);   // no FMA on the padding of a short segment
#pragma unroll 8
      for (int kk = 0; kk < kc; ++kk) {
        const T a = As[kk][row];
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c] = fmaT(a, Bs[kk][cg * CPT + c], acc[c]);
      }
      __syncthreads();
    }
  }
  if (pout) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) pout[(cg * CPT + c) * MB + row] = acc[c];
    return;
  }
  const int gm = m0 + row;
  if (gm < P.M) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int gn = n0 + cg * CPT + c;
      if (gn < P.N) {
        T* cp = P.tC ? P.C + gn + (int64_t)gm * P.ldc : P.C + gm + (int64_t)gn * P.ldc;
        T v = (T)P.alpha * acc[c];
        if (P.beta != 0.0) v += (T)P.beta * (*cp);
        *cp = v;
      }
    }
  }
}

// Very skinny variant for N <= 4 columns (matrix-vector like): 64-row tiles, 256 threads =
// 64 rows x 4 groups that split every 32-wide K chunk; the four partial sums are added in
// a fixed order through shared memory.
// A tile with t.w > 0 covers only the K range kparts[t.w - 1] = (k_lo, k_hi, slot) of the
// problem's concatenated segments and writes its unscaled partial sums to partial slot
// `slot`; k_gemm_kreduce adds the slots of a tile in order and applies alpha and beta.
template <class T, int NB>
__global__ void __launch_bounds__(256) k_gemm_k(const GemmProbT<T>* __restrict__ probs,
                                                const GemmSegT<T>* __restrict__ segs,
                                                const int4* __restrict__ tiles,
                                                const int4* __restrict__ kparts,
                                                T* __restrict__ partial) {
  constexpr int MB = 64, KB = 32;
  const int4 t = tiles[blockIdx.x];
  const GemmProbT<T> P = probs[t.x];
  const int m0 = t.y, n0 = t.z;
  int klo = 0, khi = 0x7fffffff;
  T* pout = nullptr;
  if (t.w > 0) {
    const int4 kp = kparts[t.w - 1];
    klo = kp.x;
    khi = kp.y;
    pout = partial + (int64_t)kp.z * (4 * MB);   // slots have the 4-column stride
  }
  __shared__ T As[KB][MB + 1];
  __shared__ T Bs[KB][NB];
  __shared__ T red[4][NB][MB];
  const int tid = threadIdx.x;
  const int row = tid & 63, kg = tid >> 6;
  T acc[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) acc[c] = 0;
  int kbase = 0;   // offset of the segment in the concatenated K range
  for (int sg = P.seg0; sg < P.seg1; ++sg) {
    const GemmSegT<T> S = segs[sg];
    const int ks = max(0, klo - kbase), ke = min(S.K, khi - kbase);
    kbase += S.K;
    for (int k0 = ks; k0 < ke; k0 += KB) {
#pragma unroll
      for (int r = 0; r < (MB * KB) / 256; ++r) {
        const int e = tid + 256 * r;
        int mm, kk;
        if (!S.tA) { mm = e % MB; kk = e / MB; } else { kk = e % KB; mm = e / KB; }
        const int gm = m0 + mm, gk = k0 + kk;
        T v = 0;
        if (gm < P.M && gk < ke)
          v = S.tA ? S.A[gk + (int64_t)gm * S.lda] : S.A[gm + (int64_t)gk * S.lda];
        As[kk][mm] = v;
      }
      if (tid < KB * NB) {
        const int kk = tid % KB, nn = tid / KB;
        const int gn = n0 + nn, gk = k0 + kk;
        T v = 0;
        if (gn < P.N && gk < ke)
          v = S.tB ? S.B[gn + (int64_t)gk * S.ldb] : S.B[gk + (int64_t)gn * S.ldb];
        Bs[kk][nn] = v;
      }
      __syncthreads();
      const int kc = min(KB, ke - k0);   // no FMA on the padding of a short segment
#pragma unroll
      for (int q = 0; q < KB / 4; ++q) {
        const int kk = kg * (KB / 4) + q;
        if (kk >= kc) break;
        const T a = As[kk][row];
#pragma unroll
        for (int c = 0; c < NB; ++c) acc[c] = fmaT(a, Bs[kk][c], acc[c]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c) red[kg][c][row] = acc[c];
  __syncthreads();
  if (kg == 0 && pout) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      pout[c * MB + row] = (red[0][c][row] + red[1][c][row]) + (red[2][c][row] + red[3][c][row]);
  } else if (kg == 0) {
    const int gm = m0 + row;
    if (gm < P.M) {
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const int gn = n0 + c;
        if (gn < P.N) {
          const T v0 = (red[0][c][row] + red[1][c][row]) + (red[2][c][row] + red[3][c][row]);
          T* cp = P.tC ? P.C + gn + (int64_t)gm * P.ldc : P.C + gm + (int64_t)gn * P.ldc;
          T v = (T)P.alpha * v0;
          if (P.beta != 0.0) v += (T)P.beta * (*cp);
          *cp = v;
        }
      }
    }
  }
}

// the K parts of a split tile: out = alpha * (sum of the parts in order) + beta * out.
// nparts[i] = parts | (slot width << 8): a part covers width / 4 slots of 4 columns x 64
// rows (4 for the up-to-4-column variants, the tile width otherwise), parts consecutive.
template <class T>
__global__ void __launch_bounds__(64) k_gemm_kreduce(const GemmProbT<T>* __restrict__ probs,
                                                     const int4* __restrict__ reds,
                                                     const int* __restrict__ nparts,
                                                     const T* __restrict__ partial) {
  constexpr int MB = 64;
  const int4 r = reds[blockIdx.x];   // (problem, m0, n0, first slot)
  const int np = nparts[blockIdx.x] & 255, w = nparts[blockIdx.x] >> 8;
  const GemmProbT<T> P = probs[r.x];
  const int row = threadIdx.x, gm = r.y + row;
  if (gm >= P.M) return;
  const int64_t stride = (int64_t)(w / 4) * (4 * MB);
  for (int c = 0; c < w; ++c) {
    const int gn = r.z + c;
    if (gn >= P.N) break;
    const T* src = partial + (int64_t)r.w * (4 * MB) + c * MB + row;
    T v0 = src[0];
    for (int q = 1; q < np; ++q) v0 += src[q * stride];
    T* cp = P.tC ? P.C + gn + (int64_t)gm * P.ldc : P.C + gm + (int64_t)gn * P.ldc;
    T v = (T)P.alpha * v0;
    if (P.beta != 0.0) v += (T)P.beta * (*cp);
    *cp = v;
  }
}

static int gemm_variant(int maxn) {
  if (maxn <= 1) return 1;
  if (maxn <= 2) return 2;
  if (maxn <= 4) return 4;
  if (maxn <= 8) return 8;
  if (maxn <= 16) return 16;
  if (maxn <= 32) return 32;
  return 0;
}

template <class T>
static void gemm_dispatch(int nb, int g, const GemmProbT<T>* pr, const GemmSegT<T>* sg,
                          const int4* tl, cudaStream_t s, const int4* kp = nullptr,
                          T* partial = nullptr) {
  switch (nb) {
    case 1: k_gemm_k<T, 1><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    case 2: k_gemm_k<T, 2><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    case 4: k_gemm_k<T, 4><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    case 8: k_gemm_n<T, 8><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    case 16: k_gemm_n<T, 16><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    case 32: k_gemm_n<T, 32><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
    default: k_gemm<T><<<g, 256, 0, s>>>(pr, sg, tl, kp, partial); break;
  }
}

// tile footprint of a variant: rows x columns per CTA
static inline void gemm_tile_shape(int nb, int* tm, int* tn) {
  *tm = 64;
  *tn = nb ? nb : 64;
}

// fraction of the tile FMAs that are not padding for an M x N product on variant nb
static inline double gemm_fill(int M, int N, int nb) {
  int tm, tn;
  gemm_tile_shape(nb, &tm, &tn);
  const double tiles = (double)((M + tm - 1) / tm) * (double)((N + tn - 1) / tn);
  return tiles > 0 ? (double)M * N / (tiles * tm * tn) : 1.0;
}

template <class T>
void GemmBatchT<T>::upload(cudaStream_t s) {
  tiles.clear();
  lprobs.clear();
  lsegs.clear();
  vnb.clear();
  vbeg.clear();
  flops = 0.0;
  bytes = 0.0;
  if constexpr (sizeof(T) == 4) {
    if (tc) {   // tensor cores: the problems as given, 128 x tc_nt tiles
      for (const auto& P : probs) {
        double kk = 0.0;
        for (int g = P.seg0; g < P.seg1; ++g) kk += segs[g].K;
        flops += 2.0 * P.M * (double)P.N * kk;
      }
      tiles = tc_gemm_tiles(probs, &tc_nt);
      d_segs.upload(segs, s);
      d_probs.upload(probs, s);
      d_tiles.upload(tiles, s);
      return;
    }
  }
  int maxn = 0;
  for (const auto& p : probs) maxn = std::max(maxn, p.N);
  nb = gemm_variant(maxn);
  // orientation and variant of every problem
  std::vector<int> pv(probs.size());
  for (int p = 0; p < (int)probs.size(); ++p) {
    const GemmProbT<T>& P = probs[p];
    double kk = 0.0;
    for (int g = P.seg0; g < P.seg1; ++g) {
      kk += segs[g].K;
      bytes += sizeof(T) * ((double)P.M * segs[g].K + (double)segs[g].K * P.N);
    }
    flops += 2.0 * P.M * (double)P.N * kk;
    bytes += sizeof(T) * (double)P.M * P.N * (P.beta != 0.0 ? 2.0 : 1.0);
    const int v = gemm_variant(P.N), vt = gemm_variant(P.M);
    const bool tr = gemm_fill(P.N, P.M, vt) > 2.0 * gemm_fill(P.M, P.N, v);
    GemmProbT<T> q = P;
    q.seg0 = (int)lsegs.size();
    for (int g = P.seg0; g < P.seg1; ++g) {
      GemmSegT<T> sg = segs[g];
      if (tr) {   // C^T = B^T A^T
        GemmSegT<T> t2 = sg;
        t2.A = sg.B; t2.lda = sg.ldb; t2.tA = !sg.tB;
        t2.B = sg.A; t2.ldb = sg.lda; t2.tB = !sg.tA;
        sg = t2;
      }
      lsegs.push_back(sg);
    }
    q.seg1 = (int)lsegs.size();
    if (tr) { q.M = P.N; q.N = P.M; q.tC = !P.tC; }
    lprobs.push_back(q);
    pv[p] = tr ? vt : v;
  }
  // tiles grouped by variant
  static const int kVariants[7] = {1, 2, 4, 8, 16, 32, 0};
  std::vector<int> kt;   // K of every launched problem (filled on first use)
  kparts.clear();
  reds.clear();
  rednp.clear();
  int slot = 0;
  for (int v : kVariants) {
    std::vector<int4> vt;
    int tm, tn;
    gemm_tile_shape(v, &tm, &tn);
    for (int p = 0; p < (int)lprobs.size(); ++p) {
      if (pv[p] != v) continue;
      for (int m0 = 0; m0 < lprobs[p].M; m0 += tm)
        for (int n0 = 0; n0 < lprobs[p].N; n0 += tn) vt.push_back(make_int4(p, m0, n0, 0));
    }
    if (vt.empty()) continue;
    // matrix-vector-like products of few tiles: split the K range of each tile over
    // several CTAs (partial sums, added in order by k_gemm_kreduce).  The split of a
    // problem depends on that problem alone (its tile count and K), never on the other
    // problems of the launch, so that a product gives the same bits whichever launch it is
    // part of (one instance alone, or many merged).
    // Wider products with few tiles and a long K (the coupling and pair products of small
    // problems: one tile, K in the thousands) split the same way, into parts of at least
    // 256 (the partial tile of a part is written once, for 2 x 64 x 256 FMAs per column).
    {
      const bool narrow = v >= 1 && v <= 4;
      const int ws = narrow ? 4 : tn;            // slot width of a part
      const int kmin = narrow ? 128 : 256;       // K per part at least
      std::vector<int4> nt;
      for (const int4& t : vt) {
        int K = 0;
        for (int g = lprobs[t.x].seg0; g < lprobs[t.x].seg1; ++g) K += lsegs[g].K;
        const int64_t ptiles = ceil_div((int64_t)lprobs[t.x].M, (int64_t)tm) *
                               (narrow ? 1 : ceil_div((int64_t)lprobs[t.x].N, (int64_t)tn));
        const int want = ptiles >= 2 * 152
                             ? 1
                             : (int)std::min<int64_t>(16, ceil_div((int64_t)4 * 152, ptiles));
        const int kp = std::min(want, narrow ? (K + kmin - 1) / kmin : K / kmin);
        if (kp <= 1) { nt.push_back(t); continue; }
        reds.push_back(make_int4(t.x, t.y, t.z, slot));
        rednp.push_back(kp | (ws << 8));
        for (int q = 0; q < kp; ++q) {
          const int lo = (int)((int64_t)K * q / kp), hi = (int)((int64_t)K * (q + 1) / kp);
          kparts.push_back(make_int4(lo, hi, slot + q * (ws / 4), 0));
          nt.push_back(make_int4(t.x, t.y, t.z, (int)kparts.size()));
        }
        slot += kp * (ws / 4);
      }
      vt.swap(nt);
    }
    // longest K first, so that the long tiles do not form the tail of the launch: a
    // counting sort by the power of two of K (the order only schedules: every tile's
    // arithmetic is its own)
    {
      if (kt.empty()) {
        kt.assign(lprobs.size(), 0);
        for (int q = 0; q < (int)lprobs.size(); ++q)
          for (int g = lprobs[q].seg0; g < lprobs[q].seg1; ++g) kt[q] += lsegs[g].K;
      }
      auto bucket = [&](const int4& t) {
        const int k = t.w > 0 ? kparts[t.w - 1].y - kparts[t.w - 1].x : kt[t.x];
        int b = 0;
        while (b < 31 && (1 << b) < k) ++b;
        return 31 - b;   // long K first
      };
      int cnt[33] = {0};
      std::vector<unsigned char> bk(vt.size());
      for (size_t q = 0; q < vt.size(); ++q) { bk[q] = (unsigned char)bucket(vt[q]); ++cnt[bk[q] + 1]; }
      for (int b = 0; b < 32; ++b) cnt[b + 1] += cnt[b];
      std::vector<int4> sorted(vt.size());
      for (size_t q = 0; q < vt.size(); ++q) sorted[cnt[bk[q]]++] = vt[q];
      vt.swap(sorted);
    }
    vnb.push_back(v);
    vbeg.push_back((int64_t)tiles.size());
    tiles.insert(tiles.end(), vt.begin(), vt.end());
  }
  vbeg.push_back((int64_t)tiles.size());
  if (!reds.empty()) {
    d_kparts.upload(kparts, s);
    d_reds.upload(reds, s);
    d_rednp.upload(rednp, s);
    // slots of 4 columns x 64 rows; a part of a wider tile takes width / 4 of them
    d_partial.alloc(std::max(slot, 1) * (size_t)4 * 64);
  }
  d_segs.upload(lsegs, s);
  d_probs.upload(lprobs, s);
  d_tiles.upload(tiles, s);
}

// grouped GEMMs of several instances: segments re-based, one upload, one launch
template <class T>
struct DeferredGemm : Deferred {
  std::vector<GemmSegT<T>> segs;
  std::vector<GemmProbT<T>> probs;
  const char* tag = "gemm";
  int tc = 0;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    GemmBatchT<T> m;
    m.tag = tag;
    m.tc = tc;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredGemm<T>*>(d);
      const int off = (int)m.segs.size();
      m.segs.insert(m.segs.end(), x->segs.begin(), x->segs.end());
      for (GemmProbT<T> p : x->probs) {
        p.seg0 += off;
        p.seg1 += off;
        m.probs.push_back(p);
      }
    }
    m.upload(s);
    m.launch(s);
  }
};

template <class T>
void GemmBatchT<T>::launch(cudaStream_t s) const {
  if (merging()) {
    if (probs.empty()) { merge_skip(); return; }
    std::unique_ptr<DeferredGemm<T>> d(new DeferredGemm<T>());
    d->segs = segs;
    d->probs = probs;
    d->tag = tag;
    d->tc = tc;
    merge_ctx().m->submit(sizeof(T) == 8 ? "gemm_f64" : "gemm_f32_tc" + std::to_string(tc),
                          std::move(d));
    return;
  }
  const int64_t nt = (int64_t)tiles.size();
  if (nt == 0) return;
  ProfScope ps(tag, s, flops, bytes);
  if constexpr (sizeof(T) == 4) {
    if (tc) {
      tc_gemm_launch(d_probs.p, d_segs.p, d_tiles.p, nt, tc_nt, tc == 2, tc_error_word(), s,
                     tc_stall);
      return;
    }
  }
  for (size_t v = 0; v < vnb.size(); ++v) {
    for (int64_t b0 = vbeg[v]; b0 < vbeg[v + 1]; b0 += 2147483647LL) {
      const int g = (int)std::min<int64_t>(vbeg[v + 1] - b0, 2147483647LL);
      gemm_dispatch<T>(vnb[v], g, d_probs.p, d_segs.p, d_tiles.p + b0, s, d_kparts.p, d_partial.p);
      SPD_LAUNCHED();
    }
  }
  if (!reds.empty()) {
    // the reduction reads the slots with the 4-column stride used for every split variant
    k_gemm_kreduce<T><<<(unsigned)reds.size(), 64, 0, s>>>(d_probs.p, d_reds.p, d_rednp.p,
                                                            d_partial.p);
    SPD_LAUNCHED();
  }
}

template struct GemmBatchT<double>;
template struct GemmBatchT<float>;

// ---------------------------------------------------------------------------------------
// Cholesky
// ---------------------------------------------------------------------------------------

// Blocked right-looking Cholesky, one CTA per matrix, 32 x 32 tiles: one warp factors the
// diagonal tile in shared memory, every thread solves panel rows against it, and the
// trailing lower triangle is updated tile by tile from shared-memory copies of the panel.
constexpr int PB = 32;

__global__ void __launch_bounds__(256) k_potrf_blk(const PotrfProb* __restrict__ probs, int* info) {
  const PotrfProb P = probs[blockIdx.x];
  double* A = P.A;
  const int64_t ld = P.lda;
  const int n = P.n;
  __shared__ double dk[PB][PB + 1];
  __shared__ double li[PB][PB + 1];
  __shared__ double lj[PB][PB + 1];
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_fail = 0;
  for (int k0 = 0; k0 < n; k0 += PB) {
    const int kb = min(PB, n - k0);
    for (int e = tid; e < PB * PB; e += blockDim.x) {
      const int i = e % PB, j = e / PB;
      dk[i][j] = (i < kb && j < kb && i >= j) ? A[(k0 + i) + (int64_t)(k0 + j) * ld] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < kb; ++j) {
        if (lane == 0) {
          const double d = dk[j][j];
          if (!(d > 0.0) || !isfinite(d)) {
            if (!s_fail && atomicCAS(P.info ? P.info : info, 0, P.tag + 1) == 0) (P.info ? P.info : info)[1] = P.col0 + k0 + j;
            s_fail = 1;
            dk[j][j] = 1.0;
          } else {
            dk[j][j] = sqrt(d);
          }
        }
        __syncwarp();
        const double dj = dk[j][j];
        if (lane > j && lane < kb) dk[lane][j] /= dj;
        __syncwarp();
        if (lane > j && lane < kb) {
          const double lij = dk[lane][j];
          for (int jj = j + 1; jj <= lane; ++jj) dk[lane][jj] -= lij * dk[jj][j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_fail) return;
    for (int e = tid; e < PB * PB; e += blockDim.x) {
      const int i = e % PB, j = e / PB;
      if (i < kb && j < kb && i >= j) A[(k0 + i) + (int64_t)(k0 + j) * ld] = dk[i][j];
    }
    // panel rows below the diagonal tile: L_ik = A_ik L_kk^{-T}
    for (int i = k0 + kb + tid; i < n; i += blockDim.x) {
      double x[PB];
#pragma unroll
      for (int j = 0; j < PB; ++j) x[j] = (j < kb) ? A[i + (int64_t)(k0 + j) * ld] : 0.0;
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        if (j < kb) {
          double v = x[j];
#pragma unroll
          for (int l = 0; l < j; ++l) v -= x[l] * dk[j][l];
          x[j] = v / dk[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < PB; ++j)
        if (j < kb) A[i + (int64_t)(k0 + j) * ld] = x[j];
    }
    __syncthreads();
    // trailing update of the lower triangle, one 32 x 32 tile at a time
    const int r0 = k0 + kb;
    const int nt = (n - r0 + PB - 1) / PB;
    for (int ti = 0; ti < nt; ++ti) {
      const int i0 = r0 + ti * PB, ib = min(PB, n - i0);
      for (int e = tid; e < PB * PB; e += blockDim.x) {
        const int r = e % PB, l = e / PB;
        li[r][l] = (r < ib && l < kb) ? A[(i0 + r) + (int64_t)(k0 + l) * ld] : 0.0;
      }
      for (int tj = 0; tj <= ti; ++tj) {
        const int j0 = r0 + tj * PB, jb = min(PB, n - j0);
        for (int e = tid; e < PB * PB; e += blockDim.x) {
          const int r = e % PB, l = e / PB;
          lj[r][l] = (r < jb && l < kb) ? A[(j0 + r) + (int64_t)(k0 + l) * ld] : 0.0;
        }
        __syncthreads();
        const int r = tid & 31;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = (tid >> 5) + 8 * q;
          const int gi = i0 + r, gj = j0 + c;
          if (r < ib && c < jb && gi >= gj) {
            double acc = 0.0;
#pragma unroll 8
            for (int l = 0; l < kb; ++l) acc = fma(li[r][l], lj[c][l], acc);
            A[gi + (int64_t)gj * ld] -= acc;
          }
        }
        __syncthreads();
      }
    }
  }
  for (int c = warp; c < n; c += (int)(blockDim.x >> 5))
    for (int i = lane; i < c; i += 32) A[i + (int64_t)c * ld] = 0.0;
}

// Matrices larger than kPotrfBig are factored by blocks of kPotrfNB columns over several
// launches, each covering all of them: Cholesky of the diagonal block (one CTA each), its
// triangular inverse (TRSM on the identity, one warp per column), the panel
// L_ik = A_ik L_kk^{-T} and the trailing update of the lower triangle as grouped GEMMs over
// many CTAs.  One CTA would run the whole O(n^3) factorization at the FP64 rate of a single
// SM.
constexpr int kPotrfBig = 128, kPotrfNB = 64;

static void potrf_one_launch(const Batch<PotrfProb>& b, int* d_info, cudaStream_t s);

static void potrf_blocked(const std::vector<PotrfProb>& big, int* d_info, const char* tag,
                          cudaStream_t s) {
  const int NB = kPotrfNB;
  const size_t np = big.size();
  std::vector<int64_t> soff(np + 1, 0);
  int nmax = 0;
  for (size_t q = 0; q < np; ++q) {
    soff[q + 1] = soff[q] + (int64_t)NB * NB + (int64_t)big[q].n * NB;
    nmax = std::max(nmax, big[q].n);
  }
  DevBuf<double> scratch(std::max<int64_t>(soff[np], 1));
  for (int k0 = 0; k0 < nmax; k0 += NB) {
    Batch<PotrfProb> pd;
    Batch<CopyProb> idb, back;
    Batch<TrsmProb> tb;
    GemmBatch panel, trail;
    pd.tag = tag;
    for (size_t q = 0; q < np; ++q) {
      const PotrfProb& P = big[q];
      if (P.n <= k0) continue;
      const int kb = std::min(NB, P.n - k0);
      const int64_t ld = P.lda;
      double* Akk = P.A + k0 + (int64_t)k0 * ld;
      PotrfProb d = P;
      d.A = Akk;
      d.n = kb;
      d.info = P.info ? P.info : d_info;
      d.col0 = P.col0 + k0;
      pd.push(d);
      const int r0 = k0 + kb, R = P.n - r0;
      if (R <= 0) continue;
      double* W = scratch.p + soff[q];            // kb x kb: L_kk^{-1}
      double* S = W + (int64_t)NB * NB;           // R x kb: the new panel
      CopyProb c;
      c.src = nullptr; c.lds = kb; c.dst = W; c.ldd = kb; c.m = kb; c.n = kb;
      c.trans = 0; c.accumulate = 0; c.alpha = 1.0;
      idb.push(c);
      TrsmProb t;
      t.T = Akk; t.ldt = ld; t.B = W; t.ldb = kb; t.n = kb; t.ncol = kb; t.lower = 1; t.trans = 0;
      tb.push(t);
      double* Ap = P.A + r0 + (int64_t)k0 * ld;
      panel.add(S, R, R, kb, Ap, ld, 0, W, kb, 1, kb, 1.0, 0.0);
      for (int j0 = r0; j0 < P.n; j0 += NB) {
        const int jw = std::min(NB, P.n - j0);
        trail.add(P.A + j0 + (int64_t)j0 * ld, ld, P.n - j0, jw, S + (j0 - r0), R, 0,
                  S + (j0 - r0), R, 1, kb, -1.0, 1.0);
      }
      CopyProb cb;
      cb.src = S; cb.lds = R; cb.dst = Ap; cb.ldd = ld; cb.m = R; cb.n = kb;
      cb.trans = 0; cb.accumulate = 0; cb.alpha = 1.0;
      back.push(cb);
    }
    pd.upload(s);
    potrf_one_launch(pd, d_info, s);
    if (idb.empty()) continue;
    idb.upload(s);
    identity_launch(idb, s);
    tb.tag = "trsm_potrf_inv";
    tb.upload(s);
    trsm_launch(tb, s);
    panel.tag = trail.tag = "gemm_potrf";
    panel.run(s);
    trail.run(s);
    back.upload(s);
    copy_launch(back, s);
  }
  // zeros above the diagonal blocks
  Batch<CopyProb> z;
  for (const auto& P : big)
    for (int j0 = NB; j0 < P.n; j0 += NB) {
      CopyProb c;
      c.src = nullptr; c.lds = j0; c.dst = P.A + (int64_t)j0 * P.lda; c.ldd = P.lda;
      c.m = j0; c.n = std::min(NB, P.n - j0); c.trans = 0; c.accumulate = 0; c.alpha = 1.0;
      z.push(c);
    }
  z.upload(s);
  copy_launch(z, s);
}

void potrf_launch(const Batch<PotrfProb>& b, int* d_info, cudaStream_t s) {
  if (!merging() && !b.empty()) {
    int nmax = 0;
    for (const auto& p : b.h) nmax = std::max(nmax, p.n);
    if (nmax > kPotrfBig) {
      Batch<PotrfProb> small;
      std::vector<PotrfProb> big;
      small.tag = b.tag;
      for (const auto& p : b.h) (p.n > kPotrfBig ? big.push_back(p) : small.push(p));
      if (!small.empty()) {
        small.upload(s);
        potrf_one_launch(small, d_info, s);
      }
      potrf_blocked(big, d_info, b.tag ? b.tag : "potrf", s);
      return;
    }
  }
  potrf_one_launch(b, d_info, s);
}

static void potrf_one_launch(const Batch<PotrfProb>& b, int* d_info, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    std::vector<PotrfProb> h = b.h;
    for (auto& p : h)
      if (!p.info) p.info = d_info;
    const char* tag = b.tag;
    defer_launch("potrf", h, [tag](std::vector<PotrfProb>& all, cudaStream_t st) {
      Batch<PotrfProb> m;
      m.h = std::move(all);
      m.tag = tag;
      m.upload(st);
      potrf_launch(m, nullptr, st);
    });
    return;
  }
  double f = 0.0;
  for (const auto& p : b.h) f += (double)p.n * p.n * p.n / 3.0;
  ProfScope ps(b.tag ? b.tag : "potrf", s, f);
  k_potrf_blk<<<(unsigned)b.size(), 256, 0, s>>>(b.d.p, d_info);
  SPD_LAUNCHED();
}

// ---------------------------------------------------------------------------------------
// triangular solves: one warp per right-hand-side column
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_trsm(const TrsmProb* __restrict__ probs,
                                              const int2* __restrict__ work, int64_t nwork) {
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= nwork) return;
  const int lane = threadIdx.x & 31;
  const int2 it = work[w];
  const TrsmProb P = probs[it.x];
  double* b = P.B + (int64_t)it.y * P.ldb;
  const double* T = P.T;
  const int64_t lt = P.ldt;
  const int n = P.n;
  // op(T)(i, j): element of the matrix actually solved with
  const bool fwd = (P.lower && !P.trans) || (!P.lower && P.trans);
  const bool direct = !P.trans;   // op(T)(i,j) = T[i + j*lt] when not transposed
  if (fwd) {
    for (int j = 0; j < n; ++j) {
      __syncwarp();
      const double xj = b[j] / T[j + j * lt];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int i = j + 1 + lane; i < n; i += 32) {
        const double tij = direct ? T[i + (int64_t)j * lt] : T[j + (int64_t)i * lt];
        b[i] -= tij * xj;
      }
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      __syncwarp();
      const double xj = b[j] / T[j + j * lt];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int i = lane; i < j; i += 32) {
        const double tij = direct ? T[i + (int64_t)j * lt] : T[j + (int64_t)i * lt];
        b[i] -= tij * xj;
      }
    }
  }
}

// Blocked variant: one CTA per (problem, 8 right-hand-side columns) keeps its columns in
// shared memory; 32-row diagonal blocks are solved by one warp from a staged tile, the
// remaining rows are updated by the whole CTA.  The dependent chain is n/32 block steps
// of shared-memory latency instead of n steps of global-memory latency.
constexpr int TRB = 32;

template <int TRC>
__global__ void __launch_bounds__(256) k_trsm_blk(const TrsmProb* __restrict__ probs,
                                                  const int2* __restrict__ work) {
  const int2 it = work[blockIdx.x];
  const TrsmProb P = probs[it.x];
  const int c0 = it.y;
  const int nc = min(TRC, P.ncol - c0);
  const int n = P.n;
  extern __shared__ double sm[];
  double* bs = sm;                        // column c at bs + c * n
  double* td = sm + (size_t)n * TRC;      // 32 x 33 diagonal tile of op(T)
  const double* T = P.T;
  const int64_t lt = P.ldt;
  const bool fwd = (P.lower && !P.trans) || (!P.lower && P.trans);
  const bool direct = !P.trans;
  for (int e = threadIdx.x; e < n * TRC; e += blockDim.x) {
    const int i = e % n, c = e / n;
    bs[e] = (c < nc) ? P.B[i + (int64_t)(c0 + c) * P.ldb] : 0.0;
  }
  __syncthreads();
  const int nb = (n + TRB - 1) / TRB;
  for (int bb = 0; bb < nb; ++bb) {
    const int blk = fwd ? bb : nb - 1 - bb;
    const int j0 = blk * TRB, jb = min(TRB, n - j0);
    for (int e = threadIdx.x; e < TRB * TRB; e += blockDim.x) {
      const int ii = e % TRB, jj = e / TRB;
      double v = 0.0;
      if (ii < jb && jj < jb)
        v = direct ? T[(j0 + ii) + (int64_t)(j0 + jj) * lt] : T[(j0 + jj) + (int64_t)(j0 + ii) * lt];
      td[ii * 33 + jj] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int ii = threadIdx.x;
      // reciprocal diagonal once per block (off the dependent chain)
      const double dinv = (ii < jb) ? 1.0 / td[ii * 33 + ii] : 0.0;
      for (int c = 0; c < nc; ++c) {
        double* b = bs + (size_t)c * n + j0;
        double bi = (ii < jb) ? b[ii] : 0.0;
        if (fwd) {
          for (int jj = 0; jj < jb; ++jj) {
            const double xj = __shfl_sync(0xffffffffu, bi * dinv, jj);
            if (ii == jj) bi = xj;
            if (ii > jj) bi -= td[ii * 33 + jj] * xj;
          }
        } else {
          for (int jj = jb - 1; jj >= 0; --jj) {
            const double xj = __shfl_sync(0xffffffffu, bi * dinv, jj);
            if (ii == jj) bi = xj;
            if (ii < jj) bi -= td[ii * 33 + jj] * xj;
          }
        }
        if (ii < jb) b[ii] = bi;
      }
    }
    __syncthreads();
    const int r0 = fwd ? j0 + jb : 0, r1 = fwd ? n : j0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double acc[TRC];
#pragma unroll
      for (int c = 0; c < TRC; ++c) acc[c] = 0.0;
      if (jb == TRB) {
        // full block: the 32 loads of this row are independent and issued together
        double tv[TRB];
#pragma unroll
        for (int jj = 0; jj < TRB; ++jj)
          tv[jj] = direct ? T[i + (int64_t)(j0 + jj) * lt] : T[(j0 + jj) + (int64_t)i * lt];
#pragma unroll
        for (int jj = 0; jj < TRB; ++jj)
#pragma unroll
          for (int c = 0; c < TRC; ++c) acc[c] = fma(tv[jj], bs[(size_t)c * n + j0 + jj], acc[c]);
      } else {
        for (int jj = 0; jj < jb; ++jj) {
          const double tv = direct ? T[i + (int64_t)(j0 + jj) * lt] : T[(j0 + jj) + (int64_t)i * lt];
#pragma unroll
          for (int c = 0; c < TRC; ++c) acc[c] = fma(tv, bs[(size_t)c * n + j0 + jj], acc[c]);
        }
      }
      for (int c = 0; c < nc; ++c) bs[(size_t)c * n + i] -= acc[c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * TRC; e += blockDim.x) {
    const int i = e % n, c = e / n;
    if (c < nc) P.B[i + (int64_t)(c0 + c) * P.ldb] = bs[e];
  }
}

static constexpr size_t kTrsmMaxSmem = 200 * 1024;

// Work list and variant.  A problem whose n rows of one column fit shared memory goes to
// the blocked kernel, any other to the column-per-warp kernel: the choice depends on the
// problem alone, so that its result is the same in any launch it is part of (the two
// kernels order their operations differently; the blocked kernel's columns per CTA do
// not change any column's arithmetic).  Work items of the blocked kernel come first
// (*nblk of them), variant = its columns per CTA (1, 2, 4 or 8).
static bool trsm_fits_blocked(int n) {
  return (size_t)n * sizeof(double) + TRB * 33 * sizeof(double) <= kTrsmMaxSmem;
}

template <int C>
static void trsm_blk_go(const TrsmProb* probs, const int2* work, int64_t nwork, size_t smem,
                        cudaStream_t s);

// synthetic unit lower-triangular T (1e-3 below the diagonal) and B = 1, for timing
__global__ void k_trsm_synth(double* __restrict__ T, int n, int64_t count, double* __restrict__ B,
                             int64_t nb) {
  const int64_t nt = (int64_t)n * n * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt + nb;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nt) {
      const int64_t q = e % ((int64_t)n * n);
      const int i = (int)(q % n), j = (int)(q / n);
      T[e] = i == j ? 1.0 : (i > j ? 1e-3 : 0.0);
    } else {
      B[e - nt] = 1.0;
    }
  }
}

// Time of the blocked TRSM with v columns per CTA on `count` synthetic n x n problems of
// ncol columns (private stream, CUDA events, two launches after a warm-up).
static double trsm_time_variant(int v, int n, int ncol, int count) {
  cudaStream_t ps;
  SPD_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
  double ms = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    StreamScope sc(ps);
    DevBuf<double> T((size_t)count * n * n), B((size_t)count * n * ncol);
    k_trsm_synth<<<1024, 256, 0, ps>>>(T.p, n, count, B.p, (int64_t)count * n * ncol);
    SPD_LAUNCHED();
    Batch<TrsmProb> bt;
    for (int p = 0; p < count; ++p)
      bt.push(TrsmProb{T.p + (int64_t)p * n * n, n, B.p + (int64_t)p * n * ncol, n, n, ncol, 1, 0});
    bt.upload(ps);
    std::vector<int2> w;
    for (int p = 0; p < count; ++p)
      for (int c = 0; c < ncol; c += v) w.push_back(make_int2(p, c));
    DevBuf<int2> dw;
    dw.upload(w, ps);
    const size_t smem = (size_t)n * v * sizeof(double) + TRB * 33 * sizeof(double);
    auto go = [&]() {
      switch (v) {
        case 1: trsm_blk_go<1>(bt.d.p, dw.p, (int64_t)w.size(), smem, ps); break;
        case 2: trsm_blk_go<2>(bt.d.p, dw.p, (int64_t)w.size(), smem, ps); break;
        case 4: trsm_blk_go<4>(bt.d.p, dw.p, (int64_t)w.size(), smem, ps); break;
        default: trsm_blk_go<8>(bt.d.p, dw.p, (int64_t)w.size(), smem, ps); break;
      }
      SPD_LAUNCHED();
    };
    go();
    SPD_CUDA(cudaEventCreate(&e0));
    SPD_CUDA(cudaEventCreate(&e1));
    SPD_CUDA(cudaEventRecord(e0, ps));
    for (int r = 0; r < 2; ++r) go();
    SPD_CUDA(cudaEventRecord(e1, ps));
    SPD_CUDA(cudaEventSynchronize(e1));
    float f = 0.f;
    SPD_CUDA(cudaEventElapsedTime(&f, e0, e1));
    ms = f / 2.0;
  } catch (...) {
    ms = -1.0;
    cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(ps);
  cudaStreamDestroy(ps);
  return ms;
}

static int pow2_at_least(int64_t x) {
  int p = 1;
  while (p < x && p < (1 << 30)) p *= 2;
  return p;
}

static std::vector<int2> trsm_work(const Batch<TrsmProb>& b, int* variant, size_t* smem,
                                   int64_t* nblk, cudaStream_t s = nullptr) {
  int maxn = 0, maxc = 0, nprob = 0;
  for (const auto& p : b.h)
    if (p.n > 0 && trsm_fits_blocked(p.n)) {
      maxn = std::max(maxn, p.n);
      maxc = std::max(maxc, p.ncol);
      ++nprob;
    }
  int cw = maxc <= 1 ? 1 : (maxc <= 2 ? 2 : (maxc <= 4 ? 4 : 8));
  while (cw > 1 && (size_t)maxn * cw * sizeof(double) + TRB * 33 * sizeof(double) > kTrsmMaxSmem)
    cw /= 2;
  // columns per CTA do not change a column's arithmetic: the width is tuned per device and
  // shape bucket (the rule above when tuning is off, or while the stream is being captured)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (s) cudaStreamIsCapturing(s, &cap);
  const char* forced = std::getenv("SPDHSS_TRSM_COLS");   // 1, 2, 4 or 8: a fixed width
  const int fw = forced ? std::atoi(forced) : 0;
  if (fw == 1 || fw == 2 || fw == 4 || fw == 8) {
    cw = std::min(cw, fw);
  } else if (nprob > 0 && cap == cudaStreamCaptureStatusNone && tuning_enabled()) {
    const int bn = pow2_at_least(maxn), bc = std::min(pow2_at_least(maxc), 64);
    const int bp = std::min(pow2_at_least(nprob), 4096);
    std::vector<int> cands;
    for (int v : {1, 2, 4, 8})
      if (v <= cw) cands.push_back(v);
    const std::string key = "trsm_blk n" + std::to_string(bn) + " c" + std::to_string(bc) +
                            " p" + std::to_string(bp);
    // the synthetic set: the bucket's problem count, at most 512 problems and 32 MB
    const int64_t fit = std::max<int64_t>(1, (int64_t(32) << 20) / ((int64_t)maxn * maxn * 8));
    const int count = (int)std::min<int64_t>(std::min<int64_t>(bp, 512), fit);
    const int tn = maxn, tc = maxc;
    cw = tuned_variant(key, cands, cw, [&](int v) { return trsm_time_variant(v, tn, tc, count); });
  }
  *variant = cw;
  *smem = (size_t)maxn * cw * sizeof(double) + TRB * 33 * sizeof(double);
  std::vector<int2> work;
  for (int p = 0; p < (int)b.size(); ++p)
    if (b.h[p].n > 0 && trsm_fits_blocked(b.h[p].n))
      for (int c = 0; c < b.h[p].ncol; c += cw) work.push_back(make_int2(p, c));
  *nblk = (int64_t)work.size();
  for (int p = 0; p < (int)b.size(); ++p)
    if (b.h[p].n > 0 && !trsm_fits_blocked(b.h[p].n))
      for (int c = 0; c < b.h[p].ncol; ++c) work.push_back(make_int2(p, c));
  return work;
}

template <int C>
static void trsm_blk_go(const TrsmProb* probs, const int2* work, int64_t nwork, size_t smem,
                        cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_trsm_blk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsmMaxSmem);
  });
  k_trsm_blk<C><<<(unsigned)nwork, 256, smem, s>>>(probs, work);
}

static void trsm_go(const TrsmProb* probs, const int2* work, int64_t nwork, int64_t nblk,
                    int variant, size_t smem, cudaStream_t s) {
  if (nblk > 0) {
    switch (variant) {
      case 1: trsm_blk_go<1>(probs, work, nblk, smem, s); break;
      case 2: trsm_blk_go<2>(probs, work, nblk, smem, s); break;
      case 4: trsm_blk_go<4>(probs, work, nblk, smem, s); break;
      default: trsm_blk_go<8>(probs, work, nblk, smem, s); break;
    }
    SPD_LAUNCHED();
  }
  if (nwork > nblk) {
    k_trsm<<<ceil_div(nwork - nblk, 8), 256, 0, s>>>(probs, work + nblk, nwork - nblk);
    SPD_LAUNCHED();
  }
}

void trsm_prepare(Batch<TrsmProb>& b, cudaStream_t s) {
  std::vector<int2> w = trsm_work(b, &b.variant, &b.smem, &b.nfirst, s);
  b.work.upload(w, s);
  b.nwork = (int64_t)w.size();
}

void trsm_launch(const Batch<TrsmProb>& b, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    const char* tag = b.tag;
    defer_launch("trsm", b.h, [tag](std::vector<TrsmProb>& all, cudaStream_t st) {
      Batch<TrsmProb> m;
      m.h = std::move(all);
      m.tag = tag;
      m.upload(st);
      trsm_launch(m, st);
    });
    return;
  }
  double f = 0.0;
  for (const auto& p : b.h) f += (double)p.n * p.n * p.ncol;
  if (b.nwork >= 0) {
    if (b.nwork == 0) return;
    ProfScope ps(b.tag ? b.tag : "trsm", s, f);
    trsm_go(b.d.p, b.work.p, b.nwork, b.nfirst, b.variant, b.smem, s);
    return;
  }
  int variant;
  size_t smem;
  int64_t nblk;
  std::vector<int2> work = trsm_work(b, &variant, &smem, &nblk, s);
  if (work.empty()) return;
  DevBuf<int2> dw;
  dw.upload(work, s);
  {
    ProfScope ps(b.tag ? b.tag : "trsm", s, f);
    trsm_go(b.d.p, dw.p, (int64_t)work.size(), nblk, variant, smem, s);
  }
}

// ---------------------------------------------------------------------------------------
// Householder QR with column pivoting; a cluster of C CTAs shares one matrix, CTA q owning
// the column positions p with p % C == q.  Pivot norms are downdated after every step and
// recomputed from the trailing rows when the downdate loses accuracy (qr_downdate below),
// or recomputed at every step when the problem asks for it (downdate = 0); ties go to the
// lowest position.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void argmax_merge(double& v, int& p, double v2, int p2) {
  if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Column norms are downdated after every step, |a_p(j+1:)|^2 = |a_p(j:)|^2 - R_jp^2, and
// recomputed from the column when cancellation makes the downdate unreliable: when
// (1 - (R_jp/vn1)^2) (vn1/vn2)^2 falls to sqrt(eps) or below, vn2 being the norm at the
// last recomputation (the safeguard of LAPACK's column-pivoted QR, Drmac and Bujanovic).
// Returns 1 when the caller must recompute vn1 = vn2 = |a_p(j+1:)|.
constexpr double kQrTol3z = 1.0536712127723509e-08;   // sqrt(2^-53)

__device__ __forceinline__ int qr_downdate(double rjp, double& vn1, double vn2) {
  if (vn1 == 0.0) return 0;
  double t = fabs(rjp) / vn1;
  t = fmax(1.0 - t * t, 0.0);
  const double r = vn1 / vn2;
  if (t * r * r <= kQrTol3z) return 1;
  vn1 *= sqrt(t);
  return 0;
}

template <int LPC>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
  for (int o = LPC / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Columns in global memory.  Every reduction has the shape and order of k_geqp3_smem with
// the same LPC (lanes per column), so the two kernels give bit-identical factorizations
// and the choice between them (and of the cluster size) does not change any result.
template <int LPC>
__global__ void __launch_bounds__(256) k_geqp3(const QrProb* __restrict__ probs, int pivot) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const QrProb P = probs[blockIdx.x / C];
  extern __shared__ double s_v[];
  __shared__ double s_wv[8];
  __shared__ int s_wp[8];
  __shared__ double s_cv;
  __shared__ int s_cp;
  __shared__ double s_first, s_tau, s_scale;
  __shared__ int s_stop, s_piv;
  const int m = P.m, n = P.n;
  const int kmax = min(P.kmax, min(m, n));
  double* A = P.A;
  const int64_t ld = P.lda;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;

  // first owned position >= start
  auto first_owned = [&](int start) { return start + (((q - start) % C) + C) % C; };

  if (pivot) {
    int t = 0;
    for (int p = first_owned(0); p < n; p += C, ++t) {
      if (t % nw != warp) continue;
      double s = 0.0;
      for (int i = lane; i < m; i += 32) { const double a = A[i + (int64_t)p * ld]; s += a * a; }
      s = warp_sum(s);
      if (lane == 0) { P.norms[p] = sqrt(s); P.norms[n + p] = P.norms[p]; P.piv[p] = p; }
    }
  }
  __threadfence();
  cl.sync();

  int j = 0;
  for (; j < kmax; ++j) {
    if (pivot) {
      double bv = -1.0;
      int bp = n;
      int t = 0;
      for (int p = first_owned(j); p < n; p += C, ++t)
        if (t % nw == warp) argmax_merge(bv, bp, P.norms[p], p);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
        argmax_merge(bv, bp, v2, p2);
      }
      if (lane == 0) { s_wv[warp] = bv; s_wp[warp] = bp; }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) argmax_merge(bv, bp, s_wv[w], s_wp[w]);
        s_cv = bv;
        s_cp = bp;
      }
      cl.sync();
      if (threadIdx.x == 0) {
        double gv = -1.0;
        int gp = n;
        for (int r = 0; r < C; ++r) {
          const double* pv = cl.map_shared_rank(&s_cv, r);
          const int* pp = cl.map_shared_rank(&s_cp, r);
          argmax_merge(gv, gp, *pv, *pp);
        }
        if (j == 0) s_first = gv;
        s_stop = (gv <= 0.0) || (gv <= P.rtol * s_first) || (gp >= n);
        s_piv = gp;
      }
      __syncthreads();
      if (s_stop) break;
    } else {
      if (threadIdx.x == 0) s_piv = j;
      __syncthreads();
    }
    const int pc = s_piv;
    if (q == 0) {
      if (pc != j) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          const double a = A[i + (int64_t)j * ld];
          A[i + (int64_t)j * ld] = A[i + (int64_t)pc * ld];
          A[i + (int64_t)pc * ld] = a;
        }
        if (threadIdx.x == 0) {
          const int tp = P.piv[j]; P.piv[j] = P.piv[pc]; P.piv[pc] = tp;
          const double tn = P.norms[j]; P.norms[j] = P.norms[pc]; P.norms[pc] = tn;
          const double t2 = P.norms[n + j]; P.norms[n + j] = P.norms[n + pc]; P.norms[n + pc] = t2;
        }
      }
      __syncthreads();
      double s = 0.0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        const double a = A[i + (int64_t)j * ld];
        s += a * a;
      }
      s = warp_sum(s);
      if (lane == 0) s_wv[warp] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += s_wv[w];
        const double normx = sqrt(tot);
        const double alpha = A[j + (int64_t)j * ld];
        double tau = 0.0, beta = alpha, scale = 0.0;
        if (normx > 0.0) {
          beta = alpha >= 0.0 ? -normx : normx;
          scale = 1.0 / (alpha - beta);
          tau = (beta - alpha) / beta;
        }
        s_tau = tau;
        s_scale = scale;
        P.tau[j] = tau;
        A[j + (int64_t)j * ld] = beta;
      }
      __syncthreads();
      const double scale = s_scale;
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + (int64_t)j * ld] *= scale;
      if (C > 1) __threadfence();
    }
    cl.sync();
    const double tau = P.tau[j];
    const int len = m - j;
    for (int i = threadIdx.x; i < len; i += blockDim.x)
      s_v[i] = (i == 0) ? 1.0 : A[j + i + (int64_t)j * ld];
    __syncthreads();
    {
      // LPC lanes per column, G = 32 / LPC columns per warp at a time (as k_geqp3_smem)
      constexpr int G = 32 / LPC;
      const int g = lane / LPC, sl = lane % LPC;
      const unsigned FULL = 0xffffffffu;
      const int p0 = first_owned(j + 1);
      const int cnt = (p0 < n) ? (n - p0 + C - 1) / C : 0;
      for (int t0 = warp * G; t0 < cnt; t0 += nw * G) {
        const int t = t0 + g;
        const bool act = t < cnt;
        const int p = p0 + (act ? t : 0) * C;
        double* col = A + j + (int64_t)p * ld;
        double w = 0.0;
        if (act && tau != 0.0) {
          double w0 = 0.0, w1 = 0.0;
          int i = sl;
          for (; i + LPC < len; i += 2 * LPC) {
            w0 = fma(s_v[i], col[i], w0);
            w1 = fma(s_v[i + LPC], col[i + LPC], w1);
          }
          if (i < len) w0 = fma(s_v[i], col[i], w0);
          w = w0 + w1;
        }
        w = group_sum<LPC>(w) * tau;
        double sq = 0.0;
        if (act && tau != 0.0) {
          if (pivot && !P.downdate) {   // update and recompute the norm in one pass
            for (int i = sl; i < len; i += LPC) {
              const double a = col[i] - w * s_v[i];
              col[i] = a;
              if (i > 0) sq += a * a;
            }
          } else {
#pragma unroll 4
            for (int i = sl; i < len; i += LPC) col[i] -= w * s_v[i];
          }
        }
        if (!pivot) continue;
        int rc = 1;
        if (P.downdate || tau == 0.0) {
          if (P.downdate) {
            rc = 0;
            if (act && sl == 0) {
              double v1 = P.norms[p];
              rc = qr_downdate(col[0], v1, P.norms[n + p]);
              P.norms[p] = v1;
            }
            rc = __shfl_sync(FULL, rc, g * LPC);
          }
          if (act && rc)
            for (int i = 1 + sl; i < len; i += LPC) sq += col[i] * col[i];
        }
        sq = group_sum<LPC>(sq);
        if (act && sl == 0 && rc) {
          P.norms[p] = sqrt(sq);
          if (P.downdate) P.norms[n + p] = P.norms[p];
        }
      }
    }
    if (C > 1) __threadfence();   // peers read the updated columns from global memory
    cl.sync();
  }
  if (q == 0 && threadIdx.x == 0) *P.rank = j;
  // keep every CTA of the cluster alive until peers are done reading its shared memory
  cl.sync();
}

// ---------------------------------------------------------------------------------------
// The same factorization with every column resident in shared memory: a cluster of C CTAs
// shares one matrix, CTA q holding the columns c with c % C == q for the whole
// factorization (position swaps only permute a replicated position <-> column map).  Per
// step: each CTA proposes its best remaining column, the cluster agrees on the pivot
// (largest norm, lowest position), the owner forms the reflector in its shared memory, the
// other CTAs copy it over DSMEM, and every CTA updates and re-measures its own columns.
// Every reduction has the shape and order of k_geqp3, so the results are bit-identical.
// ---------------------------------------------------------------------------------------
constexpr size_t kQrSmemBudget = 200 * 1024;

struct QrSmemLayout {
  int nown, ldm;
  size_t cols, norms, norms2, pos2col, col2pos, v, total;
};
__host__ __device__ inline QrSmemLayout qr_smem_layout(int m, int n, int C) {
  QrSmemLayout L;
  L.nown = (n + C - 1) / C;
  L.ldm = m + (m & 1);
  L.cols = 0;
  L.norms = L.cols + (size_t)L.nown * L.ldm * sizeof(double);
  L.norms2 = L.norms + (size_t)L.nown * sizeof(double);
  L.pos2col = L.norms2 + (size_t)L.nown * sizeof(double);
  L.col2pos = L.pos2col + (size_t)n * sizeof(int);
  L.v = (L.col2pos + (size_t)n * sizeof(int) + 15) & ~(size_t)15;
  L.total = L.v + (size_t)L.ldm * sizeof(double);
  return L;
}

template <int LPC>
__global__ void __launch_bounds__(256) k_geqp3_smem(const QrProb* __restrict__ probs, int mmax,
                                                    int nmax) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const QrProb P = probs[blockIdx.x / C];
  extern __shared__ __align__(16) unsigned char smem_qr[];
  const QrSmemLayout Ly = qr_smem_layout(mmax, nmax, C);
  double* cols = reinterpret_cast<double*>(smem_qr + Ly.cols);
  double* norms = reinterpret_cast<double*>(smem_qr + Ly.norms);     // downdated norms
  double* norms2 = reinterpret_cast<double*>(smem_qr + Ly.norms2);   // at the last recompute
  int* pos2col = reinterpret_cast<int*>(smem_qr + Ly.pos2col);
  int* col2pos = reinterpret_cast<int*>(smem_qr + Ly.col2pos);
  double* s_v = reinterpret_cast<double*>(smem_qr + Ly.v);   // the reflector, m - j entries
  __shared__ double s_wv[8];
  __shared__ double s_cv[2];
  __shared__ int s_cp[2];
  __shared__ double s_first, s_tau;
  __shared__ int s_stop, s_piv;
  const int m = P.m, n = P.n;
  const int kmax = min(P.kmax, min(m, n));
  const int64_t ld = P.lda;
  const int ldm = Ly.ldm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nown = (q < n) ? (n - q + C - 1) / C : 0;   // owned columns c = q + t * C

  for (int t = warp; t < nown; t += nw) {
    const double* src = P.A + (int64_t)(q + t * C) * ld;
    double* dst = cols + (int64_t)t * ldm;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double a = src[i];
      dst[i] = a;
      s += a * a;
    }
    s = warp_sum(s);
    if (lane == 0) { norms[t] = sqrt(s); norms2[t] = norms[t]; }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) { pos2col[i] = i; col2pos[i] = i; }
  cl.sync();

  int j = 0;
  for (; j < kmax; ++j) {
    // this CTA's candidate: largest norm among its columns at positions >= j, lowest position
    if (warp == 0) {
      double bv = -1.0;
      int bp = n;
      for (int t = lane; t < nown; t += 32) {
        const int p = col2pos[q + t * C];
        if (p >= j) argmax_merge(bv, bp, norms[t], p);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
        argmax_merge(bv, bp, v2, p2);
      }
      if (lane == 0) { s_cv[j & 1] = bv; s_cp[j & 1] = bp; }
    }
    cl.sync();
    if (warp == 0) {
      // the candidates of the C CTAs, one per lane (the merge order does not matter: the
      // order (largest value, then lowest position) is total)
      double gv = -1.0;
      int gp = n;
      if (lane < C) {
        gv = *cl.map_shared_rank(&s_cv[j & 1], lane);
        gp = *cl.map_shared_rank(&s_cp[j & 1], lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, gv, o);
        const int p2 = __shfl_xor_sync(0xffffffffu, gp, o);
        argmax_merge(gv, gp, v2, p2);
      }
      if (lane == 0) {
        if (j == 0) s_first = gv;
        s_stop = (gv <= 0.0) || (gv <= P.rtol * s_first) || (gp >= n);
        if (!s_stop) {
          // positions j and gp exchange their columns
          const int cj = pos2col[j], cp = pos2col[gp];
          pos2col[j] = cp; pos2col[gp] = cj;
          col2pos[cp] = j; col2pos[cj] = gp;
          s_piv = cp;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int cp = s_piv;
    const int owner = cp % C;
    if (q == owner) {
      double* x = cols + (int64_t)(cp / C) * ldm;
      double s = 0.0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) { const double a = x[i]; s += a * a; }
      s = warp_sum(s);
      if (lane == 0) s_wv[warp] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += s_wv[w];
        const double normx = sqrt(tot);
        const double alpha = x[j];
        double tau = 0.0, beta = alpha, scale = 0.0;
        if (normx > 0.0) {
          beta = alpha >= 0.0 ? -normx : normx;
          scale = 1.0 / (alpha - beta);
          tau = (beta - alpha) / beta;
        }
        s_tau = tau;
        s_wv[0] = scale;
        P.tau[j] = tau;
        x[j] = beta;
      }
      __syncthreads();
      const double scale = s_wv[0];
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) x[i] *= scale;
    }
    cl.sync();
    // the reflector v (v_0 = 1) and tau from the owner's shared memory
    const int len = m - j;
    {
      const double* xo = cl.map_shared_rank(cols + (int64_t)(cp / C) * ldm, owner);
      for (int i = threadIdx.x; i < len; i += blockDim.x) s_v[i] = (i == 0) ? 1.0 : xo[j + i];
      if (threadIdx.x == 0) s_wv[1] = *cl.map_shared_rank(&s_tau, owner);
    }
    __syncthreads();
    const double tau = s_wv[1];
    // LPC lanes per column, 32 / LPC columns per warp at a time: short columns spend their
    // FP64 issue on the products rather than on reduction trees
    constexpr int G = 32 / LPC;
    const int g = lane / LPC, sl = lane % LPC;
    const unsigned FULL = 0xffffffffu;
    for (int t0 = warp * G; t0 < nown; t0 += nw * G) {
      const int t = t0 + g;
      const bool act = t < nown && col2pos[q + min(t, nown - 1) * C] > j;
      double* col = cols + (int64_t)min(t, nown - 1) * ldm + j;
      double w = 0.0;
      if (act && tau != 0.0) {
        double w0 = 0.0, w1 = 0.0;
        int i = sl;
        for (; i + LPC < len; i += 2 * LPC) {
          w0 = fma(s_v[i], col[i], w0);
          w1 = fma(s_v[i + LPC], col[i + LPC], w1);
        }
        if (i < len) w0 = fma(s_v[i], col[i], w0);
        w = w0 + w1;
      }
      w = group_sum<LPC>(w) * tau;
      double s = 0.0;
      if (act && tau != 0.0) {
        if (!P.downdate) {   // update and recompute the norm in one pass
          for (int i = sl; i < len; i += LPC) {
            const double a = col[i] - w * s_v[i];
            col[i] = a;
            if (i > 0) s += a * a;
          }
        } else {
#pragma unroll 4
          for (int i = sl; i < len; i += LPC) col[i] -= w * s_v[i];
        }
      }
      int rc = 1;
      if (P.downdate || tau == 0.0) {
        if (P.downdate) {
          rc = 0;
          if (act && sl == 0) rc = qr_downdate(col[0], norms[t], norms2[t]);
          rc = __shfl_sync(FULL, rc, g * LPC);
        }
        if (act && rc)
          for (int i = 1 + sl; i < len; i += LPC) s += col[i] * col[i];
      }
      s = group_sum<LPC>(s);
      if (act && sl == 0 && rc) {
        norms[t] = sqrt(s);
        if (P.downdate) norms2[t] = norms[t];
      }
    }
    __syncthreads();
  }
  // columns to their final positions, the position -> column map, the rank
  for (int t = warp; t < nown; t += nw) {
    const int c = q + t * C;
    const int p = col2pos[c];
    double* dst = P.A + (int64_t)p * ld;
    const double* src = cols + (int64_t)t * ldm;
    for (int i = lane; i < m; i += 32) dst[i] = src[i];
    if (lane == 0) {
      P.piv[p] = c;
      P.norms[p] = norms[t];
    }
  }
  if (q == 0 && threadIdx.x == 0) *P.rank = j;
  // keep every CTA of the cluster alive until peers are done reading its shared memory
  cl.sync();
}

// Cluster size for the shared-memory variant, 0 to use k_geqp3.  A cluster spends C SMs
// and two cluster barriers per step on one matrix: that pays when the batch has too few
// matrices to fill the GPU one CTA each (measured on the H^2 ID: 3D leaves and the level
// above at n = 4096 gain 1.4x, batches of 500+ full-rank leaves lose 2-3x); a matrix that
// fits one CTA's shared memory always gains.
static int geqp3_smem_cluster(int mmax, int nmax, size_t nprob) {
  for (int C = 1; C <= 8; C *= 2)
    if (qr_smem_layout(mmax, nmax, C).total <= kQrSmemBudget)
      return (C == 1 || nprob <= 2 * 152) ? C : 0;
  return 0;
}

// pivoted QRs of several instances: the largest cluster and row count of the group
struct DeferredQr : Deferred {
  std::vector<QrProb> h;
  int pivot = 1, cluster = 1, max_m = 1;
  const char* tag = nullptr;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    Batch<QrProb> m;
    m.tag = tag;
    int cl = 1, mm = 1;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredQr*>(d);
      m.h.insert(m.h.end(), x->h.begin(), x->h.end());
      cl = std::max(cl, x->cluster);
      mm = std::max(mm, x->max_m);
    }
    m.upload(s);
    geqp3_launch(m, pivot, cl, mm, s);
  }
};

// lanes per column of a problem: rows per lane at least 8 where the columns are short.  A
// function of the problem alone: the factorization's arithmetic depends on it and on
// nothing else of the launch.
static int qr_lpc(int m) { return m <= 64 ? 8 : (m <= 128 ? 16 : 32); }

static int geqp3_launch_lpc(const Batch<QrProb>& b, int pivot, int cluster, int max_m, int lpc,
                            cudaStream_t s);

int geqp3_launch(const Batch<QrProb>& b, int pivot, int cluster, int max_m, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return -1; }
  if (!merging()) {
    int slot = -1;
    for (int lpc : {8, 16, 32}) {
      Batch<QrProb> sub;
      sub.tag = b.tag;
      int mm = 1;
      for (const auto& q : b.h)
        if (qr_lpc(q.m) == lpc) { sub.push(q); mm = std::max(mm, q.m); }
      if (sub.empty()) continue;
      if (sub.size() == b.size()) return geqp3_launch_lpc(b, pivot, cluster, max_m, lpc, s);
      sub.upload(s);
      const int sl = geqp3_launch_lpc(sub, pivot, cluster, std::min(max_m, mm), lpc, s);
      if (slot < 0) slot = sl;
    }
    return slot;
  }
  return geqp3_launch_lpc(b, pivot, cluster, max_m, 0, s);
}

static int geqp3_launch_lpc(const Batch<QrProb>& b, int pivot, int cluster, int max_m, int lpc,
                            cudaStream_t s) {
  if (merging()) {
    std::unique_ptr<DeferredQr> d(new DeferredQr());
    d->h = b.h;
    d->pivot = pivot;
    d->cluster = cluster;
    d->max_m = max_m;
    d->tag = b.tag;
    merge_ctx().m->submit(pivot ? "geqp3" : "geqrf", std::move(d));
    return -1;
  }
  // the largest factorizations first (CTAs start in index order), so that they do not
  // form the tail of the launch
  DevBuf<QrProb> sorted;
  const QrProb* dprobs = b.d.p;
  if (b.size() > 1) {
    std::vector<QrProb> h = b.h;
    auto cost = [](const QrProb& q) {
      const double k = std::min(q.kmax, std::min(q.m, q.n));
      return (double)q.m * q.n * k;
    };
    std::stable_sort(h.begin(), h.end(),
                     [&](const QrProb& x, const QrProb& y) { return cost(x) > cost(y); });
    sorted.upload(h, s);
    dprobs = sorted.p;
  }
  if (pivot) {
    int mmax = 1, nmax = 1;
    for (const auto& p : b.h) { mmax = std::max(mmax, p.m); nmax = std::max(nmax, p.n); }
    const int C = geqp3_smem_cluster(mmax, nmax, b.size());
    if (C > 0) {
      const size_t sm = qr_smem_layout(mmax, nmax, C).total;
      static std::once_flag once_s;
      std::call_once(once_s, [] {
        cudaFuncSetAttribute(k_geqp3_smem<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kQrSmemBudget);
        cudaFuncSetAttribute(k_geqp3_smem<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kQrSmemBudget);
        cudaFuncSetAttribute(k_geqp3_smem<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kQrSmemBudget);
      });
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(b.size() * C), 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = sm;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      ProfScope ps(b.tag ? b.tag : "geqp3", s);
      if (lpc == 8)
        SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3_smem<8>, dprobs, mmax, nmax));
      else if (lpc == 16)
        SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3_smem<16>, dprobs, mmax, nmax));
      else
        SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3_smem<32>, dprobs, mmax, nmax));
      SPD_LAUNCHED();
      return ps.slot;
    }
  }
  cluster = std::max(1, std::min(cluster, 8));
  const size_t smem = (size_t)std::max(1, max_m) * sizeof(double);
  SPD_REQUIRE(smem <= 200 * 1024, "geqp3: matrix too tall for the shared-memory reflector");
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_geqp3<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    cudaFuncSetAttribute(k_geqp3<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    cudaFuncSetAttribute(k_geqp3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b.size() * cluster), 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int slot;
  {
    ProfScope ps(b.tag ? b.tag : (pivot ? "geqp3" : "geqrf"), s);
    slot = ps.slot;
    if (lpc == 8) SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3<8>, dprobs, pivot));
    else if (lpc == 16) SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3<16>, dprobs, pivot));
    else SPD_CUDA(cudaLaunchKernelEx(&cfg, k_geqp3<32>, dprobs, pivot));
    SPD_LAUNCHED();
  }
  return slot;
}

// ---------------------------------------------------------------------------------------
// Two stacked upper triangles reduced to one: column j of [R1; R2] has its non-zeros in
// row j of R1 and rows 0..j of R2, so its reflector has j + 2 entries and touches only
// those rows of the later columns.  Both triangles are held packed in shared memory
// (column p: rows 0..p at p (p + 1) / 2).  Column p has a group of lanes of its own
// (col_group_lanes); the reflector is unnormalized as in k_proxy_qr
// (A <- A - c u (u^T A), c = -1 / (beta u_0)), and the group of column j + 1 forms the
// next reflector's scalars right after its update, so a step costs one barrier.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double tri_scalars(double* d, double n2_rest, double* u0_out) {
  const double alpha = *d;
  const double normx = sqrt(fma(alpha, alpha, n2_rest));
  double beta = alpha, c = 0.0, u0 = 0.0;
  if (normx > kHhMinNorm) {
    beta = alpha >= 0.0 ? -normx : normx;
    u0 = alpha - beta;
    c = -1.0 / (beta * u0);
  }
  *d = beta;
  *u0_out = u0;
  return c;
}

__global__ void __launch_bounds__(256) k_tri_merge(const TriMergeProb* __restrict__ probs) {
  const TriMergeProb P = probs[blockIdx.x];
  const int m = P.m;
  extern __shared__ double sT[];
  const int tri = m * (m + 1) / 2;
  double* T1 = sT;
  double* T2 = sT + tri;
  __shared__ double s_c[2], s_u0[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int lanes = col_group_lanes(m), gpw = 32 / lanes;
  const int g = tid / lanes, sl = tid % lanes;
  const int g_lo = warp * gpw, g_hi = g_lo + gpw - 1;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, p = e / m;
    if (i <= p) {
      T1[p * (p + 1) / 2 + i] = P.R1[i + (int64_t)p * m];
      T2[p * (p + 1) / 2 + i] = P.R2[i + (int64_t)p * m];
    }
  }
  __syncthreads();
  if (tid == 0) s_c[0] = tri_scalars(T1, T2[0] * T2[0], &s_u0[0]);
  __syncthreads();
  const int gc = min(g, m - 1);
  double* c1 = T1 + gc * (gc + 1) / 2;   // column g of R1 (rows 0..g)
  double* c2 = T2 + gc * (gc + 1) / 2;   // column g of R2
  for (int j = 0; j < m; ++j) {
    if (g_hi > j && g_lo < m) {   // a warp with a column > j (warp-uniform)
      const bool act = g > j && g < m;
      const double c = s_c[j & 1], u0 = s_u0[j & 1];
      const double* u2 = T2 + j * (j + 1) / 2;   // rows 0..j of R2's column j
      const bool next = g == j + 1;              // this column forms the next reflector
      double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
      if (act && c != 0.0) {
        if (sl == 0) w0 = u0 * c1[j];
        int i = sl;
        for (; i + 3 * lanes <= j; i += 4 * lanes) {   // four independent loads per lane
          w0 = fma(u2[i], c2[i], w0);
          w1 = fma(u2[i + lanes], c2[i + lanes], w1);
          w2 = fma(u2[i + 2 * lanes], c2[i + 2 * lanes], w2);
          w3 = fma(u2[i + 3 * lanes], c2[i + 3 * lanes], w3);
        }
        for (; i <= j; i += lanes) w0 = fma(u2[i], c2[i], w0);
      }
      const double w = group_sum_n((w0 + w1) + (w2 + w3), lanes) * c;
      double sq = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;   // next: squares of rows 0..j + 1
      if (act && c != 0.0) {
        if (sl == 0) c1[j] -= w * u0;
        int k = sl;
        for (; k + 3 * lanes <= j; k += 4 * lanes) {   // the column and u are disjoint
          const double a0 = c2[k], a1 = c2[k + lanes], a2 = c2[k + 2 * lanes], a3 = c2[k + 3 * lanes];
          const double v0 = u2[k], v1 = u2[k + lanes], v2 = u2[k + 2 * lanes], v3 = u2[k + 3 * lanes];
          const double b0 = a0 - w * v0, b1 = a1 - w * v1, b2 = a2 - w * v2, b3 = a3 - w * v3;
          c2[k] = b0; c2[k + lanes] = b1; c2[k + 2 * lanes] = b2; c2[k + 3 * lanes] = b3;
          if (next) {
            sq = fma(b0, b0, sq);
            q1 = fma(b1, b1, q1);
            q2 = fma(b2, b2, q2);
            q3 = fma(b3, b3, q3);
          }
        }
        for (; k <= j; k += lanes) {
          const double b = c2[k] - w * u2[k];
          c2[k] = b;
          if (next) sq = fma(b, b, sq);
        }
        sq = (sq + q1) + (q2 + q3);
      } else if (next) {
        for (int k = sl; k <= j; k += lanes) sq = fma(c2[k], c2[k], sq);
      }
      if (g_lo <= j + 1 && j + 1 <= g_hi && j + 1 < m) {   // the warp of column j + 1
        if (next && sl == (j + 1) % lanes) sq = fma(c2[j + 1], c2[j + 1], sq);
        sq = group_sum_n(sq, lanes);
        if (next && sl == 0) s_c[(j + 1) & 1] = tri_scalars(c1 + j + 1, sq, &s_u0[(j + 1) & 1]);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, q = e / m;
    P.R1[i + (int64_t)q * m] = (i <= q) ? T1[q * (q + 1) / 2 + i] : 0.0;
  }
}

// ---------------------------------------------------------------------------------------
// Column-pivoted QR of a small matrix (m, n <= kSmallQr), one CTA, every column resident
// in shared memory with a lane group of its own (col_group_lanes): per step the CTA agrees
// on the pivot (largest downdated norm, lowest position), the pivot column's group forms
// the reflector from the exact norm of its trailing rows and applies the stop test
// |R_kk| <= rtol |R_00|, and every later column is updated and its norm downdated
// (recomputed when the downdate loses accuracy, qr_downdate).  Positions are permuted
// through a column <-> position map; the columns go to their final positions at the end.
// ---------------------------------------------------------------------------------------
constexpr int kSmallQr = 160;

__global__ void __launch_bounds__(256) k_geqp3_small(const QrProb* __restrict__ probs) {
  const QrProb P = probs[blockIdx.x];
  const int m = P.m, n = P.n;
  const int lanes = col_group_lanes(n), ld = col_group_ld(m, lanes), gpw = 32 / lanes;
  extern __shared__ double sA[];   // m x n, column-major, ld
  __shared__ double s_vn1[kSmallQr], s_vn2[kSmallQr], s_diag[kSmallQr];
  __shared__ int s_pos[kSmallQr], s_col[kSmallQr];   // column -> position, position -> column
  __shared__ double s_wv[8];
  __shared__ int s_wp[8];
  __shared__ double s_c, s_first;
  __shared__ int s_piv, s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid / lanes, sl = tid % lanes;
  const bool own = g < n;
  const unsigned FULL = 0xffffffffu;
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int i = e % m, c = e / m;
    sA[i + (int64_t)c * ld] = P.A[i + (int64_t)c * P.lda];
  }
  for (int c = tid; c < n; c += blockDim.x) { s_pos[c] = c; s_col[c] = c; }
  __syncthreads();
  {
    double sq = 0.0;
    if (own)
      for (int i = sl; i < m; i += lanes) sq += sA[i + (int64_t)g * ld] * sA[i + (int64_t)g * ld];
    sq = group_sum_n(sq, lanes);
    if (own && sl == 0) { s_vn1[g] = sqrt(sq); s_vn2[g] = s_vn1[g]; }
  }
  __syncthreads();
  const int kmax = min(P.kmax, min(m, n));
  int j = 0;
  for (; j < kmax; ++j) {
    // pivot: the largest downdated norm among positions >= j, ties to the lowest position
    double bv = -1.0;
    int bp = n;
    if (own && sl == 0 && s_pos[g] >= j) { bv = s_vn1[g]; bp = s_pos[g]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(FULL, bv, o);
      const int p2 = __shfl_xor_sync(FULL, bp, o);
      argmax_merge(bv, bp, v2, p2);
    }
    if (lane == 0) { s_wv[warp] = bv; s_wp[warp] = bp; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmax_merge(bv, bp, s_wv[w], s_wp[w]);
      if (bp >= n) {   // no comparable norm left (NaN): stop
        s_stop = 1;
        s_piv = -1;
      } else {
        const int cp = s_col[bp], cj = s_col[j];
        s_col[j] = cp; s_col[bp] = cj;
        s_pos[cp] = j; s_pos[cj] = bp;
        s_piv = cp;
      }
    }
    __syncthreads();
    const int cp = s_piv;
    if (cp < 0) break;
    if (warp == cp / gpw) {   // the pivot column's group: exact norm, reflector, stop test
      double sq = 0.0;
      if (g == cp)
        for (int i = j + sl; i < m; i += lanes) sq += sA[i + (int64_t)cp * ld] * sA[i + (int64_t)cp * ld];
      sq = group_sum_n(sq, lanes);
      if (g == cp && sl == 0) {
        const double normx = sqrt(sq);
        if (j == 0) s_first = normx;
        const int stop = !(normx > 0.0) || (j > 0 && normx <= P.rtol * s_first);
        s_stop = stop;
        if (!stop) s_c = hh_scalars(&sA[j + (int64_t)cp * ld], sq, &s_diag[j]);
      }
    }
    __syncthreads();
    if (s_stop) break;
    const double c = s_c;
    const double* u = sA + (int64_t)cp * ld + j;
    const int len = m - j;
    const bool act = own && s_pos[g] > j;
    double* ap = sA + (int64_t)(act ? g : cp) * ld + j;
    double w0 = 0.0, w1 = 0.0;
    if (act) {
      int i = sl;
      for (; i + lanes < len; i += 2 * lanes) {
        w0 = fma(u[i], ap[i], w0);
        w1 = fma(u[i + lanes], ap[i + lanes], w1);
      }
      if (i < len) w0 = fma(u[i], ap[i], w0);
    }
    const double w = group_sum_n(w0 + w1, lanes) * c;
    if (act)
      for (int i = sl; i < len; i += lanes) ap[i] -= w * u[i];
    __syncwarp();
    int rc = 0;
    if (act && sl == 0) {
      double v1 = s_vn1[g];
      rc = qr_downdate(ap[0], v1, s_vn2[g]);
      s_vn1[g] = v1;
    }
    rc = __shfl_sync(FULL, rc, (lane / lanes) * lanes);
    double sq = 0.0;
    if (act && rc)
      for (int i = 1 + sl; i < len; i += lanes) sq += ap[i] * ap[i];
    sq = group_sum_n(sq, lanes);
    if (act && rc && sl == 0) { s_vn1[g] = sqrt(sq); s_vn2[g] = s_vn1[g]; }
    __syncthreads();
  }
  // columns in pivot order; R_pp on the diagonal of the factored positions
  for (int e = tid; e < m * n; e += blockDim.x) {
    const int i = e % m, p = e / m;
    const int c = s_col[p];
    P.A[i + (int64_t)p * P.lda] = (p < j && i == p) ? s_diag[p] : sA[i + (int64_t)c * ld];
  }
  for (int c = tid; c < n; c += blockDim.x) P.piv[c] = s_col[c];
  if (tid == 0) *P.rank = j;
}

int geqp3_small_launch(const Batch<QrProb>& b, const char* tag, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return -1; }
  if (merging()) {
    defer_launch("geqp3_small", b.h, [tag](std::vector<QrProb>& all, cudaStream_t st) {
      Batch<QrProb> m;
      m.h = std::move(all);
      m.upload(st);
      geqp3_small_launch(m, tag, st);
    });
    return -1;
  }
  size_t smem = 8;
  for (const auto& q : b.h) {
    SPD_REQUIRE(q.m >= 1 && q.n >= 1 && q.m <= kSmallQr && q.n <= kSmallQr,
                "geqp3_small: matrix larger than the one-CTA limit");
    smem = std::max(smem, (size_t)col_group_ld(q.m, col_group_lanes(q.n)) * q.n * sizeof(double));
  }
  constexpr int kDyn = 227 * 1024 - 8192;   // less the kernel's static arrays
  SPD_REQUIRE(smem <= (size_t)kDyn, "geqp3_small: matrix exceeds shared memory");
  static std::once_flag once;
  std::call_once(once, [] {
    SPD_CUDA(cudaFuncSetAttribute(k_geqp3_small, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn));
  });
  ProfScope ps(tag ? tag : "geqp3_small", s);
  k_geqp3_small<<<(unsigned)b.size(), 256, smem, s>>>(b.d.p);
  SPD_LAUNCHED();
  return ps.slot;
}

void tri_merge_launch(const Batch<TriMergeProb>& b, const char* tag, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    defer_launch("tri_merge", b.h, [tag](std::vector<TriMergeProb>& all, cudaStream_t st) {
      Batch<TriMergeProb> m;
      m.h = std::move(all);
      m.upload(st);
      tri_merge_launch(m, tag, st);
    });
    return;
  }
  int mmax = 1;
  double f = 0.0;
  for (const auto& p : b.h) {
    mmax = std::max(mmax, p.m);
    // column j: a reflector of j + 2 entries on m - j - 1 later columns (4 flops per entry)
    const double mm = p.m;
    f += 4.0 * (mm * mm * mm / 6.0 + mm * mm / 2.0);
  }
  const size_t smem = (size_t)mmax * (mmax + 1) * sizeof(double);
  constexpr int kDyn = 227 * 1024 - 1024;   // less the kernel's static scalars
  SPD_REQUIRE(smem <= (size_t)kDyn, "tri_merge: triangles exceed shared memory");
  static std::once_flag once;
  std::call_once(once, [] {
    SPD_CUDA(cudaFuncSetAttribute(k_tri_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn));
  });
  ProfScope ps(tag ? tag : "tri_merge", s, f);
  k_tri_merge<<<(unsigned)b.size(), 256, smem, s>>>(b.d.p);
  SPD_LAUNCHED();
}

// ---------------------------------------------------------------------------------------
// reflector application and explicit Q: one warp per column
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_hh_apply(const HhApplyProb* __restrict__ probs,
                                                  const int2* __restrict__ work, int64_t nwork,
                                                  int trans) {
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= nwork) return;
  const int lane = threadIdx.x & 31;
  const int2 it = work[w];
  const HhApplyProb P = probs[it.x];
  const int k = *P.k;
  double* b = P.B + (int64_t)it.y * P.ldb;
  for (int t = 0; t < k; ++t) {
    const int j = trans ? t : k - 1 - t;
    const double tau = P.tau[j];
    if (tau == 0.0) continue;
    const double* v = P.V + (int64_t)j * P.ldv;
    double s = 0.0;
    for (int i = j + lane; i < P.m; i += 32) s += (i == j ? 1.0 : v[i]) * b[i];
    s = warp_sum(s) * tau;
    for (int i = j + lane; i < P.m; i += 32) b[i] -= s * (i == j ? 1.0 : v[i]);
    __syncwarp();
  }
}

// The same product with the column held in registers: lane l owns rows l + 32 e (e < EPT,
// m <= 32 EPT), so each reflector costs one round of independent loads of v (issued one
// reflector ahead) and one warp reduction, instead of two passes over the column in memory.
template <int EPT>
__global__ void __launch_bounds__(256) k_hh_apply_r(const HhApplyProb* __restrict__ probs,
                                                    const int2* __restrict__ work, int64_t nwork,
                                                    int trans) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nwork) return;
  const int lane = threadIdx.x & 31;
  const int2 it = work[w];
  const HhApplyProb P = probs[it.x];
  const int k = *P.k;
  double* b = P.B + (int64_t)it.y * P.ldb;
  double x[EPT], vn[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = lane + 32 * e;
    x[e] = (i < P.m) ? b[i] : 0.0;
  }
  auto load_v = [&](int t, double* vv, double& tau) {
    const int j = trans ? t : k - 1 - t;
    const double* v = P.V + (int64_t)j * P.ldv;
    tau = P.tau[j];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = lane + 32 * e;
      vv[e] = (i > j && i < P.m) ? v[i] : (i == j ? 1.0 : 0.0);
    }
  };
  double taun = 0.0;
  if (k > 0) load_v(0, vn, taun);
  for (int t = 0; t < k; ++t) {
    double vv[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) vv[e] = vn[e];
    const double tau = taun;
    if (t + 1 < k) load_v(t + 1, vn, taun);
    if (tau == 0.0) continue;
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) s = fma(vv[e], x[e], s);
    s = warp_sum(s) * tau;
#pragma unroll
    for (int e = 0; e < EPT; ++e) x[e] -= s * vv[e];
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = lane + 32 * e;
    if (i < P.m) b[i] = x[e];
  }
}

// A problem of at most 512 rows goes to the register kernel, a taller one to the generic
// kernel: the choice depends on the problem alone (the two kernels sum in different
// orders; the register kernel's rows per lane do not change a column's arithmetic, the
// extra registers holding zeros).  EPT: registers per lane for the tallest register problem.
constexpr int kHhRegRows = 512;

static int hh_ept(const Batch<HhApplyProb>& b) {
  int mx = 1;
  for (const auto& p : b.h)
    if (p.m <= kHhRegRows) mx = std::max(mx, p.m);
  const int e = (mx + 31) / 32;
  return e <= 1 ? 1 : (e <= 2 ? 2 : (e <= 4 ? 4 : (e <= 8 ? 8 : 16)));
}

// FP64 issue is 2 FMA per clock per SM on this part: with few columns the warps are spread
// one or two per CTA so that they land on different SMs.
static void hh_go(const HhApplyProb* probs, const int2* work, int64_t nw, int64_t nreg, int ept,
                  int trans, cudaStream_t s) {
  if (nreg > 0) {
    const int wpb = nreg >= 8 * 152 ? 8 : (nreg >= 2 * 152 ? 2 : 1);   // warps per CTA
    const unsigned g = (unsigned)ceil_div(nreg, wpb);
    const int bs = 32 * wpb;
    switch (ept) {
      case 1: k_hh_apply_r<1><<<g, bs, 0, s>>>(probs, work, nreg, trans); break;
      case 2: k_hh_apply_r<2><<<g, bs, 0, s>>>(probs, work, nreg, trans); break;
      case 4: k_hh_apply_r<4><<<g, bs, 0, s>>>(probs, work, nreg, trans); break;
      case 8: k_hh_apply_r<8><<<g, bs, 0, s>>>(probs, work, nreg, trans); break;
      default: k_hh_apply_r<16><<<g, bs, 0, s>>>(probs, work, nreg, trans); break;
    }
    SPD_LAUNCHED();
  }
  if (nw > nreg) {
    k_hh_apply<<<(unsigned)ceil_div(nw - nreg, 8), 256, 0, s>>>(probs, work + nreg, nw - nreg, trans);
    SPD_LAUNCHED();
  }
}

// (problem, column) items: the register kernel's problems first (*nreg items)
static std::vector<int2> hh_work(const Batch<HhApplyProb>& b, int64_t* nreg) {
  std::vector<int2> work;
  for (int p = 0; p < (int)b.size(); ++p)
    if (b.h[p].m <= kHhRegRows)
      for (int c = 0; c < b.h[p].ncol; ++c) work.push_back(make_int2(p, c));
  *nreg = (int64_t)work.size();
  for (int p = 0; p < (int)b.size(); ++p)
    if (b.h[p].m > kHhRegRows)
      for (int c = 0; c < b.h[p].ncol; ++c) work.push_back(make_int2(p, c));
  return work;
}

void householder_prepare(Batch<HhApplyProb>& b, cudaStream_t s) {
  std::vector<int2> w = hh_work(b, &b.nfirst);
  b.work.upload(w, s);
  b.nwork = (int64_t)w.size();
  b.variant = hh_ept(b);
}

void householder_launch(const Batch<HhApplyProb>& b, int trans, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    const char* tag = b.tag;
    defer_launch(trans ? "householder_t" : "householder_n", b.h,
                 [tag, trans](std::vector<HhApplyProb>& all, cudaStream_t st) {
                   Batch<HhApplyProb> m;
                   m.h = std::move(all);
                   m.tag = tag;
                   m.upload(st);
                   householder_launch(m, trans, st);
                 });
    return;
  }
  if (b.nwork >= 0) {
    if (b.nwork == 0) return;
    ProfScope ps(b.tag ? b.tag : "householder", s);
    hh_go(b.d.p, b.work.p, b.nwork, b.nfirst, b.variant, trans, s);
    return;
  }
  int64_t nreg = 0;
  std::vector<int2> work = hh_work(b, &nreg);
  if (work.empty()) return;
  DevBuf<int2> dw;
  dw.upload(work, s);
  const int64_t nw = (int64_t)work.size();
  {
    ProfScope ps(b.tag ? b.tag : "householder", s);
    hh_go(b.d.p, dw.p, nw, nreg, hh_ept(b), trans, s);
  }
}

__global__ void __launch_bounds__(256) k_form_q(const FormQProb* __restrict__ probs,
                                                const int2* __restrict__ work, int64_t nwork) {
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= nwork) return;
  const int lane = threadIdx.x & 31;
  const int2 it = work[w];
  const FormQProb P = probs[it.x];
  const int k = *P.k;
  const int c = it.y;
  double* q = P.Q + (int64_t)c * P.ldq;
  for (int i = lane; i < P.m; i += 32) q[i] = (i == c && c < k) ? 1.0 : 0.0;
  __syncwarp();
  if (c >= k) return;
  for (int j = c; j >= 0; --j) {
    const double tau = P.tau[j];
    if (tau == 0.0) continue;
    const double* v = P.V + (int64_t)j * P.ldv;
    double s = 0.0;
    for (int i = j + lane; i < P.m; i += 32) s += (i == j ? 1.0 : v[i]) * q[i];
    s = warp_sum(s) * tau;
    for (int i = j + lane; i < P.m; i += 32) q[i] -= s * (i == j ? 1.0 : v[i]);
    __syncwarp();
  }
}

void form_q_launch(const Batch<FormQProb>& b, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    const char* tag = b.tag;
    defer_launch("form_q", b.h, [tag](std::vector<FormQProb>& all, cudaStream_t st) {
      Batch<FormQProb> m;
      m.h = std::move(all);
      m.tag = tag;
      m.upload(st);
      form_q_launch(m, st);
    });
    return;
  }
  std::vector<int2> work;
  for (int p = 0; p < (int)b.size(); ++p)
    for (int c = 0; c < b.h[p].kcols; ++c) work.push_back(make_int2(p, c));
  if (work.empty()) return;
  DevBuf<int2> dw;
  dw.upload(work, s);
  const int64_t nw = (int64_t)work.size();
  {
    ProfScope ps(b.tag ? b.tag : "form_q", s);
    k_form_q<<<ceil_div(nw, 8), 256, 0, s>>>(b.d.p, dw.p, nw);
    SPD_LAUNCHED();
  }
}

// ---------------------------------------------------------------------------------------
// batched 2-D copies
// ---------------------------------------------------------------------------------------
__global__ void k_copy(const CopyProb* __restrict__ probs, int ident) {
  const CopyProb P = probs[blockIdx.y];
  const int64_t tot = (int64_t)P.m * P.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % P.m), j = (int)(e / P.m);
    double v;
    if (ident) v = (i == j) ? 1.0 : 0.0;
    else if (!P.src) v = 0.0;
    else v = P.alpha * (P.trans ? P.src[j + (int64_t)i * P.lds] : P.src[i + (int64_t)j * P.lds]);
    double* d = P.dst + i + (int64_t)j * P.ldd;
    if (P.accumulate) *d += v; else *d = v;
  }
}

static void copy_common(const Batch<CopyProb>& b, int ident, cudaStream_t s) {
  if (b.empty()) { merge_skip(); return; }
  if (merging()) {
    const char* tag = b.tag;
    defer_launch(ident ? "identity" : "copy", b.h,
                 [tag, ident](std::vector<CopyProb>& all, cudaStream_t st) {
                   Batch<CopyProb> m;
                   m.h = std::move(all);
                   m.tag = tag;
                   m.upload(st);
                   copy_common(m, ident, st);
                 });
    return;
  }
  ProfScope ps(b.tag ? b.tag : "copy", s);
  int64_t mx = 1;
  for (const auto& p : b.h) mx = std::max<int64_t>(mx, (int64_t)p.m * p.n);
  const int gx = (int)std::min<int64_t>(ceil_div(mx, 256), 64);
  for (size_t y0 = 0; y0 < b.size(); y0 += 65535) {
    const unsigned gy = (unsigned)std::min<size_t>(65535, b.size() - y0);
    k_copy<<<dim3(gx, gy), 256, 0, s>>>(b.d.p + y0, ident);
    SPD_LAUNCHED();
  }
}

void copy_launch(const Batch<CopyProb>& b, cudaStream_t s) { copy_common(b, 0, s); }
void identity_launch(const Batch<CopyProb>& b, cudaStream_t s) { copy_common(b, 1, s); }

void copy_vec(double* dst, const double* src, int64_t count, cudaStream_t s) {
  if (count <= 0) return;
  if (merging()) {
    Batch<CopyProb> b;
    CopyProb c;
    c.src = src; c.lds = count; c.dst = dst; c.ldd = count;
    c.m = (int)count; c.n = 1; c.trans = 0; c.accumulate = 0; c.alpha = 1.0;
    SPD_REQUIRE(count < (int64_t(1) << 31), "copy_vec: vector too long to merge");
    b.h.push_back(c);
    copy_launch(b, s);
    return;
  }
  if (src) SPD_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else SPD_CUDA(cudaMemsetAsync(dst, 0, count * sizeof(double), s));
}

}  // namespace spd

// ---------------------------------------------------------------------------------------
// Launchers over descriptors that already sit in device memory (no allocation, no upload)
// ---------------------------------------------------------------------------------------
namespace spd {

std::vector<int4> gemm_tiles(const std::vector<GemmProb>& probs, int* nb_out) {
  int maxn = 0;
  for (const auto& p : probs) maxn = std::max(maxn, p.N);
  const int nb = gemm_variant(maxn);
  const int tm = nb ? 64 : GM, tn = nb ? nb : GN;
  std::vector<int4> tiles;
  for (int p = 0; p < (int)probs.size(); ++p)
    for (int m0 = 0; m0 < probs[p].M; m0 += tm)
      for (int n0 = 0; n0 < probs[p].N; n0 += tn) tiles.push_back(make_int4(p, m0, n0, 0));
  *nb_out = nb;
  return tiles;
}

void gemm_launch_raw(const GemmProb* d_probs, const GemmSeg* d_segs, const int4* d_tiles,
                     int64_t ntiles, int nb, cudaStream_t s) {
  if (ntiles <= 0) return;
  gemm_dispatch<double>(nb, (int)ntiles, d_probs, d_segs, d_tiles, s);
  SPD_LAUNCHED();
}

void trsm_launch_raw(const TrsmProb* d_probs, const int2* d_work, int64_t nwork, cudaStream_t s) {
  if (nwork <= 0) return;
  k_trsm<<<ceil_div(nwork, 8), 256, 0, s>>>(d_probs, d_work, nwork);
  SPD_LAUNCHED();
}

void householder_launch_raw(const HhApplyProb* d_probs, const int2* d_work, int64_t nwork,
                            int trans, cudaStream_t s) {
  if (nwork <= 0) return;
  k_hh_apply<<<ceil_div(nwork, 8), 256, 0, s>>>(d_probs, d_work, nwork, trans);
  SPD_LAUNCHED();
}

void copy_launch_raw(const CopyProb* d_probs, int64_t nprob, int64_t max_elems, cudaStream_t s) {
  if (nprob <= 0) return;
  const int gx = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(max_elems, 1), 256), 64);
  for (int64_t y0 = 0; y0 < nprob; y0 += 65535) {
    const unsigned gy = (unsigned)std::min<int64_t>(65535, nprob - y0);
    k_copy<<<dim3(gx, gy), 256, 0, s>>>(d_probs + y0, 0);
    SPD_LAUNCHED();
  }
}

}  // namespace spd
