// The FP32 H^2 product with every stored generator read once (Sec. 5.1: y = A x through
// the upward pass, the Type-3 couplings and the downward pass).
//
// A coupling B_ij is stored once per unordered far pair (owner i < j, k_i x k_j).  Its
// two uses, y^_i += B_ij x^_j and y^_j += B_ij^T x^_i, are made from the same tile: one
// pass over the owner's k_i x (sum k_j) region M_i = [B_ij1 B_ij2 ...] forms M_i x^ (the
// gathered x^_j) and M_i^T x^_i together.  The per-pair results go to scratch and a
// second kernel adds, per destination node, its pieces in a fixed order, so the sum
// order of every entry is fixed by the tree alone (no atomics; identical results alone
// and in a merged batch).  The upward pass (x^_i = U_i^T x) and the downward pass
// (y^_children += R_i y^_i, y = U_i y^_i) are the same kernel with one direction.
//
// Layout: every matrix (leaf basis, transfer matrix, coupling region) is an FP32
// column-major copy with its leading dimension rounded up to a multiple of 4 (zero rows),
// starting on a 16-byte boundary, so that a column range of up to 512 rows streams into
// shared memory with 16-byte asynchronous copies.  Skeleton-space vectors are
// row-interleaved (the nc right-hand sides of a row contiguous), so that the x^ entries a
// column needs are one contiguous piece.
//
// One CTA (8 warps) takes a job: rows [r0, r0 + R) (R <= 512, slices of 128 rows, a lane
// holding 4 consecutive rows) and a column range, staged S columns at a time through a
// 3-deep shared-memory pipeline of 32 KB stages.  Warps are slices x teams; a team takes every TM-th
// group of CG columns, and each warp applies both directions to the entries it loads:
//  - Direction 1 (A x): each lane accumulates its 4 rows x NC right-hand sides over the
//    columns; the teams' partial sums are added in team order at the end.
//  - Direction 2 (A^T x): for a group of CG columns each lane forms its 4 rows' share of
//    the CG x NC = V dot products and the warp reduces them across lanes with a butterfly
//    in which every level halves the values a lane holds (lane L ends with value L).  The
//    lane reads its columns and right-hand sides in an order permuted by its lane bits,
//    so that at every level the value a lane sends sits in the same register as the value
//    its partner keeps (no selects).  Slices are added in slice order.
#include <algorithm>
#include <cstdlib>

#include "h2.cuh"
#include "merge.cuh"

namespace spd {

namespace {

constexpr int kSymStages = 3;
constexpr int kSymStageFloats = 8192;   // A entries per pipeline stage (32 KB)
constexpr int kSymMaxCols = 128;        // columns per stage
constexpr int kSymRed2 = 1024;          // direction-2 slice partials per stage

__host__ __device__ constexpr int sym_cg(int nc) { return nc == 16 ? 2 : 4; }
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

size_t sym_smem(int nc) {
  return sizeof(float) * ((size_t)kSymStages * kSymStageFloats +
                          (size_t)kSymStages * kSymMaxCols * nc + kSymRed2);
}

}  // namespace

template <int NC>
__global__ void __launch_bounds__(256, NC >= 16 ? 1 : 2)
    k_sym(const SymJob* __restrict__ jobs) {
  constexpr int CG = sym_cg(NC);
  constexpr int V = CG * NC;              // dot products per column group
  constexpr int LV = ilog2c(V);           // butterfly levels that halve the values
  constexpr int LNC = ilog2c(NC);
  constexpr int NC2 = (NC + 1) / 2;
  extern __shared__ __align__(16) float sym_sm[];
  float* As = sym_sm;
  float* Xs = As + kSymStages * kSymStageFloats;
  float* red2 = Xs + kSymStages * kSymMaxCols * NC;
  // the job, read once into registers
  const SymJob& Jg = jobs[blockIdx.x];
  const float* __restrict__ A = Jg.A;
  const int64_t lda = Jg.lda;
  const int r0 = Jg.r0, R = Jg.R, c0 = Jg.c0, c1 = Jg.c1, S = Jg.S, ncol = Jg.ncol;
  float* const y1 = Jg.y1;
  const int64_t y1rs = Jg.y1rs, y1cs = Jg.y1cs;
  const int mode1 = Jg.mode1;
  const float* __restrict__ x1 = Jg.x1;
  const int* __restrict__ cmap = Jg.cmap;
  float* const z = Jg.z;
  const int64_t zcs = Jg.zcs, zrs = Jg.zrs;
  const int mode2 = Jg.mode2;
  const float* __restrict__ x2 = Jg.x2;
  const int64_t x2rs = Jg.x2rs, x2cs = Jg.x2cs;
  const int R4 = (R + 3) & ~3;
  const bool has1 = y1 != nullptr, has2 = z != nullptr;
  const int RS = (R + 127) >> 7;
  const int RSp = RS <= 1 ? 1 : (RS == 2 ? 2 : 4);
  const int TM = 8 / RSp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rs = warp % RSp, team = warp / RSp;
  const bool wact = rs < RS;              // the warp's slice holds rows of the job
  const int rbase = rs * 128 + 4 * lane;
  const bool rows_ok = wact && rbase < R4;
  const int ncols = c1 - c0;
  const int nst = ncols > 0 ? (ncols + S - 1) / S : 0;
  const int GS = S / CG;
  const int Q = R4 >> 2;   // 16-byte pieces per staged column

  // the x1 piece of this thread in every stage: column tid / NP, piece tid % NP of the
  // column's NC contiguous entries (S * NP <= 256)
  constexpr int NP = NC >= 4 ? NC / 4 : 1;
  const int xcol = threadIdx.x / NP, xp = threadIdx.x % NP;
  auto col_index = [&](int st) -> int64_t {
    const int c = c0 + st * S + xcol;
    if (st >= nst || xcol >= S || c >= c1) return -1;
    return cmap ? (int64_t)__ldg(cmap + c) : (int64_t)c;
  };
  auto issue = [&](int st, int64_t xi) {
    if (st < nst) {
      const int b = st % kSymStages;
      float* Ab = As + b * kSymStageFloats;
      const int cs = c0 + st * S;
      if (R4 == lda) {
        // the job spans whole columns: the stage is one contiguous range
        const float* src0 = A + (int64_t)cs * lda;
        const int valid = (min(c1 - cs, S) * R4) >> 2;   // 16-byte pieces inside the matrix
        for (int e = threadIdx.x; e < S * Q; e += 256)
          cp_async16(Ab + 4 * e, e < valid ? src0 + 4 * e : A, e < valid ? 16 : 0);
      } else {
        // piece e = col * Q + q; stepping e by 256 advances (col, q) by (256 / Q, 256 % Q)
        int col = threadIdx.x / Q, q = threadIdx.x - (threadIdx.x / Q) * Q;
        const int dcol = 256 / Q, dq = 256 - (256 / Q) * Q;
        for (int e = threadIdx.x; e < S * Q; e += 256) {
          const int c = cs + col;
          const bool ok = c < c1;
          const float* src = ok ? A + (int64_t)c * lda + r0 + 4 * q : A;
          cp_async16(Ab + col * R4 + 4 * q, src, ok ? 16 : 0);
          col += dcol;
          q += dq;
          if (q >= Q) { q -= Q; ++col; }
        }
      }
      if (has1 && xcol < S) {
        float* Xb = Xs + b * (kSymMaxCols * NC) + xcol * NC;
        const bool ok = xi >= 0;
        const float* src = ok ? x1 + xi * NC : x1;
        if constexpr (NC >= 4) cp_async16(Xb + 4 * xp, src + 4 * xp, ok ? 16 : 0);
        else if constexpr (NC == 2) cp_async8(Xb, src, ok ? 8 : 0);
        else cp_async4(Xb, src, ok ? 4 : 0);
      }
    }
    cp_async_commit();
  };

  // Direction 2 reads the group's columns and right-hand sides in the lane's permuted
  // order (the butterfly's layout); direction 1 follows the same column order (a fixed
  // order per lane).
  const int sig = lane >> (5 - LV);
  const int colperm = sig >> LNC, rhsperm = sig & (NC - 1);
  // acc: direction-1 sums of the lane's rows; xr: the lane's rows of x2; pairs of
  // right-hand sides share a float2 so that one packed FMA updates both
  float2 acc[4][NC2], xr[4][NC2];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int h = 0; h < NC2; ++h) { acc[k][h] = make_float2(0.f, 0.f); xr[k][h] = make_float2(0.f, 0.f); }
  if (has2 && rows_ok) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int tr = c ^ rhsperm;
        const float v = (rbase + k < R && tr < ncol) ? __ldg(x2 + (rbase + k) * x2rs + tr * x2cs) : 0.f;
        if (c & 1) xr[k][c >> 1].y = v;
        else xr[k][c >> 1].x = v;
      }
  }

  // pipeline prologue
  int64_t xi = has1 ? col_index(0) : -1;
  for (int st = 0; st < kSymStages - 1; ++st) {
    issue(st, xi);
    if (has1) xi = col_index(st + 1);
  }
  for (int st = 0; st < nst; ++st) {
    cp_async_wait<kSymStages - 2>();
    __syncthreads();
    issue(st + kSymStages - 1, xi);
    if (has1) xi = col_index(st + kSymStages);
    const int b = st % kSymStages;
    const float* Ab = As + b * kSymStageFloats;
    const float* Xb = Xs + b * (kSymMaxCols * NC);
    for (int g = team; wact && g < GS; g += TM) {
      float2 p[NC == 1 ? 2 : V / 2];   // slot pairs (2h, 2h + 1) in p[h]
#pragma unroll
      for (int cs = 0; cs < CG; ++cs) {
        const int col = g * CG + (cs ^ colperm);
        const float4 a = rows_ok ? *reinterpret_cast<const float4*>(Ab + col * R4 + rbase)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (NC == 1) {
          if (has1) {
            const float xv = Xb[col];
            acc[0][0].x = fmaf(a.x, xv, acc[0][0].x);
            acc[1][0].x = fmaf(a.y, xv, acc[1][0].x);
            acc[2][0].x = fmaf(a.z, xv, acc[2][0].x);
            acc[3][0].x = fmaf(a.w, xv, acc[3][0].x);
          }
          if (has2) {
            float v = a.x * xr[0][0].x;
            v = fmaf(a.y, xr[1][0].x, v);
            v = fmaf(a.z, xr[2][0].x, v);
            v = fmaf(a.w, xr[3][0].x, v);
            if (cs & 1) p[cs >> 1].y = v;
            else p[cs >> 1].x = v;
          }
        } else {
          const float2 ax = make_float2(a.x, a.x), ay = make_float2(a.y, a.y);
          const float2 az = make_float2(a.z, a.z), aw = make_float2(a.w, a.w);
          if (has1) {
            float2 xv[NC2];
            if constexpr (NC >= 4) {
#pragma unroll
              for (int c4 = 0; c4 < NC / 4; ++c4) {
                const float4 v = reinterpret_cast<const float4*>(Xb + col * NC)[c4];
                xv[2 * c4] = make_float2(v.x, v.y);
                xv[2 * c4 + 1] = make_float2(v.z, v.w);
              }
            } else {
              xv[0] = *reinterpret_cast<const float2*>(Xb + col * NC);
            }
#pragma unroll
            for (int h = 0; h < NC2; ++h) {
              acc[0][h] = __ffma2_rn(ax, xv[h], acc[0][h]);
              acc[1][h] = __ffma2_rn(ay, xv[h], acc[1][h]);
              acc[2][h] = __ffma2_rn(az, xv[h], acc[2][h]);
              acc[3][h] = __ffma2_rn(aw, xv[h], acc[3][h]);
            }
          }
          if (has2) {
#pragma unroll
            for (int h = 0; h < NC2; ++h) {
              float2 v = __fmul2_rn(ax, xr[0][h]);
              v = __ffma2_rn(ay, xr[1][h], v);
              v = __ffma2_rn(az, xr[2][h], v);
              p[cs * NC2 + h] = __ffma2_rn(aw, xr[3][h], v);
            }
          }
        }
      }
      if (has2) {
        // butterfly: level l keeps slots [0, H) and adds the partner's slots [H, 2H)
#pragma unroll
        for (int l = 0; l < LV; ++l) {
          const int H = V >> (l + 1);
          if (H >= 2) {
#pragma unroll
            for (int h = 0; h < H / 2; ++h) {
              const float rx = __shfl_xor_sync(0xffffffffu, p[h + H / 2].x, 16 >> l);
              const float ry = __shfl_xor_sync(0xffffffffu, p[h + H / 2].y, 16 >> l);
              p[h] = __fadd2_rn(p[h], make_float2(rx, ry));
            }
          } else {
            p[0].x += __shfl_xor_sync(0xffffffffu, p[0].y, 16 >> l);
          }
        }
        float res = p[0].x;
#pragma unroll
        for (int off = (16 >> LV); off >= 1; off >>= 1) res += __shfl_xor_sync(0xffffffffu, res, off);
        if (RS == 1) {
          if ((lane & ((32 >> LV) - 1)) == 0) {
            const int col = st * S + g * CG + (sig >> LNC);
            const int rh = sig & (NC - 1);
            if (col < ncols && rh < ncol) {
              float* zp = z + col * zcs + rh * zrs;
              *zp = mode2 ? *zp + res : res;
            }
          }
        } else {
          red2[(g * RSp + rs) * 32 + lane] = res;
        }
      }
    }
    __syncthreads();
    if (has2 && RS > 1) {
      for (int e = threadIdx.x; e < GS * 32; e += 256) {
        const int g = e >> 5, ln = e & 31;
        if (ln & ((32 >> LV) - 1)) continue;
        const int sg = ln >> (5 - LV);
        const int col = st * S + g * CG + (sg >> LNC);
        const int rh = sg & (NC - 1);
        if (col >= ncols || rh >= ncol) continue;
        float v = red2[(g * RSp) * 32 + ln];
        for (int q2 = 1; q2 < RS; ++q2) v += red2[(g * RSp + q2) * 32 + ln];
        float* zp = z + col * zcs + rh * zrs;
        *zp = mode2 ? *zp + v : v;
      }
    }
  }
  cp_async_wait<0>();
  if (!has1) return;
  __syncthreads();
  // direction 1: the teams' partial sums, added in team order
  float* red1 = As;   // [TM][R4][NC]
  if (rows_ok) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c)
        red1[((int64_t)team * R4 + rbase + k) * NC + c] = (c & 1) ? acc[k][c >> 1].y : acc[k][c >> 1].x;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * NC; e += 256) {
    const int rh = e / R, r = e - rh * R;
    if (rh >= ncol) break;
    float v = red1[r * NC + rh];
    for (int t = 1; t < TM; ++t) v += red1[((int64_t)t * R4 + r) * NC + rh];
    float* yp = y1 + r * y1rs + rh * y1cs;
    *yp = mode1 ? *yp + v : v;
  }
}

// y (+)= the sources in order (all row-interleaved with stride nc); CTA (job, chunk of
// 256 entries), one entry per thread with its source loads issued eight at a time
__global__ void __launch_bounds__(256) k_sym_sum(const SymSum* __restrict__ jobs,
                                                 const SymSrc* __restrict__ srcs) {
  const SymSum& J = jobs[blockIdx.x];
  const int rows = J.rows, ncol = J.ncol;
  const int e = blockIdx.y * 256 + threadIdx.x;
  if (e >= rows * ncol) return;
  const int r = e / ncol, c = e - r * ncol;
  const int64_t o = (int64_t)r * J.nc + c;
  float v = 0.f;
  int q = J.s0;
  for (; q + 8 <= J.s1; q += 8) {
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = __ldg(srcs[q + u].p + o);
#pragma unroll
    for (int u = 0; u < 8; ++u) v += t[u];
  }
  for (; q < J.s1; ++q) v += __ldg(srcs[q].p + o);
  float* yp = J.y + o;
  *yp = J.mode ? *yp + v : v;
}

// FP64 -> FP32 copies with the leading dimension padded by zero rows
struct PadCopy {
  const double* src;
  int64_t lds;
  int rows;
  int64_t cols;
  float* dst;
  int64_t ldd;
};
__global__ void k_pad_copy(const PadCopy* __restrict__ probs) {
  const PadCopy P = probs[blockIdx.y];
  const int64_t tot = P.ldd * P.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / P.ldd, r = e - c * P.ldd;
    P.dst[e] = r < P.rows ? (float)P.src[r + c * P.lds] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// host side

static int sym_nc(int ncol) {
  return ncol <= 1 ? 1 : (ncol <= 2 ? 2 : (ncol <= 4 ? 4 : (ncol <= 8 ? 8 : 16)));
}
static int64_t align4(int64_t x) { return (x + 3) & ~int64_t(3); }

// rows per job (multiple of 128, at most 512): 256 measured fastest on GB300 (n = 200,000
// Gaussian, 8 columns: 11.0 ms against 11.7 ms for 512, 11.0 ms for 128: fewer idle
// slices in a job, for partial sums over more row parts); SPDHSS_SYM_ROW_BLOCK selects
// 128, 256 or 512
static int sym_row_block() {
  const char* e = std::getenv("SPDHSS_SYM_ROW_BLOCK");
  if (e) {
    const int v = std::atoi(e);
    if (v == 128 || v == 256 || v == 512) return v;
  }
  return 256;
}

// columns per stage for a job of R rows: a multiple of CG x teams, a power of two,
// S * ceil4(R) <= 8192, S <= 128 (64 for 16 right-hand sides: one x1 piece per thread)
static int sym_stage_cols(int R, int nc) {
  const int R4 = (int)align4(R);
  const int RS = (R + 127) / 128;
  const int RSp = RS <= 1 ? 1 : (RS == 2 ? 2 : 4);
  const int base = sym_cg(nc) * (8 / RSp);
  int k = std::max(1, kSymStageFloats / (std::max(R4, 4) * base));
  int kp = 1;
  while (kp * 2 <= k) kp *= 2;
  int S = base * kp;
  while (S > (nc == 16 ? kSymMaxCols / 2 : kSymMaxCols)) S /= 2;
  return S;
}

bool sym_layout_fits(const spdhss_h2_s* h, cudaStream_t s) {
  if (h->sym_f.n > 0) return true;
  const size_t est = (h->coup.n + h->basis.n) * sizeof(float) * 21 / 20 +
                     (size_t)h->Ktot * 1024;
  return fits_on_device(est, s);
}

void sym_layout(spdhss_h2_s* h, cudaStream_t s) {
  if (h->sym_f.n > 0) return;
  const TreeHost& T = h->th;
  const int64_t NN = T.nn();
  h->sym_U_off.assign(NN, -1);
  h->sym_M_off.assign(NN, -1);
  h->sym_Kc.assign(NN, 0);
  h->sym_cmap_off.assign(NN + 1, 0);
  h->sym_colstart.assign(T.far_idx.size(), 0);
  std::vector<PadCopy> cps;
  std::vector<int> cmap;
  int64_t tot = 0;
  for (int64_t i = 0; i < NN; ++i) {
    const int k = h->rank(i);
    if (k == 0 || h->U_rows[i] == 0) continue;
    const int64_t ld = align4(h->U_rows[i]);
    h->sym_U_off[i] = tot;
    cps.push_back(PadCopy{h->basis.p + h->U_off[i], h->U_rows[i], h->U_rows[i], k, nullptr, ld});
    tot += ld * k;
  }
  for (int64_t i = 0; i < NN; ++i) {
    const int k = h->rank(i);
    int64_t kc = 0, first = -1;
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      if (j <= i || k == 0 || h->rank(j) == 0) continue;
      if (first < 0) first = h->far_boff[e];
      h->sym_colstart[e] = kc;
      for (int c = 0; c < h->rank(j); ++c) cmap.push_back((int)(h->skel_off[j] + c));
      kc += h->rank(j);
    }
    h->sym_cmap_off[i + 1] = (int64_t)cmap.size();
    if (kc == 0) continue;
    const int64_t ld = align4(k);
    h->sym_M_off[i] = tot;
    h->sym_Kc[i] = kc;
    cps.push_back(PadCopy{h->coup.p + first, k, k, kc, nullptr, ld});
    tot += ld * kc;
  }
  // the non-owner entries take the column start of their owner's entry
  for (int64_t i = 0; i < NN; ++i)
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      if (j >= i || h->rank(i) == 0 || h->rank(j) == 0) continue;
      const auto b0 = T.far_idx.begin() + T.far_off[j], b1 = T.far_idx.begin() + T.far_off[j + 1];
      const auto it = std::lower_bound(b0, b1, i);
      SPD_REQUIRE(it != b1 && *it == i, "h2 product: far lists are not symmetric");
      h->sym_colstart[e] = h->sym_colstart[it - T.far_idx.begin()];
    }
  h->sym_f.alloc((size_t)tot + 4);
  SPD_CUDA(cudaMemsetAsync(h->sym_f.p + tot, 0, 4 * sizeof(float), s));
  {
    size_t c = 0;
    for (int64_t i = 0; i < NN; ++i)
      if (h->sym_U_off[i] >= 0) cps[c++].dst = h->sym_f.p + h->sym_U_off[i];
    for (int64_t i = 0; i < NN; ++i)
      if (h->sym_M_off[i] >= 0) cps[c++].dst = h->sym_f.p + h->sym_M_off[i];
  }
  for (size_t b0 = 0; b0 < cps.size(); b0 += 65535) {
    std::vector<PadCopy> part(cps.begin() + b0, cps.begin() + std::min(cps.size(), b0 + 65535));
    DevBuf<PadCopy> dp;
    dp.upload(part, s);
    int64_t mx = 1;
    for (const auto& p : part) mx = std::max(mx, p.ldd * p.cols);
    const int gx = (int)std::min<int64_t>(ceil_div(mx, 256), 256);
    k_pad_copy<<<dim3(gx, (unsigned)part.size()), 256, 0, s>>>(dp.p);
    SPD_LAUNCHED();
    SPD_CUDA(cudaStreamSynchronize(s));
  }
  h->sym_cmap.upload(cmap.empty() ? std::vector<int>(1, 0) : cmap, s);
  SPD_CUDA(cudaStreamSynchronize(s));
}

namespace {

struct DeferredSym : Deferred {
  SymBatch b;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    SymBatch m;
    m.nc = b.nc;
    m.ncol = b.ncol;
    m.tag = b.tag;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredSym*>(d);
      m.jobs.insert(m.jobs.end(), x->b.jobs.begin(), x->b.jobs.end());
      m.ncol = std::max(m.ncol, x->b.ncol);
      m.bytes += x->b.bytes;
      m.flops += x->b.flops;
    }
    m.upload(s);
    m.launch(s);
  }
};

struct DeferredSymSum : Deferred {
  SymSumBatch b;
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    SymSumBatch m;
    m.ncol = b.ncol;
    m.tag = b.tag;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredSymSum*>(d);
      const int off = (int)m.srcs.size();
      m.srcs.insert(m.srcs.end(), x->b.srcs.begin(), x->b.srcs.end());
      for (SymSum j : x->b.jobs) {
        j.s0 += off;
        j.s1 += off;
        m.jobs.push_back(j);
      }
      m.ncol = std::max(m.ncol, x->b.ncol);
      m.bytes += x->b.bytes;
    }
    m.upload(s);
    m.launch(s);
  }
};

template <int NC>
void sym_go(const SymBatch& b, cudaStream_t s) {
  const size_t smem = sym_smem(NC);
  SPD_CUDA(cudaFuncSetAttribute(k_sym<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sym<NC><<<(unsigned)b.jobs.size(), 256, smem, s>>>(b.d_jobs.p);
  SPD_LAUNCHED();
}

}  // namespace

void SymBatch::upload(cudaStream_t s) {
  // the largest jobs first, so that the long ones do not form the tail
  std::stable_sort(jobs.begin(), jobs.end(), [](const SymJob& x, const SymJob& y) {
    return (int64_t)x.R * (x.c1 - x.c0) > (int64_t)y.R * (y.c1 - y.c0);
  });
  d_jobs.upload(jobs, s);
}

void SymBatch::launch(cudaStream_t s) const {
  if (merging()) {
    if (jobs.empty()) { merge_skip(); return; }
    std::unique_ptr<DeferredSym> d(new DeferredSym());
    d->b.jobs = jobs;
    d->b.nc = nc;
    d->b.ncol = ncol;
    d->b.tag = tag;
    d->b.bytes = bytes;
    d->b.flops = flops;
    merge_ctx().m->submit("sym_" + std::to_string(nc), std::move(d));
    return;
  }
  if (jobs.empty()) return;
  ProfScope ps(tag, s, flops, bytes);
  switch (nc) {
    case 1: sym_go<1>(*this, s); break;
    case 2: sym_go<2>(*this, s); break;
    case 4: sym_go<4>(*this, s); break;
    case 8: sym_go<8>(*this, s); break;
    default: sym_go<16>(*this, s); break;
  }
}

void SymSumBatch::upload(cudaStream_t s) {
  d_jobs.upload(jobs, s);
  d_srcs.upload(srcs.empty() ? std::vector<SymSrc>(1, SymSrc{nullptr}) : srcs, s);
}

void SymSumBatch::launch(cudaStream_t s) const {
  if (merging()) {
    if (jobs.empty()) { merge_skip(); return; }
    std::unique_ptr<DeferredSymSum> d(new DeferredSymSum());
    d->b.jobs = jobs;
    d->b.srcs = srcs;
    d->b.ncol = ncol;
    d->b.tag = tag;
    d->b.bytes = bytes;
    merge_ctx().m->submit("symsum", std::move(d));
    return;
  }
  if (jobs.empty()) return;
  ProfScope ps(tag, s, 0.0, bytes);
  int mx = 1;
  for (const SymSum& j : jobs) mx = std::max(mx, j.rows * j.ncol);
  k_sym_sum<<<dim3((unsigned)jobs.size(), (unsigned)ceil_div(mx, 256)), 256, 0, s>>>(d_jobs.p, d_srcs.p);
  SPD_LAUNCHED();
}

// The steps of the FP32 product of plan p (its vectors already allocated).
void sym_plan_build(const spdhss_h2_s* h, H2PlanF& p, int ncol, cudaStream_t s) {
  const TreeHost& T = h->th;
  const int64_t n = T.n, K = std::max<int64_t>(h->Ktot, 1);
  const int D = T.D;
  const int nc = sym_nc(ncol);
  const int RB = sym_row_block();
  std::shared_ptr<SymPlan> sp(new SymPlan());
  SymPlan& P = *sp;
  P.nc = nc;
  // x^ and y^, row-interleaved; the padding right-hand sides stay zero
  P.xh.alloc((size_t)K * nc);
  P.yh.alloc((size_t)K * nc);
  P.xh.zero(s);
  P.yh.zero(s);
  float* const xh = P.xh.p;
  float* const yh = P.yh.p;
  float* base = h->sym_f.p;
  const char* btag = "h2_basis_f32";
  const char* ctag = "h2_coupling_f32";
  auto new_sym = [&](const char* tag) {
    P.steps.emplace_back();
    P.steps.back().sym.reset(new SymBatch());
    SymBatch& b = *P.steps.back().sym;
    b.nc = nc;
    b.ncol = ncol;
    b.tag = tag;
    return &b;
  };
  auto new_sum = [&](const char* tag) {
    P.steps.emplace_back();
    P.steps.back().sum.reset(new SymSumBatch());
    SymSumBatch& b = *P.steps.back().sum;
    b.ncol = ncol;
    b.tag = tag;
    return &b;
  };
  auto new_job = [&]() {
    SymJob j{};
    j.ncol = ncol;
    return j;
  };
  // partial buffers (row-interleaved): offsets first, pointers patched once the buffer
  // exists
  struct Patch { int step; size_t idx; int which; int64_t off; };
  std::vector<Patch> patches;   // which: 0 job.y1, 1 job.z, 2 src.p (all into P.part)
  int64_t part_tot = 0;
  auto part_alloc = [&](int64_t rows) {
    const int64_t o = part_tot;
    part_tot += align4(rows * nc);
    return o;
  };

  // upward pass: x^_i = U_i^T x (leaves), x^_i = R_i^T x^_children (depth D-1 .. 1)
  for (int t = D; t >= 1; --t) {
    SymBatch* b = new_sym(btag);
    const int sb = (int)P.steps.size() - 1;
    SymSumBatch* sm = nullptr;
    int ssm = -1;
    for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i) {
      const int k = h->rank(i);
      if (k == 0 || h->sym_U_off[i] < 0) continue;
      const int rows = h->U_rows[i];
      const int nrp = (rows + RB - 1) / RB;
      std::vector<int64_t> offs;
      for (int rp = 0; rp < nrp; ++rp) {
        SymJob j = new_job();
        j.A = base + h->sym_U_off[i];
        j.lda = align4(rows);
        j.r0 = rp * RB;
        j.R = std::min(RB, rows - j.r0);
        j.c0 = 0;
        j.c1 = k;
        j.S = sym_stage_cols(j.R, nc);
        if (t == D) {   // x in the plan's column-major sorted-order block
          j.x2 = p.xs.p + T.begin[i] + j.r0;
          j.x2rs = 1;
          j.x2cs = n;
        } else {
          j.x2 = xh + (h->skel_off[T.child_begin[i]] + j.r0) * nc;
          j.x2rs = nc;
          j.x2cs = 1;
        }
        j.zcs = nc;
        j.zrs = 1;
        if (nrp == 1) {
          j.z = xh + h->skel_off[i] * nc;
        } else {
          const int64_t o = part_alloc(k);
          offs.push_back(o);
          patches.push_back(Patch{sb, b->jobs.size(), 1, o});
        }
        b->bytes += 4.0 * (double)j.R * k;
        b->flops += 2.0 * (double)j.R * k * ncol;
        b->jobs.push_back(j);
      }
      if (nrp > 1) {
        if (!sm) { sm = new_sum("h2_basis_sum_f32"); ssm = (int)P.steps.size() - 1; }
        SymSum q{};
        q.y = xh + h->skel_off[i] * nc;
        q.rows = k;
        q.ncol = ncol;
        q.nc = nc;
        q.mode = 0;
        q.s0 = (int)sm->srcs.size();
        for (int64_t o : offs) {
          patches.push_back(Patch{ssm, sm->srcs.size(), 2, o});
          sm->srcs.push_back(SymSrc{nullptr});
        }
        q.s1 = (int)sm->srcs.size();
        sm->jobs.push_back(q);
      }
    }
  }
  // couplings: per owner region M_i, direction 1 into partial tiles, direction 2 into the
  // per-pair pieces Z_i (Kc_i x nc, one per row part of the owner)
  SymBatch* cb = new_sym(ctag);
  const int scb = (int)P.steps.size() - 1;
  const int64_t NN = T.nn();
  std::vector<std::vector<std::vector<int64_t>>> p1(NN);   // [i][row part] -> partial offsets
  std::vector<std::vector<int64_t>> zoff(NN);               // [i][row part] -> Z offset
  const int64_t kTarget = int64_t(1) << 19;                   // entries per job (2 MB)
  for (int64_t i = 0; i < NN; ++i) {
    const int64_t kc = h->sym_Kc[i];
    const int k = h->rank(i);
    if (kc == 0 || k == 0) continue;
    const int nrp = (k + RB - 1) / RB;
    p1[i].resize(nrp);
    zoff[i].resize(nrp);
    for (int rp = 0; rp < nrp; ++rp) {
      const int r0 = rp * RB, R = std::min(RB, k - r0);
      const int S = sym_stage_cols(R, nc);
      const int64_t R4 = align4(R);
      const int64_t cpj = std::max<int64_t>(1, kTarget / (R4 * S)) * S;
      zoff[i][rp] = part_alloc(kc);
      for (int64_t cc = 0; cc < kc; cc += cpj) {
        SymJob j = new_job();
        j.A = base + h->sym_M_off[i];
        j.lda = align4(k);
        j.r0 = r0;
        j.R = R;
        j.c0 = (int)cc;
        j.c1 = (int)std::min(kc, cc + cpj);
        j.S = S;
        const int64_t o1 = part_alloc(R);
        p1[i][rp].push_back(o1);
        j.y1rs = nc;
        j.y1cs = 1;
        j.mode1 = 0;
        patches.push_back(Patch{scb, cb->jobs.size(), 0, o1});
        j.x1 = xh;
        j.cmap = h->sym_cmap.p + h->sym_cmap_off[i];
        j.zcs = nc;
        j.zrs = 1;
        j.mode2 = 0;
        patches.push_back(Patch{scb, cb->jobs.size(), 1, zoff[i][rp] + cc * nc});
        j.x2 = xh + (h->skel_off[i] + r0) * nc;
        j.x2rs = nc;
        j.x2cs = 1;
        cb->bytes += 4.0 * (double)R * (j.c1 - j.c0);
        cb->flops += 4.0 * (double)R * (j.c1 - j.c0) * ncol;
        cb->jobs.push_back(j);
      }
    }
  }
  // y^_j = its own region's direction-1 parts + the Z pieces of its owners, in order
  SymSumBatch* cs = new_sum("h2_coupling_sum_f32");
  const int scs = (int)P.steps.size() - 1;
  for (int64_t j = 0; j < NN; ++j) {
    const int k = h->rank(j);
    if (k == 0) continue;
    const int nrp = (k + RB - 1) / RB;
    for (int rp = 0; rp < nrp; ++rp) {
      const int r0 = rp * RB, R = std::min(RB, k - r0);
      SymSum q{};
      q.y = yh + (h->skel_off[j] + r0) * nc;
      q.rows = R;
      q.ncol = ncol;
      q.nc = nc;
      q.mode = 0;
      q.s0 = (int)cs->srcs.size();
      if (!p1[j].empty())
        for (int64_t o : p1[j][rp]) {
          patches.push_back(Patch{scs, cs->srcs.size(), 2, o});
          cs->srcs.push_back(SymSrc{nullptr});
        }
      for (int64_t e = T.far_off[j]; e < T.far_off[j + 1]; ++e) {
        const int64_t hh = T.far_idx[e];
        if (hh >= j || h->rank(hh) == 0) continue;
        for (size_t rq = 0; rq < zoff[hh].size(); ++rq) {
          patches.push_back(Patch{scs, cs->srcs.size(), 2,
                                  zoff[hh][rq] + (h->sym_colstart[e] + r0) * nc});
          cs->srcs.push_back(SymSrc{nullptr});
        }
      }
      q.s1 = (int)cs->srcs.size();
      cs->bytes += 4.0 * (double)R * ncol * (q.s1 - q.s0 + 1);
      cs->jobs.push_back(q);
    }
  }
  // downward pass: y^_children += R_i y^_i (depth 1 .. D-1), then y = U_i y^_i (leaves)
  for (int t = std::min(1, D); t <= D; ++t) {
    SymBatch* b = new_sym(btag);
    for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i) {
      const int k = h->rank(i);
      const bool leaf = (t == D);
      if (!leaf && (k == 0 || h->sym_U_off[i] < 0)) continue;
      const int rows = leaf ? (int)T.size(i) : h->U_rows[i];
      if (rows == 0) continue;
      const bool has = k > 0 && h->sym_U_off[i] >= 0;
      const int nrp = (rows + RB - 1) / RB;
      for (int rp = 0; rp < nrp; ++rp) {
        SymJob j = new_job();
        j.A = has ? base + h->sym_U_off[i] : base;
        j.lda = align4(rows);
        j.r0 = rp * RB;
        j.R = std::min(RB, rows - j.r0);
        j.c0 = 0;
        j.c1 = has ? k : 0;
        j.S = sym_stage_cols(j.R, nc);
        if (leaf) {
          j.y1 = p.ys.p + T.begin[i] + j.r0;
          j.y1rs = 1;
          j.y1cs = n;
          j.mode1 = 0;
        } else {
          j.y1 = yh + (h->skel_off[T.child_begin[i]] + j.r0) * nc;
          j.y1rs = nc;
          j.y1cs = 1;
          j.mode1 = 1;
        }
        j.x1 = yh + h->skel_off[i] * nc;
        j.cmap = nullptr;
        b->bytes += 4.0 * (double)j.R * (j.c1 - j.c0);
        b->flops += 2.0 * (double)j.R * (j.c1 - j.c0) * ncol;
        b->jobs.push_back(j);
      }
    }
  }
  P.part.alloc((size_t)std::max<int64_t>(part_tot, 4));
  for (const Patch& q : patches) {
    PlanStep& st = P.steps[q.step];
    if (q.which == 0) st.sym->jobs[q.idx].y1 = P.part.p + q.off;
    else if (q.which == 1) st.sym->jobs[q.idx].z = P.part.p + q.off;
    else st.sum->srcs[q.idx].p = P.part.p + q.off;
  }
  for (PlanStep& st : P.steps) {
    if (st.sym) st.sym->upload(s);
    if (st.sum) st.sum->upload(s);
  }
  SPD_CUDA(cudaStreamSynchronize(s));
  p.sym = sp;
}

void sym_plan_run(const SymPlan& P, cudaStream_t s) {
  for (const PlanStep& st : P.steps) {
    if (st.sym) st.sym->launch(s);
    if (st.sum) st.sum->launch(s);
  }
}

}  // namespace spd
