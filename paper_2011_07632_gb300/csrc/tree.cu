// Cluster tree on the device: enclosing cube, Morton keys, stable LSD radix sort, the
// 2^d-ary tree level by level (split iff a box holds more than leaf_size points; shallow
// leaves padded with single-child copies down to the deepest level), and the per-level
// near / far (Type-3) lists from the admissibility test of Sec. 5.1.  Integer logic
// after one FP64 subtract-and-multiply per coordinate, so the result is exact.
#include <algorithm>

#include "tree.cuh"

namespace spd {

// ---------------------------------------------------------------------------------------
// int64 exclusive scan
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan_local(int64_t* d, int64_t n, int64_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * 1024 + threadIdx.x * 4;
  int64_t v[4], loc[4];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < n) ? d[base + k] : 0;
    loc[k] = s;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __shared__ int64_t ws[8];
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int w = 0; w < 8; ++w) { const int64_t t = ws[w]; ws[w] = acc; acc += t; }
  }
  __syncthreads();
  const int64_t excl = x - s + ws[warp];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (base + k < n) d[base + k] = excl + loc[k];
  if (threadIdx.x == 255) bsum[blockIdx.x] = excl + s;
}

__global__ void k_scan_add(int64_t* d, int64_t n, const int64_t* boff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] += boff[i / 1024];
}

int64_t exclusive_scan_i64(int64_t* d, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  const int64_t nb = (n + 1023) / 1024;
  DevBuf<int64_t> bs(nb);
  k_scan_local<<<(unsigned)nb, 256, 0, s>>>(d, n, bs.p);
  SPD_LAUNCHED();
  int64_t total = 0;
  if (nb > 1) {
    total = exclusive_scan_i64(bs.p, nb, s);
    k_scan_add<<<ceil_div(n, 256), 256, 0, s>>>(d, n, bs.p);
    SPD_LAUNCHED();
  } else {
    SPD_CUDA(cudaMemcpyAsync(&total, bs.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  }
  SPD_CUDA(cudaStreamSynchronize(s));
  return total;
}

// ---------------------------------------------------------------------------------------
// enclosing cube
// ---------------------------------------------------------------------------------------
__global__ void k_soa_minmax(const double* __restrict__ pts, int64_t n, int dim,
                             double* __restrict__ xs, double* __restrict__ part) {
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < dim; ++a) {
      const double v = pts[p * dim + a];
      xs[a * n + p] = v;
      mn[a] = fmin(mn[a], v);
      mx[a] = fmax(mx[a], v);
    }
  }
  __shared__ double smn[3][256], smx[3][256];
  for (int a = 0; a < 3; ++a) { smn[a][threadIdx.x] = mn[a]; smx[a][threadIdx.x] = mx[a]; }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int a = 0; a < 3; ++a) {
        smn[a][threadIdx.x] = fmin(smn[a][threadIdx.x], smn[a][threadIdx.x + o]);
        smx[a][threadIdx.x] = fmax(smx[a][threadIdx.x], smx[a][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) {
      part[blockIdx.x * 6 + a] = smn[a][0];
      part[blockIdx.x * 6 + 3 + a] = smx[a][0];
    }
}

// box[0..2] = lo, box[3] = w, box[4] = 2^B / w (correctly rounded), box[5] = nonfinite flag
__global__ void k_box_final(const double* part, int nb, int dim, int B, double* box) {
  if (threadIdx.x != 0) return;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      mn[a] = fmin(mn[a], part[b * 6 + a]);
      mx[a] = fmax(mx[a], part[b * 6 + 3 + a]);
    }
  double w = 0.0;
  bool bad = false;
  for (int a = 0; a < dim; ++a) {
    box[a] = mn[a];
    w = fmax(w, __dsub_rn(mx[a], mn[a]));
    bad = bad || !isfinite(mn[a]) || !isfinite(mx[a]);
  }
  box[3] = w;
  box[4] = (w > 0.0) ? __ddiv_rn((double)(1LL << B), w) : 0.0;
  box[5] = bad ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------------------
// Morton keys: q_a = floor((x_a - lo_a) * (2^B / w)), clamped; bit b of q_a at key bit
// b*dim + (dim-1-a)
// ---------------------------------------------------------------------------------------
__global__ void k_keys(const double* __restrict__ xs, int64_t n, int dim, int B,
                       const double* __restrict__ box, uint64_t* __restrict__ keys,
                       int64_t* __restrict__ idx) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double scale = box[4];
  const int64_t top = (1LL << B) - 1;
  int64_t q[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    if (box[3] > 0.0) {
      const double f = floor(__dmul_rn(__dsub_rn(xs[a * n + p], box[a]), scale));
      int64_t v = (int64_t)f;
      v = v < 0 ? 0 : (v > top ? top : v);
      q[a] = v;
    }
  }
  uint64_t key = 0;
  for (int b = B - 1; b >= 0; --b)
    for (int a = 0; a < dim; ++a) key = (key << 1) | (uint64_t)((q[a] >> b) & 1);
  keys[p] = key;
  idx[p] = p;
}

// ---------------------------------------------------------------------------------------
// stable LSD radix sort of (key, value), 4-bit digits, 2048 items per block
// ---------------------------------------------------------------------------------------
constexpr int RS_CHUNK = 2048;

__global__ void __launch_bounds__(256) k_rs_count(const uint64_t* __restrict__ keys, int64_t n,
                                                  int shift, int64_t* __restrict__ counts,
                                                  int nb) {
  __shared__ int c[16];
  if (threadIdx.x < 16) c[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_CHUNK;
  for (int e = threadIdx.x; e < RS_CHUNK; e += 256) {
    const int64_t i = base + e;
    if (i < n) atomicAdd(&c[(keys[i] >> shift) & 15], 1);
  }
  __syncthreads();
  if (threadIdx.x < 16) counts[(int64_t)threadIdx.x * nb + blockIdx.x] = c[threadIdx.x];
}

__global__ void __launch_bounds__(256) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                    const int64_t* __restrict__ vin,
                                                    uint64_t* __restrict__ kout,
                                                    int64_t* __restrict__ vout, int64_t n,
                                                    int shift, const int64_t* __restrict__ offs,
                                                    int nb) {
  __shared__ int cnt[16][257];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * RS_CHUNK + t * 8;
  int loc[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) loc[d] = 0;
  for (int k = 0; k < 8; ++k)
    if (base + k < n) loc[(kin[base + k] >> shift) & 15]++;
#pragma unroll
  for (int d = 0; d < 16; ++d) cnt[d][t] = loc[d];
  __syncthreads();
  const int lane = t & 31, warp = t >> 5;
  for (int d = warp * 2; d < warp * 2 + 2; ++d) {
    int v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) { v[k] = cnt[d][lane * 8 + k]; s += v[k]; }
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    int e = x - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) { cnt[d][lane * 8 + k] = e; e += v[k]; }
  }
  __syncthreads();
  int64_t run[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) run[d] = offs[(int64_t)d * nb + blockIdx.x] + cnt[d][t];
  for (int k = 0; k < 8; ++k) {
    const int64_t i = base + k;
    if (i < n) {
      const uint64_t key = kin[i];
      const int d = (key >> shift) & 15;
      const int64_t pos = run[d]++;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
  }
}

static void radix_sort(uint64_t* keys, int64_t* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1) return;
  const int nb = ceil_div(n, RS_CHUNK);
  DevBuf<uint64_t> k2(n);
  DevBuf<int64_t> v2(n);
  DevBuf<int64_t> counts((size_t)16 * nb);
  uint64_t *ka = keys, *kb = k2.p;
  int64_t *va = vals, *vb = v2.p;
  int passes = (bits + 3) / 4;
  if (passes % 2) ++passes;   // even number of passes: result lands back in (keys, vals)
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 4 * ps;
    k_rs_count<<<nb, 256, 0, s>>>(ka, n, shift, counts.p, nb);
    SPD_LAUNCHED();
    exclusive_scan_i64(counts.p, (int64_t)16 * nb, s);
    k_rs_scatter<<<nb, 256, 0, s>>>(ka, va, kb, vb, n, shift, counts.p, nb);
    SPD_LAUNCHED();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  SPD_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_gather_soa(const double* __restrict__ xin, const int64_t* __restrict__ perm,
                             int64_t n, int dim, double* __restrict__ xout) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t o = perm[p];
  for (int a = 0; a < dim; ++a) xout[a * n + p] = xin[a * n + o];
}

// unknowns of a vector-valued kernel: sorted unknown k*p + c is component c of sorted
// point p, original unknown k*perm[p] + c; coordinates repeated, row `dim` holds c
__global__ void k_expand_dofs(const double* __restrict__ xs, const int64_t* __restrict__ perm,
                              int64_t n, int dim, int k, double* __restrict__ xd,
                              int64_t* __restrict__ pd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t p = e / k;
  const int c = (int)(e - p * k);
  const int64_t N = n * k;
  for (int a = 0; a < dim; ++a) xd[a * N + e] = xs[a * n + p];
  xd[dim * N + e] = (double)c;
  pd[e] = perm[p] * k + c;
}

void expand_dofs(int k, cudaStream_t s, TreeHost& th, TreeDev& td) {
  if (k <= 1) return;
  const int64_t n = th.n, N = n * k;
  DevBuf<double> xd((size_t)(th.dim + 1) * N);
  DevBuf<int64_t> pd(N);
  k_expand_dofs<<<ceil_div(N, 256), 256, 0, s>>>(td.xs.p, td.perm.p, n, th.dim, k, xd.p, pd.p);
  SPD_LAUNCHED();
  SPD_CUDA(cudaStreamSynchronize(s));
  td.xs = std::move(xd);
  td.perm = std::move(pd);
  th.n = N;
  th.dofs = k;
  for (auto& v : th.begin) v *= k;
  for (auto& v : th.end) v *= k;
  td.begin.upload(th.begin, s);
  td.end.upload(th.end, s);
}

// ---------------------------------------------------------------------------------------
// tree level by level
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t key_coord(uint64_t key, int a, int dim, int B) {
  int64_t q = 0;
  for (int b = 0; b < B; ++b) q |= (int64_t)((key >> (b * dim + (dim - 1 - a))) & 1ULL) << b;
  return q;
}

// node id of every point at this depth and node begins
__global__ void k_node_ids(const int64_t* __restrict__ flag, const int64_t* __restrict__ excl,
                           int64_t n, int64_t* __restrict__ nid, int64_t* __restrict__ nbegin) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t id = excl[p] + flag[p] - 1;
  nid[p] = id;
  if (flag[p]) nbegin[id] = p;
}

// per node: end, split flag, parent, cell
__global__ void k_node_info(int64_t nn, int64_t n, int t, int dim, int B, int leaf_size,
                            const int64_t* __restrict__ nbegin, int64_t* __restrict__ nend,
                            int64_t* __restrict__ split, const uint64_t* __restrict__ keys,
                            const int64_t* __restrict__ prev_nid, int64_t prev_off,
                            const int64_t* __restrict__ prev_split,
                            const int64_t* __restrict__ prev_cell,
                            const int64_t* __restrict__ prev_width, int64_t* __restrict__ parent,
                            int64_t* __restrict__ cell, int64_t* __restrict__ width,
                            int64_t* __restrict__ nsplit) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t b = nbegin[k];
  const int64_t e = (k + 1 < nn) ? nbegin[k + 1] : n;
  nend[k] = e;
  const int sp = (e - b > leaf_size) && (t < B);
  split[k] = sp;
  if (sp) atomicAdd((unsigned long long*)nsplit, 1ULL);
  int64_t par = -1;
  bool genuine = true;
  if (t > 0) {
    const int64_t pl = prev_nid[b];
    par = prev_off + pl;
    genuine = prev_split[pl] != 0;
    if (!genuine) {
      for (int a = 0; a < dim; ++a) cell[k * dim + a] = prev_cell[pl * dim + a];
      width[k] = prev_width[pl];
    }
  }
  parent[k] = par;
  if (genuine) {
    const int sh = B - t;
    for (int a = 0; a < dim; ++a) cell[k * dim + a] = (key_coord(keys[b], a, dim, B) >> sh) << sh;
    width[k] = 1LL << sh;
  }
}

// next depth's node starts: a split node starts a child wherever the depth-(t+1) prefix changes
__global__ void k_next_flags(int64_t* __restrict__ flag, const int64_t* __restrict__ nid,
                             const int64_t* __restrict__ split, const uint64_t* __restrict__ keys,
                             int64_t n, int shift) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || p == 0) return;
  if (flag[p]) return;
  if (split[nid[p]] && ((keys[p] >> shift) != (keys[p - 1] >> shift))) flag[p] = 1;
}

// children ranges of depth-t nodes (global ids) from the depth-(t+1) node ids
__global__ void k_children(int64_t nn, const int64_t* __restrict__ nbegin,
                           const int64_t* __restrict__ nend, const int64_t* __restrict__ next_nid,
                           int64_t next_off, int64_t* __restrict__ cb, int64_t* __restrict__ ce) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  cb[k] = next_off + next_nid[nbegin[k]];
  ce[k] = next_off + next_nid[nend[k] - 1] + 1;
}

__device__ __forceinline__ bool admissible(const int64_t* ci, int64_t wi, const int64_t* cj,
                                           int64_t wj, int dim) {
  int64_t gap = 0;
  for (int a = 0; a < dim; ++a) {
    const int64_t g1 = cj[a] - (ci[a] + wi);
    const int64_t g2 = ci[a] - (cj[a] + wj);
    const int64_t g = g1 > g2 ? g1 : g2;
    gap = g > gap ? g : gap;
  }
  return gap >= (wi > wj ? wi : wj);
}

// near / far lists of depth-t nodes from the near lists of their parents (depth t-1).
// Cells and widths are indexed by global node id; pass = 0 counts, pass = 1 fills.
__global__ void k_lists(int64_t nn, int64_t off, int dim, const int64_t* __restrict__ parent,
                        const int64_t* __restrict__ pnear_off, const int64_t* __restrict__ pnear_idx,
                        int64_t poff, const int64_t* __restrict__ child_b,
                        const int64_t* __restrict__ child_e, const int64_t* __restrict__ cell,
                        const int64_t* __restrict__ width, int pass, int64_t* __restrict__ ncnt,
                        int64_t* __restrict__ fcnt, int64_t* __restrict__ nidx,
                        int64_t* __restrict__ fidx) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const int64_t i = off + k;
  const int64_t p = parent[k] - poff;
  int64_t cn = 0, cf = 0;
  int64_t wn = pass ? ncnt[k] : 0, wf = pass ? fcnt[k] : 0;
  for (int64_t jj = pnear_off[p]; jj < pnear_off[p + 1]; ++jj) {
    const int64_t j = pnear_idx[jj] - poff;
    for (int64_t c = child_b[j]; c < child_e[j]; ++c) {
      const bool adm = admissible(cell + i * dim, width[i], cell + c * dim, width[c], dim);
      if (adm) {
        if (pass) fidx[wf++] = c;
        ++cf;
      } else {
        if (pass) nidx[wn++] = c;
        ++cn;
      }
    }
  }
  if (!pass) { ncnt[k] = cn; fcnt[k] = cf; }
}

void build_tree(const double* d_points, int64_t n, int dim, int leaf_size, cudaStream_t s,
                TreeHost& th, TreeDev& td) {
  SPD_REQUIRE(n >= 1, "h2_build: n must be >= 1");
  SPD_REQUIRE(dim == 2 || dim == 3, "h2_build: dim must be 2 or 3");
  SPD_REQUIRE(leaf_size >= 1, "h2_build: leaf_size must be >= 1");
  const int B = (dim == 3) ? 21 : 31;
  th = TreeHost();
  th.n = n;
  th.dim = dim;
  th.leaf_size = leaf_size;
  th.B = B;

  DevBuf<double> xin((size_t)dim * n);
  const int nbm = std::min(ceil_div(n, 256), 1024);
  DevBuf<double> part((size_t)nbm * 6), box(6);
  k_soa_minmax<<<nbm, 256, 0, s>>>(d_points, n, dim, xin.p, part.p);
  SPD_LAUNCHED();
  k_box_final<<<1, 32, 0, s>>>(part.p, nbm, dim, B, box.p);
  SPD_LAUNCHED();
  std::vector<double> hbox = box.download(s);
  SPD_REQUIRE(hbox[5] == 0.0, "h2_build: points contain NaN or Inf");
  for (int a = 0; a < dim; ++a) th.lo[a] = hbox[a];
  th.w = hbox[3];

  DevBuf<uint64_t> keys(n);
  td.perm.alloc(n);
  k_keys<<<ceil_div(n, 256), 256, 0, s>>>(xin.p, n, dim, B, box.p, keys.p, td.perm.p);
  SPD_LAUNCHED();
  radix_sort(keys.p, td.perm.p, n, dim * B, s);
  td.xs.alloc((size_t)dim * n);
  k_gather_soa<<<ceil_div(n, 256), 256, 0, s>>>(xin.p, td.perm.p, n, dim, td.xs.p);
  SPD_LAUNCHED();

  // level-by-level construction
  struct Depth {
    int64_t nn = 0, off = 0;
    DevBuf<int64_t> nid, begin, end, split, parent, cell, width, cb, ce;
    DevBuf<int64_t> noff, nidx, foff, fidx;
  };
  std::vector<Depth> dep;
  DevBuf<int64_t> flag(n), excl(n), nsplit(1);
  flag.zero(s);
  {
    const int64_t one = 1;
    SPD_CUDA(cudaMemcpyAsync(flag.p, &one, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }
  int64_t off = 0;
  for (int t = 0;; ++t) {
    SPD_CUDA(cudaMemcpyAsync(excl.p, flag.p, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    const int64_t nn = exclusive_scan_i64(excl.p, n, s);
    dep.emplace_back();
    Depth& d = dep.back();
    d.nn = nn;
    d.off = off;
    d.nid.alloc(n);
    d.begin.alloc(nn);
    d.end.alloc(nn);
    d.split.alloc(nn);
    d.parent.alloc(nn);
    d.cell.alloc((size_t)nn * dim);
    d.width.alloc(nn);
    k_node_ids<<<ceil_div(n, 256), 256, 0, s>>>(flag.p, excl.p, n, d.nid.p, d.begin.p);
    SPD_LAUNCHED();
    nsplit.zero(s);
    const Depth* pd = t > 0 ? &dep[t - 1] : nullptr;
    k_node_info<<<ceil_div(nn, 256), 256, 0, s>>>(
        nn, n, t, dim, B, leaf_size, d.begin.p, d.end.p, d.split.p, keys.p,
        pd ? pd->nid.p : nullptr, pd ? pd->off : 0, pd ? pd->split.p : nullptr,
        pd ? pd->cell.p : nullptr, pd ? pd->width.p : nullptr, d.parent.p, d.cell.p, d.width.p,
        nsplit.p);
    SPD_LAUNCHED();
    int64_t hs = 0;
    SPD_CUDA(cudaMemcpyAsync(&hs, nsplit.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SPD_CUDA(cudaStreamSynchronize(s));
    off += nn;
    if (hs == 0) break;
    const int shift = dim * (B - t - 1);
    k_next_flags<<<ceil_div(n, 256), 256, 0, s>>>(flag.p, d.nid.p, d.split.p, keys.p, n, shift);
    SPD_LAUNCHED();
  }
  const int D = (int)dep.size() - 1;
  th.D = D;
  th.depth_off.assign(D + 2, 0);
  for (int t = 0; t <= D; ++t) th.depth_off[t + 1] = th.depth_off[t] + dep[t].nn;
  const int64_t NN = th.depth_off[D + 1];

  // children ranges, then global cells/widths for the list kernels
  for (int t = 0; t <= D; ++t) {
    Depth& d = dep[t];
    d.cb.alloc(d.nn);
    d.ce.alloc(d.nn);
    if (t < D) {
      k_children<<<ceil_div(d.nn, 256), 256, 0, s>>>(d.nn, d.begin.p, d.end.p, dep[t + 1].nid.p,
                                                     dep[t + 1].off, d.cb.p, d.ce.p);
      SPD_LAUNCHED();
    } else {
      d.cb.zero(s);
      d.ce.zero(s);
    }
  }
  DevBuf<int64_t> gcell((size_t)NN * dim), gwidth(NN);
  for (int t = 0; t <= D; ++t) {
    SPD_CUDA(cudaMemcpyAsync(gcell.p + dep[t].off * dim, dep[t].cell.p,
                             dep[t].nn * dim * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SPD_CUDA(cudaMemcpyAsync(gwidth.p + dep[t].off, dep[t].width.p, dep[t].nn * sizeof(int64_t),
                             cudaMemcpyDeviceToDevice, s));
  }
  // lists
  {
    Depth& d0 = dep[0];
    d0.noff.upload(std::vector<int64_t>{0, 1}, s);
    d0.nidx.upload(std::vector<int64_t>{0}, s);
    d0.foff.upload(std::vector<int64_t>{0, 0}, s);
    d0.fidx.alloc(0);
  }
  for (int t = 1; t <= D; ++t) {
    Depth& d = dep[t];
    Depth& p = dep[t - 1];
    d.noff.alloc(d.nn + 1);
    d.foff.alloc(d.nn + 1);
    d.noff.zero(s);
    d.foff.zero(s);
    k_lists<<<ceil_div(d.nn, 128), 128, 0, s>>>(d.nn, d.off, dim, d.parent.p, p.noff.p, p.nidx.p,
                                                p.off, p.cb.p, p.ce.p, gcell.p, gwidth.p, 0,
                                                d.noff.p, d.foff.p, nullptr, nullptr);
    SPD_LAUNCHED();
    const int64_t tn = exclusive_scan_i64(d.noff.p, d.nn + 1, s);
    const int64_t tf = exclusive_scan_i64(d.foff.p, d.nn + 1, s);
    d.nidx.alloc(tn);
    d.fidx.alloc(tf);
    k_lists<<<ceil_div(d.nn, 128), 128, 0, s>>>(d.nn, d.off, dim, d.parent.p, p.noff.p, p.nidx.p,
                                                p.off, p.cb.p, p.ce.p, gcell.p, gwidth.p, 1,
                                                d.noff.p, d.foff.p, d.nidx.p, d.fidx.p);
    SPD_LAUNCHED();
  }

  // host mirror
  th.begin.clear(); th.end.clear(); th.parent.clear(); th.child_begin.clear();
  th.child_end.clear(); th.cell_lo.clear(); th.width.clear();
  th.near_off.assign(1, 0); th.far_off.assign(1, 0);
  th.near_idx.clear(); th.far_idx.clear();
  auto app = [](std::vector<int64_t>& dst, const std::vector<int64_t>& src) {
    dst.insert(dst.end(), src.begin(), src.end());
  };
  for (int t = 0; t <= D; ++t) {
    Depth& d = dep[t];
    app(th.begin, d.begin.download(s));
    app(th.end, d.end.download(s));
    app(th.parent, d.parent.download(s));
    app(th.child_begin, d.cb.download(s));
    app(th.child_end, d.ce.download(s));
    app(th.cell_lo, d.cell.download(s));
    app(th.width, d.width.download(s));
    std::vector<int64_t> no = d.noff.download(s), ni = d.nidx.download(s);
    std::vector<int64_t> fo = d.foff.download(s), fi = d.fidx.download(s);
    const int64_t nb0 = th.near_idx.size(), fb0 = th.far_idx.size();
    for (int64_t k = 1; k <= d.nn; ++k) {
      th.near_off.push_back(nb0 + no[k]);
      th.far_off.push_back(fb0 + fo[k]);
    }
    app(th.near_idx, ni);
    app(th.far_idx, fi);
  }
  for (int64_t i = 0; i < NN; ++i)
    if (th.child_begin[i] == th.child_end[i]) th.child_begin[i] = th.child_end[i] = 0;
  td.begin.upload(th.begin, s);
  td.end.upload(th.end, s);
  td.near_off.upload(th.near_off, s);
  td.near_idx.upload(th.near_idx, s);
  td.far_off.upload(th.far_off, s);
  td.far_idx.upload(th.far_idx, s);
  SPD_CUDA(cudaStreamSynchronize(s));
}

}  // namespace spd
