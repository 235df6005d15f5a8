// Proxy-point H^2 construction and H^2 products.
//
// Construction, bottom-up over the depths: for every node with a far field, the proxy
// matrix K(P_i, X_cand) (candidates: the node's points at the leaf level, the children's
// skeleton points above) is factored by column-pivoted QR stopped at |R_kk| <= tol |R_00|;
// the interpolative decomposition U = Pi [I; (R11^{-1} R12)^T] is the leaf basis / transfer
// matrix and the first k pivots are the skeleton.  Couplings B_ij = K(X_skel_i, X_skel_j)
// for the Type-3 pairs (Sec. 5.2.2) are stored once per unordered pair.
#include <algorithm>
#include <type_traits>

#include "h2.cuh"

namespace spd {

// ---- ID: U (m x k) from the pivots and T = R11^{-1} R12 stored over R12 ---------------
struct IdProb {
  const double* G;   // QR workspace, ld np: T[b, a-k] at G[b + a*np] for a >= k
  int64_t ldg;
  const int* piv;
  const int* rank;
  double* U;         // m x k, ld m
  int m;
};

__global__ void k_id_assemble(const IdProb* __restrict__ probs) {
  const IdProb P = probs[blockIdx.x];
  const int k = *P.rank;
  const int m = P.m;
  for (int64_t e = threadIdx.x; e < (int64_t)m * k; e += blockDim.x) {
    const int a = (int)(e % m), b = (int)(e / m);
    const double v = (a < k) ? (a == b ? 1.0 : 0.0) : P.G[b + (int64_t)a * P.ldg];
    P.U[P.piv[a] + (int64_t)b * m] = v;
  }
}

__global__ void k_gather_coords(const double* __restrict__ xs, int64_t n, int dim,
                                const int64_t* __restrict__ idx, int64_t K,
                                double* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= K) return;
  for (int a = 0; a < dim; ++a) out[a * K + r] = xs[a * n + idx[r]];
}

__global__ void k_perm_to(const double* __restrict__ X, int64_t ldx, double* __restrict__ Xs,
                          int64_t n, int ncol, const int64_t* __restrict__ perm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncol) return;
  const int64_t p = e % n, c = e / n;
  Xs[p + c * n] = X[perm[p] + c * ldx];
}

__global__ void k_perm_from(const double* __restrict__ Xs, double* __restrict__ Y, int64_t ldy,
                            int64_t n, int ncol, const int64_t* __restrict__ perm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncol) return;
  const int64_t p = e % n, c = e / n;
  Y[perm[p] + c * ldy] = Xs[p + c * n];
}

void permute_to_sorted(const double* X, int64_t ldx, double* Xs, int64_t n, int ncol,
                       const int64_t* perm, cudaStream_t s) {
  k_perm_to<<<ceil_div(n * ncol, 256), 256, 0, s>>>(X, ldx, Xs, n, ncol, perm);
  SPD_LAUNCHED();
}

void permute_from_sorted(const double* Xs, double* Y, int64_t ldy, int64_t n, int ncol,
                         const int64_t* perm, cudaStream_t s) {
  k_perm_from<<<ceil_div(n * ncol, 256), 256, 0, s>>>(Xs, Y, ldy, n, ncol, perm);
  SPD_LAUNCHED();
}

static bool has_far_field(const TreeHost& T, int64_t i) {
  const int64_t wd = T.width[i];
  const int64_t top = 1LL << T.B;
  for (int a = 0; a < T.dim; ++a) {
    const int64_t lo = T.cell_lo[i * T.dim + a];
    if (lo - wd > 0 || top - (lo + wd) - wd > 0) return true;
  }
  return false;
}

void h2_build_impl(spdhss_h2_s* h, const double* d_points, int64_t n, int dim, int leaf_size,
                   cudaStream_t s) {
  build_tree(d_points, n, dim, leaf_size, s, h->th, h->td);
  // a vector-valued kernel: from here on the tree counts unknowns, and every proxy point
  // carries one row per component
  expand_dofs(kernel_dofs(h->kfn.kind), s, h->th, h->td);
  n = h->th.n;
  const TreeHost& T = h->th;
  const int64_t NN = T.nn();
  const int D = T.D;
  const int crow = dim + (T.dofs > 1 ? 1 : 0);   // coordinate rows (+ component row)
  const int np = proxy_count(dim) * T.dofs;
  const double hg = T.w / (double)(1LL << T.B);

  std::vector<int> rank(NN, 0), mrows(NN, 0);
  std::vector<std::vector<int64_t>> skel_local(NN);   // skeleton (sorted point indices)
  std::vector<DevBuf<double>> sx(D + 2);              // per-depth skeleton coordinates
  std::vector<std::vector<int64_t>> soff(D + 2);      // per-depth local skeleton offsets
  std::vector<std::unique_ptr<DevBuf<double>>> upool;
  std::vector<double*> Uptr(NN, nullptr);

  for (int t = D; t >= 1; --t) {
    merge_stage(1, D - t);   // batched sweeps align the levels by height above the leaves
    const int64_t o = T.depth_off[t], nn = T.depth_off[t + 1] - o;
    // candidate rows
    for (int64_t k = 0; k < nn; ++k) {
      const int64_t i = o + k;
      if (t == D) mrows[i] = (int)T.size(i);
      else {
        int m = 0;
        for (int64_t c = T.child_begin[i]; c < T.child_end[i]; ++c) m += rank[c];
        mrows[i] = m;
      }
    }
    // batches bounded by scratch memory
    std::vector<int64_t> todo;
    for (int64_t k = 0; k < nn; ++k)
      if (mrows[o + k] > 0 && has_far_field(T, o + k)) todo.push_back(o + k);
    const size_t budget = (size_t)3 << 30;
    // a node with few candidates takes the blocked QR (proxy rows evaluated and factored
    // block by block in shared memory, the block triangles merged pairwise, the pivoted QR
    // on the m x m result); a wider one the pivoted QR of its whole proxy matrix
    auto blocked = [&](int m) { return m <= kIdTsqrMaxM; };
    auto nblocks = [&](int m) { return ceil_div(np, id_tsqr_rows(m, np)); };
    auto work_doubles = [&](int m) -> int64_t {
      return blocked(m) ? (int64_t)nblocks(m) * m * m : (int64_t)np * m;
    };
    // merge rounds: fixed by the proxy count (the most blocks any node can have), so that
    // every instance of a batched sweep makes the same sequence of launches
    int rounds = 0, most = 1;
    for (int m = 1; m <= kIdTsqrMaxM; ++m) most = std::max(most, nblocks(m));
    while ((1 << rounds) < most) ++rounds;
    size_t pos = 0;
    while (pos < todo.size()) {
      size_t end = pos, bytes = 0;
      while (end < todo.size()) {
        const size_t b = (size_t)work_doubles(mrows[todo[end]]) * sizeof(double);
        if (end > pos && bytes + b > budget) break;
        bytes += b;
        ++end;
      }
      const size_t nb = end - pos;
      std::vector<int64_t> goff(nb + 1, 0), coff(nb + 1, 0), ldg(nb, np);
      int maxm = 0, maxrows = 1;
      for (size_t b = 0; b < nb; ++b) {
        const int m = mrows[todo[pos + b]];
        goff[b + 1] = goff[b] + work_doubles(m);
        coff[b + 1] = coff[b] + m;
        maxm = std::max(maxm, m);
        if (blocked(m)) ldg[b] = m;
        maxrows = std::max<int>(maxrows, (int)ldg[b]);
      }
      DevBuf<double> G(goff[nb]), tau(coff[nb]), norms(2 * coff[nb]);
      DevBuf<int> piv(coff[nb]), rk(nb);
      Batch<ProxyProb> pb;
      Batch<ProxyQrProb> zb[2];                 // row blocks: narrow, wide (m > 113)
      std::vector<std::pair<int64_t, int>> tri; // blocked nodes: (R stack offset, m)
      std::vector<int> trib;                    // and their block counts
      Batch<QrProb> qb, qs;                     // pivoted QRs: whole proxy matrices, triangles
      for (size_t b = 0; b < nb; ++b) {
        const int64_t i = todo[pos + b];
        ProxyProb p;
        const double side = (double)T.width[i] * hg;
        const double hh = 0.5 * side;
        double H = 0.0;
        for (int a = 0; a < 3; ++a) p.c[a] = 0.0;
        for (int a = 0; a < dim; ++a) {
          const double blo = T.lo[a] + (double)T.cell_lo[i * dim + a] * hg;
          p.c[a] = blo + hh;
          H = std::max(H, std::max(p.c[a] - T.lo[a], T.lo[a] + T.w - p.c[a]));
        }
        p.h = hh;
        p.H = std::max(H, 3.0 * hh * (1.0 + 1e-12));
        p.scale = proxy_scale(h->kfn, hh);
        if (t == D) {
          p.xc = h->td.xs.p; p.ldxc = n; p.c0 = T.begin[i];
        } else {
          const int64_t cb = T.child_begin[i] - T.depth_off[t + 1];
          p.xc = sx[t + 1].p; p.ldxc = (int64_t)sx[t + 1].n / crow; p.c0 = soff[t + 1][cb];
        }
        const int m = mrows[i];
        p.cols = m;
        QrProb q;
        if (blocked(m)) {
          // R_b of every row block into the node's stack; the merged R in block 0
          const int br = id_tsqr_rows(m, np), nbk = nblocks(m);
          for (int k2 = 0; k2 < nbk; ++k2) {
            ProxyQrProb z;
            z.p = p;
            z.p.out = G.p + goff[b] + (int64_t)k2 * m * m;
            z.p.ldo = m;
            z.r0 = k2 * br;
            z.rows = std::min(br, np - k2 * br);
            zb[m * m > kIdTsqrBlockEntries ? 1 : 0].push(z);
          }
          tri.emplace_back(goff[b], m);
          trib.push_back(nbk);
          q.A = G.p + goff[b]; q.lda = m; q.m = m;
          q.n = m;
          q.kmax = m; q.rtol = h->tol;
          q.piv = piv.p + coff[b]; q.tau = tau.p + coff[b]; q.rank = rk.p + b;
          q.norms = norms.p + 2 * coff[b];
          qs.push(q);
          continue;
        } else {
          p.out = G.p + goff[b];
          p.ldo = np;
          pb.push(p);
          q.A = G.p + goff[b]; q.lda = np; q.m = np;
        }
        q.n = m;
        q.kmax = std::min(q.m, m); q.rtol = h->tol;
        q.piv = piv.p + coff[b]; q.tau = tau.p + coff[b]; q.rank = rk.p + b;
        q.norms = norms.p + 2 * coff[b];
        qb.push(q);
      }
      pb.upload(s);
      proxy_launch(pb, h->kfn, dim, s);
      for (auto& z : zb) {
        z.upload(s);
        proxy_qr_launch(z, h->kfn, dim, "qr_h2_id_blocks", s);
      }
      // pairwise merges of the block triangles, block q absorbing block q + 2^r
      for (int r = 0; r < rounds; ++r) {
        Batch<TriMergeProb> mb;
        for (size_t t2 = 0; t2 < tri.size(); ++t2) {
          const int m = tri[t2].second, nbk = trib[t2];
          const int64_t mm = (int64_t)m * m;
          for (int q2 = 0; q2 + (1 << r) < nbk; q2 += 2 << r)
            mb.push(TriMergeProb{G.p + tri[t2].first + q2 * mm,
                                 G.p + tri[t2].first + (q2 + (1 << r)) * mm, m});
        }
        mb.upload(s);
        tri_merge_launch(mb, "qr_h2_id_merge", s);
      }
      qs.upload(s);
      const int sslot = geqp3_small_launch(qs, "qr_h2_id_pivot", s);
      qb.tag = "geqp3_h2_id";
      qb.upload(s);
      // cluster size: by the widest matrix, and wide enough that small batches still put
      // about two CTAs on every SM (the columns of a matrix are split over its cluster)
      int cl = maxm <= 128 ? 1 : (maxm <= 256 ? 2 : (maxm <= 512 ? 4 : 8));
      while (cl < 8 && (int64_t)nb * cl < 2 * 152 && maxm >= 32 * cl) cl *= 2;
      const int pslot = geqp3_launch(qb, 1, cl, maxrows, s);
      std::vector<int> hrk = rk.download(s);
      {
        double f = 0.0, fs = 0.0;
        for (size_t b = 0; b < nb; ++b) {
          const double fb = qr_flops((int)ldg[b], mrows[todo[pos + b]], hrk[b], true);
          (blocked(mrows[todo[pos + b]]) ? fs : f) += fb;
        }
        if (pslot >= 0) prof_add_flops(pslot, f);
        if (sslot >= 0) prof_add_flops(sslot, fs);
      }
      std::vector<int> hpiv = piv.download(s);
      // T = R11^{-1} R12 in place, then U
      Batch<TrsmProb> tb;
      Batch<IdProb> ib;
      size_t ubytes = 0;
      for (size_t b = 0; b < nb; ++b) ubytes += (size_t)mrows[todo[pos + b]] * hrk[b];
      upool.emplace_back(new DevBuf<double>(std::max<size_t>(ubytes, 1)));
      double* up = upool.back()->p;
      for (size_t b = 0; b < nb; ++b) {
        const int64_t i = todo[pos + b];
        const int k = hrk[b], m = mrows[i];
        rank[i] = k;
        Uptr[i] = up;
        if (k < m && k > 0) {
          TrsmProb tp;
          tp.T = G.p + goff[b]; tp.ldt = ldg[b];
          tp.B = G.p + goff[b] + (int64_t)k * ldg[b]; tp.ldb = ldg[b];
          tp.n = k; tp.ncol = m - k; tp.lower = 0; tp.trans = 0;
          tb.push(tp);
        }
        IdProb ip;
        ip.G = G.p + goff[b]; ip.ldg = ldg[b]; ip.piv = piv.p + coff[b]; ip.rank = rk.p + b;
        ip.U = up; ip.m = m;
        ib.push(ip);
        up += (size_t)m * k;
        // skeleton: candidates in pivot order
        std::vector<int64_t>& sk = skel_local[i];
        sk.resize(k);
        for (int a = 0; a < k; ++a) {
          const int pv = hpiv[coff[b] + a];
          if (t == D) sk[a] = T.begin[i] + pv;
          else {
            int acc = 0;
            int64_t cnode = T.child_begin[i];
            for (; cnode < T.child_end[i]; ++cnode) {
              if (pv < acc + rank[cnode]) break;
              acc += rank[cnode];
            }
            sk[a] = skel_local[cnode][pv - acc];
          }
        }
      }
      tb.tag = "trsm_h2_id";
      tb.upload(s);
      trsm_launch(tb, s);
      ib.upload(s);
      if (!ib.empty()) {
        k_id_assemble<<<(unsigned)ib.size(), 256, 0, s>>>(ib.d.p);
        SPD_LAUNCHED();
      }
      pos = end;
    }
    // per-depth skeleton offsets and coordinates
    soff[t].assign(nn + 1, 0);
    std::vector<int64_t> sidx;
    for (int64_t k = 0; k < nn; ++k) {
      soff[t][k + 1] = soff[t][k] + rank[o + k];
      for (int64_t v : skel_local[o + k]) sidx.push_back(v);
    }
    const int64_t Kt = soff[t][nn];
    sx[t].alloc((size_t)std::max<int64_t>(Kt, 1) * crow);
    if (Kt > 0) {
      DevBuf<int64_t> di;
      di.upload(sidx, s);
      k_gather_coords<<<ceil_div(Kt, 256), 256, 0, s>>>(h->td.xs.p, n, crow, di.p, Kt, sx[t].p);
      SPD_LAUNCHED();
    }
    // sx[t].n is used as the leading dimension holder: crow * Kt entries
    if (Kt == 0) sx[t].n = crow;
  }

  // global skeleton arrays (node-major) and bases
  merge_stage(2, 0);
  h->skel_off.assign(NN + 1, 0);
  h->skel_idx.clear();
  h->U_rows.assign(NN, 0);
  h->U_off.assign(NN, 0);
  int mxr = 0;
  for (int64_t i = 0; i < NN; ++i) {
    h->skel_off[i + 1] = h->skel_off[i] + rank[i];
    for (int64_t v : skel_local[i]) h->skel_idx.push_back(v);
    h->U_rows[i] = mrows[i];
    mxr = std::max(mxr, rank[i]);
  }
  h->max_rank = mxr;
  h->Ktot = h->skel_off[NN];
  // one contiguous basis pool
  int64_t btot = 0;
  for (int64_t i = 0; i < NN; ++i) { h->U_off[i] = btot; btot += (int64_t)mrows[i] * rank[i]; }
  h->basis.alloc(std::max<int64_t>(btot, 1));
  {
    Batch<CopyProb> cb;
    for (int64_t i = 0; i < NN; ++i)
      if ((int64_t)mrows[i] * rank[i] > 0) {
        CopyProb c;
        c.src = Uptr[i]; c.lds = mrows[i]; c.dst = h->basis.p + h->U_off[i]; c.ldd = mrows[i];
        c.m = mrows[i]; c.n = rank[i]; c.trans = 0; c.accumulate = 0; c.alpha = 1.0;
        cb.push(c);
      }
    cb.upload(s);
    copy_launch(cb, s);
  }
  upool.clear();
  const int64_t K = h->Ktot;
  h->skel_x.alloc((size_t)std::max<int64_t>(K, 1) * crow);
  if (K > 0) {
    DevBuf<int64_t> di;
    di.upload(h->skel_idx, s);
    k_gather_coords<<<ceil_div(K, 256), 256, 0, s>>>(h->td.xs.p, n, crow, di.p, K, h->skel_x.p);
    SPD_LAUNCHED();
  }

  // couplings, once per unordered far pair
  const int64_t nfar = (int64_t)T.far_idx.size();
  h->far_boff.assign(nfar, 0);
  h->far_trans.assign(nfar, 0);
  int64_t ctot = 0;
  std::vector<int64_t> own(nfar, -1);
  for (int64_t i = 0; i < NN; ++i)
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      if (i < j) { own[e] = ctot; ctot += (int64_t)rank[i] * rank[j]; }
    }
  for (int64_t i = 0; i < NN; ++i)
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      if (i < j) { h->far_boff[e] = own[e]; h->far_trans[e] = 0; }
      else {
        const auto b0 = T.far_idx.begin() + T.far_off[j], b1 = T.far_idx.begin() + T.far_off[j + 1];
        const auto it = std::lower_bound(b0, b1, i);
        SPD_REQUIRE(it != b1 && *it == i, "h2_build: far lists are not symmetric");
        h->far_boff[e] = own[it - T.far_idx.begin()];
        h->far_trans[e] = 1;
      }
    }
  h->coup.alloc(std::max<int64_t>(ctot, 1));
  Batch<TileProb> tb;
  for (int64_t i = 0; i < NN; ++i)
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      if (!(i < j) || rank[i] == 0 || rank[j] == 0) continue;
      TileProb p;
      p.xr = h->skel_x.p; p.ldxr = K; p.r0 = h->skel_off[i]; p.rows = rank[i];
      p.xc = h->skel_x.p; p.ldxc = K; p.c0 = h->skel_off[j]; p.cols = rank[j];
      p.out = h->coup.p + own[e]; p.ldo = rank[i]; p.diag_add = 0.0;
      tb.push(p);
      if (tb.size() >= 200000) { tb.upload(s); tile_launch(tb, h->kfn, dim, s); tb.h.clear(); }
    }
  tb.upload(s);
  tile_launch(tb, h->kfn, dim, s);
  SPD_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------------------
// products
// ---------------------------------------------------------------------------------------
static int lca_level(const TreeHost& T, int64_t i, int64_t j) {
  while (i != j) { i = T.parent[i]; j = T.parent[j]; }
  return T.level_of_depth(T.depth_of(i));
}

// Near blocks are stored (instead of evaluated in every product) when they take at most
// this many bytes: every later product then reads them once instead of spending ~40 FP64
// operations per entry on the kernel function.
constexpr int64_t kNearStoreBytes = int64_t(16) << 30;

static bool near_store(spdhss_h2_s* h, cudaStream_t s) {
  if (h->near_state) return h->near_state == 1;
  const TreeHost& T = h->th;
  const int D = T.D;
  h->near_boff.assign(T.near_idx.size(), 0);
  int64_t tot = 0;
  for (int64_t i = T.depth_off[D]; i < T.depth_off[D + 1]; ++i)
    for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
      h->near_boff[e] = tot;
      tot += T.size(i) * T.size(T.near_idx[e]);
    }
  if (tot * (int64_t)sizeof(double) > kNearStoreBytes) {
    h->near_state = 2;
    return false;
  }
  h->near_blk.alloc(std::max<int64_t>(tot, 1));
  Batch<TileProb> tb;
  for (int64_t i = T.depth_off[D]; i < T.depth_off[D + 1]; ++i)
    for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
      const int64_t j = T.near_idx[e];
      TileProb tp;
      tp.xr = h->td.xs.p; tp.ldxr = T.n; tp.r0 = T.begin[i]; tp.rows = (int)T.size(i);
      tp.xc = h->td.xs.p; tp.ldxc = T.n; tp.c0 = T.begin[j]; tp.cols = (int)T.size(j);
      tp.out = h->near_blk.p + h->near_boff[e]; tp.ldo = T.size(i);
      tp.diag_add = (i == j) ? h->kfn.shift : 0.0;
      tb.push(tp);
    }
  tb.upload(s);
  tile_launch(tb, h->kfn, T.dim, s);
  h->near_state = 1;
  return true;
}

template <class F>
static void h2_plan_build_t(const spdhss_h2_s* h, H2PlanT<F>& p, int ncol, int nslot,
                            const F* Ub, const F* Cb, cudaStream_t s, int tc = 0,
                            bool basis = true) {
  const TreeHost& T = h->th;
  const int64_t n = T.n, K = std::max<int64_t>(h->Ktot, 1);
  const int D = T.D;
  p.ncol = ncol;
  p.nslot = nslot;
  const int W = ncol * nslot;
  p.xs.alloc((size_t)n * ncol);
  p.ys.alloc((size_t)n * W);
  p.xhat.alloc((size_t)K * ncol);
  p.yhat.alloc((size_t)K * W);
  auto U = [&](int64_t i) { return Ub + h->U_off[i]; };
  // upward
  p.up_leaf = GemmBatchT<F>();
  for (int64_t i = T.depth_off[D]; basis && i < T.depth_off[D + 1]; ++i)
    if (h->rank(i) > 0)
      p.up_leaf.add(p.xhat.p + h->skel_off[i], K, h->rank(i), ncol, U(i), h->U_rows[i], 1,
                    p.xs.p + T.begin[i], n, 0, h->U_rows[i], 1.0, 0.0);
  p.up.clear();
  for (int t = D - 1; basis && t >= 1; --t) {
    p.up.emplace_back();
    GemmBatchT<F>& g = p.up.back();
    for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i)
      if (h->rank(i) > 0)
        g.add(p.xhat.p + h->skel_off[i], K, h->rank(i), ncol, U(i), h->U_rows[i], 1,
              p.xhat.p + h->skel_off[T.child_begin[i]], K, 0, h->U_rows[i], 1.0, 0.0);
  }
  // coupling
  p.coupling = GemmBatchT<F>();
  for (int64_t i = 0; Cb != nullptr && i < T.nn(); ++i) {
    if (h->rank(i) == 0) continue;
    const int lev = T.level_of_depth(T.depth_of(i));
    for (int sl = 0; sl < nslot; ++sl) {
      bool opened = false;
      for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
        const int64_t j = T.far_idx[e];
        if (h->rank(j) == 0) continue;
        if (nslot > 1 && lca_level(T, i, j) - 2 != sl) continue;
        if (!opened) {
          p.coupling.prob(p.yhat.p + h->skel_off[i] + (int64_t)sl * ncol * K, K, h->rank(i),
                          ncol, 1.0, 1.0);
          opened = true;
        }
        const int tr = h->far_trans[e];
        p.coupling.seg(Cb + h->far_boff[e], tr ? h->rank(j) : h->rank(i), tr,
                       p.xhat.p + h->skel_off[j], K, 0, h->rank(j));
      }
    }
    (void)lev;
  }
  // downward
  p.down.clear();
  for (int t = 1; basis && t <= D - 1; ++t) {
    p.down.emplace_back();
    GemmBatchT<F>& g = p.down.back();
    for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i) {
      if (h->rank(i) == 0) continue;
      const int lev = T.level_of_depth(t);
      const int s0 = nslot == 1 ? 0 : lev - 1;
      if (s0 >= nslot) continue;
      const int64_t cs = (int64_t)s0 * ncol * K;
      g.add(p.yhat.p + h->skel_off[T.child_begin[i]] + cs, K, h->U_rows[i], (nslot - s0) * ncol,
            U(i), h->U_rows[i], 0, p.yhat.p + h->skel_off[i] + cs, K, 0, h->rank(i), 1.0, 1.0);
    }
  }
  // leaves
  p.leaf_out = GemmBatchT<F>();
  for (int64_t i = T.depth_off[D]; basis && i < T.depth_off[D + 1]; ++i) {
    p.leaf_out.prob(p.ys.p + T.begin[i], n, (int)T.size(i), W, 1.0, 0.0);
    if (h->rank(i) > 0)
      p.leaf_out.seg(U(i), h->U_rows[i], 0, p.yhat.p + h->skel_off[i], K, 0, h->rank(i));
  }
  // near field: grouped GEMMs over the stored blocks (FP64), else evaluated on the fly
  p.near = NearBatchT<F>();
  p.near_g = GemmBatchT<F>();
  p.near_stored = false;
  if constexpr (std::is_same<F, double>::value) {
    if (near_store(const_cast<spdhss_h2_s*>(h), s)) {   // the blocks are a cache of the handle
      p.near_stored = true;
      p.near_rows = (nslot == 1 && ncol <= 4);
      if (p.near_rows) {
        // each leaf's blocks form one |I_i| x sum |I_j| row block: stream it like the couplings
        RowCoupBatchT<F>& rb = p.near_r;
        rb.ncol = ncol;
        rb.tag = "near_h2_stored";
        for (int64_t i = T.depth_off[D]; i < T.depth_off[D + 1]; ++i) {
          if (T.near_off[i] == T.near_off[i + 1] || T.size(i) == 0) continue;
          RowCoupProbT<F> pr;
          pr.C = p.ys.p + T.begin[i];
          pr.ldc = n;
          pr.M = (int)T.size(i);
          pr.ncol = ncol;
          pr.A = h->near_blk.p + h->near_boff[T.near_off[i]];
          pr.beta = 1;
          pr.ch0 = (int)rb.chunks.size();
          int64_t col = 0;
          for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
            const int64_t j = T.near_idx[e];
            const int sj = (int)T.size(j);
            for (int k0 = 0; k0 < sj; k0 += kRowChunk)
              rb.chunks.push_back(RowCoupChunkT<F>{p.xs.p + T.begin[j] + k0, n, col + k0,
                                                   std::min(kRowChunk, sj - k0)});
            col += sj;
          }
          pr.ch1 = (int)rb.chunks.size();
          rb.probs.push_back(pr);
        }
        rb.upload(s);
      }
      for (int64_t i = T.depth_off[D]; !p.near_rows && i < T.depth_off[D + 1]; ++i) {
        for (int sl = 0; sl < nslot; ++sl) {
          bool opened = false;
          for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
            const int64_t j = T.near_idx[e];
            if (nslot > 1) {
              if (j == i) continue;
              if (lca_level(T, i, j) - 2 != sl) continue;
            }
            if (!opened) {
              p.near_g.prob(p.ys.p + T.begin[i] + (int64_t)sl * ncol * n, n, (int)T.size(i),
                            ncol, 1.0, 1.0);
              opened = true;
            }
            p.near_g.seg(h->near_blk.p + h->near_boff[e], T.size(i), 0, p.xs.p + T.begin[j], n,
                         0, (int)T.size(j));
          }
        }
      }
    }
  }
  for (int64_t i = T.depth_off[D]; !p.near_stored && i < T.depth_off[D + 1]; ++i) {
    for (int sl = 0; sl < nslot; ++sl) {
      bool opened = false;
      for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
        const int64_t j = T.near_idx[e];
        if (nslot > 1) {
          if (j == i) continue;
          if (lca_level(T, i, j) - 2 != sl) continue;
        }
        if (!opened) {
          p.near.prob(T.begin[i], (int)T.size(i), p.ys.p + T.begin[i] + (int64_t)sl * ncol * n, n,
                      ncol, 1);
          opened = true;
        }
        p.near.seg(T.begin[j], (int)T.size(j), p.xs.p + T.begin[j], n, j == i ? 1 : 0);
      }
    }
  }
  const bool f32 = sizeof(F) == 4;
  p.coupling.tag = nslot > 1 ? "h2_coupling_sample" : (f32 ? "h2_coupling_f32" : "h2_coupling");
  p.near.tag = nslot > 1 ? "near_sample" : (f32 ? "near_h2_f32" : "near_h2");
  p.near_g.tag = nslot > 1 ? "near_sample_stored" : "near_h2_stored";
  p.near_g.upload(s);
  const char* btag = f32 ? "h2_basis_f32" : "h2_basis";
  p.up_leaf.tag = p.leaf_out.tag = btag;
  for (auto& g : p.up) g.tag = btag;
  for (auto& g : p.down) g.tag = btag;
  if (tc) {   // FP32 plans: the basis and coupling products on the tensor cores
    p.up_leaf.tc = p.leaf_out.tc = p.coupling.tc = tc;
    for (auto& g : p.up) g.tc = tc;
    for (auto& g : p.down) g.tc = tc;
    const char* ttag = nslot > 1 ? "h2_basis_sample_tc" : "h2_basis_tc";
    p.up_leaf.tag = p.leaf_out.tag = ttag;
    for (auto& g : p.up) g.tag = ttag;
    for (auto& g : p.down) g.tag = ttag;
    p.coupling.tag = nslot > 1 ? "h2_coupling_sample_tc" : "h2_coupling_tc";
    p.near.tag = nslot > 1 ? "near_sample_f32" : "near_h2_f32";
  }
  p.up_leaf.upload(s);
  for (auto& g : p.up) g.upload(s);
  p.coupling.upload(s);
  for (auto& g : p.down) g.upload(s);
  p.leaf_out.upload(s);
  p.near.upload(s);
}


__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

__global__ void k_f2d(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}

void convert_d2f(const double* x, float* y, int64_t count, cudaStream_t s) {
  if (count <= 0) return;
  k_d2f<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 16), 256, 0, s>>>(x, y, count);
  SPD_LAUNCHED();
}

void convert_f2d(const float* x, double* y, int64_t count, cudaStream_t s) {
  if (count <= 0) return;
  k_f2d<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 16), 256, 0, s>>>(x, y, count);
  SPD_LAUNCHED();
}

// FP64 coupling block (owner orientation, possibly transposed) -> destination-major copy
template <class TD>
struct CopyDM {
  const double* src;
  int64_t lds;
  int trans;
  TD* dst;
  int64_t ldd;
  int m, n;
};

template <class TD>
__global__ void k_copy_dm(const CopyDM<TD>* __restrict__ probs) {
  const CopyDM<TD> P = probs[blockIdx.y];
  const int64_t tot = (int64_t)P.m * P.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % P.m), j = (int)(e / P.m);
    const double v = P.trans ? P.src[j + (int64_t)i * P.lds] : P.src[i + (int64_t)j * P.lds];
    P.dst[i + (int64_t)j * P.ldd] = (TD)v;
  }
}

// CTA of 256 threads on rows [r0, r0 + 256) of node i's coupling matrix and a range of
// its chunks.  With Mw warps of rows, the CTA holds G = 8 / Mw groups; in round t group g
// takes chunk t * G + g.  Partial sums of the groups are added in group order, and the
// parts of a node split over several CTAs are added in part order (deterministic).
// coupling entries per CTA: about total / (152 SMs x 16), within [4096, 2^20], so that small
// products still spread over many CTAs and large ones keep long streams
constexpr int64_t kRowItemMax = int64_t(1) << 20;
constexpr int64_t kRowItemMin = 4096;

__host__ __device__ constexpr int rowcoup_ncp(int nc) { return nc < 4 ? nc : 4 * ((nc + 3) / 4); }

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <class T, int NC>
__global__ void __launch_bounds__(256) k_coupling_rows(const RowCoupProbT<T>* __restrict__ probs,
                                                       const RowCoupChunkT<T>* __restrict__ chunks,
                                                       const RowCoupWork* __restrict__ work,
                                                       T* __restrict__ partial, int c0) {
  constexpr int NCP = rowcoup_ncp(NC);
  extern __shared__ __align__(16) unsigned char smem_rc_raw[];
  T* smem_rc = reinterpret_cast<T*>(smem_rc_raw);
  T* xs = smem_rc;                            // [G][kRowChunk][NCP]
  const RowCoupWork W = work[blockIdx.x];
  const RowCoupProbT<T> P = probs[W.p];
  const int rows = min(P.M - W.r0, 256);
  const int Mw = (rows + 31) / 32;
  const int G = 8 / Mw;
  const int RW = 32 * Mw;
  const int tid = threadIdx.x;
  const int g = tid / RW, rl = tid % RW;
  const int r = W.r0 + rl;
  const bool active = g < G && rl < rows;
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  const int64_t M = P.M;
  const int nch = W.ch1 - W.ch0;
  const int rounds = (nch + G - 1) / G;
  const int ncl = min(NC, P.ncol - c0);   // columns c0 .. c0 + ncl - 1 of this launch
  for (int t = 0; t < rounds; ++t) {
    // stage: element e -> (group gg, column c, row kk), kk fastest for coalesced reads
    for (int e = tid; e < G * NC * kRowChunk; e += 256) {
      const int gg = e / (NC * kRowChunk);
      const int rem = e - gg * NC * kRowChunk;
      const int c = rem / kRowChunk, kk = rem - c * kRowChunk;
      const int ch = t * G + gg;
      T v = T(0);
      if (ch < nch) {
        const RowCoupChunkT<T> C = chunks[W.ch0 + ch];
        if (kk < C.K && c < ncl) v = C.x[(int64_t)(c0 + c) * C.ldx + kk];
      }
      xs[(gg * kRowChunk + kk) * NCP + c] = v;
    }
    __syncthreads();
    const int ch = t * G + g;
    if (active && ch < nch) {
      const RowCoupChunkT<T> C = chunks[W.ch0 + ch];
      const T* a = P.A + r + C.col * M;
      const T* xg = xs + g * kRowChunk * NCP;
      int kk0 = 0;
      for (; kk0 + 16 <= C.K; kk0 += 16) {
        T b[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) b[u] = __ldg(a + (int64_t)(kk0 + u) * M);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const T* xr = xg + (kk0 + u) * NCP;
          if constexpr (NC >= 4 && sizeof(T) == 4) {
#pragma unroll
            for (int c4 = 0; c4 < NCP / 4; ++c4) {
              const float4 v = reinterpret_cast<const float4*>(xr)[c4];
              if (4 * c4 + 0 < NC) acc[4 * c4 + 0] = fma_t(b[u], v.x, acc[4 * c4 + 0]);
              if (4 * c4 + 1 < NC) acc[4 * c4 + 1] = fma_t(b[u], v.y, acc[4 * c4 + 1]);
              if (4 * c4 + 2 < NC) acc[4 * c4 + 2] = fma_t(b[u], v.z, acc[4 * c4 + 2]);
              if (4 * c4 + 3 < NC) acc[4 * c4 + 3] = fma_t(b[u], v.w, acc[4 * c4 + 3]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fma_t(b[u], xr[c], acc[c]);
          }
        }
      }
      // the rest of the chunk, without padding FMAs
      for (; kk0 < C.K; ++kk0) {
        const T bu = __ldg(a + (int64_t)kk0 * M);
        const T* xr = xg + kk0 * NCP;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma_t(bu, xr[c], acc[c]);
      }
    }
    __syncthreads();
  }
  // group partial sums through shared memory: red[g][c][rl]
  T* red = smem_rc;
  if (G > 1) {
    if (active)
#pragma unroll
      for (int c = 0; c < NC; ++c) red[(g * NC + c) * RW + rl] = acc[c];
    __syncthreads();
    if (g == 0 && active) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T v = red[c * RW + rl];
        for (int gg = 1; gg < G; ++gg) v += red[(gg * NC + c) * RW + rl];
        acc[c] = v;
      }
    }
  }
  if (g == 0 && active) {
    if (W.part < 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < ncl) {
          T* cp = P.C + r + (int64_t)(c0 + c) * P.ldc;
          *cp = P.beta ? *cp + acc[c] : acc[c];
        }
    } else {
      T* pt = partial + W.part * (NC * 256);
#pragma unroll
      for (int c = 0; c < NC; ++c) pt[c * 256 + rl] = acc[c];
    }
  }
}

template <class T, int NC>
__global__ void __launch_bounds__(256) k_coupling_rows_reduce(const RowCoupProbT<T>* __restrict__ probs,
                                                              const RowCoupRed* __restrict__ red,
                                                              const T* __restrict__ partial,
                                                              int c0) {
  const RowCoupRed R = red[blockIdx.x];
  const RowCoupProbT<T> P = probs[R.p];
  const int rl = threadIdx.x;
  if (rl >= min(P.M - R.r0, 256)) return;
  const int ncl = min(NC, P.ncol - c0);
  for (int c = 0; c < ncl; ++c) {
    T v = T(0);
    for (int q = 0; q < R.nparts; ++q) v += partial[(R.part0 + q) * (NC * 256) + c * 256 + rl];
    T* cp = P.C + R.r0 + rl + (int64_t)(c0 + c) * P.ldc;
    *cp = P.beta ? *cp + v : v;
  }
}

static int rowcoup_nc(int ncol) {
  return ncol <= 1 ? 1 : (ncol <= 2 ? 2 : (ncol <= 4 ? 4 : (ncol <= 8 ? 8 : 16)));
}

template <class T>
void RowCoupBatchT<T>::upload(cudaStream_t s) {
  work.clear();
  red.clear();
  flops = bytes = 0.0;
  int64_t nparts = 0, total = 0;
  for (const auto& P : probs)
    for (int g = P.ch0; g < P.ch1; ++g) total += (int64_t)P.M * chunks[g].K;
  const int64_t item0 = std::min(kRowItemMax, std::max(kRowItemMin, total / (152 * 16)));
  for (auto& P : probs)
    if (P.item == 0) P.item = item0;
  for (int p = 0; p < (int)probs.size(); ++p) {
    const RowCoupProbT<T>& P = probs[p];
    const int64_t item = P.item;
    int64_t kt = 0;
    for (int g = P.ch0; g < P.ch1; ++g) kt += chunks[g].K;
    flops += 2.0 * P.M * (double)kt * P.ncol;
    bytes += sizeof(T) * (double)P.M * (double)kt;
    for (int r0 = 0; r0 < P.M; r0 += 256) {
      const int rows = std::min(P.M - r0, 256);
      // cut the chunk range into parts of about `item` entries
      std::vector<std::pair<int, int>> parts;
      int start = P.ch0;
      int64_t acc = 0;
      for (int g = P.ch0; g < P.ch1; ++g) {
        acc += (int64_t)rows * chunks[g].K;
        if (acc >= item && g + 1 < P.ch1) {
          parts.emplace_back(start, g + 1);
          start = g + 1;
          acc = 0;
        }
      }
      parts.emplace_back(start, P.ch1);
      if (parts.size() == 1) {
        work.push_back(RowCoupWork{p, r0, parts[0].first, parts[0].second, -1});
      } else {
        red.push_back(RowCoupRed{p, r0, nparts, (int)parts.size()});
        for (auto& pr : parts) work.push_back(RowCoupWork{p, r0, pr.first, pr.second, nparts++});
      }
    }
  }
  // the largest items first, so that the long ones do not form the tail
  std::stable_sort(work.begin(), work.end(), [&](const RowCoupWork& x, const RowCoupWork& y) {
    auto sz = [&](const RowCoupWork& w) {
      int64_t k = 0;
      for (int g = w.ch0; g < w.ch1; ++g) k += chunks[g].K;
      return k * std::min(probs[w.p].M - w.r0, 256);
    };
    return sz(x) > sz(y);
  });
  d_probs.upload(probs, s);
  d_chunks.upload(chunks, s);
  d_work.upload(work, s);
  d_red.upload(red, s);
  partial.alloc(std::max<int64_t>(nparts, 1) * rowcoup_nc(ncol) * 256);
}

template <class T, int NC>
static void rowcoup_go(const RowCoupBatchT<T>& b, cudaStream_t s) {
  constexpr int NCP = rowcoup_ncp(NC);
  const size_t smem = (size_t)8 * kRowChunk * NCP * sizeof(T);
  // the reduction reuses the staging buffer: G * NC * RW <= 256 * NC entries
  static_assert(8 * kRowChunk * NCP >= 256 * NC, "reduction buffer");
  if (smem > 48 * 1024)
    SPD_CUDA(cudaFuncSetAttribute(k_coupling_rows<T, NC>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int c0 = 0; c0 < b.ncol; c0 += NC) {
    k_coupling_rows<T, NC><<<(unsigned)b.work.size(), 256, smem, s>>>(
        b.d_probs.p, b.d_chunks.p, b.d_work.p, b.partial.p, c0);
    SPD_LAUNCHED();
    if (!b.red.empty()) {
      k_coupling_rows_reduce<T, NC><<<(unsigned)b.red.size(), 256, 0, s>>>(
          b.d_probs.p, b.d_red.p, b.partial.p, c0);
      SPD_LAUNCHED();
    }
  }
}

// several instances' coupling steps (batched sweep): problems and chunks concatenated
template <class T>
struct DeferredRowCoup : Deferred {
  std::vector<RowCoupProbT<T>> probs;
  std::vector<RowCoupChunkT<T>> chunks;
  int ncol = 1;
  const char* tag = "h2_coupling";
  void launch_merged(const std::vector<Deferred*>& group, cudaStream_t s) override {
    RowCoupBatchT<T> m;
    m.tag = tag;
    for (Deferred* d : group) {
      const auto* x = static_cast<const DeferredRowCoup<T>*>(d);
      const int off = (int)m.chunks.size();
      m.chunks.insert(m.chunks.end(), x->chunks.begin(), x->chunks.end());
      for (RowCoupProbT<T> p : x->probs) {
        p.ch0 += off;
        p.ch1 += off;
        m.probs.push_back(p);
      }
      m.ncol = std::max(m.ncol, x->ncol);
    }
    m.upload(s);
    m.launch(s);
  }
};

template <class T>
void RowCoupBatchT<T>::launch(cudaStream_t s) const {
  if (merging()) {
    if (probs.empty()) { merge_skip(); return; }
    std::unique_ptr<DeferredRowCoup<T>> d(new DeferredRowCoup<T>());
    d->probs = probs;
    d->chunks = chunks;
    d->ncol = ncol;
    d->tag = tag;
    merge_ctx().m->submit(std::string(sizeof(T) == 8 ? "rowcoup_f64_" : "rowcoup_f32_") +
                              std::to_string(rowcoup_nc(ncol)), std::move(d));
    return;
  }
  if (work.empty()) return;
  ProfScope ps(tag, s, flops, bytes);
  switch (rowcoup_nc(ncol)) {
    case 1: rowcoup_go<T, 1>(*this, s); break;
    case 2: rowcoup_go<T, 2>(*this, s); break;
    case 4: rowcoup_go<T, 4>(*this, s); break;
    case 8: rowcoup_go<T, 8>(*this, s); break;
    default: rowcoup_go<T, 16>(*this, s); break;
  }
}

template struct RowCoupBatchT<double>;
template struct RowCoupBatchT<float>;

// Offsets of the destination-major coupling matrices (once per handle).
static void coup_dm_offsets(spdhss_h2_s* h) {
  if (!h->coup_dm_off.empty()) return;
  const TreeHost& T = h->th;
  const int64_t NN = T.nn();
  h->coup_dm_off.assign(NN + 1, 0);
  for (int64_t i = 0; i < NN; ++i) {
    int64_t kt = 0;
    if (h->rank(i) > 0)
      for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) kt += h->rank(T.far_idx[e]);
    h->coup_dm_off[i + 1] = h->coup_dm_off[i] + (int64_t)h->rank(i) * kt;
  }
}

// The destination-major copy of the couplings in type TD.
template <class TD>
static void coup_dm_build(spdhss_h2_s* h, DevBuf<TD>& out, cudaStream_t s) {
  const TreeHost& T = h->th;
  const int64_t NN = T.nn();
  coup_dm_offsets(h);
  out.alloc(std::max<int64_t>(h->coup_dm_off[NN], 1));
  std::vector<CopyDM<TD>> cps;
  int64_t maxe = 1;
  for (int64_t i = 0; i < NN; ++i) {
    const int ki = h->rank(i);
    if (ki == 0) continue;
    int64_t col = 0;
    for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
      const int64_t j = T.far_idx[e];
      const int kj = h->rank(j);
      if (kj == 0) continue;
      CopyDM<TD> c;
      c.src = h->coup.p + h->far_boff[e];
      c.trans = h->far_trans[e];
      c.lds = c.trans ? kj : ki;
      c.dst = out.p + h->coup_dm_off[i] + col * ki;
      c.ldd = ki;
      c.m = ki;
      c.n = kj;
      cps.push_back(c);
      maxe = std::max<int64_t>(maxe, (int64_t)ki * kj);
      col += kj;
    }
  }
  for (size_t b0 = 0; b0 < cps.size(); b0 += 65535) {
    std::vector<CopyDM<TD>> part(cps.begin() + b0, cps.begin() + std::min(cps.size(), b0 + 65535));
    DevBuf<CopyDM<TD>> dp;
    dp.upload(part, s);
    const int gx = (int)std::min<int64_t>(ceil_div(maxe, 256), 16);
    k_copy_dm<TD><<<dim3(gx, (unsigned)part.size()), 256, 0, s>>>(dp.p);
    SPD_LAUNCHED();
    SPD_CUDA(cudaStreamSynchronize(s));
  }
}

// The destination-major coupling step of plan p (one streaming problem per node).
template <class T>
static void rowcoup_plan(const spdhss_h2_s* h, H2PlanT<T>& p, int ncol, const T* A,
                         cudaStream_t s) {
  const TreeHost& T_ = h->th;
  const int64_t K = std::max<int64_t>(h->Ktot, 1);
  RowCoupBatchT<T>& rb = p.rowcoup;
  rb.ncol = ncol;
  rb.tag = sizeof(T) == 4 ? "h2_coupling_f32" : "h2_coupling";
  for (int64_t i = 0; i < T_.nn(); ++i) {
    const int ki = h->rank(i);
    if (ki == 0 || T_.far_off[i] == T_.far_off[i + 1]) continue;
    RowCoupProbT<T> pr;
    pr.C = p.yhat.p + h->skel_off[i];
    pr.ldc = K;
    pr.M = ki;
    pr.ncol = ncol;
    pr.A = A + h->coup_dm_off[i];
    pr.ch0 = (int)rb.chunks.size();
    int64_t col = 0;
    for (int64_t e = T_.far_off[i]; e < T_.far_off[i + 1]; ++e) {
      const int64_t j = T_.far_idx[e];
      const int kj = h->rank(j);
      for (int k0 = 0; k0 < kj; k0 += kRowChunk)
        rb.chunks.push_back(RowCoupChunkT<T>{p.xhat.p + h->skel_off[j] + k0, K, col + k0,
                                             std::min(kRowChunk, kj - k0)});
      col += kj;
    }
    pr.ch1 = (int)rb.chunks.size();
    rb.probs.push_back(pr);
  }
  rb.upload(s);
  p.use_rowcoup = true;
  p.coupling = GemmBatchT<T>();
}

void h2_plan_build(const spdhss_h2_s* h, H2Plan& p, int ncol, int nslot, cudaStream_t s) {
  // Few columns: the coupling step streams the destination-major FP64 copy (each entry read
  // once, coalesced, spread over many CTAs); the grouped GEMM would give every node one CTA
  // with a long serial loop over its partners.  The copy is made on first use and kept.
  // (each unordered pair twice: twice the bytes of the FP64 couplings; made only when it
  // fits beside everything else, else the grouped GEMM over the stored couplings)
  spdhss_h2_s* hm = const_cast<spdhss_h2_s*>(h);   // a cache of the handle
  if (nslot == 1 && ncol <= 4 &&
      (hm->coup_dd.n > 0 || fits_on_device(2 * h->coup.bytes(), s))) {
    if (hm->coup_dd.n == 0) coup_dm_build<double>(hm, hm->coup_dd, s);
    h2_plan_build_t<double>(h, p, ncol, nslot, h->basis.p, nullptr, s);
    rowcoup_plan<double>(h, p, ncol, h->coup_dd.p, s);
    return;
  }
  h2_plan_build_t<double>(h, p, ncol, nslot, h->basis.p, h->coup.p, s);
}

// The sampling product of the precision mode: an FP32 plan with LCA slots over FP32
// copies of the bases and (source-major) couplings, its GEMMs on the tensor cores
// (tc = 1: TF32, 2: 3xTF32), the near field evaluated in FP32 on the fly.
void h2_plan_sample_f(spdhss_h2_s* h, H2PlanF& p, int ncol, int nslot, int tc, cudaStream_t s) {
  if (h->basis_f.n == 0) {
    h->basis_f.alloc(std::max<size_t>(h->basis.n, 1));
    convert_d2f(h->basis.p, h->basis_f.p, (int64_t)h->basis.n, s);
  }
  // the source-major FP32 couplings live as long as the plan (half the FP64 couplings'
  // bytes; made again per build rather than kept beside the destination-major copy of the
  // FP32 products)
  p.coup_src.alloc(std::max<size_t>(h->coup.n, 1));
  if (h->coup.n) convert_d2f(h->coup.p, p.coup_src.p, (int64_t)h->coup.n, s);
  h2_plan_build_t<float>(h, p, ncol, nslot, h->basis_f.p, p.coup_src.p, s, tc);
}

H2PlanF& h2_plan_f(spdhss_h2_s* h, int ncol, cudaStream_t s) {
  // up to 16 columns: the once-read product over the padded FP32 layout (made on first use,
  // about half the bytes of the FP64 generators); else, or when the layout does not fit,
  // each plan converts the couplings once and runs the grouped GEMMs over them
  auto it = h->plans_f.find(ncol);
  if (it == h->plans_f.end()) {
    std::unique_ptr<H2PlanF> p(new H2PlanF());
    if (ncol <= 16 && sym_layout_fits(h, s)) {
      sym_layout(h, s);
      h2_plan_build_t<float>(h, *p, ncol, 1, nullptr, nullptr, s, 0, false);
      sym_plan_build(h, *p, ncol, s);
    } else {
      if (h->basis_f.n == 0) {
        h->basis_f.alloc(std::max<size_t>(h->basis.n, 1));
        convert_d2f(h->basis.p, h->basis_f.p, (int64_t)h->basis.n, s);
      }
      p->coup_src.alloc(std::max<size_t>(h->coup.n, 1));
      if (h->coup.n) convert_d2f(h->coup.p, p->coup_src.p, (int64_t)h->coup.n, s);
      h2_plan_build_t<float>(h, *p, ncol, 1, h->basis_f.p, p->coup_src.p, s);
    }
    it = h->plans_f.emplace(ncol, std::move(p)).first;
  }
  return *it->second;
}

template <class T>
static void h2_plan_run_t(const spdhss_h2_s* h, const H2PlanT<T>& p, cudaStream_t s) {
  if (p.sym) {
    sym_plan_run(*p.sym, s);
    p.near.launch(h->kfn, h->td.xs.p, h->th.n, h->th.dim, s);
    return;
  }
  p.up_leaf.launch(s);
  for (const auto& g : p.up) g.launch(s);
  if constexpr (std::is_same<T, double>::value) copy_vec(p.yhat.p, nullptr, (int64_t)p.yhat.n, s);
  else SPD_CUDA(cudaMemsetAsync(p.yhat.p, 0, p.yhat.bytes(), s));
  if (p.use_rowcoup) p.rowcoup.launch(s);
  else p.coupling.launch(s);
  for (const auto& g : p.down) g.launch(s);
  p.leaf_out.launch(s);
  if (p.near_rows) p.near_r.launch(s);
  else if (p.near_stored) p.near_g.launch(s);
  else p.near.launch(h->kfn, h->td.xs.p, h->th.n, h->th.dim, s);
}

void h2_plan_run(const spdhss_h2_s* h, const H2Plan& p, cudaStream_t s) { h2_plan_run_t(h, p, s); }
void h2_plan_run(const spdhss_h2_s* h, const H2PlanF& p, cudaStream_t s) { h2_plan_run_t(h, p, s); }

}  // namespace spd
