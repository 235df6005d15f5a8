// Symmetric ULV factorization of the SPD HSS matrix (reading of the ULV decomposition the
// paper applies, Sec. 1 and Sec. 6): per node, bottom-up,
//   W_i = Q_i [U~_i; 0]            (Householder QR of the basis: leaf U_i, above diag(U~_c) R_i)
//   Q_i^T D_i Q_i = [[D_pp, D_pq], [D_qp, D_qq]]
//   D_qq = L_q L_q^T,  X = L_q^{-1} D_qp,  D^_i = D_pp - X^T X
// where D_i is the leaf block A_ii + sigma I or, above, the children's reduced blocks D^_c
// coupled by U~_a B_ab U~_b^T; a dense Cholesky factorization closes the root.  The solve
// is the matching forward and backward sweep.
#include <algorithm>

#include "ulv.cuh"

namespace spd {

__global__ void k_triu(const double* const* __restrict__ src, const int64_t* __restrict__ lds,
                       double* const* __restrict__ dst, const int* __restrict__ rr, int nprob) {
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const int r = rr[p];
  const double* a = src[p];
  double* b = dst[p];
  const int64_t ld = lds[p];
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    b[i + (int64_t)j * r] = (i <= j) ? a[i + (int64_t)j * ld] : 0.0;
  }
}

void ulv_factor_impl(spdhss_ulv_s* u, const spdhss_hss_s* hs, cudaStream_t s) {
  // the allocation-free solve's arrays are loaded here, where allocating is allowed
  ulv_noalloc_prepare_device();
  const spdhss_h2_s* h2 = hs->h2;
  const TreeHost& T = h2->th;
  const int64_t n = T.n;
  const int D = T.D, L = D + 1;
  const int NN = (int)T.nn();
  u->hs = hs;
  u->L = L;
  u->D = D;
  u->m.assign(NN, 0);
  u->r.assign(NN, 0);
  for (int i = 0; i < NN; ++i) { u->m[i] = hs->mrow[i]; u->r[i] = hs->rk[i]; }
  DevBuf<int> info(2);
  if (D == 0) {
    u->mroot = (int)n;
    u->root.alloc((size_t)n * n);
    Batch<TileProb> tb;
    TileProb tp;
    tp.xr = h2->td.xs.p; tp.ldxr = n; tp.r0 = 0; tp.rows = (int)n;
    tp.xc = h2->td.xs.p; tp.ldxc = n; tp.c0 = 0; tp.cols = (int)n;
    tp.out = u->root.p; tp.ldo = n; tp.diag_add = h2->kfn.shift;
    tb.push(tp);
    tb.upload(s);
    tile_launch(tb, h2->kfn, T.dim, s);
    Batch<PotrfProb> pb;
    pb.push(PotrfProb{u->root.p, n, (int)n, 0});
    pb.upload(s);
    info.zero(s);
    potrf_launch(pb, info.p, s);
    std::vector<int> hi = info.download(s);
    if (hi[0]) throw Error(SPDHSS_NOT_SPD, "ulv_factor: the dense block is not positive definite");
    return;
  }
  // storage
  u->Doff.assign(NN, 0);
  u->Woff.assign(NN, 0);
  u->toff.assign(NN, 0);
  u->Uoff.assign(NN, 0);
  int64_t dt = 0, wt = 0, tt = 0, ut = 0;
  for (int i = 0; i < NN; ++i) {
    if (T.depth_of(i) == 0) continue;
    const int64_t m = u->m[i], r = u->r[i];
    u->Doff[i] = dt; dt += m * m;
    u->Woff[i] = wt; wt += m * r;
    u->toff[i] = tt; tt += std::max<int64_t>(r, 1);
    u->Uoff[i] = ut; ut += r * r;
  }
  u->Dbuf.alloc(std::max<int64_t>(dt, 1));
  u->Wbuf.alloc(std::max<int64_t>(wt, 1));
  u->taub.alloc(std::max<int64_t>(tt, 1));
  u->Ubuf.alloc(std::max<int64_t>(ut, 1));
  u->rdev.upload(u->r, s);
  auto Dp = [&](int64_t i) { return u->Dbuf.p + u->Doff[i]; };
  auto Wp = [&](int64_t i) { return u->Wbuf.p + u->Woff[i]; };
  auto Up = [&](int64_t i) { return u->Ubuf.p + u->Uoff[i]; };

  for (int k = 1; k <= L - 1; ++k) {
    merge_stage(6, k);
    const int t = D + 1 - k;
    const int64_t o = T.depth_off[t], nn = T.depth_off[t + 1] - o;
    // (1) D_i and W_i
    {
      Batch<TileProb> tb;
      Batch<CopyProb> cb;
      GemmBatch gw, g1, g2;
      struct Off { int64_t a, b, e; double* dst; int64_t ld; };
      std::vector<Off> offs;
      int64_t tmpn = 0;
      for (int64_t i = o; i < o + nn; ++i) {
        const int m = u->m[i], r = u->r[i];
        if (m == 0) continue;
        if (k == 1) {
          TileProb tp;
          tp.xr = h2->td.xs.p; tp.ldxr = n; tp.r0 = T.begin[i]; tp.rows = m;
          tp.xc = h2->td.xs.p; tp.ldxc = n; tp.c0 = T.begin[i]; tp.cols = m;
          tp.out = Dp(i); tp.ldo = m; tp.diag_add = h2->kfn.shift;
          tb.push(tp);
          if (r > 0) {
            CopyProb cp{};
            cp.src = hs->gen.p + hs->gen_off[i]; cp.lds = m; cp.dst = Wp(i); cp.ldd = m;
            cp.m = m; cp.n = r; cp.alpha = 1.0;
            cb.push(cp);
          }
        } else {
          int64_t ra = 0;
          for (int64_t a = T.child_begin[i]; a < T.child_end[i]; ++a) {
            const int rA = u->r[a];
            if (rA > 0) {
              CopyProb cp{};
              cp.src = Dp(a); cp.lds = u->m[a]; cp.dst = Dp(i) + ra + ra * m; cp.ldd = m;
              cp.m = rA; cp.n = rA; cp.alpha = 1.0;
              cb.push(cp);
              if (r > 0)
                gw.add(Wp(i) + ra, m, rA, r, Up(a), rA, 0,
                       hs->gen.p + hs->gen_off[i] + ra, m, 0, rA, 1.0, 0.0);
            }
            int64_t rb = 0;
            for (int64_t b = T.child_begin[i]; b < T.child_end[i]; ++b) {
              const int rB = u->r[b];
              if (a != b && rA > 0 && rB > 0) {
                int64_t e = -1;
                for (int64_t q = hs->sib_off[a]; q < hs->sib_off[a + 1]; ++q)
                  if (hs->sib_node[q] == b) { e = q; break; }
                SPD_REQUIRE(e >= 0, "ulv_factor: missing sibling coupling");
                offs.push_back(Off{a, b, e, Dp(i) + ra + rb * m, m});
                tmpn += (int64_t)rA * rB;
              }
              rb += rB;
            }
            ra += rA;
          }
        }
      }
      DevBuf<double> tmp(std::max<int64_t>(tmpn, 1));
      int64_t to = 0;
      for (const Off& f : offs) {
        const int rA = u->r[f.a], rB = u->r[f.b];
        // tmp = B_ab U~_b^T ; block = U~_a tmp
        g1.add(tmp.p + to, rA, rA, rB, hs->sib.p + hs->sib_boff[f.e], rA, 0, Up(f.b), rB, 1, rB,
               1.0, 0.0);
        g2.add(f.dst, f.ld, rA, rB, Up(f.a), rA, 0, tmp.p + to, rA, 0, rA, 1.0, 0.0);
        to += (int64_t)rA * rB;
      }
      tb.upload(s);
      tile_launch(tb, h2->kfn, T.dim, s);
      cb.upload(s);
      copy_launch(cb, s);
      gw.run(s);
      g1.run(s);
      g2.run(s);
    }
    // (2) QR of W_i, U~_i
    {
      Batch<QrProb> qb;
      int maxm = 1;
      for (int64_t i = o; i < o + nn; ++i) {
        const int m = u->m[i], r = u->r[i];
        if (m == 0 || r == 0) continue;
        maxm = std::max(maxm, m);
        QrProb q{};
        q.A = Wp(i); q.lda = m; q.m = m; q.n = r; q.kmax = r; q.rtol = 0.0;
        q.piv = nullptr; q.tau = u->taub.p + u->toff[i]; q.rank = u->rdev.p + i; q.norms = nullptr;
        qb.push(q);
      }
      qb.upload(s);
      const int pslot = geqp3_launch(qb, 0, 1, maxm, s);
      if (pslot >= 0) {
        double f = 0.0;
        for (const auto& q : qb.h) f += qr_flops(q.m, q.n, q.kmax, false);
        prof_add_flops(pslot, f);
      }
      std::vector<const double*> src;
      std::vector<double*> dst;
      std::vector<int64_t> lds;
      std::vector<int> rr;
      for (int64_t i = o; i < o + nn; ++i)
        if (u->m[i] > 0 && u->r[i] > 0) {
          src.push_back(Wp(i)); dst.push_back(Up(i)); lds.push_back(u->m[i]); rr.push_back(u->r[i]);
        }
      if (!src.empty()) {
        DevBuf<const double*> ds; DevBuf<double*> dd; DevBuf<int64_t> dl; DevBuf<int> dr;
        ds.upload(src, s); dd.upload(dst, s); dl.upload(lds, s); dr.upload(rr, s);
        k_triu<<<(unsigned)src.size(), 256, 0, s>>>(ds.p, dl.p, dd.p, dr.p, (int)src.size());
        SPD_LAUNCHED();
      }
    }
    // (3) Q^T D Q
    {
      std::vector<int64_t> sz;
      int64_t tot = 0;
      for (int64_t i = o; i < o + nn; ++i) { sz.push_back(tot); tot += (int64_t)u->m[i] * u->m[i]; }
      DevBuf<double> Dt(std::max<int64_t>(tot, 1));
      Batch<HhApplyProb> h1, h2b;
      Batch<CopyProb> tr, back;
      for (int64_t i = o; i < o + nn; ++i) {
        const int m = u->m[i], r = u->r[i];
        if (m == 0 || r == 0) continue;
        HhApplyProb hp;
        hp.V = Wp(i); hp.ldv = m; hp.tau = u->taub.p + u->toff[i]; hp.k = u->rdev.p + i;
        hp.B = Dp(i); hp.ldb = m; hp.m = m; hp.ncol = m;
        h1.push(hp);
        hp.B = Dt.p + sz[i - o];
        h2b.push(hp);
        CopyProb cp{};
        cp.src = Dp(i); cp.lds = m; cp.dst = Dt.p + sz[i - o]; cp.ldd = m; cp.m = m; cp.n = m;
        cp.trans = 1; cp.alpha = 1.0;
        tr.push(cp);
        cp.src = Dt.p + sz[i - o]; cp.dst = Dp(i); cp.trans = 0;
        back.push(cp);
      }
      h1.tag = h2b.tag = "hh_ulv_factor";
      h1.upload(s); householder_launch(h1, 1, s);
      tr.upload(s); copy_launch(tr, s);
      h2b.upload(s); householder_launch(h2b, 1, s);
      back.upload(s); copy_launch(back, s);
    }
    // (4) eliminate the complement
    {
      Batch<PotrfProb> pb;
      Batch<TrsmProb> tb;
      GemmBatch gb;
      for (int64_t i = o; i < o + nn; ++i) {
        const int m = u->m[i], r = u->r[i];
        if (m - r <= 0) continue;
        double* Di = Dp(i);
        pb.push(PotrfProb{Di + r + (int64_t)r * m, m, m - r, (int)(i - o)});
        if (r > 0) {
          TrsmProb tp;
          tp.T = Di + r + (int64_t)r * m; tp.ldt = m; tp.B = Di + r; tp.ldb = m;
          tp.n = m - r; tp.ncol = r; tp.lower = 1; tp.trans = 0;
          tb.push(tp);
          gb.add(Di, m, r, r, Di + r, m, 1, Di + r, m, 0, m - r, -1.0, 1.0);
        }
      }
      info.zero(s);
      pb.tag = "potrf_ulv";
      tb.tag = "trsm_ulv_factor";
      gb.tag = "gemm_ulv_factor";
      pb.upload(s);
      potrf_launch(pb, info.p, s);
      std::vector<int> hi = info.download(s);
      if (hi[0]) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "ulv_factor: Cholesky failed at node %lld",
                      (long long)(o + hi[0] - 1));
        throw Error(SPDHSS_NOT_SPD, buf);
      }
      tb.upload(s);
      trsm_launch(tb, s);
      gb.run(s);
    }
  }
  // root block from the level L-1 reduced blocks
  merge_stage(7, 0);
  {
    int mr = 0;
    for (int64_t c = T.child_begin[0]; c < T.child_end[0]; ++c) mr += u->r[c];
    u->mroot = mr;
    u->root.alloc((size_t)std::max(mr, 1) * std::max(mr, 1));
    Batch<CopyProb> cb;
    GemmBatch g1, g2;
    int64_t tmpn = 0;
    for (int64_t a = T.child_begin[0]; a < T.child_end[0]; ++a)
      for (int64_t b = T.child_begin[0]; b < T.child_end[0]; ++b)
        if (a != b) tmpn += (int64_t)u->r[a] * u->r[b];
    DevBuf<double> tmp(std::max<int64_t>(tmpn, 1));
    int64_t ra = 0, to = 0;
    for (int64_t a = T.child_begin[0]; a < T.child_end[0]; ++a) {
      const int rA = u->r[a];
      if (rA > 0) {
        CopyProb cp{};
        cp.src = Dp(a); cp.lds = u->m[a]; cp.dst = u->root.p + ra + ra * (int64_t)mr; cp.ldd = mr;
        cp.m = rA; cp.n = rA; cp.alpha = 1.0;
        cb.push(cp);
      }
      int64_t rb = 0;
      for (int64_t b = T.child_begin[0]; b < T.child_end[0]; ++b) {
        const int rB = u->r[b];
        if (a != b && rA > 0 && rB > 0) {
          int64_t e = -1;
          for (int64_t q = hs->sib_off[a]; q < hs->sib_off[a + 1]; ++q)
            if (hs->sib_node[q] == b) { e = q; break; }
          SPD_REQUIRE(e >= 0, "ulv_factor: missing root sibling coupling");
          g1.add(tmp.p + to, rA, rA, rB, hs->sib.p + hs->sib_boff[e], rA, 0, Up(b), rB, 1, rB,
                 1.0, 0.0);
          g2.add(u->root.p + ra + rb * (int64_t)mr, mr, rA, rB, Up(a), rA, 0, tmp.p + to, rA, 0,
                 rA, 1.0, 0.0);
          to += (int64_t)rA * rB;
        }
        rb += rB;
      }
      ra += rA;
    }
    cb.upload(s);
    copy_launch(cb, s);
    g1.run(s);
    g2.run(s);
    if (mr > 0) {
      Batch<PotrfProb> pb;
      pb.push(PotrfProb{u->root.p, mr, mr, 0});
      pb.upload(s);
      info.zero(s);
      potrf_launch(pb, info.p, s);
      std::vector<int> hi = info.download(s);
      if (hi[0]) throw Error(SPDHSS_NOT_SPD, "ulv_factor: Cholesky failed at the root");
    }
    SPD_CUDA(cudaStreamSynchronize(s));
  }
}

// F_i and B_i for every node and the root's explicit triangular inverses: the forward and
// backward steps of the solve applied to identity matrices, with the batched kernels of the
// factorization (the same operations as a solve, with m_i columns).
static void ulv_explicit(spdhss_ulv_s* u, cudaStream_t s) {
  if (!u->Foff.empty()) return;
  const TreeHost& T = u->hs->h2->th;
  const int64_t NN = T.nn();
  u->Foff.assign(NN + 1, 0);
  for (int64_t i = 0; i < NN; ++i) {
    const int64_t m = (T.depth_of(i) == 0) ? 0 : u->m[i];
    u->Foff[i + 1] = u->Foff[i] + m * m;
  }
  u->Fbuf.alloc(std::max<int64_t>(u->Foff[NN], 1));
  u->Bbuf.alloc(std::max<int64_t>(u->Foff[NN], 1));
  Batch<CopyProb> id;
  Batch<HhApplyProb> qt, q;
  Batch<TrsmProb> fw, bk;
  GemmBatch uf, ub;
  for (int64_t i = 0; i < NN; ++i) {
    const int m = (T.depth_of(i) == 0) ? 0 : u->m[i];
    if (m == 0) continue;
    const int r = u->r[i];
    double* F = u->Fbuf.p + u->Foff[i];
    double* B = u->Bbuf.p + u->Foff[i];
    double* Di = u->Dbuf.p + u->Doff[i];
    for (double* X : {F, B}) {
      CopyProb c{};
      c.src = nullptr; c.lds = m; c.dst = X; c.ldd = m; c.m = m; c.n = m; c.alpha = 1.0;
      id.push(c);
    }
    if (r > 0) {
      HhApplyProb hp;
      hp.V = u->Wbuf.p + u->Woff[i]; hp.ldv = m; hp.tau = u->taub.p + u->toff[i];
      hp.k = u->rdev.p + i; hp.m = m; hp.ncol = m;
      hp.B = F; hp.ldb = m;
      qt.push(hp);
      hp.B = B;
      q.push(hp);
    }
    if (m - r > 0) {
      fw.push(TrsmProb{Di + r + (int64_t)r * m, m, F + r, m, m - r, m, 1, 0});
      bk.push(TrsmProb{Di + r + (int64_t)r * m, m, B + r, m, m - r, m, 1, 1});
      if (r > 0) {
        uf.add(F, m, r, m, Di + r, m, 1, F + r, m, 0, m - r, -1.0, 1.0);
        ub.add(B + r, m, m - r, m, Di + r, m, 0, B, m, 0, r, -1.0, 1.0);
      }
    }
  }
  id.upload(s);
  identity_launch(id, s);
  // forward: Q^T, complement solve, kept rows
  qt.tag = q.tag = "hh_ulv_explicit";
  qt.upload(s);
  householder_launch(qt, 1, s);
  fw.tag = bk.tag = "trsm_ulv_explicit";
  fw.upload(s);
  trsm_launch(fw, s);
  uf.tag = ub.tag = "gemm_ulv_explicit";
  uf.run(s);
  // backward: kept rows into the complement, transposed complement solve, Q
  ub.run(s);
  bk.upload(s);
  trsm_launch(bk, s);
  q.upload(s);
  householder_launch(q, 0, s);
  // root: L^{-1} and L^{-T}
  const int mr = u->mroot;
  if (mr > 0) {
    u->rootF.alloc((size_t)mr * mr);
    u->rootB.alloc((size_t)mr * mr);
    Batch<CopyProb> ir;
    for (double* X : {u->rootF.p, u->rootB.p}) {
      CopyProb c{};
      c.src = nullptr; c.lds = mr; c.dst = X; c.ldd = mr; c.m = mr; c.n = mr; c.alpha = 1.0;
      ir.push(c);
    }
    ir.upload(s);
    identity_launch(ir, s);
    Batch<TrsmProb> rt;
    rt.push(TrsmProb{u->root.p, mr, u->rootF.p, mr, mr, mr, 1, 0});
    rt.push(TrsmProb{u->root.p, mr, u->rootB.p, mr, mr, mr, 1, 1});
    rt.tag = "trsm_ulv_explicit";
    rt.upload(s);
    trsm_launch(rt, s);
  }
  SPD_CUDA(cudaStreamSynchronize(s));
}

UlvPlan& ulv_plan(spdhss_ulv_s* u, int ncol, cudaStream_t s) {
  auto it = u->plans.find(ncol);
  if (it != u->plans.end()) return *it->second;
  ulv_explicit(u, s);
  std::unique_ptr<UlvPlan> pp(new UlvPlan());
  UlvPlan& P = *pp;
  const TreeHost& T = u->hs->h2->th;
  const int64_t n = T.n;
  const int L = u->L, D = u->D;
  P.ncol = ncol;
  const int nlev = std::max(L - 1, 0);
  P.bw.resize(nlev + 1);
  P.tw.resize(nlev + 1);
  P.ldk.assign(nlev + 1, 0);
  P.fwd.resize(nlev); P.bwd.resize(nlev); P.up.resize(nlev); P.down.resize(nlev);
  // per-level row offsets of every node block
  std::vector<int64_t> moff(T.nn(), 0);
  if (D > 0) {
    for (int k = 1; k <= L - 1; ++k) {
      const int t = D + 1 - k;
      const int64_t o = T.depth_off[t], nn = T.depth_off[t + 1] - o;
      int64_t tot = 0;
      for (int64_t i = o; i < o + nn; ++i) {
        moff[i] = (k == 1) ? T.begin[i] : tot;
        tot += u->m[i];
      }
      if (k == 1) tot = n;
      P.ldk[k - 1] = std::max<int64_t>(tot, 1);
      P.bw[k - 1].alloc((size_t)P.ldk[k - 1] * ncol);
      P.tw[k - 1].alloc((size_t)P.ldk[k - 1] * ncol);
    }
  }
  P.ldk[nlev] = (D == 0) ? n : std::max(u->mroot, 1);
  P.bw[nlev].alloc((size_t)P.ldk[nlev] * ncol);
  P.tw[nlev].alloc((size_t)P.ldk[nlev] * ncol);
  for (int k = 1; k <= L - 1 && D > 0; ++k) {
    const int t = D + 1 - k;
    const int64_t o = T.depth_off[t], nn = T.depth_off[t + 1] - o;
    const int64_t ld = P.ldk[k - 1];
    const int64_t ldn = P.ldk[k];
    double* bn = P.bw[k].p;
    for (int64_t i = o; i < o + nn; ++i) {
      const int m = u->m[i], r = u->r[i];
      if (m == 0) continue;
      double* blk = P.bw[k - 1].p + moff[i];
      double* tb = P.tw[k - 1].p + moff[i];
      P.fwd[k - 1].add(tb, ld, m, ncol, u->Fbuf.p + u->Foff[i], m, 0, blk, ld, 0, m, 1.0, 0.0);
      P.bwd[k - 1].add(blk, ld, m, ncol, u->Bbuf.p + u->Foff[i], m, 0, tb, ld, 0, m, 1.0, 0.0);
      // position of i's kept rows inside its parent's block (or the root block)
      if (r > 0) {
        const int64_t par = T.parent[i];
        int64_t pos = 0;
        for (int64_t c = T.child_begin[par]; c < i; ++c) pos += u->r[c];
        const int64_t pbase = (k == L - 1) ? 0 : moff[par];
        CopyProb cu{};
        cu.src = tb; cu.lds = ld; cu.dst = bn + pbase + pos; cu.ldd = ldn; cu.m = r; cu.n = ncol;
        cu.alpha = 1.0;
        P.up[k - 1].push(cu);
        CopyProb cd{};
        cd.src = bn + pbase + pos; cd.lds = ldn; cd.dst = tb; cd.ldd = ld; cd.m = r; cd.n = ncol;
        cd.alpha = 1.0;
        P.down[k - 1].push(cd);
      }
    }
  }
  const int mr = (D == 0) ? (int)n : u->mroot;
  if (mr > 0) {
    const int64_t ldr = P.ldk[nlev];
    P.root_f.add(P.tw[nlev].p, ldr, mr, ncol, u->rootF.p, mr, 0, P.bw[nlev].p, ldr, 0, mr, 1.0, 0.0);
    P.root_b.add(P.bw[nlev].p, ldr, mr, ncol, u->rootB.p, mr, 0, P.tw[nlev].p, ldr, 0, mr, 1.0, 0.0);
  }
  for (int k = 0; k < nlev; ++k) {
    P.fwd[k].tag = P.bwd[k].tag = "gemm_ulv_solve";
    P.up[k].tag = P.down[k].tag = "copy_ulv_solve";
    P.fwd[k].upload(s);
    P.bwd[k].upload(s);
    P.up[k].upload(s);
    P.down[k].upload(s);
  }
  P.root_f.tag = P.root_b.tag = "gemm_ulv_root";
  P.root_f.upload(s);
  P.root_b.upload(s);
  it = u->plans.emplace(ncol, std::move(pp)).first;
  return *it->second;
}

void ulv_solve_sorted(const spdhss_ulv_s* u, const UlvPlan& P, cudaStream_t s) {
  const int nlev = std::max(u->L - 1, 0);
  for (int k = 0; k < nlev; ++k) {
    P.fwd[k].launch(s);
    copy_launch(P.up[k], s);
  }
  P.root_f.launch(s);
  P.root_b.launch(s);
  for (int k = nlev - 1; k >= 0; --k) {
    copy_launch(P.down[k], s);
    P.bwd[k].launch(s);
  }
}

}  // namespace spd
