// Accelerated SPD HSS construction (Alg. 5.3) on the device.
//
//  Y^(k) = (A - blkdiag_k A) Omega for all k (Eq. Yk) from ONE H^2 pass: every block is
//  routed to the HSS level of its lowest common ancestor, Y^(k) = sum over levels > k.
//  Leaf level: A_ii = S_i S_i^T; S_i^{-1} Y_i; pivoted QR -> V_i; T_i = V_i^T S_i^{-1} Y_i^(k)
//  (Alg. 5.2); G_i = S_i^{-T} V_i so that Phi_i = G_i^T; Phi U^H2; Type-1 B_ij = G_i^T A_ij G_j
//  (A_ij on the fly); Type-3 B_ij = (Phi U^H2)_i B^H2_ij (Phi U^H2)_j^T; U_i = S_i V_i.
//  Level k >= 2: I + bold B_ii = L_i L_i^T (Cholesky in place of the symmetric square root
//  of Eq. Si0); Lambda_i = L_i^{-1} [T_children]; pivoted QR -> Vbar_i; T pushed up; Gbar_i =
//  L_i^{-T} Vbar_i; Phi U^H2 by its recursion; Type-1 B_ij = Gbar_i^T bold B_ij Gbar_j
//  (Eq. Mijk); Type-3 as above; R_i = L_i Vbar_i (Eq. Rik).
//  Type-2 pairs are never formed (Sec. 5.2.2): every needed pair is a near or far pair.
#include <algorithm>
#include <cstring>

#include "spdhss.cuh"

namespace spd {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t* c, const uint32_t* k) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0], n1 = lo1, n2 = hi0 ^ c[3] ^ k[1], n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

__global__ void k_philox_normal(double* out, int64_t n, int ncol, int64_t ld, uint64_t seed) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * ncol) return;
  const int64_t i = e % n, j = e / n;
  uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)j, 0u};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
  const uint64_t a = ((uint64_t)c[0] << 21) ^ (uint64_t)c[1];
  const uint64_t b = ((uint64_t)c[2] << 21) ^ (uint64_t)c[3];
  const double u1 = ((double)(a & ((1ULL << 53) - 1)) + 1.0) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(b & ((1ULL << 53) - 1)) * (1.0 / 9007199254740992.0);
  out[i + j * ld] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

void philox_normal(double* out, int64_t n, int ncol, int64_t ld, uint64_t seed, cudaStream_t s) {
  k_philox_normal<<<ceil_div(n * ncol, 256), 256, 0, s>>>(out, n, ncol, ld, seed);
  SPD_LAUNCHED();
}

// Y^(k) = sum of the slots of levels > k: in-place suffix sum over the slots
__global__ void k_suffix_slots(double* z, int64_t slot_elems, int nslot) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= slot_elems) return;
  double acc = 0.0;
  for (int sl = nslot - 1; sl >= 0; --sl) {
    acc += z[(int64_t)sl * slot_elems + e];
    z[(int64_t)sl * slot_elems + e] = acc;
  }
}

namespace {

struct PairRef {
  const double* p = nullptr;   // stored block (owner orientation)
  int trans = 0;               // 1: the pair uses the transpose of the stored block
  int ld = 0;                  // leading dimension of the stored block
};

// offsets of an n-vector of sizes
std::vector<int64_t> prefix(const std::vector<int64_t>& v) {
  std::vector<int64_t> o(v.size() + 1, 0);
  for (size_t a = 0; a < v.size(); ++a) o[a + 1] = o[a] + v[a];
  return o;
}

int64_t find_entry(const std::vector<int64_t>& off, const std::vector<int64_t>& idx, int64_t i,
                   int64_t j) {
  const auto b0 = idx.begin() + off[i], b1 = idx.begin() + off[i + 1];
  const auto it = std::lower_bound(b0, b1, j);
  if (it != b1 && *it == j) return it - idx.begin();
  return -1;
}

void check_info(DevBuf<int>& info, const char* what, int64_t base, cudaStream_t s) {
  std::vector<int> h = info.download(s);
  if (h[0] != 0) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: Cholesky failed at node %lld (column %d)", what,
                  (long long)(base + h[0] - 1), h[1]);
    throw Error(SPDHSS_NOT_SPD, buf);
  }
}

}  // namespace

void spdhss_build_impl(spdhss_hss_s* hs, const spdhss_h2_s* h2, int r, int p,
                       const double* omega, uint64_t seed, cudaStream_t s, double rtol,
                       int precision) {
  const TreeHost& T = h2->th;
  const int64_t n = T.n;
  const int D = T.D;
  const int dim = T.dim;
  const int NN = (int)T.nn();
  const int sc = r + p;   // sketch columns s
  hs->h2 = h2;
  hs->r = r;
  hs->p = p;
  hs->s = sc;
  hs->L = D + 1;
  const int L = D + 1;
  hs->rk.assign(NN, 0);
  hs->mrow.assign(NN, 0);
  std::vector<int>& rk = hs->rk;
  std::vector<int>& mrow = hs->mrow;
  const double* xs = h2->td.xs.p;

  if (D == 0) {   // a single leaf: the HSS matrix is the dense matrix itself
    mrow[0] = (int)n;
    hs->hoff.assign(NN + 1, 0);
    hs->gen_off.assign(NN, 0);
    hs->sib_off.assign(NN + 1, 0);
    return;
  }

  // ---- sampling: Y^(k), k = 1 .. L-1, in sorted order: ys column block (k-1)*s ----------
  merge_stage(3, 0);
  const int nslot = L - 1;
  H2Plan plan;
  DevBuf<double> Ymixed;
  double* Y = nullptr;            // n x (s * (L-1)), ld n
  if (precision == 0) {
    h2_plan_build(h2, plan, sc, nslot, s);
    if (omega) permute_to_sorted(omega, n, plan.xs.p, n, sc, h2->td.perm.p, s);
    else {
      DevBuf<double> om((size_t)n * sc);
      philox_normal(om.p, n, sc, n, seed, s);
      permute_to_sorted(om.p, n, plan.xs.p, n, sc, h2->td.perm.p, s);
    }
    h2_plan_run(h2, plan, s);
    Y = plan.ys.p;
  } else {
    // precision mode: the sampling product in FP32 (FP32 generators and kernel entries,
    // basis and coupling GEMMs on the tensor cores, FP32 accumulation), then FP64 again
    spdhss_h2_s* hm = const_cast<spdhss_h2_s*>(h2);   // FP32 copies: a cache of the handle
    H2PlanF fp;
    h2_plan_sample_f(hm, fp, sc, nslot, precision == 2 ? 1 : 2, s);
    DevBuf<double> om((size_t)n * sc);
    if (omega) permute_to_sorted(omega, n, om.p, n, sc, h2->td.perm.p, s);
    else {
      DevBuf<double> o2((size_t)n * sc);
      philox_normal(o2.p, n, sc, n, seed, s);
      permute_to_sorted(o2.p, n, om.p, n, sc, h2->td.perm.p, s);
    }
    convert_d2f(om.p, fp.xs.p, n * sc, s);
    h2_plan_run(h2, fp, s);
    Ymixed.alloc((size_t)n * sc * nslot);
    convert_f2d(fp.ys.p, Ymixed.p, n * sc * nslot, s);
    tc_check(s);
    Y = Ymixed.p;
  }
  k_suffix_slots<<<ceil_div(n * sc, 256), 256, 0, s>>>(Y, n * sc, nslot);
  SPD_LAUNCHED();
  const int64_t ycols = (int64_t)sc * nslot;

  DevBuf<int> info(2);
  // per-level persistent pieces
  std::vector<std::unique_ptr<DevBuf<double>>> genpool(NN);   // U_i / R_i per level batches
  std::vector<double*> genp(NN, nullptr);
  // level-to-level state
  DevBuf<double> Tprev, PhiUprev, Bprev;
  std::vector<int64_t> troff_prev;            // row offsets in Tprev by local node index
  std::vector<int64_t> phiu_off_prev;         // offsets of PhiU in PhiUprev by local index
  std::vector<PairRef> nearB_prev(T.near_idx.size()), farB_prev(T.far_idx.size());
  // sibling blocks kept for the final HSS: (node a, partner b) -> host copy of location
  struct SibSrc { int64_t a, b; PairRef ref; };
  std::vector<SibSrc> sib_src;
  std::vector<std::unique_ptr<DevBuf<double>>> keep_pools;   // pools holding sibling blocks
  const double* UH = h2->basis.p;

  for (int k = 1; k <= L - 1; ++k) {
    merge_stage(4, k);
    const int t = D + 1 - k;
    const int64_t o = T.depth_off[t], nn = T.depth_off[t + 1] - o;
    const bool leaf = (k == 1);
    // rows of every node's local problem
    for (int64_t a = 0; a < nn; ++a) {
      const int64_t i = o + a;
      if (leaf) mrow[i] = (int)T.size(i);
      else {
        int m = 0;
        for (int64_t c = T.child_begin[i]; c < T.child_end[i]; ++c) m += rk[c];
        mrow[i] = m;
      }
    }
    std::vector<int64_t> msz(nn), mm(nn), qsz(nn), wsz(nn);
    for (int64_t a = 0; a < nn; ++a) {
      const int64_t m = mrow[o + a];
      msz[a] = m;
      mm[a] = m * m;
      qsz[a] = m * sc;
      wsz[a] = m * (int64_t)sc * (L - k);
    }
    const std::vector<int64_t> mmo = prefix(mm), qo = prefix(qsz), wo = prefix(wsz), mo = prefix(msz);
    DevBuf<double> F(std::max<int64_t>(mmo[nn], 1));      // S_i or L_i
    DevBuf<double> W(std::max<int64_t>(wo[nn], 1));       // nonleaf: Lambda_i, all pending slots
    DevBuf<double> Q(std::max<int64_t>(qo[nn], 1));       // QR workspace (m x s)
    DevBuf<double> tau(std::max<int64_t>(mo[nn], 1)), norms(std::max<int64_t>(2 * nn * sc, 1));
    DevBuf<int> piv(std::max<int64_t>(nn * sc, 1)), rkd(std::max<int64_t>(nn, 1));

    // (a) factor the diagonal blocks
    {
      Batch<TileProb> tb;
      Batch<CopyProb> ib, cb;
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        const int m = mrow[i];
        if (m == 0) continue;
        double* Fi = F.p + mmo[a];
        if (leaf) {
          TileProb tp;
          tp.xr = xs; tp.ldxr = n; tp.r0 = T.begin[i]; tp.rows = m;
          tp.xc = xs; tp.ldxc = n; tp.c0 = T.begin[i]; tp.cols = m;
          tp.out = Fi; tp.ldo = m; tp.diag_add = h2->kfn.shift;
          tb.push(tp);
        } else {
          CopyProb id{};
          id.dst = Fi; id.ldd = m; id.m = m; id.n = m;
          ib.push(id);
          // off-diagonal blocks B_{c_a c_b} from the previous level
          int64_t ra = 0;
          for (int64_t ca = T.child_begin[i]; ca < T.child_end[i]; ++ca) {
            int64_t rb = 0;
            for (int64_t cbn = T.child_begin[i]; cbn < T.child_end[i]; ++cbn) {
              if (ca != cbn && rk[ca] > 0 && rk[cbn] > 0) {
                int64_t e = find_entry(T.near_off, T.near_idx, ca, cbn);
                PairRef ref;
                if (e >= 0) ref = nearB_prev[e];
                else {
                  e = find_entry(T.far_off, T.far_idx, ca, cbn);
                  SPD_REQUIRE(e >= 0, "spdhss_build: sibling pair missing from the lists");
                  ref = farB_prev[e];
                }
                CopyProb cp{};
                cp.src = ref.p; cp.lds = ref.ld; cp.trans = ref.trans;
                cp.dst = Fi + ra + rb * m; cp.ldd = m;
                cp.m = rk[ca]; cp.n = rk[cbn]; cp.accumulate = 0; cp.alpha = 1.0;
                cb.push(cp);
              }
              rb += rk[cbn];
            }
            ra += rk[ca];
          }
        }
      }
      if (leaf) { tb.upload(s); tile_launch(tb, h2->kfn, dim, s); }
      else {
        ib.upload(s); identity_launch(ib, s);
        cb.upload(s); copy_launch(cb, s);
      }
      Batch<PotrfProb> pb;
      for (int64_t a = 0; a < nn; ++a)
        if (mrow[o + a] > 0) pb.push(PotrfProb{F.p + mmo[a], mrow[o + a], mrow[o + a], (int)a});
      info.zero(s);
      pb.tag = "potrf_hss";
      pb.upload(s);
      potrf_launch(pb, info.p, s);
      check_info(info, "spdhss_build", o, s);
    }

    // (b) Lambda for every pending slot: leaf S^{-1} Y_i in place; nonleaf L^{-1}[T_children]
    {
      Batch<TrsmProb> tb;
      Batch<CopyProb> cb;
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        const int m = mrow[i];
        if (m == 0) continue;
        TrsmProb tp;
        tp.T = F.p + mmo[a]; tp.ldt = m; tp.n = m; tp.lower = 1; tp.trans = 0;
        if (leaf) {
          tp.B = Y + T.begin[i]; tp.ldb = n; tp.ncol = (int)ycols;
        } else {
          CopyProb cp{};
          const int64_t cl = T.child_begin[i] - T.depth_off[t + 1];
          cp.src = Tprev.p + troff_prev[cl] + (int64_t)(k - 1) * sc * troff_prev.back();
          cp.lds = troff_prev.back();
          cp.dst = W.p + wo[a]; cp.ldd = m; cp.m = m; cp.n = sc * (L - k); cp.alpha = 1.0;
          cb.push(cp);
          tp.B = W.p + wo[a]; tp.ldb = m; tp.ncol = sc * (L - k);
        }
        tb.push(tp);
      }
      cb.upload(s); copy_launch(cb, s);
      tb.tag = "trsm_hss_lambda";
      tb.upload(s); trsm_launch(tb, s);
    }
    // Lambda of slot k (the current level) for node a: pointer and ld
    auto lam = [&](int64_t a, int64_t slot_rel, int64_t& ld) -> double* {
      const int64_t i = o + a;
      if (leaf) { ld = n; return Y + T.begin[i] + (slot_rel + k - 1) * sc * n; }
      ld = mrow[i];
      return W.p + wo[a] + slot_rel * sc * (int64_t)mrow[i];
    };

    // (c) pivoted QR of Lambda_i Omega -> V_i (or Vbar_i)
    {
      Batch<CopyProb> cb;
      Batch<QrProb> qb;
      int maxm = 1;
      for (int64_t a = 0; a < nn; ++a) {
        const int m = mrow[o + a];
        maxm = std::max(maxm, m);
        int64_t ld;
        const double* src = lam(a, 0, ld);
        if (m > 0) {
          CopyProb cp{};
          cp.src = src; cp.lds = ld; cp.dst = Q.p + qo[a]; cp.ldd = m; cp.m = m; cp.n = sc;
          cp.alpha = 1.0;
          cb.push(cp);
        }
        QrProb q;
        q.A = Q.p + qo[a]; q.lda = std::max(m, 1); q.m = m; q.n = sc;
        q.kmax = std::min(r, std::min(m, sc)); q.rtol = std::max(rtol, 1e-14);
        q.piv = piv.p + a * sc; q.tau = tau.p + mo[a]; q.rank = rkd.p + a;
        q.norms = norms.p + 2 * a * sc;
        q.downdate = 0;   // sketches are close to full rank: every norm would be recomputed
        qb.push(q);
      }
      cb.upload(s); copy_launch(cb, s);
      qb.tag = "geqp3_hss";
      qb.upload(s);
      const int pslot = geqp3_launch(qb, 1, 1, maxm, s);
      std::vector<int> hr = rkd.download(s);
      if (pslot >= 0) {
        double f = 0.0;
        for (int64_t a = 0; a < nn; ++a) f += qr_flops(mrow[o + a], sc, hr[a], true);
        prof_add_flops(pslot, f);
      }
      for (int64_t a = 0; a < nn; ++a) rk[o + a] = mrow[o + a] > 0 ? hr[a] : 0;
    }
    // sizes that depend on the ranks
    std::vector<int64_t> vsz(nn), rr(nn), phs(nn);
    for (int64_t a = 0; a < nn; ++a) {
      vsz[a] = (int64_t)mrow[o + a] * rk[o + a];
      rr[a] = rk[o + a];
      phs[a] = (int64_t)rk[o + a] * h2->rank(o + a);
    }
    const std::vector<int64_t> vo = prefix(vsz), ro = prefix(rr), pho = prefix(phs);
    const int64_t Rl = std::max<int64_t>(ro[nn], 1);
    DevBuf<double> V(std::max<int64_t>(vo[nn], 1)), G(std::max<int64_t>(vo[nn], 1));
    DevBuf<double> Tcur((size_t)Rl * ycols), PhiU(std::max<int64_t>(pho[nn], 1));
    Tcur.zero(s);
    genpool[o] = std::unique_ptr<DevBuf<double>>(new DevBuf<double>(std::max<int64_t>(vo[nn], 1)));
    for (int64_t a = 0; a < nn; ++a) genp[o + a] = genpool[o]->p + vo[a];
    {
      Batch<FormQProb> fb;
      for (int64_t a = 0; a < nn; ++a) {
        const int m = mrow[o + a];
        if (m == 0 || rk[o + a] == 0) continue;
        FormQProb f;
        f.V = Q.p + qo[a]; f.ldv = m; f.tau = tau.p + mo[a]; f.k = rkd.p + a;
        f.Q = V.p + vo[a]; f.ldq = m; f.m = m; f.kcols = rk[o + a];
        fb.push(f);
      }
      fb.upload(s);
      form_q_launch(fb, s);
    }
    // (d) T pushed up (Alg. 5.2), G = F^{-T} V, U or R = F V, Phi U^H2
    {
      GemmBatch gb;
      Batch<CopyProb> cb;
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        const int m = mrow[i], ri = rk[i];
        if (m == 0 || ri == 0) continue;
        const int pend = L - 1 - k;   // slots k+1 .. L-1
        if (pend > 0) {
          int64_t ld;
          const double* src = lam(a, 1, ld);
          gb.add(Tcur.p + ro[a] + (int64_t)k * sc * Rl, Rl, ri, sc * pend, V.p + vo[a], m, 1, src,
                 ld, 0, m, 1.0, 0.0);
        }
        gb.add(genp[i], m, m, ri, F.p + mmo[a], m, 0, V.p + vo[a], m, 0, m, 1.0, 0.0);
        CopyProb cp{};
        cp.src = V.p + vo[a]; cp.lds = m; cp.dst = G.p + vo[a]; cp.ldd = m; cp.m = m; cp.n = ri;
        cp.alpha = 1.0;
        cb.push(cp);
      }
      gb.run(s);
      cb.upload(s);
      copy_launch(cb, s);
      Batch<TrsmProb> tb;
      for (int64_t a = 0; a < nn; ++a) {
        const int m = mrow[o + a], ri = rk[o + a];
        if (m == 0 || ri == 0) continue;
        TrsmProb tp;
        tp.T = F.p + mmo[a]; tp.ldt = m; tp.B = G.p + vo[a]; tp.ldb = m; tp.n = m; tp.ncol = ri;
        tp.lower = 1; tp.trans = 1;
        tb.push(tp);
      }
      tb.tag = "trsm_hss_G";
      tb.upload(s);
      trsm_launch(tb, s);
      // Phi U^H2: leaf G^T U^H2; nonleaf Gbar^T (diag(PhiU_c) R^H2_i)
      std::vector<int64_t> zsz(nn);
      for (int64_t a = 0; a < nn; ++a) zsz[a] = leaf ? 0 : (int64_t)mrow[o + a] * h2->rank(o + a);
      const std::vector<int64_t> zo = prefix(zsz);
      DevBuf<double> Z(std::max<int64_t>(zo[nn], 1));
      GemmBatch zb, pbt;
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        const int m = mrow[i], ri = rk[i], ki = h2->rank(i);
        if (m == 0 || ri == 0 || ki == 0) continue;
        if (leaf) {
          pbt.add(PhiU.p + pho[a], ri, ri, ki, G.p + vo[a], m, 1, UH + h2->U_off[i],
                  h2->U_rows[i], 0, m, 1.0, 0.0);
        } else {
          int64_t roff = 0, koff = 0;
          for (int64_t c = T.child_begin[i]; c < T.child_end[i]; ++c) {
            const int64_t cl = c - T.depth_off[t + 1];
            const int rc = rk[c], kc = h2->rank(c);
            if (rc > 0) {
              zb.prob(Z.p + zo[a] + roff, m, rc, ki, 1.0, 0.0);
              if (kc > 0)
                zb.seg(PhiUprev.p + phiu_off_prev[cl], rc, 0, UH + h2->U_off[i] + koff,
                       h2->U_rows[i], 0, kc);
            }
            roff += rc;
            koff += kc;
          }
          pbt.add(PhiU.p + pho[a], ri, ri, ki, G.p + vo[a], m, 1, Z.p + zo[a], m, 0, m, 1.0, 0.0);
        }
      }
      zb.run(s);
      pbt.run(s);
    }

    // (e) coefficient matrices for every near (!= self) and far pair of this level, i < j
    std::vector<PairRef> nearB(T.near_idx.size()), farB(T.far_idx.size());
    {
      std::vector<int64_t> bsz;
      std::vector<std::pair<int64_t, int64_t>> own;   // (list kind*big + entry)
      int64_t tot = 0;
      std::vector<int64_t> noff(T.near_idx.size(), -1), foff(T.far_idx.size(), -1);
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
          const int64_t j = T.near_idx[e];
          if (i < j && rk[i] > 0 && rk[j] > 0) { noff[e] = tot; tot += (int64_t)rk[i] * rk[j]; }
        }
        for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
          const int64_t j = T.far_idx[e];
          if (i < j && rk[i] > 0 && rk[j] > 0) { foff[e] = tot; tot += (int64_t)rk[i] * rk[j]; }
        }
      }
      std::unique_ptr<DevBuf<double>> Bpool(new DevBuf<double>(std::max<int64_t>(tot, 1)));
      double* BP = Bpool->p;
      // references for both orientations
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e) {
          const int64_t j = T.near_idx[e];
          if (j == i || rk[i] == 0 || rk[j] == 0) continue;
          if (i < j) nearB[e] = PairRef{BP + noff[e], 0, rk[i]};
          else nearB[e] = PairRef{BP + noff[find_entry(T.near_off, T.near_idx, j, i)], 1, rk[j]};
        }
        for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e) {
          const int64_t j = T.far_idx[e];
          if (rk[i] == 0 || rk[j] == 0) continue;
          if (i < j) farB[e] = PairRef{BP + foff[e], 0, rk[i]};
          else farB[e] = PairRef{BP + foff[find_entry(T.far_off, T.far_idx, j, i)], 1, rk[j]};
        }
      }
      // chunks of pairs whose intermediates fit a budget
      const int64_t budget = (int64_t)1 << 28;   // doubles (2 GiB)
      struct Job { int64_t i, j, e; int far; };
      std::vector<Job> jobs;
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        for (int64_t e = T.near_off[i]; e < T.near_off[i + 1]; ++e)
          if (noff[e] >= 0) jobs.push_back(Job{i, T.near_idx[e], e, 0});
        for (int64_t e = T.far_off[i]; e < T.far_off[i + 1]; ++e)
          if (foff[e] >= 0) jobs.push_back(Job{i, T.far_idx[e], e, 1});
      }
      auto tmp_rows = [&](const Job& jb) -> int64_t {
        return jb.far ? h2->rank(jb.i) : mrow[jb.i];
      };
      size_t pos = 0;
      while (pos < jobs.size()) {
        size_t end = pos;
        int64_t need = 0;
        while (end < jobs.size()) {
          const int64_t b = tmp_rows(jobs[end]) * rk[jobs[end].j];
          if (end > pos && need + b > budget) break;
          need += b;
          ++end;
        }
        DevBuf<double> tmp(std::max<int64_t>(need, 1));
        NearBatch nb;
        GemmBatch g1, g2;
        int64_t to = 0;
        for (size_t q = pos; q < end; ++q) {
          const Job& jb = jobs[q];
          const int64_t i = jb.i, j = jb.j;
          const int64_t al = i - o, bl = j - o;
          const int ri = rk[i], rj = rk[j];
          double* Bij = BP + (jb.far ? foff[jb.e] : noff[jb.e]);
          double* tp = tmp.p + to;
          if (jb.far) {
            const int ki = h2->rank(i), kj = h2->rank(j);
            const int64_t he = jb.e;
            if (ki == 0 || kj == 0) {
              g2.prob(Bij, ri, ri, rj, 1.0, 0.0);   // zero block
            } else {
              const int tr = h2->far_trans[he];
              // tmp = B^H2_ij (PhiU_j)^T  (k_i x r_j)
              g1.add(tp, ki, ki, rj, h2->coup.p + h2->far_boff[he], tr ? kj : ki, tr,
                     PhiU.p + pho[bl], rj, 1, kj, 1.0, 0.0);
              g2.add(Bij, ri, ri, rj, PhiU.p + pho[al], ri, 0, tp, ki, 0, ki, 1.0, 0.0);
            }
          } else if (leaf) {
            // tmp = A_ij G_j on the fly (|I_i| x r_j); B_ij = G_i^T tmp
            nb.prob(T.begin[i], mrow[i], tp, mrow[i], rj, 0);
            nb.seg(T.begin[j], mrow[j], G.p + vo[bl], mrow[j], 0);
            g2.add(Bij, ri, ri, rj, G.p + vo[al], mrow[i], 1, tp, mrow[i], 0, mrow[i], 1.0, 0.0);
          } else {
            // tmp = bold B_ij Gbar_j (M_i x r_j) from the children's blocks (Eq. Mijk)
            int64_t roff = 0;
            for (int64_t ca = T.child_begin[i]; ca < T.child_end[i]; ++ca) {
              const int rca = rk[ca];
              if (rca == 0) continue;
              g1.prob(tp + roff, mrow[i], rca, rj, 1.0, 0.0);
              int64_t coff = 0;
              for (int64_t cbn = T.child_begin[j]; cbn < T.child_end[j]; ++cbn) {
                const int rcb = rk[cbn];
                if (rcb == 0) continue;
                int64_t e2 = find_entry(T.near_off, T.near_idx, ca, cbn);
                PairRef ref;
                if (e2 >= 0) ref = nearB_prev[e2];
                else {
                  e2 = find_entry(T.far_off, T.far_idx, ca, cbn);
                  SPD_REQUIRE(e2 >= 0, "spdhss_build: child pair missing from the lists");
                  ref = farB_prev[e2];
                }
                g1.seg(ref.p, ref.ld, ref.trans, G.p + vo[bl] + coff, mrow[j], 0, rcb);
                coff += rcb;
              }
              roff += rca;
            }
            g2.add(Bij, ri, ri, rj, G.p + vo[al], mrow[i], 1, tp, mrow[i], 0, mrow[i], 1.0, 0.0);
          }
          to += tmp_rows(jb) * rj;
        }
        nb.tag = "near_hss_type1";
        g1.tag = g2.tag = "gemm_hss_pairs";
        nb.upload(s);
        nb.launch(h2->kfn, xs, n, dim, s);
        g1.run(s);
        g2.run(s);
        pos = end;
      }
      // sibling pairs of this level, kept for the final HSS
      for (int64_t a = 0; a < nn; ++a) {
        const int64_t i = o + a;
        if (T.parent[i] < 0) continue;
        const int64_t par = T.parent[i];
        for (int64_t j = T.child_begin[par]; j < T.child_end[par]; ++j) {
          if (j == i || rk[i] == 0 || rk[j] == 0) continue;
          int64_t e = find_entry(T.near_off, T.near_idx, i, j);
          PairRef ref = e >= 0 ? nearB[e] : farB[find_entry(T.far_off, T.far_idx, i, j)];
          sib_src.push_back(SibSrc{i, j, ref});
        }
      }
      keep_pools.push_back(std::move(Bpool));
    }
    // hand over to the next level
    Tprev = std::move(Tcur);
    troff_prev = ro;
    troff_prev.back() = Rl;   // last entry: leading dimension of Tprev
    PhiUprev = std::move(PhiU);
    phiu_off_prev = pho;
    nearB_prev = std::move(nearB);
    farB_prev = std::move(farB);
    // pools two levels back are no longer needed except for their sibling blocks: keep
    // them (sibling blocks are compacted below)
  }

  // ---- compact the generators and the sibling blocks ---------------------------------
  merge_stage(5, 0);
  hs->hoff.assign(NN + 1, 0);
  for (int i = 0; i < NN; ++i) hs->hoff[i + 1] = hs->hoff[i] + rk[i];
  hs->Rtot = hs->hoff[NN];
  hs->gen_off.assign(NN, 0);
  int64_t gt = 0;
  for (int i = 0; i < NN; ++i) { hs->gen_off[i] = gt; gt += (int64_t)mrow[i] * rk[i]; }
  hs->gen.alloc(std::max<int64_t>(gt, 1));
  for (int i = 0; i < NN; ++i)
    if ((int64_t)mrow[i] * rk[i] > 0)
      SPD_CUDA(cudaMemcpyAsync(hs->gen.p + hs->gen_off[i], genp[i],
                               (size_t)mrow[i] * rk[i] * sizeof(double), cudaMemcpyDeviceToDevice,
                               s));
  std::sort(sib_src.begin(), sib_src.end(), [](const SibSrc& x, const SibSrc& y) {
    return x.a != y.a ? x.a < y.a : x.b < y.b;
  });
  hs->sib_off.assign(NN + 1, 0);
  hs->sib_node.clear();
  hs->sib_boff.clear();
  int64_t st = 0;
  Batch<CopyProb> cb;
  std::vector<int64_t> cnt(NN, 0);
  for (const auto& x : sib_src) cnt[x.a]++;
  for (int i = 0; i < NN; ++i) hs->sib_off[i + 1] = hs->sib_off[i] + cnt[i];
  for (const auto& x : sib_src) {
    hs->sib_node.push_back(x.b);
    hs->sib_boff.push_back(st);
    st += (int64_t)rk[x.a] * rk[x.b];
  }
  hs->sib.alloc(std::max<int64_t>(st, 1));
  for (size_t q = 0; q < sib_src.size(); ++q) {
    const auto& x = sib_src[q];
    CopyProb cp{};
    cp.src = x.ref.p; cp.lds = x.ref.ld; cp.trans = x.ref.trans;
    cp.dst = hs->sib.p + hs->sib_boff[q]; cp.ldd = rk[x.a];
    cp.m = rk[x.a]; cp.n = rk[x.b]; cp.alpha = 1.0;
    cb.push(cp);
  }
  cb.upload(s);
  copy_launch(cb, s);
  SPD_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------------------
// HSS product: upward (U^T, R^T), sibling couplings, downward (R, U), dense leaf blocks
// ---------------------------------------------------------------------------------------
struct HssPlan {
  int ncol = 0;
  DevBuf<double> xs, ys, xhat, yhat;
  GemmBatch up_leaf, coupling, leaf_out;
  std::vector<GemmBatch> up, down;
  NearBatch near;
};

static void hss_plan_build(const spdhss_hss_s* hs, HssPlan& P, int ncol, cudaStream_t s) {
  const spdhss_h2_s* h2 = hs->h2;
  const TreeHost& T = h2->th;
  const int64_t n = T.n, K = std::max<int64_t>(hs->Rtot, 1);
  const int D = T.D;
  P.ncol = ncol;
  P.xs.alloc((size_t)n * ncol);
  P.ys.alloc((size_t)n * ncol);
  P.xhat.alloc((size_t)K * ncol);
  P.yhat.alloc((size_t)K * ncol);
  const std::vector<int>& rk = hs->rk;
  auto gen = [&](int64_t i) { return hs->gen.p + hs->gen_off[i]; };
  if (D > 0) {
    for (int64_t i = T.depth_off[D]; i < T.depth_off[D + 1]; ++i)
      if (rk[i] > 0)
        P.up_leaf.add(P.xhat.p + hs->hoff[i], K, rk[i], ncol, gen(i), hs->mrow[i], 1,
                      P.xs.p + T.begin[i], n, 0, hs->mrow[i], 1.0, 0.0);
    for (int t = D - 1; t >= 1; --t) {
      P.up.emplace_back();
      for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i)
        if (rk[i] > 0)
          P.up.back().add(P.xhat.p + hs->hoff[i], K, rk[i], ncol, gen(i), hs->mrow[i], 1,
                          P.xhat.p + hs->hoff[T.child_begin[i]], K, 0, hs->mrow[i], 1.0, 0.0);
    }
    for (int64_t a = 0; a < T.nn(); ++a) {
      if (rk[a] == 0 || hs->sib_off[a] == hs->sib_off[a + 1]) continue;
      P.coupling.prob(P.yhat.p + hs->hoff[a], K, rk[a], ncol, 1.0, 1.0);
      for (int64_t e = hs->sib_off[a]; e < hs->sib_off[a + 1]; ++e) {
        const int64_t b = hs->sib_node[e];
        P.coupling.seg(hs->sib.p + hs->sib_boff[e], rk[a], 0, P.xhat.p + hs->hoff[b], K, 0, rk[b]);
      }
    }
    for (int t = 1; t <= D - 1; ++t) {
      P.down.emplace_back();
      for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i)
        if (rk[i] > 0)
          P.down.back().add(P.yhat.p + hs->hoff[T.child_begin[i]], K, hs->mrow[i], ncol, gen(i),
                            hs->mrow[i], 0, P.yhat.p + hs->hoff[i], K, 0, rk[i], 1.0, 1.0);
    }
  }
  for (int64_t i = T.depth_off[D]; i < T.depth_off[D + 1]; ++i) {
    P.leaf_out.prob(P.ys.p + T.begin[i], n, (int)T.size(i), ncol, 1.0, 0.0);
    if (D > 0 && rk[i] > 0)
      P.leaf_out.seg(gen(i), hs->mrow[i], 0, P.yhat.p + hs->hoff[i], K, 0, rk[i]);
    P.near.prob(T.begin[i], (int)T.size(i), P.ys.p + T.begin[i], n, ncol, 1);
    P.near.seg(T.begin[i], (int)T.size(i), P.xs.p + T.begin[i], n, 1);
  }
  P.up_leaf.upload(s);
  for (auto& g : P.up) g.upload(s);
  P.coupling.upload(s);
  for (auto& g : P.down) g.upload(s);
  P.leaf_out.upload(s);
  P.near.upload(s);
}

void hss_matmul_impl(spdhss_hss_s* hs, const double* X, double* Y, int nrhs, int64_t ld,
                     cudaStream_t s) {
  auto it = hs->plans.find(nrhs);
  if (it == hs->plans.end()) {
    std::shared_ptr<HssPlan> p(new HssPlan());
    hss_plan_build(hs, *p, nrhs, s);
    it = hs->plans.emplace(nrhs, std::static_pointer_cast<void>(p)).first;
  }
  const HssPlan& P = *std::static_pointer_cast<HssPlan>(it->second);
  const spdhss_h2_s* h2 = hs->h2;
  const int64_t n = h2->th.n;
  permute_to_sorted(X, ld, P.xs.p, n, nrhs, h2->td.perm.p, s);
  P.up_leaf.launch(s);
  for (const auto& g : P.up) g.launch(s);
  SPD_CUDA(cudaMemsetAsync(P.yhat.p, 0, P.yhat.bytes(), s));
  P.coupling.launch(s);
  for (const auto& g : P.down) g.launch(s);
  P.leaf_out.launch(s);
  P.near.launch(h2->kfn, h2->td.xs.p, n, h2->th.dim, s);
  permute_from_sorted(P.ys.p, Y, ld, n, nrhs, h2->td.perm.p, s);
}

}  // namespace spd
