// ulv_solve_noalloc: the ULV solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that has reserved all device memory
// for its own allocator, or a latency-critical path that cannot afford the implicit device
// synchronization of cudaMalloc / cudaFree.  ulv_solve sizes and allocates its level
// buffers and launch descriptors on first use per column count; this variant instead
// works in two fixed file-scope device arrays: one for the level buffers (48 MiB) and one
// for the launch descriptors (8 MiB).  They are part of the library's device image, so
// every GPU that loads them holds them until the process exits.
//
// The library's modules are loaded lazily: the module holding the two arrays is loaded
// (its 56 MiB taken from the device) the first time their addresses are looked up.  That
// look-up (cudaGetSymbolAddress, with the device current) is made once per device by
// ulv_factor, which allocates anyway, so that the solve itself allocates nothing; a solve
// on a device where no factorization has run makes the look-up itself.
//
// The descriptors of one column count depend only on the handle and the device's arrays:
// they are built once per (handle, column count) into a host image that the handle keeps
// unchanged until it is destroyed, and every call copies that image into the descriptor
// array.  Every call shares the two arrays and leaves its data in them; the solve writes
// every element it later reads (the right-hand side into the leaf-level buffer, the
// reduced parts into every block above), so nothing has to start at zero.  Two calls
// whose work overlaps on the GPU (different streams) race on the arrays.
//
// The sweeps are those of the ULV solve in the reflector-and-substitution form: each
// node's stored Householder reflectors (Wbuf, taub) and its complement Cholesky factor
// (Dbuf) are applied directly, where ulv_solve multiplies by the explicit per-node solve
// matrices made from the same factors.  Both are exact forms of the same solve.
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>

#include "ulv.cuh"

namespace spd {
namespace {

constexpr size_t kScratchDoubles = (size_t)6 << 20;   // 6 Mi doubles = 48 MiB
constexpr size_t kDescBytes = (size_t)8 << 20;        // 8 MiB of launch descriptors

static __device__ __align__(256) double g_ulv_scratch[kScratchDoubles];
static __device__ __align__(256) unsigned char g_ulv_desc[kDescBytes];

constexpr int kMaxDevices = 128;
struct DeviceArrays {
  double* scratch = nullptr;
  unsigned char* desc = nullptr;
};
static DeviceArrays g_arrays[kMaxDevices];
static std::mutex g_arrays_mu;

// Device addresses of the two arrays for the current device (set up once per device).
DeviceArrays arrays_for_current_device() {
  int dev = -1;
  SPD_CUDA(cudaGetDevice(&dev));
  SPD_REQUIRE(dev >= 0 && dev < kMaxDevices, "ulv_solve_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_arrays_mu);
  DeviceArrays& a = g_arrays[dev];
  if (a.scratch == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_ulv_scratch);
    if (e != cudaSuccess)
      throw Error(SPDHSS_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_ulv_desc);
    if (e != cudaSuccess)
      throw Error(SPDHSS_ECUDA, std::string("cudaGetSymbolAddress(descriptors): ") + cudaGetErrorString(e));
    a.desc = (unsigned char*)q;
    a.scratch = (double*)p;
  }
  return a;
}

}  // namespace

void ulv_noalloc_prepare_device() { (void)arrays_for_current_device(); }

namespace {

// Host image of the descriptor array: typed blocks at 256-byte aligned offsets.
struct Stage {
  std::vector<unsigned char> bytes;
  template <class T>
  size_t put(const std::vector<T>& v) {
    size_t off = (bytes.size() + 255) & ~(size_t)255;
    bytes.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

struct LevelOps {
  size_t qt = 0, qw = 0; int64_t nq = 0;            // reflectors + (prob, col) work
  size_t fw = 0, bk = 0, tw = 0; int64_t nt = 0;    // triangular solves + work
  size_t gfp = 0, gfs = 0, gft = 0; int64_t nft = 0; int nbf = 0;   // b_p -= X^T y_q
  size_t gbp = 0, gbs = 0, gbt = 0; int64_t nbt = 0; int nbb = 0;   // y_q -= X x_p
  size_t up = 0, dn = 0; int64_t ncp = 0, cmax = 0;                  // copies to / from parent
};

}  // namespace

// Everything one column count needs: the host image of the descriptors (never modified
// once built), the offsets of its blocks and the level buffers' layout in the scratch.
struct NoallocPlan {
  Stage st;
  std::vector<LevelOps> ops;
  std::vector<int64_t> boff;
  size_t orf = 0, orb = 0, orw = 0;
  int64_t nrw = 0;
  double* scratch = nullptr;
};

// The plan of one column count for the current device (EINVAL when it exceeds the arrays).
static std::shared_ptr<NoallocPlan> noalloc_plan(const spdhss_ulv_s* u, int ncol,
                                                 const DeviceArrays& dev) {
  const TreeHost& T = u->hs->h2->th;
  const int64_t n = T.n;
  const int L = u->L, D = u->D;
  const int nlev = std::max(L - 1, 0);
  std::shared_ptr<NoallocPlan> plan = std::make_shared<NoallocPlan>();
  plan->scratch = dev.scratch;
  // ---- level buffers inside the scratch array --------------------------------------
  std::vector<int64_t> ldk(nlev + 1, 0);
  std::vector<int64_t>& boff = plan->boff;
  std::vector<int64_t> moff(T.nn(), 0);
  if (D == 0) {
    ldk.assign(1, n);
  } else {
    for (int k = 1; k <= L - 1; ++k) {
      const int t = D + 1 - k;
      int64_t tot = 0;
      for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i) {
        moff[i] = (k == 1) ? T.begin[i] : tot;
        tot += u->m[i];
      }
      ldk[k - 1] = (k == 1) ? n : std::max<int64_t>(tot, 1);
    }
    ldk[nlev] = std::max(u->mroot, 1);
  }
  boff.assign(ldk.size() + 1, 0);
  for (size_t k = 0; k < ldk.size(); ++k) boff[k + 1] = boff[k] + ldk[k] * ncol;
  const size_t need = (size_t)boff.back();
  if (need > kScratchDoubles) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "ulv_solve_noalloc needs %zu doubles of level buffers for %d columns; the "
                  "fixed scratch holds %zu (48 MiB); use fewer columns or ulv_solve",
                  need, ncol, kScratchDoubles);
    throw Error(SPDHSS_EINVAL, msg);
  }
  auto bw = [&](int k) { return dev.scratch + boff[k]; };

  // ---- descriptors (host image, then one copy into the descriptor array) ----------------
  Stage& st = plan->st;
  std::vector<LevelOps>& ops = plan->ops;
  ops.assign(nlev, LevelOps());
  for (int k = 1; k <= nlev; ++k) {
    const int t = D + 1 - k;
    const int64_t ldb = ldk[k - 1], ldn = ldk[k];
    double* lev = bw(k - 1);
    double* par = bw(k);
    std::vector<HhApplyProb> hh;
    std::vector<TrsmProb> tf, tb;
    std::vector<int2> hw, tw;
    std::vector<GemmProb> gfp, gbp;
    std::vector<GemmSeg> gfs, gbs;
    std::vector<CopyProb> cu, cd;
    int64_t cmax = 1;
    for (int64_t i = T.depth_off[t]; i < T.depth_off[t + 1]; ++i) {
      const int m = u->m[i], r = u->r[i];
      if (m == 0) continue;
      double* blk = lev + moff[i];
      const double* Di = u->Dbuf.p + u->Doff[i];
      if (r > 0) {
        HhApplyProb hp;
        hp.V = u->Wbuf.p + u->Woff[i]; hp.ldv = m; hp.tau = u->taub.p + u->toff[i];
        hp.k = u->rdev.p + i; hp.B = blk; hp.ldb = ldb; hp.m = m; hp.ncol = ncol;
        for (int c = 0; c < ncol; ++c) hw.push_back(make_int2((int)hh.size(), c));
        hh.push_back(hp);
      }
      if (m - r > 0) {
        for (int c = 0; c < ncol; ++c) tw.push_back(make_int2((int)tf.size(), c));
        tf.push_back(TrsmProb{Di + r + (int64_t)r * m, m, blk + r, ldb, m - r, ncol, 1, 0});
        tb.push_back(TrsmProb{Di + r + (int64_t)r * m, m, blk + r, ldb, m - r, ncol, 1, 1});
        if (r > 0) {
          GemmProb p{};
          p.C = blk; p.ldc = ldb; p.M = r; p.N = ncol; p.alpha = -1.0; p.beta = 1.0;
          p.seg0 = (int)gfs.size(); p.seg1 = p.seg0 + 1;
          gfp.push_back(p);
          gfs.push_back(GemmSeg{Di + r, blk + r, m, ldb, m - r, 1, 0});
          GemmProb q{};
          q.C = blk + r; q.ldc = ldb; q.M = m - r; q.N = ncol; q.alpha = -1.0; q.beta = 1.0;
          q.seg0 = (int)gbs.size(); q.seg1 = q.seg0 + 1;
          gbp.push_back(q);
          gbs.push_back(GemmSeg{Di + r, blk, m, ldb, r, 0, 0});
        }
      }
      if (r > 0) {
        const int64_t p = T.parent[i];
        int64_t pos = 0;
        for (int64_t c = T.child_begin[p]; c < i; ++c) pos += u->r[c];
        const int64_t pbase = (k == L - 1) ? 0 : moff[p];
        CopyProb a{};
        a.src = blk; a.lds = ldb; a.dst = par + pbase + pos; a.ldd = ldn; a.m = r; a.n = ncol;
        a.alpha = 1.0;
        cu.push_back(a);
        CopyProb d{};
        d.src = par + pbase + pos; d.lds = ldn; d.dst = blk; d.ldd = ldb; d.m = r; d.n = ncol;
        d.alpha = 1.0;
        cd.push_back(d);
        cmax = std::max<int64_t>(cmax, (int64_t)r * ncol);
      }
    }
    LevelOps& o = ops[k - 1];
    o.qt = st.put(hh); o.qw = st.put(hw); o.nq = (int64_t)hw.size();
    o.fw = st.put(tf); o.bk = st.put(tb); o.tw = st.put(tw); o.nt = (int64_t)tw.size();
    std::vector<int4> tfl = gemm_tiles(gfp, &o.nbf), tbl = gemm_tiles(gbp, &o.nbb);
    o.gfp = st.put(gfp); o.gfs = st.put(gfs); o.gft = st.put(tfl); o.nft = (int64_t)tfl.size();
    o.gbp = st.put(gbp); o.gbs = st.put(gbs); o.gbt = st.put(tbl); o.nbt = (int64_t)tbl.size();
    o.up = st.put(cu); o.dn = st.put(cd); o.ncp = (int64_t)cu.size(); o.cmax = cmax;
  }
  // root: dense Cholesky solve on the top buffer
  std::vector<TrsmProb> rf, rb;
  std::vector<int2> rw;
  const int mr = (D == 0) ? (int)n : u->mroot;
  double* top = (D == 0) ? bw(0) : bw(nlev);
  const int64_t ldtop = (D == 0) ? n : ldk[nlev];
  if (mr > 0) {
    rf.push_back(TrsmProb{u->root.p, mr, top, ldtop, mr, ncol, 1, 0});
    rb.push_back(TrsmProb{u->root.p, mr, top, ldtop, mr, ncol, 1, 1});
    for (int c = 0; c < ncol; ++c) rw.push_back(make_int2(0, c));
  }
  plan->orf = st.put(rf);
  plan->orb = st.put(rb);
  plan->orw = st.put(rw);
  plan->nrw = (int64_t)rw.size();
  if (st.bytes.size() > kDescBytes) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "ulv_solve_noalloc needs %zu bytes of launch descriptors; the fixed array "
                  "holds %zu (8 MiB); use fewer columns or ulv_solve", st.bytes.size(), kDescBytes);
    throw Error(SPDHSS_EINVAL, msg);
  }
  return plan;
}

void ulv_solve_noalloc_impl(spdhss_ulv_s* u, const double* B, double* X, int ncol, int64_t ld,
                            cudaStream_t s) {
  const DeviceArrays dev = arrays_for_current_device();
  const int64_t n = u->hs->h2->th.n;
  const int nlev = std::max(u->L - 1, 0);
  const int D = u->D;
  const int64_t* perm = u->hs->h2->td.perm.p;
  std::shared_ptr<NoallocPlan>& slot = u->noalloc_plans[ncol];
  if (!slot || slot->scratch != dev.scratch) slot = noalloc_plan(u, ncol, dev);
  const NoallocPlan& P = *slot;
  const std::vector<LevelOps>& ops = P.ops;
  auto bw = [&](int k) { return dev.scratch + P.boff[k]; };
  // the plan's descriptor image, unchanged since it was built, into the descriptor array
  if (!P.st.bytes.empty())
    SPD_CUDA(cudaMemcpyAsync(dev.desc, P.st.bytes.data(), P.st.bytes.size(),
                             cudaMemcpyHostToDevice, s));
  auto D_ = [&](size_t off) { return (const void*)(dev.desc + off); };
  const size_t orf = P.orf, orb = P.orb, orw = P.orw;
  const int64_t nrw = P.nrw;
  (void)D;

  // ---- the solve: ULV sweeps up the levels, root solves, sweeps down ------------------
  permute_to_sorted(B, ld, bw(0), n, ncol, perm, s);
  for (int k = 0; k < nlev; ++k) {
    const LevelOps& o = ops[k];
    householder_launch_raw((const HhApplyProb*)D_(o.qt), (const int2*)D_(o.qw), o.nq, 1, s);
    trsm_launch_raw((const TrsmProb*)D_(o.fw), (const int2*)D_(o.tw), o.nt, s);
    gemm_launch_raw((const GemmProb*)D_(o.gfp), (const GemmSeg*)D_(o.gfs), (const int4*)D_(o.gft),
                    o.nft, o.nbf, s);
    copy_launch_raw((const CopyProb*)D_(o.up), o.ncp, o.cmax, s);
  }
  trsm_launch_raw((const TrsmProb*)D_(orf), (const int2*)D_(orw), nrw, s);
  trsm_launch_raw((const TrsmProb*)D_(orb), (const int2*)D_(orw), nrw, s);
  for (int k = nlev - 1; k >= 0; --k) {
    const LevelOps& o = ops[k];
    copy_launch_raw((const CopyProb*)D_(o.dn), o.ncp, o.cmax, s);
    gemm_launch_raw((const GemmProb*)D_(o.gbp), (const GemmSeg*)D_(o.gbs), (const int4*)D_(o.gbt),
                    o.nbt, o.nbb, s);
    trsm_launch_raw((const TrsmProb*)D_(o.bk), (const int2*)D_(o.tw), o.nt, s);
    householder_launch_raw((const HhApplyProb*)D_(o.qt), (const int2*)D_(o.qw), o.nq, 0, s);
  }
  permute_from_sorted(bw(0), X, ld, n, ncol, perm, s);
}

}  // namespace spd

extern "C" spdhss_status ulv_solve_noalloc(ulv_handle u, const double* B, double* X, int nrhs,
                                           int64_t ld, void* stream) {
  try {
    SPD_REQUIRE(u && B && X, "ulv_solve_noalloc: NULL argument");
    SPD_REQUIRE(nrhs >= 1, "ulv_solve_noalloc: nrhs must be >= 1");
    SPD_REQUIRE(ld >= u->hs->h2->th.n, "ulv_solve_noalloc: ld must be >= n");
    spd::ulv_solve_noalloc_impl(u, B, X, nrhs, ld, (cudaStream_t)stream);
    return SPDHSS_OK;
  } catch (const spd::Error& e) {
    spd::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    spd::set_last_error(std::string("ulv_solve_noalloc: ") + e.what());
    return SPDHSS_ECUDA;
  }
}
