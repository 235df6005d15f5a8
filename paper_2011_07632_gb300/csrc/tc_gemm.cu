// Grouped FP32 GEMMs on the fifth-generation tensor cores (tcgen05.mma, kind::tf32).
//
// One CTA of 128 threads computes a 128 x NT tile of C = alpha sum_s op(A_s) op(B_s) +
// beta C for one problem of a grouped batch (the same problems, segments and tiles as
// the CUDA-core k_gemm).  The K range of every segment is walked in chunks of 32: the four
// warps stage the chunk of A (128 rows) and of B (NT rows) into shared memory, converted to
// TF32 and laid out in the canonical K-major core-matrix layout without swizzle (core
// matrix = 8 rows x 16 bytes, K-adjacent cores 128 bytes apart, M/N-adjacent cores 256
// bytes apart), two stages deep; one elected thread issues the MMAs of the chunk
// (K = 8 each) into an FP32 accumulator in tensor memory and commits them to the stage's
// mbarrier, which the stagers wait on before they overwrite the stage.  The epilogue reads
// the accumulator with tcgen05.ld (warp w owns TMEM lanes 32 w .. 32 w + 31 = tile rows).
//
// Split mode (3xTF32): every operand is split into a TF32 head and a TF32 tail
// (x = hi + lo, hi = x rounded to TF32, lo = x - hi exactly in FP32) and every product is
// accumulated as lo_a hi_b + hi_a lo_b + hi_a hi_b (the lo lo term is below FP32 rounding),
// which gives FP32-accurate products on the tensor cores (Markidis et al., IPDPSW 2018;
// Ootomo and Yokota, IJHPCA 2022).
//
// Every wait on an mbarrier gives up after a bounded number of tries: the kernel then
// records the failure in the error word, waits (bounded) for its MMAs once more, frees its
// tensor memory and returns; the launcher turns the record into SPDHSS_TIMEOUT.
#include <algorithm>
#include <mutex>

#include "dense.cuh"

namespace spd {
namespace {

constexpr int TC_M = 128;     // tile rows (TMEM lanes)
constexpr int TC_KC = 32;     // K elements per stage
constexpr int TC_KS = 8;      // K per MMA instruction (32 bytes of TF32)
constexpr long long kTcWaitCycles = 1LL << 31;   // about one second at the SM clock

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a K-major stage tile (k < 32): sub-tile k / 8 of
// rows x 32 bytes, core (r / 8, (k % 8) / 4), row r % 8 (16 bytes), element k % 4
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int rows) {
  return (uint32_t)((k >> 3) * rows * 32 + (r >> 3) * 256 + ((k >> 2) & 1) * 128 +
                    (r & 7) * 16 + (k & 3) * 4);
}

// shared memory matrix descriptor, K-major, no swizzle: start, LBO = 128 B (K direction),
// SBO = 256 B (M/N direction), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, N, M
__host__ __device__ constexpr uint32_t tf32_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// true once the phase with the given parity has completed; false after about a second
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (clock64() - t0 < kTcWaitCycles) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// stage bytes of one operand tile: rows x 32 TF32 values
__host__ __device__ constexpr int stage_bytes(int rows) { return rows * TC_KC * 4; }

template <int NT, bool SPLIT>
__global__ void __launch_bounds__(128) k_gemm_tf32(const GemmProbT<float>* __restrict__ probs,
                                                   const GemmSegT<float>* __restrict__ segs,
                                                   const int4* __restrict__ tiles,
                                                   int* __restrict__ err, int stall) {
  constexpr int NOP = SPLIT ? 2 : 1;                        // hi (, lo) per operand
  constexpr int SA = stage_bytes(TC_M), SB = stage_bytes(NT);
  constexpr int STAGE = NOP * (SA + SB);
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint64_t s_bar[2];
  __shared__ uint32_t s_taddr;
  const int4 t = tiles[blockIdx.x];
  const GemmProbT<float> P = probs[t.x];
  const int m0 = t.y, n0 = t.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_taddr)),
                 "r"(NT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = s_taddr;
  const uint32_t idesc = tf32_idesc(TC_M, NT);
  const uint32_t sbase = smem_u32(tc_smem);

  bool ok = true;
  int chunk = 0;        // chunks staged so far (stage = chunk & 1)
  uint32_t issued = 0;  // MMAs issued (0: the accumulator holds nothing yet)
  for (int sg = P.seg0; sg < P.seg1; ++sg) {
    const GemmSegT<float> S = segs[sg];
    for (int k0 = 0; k0 < S.K; k0 += TC_KC, ++chunk) {
      const int st = chunk & 1;
      // the MMAs that read this stage two chunks ago must be done before it is overwritten
      // (every thread waits; the verdict is made uniform over the CTA)
      const bool w = chunk < 2 || mbar_wait(&s_bar[st], ((chunk - 2) >> 1) & 1);
      if (!__syncthreads_and(w)) { ok = false; break; }
      unsigned char* sa = tc_smem + st * STAGE;
      unsigned char* sb = sa + NOP * SA;
      // A chunk: 128 rows x 32 k; consecutive threads take consecutive rows (column-major
      // A) or consecutive k (transposed A), so that global reads are coalesced
      for (int e = tid; e < TC_M * TC_KC; e += 128) {
        int r, k;
        if (!S.tA) { r = e % TC_M; k = e / TC_M; } else { k = e % TC_KC; r = e / TC_KC; }
        const int gm = m0 + r, gk = k0 + k;
        float v = 0.f;
        if (gm < P.M && gk < S.K)
          v = S.tA ? S.A[gk + (int64_t)gm * S.lda] : S.A[gm + (int64_t)gk * S.lda];
        const uint32_t off = kmajor_off(r, k, TC_M);
        const float hi = to_tf32(v);
        *reinterpret_cast<float*>(sa + off) = hi;
        if (SPLIT) *reinterpret_cast<float*>(sa + SA + off) = to_tf32(v - hi);
      }
      // B chunk: NT columns x 32 k, stored as NT rows of K
      for (int e = tid; e < NT * TC_KC; e += 128) {
        int nn, k;
        if (!S.tB) { k = e % TC_KC; nn = e / TC_KC; } else { nn = e % NT; k = e / NT; }
        const int gn = n0 + nn, gk = k0 + k;
        float v = 0.f;
        if (gn < P.N && gk < S.K)
          v = S.tB ? S.B[gn + (int64_t)gk * S.ldb] : S.B[gk + (int64_t)gn * S.ldb];
        const uint32_t off = kmajor_off(nn, k, NT);
        const float hi = to_tf32(v);
        *reinterpret_cast<float*>(sb + off) = hi;
        if (SPLIT) *reinterpret_cast<float*>(sb + SB + off) = to_tf32(v - hi);
      }
      // the staged chunk, visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0 && !stall) {   // stall (test of the bounded waits): nothing is issued
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = sbase + st * STAGE, b0 = a0 + NOP * SA;
#pragma unroll
        for (int ks = 0; ks < TC_KC / TC_KS; ++ks) {
          const uint32_t ao = ks * TC_M * 32, bo = ks * NT * 32;
          if (SPLIT) {
            tc_mma(tbase, smem_desc(a0 + SA + ao), smem_desc(b0 + bo), idesc, issued++);
            tc_mma(tbase, smem_desc(a0 + ao), smem_desc(b0 + SB + bo), idesc, issued++);
          }
          tc_mma(tbase, smem_desc(a0 + ao), smem_desc(b0 + bo), idesc, issued++);
        }
        tc_commit(&s_bar[st]);
      }
      __syncthreads();
    }
    if (!ok) break;
  }
  // all MMAs done: the last commit covers every earlier one
  const int nch = chunk;
  {
    const bool w = !ok || nch == 0 || mbar_wait(&s_bar[(nch - 1) & 1], ((nch - 1) >> 1) & 1);
    ok = __syncthreads_and(ok && w);
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // bounded second wait for whatever is still in flight before the memory is freed
    if (nch > 0) (void)mbar_wait(&s_bar[(nch - 1) & 1], ((nch - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: row m0 + 32 warp + lane, 16 columns per load
  const int gm = m0 + warp * 32 + lane;
  const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
  const float alpha = (float)P.alpha, beta = (float)P.beta;
  if (ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
      float v[16];
      if (nch > 0) tmem_ld16(lane_base + (uint32_t)c0, v);
      else
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      if (gm < P.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int gn = n0 + c0 + i;
          if (gn >= P.N) break;
          float* cp = P.tC ? P.C + gn + (int64_t)gm * P.ldc : P.C + gm + (int64_t)gn * P.ldc;
          float o = alpha * v[i];
          if (beta != 0.f) o += beta * (*cp);
          *cp = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NT)
                 : "memory");
}

template <int NT, bool SPLIT>
constexpr int tc_smem_bytes() {
  return 2 * (SPLIT ? 2 : 1) * (stage_bytes(TC_M) + stage_bytes(NT));
}

template <int NT, bool SPLIT>
void tc_go(const GemmProbT<float>* pr, const GemmSegT<float>* sg, const int4* tl, int64_t nt,
           int* err, int stall, cudaStream_t s) {
  constexpr int smem = tc_smem_bytes<NT, SPLIT>();
  static std::once_flag once;
  std::call_once(once, [] {
    SPD_CUDA(cudaFuncSetAttribute(k_gemm_tf32<NT, SPLIT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  });
  for (int64_t b0 = 0; b0 < nt; b0 += 2147483647LL) {
    const unsigned g = (unsigned)std::min<int64_t>(nt - b0, 2147483647LL);
    k_gemm_tf32<NT, SPLIT><<<g, 128, smem, s>>>(pr, sg, tl + b0, err, stall);
    SPD_LAUNCHED();
  }
}

}  // namespace

// Tiles of the tensor-core kernel: 128 x 64 for a problem of at most 64 columns, 128 x 128
// otherwise (a choice of the problem alone, so that its arithmetic does not depend on the
// other problems of the launch).  The 64-column tiles come first, *n64_out of them.
std::vector<int4> tc_gemm_tiles(const std::vector<GemmProbT<float>>& probs, int* n64_out) {
  std::vector<int4> tiles;
  for (int pass = 0; pass < 2; ++pass) {
    for (int p = 0; p < (int)probs.size(); ++p) {
      const int nt = probs[p].N <= 64 ? 64 : 128;
      if ((nt == 64) != (pass == 0)) continue;
      for (int m0 = 0; m0 < probs[p].M; m0 += TC_M)
        for (int n0 = 0; n0 < probs[p].N; n0 += nt) tiles.push_back(make_int4(p, m0, n0, 0));
    }
    if (pass == 0) *n64_out = (int)tiles.size();
  }
  return tiles;
}

void tc_gemm_launch(const GemmProbT<float>* d_probs, const GemmSegT<float>* d_segs,
                    const int4* d_tiles, int64_t ntiles, int n64, bool split, int* d_err,
                    cudaStream_t s, int stall) {
  if (ntiles <= 0) return;
  if (n64 > 0) {
    if (split) tc_go<64, true>(d_probs, d_segs, d_tiles, n64, d_err, stall, s);
    else tc_go<64, false>(d_probs, d_segs, d_tiles, n64, d_err, stall, s);
  }
  if (ntiles > n64) {
    if (split) tc_go<128, true>(d_probs, d_segs, d_tiles + n64, ntiles - n64, d_err, stall, s);
    else tc_go<128, false>(d_probs, d_segs, d_tiles + n64, ntiles - n64, d_err, stall, s);
  }
}

int* tc_error_word() {
  static std::mutex mu;
  static int* words[128] = {nullptr};
  int dev = 0;
  SPD_CUDA(cudaGetDevice(&dev));
  SPD_REQUIRE(dev >= 0 && dev < 128, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!words[dev]) {
    SPD_CUDA(cudaMalloc(&words[dev], sizeof(int)));   // one word per device, kept
    SPD_CUDA(cudaMemset(words[dev], 0, sizeof(int)));
  }
  return words[dev];
}

void tc_check(cudaStream_t s) {
  int* w = tc_error_word();
  int h = 0;
  SPD_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPD_CUDA(cudaStreamSynchronize(s));
  if (h) {
    SPD_CUDA(cudaMemsetAsync(w, 0, sizeof(int), s));
    throw Error(SPDHSS_TIMEOUT, "tensor-core GEMM: an mbarrier wait gave up");
  }
}

}  // namespace spd

// One FP32 GEMM through the library's grouped GEMM (test and benchmark hook).
extern "C" spdhss_status spdhss_gemm_f32(int M, int N, int K, const float* A, int64_t lda,
                                         int tA, const float* B, int64_t ldb, int tB, float* C,
                                         int64_t ldc, float alpha, float beta, int mode,
                                         void* stream) {
  try {
    SPD_REQUIRE(M >= 1 && N >= 1 && K >= 0, "spdhss_gemm_f32: bad sizes");
    SPD_REQUIRE(C && (K == 0 || (A && B)), "spdhss_gemm_f32: NULL argument");
    SPD_REQUIRE(mode >= 0 && mode <= 3, "spdhss_gemm_f32: mode must be 0, 1, 2 or 3");
    SPD_REQUIRE(ldc >= M && lda >= (tA ? K : M) && ldb >= (tB ? N : K),
                "spdhss_gemm_f32: leading dimension too small");
    cudaStream_t s = (cudaStream_t)stream;
    spd::StreamScope ss(s);
    spd::GemmBatchT<float> g;
    g.tc = mode == 3 ? 2 : mode;
    g.tc_stall = mode == 3;
    g.tag = "gemm_f32";
    g.prob(C, ldc, M, N, alpha, beta);
    if (K > 0) g.seg(A, lda, tA, B, ldb, tB, K);
    g.run(s);
    spd::tc_check(s);
    return SPDHSS_OK;
  } catch (const spd::Error& e) {
    spd::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    spd::set_last_error(std::string("spdhss_gemm_f32: ") + e.what());
    return SPDHSS_ECUDA;
  }
}
