// Perturbative triples (Sec. II.A) on the tensor cores: the W contractions
//   W_ijk^abc += sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab
// of every ordering of P, as batched split-BF16 GEMMs on tcgen05.
//
// For one (i, j) and one ordering of P the contraction is a GEMM batched over
// k: rows m = (alpha, beta) (or (beta, alpha)) of v^2, columns n = gamma (v),
// and two K segments into the same accumulators:
//   segment 1 (K = d, v):  A1[m][d] = (beta d | alpha x), B1[n][d] = t_zy^{gamma d}
//   segment 2 (K = l, o):  A2[m][l] = t_xl^{alpha beta}, B2[n][l] = -(gamma z | y l)
// with (x, y, z) the ordering of (i, j, k).  The operands are the FP32
// integrals and amplitudes of the FP32 path, cut into three BF16 slices each
// (exact for FP32 inputs), K-major and zero-padded; a product is the sum of
// the six slice products p + q < 3, the hi*hi product in one TMEM accumulator
// and the five smaller ones in another (the tensor core's FP32 accumulation
// error scales with the accumulator it lands in).  The epilogue adds the two
// accumulators and writes (or adds) W[k][a][b][c] through the ordering's
// strides, as the CUDA-core path's kEpiAcc3 epilogue does.
//
// Warp roles (320 threads): warp 0 TMA producer, warp 1 MMA issuer, warps 2-9
// epilogue (two per TMEM lane quadrant).  Persistent: CTAs walk the work units
// (batch, 128-row tile); the accumulators are double-buffered in TMEM when
// both pairs fit (N <= 128 columns).
#include "kernels.h"
#include "tc_ptx.cuh"

namespace ladder {
namespace {
using namespace tc;

constexpr int kThreads = 320;
constexpr int kEpi = 256;
constexpr int kS = 3;                      // slices per operand
constexpr int kK1 = 32;                    // segment-1 K-step (64-byte rows)
constexpr int kK2 = 16;                    // segment-2 K-step (32-byte rows)
constexpr uint32_t kStageA = kS * 128u * kK1 * 2u;  // 24 KB
constexpr uint32_t kSmemBudget = 230400u;

__device__ __forceinline__ uint32_t desc_hi(uint32_t sbo_bytes, uint32_t layout) {
  return ((sbo_bytes >> 4) & 0x3FFFu) | (1u << 14) | (layout << 29);
}
__device__ __forceinline__ uint64_t desc64(uint32_t saddr, uint32_t hi) {
  return ((uint64_t)hi << 32) | (uint64_t)(((saddr >> 4) & 0x3FFFu) | (1u << 16));
}

struct DrainWatch {
  int zero = 0;
  Watchdog wd;
  __device__ DrainWatch(int *status, uint64_t deadline) : wd{status, &zero, deadline} {}
};

// slice products p + q < 3, hi*hi first
__device__ __forceinline__ constexpr int kPa(int q) { return q == 2 || q == 4 ? 1 : (q == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int kPb(int q) { return q == 1 || q == 4 ? 1 : (q == 3 ? 2 : 0); }

struct Bars {
  uint32_t base;
  int stages;
  __device__ uint32_t full(int s) const { return base + 8u * s; }
  __device__ uint32_t empty(int s) const { return base + 8u * (stages + s); }
  __device__ uint32_t cfull(int b) const { return base + 8u * (2 * stages + b); }
  __device__ uint32_t cfree(int b) const { return base + 8u * (2 * stages + 2 + b); }
  __device__ uint32_t done() const { return base + 8u * (2 * stages + 4); }
};

// Outer tensor index of an operand for batch b: fixed, or the batch itself.
__device__ __forceinline__ int outer(int fixed, int mul, int b) { return fixed + mul * b; }

__global__ void __launch_bounds__(kThreads, 1) tw_gemm_kernel(const __grid_constant__ TwArgs A) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  const uint32_t stageB = (uint32_t)kS * A.Nt * kK1 * 2u;
  const uint32_t kStage = (kStageA + stageB + 1023u) / 1024u * 1024u;
  const int stages = min(8, (int)(kSmemBudget / kStage));
  Bars bars{ring + kStage * stages, stages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + kStage * stages + 8 * (2 * stages + 5));
  int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nbuf = (4 * A.Nt <= 512) ? 2 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars.cfull(b), 1);
      mbar_init(bars.cfree(b), kEpi);
    }
    mbar_init(bars.done(), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const Watchdog wd{A.status, abort_flag, A.timeout_ns};
  const int mtiles = (A.M + 127) / 128;
  const int nunits = A.batch * mtiles;
  const int nk1 = A.K1p / kK1, nk2 = A.K2p / kK2;
  const int nks = A.nord * (nk1 + nk2);  // K steps of one unit over its orderings

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const int b = u / mtiles, m0 = (u % mtiles) * 128;
        for (int kq = 0; ok && kq < nks; ++kq) {
          if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
          const uint32_t dst = ring + (uint32_t)stage * kStage;
          const bool o2 = kq >= nk1 + nk2;  // the second ordering's segments
          const int ks = o2 ? kq - (nk1 + nk2) : kq;
          const int a1 = o2 ? outer(A.a1b_fix, A.a1b_mul, b) : outer(A.a1_fix, A.a1_mul, b);
          const int b1 = o2 ? outer(A.b1b_fix, A.b1b_mul, b) : outer(A.b1_fix, A.b1_mul, b);
          const int a2 = o2 ? a1 : outer(A.a2_fix, A.a2_mul, b), b2 = o2 ? b1 : outer(A.b2_fix, A.b2_mul, b);
          const bool seg1 = ks < nk1;
          const uint32_t bytes = seg1 ? (uint32_t)kS * (128u + A.Nt) * kK1 * 2u
                                      : (uint32_t)kS * (128u + A.Nt) * kK2 * 2u;
          mbar_arrive_expect_tx(bars.full(stage), bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          if (seg1) {
            tma_load_4d(dst, o2 ? &A.tmA1b : &A.tmA1, bars.full(stage), ks * kK1, m0, a1, 0);
            tma_load_4d(dst + kStageA, &A.tmB1, bars.full(stage), ks * kK1, 0, b1, 0);
          } else {
            const int k2 = ks - nk1;
            tma_load_4d(dst, o2 ? &A.tmA2b : &A.tmA2, bars.full(stage), k2 * kK2, m0, a2, 0);
            tma_load_4d(dst + kStageA, &A.tmB2, bars.full(stage), k2 * kK2, 0, b2, 0);
          }
          if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        DrainWatch dw(A.status, A.timeout_ns);
        for (int s = 0; s < stages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, g = 0;
      const uint32_t hi64 = desc_hi(512, kSwizzle64), hi32 = desc_hi(256, kSwizzle32);
      const uint32_t id = idesc_bf16(128, A.Nt);
      bool ok = true;
      for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
        const uint32_t buf = (uint32_t)(g % nbuf);
        if (!(ok = mbar_wait(bars.cfree(buf), ((g / nbuf) & 1u) ^ 1u, wd, kSiteXYFree))) break;
        tc_fence_after();
        const uint32_t d0 = tmem + buf * 256u;  // acc0 [0, Nt), acc1 [Nt, 2 Nt) of the buffer
        for (int kq = 0; ok && kq < nks; ++kq) {
          if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
          tc_fence_after();
          const uint32_t st = ring + (uint32_t)stage * kStage;
          const bool seg1 = (kq % (nk1 + nk2)) < nk1;
          const int kk_n = seg1 ? kK1 / 16 : 1;
          const uint32_t rowb = seg1 ? kK1 * 2u : kK2 * 2u;  // bytes per operand row
          const uint32_t hi = seg1 ? hi64 : hi32;
          for (int kk = 0; kk < kk_n; ++kk)
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const uint64_t ad = desc64(st + kPa(q) * 128u * rowb + kk * 32, hi);
              const uint64_t bd = desc64(st + kStageA + kPb(q) * A.Nt * rowb + kk * 32, hi);
              const bool first = kq == 0 && kk == 0 && q <= 1;
              mma_bf16(d0 + (q > 0 ? (uint32_t)A.Nt : 0u), ad, bd, id, first ? 0u : 1u);
            }
          mma_commit(bars.empty(stage));
          if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(bars.cfull(buf));
        ++g;
      }
      mma_commit(bars.done());
      DrainWatch dw(A.status, A.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ epilogue
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // 16-column groups 16 half + 32 k
    const int L = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    uint32_t g = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      const int b = u / mtiles, m = (u % mtiles) * 128 + L;
      const uint32_t buf = (uint32_t)(g % nbuf);
      if (!(ok = mbar_wait(bars.cfull(buf), (g / nbuf) & 1u, wd, kSiteRFull))) break;
      ++g;
      tc_fence_after();
      float *O = A.W + (long long)b * A.so_batch + (long long)(m / A.pv) * A.s1 + (long long)(m % A.pv) * A.s2;
      for (int c0 = 16 * half; c0 < A.Nt; c0 += 32) {
        float x[16], y[16];
        tmem_ld16(tl + buf * 256u + c0, x);
        tmem_ld16(tl + buf * 256u + A.Nt + c0, y);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) x[e] += y[e];
        if (m >= A.M) continue;
        float *w0 = O + (long long)c0 * A.s3;
        if (A.s3 == 1 && c0 + 16 <= A.N && (reinterpret_cast<uintptr_t>(w0) & 15u) == 0) {
          // the 16 columns are contiguous: four 16-byte accesses, loads first
          float4 *w4 = reinterpret_cast<float4 *>(w0);
          float4 old[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) old[h] = A.acc ? w4[h] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int h = 0; h < 4; ++h)
            w4[h] = make_float4(old[h].x + x[4 * h], old[h].y + x[4 * h + 1], old[h].z + x[4 * h + 2],
                                old[h].w + x[4 * h + 3]);
        } else {
          // every load of the group is issued before the first add, so the
          // read-modify-write costs one memory latency per 16 columns
          float old[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) old[e] = (A.acc && c0 + e < A.N) ? w0[(long long)e * A.s3] : 0.f;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < A.N) w0[(long long)e * A.s3] = old[e] + x[e];
        }
      }
      tc_fence_before();
      mbar_arrive(bars.cfree(buf));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// dst[s][g][r][k] = slice s of src(g, r, k) for r < rows_pad, k < K_pad (zero
// beyond rows, K), src(g, r, k) = src[g * sg + r * sr + k * sk]: the operand
// layouts of the W GEMMs (rows of one outer index g padded to rows_pad,
// K-major, K padded).  A value is cut into BF16 slices by rounding to
// nearest, each slice taking what the earlier ones leave (exact for FP32
// inputs with three slices).
__global__ void tw_slice_kernel(const float *__restrict__ src, long long sg, long long sr, long long sk, int G,
                                int rows, int rows_pad, int K, int K_pad, __nv_bfloat16 *__restrict__ dst) {
  const long long per = (long long)rows_pad * K_pad, n = (long long)G * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long g = e / per, rk = e % per;
    const int r = (int)(rk / K_pad), k = (int)(rk % K_pad);
    float x = (r < rows && k < K) ? src[g * sg + (long long)r * sr + (long long)k * sk] : 0.f;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      dst[s * n + e] = h;
      x -= __bfloat162float(h);
    }
  }
}

}  // namespace

uint32_t tw_smem_bytes(int Nt) {
  const uint32_t kStage = (kStageA + (uint32_t)kS * Nt * kK1 * 2u + 1023u) / 1024u * 1024u;
  const int stages = (int)(kSmemBudget / kStage) < 8 ? (int)(kSmemBudget / kStage) : 8;
  return kStage * stages + 256 + 1024;
}

cudaError_t tw_init_attributes() {
  return cudaFuncSetAttribute(tw_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tw_smem_bytes(256));
}

cudaError_t launch_tw_gemm(const TwArgs &a, int grid, cudaStream_t s) {
  tw_gemm_kernel<<<grid, kThreads, tw_smem_bytes(a.Nt), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tw_slice(const float *src, long long sg, long long sr, long long sk, int G, int rows,
                            int rows_pad, int K, int K_pad, __nv_bfloat16 *dst, cudaStream_t s) {
  const long long n = (long long)G * rows_pad * K_pad;
  const long long blocks = std::min<long long>((n + 255) / 256, 152 * 32);
  if (blocks > 0) tw_slice_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, sg, sr, sk, G, rows, rows_pad, K, K_pad, dst);
  return cudaGetLastError();
}

}  // namespace ladder
