// Split-BF16 gradient of E = sum W_ij^ab R_ij^ab with respect to the RI
// factor, on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
//   dB^P_xy = 2 sum_{b,d} Gamma^{xb}_{yd} B^P_bd,
//   Gamma^{xb}_{yd} = sum_ij W_ij^{xb} tau_ij^{yd}
// (the two terms of the derivative of Eq. RIM inside Eq. pp-Ladder-0 are equal
// under the pair symmetry of W and tau, Sec. II.C).
//
// One CTA owns 128 output pairs (x in a 16-block, y in an 8-block), one chunk
// of up to 128 auxiliary functions, and loops over all (b, d) blocks of 8 x 8:
//   Gamma2[(x,b),(y,d)] = sum_ij Wt[(x,b)][ij] taut[(y,d)][ij]   (M=128, N=64,
//       K = o^2; K-major BF16 slices; hi*hi and smaller products in separate
//       TMEM accumulators);
//   the lane holding (x,b) writes row (x,y), K-chunk b of the Gamma operand
//       (128 x 64 slots, BF16 slices, 128-byte swizzle) -- no exchange needed;
//   S[(x,y)][P] = Gamma[(x,y)][(b,d)] Bs[P][(b,d)]^T  (M=128, N=P chunk, K=16
//       slots per piece) into a fresh TMEM accumulator, summed by the
//       conversion warps into a TMEM running sum and flushed to FP64.
// Accumulation chains are short for the same reason as in the forward kernel
// (the tensor core's FP32 accumulation error grows with the MMAs per
// accumulator).  An unpack kernel writes dB = 2 x the double-single sums.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace ladder {
namespace {
using namespace tc;

constexpr int kThreads = 320;
constexpr int kEpi = 256;
constexpr int KSTEP = 32;                        // occupied pairs per Gamma2 stage
constexpr uint32_t A_TILE = 128u * KSTEP * 2u;   // 8 KB: rows (x,b)
constexpr uint32_t B_TILE = 64u * KSTEP * 2u;    // 4 KB: rows (y,d)
constexpr int TPIECE = 16;                       // slots per B^P piece (32-byte rows)
constexpr uint32_t G_TILE = 128u * SLOTS * 2u;   // 16 KB: 128 (x,y) rows x 64 slots
constexpr uint32_t kColS = 256;                  // TMEM: Gamma2 [0,256), S, R

template <int S>
struct Cfg {
  static constexpr uint32_t kStage = 12288u * S;
  static constexpr int kStages = (S == 2) ? 6 : 4;
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kG = (uint32_t)S * G_TILE;
  static constexpr uint32_t kBar = 256;
  static constexpr uint32_t kSmem = kRing + kG + kBar + 1024;
  static constexpr int kProducts = (S == 2) ? 3 : 6;
};
static_assert(12288u >= kGradTcPChunk * 32u * 1u, "B^P stage size");

__device__ __forceinline__ constexpr int kPa(int q) { return q == 2 || q == 4 ? 1 : (q == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int kPb(int q) { return q == 1 || q == 4 ? 1 : (q == 3 ? 2 : 0); }

__device__ __forceinline__ uint32_t desc_hi(uint32_t sbo_bytes, uint32_t layout) {
  return ((sbo_bytes >> 4) & 0x3FFFu) | (1u << 14) | (layout << 29);
}
__device__ __forceinline__ uint64_t desc64(uint32_t saddr, uint32_t hi) {
  return ((uint64_t)hi << 32) | (uint64_t)(((saddr >> 4) & 0x3FFFu) | (1u << 16));
}

__device__ __forceinline__ uint4 pack_slice(float (&rem)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(rem[2 * h], rem[2 * h + 1]);
    const float2 back = __bfloat1622float2(b2);
    rem[2 * h] -= back.x;
    rem[2 * h + 1] -= back.y;
    w[h] = *reinterpret_cast<const uint32_t *>(&b2);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

struct Bars {
  uint32_t base;
  int stages;
  __device__ uint32_t full(int s) const { return base + 8u * s; }
  __device__ uint32_t empty(int s) const { return base + 8u * (stages + s); }
  __device__ uint32_t cfull(int b) const { return base + 8u * (2 * stages + b); }
  __device__ uint32_t cfree(int b) const { return base + 8u * (2 * stages + 2 + b); }
  __device__ uint32_t g_full() const { return base + 8u * (2 * stages + 4); }
  __device__ uint32_t g_free() const { return base + 8u * (2 * stages + 5); }
  __device__ uint32_t s_full() const { return base + 8u * (2 * stages + 6); }
  __device__ uint32_t s_free() const { return base + 8u * (2 * stages + 7); }
  __device__ uint32_t done() const { return base + 8u * (2 * stages + 8); }
  static constexpr int kCount = 9;
};

struct DrainWatch {
  int zero = 0;
  Watchdog wd;
  __device__ DrainWatch(int *status, uint64_t deadline) : wd{status, &zero, deadline} {}
};

template <int S>
__global__ void __launch_bounds__(kThreads, 1) grad_B_tc_kernel(const __grid_constant__ GradTcArgs A) {
  using C = Cfg<S>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  const uint32_t gbase = ring + C::kRing;
  Bars bars{gbase + C::kG, C::kStages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(
      smem + C::kRing + C::kG + 8 * (2 * C::kStages + Bars::kCount));
  int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  // work item: (x 16-block, y 8-block) tile and chunk of auxiliary functions
  const int item = blockIdx.x;
  const int pc = item % A.npc, tile = item / A.npc;
  const int X0 = (tile / A.nY8) * 16, Y0 = (tile % A.nY8) * CB;
  const int P0 = pc * kGradTcPChunk;
  const uint32_t ncol = (uint32_t)min(kGradTcPChunk, A.Np - P0);  // multiple of 16
  const int nb = A.vp / CB, nq = nb * nb;                          // (b, d) blocks
  float2 *racc = A.racc + (size_t)item * 128 * kGradTcPChunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars.cfull(b), 1);
      mbar_init(bars.cfree(b), kEpi);
    }
    mbar_init(bars.g_full(), kEpi);
    mbar_init(bars.g_free(), 1);
    mbar_init(bars.s_full(), 1);
    mbar_init(bars.s_free(), kEpi);
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
  const int kc = A.kc;
  const int nch = (A.nks + kc - 1) / kc;  // Gamma2 chains per block

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&A.tmW);
      tma_prefetch_desc(&A.tmT);
      tma_prefetch_desc(&A.tmBs);
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      const uint32_t bbytes = ncol * 32u;  // one slice of a B^P piece
      bool ok = true;
      for (int q = 0; ok && q <= nq; ++q) {
        if (q < nq) {
          const int Bb0 = (q / nb) * CB, Dd0 = (q % nb) * CB;
          for (int ks = 0; ok && ks < A.nks; ++ks) {
            if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
            const uint32_t dst = ring + (uint32_t)stage * C::kStage;
            mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * (A_TILE + B_TILE));
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
#pragma unroll
            for (int s = 0; s < S; ++s) {
              tma_load_3d(dst + s * A_TILE, &A.tmW, bars.full(stage), ks * KSTEP, Bb0, s * A.vp + X0);
              tma_load_3d(dst + S * A_TILE + s * B_TILE, &A.tmT, bars.full(stage), ks * KSTEP, Dd0,
                          s * A.vp + Y0);
            }
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (ok && q > 0) {
          const int Bb0 = ((q - 1) / nb) * CB, Dd0 = ((q - 1) % nb) * CB;
          for (int piece = 0; piece < SLOTS / TPIECE; ++piece) {
            if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
            const uint32_t dst = ring + (uint32_t)stage * C::kStage;
            mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * bbytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
#pragma unroll
            for (int s = 0; s < S; ++s)
              for (uint32_t r = 0; r < ncol; r += 16)
                tma_load_3d(dst + s * bbytes + r * 32, &A.tmBs, bars.full(stage),
                            (Bb0 + 2 * piece) * CB, Dd0 / CB, s * A.Np + P0 + (int)r);
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        DrainWatch dw(A.status, A.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, g = 0, g_use = 0, s_use = 0;
      const uint32_t id1 = idesc_bf16(128, 64);
      const uint32_t id2 = idesc_bf16(128, (int)ncol);
      const uint32_t hi64 = desc_hi(512, kSwizzle64), hi128 = desc_hi(1024, kSwizzle128),
                     hi32 = desc_hi(256, kSwizzle32);
      const uint32_t bbytes = ncol * 32u;
      bool ok = true;
      for (int q = 0; ok && q <= nq; ++q) {
        if (q < nq) {
          for (int c = 0; ok && c < nch; ++c) {
            const int buf = (int)(g & 1u);
            if (!(ok = mbar_wait(bars.cfree(buf), ((g >> 1) & 1u) ^ 1u, wd, kSiteXYFree))) break;
            tc_fence_after();
            const int ks0 = c * kc, ks1 = min(A.nks, ks0 + kc);
            for (int ks = ks0; ok && ks < ks1; ++ks) {
              if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
              tc_fence_after();
              const uint32_t st = ring + (uint32_t)stage * C::kStage;
              const uint32_t dT = tmem + (uint32_t)buf * 128u;
#pragma unroll
              for (int kk = 0; kk < KSTEP / 16; ++kk)
#pragma unroll
                for (int qq = 0; qq < C::kProducts; ++qq) {
                  const uint64_t ad = desc64(st + kPa(qq) * A_TILE + kk * 32, hi64);
                  const uint64_t bd = desc64(st + S * A_TILE + kPb(qq) * B_TILE + kk * 32, hi64);
                  // hi*hi product into the large accumulator, the rest 64 columns on
                  const bool small = qq > 0;
                  const bool first = (ks == ks0) && kk == 0 && qq <= 1;
                  mma_bf16(dT + (small ? 64u : 0u), ad, bd, id1, first ? 0u : 1u);
                }
              mma_commit(bars.empty(stage));
              if (++stage == C::kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
            if (!ok) break;
            mma_commit(bars.cfull(buf));
            ++g;
          }
          if (!ok) break;
        }
        if (q > 0) {
          if (!(ok = mbar_wait(bars.g_full(), g_use & 1u, wd, kSiteVFull))) break;
          tc_fence_after();
          for (int piece = 0; ok && piece < SLOTS / TPIECE; ++piece) {
            const bool first = (piece % A.s_pieces) == 0;
            if (first) {
              if (!(ok = mbar_wait(bars.s_free(), (s_use & 1u) ^ 1u, wd, kSiteRFree))) break;
              tc_fence_after();
            }
            if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
            tc_fence_after();
            const uint32_t st = ring + (uint32_t)stage * C::kStage;
#pragma unroll
            for (int qq = 0; qq < C::kProducts; ++qq) {
              const uint64_t ap = desc64(gbase + kPa(qq) * G_TILE + piece * 32, hi128);
              const uint64_t bp = desc64(st + kPb(qq) * bbytes, hi32);
              mma_bf16(tmem + kColS, ap, bp, id2, (first && qq == 0) ? 0u : 1u);
            }
            mma_commit(bars.empty(stage));
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
            if ((piece + 1) % A.s_pieces == 0) {
              mma_commit(bars.s_full());
              ++s_use;
            }
          }
          if (!ok) break;
          mma_commit(bars.g_free());
          ++g_use;
        }
      }
      mma_commit(bars.done());
      DrainWatch dw(A.status, A.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ conversion warps
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // y in [4*half, 4*half+4)
    const int L = quad * 32 + lane;    // TMEM lane
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const int x_l = L >> 3, b_l = L & 7;
    const uint64_t pol = l2_evict_last_policy();
    uint32_t g = 0, g_use = 0, s_use = 0;
    int nacc = 0, nflush = 0;
    bool ok = true;

    auto take_S = [&]() -> bool {
      if (!mbar_wait(bars.s_full(), s_use & 1u, wd, kSiteRFull)) return false;
      ++s_use;
      tc_fence_after();
      for (uint32_t c0 = 16u * half; c0 < ncol; c0 += 32) {
        float sv[16], r[16];
        tmem_ld16(tl + kColS + c0, sv);
        if (nacc > 0) tmem_ld16(tl + kColS + ncol + c0, r);
        tmem_ld_wait();
        if (nacc > 0) {
#pragma unroll
          for (int u = 0; u < 16; ++u) sv[u] += r[u];
        }
        tmem_st16(tl + kColS + ncol + c0, sv);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(bars.s_free());
      ++nacc;
      return true;
    };
    auto flush_R = [&]() {
      for (uint32_t c0 = 16u * half; c0 < ncol; c0 += 32) {
        float r[16];
        tmem_ld16(tl + kColS + ncol + c0, r);
        tmem_ld_wait();
        flush16_ds(racc + (size_t)c0 * 128 + L, r, nflush != 0, pol);
      }
      ++nflush;
      nacc = 0;
    };

    for (int q = 0; q < nq; ++q) {
      float X[32];  // Gamma2 row of lane (x, b): columns (y, d) for y in this half
      for (int c = 0; c < nch; ++c) {
        const int buf = (int)(g & 1u);
        if (!(ok = mbar_wait(bars.cfull(buf), (g >> 1) & 1u, wd, kSiteXYFull))) break;
        ++g;
        tc_fence_after();
        const uint32_t cX = tl + (uint32_t)buf * 128u + 32u * half;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float tb[16], ts[16];
          tmem_ld16(cX + h * 16, tb);
          tmem_ld16(cX + 64u + h * 16, ts);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) X[h * 16 + i] = c ? X[h * 16 + i] + (tb[i] + ts[i]) : tb[i] + ts[i];
        }
        tc_fence_before();
        mbar_arrive(bars.cfree(buf));
      }
      if (!ok) break;
      if (q > 0) {
        for (int gs = 0; ok && gs < SLOTS / TPIECE / A.s_pieces; ++gs) {
          ok = take_S();
          if (ok && nacc >= A.flush_every) flush_R();
        }
        if (!ok) break;
      }
      if (!(ok = mbar_wait(bars.g_free(), (g_use & 1u) ^ 1u, wd, kSiteVFree))) break;
      ++g_use;
      // row (x, y) of the Gamma operand, K-chunk b = this lane's b: 8 slots d
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int row = x_l * 8 + 4 * half + y;
        const uint32_t off = (uint32_t)row * 128u + (uint32_t)((b_l ^ (row & 7)) * 16);
        float rem[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) rem[d] = X[y * 8 + d];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const uint4 w = pack_slice(rem);
          *reinterpret_cast<uint4 *>(smem + C::kRing + (uint32_t)s * G_TILE + off) = w;
        }
      }
      fence_async_smem();
      mbar_arrive(bars.g_full());
    }
    for (int gs = 0; ok && gs < SLOTS / TPIECE / A.s_pieces; ++gs) ok = take_S();
    if (ok) flush_R();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- two-pass dB, storing pass
// Gamma^{xb}_{yd} of every (x 16-block, y 8-block) tile and (b, d) block,
// computed once (Gamma2 as above, K = occupied pairs) and stored as S bf16
// slices in the layout of the GEMM2 kernel's first operand: plane
// ((tile * nq + q) * S + s), 128 rows (x, y) x 64 slots (b, d).  The
// contraction with B^P then runs in that kernel over aux chunks of up to 192,
// without recomputing Gamma per chunk.  A work unit is a tile and a range of
// (b, d) blocks (no accumulator depends on the grouping).
template <int S>
struct CfgG {
  static constexpr uint32_t kStage = 12288u * S;
  static constexpr int kStages = (int)((230400u) / kStage);
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kBar = 256;
  static constexpr uint32_t kSmem = kRing + kBar + 1024;
  static constexpr int kProducts = (S == 2) ? 3 : 6;
};

template <int S>
__global__ void __launch_bounds__(kThreads, 1) grad_gamma_store_kernel(const __grid_constant__ GradTcArgs A) {
  using C = CfgG<S>;
  static_assert(8 * (2 * C::kStages + Bars::kCount) + 8 <= C::kBar, "barrier area");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  Bars bars{ring + C::kRing, C::kStages};
  uint32_t *tmem_holder =
      reinterpret_cast<uint32_t *>(smem + C::kRing + 8 * (2 * C::kStages + Bars::kCount));
  int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  const int nb = A.vp / CB, nq = nb * nb;
  const int item = blockIdx.x;
  const int tile = item / A.qsplit, r = item % A.qsplit;
  const int q0 = (int)((long long)nq * r / A.qsplit), q1 = (int)((long long)nq * (r + 1) / A.qsplit);
  const int X0 = (tile / A.nY8) * 16, Y0 = (tile % A.nY8) * CB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
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
  const int kc = A.kc;
  const int nch = (A.nks + kc - 1) / kc;

  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_desc(&A.tmW);
      tma_prefetch_desc(&A.tmT);
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      bool ok = true;
      for (int q = q0; ok && q < q1; ++q) {
        const int Bb0 = (q / nb) * CB, Dd0 = (q % nb) * CB;
        for (int ks = 0; ok && ks < A.nks; ++ks) {
          if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
          const uint32_t dst = ring + (uint32_t)stage * C::kStage;
          mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * (A_TILE + B_TILE));
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            tma_load_3d(dst + s * A_TILE, &A.tmW, bars.full(stage), ks * KSTEP, Bb0, s * A.vp + X0);
            tma_load_3d(dst + S * A_TILE + s * B_TILE, &A.tmT, bars.full(stage), ks * KSTEP, Dd0,
                        s * A.vp + Y0);
          }
          if (++stage == C::kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        DrainWatch dw(A.status, A.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, g = 0;
      const uint32_t hi64 = desc_hi(512, kSwizzle64);
      bool ok = true;
      for (int q = q0; ok && q < q1; ++q)
        for (int c = 0; ok && c < nch; ++c) {
          const int buf = (int)(g & 1u);
          if (!(ok = mbar_wait(bars.cfree(buf), ((g >> 1) & 1u) ^ 1u, wd, kSiteXYFree))) break;
          tc_fence_after();
          const int ks0 = c * kc, ks1 = min(A.nks, ks0 + kc);
          for (int ks = ks0; ok && ks < ks1; ++ks) {
            if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
            const uint32_t st = ring + (uint32_t)stage * C::kStage;
            // merged slice products (as in the forward storing pass): slice
            // pa of W times tau slices 0..S-1-pa, back to back in shared
            // memory, is one MMA of N = 64 (S - pa) at column 64 pa, so the
            // products of slice order pa + qb land in 64-column block pa + qb
            // (block 0 = hi*hi, the large accumulator); buffers at 0 and 256
            const uint32_t dT = tmem + (uint32_t)buf * 256u;
#pragma unroll
            for (int kk = 0; kk < KSTEP / 16; ++kk)
#pragma unroll
              for (int pa = 0; pa < S; ++pa) {
                const uint64_t ad = desc64(st + pa * A_TILE + kk * 32, hi64);
                const uint64_t bd = desc64(st + S * A_TILE + kk * 32, hi64);
                const bool first = (ks == ks0) && kk == 0 && pa == 0;
                mma_bf16(dT + 64u * pa, ad, bd, idesc_bf16(128, 64 * (S - pa)), first ? 0u : 1u);
              }
            mma_commit(bars.empty(stage));
            if (++stage == C::kStages) {
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
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // y in [4*half, 4*half+4)
    const int L = quad * 32 + lane;    // TMEM lane = (x, b)
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const int x_l = L >> 3, b_l = L & 7;
    uint32_t g = 0;
    bool ok = true;
    for (int q = q0; ok && q < q1; ++q) {
      float X[32];  // Gamma2 row of lane (x, b): columns (y, d) for y in this half
      for (int c = 0; c < nch; ++c) {
        const int buf = (int)(g & 1u);
        if (!(ok = mbar_wait(bars.cfull(buf), (g >> 1) & 1u, wd, kSiteXYFull))) break;
        ++g;
        tc_fence_after();
        const uint32_t cX = tl + (uint32_t)buf * 256u + 32u * half;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float b0[16], b1[16], b2[16];
          tmem_ld16(cX + h * 16, b0);
          tmem_ld16(cX + 64u + h * 16, b1);
          if (S == 3) tmem_ld16(cX + 128u + h * 16, b2);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float t = b0[i] + (S == 3 ? b1[i] + b2[i] : b1[i]);
            X[h * 16 + i] = c ? X[h * 16 + i] + t : t;
          }
        }
        tc_fence_before();
        mbar_arrive(bars.cfree(buf));
      }
      if (!ok) break;
      // row (x, y) of plane (tile, q, s), slots (b_l, 0..7): whole 128-byte rows per warp
      __nv_bfloat16 *gp = A.Gst + (size_t)(tile * nq + q) * S * (128 * SLOTS);
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int row = x_l * 8 + 4 * half + y;
        float rem[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) rem[d] = X[y * 8 + d];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const uint4 w = pack_slice(rem);
          __stcs(reinterpret_cast<uint4 *>(gp + (size_t)s * (128 * SLOTS) + row * SLOTS + b_l * CB), w);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// dB[P][x][y] = 2 x the double-single sum of work unit (tile, chunk); lane = (x, y).
__global__ void __launch_bounds__(128) grad_unpack_kernel(const __grid_constant__ GradTcArgs A) {
  const int item = blockIdx.x;
  const int pc = item % A.npc, tile = item / A.npc;
  const int L = threadIdx.x;
  const int x = (tile / A.nY8) * 16 + (L >> 3), y = (tile % A.nY8) * CB + (L & 7);
  if (x >= A.v || y >= A.v) return;
  const float2 *src = A.racc + (size_t)item * 128 * kGradTcPChunk + L;
  const int P0 = pc * kGradTcPChunk;
  const int n = min(kGradTcPChunk, A.N - P0);
  for (int c = 0; c < n; ++c)
    A.dB[((size_t)(P0 + c) * A.v + x) * A.v + y] = 2.0 * ds_value(src[(size_t)c * 128]);
}

}  // namespace

cudaError_t grad_tc_init_attributes(int nslices) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if (nslices == 2) {
    e = cudaFuncSetAttribute(grad_B_tc_kernel<2>, at, (int)Cfg<2>::kSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(grad_gamma_store_kernel<2>, at, (int)CfgG<2>::kSmem);
  } else {
    e = cudaFuncSetAttribute(grad_B_tc_kernel<3>, at, (int)Cfg<3>::kSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(grad_gamma_store_kernel<3>, at, (int)CfgG<3>::kSmem);
  }
  return e;
}

cudaError_t launch_grad_gamma_store(const GradTcArgs &a, int nslices, cudaStream_t s) {
  const int items = a.ntiles * a.qsplit;
  if (nslices == 2)
    grad_gamma_store_kernel<2><<<items, kThreads, CfgG<2>::kSmem, s>>>(a);
  else
    grad_gamma_store_kernel<3><<<items, kThreads, CfgG<3>::kSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grad_B_tc(const GradTcArgs &a, int nslices, cudaStream_t s) {
  const int items = a.ntiles * a.npc;
  if (nslices == 2)
    grad_B_tc_kernel<2><<<items, kThreads, Cfg<2>::kSmem, s>>>(a);
  else
    grad_B_tc_kernel<3><<<items, kThreads, Cfg<3>::kSmem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grad_unpack_kernel<<<items, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ladder
