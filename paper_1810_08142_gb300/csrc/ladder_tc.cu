// Split-BF16 fused ladder kernel on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
// R_ij^ab = sum_cd (ac|bd) tau_ij^cd (Eq. pp-Ladder-0) with (ac|bd) =
// sum_P B^P_ac B^P_bd (Eq. RIM), in the slot form of the symmetric /
// antisymmetric pair scheme (Sec. II.C): virtual indices in blocks of 8,
// block pairs k <= l, V+-_ab[(c,d)] = (ac|bd) +- (ad|bc), R+- = sum T+- V+-.
// Every operand x is carried as S bfloat16 slices x = x_0 + x_1 (+ x_2) and a
// product as the sum of the slice products x_p y_q with p + q < S.
//
// Accumulation.  The tensor core rounds its FP32 accumulator on every MMA
// instruction with a bias, so the error of one accumulator grows linearly
// with the number of MMAs that feed it.  Every FP32 accumulation chain here is
// therefore short, and chains are summed outside the tensor core:
//   GEMM1 (K = aux functions) runs in chains of `kc` K-steps; the
//         conversion warps sum the chains in registers (FP32, round to
//         nearest).  With `xy_split` the hi*hi slice product and the smaller
//         products go to separate accumulators: the error an MMA adds scales
//         with the accumulator it lands in, so the small products then cost
//         almost nothing and chains can be long; without it, chains alternate
//         between two TMEM buffers;
//   GEMM2 (K = slots) starts a fresh TMEM accumulator S every `s_pieces`
//         pieces of 16 slots (a block pair has 4);
//         the conversion warps add S into a TMEM running sum R (FP32, round to
//         nearest) and every `flush_every` S add R into a double-single
//         accumulator (an FP32 pair updated with TwoSum) in the workspace.
// A separate unpack kernel turns the accumulators into R_ij^ab in FP64.
//
// One CTA owns 128 virtual pairs (a in a 16-block, b in an 8-block), one
// chunk of occupied pairs (at most 128 TMEM columns) and one range of block
// pairs.  Warp roles:
//   warp 0    TMA producer: B slices (GEMM1 operands) and tau+- pieces into a
//             ring of shared-memory stages;
//   warp 1    MMA issuer (one thread): GEMM1 X[(a,c),(b,d)], Y[(a,d),(b,c)]
//             (M=128, N=64) and GEMM2 S+-[ab][lambda] = V+-[ab][slots]
//             T+-[lambda][slots]^T (M=128, N=lambda);
//   warps 2-9 conversion (two per TMEM lane quadrant, each owning half of the
//             columns: b = 0-3 or 4-7 of X and Y, every other 16 columns of S
//             and R): TMEM -> registers, exchange of Y within groups of 8
//             lanes by shuffles, V+- = X +- Y', BF16 slicing, swizzled stores
//             into the GEMM2 operand tile; S -> R sums; flushes.
// The integral tiles live only in TMEM, registers and shared memory.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace ladder {
namespace {
using namespace tc;

constexpr int kThreads = 320;   // warp 0 TMA, warp 1 MMA, warps 2-9 conversion
constexpr int kEpi = 256;       // two conversion warps per TMEM lane quadrant
constexpr int KSTEP = 32;                             // aux functions per GEMM1 stage
constexpr uint32_t A_TILE = 128u * KSTEP * 2u;        // 8 KB: rows (a,c), 64-byte rows
constexpr uint32_t B_TILE = 64u * KSTEP * 2u;         // 4 KB: rows (b,d)
constexpr int TPIECE = 16;                            // slots per tau+- stage (32-byte rows)
constexpr uint32_t V_TILE = 128u * SLOTS * 2u;        // 16 KB: 128 ab rows x 64 slots
constexpr uint32_t kColS = 256;                       // TMEM: XY0 [0,128), XY1 [128,256), S, R

// Shared memory of the fused kernel: a ring of TMA stages and the V+- tile
// (the GEMM2 operand).  The storing pass writes V+- straight to global
// memory, so its ring takes the whole budget.
template <int S, bool kStoreV>
struct Cfg {
  static constexpr uint32_t kStage = 12288u * S;      // S*(A_TILE+B_TILE) >= S*kTcMaxCols*32
  static constexpr int kStages = kStoreV ? (int)((232448u - 2048u) / kStage) : ((S == 2) ? 5 : 3);
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kV = kStoreV ? 0u : 2u * S * V_TILE;
  static constexpr uint32_t kBar = 256;
  static constexpr uint32_t kSmem = kRing + kV + kBar + 1024;
  static constexpr int kProducts = (S == 2) ? 3 : 6;
};
static_assert(12288u == A_TILE + B_TILE, "stage size");
static_assert(12288u >= kTcMaxCols * 32u, "tau stage size");
static_assert(kColS + 2 * kTcMaxCols <= 512, "TMEM columns");

// slice pairs (p, q) with p + q < S, larger terms first
__device__ __forceinline__ constexpr int kPa(int q) { return q == 2 || q == 4 ? 1 : (q == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int kPb(int q) { return q == 1 || q == 4 ? 1 : (q == 3 ? 2 : 0); }

// 8x8 transpose across the 8 lanes of a group: lane x holds row x on entry
// and column x on exit (three butterfly stages).
__device__ __forceinline__ void transpose8(float (&r)[8], int x) {
#pragma unroll
  for (int s = 1; s < 8; s <<= 1) {
    const bool up = (x & s) != 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j & s) continue;
      const float send = up ? r[j] : r[j ^ s];
      const float recv = __shfl_xor_sync(0xffffffffu, send, s);
      if (up)
        r[j] = recv;
      else
        r[j ^ s] = recv;
    }
  }
}

// Shared-memory descriptor from an address and a precomputed high word
// (stride byte offset, fixed bits, layout type; see sdesc).
__device__ __forceinline__ uint32_t desc_hi(uint32_t sbo_bytes, uint32_t layout) {
  return ((sbo_bytes >> 4) & 0x3FFFu) | (1u << 14) | (layout << 29);
}
__device__ __forceinline__ uint64_t desc64(uint32_t saddr, uint32_t hi) {
  return ((uint64_t)hi << 32) | (uint64_t)(((saddr >> 4) & 0x3FFFu) | (1u << 16));
}

// One BF16 slice of 8 values (round to nearest); `rem` keeps what is left.
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
  __device__ uint32_t v_full() const { return base + 8u * (2 * stages + 4); }
  __device__ uint32_t v_free() const { return base + 8u * (2 * stages + 5); }
  __device__ uint32_t s_full() const { return base + 8u * (2 * stages + 6); }
  __device__ uint32_t s_free() const { return base + 8u * (2 * stages + 7); }
  __device__ uint32_t done() const { return base + 8u * (2 * stages + 8); }
  static constexpr int kCount = 9;  // + 2 * stages
};

// A Watchdog that ignores the CTA's abort flag: used only to let copies and
// MMAs already in flight land before the CTA releases its resources.
struct DrainWatch {
  int zero = 0;
  Watchdog wd;
  __device__ DrainWatch(int *status, uint64_t deadline) : wd{status, &zero, deadline} {}
};

// Work item of the fused kernel: an (a 16-block, b 8-block) tile, an
// occupied-pair chunk and a range [p0, p1) of block pairs of one molecule.
struct Item {
  int tile, iA, jB, A0, B0, p0, p1;
  TcChunk CH;
  uint32_t sc;   // TMEM columns of S and of R (nps + nms)
  float2 *racc;  // this item's double-single accumulators, [col][lane]
};

__device__ __forceinline__ Item decode_item(const TcArgs &A, int item) {
  Item I;
  const int ksl = item % A.ksplit;
  const int tc = item / A.ksplit;
  const int tile = tc / A.nchunks, ch = tc % A.nchunks;
  int iA = 0, t = tile + A.tile0;  // tile0: first tile of the plan's range
  if (A.square) {
    iA = tile / A.nB8;
    t = tile % A.nB8 - 2 * iA;
  } else {
    while (t >= A.nB8 - 2 * iA) {
      t -= A.nB8 - 2 * iA;
      ++iA;
    }
  }
  I.tile = tile;
  I.iA = iA;
  I.jB = 2 * iA + t;
  I.A0 = iA * 16;
  I.B0 = I.jB * CB;
  I.CH = A.chunks[ch];
  I.p0 = (int)((long long)A.nbp * ksl / A.ksplit);
  I.p1 = (int)((long long)A.nbp * (ksl + 1) / A.ksplit);
  I.sc = (uint32_t)(I.CH.nps + I.CH.nms);
  I.racc = A.racc + (size_t)item * 128 * A.racc_cols;
  return I;
}

// The molecule's arguments and the local item index of global work unit `it`.
// A single-molecule launch reads its arguments straight from the launch
// parameters; a batch reads them from the device table.
template <bool kBatch>
__device__ __forceinline__ const TcArgs &item_args(const TcLaunch &Lp, int it, int &local) {
  if constexpr (!kBatch) {
    local = it;
    return Lp.one;
  } else {
    const int2 w = Lp.items[it];
    local = w.y;
    return Lp.mols[w.x];
  }
}

// Work units of the storing pass in range-major order: unit u takes
// block-pair range u / tiles of tile u % tiles, so the CTAs resident at one
// time work in one window of block pairs and share its B-slice panels in L2.
// (The storing pass keeps no accumulators, so any order gives the same
// result.)  Returns the slot that decode_item maps to (tile, range).
__device__ __forceinline__ int vstore_slot(const TcArgs &A, int u) {
  return (u % A.ntiles) * A.ksplit + u / A.ntiles;
}

template <int S, bool kBatch, bool kStoreV>
__global__ void __launch_bounds__(kThreads, 1) ladder_tc_kernel(const __grid_constant__ TcLaunch Lp) {
  using C = Cfg<S, kStoreV>;
  static_assert(C::kStages >= 3 && 8 * (2 * C::kStages + Bars::kCount) + 8 <= C::kBar, "ring");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  const uint32_t vbase = ring + C::kRing;
  Bars bars{vbase + C::kV, C::kStages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(
      smem + C::kRing + C::kV + 8 * (2 * C::kStages + Bars::kCount));
  int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars.cfull(b), 1);
      mbar_init(bars.cfree(b), kEpi);
    }
    mbar_init(bars.v_full(), kEpi);
    mbar_init(bars.v_free(), 1);
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
  // every role walks the same sequence of work items; barrier phases carry
  // over from one item to the next
  const int it0 = blockIdx.x, itstep = gridDim.x, nit = Lp.nitems;
  const TcArgs &A0args = kBatch ? Lp.mols[0] : Lp.one;
  const Watchdog wd{A0args.status, abort_flag, Lp.timeout_ns};

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_par = 0;  // per stage: armed at least once / parity armed last
      bool ok = true;
      for (int it = it0; ok && it < nit; it += itstep) {
        int local;
        const TcArgs &A = item_args<kBatch>(Lp, it, local);
        const Item I = decode_item(A, kStoreV ? vstore_slot(A, local) : local);
        const TcChunk &CH = I.CH;
        const int A0 = I.A0, B0 = I.B0, p0 = I.p0, p1 = I.p1;
        const uint32_t tbytes = I.sc * 32u;
        tma_prefetch_desc(&A.tmA);
        tma_prefetch_desc(&A.tmB);
        if (!kStoreV) {
          tma_prefetch_desc(&A.tmTp);
          tma_prefetch_desc(&A.tmTm);
        }
        for (int p = p0; ok && p <= p1; ++p) {
          if (p < p1) {
            int k, l;
            pair_of(p, k, l);
            const int ntile = (k == l) ? 1 : 2;
            for (int ks = 0; ok && ks < A.nks; ++ks)
              for (int tt = 0; tt < ntile; ++tt) {
                if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
                const uint32_t dst = ring + (uint32_t)stage * C::kStage;
                mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * (A_TILE + B_TILE));
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                const int ca = (tt == 0 ? k : l) * CB, cb = (tt == 0 ? l : k) * CB;
                // all S slices of each operand tile in one 4-D box
                tma_load_4d(dst, &A.tmA, bars.full(stage), ks * KSTEP, ca, A0, 0);
                tma_load_4d(dst + S * A_TILE, &A.tmB, bars.full(stage), ks * KSTEP, cb, B0, 0);
                if (++stage == C::kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
          }
          if (!kStoreV && ok && p > p0) {
            for (int piece = 0; piece < SLOTS / TPIECE; ++piece) {
              if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
              const uint32_t dst = ring + (uint32_t)stage * C::kStage;
              mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * tbytes);
              armed |= 1u << stage;
              armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
              const int x = (p - 1) * SLOTS + piece * TPIECE;
  #pragma unroll
              for (int s = 0; s < S; ++s) {
                for (int r = 0; r < CH.nps; r += 16)
                  tma_load_3d(dst + s * tbytes + r * 32, &A.tmTp, bars.full(stage), x, CH.lp0 + r, s);
                for (int r = 0; r < CH.nms; r += 16)
                  tma_load_3d(dst + s * tbytes + (CH.nps + r) * 32, &A.tmTm, bars.full(stage), x,
                              CH.lm0 + r, s);
              }
              if (++stage == C::kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
          }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA leaves
        DrainWatch dw(A0args.status, Lp.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t g = 0, v_use = 0, s_use = 0;  // chains issued, V tiles and S tiles consumed
      const uint32_t id1 = idesc_bf16(128, 64);
      const uint32_t hi64 = desc_hi(512, kSwizzle64), hi128 = desc_hi(1024, kSwizzle128),
                     hi32 = desc_hi(256, kSwizzle32);
      bool ok = true;
      for (int it = it0; ok && it < nit; it += itstep) {
        int local;
        const TcArgs &A = item_args<kBatch>(Lp, it, local);
        const Item I = decode_item(A, kStoreV ? vstore_slot(A, local) : local);
        const TcChunk &CH = I.CH;
        const int p0 = I.p0, p1 = I.p1;
        const uint32_t idp = idesc_bf16(128, CH.nps > 0 ? CH.nps : 16);
        const uint32_t idm = idesc_bf16(128, CH.nms > 0 ? CH.nms : 16);
        const uint32_t tbytes = I.sc * 32u;
        const int kc = A.kc;
        const int nch_full = (A.nks + kc - 1) / kc;
        const bool split = A.xy_split != 0;
        const uint32_t nbuf = (kStoreV || split) ? 1u : 2u;
        for (int p = p0; ok && p <= p1; ++p) {
          if (p < p1) {
            int k, l;
            pair_of(p, k, l);
            const int ntile = (k == l) ? 1 : 2;
            for (int c = 0; ok && c < nch_full; ++c) {
              const int buf = (int)(g % nbuf);
              if (!(ok = mbar_wait(bars.cfree(buf), ((g / nbuf) & 1u) ^ 1u, wd, kSiteXYFree))) break;
              tc_fence_after();
              const int ks0 = c * kc, ks1 = min(A.nks, ks0 + kc);
              for (int ks = ks0; ok && ks < ks1; ++ks)
                for (int tt = 0; tt < ntile; ++tt) {
                  // operands written by TMA and read by the MMA (both async
                  // proxy): the barrier's transaction count orders them
                  if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
                  const uint32_t st = ring + (uint32_t)stage * C::kStage;
                  if constexpr (kStoreV) {
                    // The S slices of B sit back to back (64 rows each), so
                    // slice p of A times slices 0..S-1-p of B is one MMA of
                    // N = 64 (S - p) at column offset 64 p: the products of
                    // slice order p + q land in the 64-column block p + q.
                    // Block 0 (hi*hi) is the large accumulator, blocks 1 and
                    // 2 the small ones; X at columns [0, 64 S), Y after it.
                    const uint32_t dT = tmem + (tt ? (uint32_t)(64 * S) : 0u);
  #pragma unroll
                    for (int kk = 0; kk < KSTEP / 16; ++kk)
  #pragma unroll
                      for (int pa = 0; pa < S; ++pa) {
                        const uint64_t ad = desc64(st + pa * A_TILE + kk * 32, hi64);
                        const uint64_t bd = desc64(st + S * A_TILE + kk * 32, hi64);
                        const bool first = (ks == ks0) && kk == 0 && pa == 0;
                        mma_bf16(dT + 64u * pa, ad, bd, idesc_bf16(128, 64 * (S - pa)), first ? 0u : 1u);
                      }
                  } else {
                    const uint32_t dT = tmem + (split ? 0u : (uint32_t)buf * 128u) + (tt ? 64u : 0u);
  #pragma unroll
                    for (int kk = 0; kk < KSTEP / 16; ++kk)
  #pragma unroll
                      for (int q = 0; q < C::kProducts; ++q) {
                        const uint64_t ad = desc64(st + kPa(q) * A_TILE + kk * 32, hi64);
                        const uint64_t bd = desc64(st + S * A_TILE + kPb(q) * B_TILE + kk * 32, hi64);
                        // split: the hi*hi product into the "big" accumulator,
                        // every smaller product into the "small" one (128 columns on)
                        const bool small = split && q > 0;
                        const bool first = (ks == ks0) && kk == 0 && (split ? (q <= 1) : (q == 0));
                        mma_bf16(dT + (small ? 128u : 0u), ad, bd, id1, first ? 0u : 1u);
                      }
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
          if (!kStoreV && p > p0) {
            if (!(ok = mbar_wait(bars.v_full(), v_use & 1u, wd, kSiteVFull))) break;
            tc_fence_after();
            for (int piece = 0; ok && piece < SLOTS / TPIECE; ++piece) {
              const bool first = (piece % A.s_pieces) == 0;
              if (first) {
                // a fresh S accumulator: the previous one has been taken
                if (!(ok = mbar_wait(bars.s_free(), (s_use & 1u) ^ 1u, wd, kSiteRFree))) break;
                tc_fence_after();
              }
              if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
              tc_fence_after();
              const uint32_t st = ring + (uint32_t)stage * C::kStage;
  #pragma unroll
              for (int q = 0; q < C::kProducts; ++q) {
                const uint32_t acc = (first && q == 0) ? 0u : 1u;
                const uint64_t ap = desc64(vbase + (0 * S + kPa(q)) * V_TILE + piece * 32, hi128);
                const uint64_t bp = desc64(st + kPb(q) * tbytes, hi32);
                mma_bf16(tmem + kColS, ap, bp, idp, acc);
                if (CH.nms > 0) {
                  const uint64_t am = desc64(vbase + (1 * S + kPa(q)) * V_TILE + piece * 32, hi128);
                  const uint64_t bm = desc64(st + kPb(q) * tbytes + CH.nps * 32, hi32);
                  mma_bf16(tmem + kColS + CH.nps, am, bm, idm, acc);
                }
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
            mma_commit(bars.v_free());
            ++v_use;
          }
        }
      }
      // every MMA of this CTA completes before TMEM is released
      mma_commit(bars.done());
      DrainWatch dw(A0args.status, Lp.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ conversion warps
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // which half of the columns this warp owns
    const int L = quad * 32 + lane;    // TMEM lane
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const int a_l = L >> 3, x_l = L & 7;
    const uint64_t pol = l2_evict_last_policy();
    uint32_t g = 0, v_use = 0, s_use = 0;
    bool ok = true;
    for (int it = it0; ok && it < nit; it += itstep) {
      int local;
      const TcArgs &A = item_args<kBatch>(Lp, it, local);
      const Item I = decode_item(A, kStoreV ? vstore_slot(A, local) : local);
      const int p0 = I.p0, p1 = I.p1;
      const uint32_t sc = I.sc;
      float2 *racc = I.racc;
      const int kc = A.kc;
      const int nch_full = (A.nks + kc - 1) / kc;
      const bool split = A.xy_split != 0;
      const uint32_t nbuf = (kStoreV || split) ? 1u : 2u;
      int nacc = 0, nflush = 0;
      // S (fresh GEMM2 result of one block pair) -> R (TMEM running sum, FP32)
      auto take_S = [&]() -> bool {
        if (!mbar_wait(bars.s_full(), s_use & 1u, wd, kSiteRFull)) return false;
        ++s_use;
        tc_fence_after();
        for (uint32_t c0 = 16u * half; c0 < sc; c0 += 32) {
          float s[16], r[16];
          tmem_ld16(tl + kColS + c0, s);
          if (nacc > 0) tmem_ld16(tl + kColS + sc + c0, r);
          tmem_ld_wait();
          if (nacc > 0) {
  #pragma unroll
            for (int u = 0; u < 16; ++u) s[u] += r[u];
          }
          tmem_st16(tl + kColS + sc + c0, s);
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(bars.s_free());
        ++nacc;
        return true;
      };
      // R (FP32, TMEM) -> double-single accumulator in the workspace, [col][lane]
      auto flush_R = [&]() {
        for (uint32_t c0 = 16u * half; c0 < sc; c0 += 32) {
          float r[16];
          tmem_ld16(tl + kColS + sc + c0, r);
          tmem_ld_wait();
          flush16_ds(racc + (size_t)c0 * 128 + L, r, nflush != 0, pol);
        }
        ++nflush;
        nacc = 0;
      };

      for (int p = p0; p < p1; ++p) {
        int k, l;
        pair_of(p, k, l);
        const bool diag = (k == l);
        float X[32], Y[32];  // columns (b, 0..7) for b in [4*half, 4*half+4)
        for (int c = 0; c < nch_full; ++c) {
          const int buf = (int)(g % nbuf);
          if (!(ok = mbar_wait(bars.cfull(buf), (g / nbuf) & 1u, wd, kSiteXYFull))) break;
          ++g;
          tc_fence_after();
          if constexpr (kStoreV) {
            // X = block 0 + (block 1 [+ block 2]) of the merged slice products
            const uint32_t cX = tl + 32u * half;
            const uint32_t cY = diag ? cX : cX + (uint32_t)(64 * S);
  #pragma unroll
            for (int q = 0; q < 2; ++q) {
  #pragma unroll
              for (int xy = 0; xy < 2; ++xy) {
                float b0[16], b1[16], b2[16];
                const uint32_t ca = (xy ? cY : cX) + q * 16;
                tmem_ld16(ca, b0);
                tmem_ld16(ca + 64u, b1);
                if (S == 3) tmem_ld16(ca + 128u, b2);
                tmem_ld_wait();
                float *dst = xy ? Y : X;
  #pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const float t = b0[i] + (S == 3 ? b1[i] + b2[i] : b1[i]);
                  dst[q * 16 + i] = c ? dst[q * 16 + i] + t : t;
                }
              }
            }
            tc_fence_before();
            mbar_arrive(bars.cfree(buf));
            continue;
          }
          const uint32_t cX = tl + (split ? 0u : (uint32_t)buf * 128u) + 32u * half;
          const uint32_t cY = diag ? cX : cX + 64u;
  #pragma unroll
          for (int q = 0; q < 2; ++q) {
            float tx[16], ty[16];
            tmem_ld16(cX + q * 16, tx);
            tmem_ld16(cY + q * 16, ty);
            if (split) {
              float sx[16], sy[16];
              tmem_ld16(cX + 128u + q * 16, sx);
              tmem_ld16(cY + 128u + q * 16, sy);
              tmem_ld_wait();
  #pragma unroll
              for (int i = 0; i < 16; ++i) {
                tx[i] += sx[i];
                ty[i] += sy[i];
              }
            } else {
              tmem_ld_wait();
            }
  #pragma unroll
            for (int i = 0; i < 16; ++i) {
              X[q * 16 + i] = c ? X[q * 16 + i] + tx[i] : tx[i];
              Y[q * 16 + i] = c ? Y[q * 16 + i] + ty[i] : ty[i];
            }
          }
          tc_fence_before();
          mbar_arrive(bars.cfree(buf));
        }
        if (!ok) break;
        // S chains of the previous block pair (GEMM2 runs after this pair's GEMM1)
        if (!kStoreV && p > p0) {
          for (int gs = 0; ok && gs < SLOTS / TPIECE / A.s_pieces; ++gs) {
            ok = take_S();
            if (ok && nacc >= A.flush_every) flush_R();
          }
          if (!ok) break;
        }
        // Y row of lane (a, d=x_l) holds (ad|bc) at column (b, c); after the
        // transpose lane (a, c=x_l) holds (ad|bc) at index (b, d).
  #pragma unroll
        for (int b = 0; b < 4; ++b) {
          float r[8];
  #pragma unroll
          for (int j = 0; j < 8; ++j) r[j] = Y[b * 8 + j];
          transpose8(r, x_l);
  #pragma unroll
          for (int j = 0; j < 8; ++j) Y[b * 8 + j] = r[j];
        }
        if constexpr (kStoreV) {
          // V+- slices straight to the planes [tile][pair][sign][slice][128
          // rows][64 slots]: a warp writes whole 128-byte rows
          // (lambda-only form: X and Y' themselves, no +- combination)
          __nv_bfloat16 *vp = A.Vst + (size_t)(I.tile * A.nbp + p) * 2 * S * (128 * SLOTS);
          const bool lam = A.lam_only != 0;
  #pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int row = a_l * 8 + 4 * half + b;
  #pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
              float rem[8];
  #pragma unroll
              for (int d = 0; d < 8; ++d)
                rem[d] = lam ? (sg ? Y[b * 8 + d] : X[b * 8 + d])
                             : (sg ? X[b * 8 + d] - Y[b * 8 + d] : X[b * 8 + d] + Y[b * 8 + d]);
  #pragma unroll
              for (int s = 0; s < S; ++s) {
                const uint4 w = pack_slice(rem);
                __stcs(reinterpret_cast<uint4 *>(vp + (size_t)(sg * S + s) * (128 * SLOTS) + row * SLOTS +
                                                 x_l * CB),
                       w);
              }
            }
          }
          continue;
        }
        if (!(ok = mbar_wait(bars.v_free(), (v_use & 1u) ^ 1u, wd, kSiteVFree))) break;
        ++v_use;
  #pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int row = a_l * 8 + 4 * half + b;
          const uint32_t off = (uint32_t)row * 128u + (uint32_t)((x_l ^ (row & 7)) * 16);
  #pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            float rem[8];
  #pragma unroll
            for (int d = 0; d < 8; ++d) rem[d] = sg ? X[b * 8 + d] - Y[b * 8 + d] : X[b * 8 + d] + Y[b * 8 + d];
  #pragma unroll
            for (int s = 0; s < S; ++s) {
              const uint4 w = pack_slice(rem);
              *reinterpret_cast<uint4 *>(smem + C::kRing + (uint32_t)(sg * S + s) * V_TILE + off) = w;
            }
          }
        }
        fence_async_smem();
        mbar_arrive(bars.v_full());
      }
      // S chains of the last block pair, then the final flush
      if (!kStoreV) {
        for (int gs = 0; ok && gs < SLOTS / TPIECE / A.s_pieces; ++gs) ok = take_S();
        if (ok) flush_R();
      }
    }
  }

  // ---- teardown: all roles done (or given up); release TMEM
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- unpack
// R_ij^ab from the accumulators of every block-pair range of a
// (tile, chunk): lane = ab slot (a = A0 + lane/8, b = B0 + lane%8),
//   R_ij^ab = R+ + R-, R_ij^ba = R+ - R-, R_ji^ba = R_ij^ab, R_ji^ab = R_ij^ba,
// with R- = 0 when i = j or a = b.  Every element of R is written once.
__global__ void __launch_bounds__(128) unpack_kernel(const __grid_constant__ TcLaunch Lp) {
  int tc;
  const TcArgs &A = Lp.mols ? Lp.mols[Lp.tcs[blockIdx.x].x] : Lp.one;
  tc = Lp.mols ? Lp.tcs[blockIdx.x].y : (int)blockIdx.x;
  const int tile = tc / A.nchunks, ch = tc % A.nchunks;
  int iA = 0, t = tile + A.tile0;
  while (t >= A.nB8 - 2 * iA) {
    t -= A.nB8 - 2 * iA;
    ++iA;
  }
  const int jB = 2 * iA + t;
  const TcChunk CH = A.chunks[ch];
  const int L = threadIdx.x;
  const int a = iA * 16 + (L >> 3), b = jB * CB + (L & 7);
  const bool diag_ab = (jB >> 1) == iA;
  if (!(a < A.v && b < A.v && (!diag_ab || a <= b))) return;
  const size_t per_item = (size_t)128 * A.racc_cols;
  const float2 *base = A.racc + (size_t)tc * A.ksplit * per_item + L;
  const size_t vv = (size_t)A.v * A.v, o = (size_t)A.o;
  int i = 0, j = 0;
  lam_plus(CH.lp0, i, j);
  for (int c = 0; c < CH.np; ++c) {
    // the ranges' partial sums added in double-single form, then widened once
    float2 ps = base[(size_t)c * 128], ms = make_float2(0.f, 0.f);
    for (int k = 1; k < A.ksplit; ++k) ps = ds_add2(ps, base[k * per_item + (size_t)c * 128]);
    if (i < j && a != b) {
      const int cm = CH.nps + (pneg(j) + i - CH.lm0);
      for (int k = 0; k < A.ksplit; ++k) ms = ds_add2(ms, base[k * per_item + (size_t)cm * 128]);
    }
    const double pv = ds_value(ps), mv = ds_value(ms);
    A.R[(i * o + j) * vv + (size_t)a * A.v + b] = pv + mv;
    A.R[(i * o + j) * vv + (size_t)b * A.v + a] = pv - mv;
    A.R[(j * o + i) * vv + (size_t)b * A.v + a] = pv + mv;
    A.R[(j * o + i) * vv + (size_t)a * A.v + b] = pv - mv;
    if (++i > j) {
      ++j;
      i = 0;
    }
  }
}

// ---------------------------------------------------------------- GEMM2 from stored V+-
// Second pass of the two-pass form.  The store mode of the fused kernel has
// written the V+- slices of every (tile, block pair) to global memory, as
// planes [tile][pair][sign][slice] of 128 ab rows x 64 slots.  This kernel
// contracts them with tau+- for one chunk of up to kTcMaxColsV occupied
// pairs of one sign (lambda+ or lambda-), so each MMA is N = the chunk's
// columns wide and only that sign's planes are read; GEMM1 thus runs once per
// tile instead of once per chunk.
// Accumulation: a fresh FP32 accumulator S every s_pieces pieces (as in the
// fused kernel), double-buffered in TMEM so that the next pieces' MMAs run
// while the conversion warps take the last S; the running FP32 sum R lives in
// the conversion warps' registers and is added into the accumulators in
// the workspace every flush_every S.
//   warp 0    TMA: per 16-slot piece, the S V planes of the sign (one 3-D box) and the
//             chunk's tau+- rows (one bulk copy from the chunk-major copy);
//   warp 1    MMA issuer: S+-[ab][lambda] (+)= V+-[ab][piece] T+-[lambda][piece]^T;
//   warps 2-9 S -> R (registers) and flushes; lane = ab row, each warp
//             owns every other group of 16 columns.
constexpr uint32_t VP_PLANE = 128u * TPIECE * 2u;  // 4 KB: 128 ab rows x 16 slots
constexpr uint32_t kColS1 = 256;                   // TMEM: S0 [0, 192), S1 [256, 448)
constexpr int kGroupsV = kTcMaxColsV / 32;         // 16-column groups per conversion warp
constexpr int kPPS = 2;                            // 16-slot pieces per TMA stage
static_assert(kPPS == 2, "the lambda-only form puts its two planes where the two pieces go");

template <int S>
struct Cfg2 {
  static constexpr uint32_t kV1 = (uint32_t)S * VP_PLANE;  // V planes of one piece
  static constexpr uint32_t kV = kPPS * kV1;
  static constexpr uint32_t kT = (uint32_t)kPPS * S * kTcMaxColsV * 32u;
  static constexpr uint32_t kStage = (kV + kT + 1023u) / 1024u * 1024u;
  static constexpr int kStages = (230400u / kStage) < 10u ? (int)(230400u / kStage) : 10;  // <= 225 KB
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kSmem = kRing + 256 + 1024;
  static constexpr int kProducts = (S == 2) ? 3 : 6;
};
static_assert(kColS1 + kTcMaxColsV <= 512, "TMEM columns of the GEMM2 kernel");
static_assert(kTcMaxColsV % 32 == 0, "column groups");
static_assert(8 * (2 * 10 + Bars::kCount) + 8 <= 256, "barrier area");

// Work units of the GEMM2 kernel in range-major order: unit u takes block-pair
// range u / (tiles * chunks) of (tile, chunk) u % (tiles * chunks), so the CTAs
// resident at one time share one window of block pairs (and with it the
// tau+- rows and V+- planes they read from L2).  Returns the accumulator
// slot of the unit, which decode_item maps to (tile, chunk, range).
__device__ __forceinline__ int gemm2_slot(const TcArgs &A, int u) {
  const int tcs = A.ntiles * A.nchunks;
  return (u % tcs) * A.ksplit + u / tcs;
}

template <int S, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1) ladder_gemm2_kernel(const __grid_constant__ TcLaunch Lp) {
  using C = Cfg2<S>;
  static_assert(C::kStages >= 3 && C::kStages <= 10, "ring depth");
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

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bars.cfull(b), 1);     // S buffer b holds a finished accumulator
      mbar_init(bars.cfree(b), kEpi);  // S buffer b has been taken
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
  const int it0 = blockIdx.x, itstep = gridDim.x, nit = Lp.nitems;
  const TcArgs &A0args = kBatch ? Lp.mols[0] : Lp.one;
  const Watchdog wd{A0args.status, abort_flag, Lp.timeout_ns};
  constexpr int kPieces = SLOTS / TPIECE;

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t armed = 0, armed_par = 0;
      bool ok = true;
      for (int it = it0; ok && it < nit; it += itstep) {
        int local;
        const TcArgs &A = item_args<kBatch>(Lp, it, local);
        const Item I = decode_item(A, gemm2_slot(A, local));
        tma_prefetch_desc(&A.tmVl);
        const TcChunk &CH = I.CH;
        const uint32_t tbytes = I.sc * 32u;
        const int sg = CH.nps > 0 ? 0 : 1;  // the chunk's sign
        // a stage holds kPPS pieces of the chunk's sign, or (lambda-only) one
        // piece of both planes; the bytes are the same
        const bool lam = A.lam_only != 0;
        const int pstep = lam ? 1 : kPPS;
        for (int p = I.p0; ok && p < I.p1; ++p) {
          const int zb = (I.tile * A.nbp + p) * A.nsign;
          for (int piece = 0; piece < kPieces; piece += pstep) {
            if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
            const uint32_t dst = ring + (uint32_t)stage * C::kStage;
            mbar_arrive_expect_tx(bars.full(stage), C::kV + (uint32_t)(kPPS * S) * tbytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            // (default L2 policy for both: marking the tau+- copy evict-last
            // or the V+- planes evict-first measured slower)
            for (int j = 0; j < kPPS; ++j)
              tma_load_3d(dst + j * C::kV1, &A.tmVl, bars.full(stage), (lam ? piece : piece + j) * TPIECE, 0,
                          (zb + (lam ? j : sg)) * S);
            // the chunk's tau rows of these pieces, every slice: one bulk copy
            bulk_load(dst + C::kV, A.T2 + CH.t2off + (size_t)(p * kPieces + piece) * (lam ? 2 : 1) * S * tbytes,
                      (uint32_t)(kPPS * S) * tbytes, bars.full(stage));
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        DrainWatch dw(A0args.status, Lp.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, g = 0;  // g: S accumulators started
      const uint32_t hi32 = desc_hi(256, kSwizzle32);
      bool ok = true;
      for (int it = it0; ok && it < nit; it += itstep) {
        int local;
        const TcArgs &A = item_args<kBatch>(Lp, it, local);
        const Item I = decode_item(A, gemm2_slot(A, local));
        const uint32_t id = idesc_bf16(128, (int)I.sc);
        const uint32_t tbytes = I.sc * 32u;
        const bool lam = A.lam_only != 0;
        const int pstep = lam ? 1 : kPPS;
        for (int p = I.p0; ok && p < I.p1; ++p)
          for (int piece0 = 0; ok && piece0 < kPieces; piece0 += pstep) {
            if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
            const uint32_t st = ring + (uint32_t)stage * C::kStage;
            for (int j = 0; ok && j < kPPS; ++j) {
              // lambda-only: j is the plane (X by tau^cd, Y' by tau^dc) of one piece
              const int piece = lam ? piece0 : piece0 + j;
              const bool first = (piece % A.s_pieces) == 0 && (!lam || j == 0);
              const uint32_t buf = g & 1u;
              if (first) {
                if (!(ok = mbar_wait(bars.cfree(buf), ((g >> 1) & 1u) ^ 1u, wd, kSiteRFree))) break;
                tc_fence_after();
              }
              const uint32_t dS = tmem + buf * kColS1;
              const uint32_t sv = st + j * C::kV1, stt = st + C::kV + (uint32_t)(j * S) * tbytes;
#pragma unroll
              for (int q = 0; q < C::kProducts; ++q)
                mma_bf16(dS, desc64(sv + (uint32_t)kPa(q) * VP_PLANE, hi32), desc64(stt + kPb(q) * tbytes, hi32),
                         id, (first && q == 0) ? 0u : 1u);
              if ((piece + 1) % A.s_pieces == 0 && (!lam || j == kPPS - 1)) {
                mma_commit(bars.cfull(buf));
                ++g;
              }
            }
            if (!ok) break;
            mma_commit(bars.empty(stage));
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
      }
      mma_commit(bars.done());
      DrainWatch dw(A0args.status, Lp.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ S -> R -> accumulators
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int L = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    uint32_t g = 0;
    bool ok = true;
    const uint64_t pol = l2_evict_last_policy();
    float R[kGroupsV * 16];
    for (int it = it0; ok && it < nit; it += itstep) {
      int local;
      const TcArgs &A = item_args<kBatch>(Lp, it, local);
      const Item I = decode_item(A, gemm2_slot(A, local));
      const int sc = (int)I.sc;
      const int ng = (sc - 16 * half + 31) / 32;  // this warp's groups: columns 16*half + 32*k
      float2 *racc = I.racc + L;
      int nacc = 0, nflush = 0;
#pragma unroll
      for (int u = 0; u < kGroupsV * 16; ++u) R[u] = 0.f;
      const int ntake = (I.p1 - I.p0) * (kPieces / A.s_pieces);
      for (int t = 0; ok && t < ntake; ++t) {
        const uint32_t buf = g & 1u;
        if (!(ok = mbar_wait(bars.cfull(buf), (g >> 1) & 1u, wd, kSiteRFull))) break;
        ++g;
        tc_fence_after();
        const uint32_t cS = tl + buf * kColS1 + 16u * half;
#pragma unroll
        for (int k = 0; k < kGroupsV; k += 2) {
          float a[16], b[16];
          if (k < ng) tmem_ld16(cS + 32u * k, a);
          if (k + 1 < ng) tmem_ld16(cS + 32u * (k + 1), b);
          tmem_ld_wait();
          if (k < ng) {
#pragma unroll
            for (int u = 0; u < 16; ++u) R[k * 16 + u] += a[u];
          }
          if (k + 1 < ng) {
#pragma unroll
            for (int u = 0; u < 16; ++u) R[(k + 1) * 16 + u] += b[u];
          }
        }
        tc_fence_before();
        mbar_arrive(bars.cfree(buf));
        if (++nacc >= A.flush_every || t + 1 == ntake) {
#pragma unroll
          for (int k = 0; k < kGroupsV; ++k)
            if (k < ng) flush16_ds(racc + (size_t)(16 * half + 32 * k) * 128, &R[k * 16], nflush != 0, pol);
#pragma unroll
          for (int u = 0; u < kGroupsV * 16; ++u) R[u] = 0.f;
          ++nflush;
          nacc = 0;
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

// ---------------------------------------------------------------- unpack (two-pass)
// R_ij^ab from the accumulators of the GEMM2 pass, whose chunks hold
// lambda+ columns [c wplus, (c+1) wplus) or lambda- columns [c wminus, ...):
// block (tile, plus chunk c) writes every (i <= j) of that lambda+ range,
// taking R- from the minus chunk of lambda- = j(j-1)/2 + i.  Lane = ab slot,
// as in unpack_kernel; every element of R is written once.
__global__ void __launch_bounds__(128) unpack2_kernel(const __grid_constant__ TcLaunch Lp) {
  // a batch lists its blocks as (molecule, block of that molecule) in tcs
  const TcArgs &A = Lp.mols ? Lp.mols[Lp.tcs[blockIdx.x].x] : Lp.one;
  const int blk = Lp.mols ? Lp.tcs[blockIdx.x].y : (int)blockIdx.x;
  const int tile = blk / A.nplus, cp = blk % A.nplus;
  int iA = 0, t = tile + A.tile0;
  while (t >= A.nB8 - 2 * iA) {
    t -= A.nB8 - 2 * iA;
    ++iA;
  }
  const int jB = 2 * iA + t;
  const int L = threadIdx.x;
  const int a = iA * 16 + (L >> 3), b = jB * CB + (L & 7);
  const bool diag_ab = (jB >> 1) == iA;
  if (!(a < A.v && b < A.v && (!diag_ab || a <= b))) return;
  const size_t per_item = (size_t)128 * A.racc_cols;
  // work item (tile, chunk, range k) sits at ((tile * nchunks + chunk) * ksplit + k)
  const float2 *base = A.racc + (size_t)tile * A.nchunks * A.ksplit * per_item + L;
  const size_t vv = (size_t)A.v * A.v, o = (size_t)A.o;
  const TcChunk CH = A.chunks[cp];
  int i = 0, j = 0;
  lam_plus(CH.lp0, i, j);
  for (int c = 0; c < CH.np; ++c) {
    // the ranges' partial sums added in double-single form, then widened once
    const float2 *bp = base + ((size_t)cp * A.ksplit) * per_item + (size_t)c * 128;
    float2 ps = bp[0], ms = make_float2(0.f, 0.f);
    for (int k = 1; k < A.ksplit; ++k) ps = ds_add2(ps, bp[k * per_item]);
    if (i < j && a != b) {
      const int lm = pneg(j) + i;
      const int cm = A.nplus + lm / A.wminus;
      const float2 *bm = base + ((size_t)cm * A.ksplit) * per_item + (size_t)(lm % A.wminus) * 128;
      for (int k = 0; k < A.ksplit; ++k) ms = ds_add2(ms, bm[k * per_item]);
    }
    const double pv = ds_value(ps), mv = ds_value(ms);
    A.R[(i * o + j) * vv + (size_t)a * A.v + b] = pv + mv;
    A.R[(i * o + j) * vv + (size_t)b * A.v + a] = pv - mv;
    A.R[(j * o + i) * vv + (size_t)b * A.v + a] = pv + mv;
    A.R[(j * o + i) * vv + (size_t)a * A.v + b] = pv - mv;
    if (++i > j) {
      ++j;
      i = 0;
    }
  }
}

// ---------------------------------------------------------------- unpack (lambda-only)
// One block per (tile, chunk) of the lambda-only form; lane = ab slot with
// a <= b.  Column c of the chunk is the ordered pair ij = lp0 + c, and
//   R_ij^ab = sum over the block-pair ranges,  R_ji^ba = R_ij^ab,
// which writes every element of R once (a = b is written from ij and ji).
__global__ void __launch_bounds__(128) unpack_lam_kernel(const __grid_constant__ TcLaunch Lp) {
  const TcArgs &A = Lp.one;
  const int tc = blockIdx.x, tile = tc / A.nchunks, ch = tc % A.nchunks;
  int iA = 0, t = tile + A.tile0;
  while (t >= A.nB8 - 2 * iA) {
    t -= A.nB8 - 2 * iA;
    ++iA;
  }
  const int jB = 2 * iA + t;
  const int L = threadIdx.x;
  const int a = iA * 16 + (L >> 3), b = jB * CB + (L & 7);
  const bool diag_ab = (jB >> 1) == iA;
  if (!(a < A.v && b < A.v && (!diag_ab || a <= b))) return;
  const size_t per_item = (size_t)128 * A.racc_cols;
  const float2 *base = A.racc + (size_t)tc * A.ksplit * per_item + L;
  const size_t vv = (size_t)A.v * A.v, o = (size_t)A.o;
  const TcChunk CH = A.chunks[ch];
  for (int c = 0; c < CH.np; ++c) {
    const float2 *bp = base + (size_t)c * 128;
    float2 acc = bp[0];
    for (int k = 1; k < A.ksplit; ++k) acc = ds_add2(acc, bp[k * per_item]);
    const size_t ij = (size_t)CH.lp0 + c, i = ij / o, j = ij % o;
    const double val = ds_value(acc);
    A.R[(i * o + j) * vv + (size_t)a * A.v + b] = val;
    A.R[(j * o + i) * vv + (size_t)b * A.v + a] = val;
  }
}

// ---------------------------------------------------------------- unpack (two-pass dB)
// dB[P][x][y] = 2 x the block-range sums of the GEMM2 kernel's accumulators
// for tile (x 16-block, y 8-block) and aux chunk; lane = (x, y).
__global__ void __launch_bounds__(128) grad_unpack2_kernel(const __grid_constant__ TcLaunch Lp, double *dB,
                                                           int N) {
  const TcArgs &A = Lp.one;
  const int tc = blockIdx.x, tile = tc / A.nchunks, ch = tc % A.nchunks;
  const int L = threadIdx.x;
  const int x = (tile / A.nB8) * 16 + (L >> 3), y = (tile % A.nB8) * CB + (L & 7);
  if (x >= A.v || y >= A.v) return;
  const TcChunk CH = A.chunks[ch];
  const size_t per_item = (size_t)128 * A.racc_cols;
  const float2 *base = A.racc + (size_t)tc * A.ksplit * per_item + L;
  for (int c = 0; c < CH.np && CH.lp0 + c < N; ++c) {
    float2 acc = base[(size_t)c * 128];
    for (int k = 1; k < A.ksplit; ++k) acc = ds_add2(acc, base[k * per_item + (size_t)c * 128]);
    dB[((size_t)(CH.lp0 + c) * A.v + x) * A.v + y] = 2.0 * ds_value(acc);
  }
}

}  // namespace

cudaError_t launch_grad_unpack2(const TcLaunch &a, double *dB, int N, int nblocks, cudaStream_t s) {
  grad_unpack2_kernel<<<nblocks, 128, 0, s>>>(a, dB, N);
  return cudaGetLastError();
}

uint32_t tc_smem_bytes(int nslices) {
  return nslices == 2 ? Cfg<2, false>::kSmem : Cfg<3, false>::kSmem;
}

template <int S>
static cudaError_t set_smem_attrs() {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(ladder_tc_kernel<S, false, false>, at, (int)Cfg<S, false>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ladder_tc_kernel<S, true, false>, at, (int)Cfg<S, false>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ladder_tc_kernel<S, false, true>, at, (int)Cfg<S, true>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ladder_tc_kernel<S, true, true>, at, (int)Cfg<S, true>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(ladder_gemm2_kernel<S, false>, at, (int)Cfg2<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(ladder_gemm2_kernel<S, true>, at, (int)Cfg2<S>::kSmem);
  return e;
}

cudaError_t tc_init_attributes(int nslices) {
  return nslices == 2 ? set_smem_attrs<2>() : set_smem_attrs<3>();
}

cudaError_t launch_ladder_tc(const TcLaunch &a, int nslices, int grid, cudaStream_t s) {
  const bool batch = a.mols != nullptr;
  if (nslices == 2) {
    if (batch)
      ladder_tc_kernel<2, true, false><<<grid, kThreads, Cfg<2, false>::kSmem, s>>>(a);
    else
      ladder_tc_kernel<2, false, false><<<grid, kThreads, Cfg<2, false>::kSmem, s>>>(a);
  } else {
    if (batch)
      ladder_tc_kernel<3, true, false><<<grid, kThreads, Cfg<3, false>::kSmem, s>>>(a);
    else
      ladder_tc_kernel<3, false, false><<<grid, kThreads, Cfg<3, false>::kSmem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_ladder_vstore(const TcLaunch &a, int nslices, int grid, cudaStream_t s) {
  const bool batch = a.mols != nullptr;
  if (nslices == 2) {
    if (batch)
      ladder_tc_kernel<2, true, true><<<grid, kThreads, Cfg<2, true>::kSmem, s>>>(a);
    else
      ladder_tc_kernel<2, false, true><<<grid, kThreads, Cfg<2, true>::kSmem, s>>>(a);
  } else {
    if (batch)
      ladder_tc_kernel<3, true, true><<<grid, kThreads, Cfg<3, true>::kSmem, s>>>(a);
    else
      ladder_tc_kernel<3, false, true><<<grid, kThreads, Cfg<3, true>::kSmem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_ladder_gemm2(const TcLaunch &a, int nslices, int grid, cudaStream_t s) {
  const bool batch = a.mols != nullptr;
  if (nslices == 2) {
    if (batch)
      ladder_gemm2_kernel<2, true><<<grid, kThreads, Cfg2<2>::kSmem, s>>>(a);
    else
      ladder_gemm2_kernel<2, false><<<grid, kThreads, Cfg2<2>::kSmem, s>>>(a);
  } else {
    if (batch)
      ladder_gemm2_kernel<3, true><<<grid, kThreads, Cfg2<3>::kSmem, s>>>(a);
    else
      ladder_gemm2_kernel<3, false><<<grid, kThreads, Cfg2<3>::kSmem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(const TcLaunch &a, int nblocks, cudaStream_t s) {
  unpack_kernel<<<nblocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_unpack_lam(const TcLaunch &a, int nblocks, cudaStream_t s) {
  if (nblocks > 0) unpack_lam_kernel<<<nblocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_unpack2(const TcLaunch &a, int nblocks, cudaStream_t s) {
  unpack2_kernel<<<nblocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ladder

namespace ladder {
namespace {
// One warp waits, with the library's bounded wait, on an mbarrier that
// nothing ever arrives at; the wait gives up after `timeout_ns`, records
// `site` in the status word and the kernel returns normally.
__global__ void selftest_wait_kernel(int *status, unsigned long long timeout_ns, int site) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    tc::mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const tc::Watchdog wd{status, &abort_flag, timeout_ns};
    tc::mbar_wait(b, 0, wd, site);
  }
  __syncthreads();
}
}  // namespace

cudaError_t launch_selftest_wait(int *status, unsigned long long timeout_ns, int site,
                                 cudaStream_t s) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(status, timeout_ns, site);
  return cudaGetLastError();
}
}  // namespace ladder
