// Error-free split-BF16 ladder (LADDER_OZAKI): the two-pass form of the
// tensor-core path with an error-free splitting of every operand, after the
// scheme of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), so that
// R and E_L come out with FP64-class accuracy from BF16 tensor-core products.
//
// R_ij^ab = sum_cd (ac|bd) tau_ij^cd (Eq. pp-Ladder-0), (ac|bd) = sum_P
// B^P_ac B^P_bd (Eq. RIM), in the slot form of the symmetric / antisymmetric
// pair scheme (Sec. II.C) used by the other tensor-core kernels: virtual
// indices in blocks of 8, block pairs k <= l, V+-_ab[(c,d)] = (ac|bd) +-
// (ad|bc), R+- = sum T+- V+-.
//
// Splitting.  A row x of an operand (the K index running along it) is held as
// S slices of fixed-point numbers under one power-of-two scale per row:
//   x = scale * sum_s x_s 2^(-8 s),  x_0 in [-256, 256], x_s in [-129, 129],
// each x_s an integer, stored as the BF16 number x_s 2^(-8 s) (exact: at most
// 8 significant bits).  A product of slices p and q is exact in FP32 and is an
// integer multiple of 2^(-8 (p + q)) below 2^16 of that unit.
//
// Accumulation.  The tensor core rounds its FP32 accumulator with a bias, so a
// sum of products is exact only while every partial sum is representable.  A
// TMEM accumulator here receives products of one slice order p + q only
// (orders 0, 1 and 2 each in their own, orders >= 3 together, 2^-24 below the
// result where rounding no longer matters), over an exactness window short
// enough that its partial sums stay below 2^24 units:
//   GEMM1 (K = aux functions): windows of 128 (4 K-steps of 32); every row of
//         B has one scale over all P, so windows add without rescaling;
//   GEMM2 (K = slots): one block pair (64 slots) per window; V+- and tau+-
//         rows have one scale per block pair, applied when the window's four
//         accumulators are drained.
// The conversion warps drain each window's four accumulators into a
// double-single sum (an FP32 pair kept with TwoSum, about 48 bits).
//
// Pass 1 (oz_vstore_kernel): per (ab tile, block pair): X = (ac|bd) and
// Y = (ad|bc) windows alternate between two TMEM halves (X drains while Y's
// MMAs run); at the end V+- = X +- Y' (Y transposed across lanes), cut into S
// fixed-point slices with one scale per (ab row, block pair), stored to the
// workspace with their scales.  Pass 2 (oz_gemm2_kernel): per (tile, chunk of
// <= 128 occupied pairs of one sign, block-pair range): the S x S slice
// products of every 16-slot piece with p + q < S, issued and drained by order
// group so that draining one group overlaps the MMAs of the others.  The unpack kernel of the two-pass form then writes R.
//
// Warp roles (576 threads): warp 0 TMA producer, warp 1 MMA issuer (one
// thread), warps 2-17 conversion (four per TMEM lane quadrant, each owning a
// quarter of the columns).
#include <algorithm>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace ladder {
namespace {
using namespace tc;

constexpr int kThreads = 576;
constexpr int kEpi = 512;
constexpr int KSTEP = 32;                             // aux functions per GEMM1 stage
constexpr uint32_t A_TILE = 128u * KSTEP * 2u;        // 8 KB: rows (a,c), 64-byte rows
constexpr uint32_t B_TILE = 64u * KSTEP * 2u;         // 4 KB: rows (b,d)
constexpr int TPIECE = 16;                            // slots per GEMM2 piece
constexpr uint32_t VP_PLANE = 128u * TPIECE * 2u;     // 4 KB: 128 ab rows x 16 slots
constexpr uint32_t kSmemBudget = 230400u;             // ring bytes available per CTA

// round to the nearest integer (ties to even) for |x| <= 2^22, on the FP32 pipe
__device__ __forceinline__ float rint_small(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Two FP32 lanes per instruction (add / sub / mul .f32x2, sm_100 and later),
// each lane rounded to nearest exactly like the scalar instruction.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
// two_sum on two lanes at once
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// (H, L) += (h, l) and (H, L) += x, two accumulators at once (as ds_acc)
__device__ __forceinline__ void ds_acc2(float2 &H, float2 &L, float2 h, float2 l) {
  float2 s, e;
  two_sum2(H, h, s, e);
  H = s;
  L = add2(L, add2(l, e));
}
__device__ __forceinline__ void ds_add2(float2 &H, float2 &L, float2 x) {
  float2 s, e;
  two_sum2(H, x, s, e);
  H = s;
  L = add2(L, e);
}

// One exactness window of pass 1 into the double-single sums of 16 columns,
// two columns per f32x2 instruction.  The window's value comes from its four
// order accumulators g0..g3 (TMEM columns cbase + 64 g) as a double-single
// (h, l) with |l| <= ulp(h) / 2.  In units of the order-0 products:
// h0 + e = g0 + g1 exactly (TwoSum); e is a multiple of 2^-8 below 1/2 and g2
// a multiple of 2^-16 below 2^7, so e + g2 is exact in FP32; the TwoSum with
// h0 then leaves a remainder of at most ulp(h) / 2, to which the tail orders
// (2^-24 below h) are added with a rounding 2^-48 below h.  (Adding g2
// straight into the low word would round it 2^-40 below h.)  (h, l) then goes
// into the running sum as ds_acc2 does.
__device__ __forceinline__ void drain_window(uint32_t cbase, float2 (&acc)[16]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float g0[4], g1[4], g2[4], g3[4];
    const uint32_t c0 = cbase + 4u * h;
    tmem_ld4(c0, g0);
    tmem_ld4(c0 + 64u, g1);
    tmem_ld4(c0 + 128u, g2);
    tmem_ld4(c0 + 192u, g3);
    tmem_ld_wait();
#pragma unroll
    for (int e = 0; e < 4; e += 2) {
      float2 h0, er, hh, ll;
      two_sum2(make_float2(g0[e], g0[e + 1]), make_float2(g1[e], g1[e + 1]), h0, er);
      two_sum2(h0, add2(er, make_float2(g2[e], g2[e + 1])), hh, ll);
      ll = add2(ll, make_float2(g3[e], g3[e + 1]));
      float2 H = make_float2(acc[4 * h + e].x, acc[4 * h + e + 1].x);
      float2 L = make_float2(acc[4 * h + e].y, acc[4 * h + e + 1].y);
      ds_acc2(H, L, hh, ll);
      acc[4 * h + e] = make_float2(H.x, L.x);
      acc[4 * h + e + 1] = make_float2(H.y, L.y);
    }
  }
}

// 2^e as a float for -126 <= e <= 127
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Exponent E with m < 2^E for m > 0 (m finite, normal).
__device__ __forceinline__ int exp_above(float m) { return ((__float_as_int(m) >> 23) & 0xff) - 126; }

// 8x8 transpose across the 8 lanes of a group (lane x holds row x on entry,
// column x on exit).
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

// Work unit (tile, chunk, range) as in the other tensor-core kernels: tile =
// (a 16-block iA, b 8-block jB >= 2 iA), range [p0, p1) of block pairs.
struct Item {
  int tile, ch, A0, B0, p0, p1;
  TcChunk CH;
  float2 *racc;
};
__device__ __forceinline__ Item decode(const OzArgs &A, int slot, int nchunks) {
  Item I;
  const int ksl = slot % A.ksplit;
  const int tc = slot / A.ksplit;
  const int tile = tc / nchunks;
  I.ch = tc % nchunks;
  int iA = 0, t = tile + A.tile0;  // tile0: first tile of the plan's range
  while (t >= A.nB8 - 2 * iA) {
    t -= A.nB8 - 2 * iA;
    ++iA;
  }
  I.tile = tile;
  I.A0 = iA * 16;
  I.B0 = (2 * iA + t) * CB;
  I.CH = A.chunks[I.ch];
  I.p0 = (int)((long long)A.nbp * ksl / A.ksplit);
  I.p1 = (int)((long long)A.nbp * (ksl + 1) / A.ksplit);
  I.racc = A.racc ? A.racc + (size_t)slot * 128 * A.racc_cols : nullptr;
  return I;
}

// The molecule's arguments and the local unit index of work unit u: a single
// molecule reads them from the launch parameters, a batch from its device table.
template <bool kBatch>
__device__ __forceinline__ const OzArgs &oz_args(const OzLaunch &Lp, int u, int &local) {
  if constexpr (!kBatch) {
    local = u;
    return Lp.one;
  } else {
    const int2 w = Lp.items[u];
    local = w.y;
    return Lp.mols[w.x];
  }
}
// Pass 1 units walk range-major (unit u: range u / tiles of tile u % tiles) so
// the resident CTAs share B panels in L2; pass 2 likewise over (tile, chunk).
__device__ __forceinline__ int vstore_slot(const OzArgs &A, int u) {
  return (u % A.ntiles) * A.ksplit + u / A.ntiles;
}
__device__ __forceinline__ int gemm2_slot(const OzArgs &A, int u) {
  const int tcs = A.ntiles * A.nchunks;
  return (u % tcs) * A.ksplit + u / tcs;
}

struct Bars {
  uint32_t base;
  int stages;
  __device__ uint32_t full(int s) const { return base + 8u * s; }
  __device__ uint32_t empty(int s) const { return base + 8u * (stages + s); }
  __device__ uint32_t cfull(int b) const { return base + 8u * (2 * stages + b); }
  __device__ uint32_t cfree(int b) const { return base + 8u * (2 * stages + 3 + b); }
  __device__ uint32_t done() const { return base + 8u * (2 * stages + 6); }
  static constexpr int kCount = 7;  // + 2 * stages
};

template <int S>
struct Cfg1 {
  static constexpr uint32_t kStage = (uint32_t)S * (A_TILE + B_TILE);
  static constexpr int kStages = (int)(kSmemBudget / kStage);
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kSmem = kRing + 256 + 1024;
};
template <int S>
struct Cfg2 {
  static constexpr uint32_t kStage = (uint32_t)S * (VP_PLANE + kOzMaxCols * 32u);
  static constexpr int kStages = (int)(kSmemBudget / kStage) < 8 ? (int)(kSmemBudget / kStage) : 8;
  static constexpr uint32_t kRing = kStage * kStages;
  static constexpr uint32_t kSmem = kRing + 256 + 1024;
};

// V+- = X +- Y' of one ab row (double-single, renormalised; this lane holds
// the 8 slots (c = x_l, d = 0..7) of it in Xj and Yj, two columns per f32x2
// instruction), then per sign the row's scale (a power of two above the
// largest of its 64 slots, taken over the 8 lanes x_l) and the S fixed-point
// slices, stored to the row of the stored planes.
template <int S>
__device__ __forceinline__ void vpm_store(const float2 *Xj, const float2 *Yj, __nv_bfloat16 *vbase, float *sbase,
                                          int row, int x_l) {
  float2 Vp[8], Vm[8];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const float2 xh = make_float2(Xj[e].x, Xj[e + 1].x), xl = make_float2(Xj[e].y, Xj[e + 1].y);
    const float2 yh = make_float2(Yj[e].x, Yj[e + 1].x), yl = make_float2(Yj[e].y, Yj[e + 1].y);
    float2 sm, er, hi, lo;
    two_sum2(xh, yh, sm, er);
    two_sum2(sm, add2(add2(xl, yl), er), hi, lo);
    Vp[e] = make_float2(hi.x, lo.x);
    Vp[e + 1] = make_float2(hi.y, lo.y);
    two_sum2(xh, mul2(yh, make_float2(-1.f, -1.f)), sm, er);
    two_sum2(sm, add2(sub2(xl, yl), er), hi, lo);
    Vm[e] = make_float2(hi.x, lo.x);
    Vm[e + 1] = make_float2(hi.y, lo.y);
  }
#pragma unroll
  for (int sg = 0; sg < 2; ++sg) {
    const float2 *V = sg ? Vm : Vp;
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) m = fmaxf(m, fabsf(V[e].x));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    // rows below 2^-119 (far under any integral of interest) count as zero,
    // which keeps both powers of two normal floats
    float inv = 0.f, scale = 0.f;
    const int E = exp_above(m);
    if (m > 0.f && E >= -118) {
      inv = pow2f(8 - E);
      scale = pow2f(E - 8);
    }
    // slices two columns at a time (f32x2): x_s = rint(h), (h, l) =
    // 256 (h - x_s + l) as a TwoSum pair, x_s stored as x_s 2^(-8 s)
    uint4 out[S];
    const float2 inv2 = make_float2(inv, inv), magic = make_float2(12582912.0f, 12582912.0f);
    const float2 c256 = make_float2(256.f, 256.f);
#pragma unroll
    for (int e2 = 0; e2 < 4; ++e2) {
      float2 hs = mul2(make_float2(V[2 * e2].x, V[2 * e2 + 1].x), inv2);
      float2 ls = mul2(make_float2(V[2 * e2].y, V[2 * e2 + 1].y), inv2);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const float2 xs = sub2(add2(hs, magic), magic);
        float2 r, er;
        two_sum2(sub2(hs, xs), ls, r, er);
        hs = mul2(r, c256);
        ls = mul2(er, c256);
        const float ps = pow2f(-8 * s);
        const float2 xo = mul2(xs, make_float2(ps, ps));
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(xo.x, xo.y);
        (&out[s].x)[e2] = *reinterpret_cast<const uint32_t *>(&b2);
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      __stcs(reinterpret_cast<uint4 *>(vbase + (size_t)(sg * S + s) * (128 * SLOTS) + row * SLOTS + x_l * CB),
             out[s]);
    if (x_l == 0) sbase[sg * 128 + row] = scale;
  }
}

// ============================================================================ pass 1
// GEMM1 of every (tile, block pair) in exact windows, V+- = X +- Y', fixed-point
// slices of V+- to the workspace.  Work units walk range-major (unit u: range
// u / tiles of tile u % tiles) so the resident CTAs share B panels in L2.
template <int S, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1) oz_vstore_kernel(const __grid_constant__ OzLaunch Lp) {
  using C = Cfg1<S>;
  static_assert(C::kStages >= 3 && 8 * (2 * C::kStages + Bars::kCount) + 8 <= 256, "ring");
  static_assert(S >= 4 && S <= 6, "slices");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  Bars bars{ring + C::kRing, C::kStages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + C::kRing + 8 * (2 * C::kStages + Bars::kCount));
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
  const Watchdog wd{Lp.status, abort_flag, Lp.timeout_ns};

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const Item I = decode(A, vstore_slot(A, local), 1);
        const int nwin = (A.nks + kOzKc - 1) / kOzKc;
        tma_prefetch_desc(&A.tmA);
        tma_prefetch_desc(&A.tmB);
        for (int p = I.p0; ok && p < I.p1; ++p) {
          int k, l;
          pair_of(p, k, l);
          const int ntile = (k == l) ? 1 : 2;
          for (int w = 0; ok && w < nwin; ++w)
            for (int tt = 0; ok && tt < ntile; ++tt)
              for (int ks = w * kOzKc; ok && ks < min(A.nks, (w + 1) * kOzKc); ++ks) {
                if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
                const uint32_t dst = ring + (uint32_t)stage * C::kStage;
                mbar_arrive_expect_tx(bars.full(stage), C::kStage);
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                // X: rows (a, c in block k) x (b, d in block l); Y: the blocks swapped
                const int ca = (tt == 0 ? k : l) * CB, cb = (tt == 0 ? l : k) * CB;
                tma_load_4d(dst, &A.tmA, bars.full(stage), ks * KSTEP, ca, I.A0, 0);
                tma_load_4d(dst + S * A_TILE, &A.tmB, bars.full(stage), ks * KSTEP, cb, I.B0, 0);
                if (++stage == C::kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
        }
      }
      if (!ok) {
        DrainWatch dw(Lp.status, Lp.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t use[2] = {0, 0};
      const uint32_t hi64 = desc_hi(512, kSwizzle64);
      const uint32_t id64 = idesc_bf16(128, 64);
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const Item I = decode(A, vstore_slot(A, local), 1);
        const int nwin = (A.nks + kOzKc - 1) / kOzKc;
        for (int p = I.p0; ok && p < I.p1; ++p) {
          int k, l;
          pair_of(p, k, l);
          const int ntile = (k == l) ? 1 : 2;
          for (int w = 0; ok && w < nwin; ++w)
            for (int tt = 0; ok && tt < ntile; ++tt) {
              if (!(ok = mbar_wait(bars.cfree(tt), (use[tt] & 1u) ^ 1u, wd, kSiteXYFree))) break;
              tc_fence_after();
              const uint32_t dT = tmem + 256u * tt;
              const int ks0 = w * kOzKc;
              for (int ks = ks0; ok && ks < min(A.nks, ks0 + kOzKc); ++ks) {
                if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
                const uint32_t st = ring + (uint32_t)stage * C::kStage;
                const uint32_t sb = st + S * A_TILE;
#pragma unroll
                for (int kk = 0; kk < KSTEP / 16; ++kk) {
#pragma unroll
                  for (int pa = 0; pa < S; ++pa) {
                    const uint64_t ad = desc64(st + pa * A_TILE + kk * 32, hi64);
                    // slices q <= 3 - pa of B sit back to back: one MMA of
                    // N = 64 (4 - pa) puts order pa + q into column block pa + q
                    if (pa <= 3) {
                      const bool first = ks == ks0 && kk == 0 && pa == 0;
                      mma_bf16(dT + 64u * pa, ad, desc64(sb + kk * 32, hi64), idesc_bf16(128, 64 * (4 - pa)),
                               first ? 0u : 1u);
                    }
                    // the remaining products of order >= 4 into block 3
#pragma unroll
                    for (int q = (pa <= 4 ? 4 - pa : 0); q <= S - 1 - pa; ++q)
                      mma_bf16(dT + 192u, ad, desc64(sb + q * B_TILE + kk * 32, hi64), id64, 1u);
                  }
                }
                mma_commit(bars.empty(stage));
                if (++stage == C::kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
              if (!ok) break;
              mma_commit(bars.cfull(tt));
              ++use[tt];
            }
        }
      }
      mma_commit(bars.done());
      DrainWatch dw(Lp.status, Lp.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ conversion warps
    const int quad = warp & 3;
    const int qw = (warp - 2) >> 2;      // columns 16 qw .. 16 qw + 15 of each block: b = 2 qw + j
    const int L = quad * 32 + lane;      // TMEM lane = A row (a, c): a = A0 + L / 8, c = 8 k + L % 8
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + 16u * qw;
    const int a_l = L >> 3, x_l = L & 7;
    uint32_t use[2] = {0, 0};
    bool ok = true;
    for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
      int local;
      const OzArgs &A = oz_args<kBatch>(Lp, u, local);
      const Item I = decode(A, vstore_slot(A, local), 1);
      const int nwin = (A.nks + kOzKc - 1) / kOzKc;
      const int a = I.A0 + a_l;
      for (int p = I.p0; ok && p < I.p1; ++p) {
        int k, l;
        pair_of(p, k, l);
        const bool diag = (k == l);
        float2 X[16], Y[16];  // (hi, lo) sums of columns (b = 2 qw + j, d = 0..7), j = e / 8
#pragma unroll
        for (int e = 0; e < 16; ++e) X[e] = Y[e] = make_float2(0.f, 0.f);
        for (int w = 0; ok && w < nwin; ++w)
          for (int tt = 0; tt < (diag ? 1 : 2); ++tt) {
            if (!(ok = mbar_wait(bars.cfull(tt), use[tt] & 1u, wd, kSiteXYFull))) break;
            ++use[tt];
            tc_fence_after();
            if (tt == 0)
              drain_window(tl, X);
            else
              drain_window(tl + 256u, Y);
            tc_fence_before();
            mbar_arrive(bars.cfree(tt));
          }
        if (!ok) break;
        // scale to B units: X[(a, c), (b, d)] by scale(a, c) scale(b, d), c = 8k + x_l, d = 8l + e;
        // Y[(a, d'), (b, c')] with d' = 8l + x_l, c' = 8k + e
        const float rX = A.rsB[(size_t)a * A.vp + k * CB + x_l];
        const float rY = A.rsB[(size_t)a * A.vp + l * CB + x_l];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int b = I.B0 + 2 * qw + j;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float sx = rX * A.rsB[(size_t)b * A.vp + l * CB + e];
            X[8 * j + e].x *= sx;
            X[8 * j + e].y *= sx;
            if (!diag) {
              const float sy = rY * A.rsB[(size_t)b * A.vp + k * CB + e];
              Y[8 * j + e].x *= sy;
              Y[8 * j + e].y *= sy;
            }
          }
        }
        // Y' : lane (a, c = 8k + x_l) gets (ad|bc) for d = 8l + e (transpose across the 8 lanes)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float rh[8], rl[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            rh[e] = diag ? X[8 * j + e].x : Y[8 * j + e].x;
            rl[e] = diag ? X[8 * j + e].y : Y[8 * j + e].y;
          }
          transpose8(rh, x_l);
          transpose8(rl, x_l);
#pragma unroll
          for (int e = 0; e < 8; ++e) Y[8 * j + e] = make_float2(rh[e], rl[e]);
        }
        __nv_bfloat16 *vbase = A.Vst + (size_t)(I.tile * A.nbp + p) * 2 * S * (128 * SLOTS);
        float *sbase = A.sV + (size_t)(I.tile * A.nbp + p) * 2 * 128;
#pragma unroll
        for (int j = 0; j < 2; ++j) vpm_store<S>(X + 8 * j, Y + 8 * j, vbase, sbase, a_l * 8 + 2 * qw + j, x_l);
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

// ============================================================================ symmetric B
// With B^P_ac = B^P_ca for every P (the RI factors of real orbitals) the
// integral (ac|bd) = sum_P B^P_ac B^P_bd depends only on the unordered pairs
// {a, c} and {b, d}, and on them in either order.  Rows (a, c) of B with a in
// virtual block alpha and c in block gamma, alpha <= gamma, form the row block
// pair r = (alpha, gamma) (numbered as the block pairs of the slot scheme);
// the distinct integrals are the 64 x 64 tiles
//   X'(r, q)[(i % 8) * 8 + j % 8][(i' % 8) * 8 + j' % 8] = sum_P B^P_ij B^P_i'j',
// i in alpha, j in gamma, i' in beta, j' in lambda, q = (beta, lambda), r <= q,
// both orders of a diagonal block pair present.  They are computed once each
// (about a quarter of the general pass 1's GEMM1) in the same exact windows
// and kept as double-single sums in B units; the formation kernel then builds
// V+- of every (ab tile, block pair) from them and slices it as pass 1 does.

// Tile (r, q), r <= q, of the distinct integrals in row-major triangular order.
__device__ __forceinline__ size_t xtri(int r, int q, int nbp) {
  return (size_t)r * nbp - (size_t)r * (r - 1) / 2 + (size_t)(q - r);
}

// Element (ac|bd) of the distinct integral tiles.
__device__ __forceinline__ size_t xaddr(int a, int c, int b, int d, int nbp) {
  const int ba = a >> 3, bc = c >> 3, bb = b >> 3, bd = d >> 3;
  int r, row, q, col;
  if (ba <= bc) {
    r = ppos(bc) + ba;
    row = (a & 7) * 8 + (c & 7);
  } else {
    r = ppos(ba) + bc;
    row = (c & 7) * 8 + (a & 7);
  }
  if (bb <= bd) {
    q = ppos(bd) + bb;
    col = (b & 7) * 8 + (d & 7);
  } else {
    q = ppos(bb) + bd;
    col = (d & 7) * 8 + (b & 7);
  }
  return r <= q ? xtri(r, q, nbp) * 4096 + (size_t)(row * 64 + col) : xtri(q, r, nbp) * 4096 + (size_t)(col * 64 + row);
}

// Pass 1 of the symmetric form.  A work unit (xunits[u] = (iA, kk, q0, q1)) is
// the row tile of rows (a in the 16-block iA, c in block kk >= 2 iA), i.e. the
// row block pairs r = (2 iA, kk) and (2 iA + 1, kk), against the column block
// pairs q0 .. q1 - 1, taken two at a time: their windows alternate between the
// two TMEM halves as X and Y do in pass 1.  Tiles with r > q are computed but
// not stored (their transposes are the tiles (q, r)), and nor is the half
// (2 iA + 1, 2 iA) of the row tile kk = 2 iA (the half (2 iA, 2 iA + 1) of the
// row tile kk = 2 iA + 1 holds it).
template <int S, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1) oz_xsym_kernel(const __grid_constant__ OzLaunch Lp) {
  using C = Cfg1<S>;
  static_assert(C::kStages >= 3 && 8 * (2 * C::kStages + Bars::kCount) + 8 <= 256, "ring");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  Bars bars{ring + C::kRing, C::kStages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + C::kRing + 8 * (2 * C::kStages + Bars::kCount));
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
  const Watchdog wd{Lp.status, abort_flag, Lp.timeout_ns};

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const int4 U = A.xunits[local];
        const int nwin = (A.nks + kOzKc - 1) / kOzKc;
        tma_prefetch_desc(&A.tmA);
        tma_prefetch_desc(&A.tmB);
        for (int q = U.z; ok && q < U.w; q += 2) {
          const int ntile = min(2, U.w - q);
          for (int w = 0; ok && w < nwin; ++w)
            for (int tt = 0; ok && tt < ntile; ++tt) {
              int bq, lq;
              pair_of(q + tt, bq, lq);
              for (int ks = w * kOzKc; ok && ks < min(A.nks, (w + 1) * kOzKc); ++ks) {
                if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
                const uint32_t dst = ring + (uint32_t)stage * C::kStage;
                mbar_arrive_expect_tx(bars.full(stage), C::kStage);
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                // rows (a in 16-block iA, c in block kk) x rows (b in block bq, d in block lq)
                tma_load_4d(dst, &A.tmA, bars.full(stage), ks * KSTEP, U.y * CB, U.x * 16, 0);
                tma_load_4d(dst + S * A_TILE, &A.tmB, bars.full(stage), ks * KSTEP, lq * CB, bq * CB, 0);
                if (++stage == C::kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
            }
        }
      }
      if (!ok) {
        DrainWatch dw(Lp.status, Lp.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer (as in pass 1)
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t use[2] = {0, 0};
      const uint32_t hi64 = desc_hi(512, kSwizzle64);
      const uint32_t id64 = idesc_bf16(128, 64);
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const int4 U = A.xunits[local];
        const int nwin = (A.nks + kOzKc - 1) / kOzKc;
        for (int q = U.z; ok && q < U.w; q += 2) {
          const int ntile = min(2, U.w - q);
          for (int w = 0; ok && w < nwin; ++w)
            for (int tt = 0; ok && tt < ntile; ++tt) {
              if (!(ok = mbar_wait(bars.cfree(tt), (use[tt] & 1u) ^ 1u, wd, kSiteXYFree))) break;
              tc_fence_after();
              const uint32_t dT = tmem + 256u * tt;
              const int ks0 = w * kOzKc;
              for (int ks = ks0; ok && ks < min(A.nks, ks0 + kOzKc); ++ks) {
                if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
                const uint32_t st = ring + (uint32_t)stage * C::kStage;
                const uint32_t sb = st + S * A_TILE;
#pragma unroll
                for (int kk = 0; kk < KSTEP / 16; ++kk) {
#pragma unroll
                  for (int pa = 0; pa < S; ++pa) {
                    const uint64_t ad = desc64(st + pa * A_TILE + kk * 32, hi64);
                    if (pa <= 3) {
                      const bool first = ks == ks0 && kk == 0 && pa == 0;
                      mma_bf16(dT + 64u * pa, ad, desc64(sb + kk * 32, hi64), idesc_bf16(128, 64 * (4 - pa)),
                               first ? 0u : 1u);
                    }
#pragma unroll
                    for (int qq = (pa <= 4 ? 4 - pa : 0); qq <= S - 1 - pa; ++qq)
                      mma_bf16(dT + 192u, ad, desc64(sb + qq * B_TILE + kk * 32, hi64), id64, 1u);
                  }
                }
                mma_commit(bars.empty(stage));
                if (++stage == C::kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
              if (!ok) break;
              mma_commit(bars.cfull(tt));
              ++use[tt];
            }
        }
      }
      mma_commit(bars.done());
      DrainWatch dw(Lp.status, Lp.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ conversion warps
    const int quad = warp & 3;
    const int qw = (warp - 2) >> 2;  // columns 16 qw .. 16 qw + 15: b % 8 = 2 qw + j, d % 8 = e
    const int L = quad * 32 + lane;  // TMEM lane = row (a, c): a = 16 iA + L / 8, c = 8 kk + L % 8
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + 16u * qw;
    const int a_l = L >> 3, x_l = L & 7, h = a_l >> 3;
    uint32_t use[2] = {0, 0};
    bool ok = true;
    for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
      int local;
      const OzArgs &A = oz_args<kBatch>(Lp, u, local);
      const int4 U = A.xunits[local];
      const int nwin = (A.nks + kOzKc - 1) / kOzKc;
      const int a = U.x * 16 + a_l, c = U.y * CB + x_l;
      const int r = ppos(U.y) + 2 * U.x + h;  // row block pair (2 iA + h, kk)
      const bool dup = h == 1 && U.y == 2 * U.x;
      const float ra = A.rsB[(size_t)a * A.vp + c];
      for (int q = U.z; ok && q < U.w; q += 2) {
        const int ntile = min(2, U.w - q);
        float2 X[2][16];
#pragma unroll
        for (int e = 0; e < 16; ++e) X[0][e] = X[1][e] = make_float2(0.f, 0.f);
        for (int w = 0; ok && w < nwin; ++w)
          for (int tt = 0; tt < ntile; ++tt) {
            if (!(ok = mbar_wait(bars.cfull(tt), use[tt] & 1u, wd, kSiteXYFull))) break;
            ++use[tt];
            tc_fence_after();
            if (tt == 0)
              drain_window(tl, X[0]);
            else
              drain_window(tl + 256u, X[1]);
            tc_fence_before();
            mbar_arrive(bars.cfree(tt));
          }
        if (!ok) break;
#pragma unroll
        for (int tt = 0; tt < 2; ++tt) {
          const int qt = q + tt;
          if (tt >= ntile || dup || r > qt) continue;
          int bq, lq;
          pair_of(qt, bq, lq);
          float4 *dst = reinterpret_cast<float4 *>(A.Xs + xtri(r, qt, A.nbp) * 4096 + (size_t)((L & 63) * 64 + 16 * qw));
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int b = bq * CB + 2 * qw + j;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const float s0 = ra * A.rsB[(size_t)b * A.vp + lq * CB + e];
              const float s1 = ra * A.rsB[(size_t)b * A.vp + lq * CB + e + 1];
              const float2 v0 = X[tt][8 * j + e], v1 = X[tt][8 * j + e + 1];
              dst[(8 * j + e) / 2] = make_float4(v0.x * s0, v0.y * s0, v1.x * s1, v1.y * s1);
            }
          }
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

// V+- of every (ab tile, block pair) of the plan's tile range from the
// distinct integral tiles: X[(a, c), (b, d)] = (ac|bd) and Y'[(a, c), (b, d)]
// = (ad|bc) read straight from them, then vpm_store as in pass 1.  Local work
// unit (of a molecule of a batch, or of `one`) = (local tile / nbp, block
// pair % nbp); 512 threads, each the ab rows
// (a = A0 + L / 8, b = B0 + 2 qw + j) and the slot row c = 8 k + L % 8, as
// pass 1's conversion warps.
// The 8 values of one thread: (a c | b d) (y = false) or (a d | b c) (y =
// true) for d = d0 .. d0 + 7.  Where the tile holds them at 8 consecutive
// places (the thread's own 64 bytes) they come in four 16-byte loads; else
// (the lanes of the warp hold consecutive places) one 8-byte load each.
__device__ __forceinline__ void vf_gather(const float2 *__restrict__ Xs, int nbp, int a, int c, int b, int d0, bool y,
                                          float2 (&v)[8]) {
  const size_t p0 = y ? xaddr(a, d0, b, c, nbp) : xaddr(a, c, b, d0, nbp);
  const size_t p7 = y ? xaddr(a, d0 + 7, b, c, nbp) : xaddr(a, c, b, d0 + 7, nbp);
  if (p7 == p0 + 7) {
    const float4 *q = reinterpret_cast<const float4 *>(Xs + p0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 t = __ldg(q + i);
      v[2 * i] = make_float2(t.x, t.y);
      v[2 * i + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __ldg(Xs + (y ? xaddr(a, d0 + e, b, c, nbp) : xaddr(a, c, b, d0 + e, nbp)));
  }
}

template <int S, bool kBatch>
__global__ void __launch_bounds__(512) oz_vform_kernel(const __grid_constant__ OzLaunch Lp) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int L = (warp & 3) * 32 + lane, qw = warp >> 2;
  const int a_l = L >> 3, x_l = L & 7;
  for (int u = blockIdx.x; u < Lp.nitems; u += gridDim.x) {
    int local;
    const OzArgs &A = oz_args<kBatch>(Lp, u, local);
    const float2 *__restrict__ Xs = A.Xs;
    const int t = local / A.nbp, p = local - t * A.nbp;
    int iA = 0, tr = t + A.tile0;
    while (tr >= A.nB8 - 2 * iA) {
      tr -= A.nB8 - 2 * iA;
      ++iA;
    }
    const int a = iA * 16 + a_l, B0 = (2 * iA + tr) * CB;
    int k, l;
    pair_of(p, k, l);
    const int c = k * CB + x_l;
    __nv_bfloat16 *vbase = A.Vst + (size_t)(t * A.nbp + p) * 2 * S * (128 * SLOTS);
    float *sbase = A.sV + (size_t)(t * A.nbp + p) * 2 * 128;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int b = B0 + 2 * qw + j;
      float2 X[8], Y[8];
      vf_gather(Xs, A.nbp, a, c, b, l * CB, false, X);  // (a c | b d), d = 8 l + e
      vf_gather(Xs, A.nbp, a, c, b, l * CB, true, Y);   // (a d | b c)
      vpm_store<S>(X, Y, vbase, sbase, a_l * 8 + 2 * qw + j, x_l);
    }
  }
}

// B^P_ac = B^P_ca for every P and a, c < v (bitwise), checked on 32 x 32
// tiles of the upper triangle; a mismatch records kSiteAsymmetric.
__global__ void oz_symcheck_kernel(int N, int v, const double *__restrict__ B, int *status) {
  __shared__ double t[32][33];
  const int ta = blockIdx.x, tc = blockIdx.y;
  if (tc < ta) return;
  bool bad = false;
  for (int P = blockIdx.z; P < N; P += gridDim.z) {
    const double *Bp = B + (size_t)P * v * v;
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int a = tc * 32 + y, c = ta * 32 + threadIdx.x;
      if (a < v && c < v) t[y][threadIdx.x] = Bp[(size_t)a * v + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      const int a = ta * 32 + y, c = tc * 32 + threadIdx.x;
      if (a < v && c < v)
        bad |= __double_as_longlong(Bp[(size_t)a * v + c]) != __double_as_longlong(t[threadIdx.x][y]);
    }
  }
  if (bad) record_status(status, kSiteAsymmetric);
}

// ============================================================================ pass 2
// GEMM2 of one (tile, chunk of <= 128 occupied pairs of one sign, block-pair
// range): per block pair the slice products V_p T_q^T (p + q < S) of its four
// 16-slot pieces into the four order accumulators (columns 0, 128, 256, 384),
// issued and drained group by group (orders 0-1, 2, >= 3) with the pair's row
// scales into double-single sums in registers.  Work units walk range-major
// (unit u: range u / (tiles * chunks)).
template <int S, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1) oz_gemm2_kernel(const __grid_constant__ OzLaunch Lp) {
  using C = Cfg2<S>;
  static_assert(C::kStages >= SLOTS / TPIECE && 8 * (2 * C::kStages + Bars::kCount) + 8 <= 256, "ring");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t *smem = smem_raw + pad;
  const uint32_t ring = raw + pad;
  Bars bars{ring + C::kRing, C::kStages};
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + C::kRing + 8 * (2 * C::kStages + Bars::kCount));
  int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(bars.full(s), 1);
      mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 3; ++b) {
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
  const Watchdog wd{Lp.status, abort_flag, Lp.timeout_ns};
  constexpr int kPieces = SLOTS / TPIECE;

  if (warp == 0) {
    // ================================================================ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, armed = 0, armed_par = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const Item I = decode(A, gemm2_slot(A, local), A.nchunks);
        tma_prefetch_desc(&A.tmVl);
        const uint32_t sc = (uint32_t)(I.CH.nps + I.CH.nms);
        const int sg = I.CH.nps > 0 ? 0 : 1;
        const uint32_t tbytes = (uint32_t)S * sc * 32u;
        for (int p = I.p0; ok && p < I.p1; ++p) {
          const int plane0 = ((I.tile * A.nbp + p) * 2 + sg) * S;
          for (int piece = 0; piece < kPieces; ++piece) {
            if (!(ok = mbar_wait(bars.empty(stage), phase ^ 1u, wd, kSiteTmaEmpty))) break;
            const uint32_t dst = ring + (uint32_t)stage * C::kStage;
            mbar_arrive_expect_tx(bars.full(stage), (uint32_t)S * VP_PLANE + tbytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            tma_load_3d(dst, &A.tmVl, bars.full(stage), piece * TPIECE, 0, plane0);
            bulk_load(dst + S * VP_PLANE, A.T2 + I.CH.t2off + (size_t)(p * kPieces + piece) * tbytes, tbytes,
                      bars.full(stage));
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        DrainWatch dw(Lp.status, Lp.timeout_ns);
        for (int s = 0; s < C::kStages; ++s)
          if (armed & (1u << s)) mbar_wait(bars.full(s), (armed_par >> s) & 1u, dw.wd, kSiteTmaFull);
      }
    }
  } else if (warp == 1) {
    // ================================================================ MMA issuer
    // Per block pair the products go out by order group: orders 0 and 1
    // (accumulators 0 and 1, 3 MMAs per piece), order 2 (accumulator 2, 3
    // per piece), orders >= 3 (accumulator 3).  Each group is committed on its
    // own barrier, so the drain of a group overlaps the MMAs of the later
    // groups, and the next pair's group starts as soon as its accumulator has
    // been drained.  The four pieces of a pair stay in the ring until their
    // last (order >= 3) MMAs.
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, g = 0;
      const uint32_t hi32 = desc_hi(256, kSwizzle32);
      bool ok = true;
      for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
        int local;
        const OzArgs &A = oz_args<kBatch>(Lp, u, local);
        const Item I = decode(A, gemm2_slot(A, local), A.nchunks);
        const uint32_t sc = (uint32_t)(I.CH.nps + I.CH.nms);
        const uint32_t id = idesc_bf16(128, (int)sc);
        for (int p = I.p0; ok && p < I.p1; ++p) {
          int sidx[kPieces];
          // orders 0 and 1, waiting for each piece's operands
          if (!(ok = mbar_wait(bars.cfree(0), (g & 1u) ^ 1u, wd, kSiteRFree))) break;
          tc_fence_after();
          for (int piece = 0; ok && piece < kPieces; ++piece) {
            if (!(ok = mbar_wait(bars.full(stage), phase, wd, kSiteTmaFull))) break;
            sidx[piece] = stage;
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
            const uint32_t st = ring + (uint32_t)sidx[piece] * C::kStage, stt = st + S * VP_PLANE;
            const uint32_t acc = piece ? 1u : 0u;
            mma_bf16(tmem, desc64(st, hi32), desc64(stt, hi32), id, acc);
            mma_bf16(tmem + 128u, desc64(st, hi32), desc64(stt + sc * 32u, hi32), id, acc);
            mma_bf16(tmem + 128u, desc64(st + VP_PLANE, hi32), desc64(stt, hi32), id, 1u);
          }
          if (!ok) break;
          mma_commit(bars.cfull(0));
          // order 2
          if (!(ok = mbar_wait(bars.cfree(1), (g & 1u) ^ 1u, wd, kSiteRFree))) break;
          tc_fence_after();
          for (int piece = 0; piece < kPieces; ++piece) {
            const uint32_t st = ring + (uint32_t)sidx[piece] * C::kStage, stt = st + S * VP_PLANE;
#pragma unroll
            for (int pa = 0; pa <= 2; ++pa)
              mma_bf16(tmem + 256u, desc64(st + pa * VP_PLANE, hi32), desc64(stt + (2 - pa) * sc * 32u, hi32), id,
                       (piece == 0 && pa == 0) ? 0u : 1u);
          }
          mma_commit(bars.cfull(1));
          // orders >= 3; a piece's stage goes back to the producer after them
          if (!(ok = mbar_wait(bars.cfree(2), (g & 1u) ^ 1u, wd, kSiteRFree))) break;
          tc_fence_after();
          for (int piece = 0; piece < kPieces; ++piece) {
            const uint32_t st = ring + (uint32_t)sidx[piece] * C::kStage, stt = st + S * VP_PLANE;
#pragma unroll
            for (int pa = 0; pa < S; ++pa)
#pragma unroll
              for (int q = (pa < 3 ? 3 - pa : 0); q < S - pa; ++q)
                mma_bf16(tmem + 384u, desc64(st + pa * VP_PLANE, hi32), desc64(stt + q * sc * 32u, hi32), id,
                         (piece == 0 && pa == 0 && q == 3) ? 0u : 1u);
            mma_commit(bars.empty(sidx[piece]));
          }
          mma_commit(bars.cfull(2));
          ++g;
        }
      }
      mma_commit(bars.done());
      DrainWatch dw(Lp.status, Lp.timeout_ns);
      mbar_wait(bars.done(), 0, dw.wd, kSiteRFull);
    }
  } else {
    // ================================================================ drains -> sums
    // Group by group, as the MMA issuer commits them, each scaled by the
    // pair's row scales (exact powers of two): orders 0 + 1 as one TwoSum
    // pair into the double-single sums, order 2 (2^-16 below the window) with
    // a TwoSum, orders >= 3 (2^-24 below) fused into the low words, where the
    // rounding is 2^-48 of the window; two columns per f32x2 instruction.
    const int quad = warp & 3;
    const int qw = (warp - 2) >> 2;  // columns 32 qw .. 32 qw + 31
    const int L = quad * 32 + lane;  // TMEM lane = ab row of the tile
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + 32u * qw;
    uint32_t g = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < Lp.nitems; u += gridDim.x) {
      int local;
      const OzArgs &A = oz_args<kBatch>(Lp, u, local);
      const Item I = decode(A, gemm2_slot(A, local), A.nchunks);
      const int sc = I.CH.nps + I.CH.nms;
      const int sg = I.CH.nps > 0 ? 0 : 1;
      const int ng = min(8, max(0, (sc - 32 * qw) / 4));  // this thread's 4-column groups
      float2 H[16], Lo[16];  // (hi, lo) sums of columns 32 qw + 2k and 2k + 1 (as .x and .y)
#pragma unroll
      for (int e = 0; e < 16; ++e) H[e] = Lo[e] = make_float2(0.f, 0.f);
      for (int p = I.p0; ok && p < I.p1; ++p) {
        const float *svp = A.sV + ((size_t)(I.tile * A.nbp + p) * 2 + sg) * 128 + L;
        const float *st = A.sT + ((size_t)I.ch * A.nbp + p) * kOzMaxCols + 32 * qw;
        // this pair's scales into L1 while its MMAs run
        asm volatile("prefetch.global.L1 [%0];" ::"l"(st));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(svp));
        if (!(ok = mbar_wait(bars.cfull(0), g & 1u, wd, kSiteRFull))) break;
        tc_fence_after();
        const float sv = *svp;
        const float2 sv2 = make_float2(sv, sv);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          if (h < ng) {
            float g0[4], g1[4];
            const uint32_t c0 = tl + 4u * h;
            tmem_ld4(c0, g0);
            tmem_ld4(c0 + 128u, g1);
            const float4 t0 = *reinterpret_cast<const float4 *>(st + 4 * h);
            tmem_ld_wait();
            const float2 s01 = mul2(sv2, make_float2(t0.x, t0.y)), s23 = mul2(sv2, make_float2(t0.z, t0.w));
            float2 hh, ll;
            two_sum2(make_float2(g0[0], g0[1]), make_float2(g1[0], g1[1]), hh, ll);
            ds_acc2(H[2 * h], Lo[2 * h], mul2(hh, s01), mul2(ll, s01));
            two_sum2(make_float2(g0[2], g0[3]), make_float2(g1[2], g1[3]), hh, ll);
            ds_acc2(H[2 * h + 1], Lo[2 * h + 1], mul2(hh, s23), mul2(ll, s23));
          }
        }
        tc_fence_before();
        mbar_arrive(bars.cfree(0));
#pragma unroll
        for (int grp = 2; grp < 4; ++grp) {
          if (!(ok = mbar_wait(bars.cfull(grp - 1), g & 1u, wd, kSiteRFull))) break;
          tc_fence_after();
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            if (h < ng) {
              float gg[4];
              tmem_ld4(tl + 4u * h + 128u * grp, gg);
              const float4 t0 = *reinterpret_cast<const float4 *>(st + 4 * h);
              tmem_ld_wait();
              const float2 s01 = mul2(sv2, make_float2(t0.x, t0.y)), s23 = mul2(sv2, make_float2(t0.z, t0.w));
              if (grp == 2) {
                ds_add2(H[2 * h], Lo[2 * h], mul2(make_float2(gg[0], gg[1]), s01));
                ds_add2(H[2 * h + 1], Lo[2 * h + 1], mul2(make_float2(gg[2], gg[3]), s23));
              } else {
                Lo[2 * h] = fma2(make_float2(gg[0], gg[1]), s01, Lo[2 * h]);
                Lo[2 * h + 1] = fma2(make_float2(gg[2], gg[3]), s23, Lo[2 * h + 1]);
              }
            }
          }
          tc_fence_before();
          mbar_arrive(bars.cfree(grp - 1));
        }
        if (!ok) break;
        ++g;
      }
      if (!ok) break;
      // this unit's sums, [col][lane]
#pragma unroll
      for (int h = 0; h < 8; ++h)
        if (h < ng)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const size_t c = (size_t)(32 * qw + 4 * h + 2 * k);
            I.racc[c * 128 + L] = make_float2(H[2 * h + k].x, Lo[2 * h + k].x);
            I.racc[(c + 1) * 128 + L] = make_float2(H[2 * h + k].y, Lo[2 * h + k].y);
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

// ============================================================================ preparation
// One thread per row (a, c) of B: the smallest E with max_P |B^P_ac| < 2^E
// gives the row's scale 2^(E - 8) (0 for a zero row or a padding row).
// A NaN or infinite element records kSiteNonFinite in the status word.
__global__ void oz_rowscale_kernel(int N, int v, int vp, const double *__restrict__ B, float *__restrict__ rs,
                                   int *status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vp * vp) return;
  const int a = idx / vp, c = idx % vp;
  // the largest |B^P_ac| as the largest magnitude bit pattern (the order of
  // non-negative doubles), and NaN or infinity as an all-ones exponent: both
  // on the integer pipe
  unsigned long long mb = 0;
  if (a < v && c < v)
    for (int P = 0; P < N; ++P) {
      const unsigned long long x = (unsigned long long)__double_as_longlong(B[((size_t)P * v + a) * v + c]);
      mb = max(mb, x & 0x7fffffffffffffffull);
    }
  const bool bad = mb >= 0x7ff0000000000000ull;
  const double m = __longlong_as_double((long long)mb);
  if (bad) record_status(status, kSiteNonFinite);
  float r = 0.f;
  if (m > 0.0 && !bad) {
    int E;
    frexp(m, &E);  // m = f 2^E, 1/2 <= f < 1
    r = (float)ldexp(1.0, E - 8);
  }
  rs[idx] = r;
}

// y (|y| <= 256, the element over its row's scale) = x_0 + x_1 2^-8 + ... with
// x_s = nearest integer of what is left: slice s stored as the BF16 number
// x_s 2^(-8 s) (exact).  y is carried as a double-single (hi, lo), about 48
// bits, and every step runs on the FP32 pipe: x = rint(hi) and hi - x are
// exact, TwoSum renormalises the remainder, and the scaling by 256 is exact.
template <int S>
__device__ __forceinline__ void fixed_slices(double y, __nv_bfloat16 (&out)[S]) {
  float hi = __double2float_rn(y);
  float lo = __double2float_rn(y - (double)hi);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float x = rint_small(hi);
    float r, er;
    two_sum(__fsub_rn(hi, x), lo, r, er);
    hi = r * 256.f;
    lo = er * 256.f;
    out[s] = __float2bfloat16_rn(x * pow2f(-8 * s));
  }
}

// Bt[s][a][c][P] = slice s of B^P_ac / scale(a, c), 32x32 tiles through shared
// memory (read c fastest, write P fastest); zero beyond v and N.
template <int S>
__global__ void oz_split_B_kernel(int N, int v, int vp, int Np, const double *__restrict__ B,
                                  const float *__restrict__ rs, __nv_bfloat16 *__restrict__ Bt) {
  __shared__ double tile[32][33];
  const int a = blockIdx.z;
  const int c0 = blockIdx.x * 32, P0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int P = P0 + r, c = c0 + tx;
    tile[r][tx] = (P < N && c < v && a < v) ? B[((size_t)P * v + a) * v + c] : 0.0;
  }
  __syncthreads();
  const size_t slice = (size_t)vp * vp * Np;
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, P = P0 + tx;
    if (c < vp && P < Np) {
      const float sc = rs[(size_t)a * vp + c];
      // 1 / sc exactly (sc is a power of two): built from its exponent for a
      // normal sc, which spares the FP64 division; a subnormal sc divides
      const int eb = (__float_as_int(sc) >> 23) & 0xff;
      const double inv = eb ? __longlong_as_double((long long)(1023 + 127 - eb) << 52)
                            : (sc > 0.f ? 1.0 / (double)sc : 0.0);
      __nv_bfloat16 sl[S];
      fixed_slices<S>(tile[tx][r] * inv, sl);
      const size_t off = ((size_t)a * vp + c) * Np + P;
#pragma unroll
      for (int q = 0; q < S; ++q) Bt[q * slice + off] = sl[q];
    }
  }
}

// GEMM2 operand: for chunk c, 16-slot piece x (block pair x / 4) and slice s,
// the chunk's rows (lambda+ rows, padding, lambda- rows, padding) of 32 bytes,
// stored [x][s][row] in the 32-byte-swizzled order of shared memory, as
// pack_t2 does.  Eight threads share one (row, block pair): thread cl takes
// c = 8k + cl, d = 8l + 0..7 (piece cl / 2, half cl % 2), the group's maximum
// gives the row's scale for the pair, written to sT[c][pair][row].
//   tau+ = w (tau^cd + tau^dc),  tau- = w (tau^cd - tau^dc),  w = 1/4 (k = l), 1/2.
template <int S>
__global__ void oz_pack_t2_kernel(const __grid_constant__ OzPackArgs a) {
  const TcChunk CH = a.chunks[blockIdx.y];
  const int sc = CH.nps + CH.nms;
  const size_t groups = (size_t)sc * a.nbp;
  uint4 *dst = reinterpret_cast<uint4 *>(a.T2 + CH.t2off);
  const int cl = threadIdx.x & 7;
  const size_t g0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const size_t gstep = ((size_t)gridDim.x * blockDim.x) >> 3;
  const size_t vv = (size_t)a.v * a.v;
  // every thread runs the same number of iterations (the shuffles below take
  // the whole warp)
  const size_t niter = (groups + gstep - 1) / gstep;
  for (size_t it = 0; it < niter; ++it) {
    const size_t gi = g0 + it * gstep;
    const bool live_g = gi < groups;
    const int row = live_g ? (int)(gi % sc) : 0;
    const int p = live_g ? (int)(gi / sc) : 0;
    int k, l;
    pair_of(p, k, l);
    int i = 0, j = 0;
    bool live = false, plus = true;
    if (live_g && row < CH.np) {
      lam_plus(CH.lp0 + row, i, j);
      live = true;
    } else if (live_g && row >= CH.nps && row - CH.nps < CH.nm) {
      lam_minus(CH.lm0 + (row - CH.nps), i, j);
      live = true;
      plus = false;
    }
    const int c = k * CB + cl;
    const double w = (k == l) ? 0.25 : 0.5;
    const double *tij = a.tau + ((size_t)i * a.o + j) * vv;
    double val[8];
    double m = 0.0;
    bool bad = false;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int d = l * CB + e;
      double x = 0.0;
      if (live && c < a.v && d < a.v) {
        const double t_cd = tij[(size_t)c * a.v + d], t_dc = tij[(size_t)d * a.v + c];
        bad |= !(isfinite(t_cd) && isfinite(t_dc));
        x = plus ? w * (t_cd + t_dc) : w * (t_cd - t_dc);
      }
      val[e] = x;
      m = fmax(m, fabs(x));
    }
    if (bad) record_status(a.status, kSiteNonFinite);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, 4));
    if (!live_g) continue;
    double inv = 0.0;
    float scale = 0.f;
    if (m > 0.0 && isfinite(m)) {
      int E;
      frexp(m, &E);
      inv = ldexp(1.0, 8 - E);
      scale = (float)ldexp(1.0, E - 8);
    }
    __nv_bfloat16 sl[S][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      __nv_bfloat16 xs[S];
      fixed_slices<S>(val[e] * inv, xs);
#pragma unroll
      for (int s = 0; s < S; ++s) sl[s][e] = xs[s];
    }
    const size_t x = (size_t)p * 4 + cl / 2;
    const int h = cl & 1;
#pragma unroll
    for (int s = 0; s < S; ++s)
      dst[((x * S + s) * sc + row) * 2 + (h ^ ((row >> 2) & 1))] = *reinterpret_cast<const uint4 *>(sl[s]);
    if (cl == 0) a.sT[((size_t)blockIdx.y * a.nbp + p) * kOzMaxCols + row] = scale;
  }
}

}  // namespace

void launch_oz_rowscale(int N, int v, int vp, const double *B, float *rs, int *status, cudaStream_t s) {
  const int n = vp * vp;
  oz_rowscale_kernel<<<(n + 255) / 256, 256, 0, s>>>(N, v, vp, B, rs, status);
}

void launch_oz_split_B(int N, int v, int vp, int Np, int nslices, const double *B, const float *rs,
                       __nv_bfloat16 *Bt, cudaStream_t s) {
  dim3 grid((vp + 31) / 32, (Np + 31) / 32, vp), block(32, 8);
  if (nslices == 5)
    oz_split_B_kernel<5><<<grid, block, 0, s>>>(N, v, vp, Np, B, rs, Bt);
  else
    oz_split_B_kernel<6><<<grid, block, 0, s>>>(N, v, vp, Np, B, rs, Bt);
}

void launch_oz_pack_t2(const OzPackArgs &a, cudaStream_t s) {
  dim3 grid(512, a.nchunks);
  if (a.S == 5)
    oz_pack_t2_kernel<5><<<grid, 256, 0, s>>>(a);
  else
    oz_pack_t2_kernel<6><<<grid, 256, 0, s>>>(a);
}

uint32_t oz_smem_bytes(int pass, int nslices) {
  if (pass == 1) return nslices == 5 ? Cfg1<5>::kSmem : Cfg1<6>::kSmem;
  return nslices == 5 ? Cfg2<5>::kSmem : Cfg2<6>::kSmem;
}

template <int S>
cudaError_t oz_attrs() {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(oz_vstore_kernel<S, false>, at, (int)Cfg1<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(oz_vstore_kernel<S, true>, at, (int)Cfg1<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(oz_gemm2_kernel<S, false>, at, (int)Cfg2<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(oz_gemm2_kernel<S, true>, at, (int)Cfg2<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(oz_xsym_kernel<S, false>, at, (int)Cfg1<S>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(oz_xsym_kernel<S, true>, at, (int)Cfg1<S>::kSmem);
  return e;
}

cudaError_t oz_init_attributes(int nslices) { return nslices == 5 ? oz_attrs<5>() : oz_attrs<6>(); }

// one CTA per work unit
cudaError_t launch_oz_vstore(const OzLaunch &L, int nslices, cudaStream_t s) {
  if (L.nitems <= 0) return cudaSuccess;
  const bool b = L.mols != nullptr;
  if (nslices == 5) {
    if (b)
      oz_vstore_kernel<5, true><<<L.nitems, kThreads, Cfg1<5>::kSmem, s>>>(L);
    else
      oz_vstore_kernel<5, false><<<L.nitems, kThreads, Cfg1<5>::kSmem, s>>>(L);
  } else {
    if (b)
      oz_vstore_kernel<6, true><<<L.nitems, kThreads, Cfg1<6>::kSmem, s>>>(L);
    else
      oz_vstore_kernel<6, false><<<L.nitems, kThreads, Cfg1<6>::kSmem, s>>>(L);
  }
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm2(const OzLaunch &L, int nslices, cudaStream_t s) {
  if (L.nitems <= 0) return cudaSuccess;
  const bool b = L.mols != nullptr;
  if (nslices == 5) {
    if (b)
      oz_gemm2_kernel<5, true><<<L.nitems, kThreads, Cfg2<5>::kSmem, s>>>(L);
    else
      oz_gemm2_kernel<5, false><<<L.nitems, kThreads, Cfg2<5>::kSmem, s>>>(L);
  } else {
    if (b)
      oz_gemm2_kernel<6, true><<<L.nitems, kThreads, Cfg2<6>::kSmem, s>>>(L);
    else
      oz_gemm2_kernel<6, false><<<L.nitems, kThreads, Cfg2<6>::kSmem, s>>>(L);
  }
  return cudaGetLastError();
}

// one CTA per work unit of the distinct integral tiles
cudaError_t launch_oz_xsym(const OzLaunch &L, int nslices, cudaStream_t s) {
  if (L.nitems <= 0) return cudaSuccess;
  const bool b = L.mols != nullptr;
  if (nslices == 5) {
    if (b)
      oz_xsym_kernel<5, true><<<L.nitems, kThreads, Cfg1<5>::kSmem, s>>>(L);
    else
      oz_xsym_kernel<5, false><<<L.nitems, kThreads, Cfg1<5>::kSmem, s>>>(L);
  } else {
    if (b)
      oz_xsym_kernel<6, true><<<L.nitems, kThreads, Cfg1<6>::kSmem, s>>>(L);
    else
      oz_xsym_kernel<6, false><<<L.nitems, kThreads, Cfg1<6>::kSmem, s>>>(L);
  }
  return cudaGetLastError();
}

// two blocks per SM, each walking the units
cudaError_t launch_oz_vform(const OzLaunch &L, int nslices, int sm_count, cudaStream_t s) {
  if (L.nitems <= 0) return cudaSuccess;
  const int grid = std::min(L.nitems, 2 * sm_count);
  const bool b = L.mols != nullptr;
  if (nslices == 5) {
    if (b)
      oz_vform_kernel<5, true><<<grid, 512, 0, s>>>(L);
    else
      oz_vform_kernel<5, false><<<grid, 512, 0, s>>>(L);
  } else {
    if (b)
      oz_vform_kernel<6, true><<<grid, 512, 0, s>>>(L);
    else
      oz_vform_kernel<6, false><<<grid, 512, 0, s>>>(L);
  }
  return cudaGetLastError();
}

void launch_oz_symcheck(int N, int v, const double *B, int *status, cudaStream_t s) {
  const int nt = (v + 31) / 32;
  oz_symcheck_kernel<<<dim3(nt, nt, std::min(N, 4096)), dim3(32, 8), 0, s>>>(N, v, B, status);
}

}  // namespace ladder
