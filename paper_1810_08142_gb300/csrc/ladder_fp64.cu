// FP64 fused ladder kernel: the plain method, exact up to FP64 rounding.
//
// R_ij^ab = sum_cd (ac|bd) tau_ij^cd (Eq. pp-Ladder-0) with (ac|bd) =
// sum_P B^P_ac B^P_bd (Eq. RIM), evaluated through the symmetric /
// antisymmetric pair combinations (Sec. II.C cites the quarter-cost split;
// the slot form used here: virtual indices in blocks of 8, block pairs k <= l,
// V+-_ab[(c,d)] = (ac|bd) +- (ad|bc), R+- = sum_slots T+- V+-).
//
// One CTA owns an (a-block, b-block) tile of 8 x 8 virtual pairs (a-block <=
// b-block) and one chunk of occupied pairs.  For every (c,d) block pair it
//   1. forms the two 64x64 integral tiles X[(a,c),(b,d)] and Y[(a,d),(b,c)]
//      with FP64 tensor-core MMAs (m8n8k4) over P, staged in shared memory,
//   2. combines them into V+ and V- (64 ab x 64 slots) in shared memory,
//   3. multiplies T+- (occupied pairs x slots) into register accumulators.
// The integral tiles never leave the SM.  When the occupied pairs need more
// than one chunk, the first chunk spills V+- to a per-CTA slab and the later
// chunks read it back instead of recomputing the integrals.
#include "kernels.h"

namespace ladder {
namespace {

constexpr int NT = 256;             // 8 warps
constexpr int KP = 16;              // aux functions per panel
constexpr int PSTR = 4 * 64 + 4;    // panel stride per P (4 row sets of 64, padded)
constexpr int VSTR = SLOTS + 4;     // padded row stride of V and T tiles
constexpr int LT = kFp64LamTile;    // 64 occupied pairs per sign and chunk

constexpr size_t kPanelDoubles = (size_t)KP * PSTR;
constexpr size_t kSmemDoubles = 2 * kPanelDoubles + 2 * 64 * VSTR + 2 * LT * VSTR;

__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Four row sets of the integral tiles for block pair (k, l):
//   0: (a, c in C_k)   1: (b, d in C_l)   2: (a, d in C_l)   3: (b, c in C_k)
// row r = x*8 + y with x the a (or b) offset and y the c (or d) offset.
__device__ __forceinline__ void load_panel(double *panel, const Fp64Args &A, int P0, int A0,
                                           int B0, int k, int l, bool diag) {
  const int nsets = diag ? 2 : 4;
  for (int e = threadIdx.x; e < KP * nsets * 64; e += NT) {
    const int P = e / (nsets * 64), rem = e % (nsets * 64);
    const int set = rem / 64, r = rem % 64;
    const int x = ((set == 0 || set == 2) ? A0 : B0) + r / 8;
    const int y = ((set == 0 || set == 3) ? k : l) * CB + r % 8;
    const int PP = P0 + P;
    const bool ok = PP < A.N && x < A.v && y < A.v;
    // transB: the factor is read as B^P_yx (the transposed ladder of the adjoint)
    const size_t off = A.transB ? ((size_t)PP * A.v + y) * A.v + x : ((size_t)PP * A.v + x) * A.v + y;
    const double *src = ok ? A.B + off : A.B;
    cp_async8(panel + P * PSTR + set * 64 + r, src, ok ? 8 : 0);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(NT, 1) ladder_fp64_kernel(const __grid_constant__ Fp64Args A) {
  extern __shared__ double smem[];
  double *panels = smem;
  double *Vp = smem + 2 * kPanelDoubles;
  double *Vm = Vp + 64 * VSTR;
  double *Tps = Vm + 64 * VSTR;
  double *Tms = Tps + LT * VSTR;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = lane / 4, q = lane % 4;
  const int nb = A.vp / CB, nbp = ppos(nb);
  const size_t slab_per_pair = 2 * 64 * SLOTS;
  double *slab = A.slab ? A.slab + (size_t)blockIdx.x * nbp * slab_per_pair : nullptr;

  for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
    int ia, ib;
    pair_of(tile, ia, ib);
    const int A0 = ia * CB, B0 = ib * CB;
    for (int ch = 0; ch < A.nchunks; ++ch) {
      const int lp0 = ppos(A.chunks[ch].j0), lp1 = ppos(A.chunks[ch].j1);
      const int lm0 = pneg(A.chunks[ch].j0), lm1 = pneg(A.chunks[ch].j1);
      double accP[8][2], accM[8][2];
#pragma unroll
      for (int n = 0; n < 8; ++n) accP[n][0] = accP[n][1] = accM[n][0] = accM[n][1] = 0.0;

      for (int p = 0; p < nbp; ++p) {
        int k, l;
        pair_of(p, k, l);
        const bool diag = (k == l);
        if (ch == 0) {
          // ---- 1. integral tiles X (and Y) over P, double-buffered panels
          double X[8][2], Y[8][2];
#pragma unroll
          for (int n = 0; n < 8; ++n) X[n][0] = X[n][1] = Y[n][0] = Y[n][1] = 0.0;
          const int npan = (A.N + KP - 1) / KP;
          load_panel(panels, A, 0, A0, B0, k, l, diag);
          for (int pan = 0; pan < npan; ++pan) {
            if (pan + 1 < npan) {
              load_panel(panels + ((pan + 1) & 1) * kPanelDoubles, A, (pan + 1) * KP, A0, B0, k, l,
                         diag);
              cp_async_wait<1>();
            } else {
              cp_async_wait<0>();
            }
            __syncthreads();
            const double *pn = panels + (pan & 1) * kPanelDoubles;
#pragma unroll
            for (int kk = 0; kk < KP / 4; ++kk) {
              const double *pr = pn + (kk * 4 + q) * PSTR;
              const double ax = pr[0 * 64 + warp * 8 + g];
#pragma unroll
              for (int n = 0; n < 8; ++n) dmma(X[n][0], X[n][1], ax, pr[1 * 64 + n * 8 + g]);
              if (!diag) {
                const double ay = pr[2 * 64 + warp * 8 + g];
#pragma unroll
                for (int n = 0; n < 8; ++n) dmma(Y[n][0], Y[n][1], ay, pr[3 * 64 + n * 8 + g]);
              }
            }
            __syncthreads();
          }
          // ---- 2. V+ = X + Y', V- = X - Y' with Y'[(c,d)] = (ad|bc)
          // X fragment: row c = g, col d = 2q + e of tile (a = warp, b = n).
          // Y fragment: row d = g, col c = 2q + e.  On a diagonal block pair
          // Y is X itself read transposed.
#pragma unroll
          for (int n = 0; n < 8; ++n) {
            const int ab = warp * 8 + n;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              Vp[ab * VSTR + g * CB + 2 * q + e] = X[n][e];
              Vm[ab * VSTR + (2 * q + e) * CB + g] = diag ? X[n][e] : Y[n][e];
            }
          }
          __syncthreads();
          for (int e = tid; e < 64 * SLOTS; e += NT) {
            const int ab = e / SLOTS, s = e % SLOTS;
            const double x = Vp[ab * VSTR + s], y = Vm[ab * VSTR + s];
            Vp[ab * VSTR + s] = x + y;
            Vm[ab * VSTR + s] = x - y;
          }
          __syncthreads();
          if (slab && A.nchunks > 1) {
            double *dst = slab + (size_t)p * slab_per_pair;
            for (int e = tid; e < 2 * 64 * SLOTS; e += NT) {
              const int sgn = e / (64 * SLOTS), rem = e % (64 * SLOTS);
              dst[e] = (sgn ? Vm : Vp)[(rem / SLOTS) * VSTR + rem % SLOTS];
            }
          }
        } else {
          const double *src = slab + (size_t)p * slab_per_pair;
          for (int e = tid; e < 64 * 64 / 2 * 2; e += NT) {  // pairs of doubles
            const int sgn = e / (64 * SLOTS / 2), rem = (e % (64 * SLOTS / 2)) * 2;
            cp_async16((sgn ? Vm : Vp) + (rem / SLOTS) * VSTR + rem % SLOTS,
                       src + (size_t)sgn * 64 * SLOTS + rem, 16);
          }
          cp_async_commit();
        }
        // ---- 3. T+- tiles for this block pair and chunk
        for (int e = tid; e < 2 * LT * SLOTS / 2; e += NT) {
          const int sgn = e / (LT * SLOTS / 2), rem = (e % (LT * SLOTS / 2)) * 2;
          const int r = rem / SLOTS, s = rem % SLOTS;
          const int row = (sgn ? lm0 : lp0) + r;
          const bool ok = row < (sgn ? lm1 : lp1);
          const double *src = (sgn ? A.Tm : A.Tp) + (ok ? (size_t)row * A.K + (size_t)p * SLOTS + s : 0);
          cp_async16((sgn ? Tms : Tps) + r * VSTR + s, src, ok ? 16 : 0);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        // ---- 4. R+- += T+- V+-^T : warp owns occupied rows 8*warp .. 8*warp+7
#pragma unroll 4
        for (int kk = 0; kk < SLOTS / 4; ++kk) {
          const int s = kk * 4 + q;
          const double ap = Tps[(warp * 8 + g) * VSTR + s];
          const double am = Tms[(warp * 8 + g) * VSTR + s];
#pragma unroll
          for (int n = 0; n < 8; ++n) {
            dmma(accP[n][0], accP[n][1], ap, Vp[(n * 8 + g) * VSTR + s]);
            dmma(accM[n][0], accM[n][1], am, Vm[(n * 8 + g) * VSTR + s]);
          }
        }
        __syncthreads();
      }
      // ---- 5. unpack: R_ij^ab = R+ + R-, R_ij^ba = R+ - R-, mirrored to (j, i)
      // accumulator element (row 8*warp + g, col 8*n + 2q + e) -> a = A0 + n, b = B0 + 2q + e
      {
        const int lam = lp0 + warp * 8 + g;
        if (lam < lp1) {
          int i, j;
          lam_plus(lam, i, j);
#pragma unroll
          for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int a = A0 + n, b = B0 + 2 * q + e;
              if (a < A.v && b < A.v && (ia < ib || a <= b)) {
                const double val = accP[n][e];
                const size_t vv = (size_t)A.v * A.v;
                A.R[((size_t)i * A.o + j) * vv + (size_t)a * A.v + b] = val;
                A.R[((size_t)i * A.o + j) * vv + (size_t)b * A.v + a] = val;
                A.R[((size_t)j * A.o + i) * vv + (size_t)b * A.v + a] = val;
                A.R[((size_t)j * A.o + i) * vv + (size_t)a * A.v + b] = val;
              }
            }
        }
      }
      __syncthreads();
      {
        const int lam = lm0 + warp * 8 + g;
        if (lam < lm1) {
          int i, j;
          lam_minus(lam, i, j);
#pragma unroll
          for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int a = A0 + n, b = B0 + 2 * q + e;
              if (a < A.v && b < A.v && (ia < ib || a < b)) {
                const double m = accM[n][e];
                const size_t vv = (size_t)A.v * A.v;
                A.R[((size_t)i * A.o + j) * vv + (size_t)a * A.v + b] += m;
                A.R[((size_t)i * A.o + j) * vv + (size_t)b * A.v + a] -= m;
                A.R[((size_t)j * A.o + i) * vv + (size_t)b * A.v + a] += m;
                A.R[((size_t)j * A.o + i) * vv + (size_t)a * A.v + b] -= m;
              }
            }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

int fp64_grid(const Fp64Args &a, int sm_count) {
  int g = a.ntiles < sm_count ? a.ntiles : sm_count;  // one resident CTA per SM
  return g < 1 ? 1 : g;
}

size_t fp64_slab_doubles(int K, int grid) { return (size_t)K / SLOTS * 2 * 64 * SLOTS * grid; }

cudaError_t launch_ladder_fp64(const Fp64Args &a, int grid, cudaStream_t s) {
  const size_t smem = kSmemDoubles * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(ladder_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ladder_fp64_kernel<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ladder
