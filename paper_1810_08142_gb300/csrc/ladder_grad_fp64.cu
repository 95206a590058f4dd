// Gradient of E = sum_ijab W_ij^ab R_ij^ab with respect to the RI factor,
// FP64 (m8n8k4 f64 tensor-core MMAs), for fixed W and tau.
//
// Differentiating (ac|bd) = sum_P B^P_ac B^P_bd (Eq. RIM) inside
// Eq. pp-Ladder-0 gives two terms; with the pair symmetry of W and tau
// (Sec. II.C) they are equal:
//   dB^P_xy = 2 sum_{b,d} Gamma^{xb}_{yd} B^P_bd,
//   Gamma^{xb}_{yd} = sum_ij W_ij^{xb} tau_ij^{yd}.
// One CTA owns an (x-block, y-block) tile of 8 x 8 output pairs.  For every
// (b-block, d-block) it forms the 64 x 64 tile Gamma[(x,y),(b,d)] (K = o^2
// occupied pairs) in shared memory and contracts it with B^P_bd for a chunk
// of 64 auxiliary functions into register accumulators.  Gamma is formed once
// per tile: the first P-chunk spills it to a per-CTA slab and the later
// chunks read it back.
#include "kernels.h"

namespace ladder {
namespace {

constexpr int NT = 256;                 // 8 warps
constexpr int KI = 16;                  // occupied pairs per panel
constexpr int PROW = 2 * 64 + 4;        // panel row: W rows (x,b), tau rows (y,d), padded
constexpr int GSTR = 64 + 4;            // padded row stride of the Gamma and B tiles
constexpr int PC = kGradPChunk;         // auxiliary functions per chunk
constexpr size_t kPanel = (size_t)KI * PROW;
constexpr size_t kSmemDoubles = 2 * kPanel + 64 * GSTR + PC * GSTR;

__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Panel of KI occupied pairs: rows 0-63 W_ij^{x b} (x = X0 + r/8, b = Bb0 + r%8),
// rows 64-127 tau_ij^{y d} (y = Y0 + r/8, d = Dd0 + r%8).
__device__ __forceinline__ void load_panel(double *panel, const GradArgs &A, int ij0, int X0,
                                           int Y0, int Bb0, int Dd0) {
  const int o2 = A.o * A.o;
  for (int e = threadIdx.x; e < KI * 128; e += NT) {
    const int k = e / 128, r = e % 128;
    const int ij = ij0 + k;
    const bool w = r < 64;
    const int rr = w ? r : r - 64;
    const int x = (w ? X0 : Y0) + rr / 8, y = (w ? Bb0 : Dd0) + rr % 8;
    const bool ok = ij < o2 && x < A.v && y < A.v;
    const double *base = w ? A.W : A.tau;
    const double *src = ok ? base + ((size_t)ij * A.v + x) * A.v + y : base;
    cp_async8(panel + k * PROW + r, src, ok ? 8 : 0);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(NT, 1) grad_B_fp64_kernel(const __grid_constant__ GradArgs A) {
  extern __shared__ double smem[];
  double *panels = smem;
  double *G = smem + 2 * kPanel;
  double *Bs = G + 64 * GSTR;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = lane / 4, q = lane % 4;
  const int nb = A.vp / CB, nbd = nb * nb;
  const int npc = (A.N + PC - 1) / PC;
  const int o2 = A.o * A.o;
  const int npan = (o2 + KI - 1) / KI;
  double *slab = A.slab ? A.slab + (size_t)blockIdx.x * nbd * 64 * 64 : nullptr;

  for (int tile = blockIdx.x; tile < nb * nb; tile += gridDim.x) {
    const int X0 = (tile / nb) * CB, Y0 = (tile % nb) * CB;
    for (int pc = 0; pc < npc; ++pc) {
      const int P0 = pc * PC;
      double acc[8][2];
#pragma unroll
      for (int n = 0; n < 8; ++n) acc[n][0] = acc[n][1] = 0.0;
      for (int bd = 0; bd < nbd; ++bd) {
        const int Bb0 = (bd / nb) * CB, Dd0 = (bd % nb) * CB;
        if (pc == 0) {
          // ---- Gamma2[(x,b),(y,d)] over the occupied pairs; warp = x offset
          double c2[8][2];
#pragma unroll
          for (int n = 0; n < 8; ++n) c2[n][0] = c2[n][1] = 0.0;
          load_panel(panels, A, 0, X0, Y0, Bb0, Dd0);
          for (int pan = 0; pan < npan; ++pan) {
            if (pan + 1 < npan) {
              load_panel(panels + ((pan + 1) & 1) * kPanel, A, (pan + 1) * KI, X0, Y0, Bb0, Dd0);
              cp_async_wait<1>();
            } else {
              cp_async_wait<0>();
            }
            __syncthreads();
            const double *pn = panels + (pan & 1) * kPanel;
#pragma unroll
            for (int kk = 0; kk < KI / 4; ++kk) {
              const double *pr = pn + (kk * 4 + q) * PROW;
              const double a = pr[warp * 8 + g];
#pragma unroll
              for (int n = 0; n < 8; ++n) dmma(c2[n][0], c2[n][1], a, pr[64 + n * 8 + g]);
            }
            __syncthreads();
          }
          // fragment (row b = g, col d = 2q + e) of tile (x = warp, y = n)
          // -> Gamma[(x,y)][(b,d)]
#pragma unroll
          for (int n = 0; n < 8; ++n)
#pragma unroll
            for (int e = 0; e < 2; ++e) G[(warp * 8 + n) * GSTR + g * CB + 2 * q + e] = c2[n][e];
          __syncthreads();
          if (slab && npc > 1) {
            double *dst = slab + (size_t)bd * 64 * 64;
            for (int e = tid; e < 64 * 64; e += NT) dst[e] = G[(e / 64) * GSTR + e % 64];
          }
        } else {
          const double *src = slab + (size_t)bd * 64 * 64;
          for (int e = tid; e < 64 * 64; e += NT) G[(e / 64) * GSTR + e % 64] = src[e];
        }
        // ---- B^P_bd for this chunk: Bs[P][(b,d)]
        for (int e = tid; e < PC * 64; e += NT) {
          const int P = P0 + e / 64, s = e % 64;
          const int b = Bb0 + s / CB, d = Dd0 + s % CB;
          const bool ok = P < A.N && b < A.v && d < A.v;
          cp_async8(Bs + (e / 64) * GSTR + s, ok ? A.B + ((size_t)P * A.v + b) * A.v + d : A.B,
                    ok ? 8 : 0);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        // ---- acc[(x,y)][P] += Gamma[(x,y)][(b,d)] B^P_bd; warp = rows 8*warp..
#pragma unroll 4
        for (int kk = 0; kk < 64 / 4; ++kk) {
          const int s = kk * 4 + q;
          const double a = G[(warp * 8 + g) * GSTR + s];
#pragma unroll
          for (int n = 0; n < 8; ++n) dmma(acc[n][0], acc[n][1], a, Bs[(n * 8 + g) * GSTR + s]);
        }
        __syncthreads();
      }
      // ---- dB[P][x][y] = 2 acc; row = (x = X0 + warp, y = Y0 + g), col = P
      const int x = X0 + warp, y = Y0 + g;
      if (x < A.v && y < A.v) {
#pragma unroll
        for (int n = 0; n < 8; ++n)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int P = P0 + n * 8 + 2 * q + e;
            if (P < A.N) A.dB[((size_t)P * A.v + x) * A.v + y] = 2.0 * acc[n][e];
          }
      }
    }
  }
}

}  // namespace

int grad_fp64_grid(int vp, int sm_count) {
  const int nb = vp / CB;
  const int tiles = nb * nb;
  return tiles < sm_count ? tiles : sm_count;
}

size_t grad_fp64_slab_doubles(int vp, int N, int grid) {
  if (N <= kGradPChunk) return 0;
  const size_t nb = (size_t)vp / CB;
  return nb * nb * 64 * 64 * (size_t)grid;
}

cudaError_t launch_grad_B_fp64(const GradArgs &a, int grid, cudaStream_t s) {
  const size_t smem = kSmemDoubles * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(grad_B_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  grad_B_fp64_kernel<<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ladder
