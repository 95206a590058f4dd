// Perturbative triples (Sec. II.A): the energy kernels.
//
//   E(T) = sum_ijk sum_abc (4 W_ijk^abc + W_ijk^bca + W_ijk^cab)
//                          (V_ijk^abc - V_ijk^cba) / (3 D_ijk^abc)
//   V_ijk^abc = W_ijk^abc + v_jk^bc t_i^a + v_ik^ac t_j^b + v_ij^ab t_k^c
//   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c
//
// W_ijk^abc itself (the permutation operator P over the six orderings of the
// two contractions of Sec. II.A, one two-segment GEMM per ordering) is
// accumulated by the CUDA-core GEMM of dress.cu, for one (i, j) and every k
// at a time, into W[k][a][b][c].  These
// kernels read that W, form V from it and the integrals v_jk^bc = (bj|ck)
// (stored [j][k][b][c]), and reduce the energy in a fixed order:
//   triples_energy_kernel   one partial sum per (i, j, k, block of abc)
//   triples_final_kernel    the partials of all (i, j, k), one block, fixed order
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace ladder {
namespace {

constexpr int kTE = 256;  // threads per energy block
constexpr int kTC = 8;    // edge of the (a, b, c) cube of one block

// One block per (8x8 (a, b) tile, k), walking the 8-wide blocks of c: for
// each 8x8x8 cube the three permuted sub-cubes of W the terms need (W^bca,
// W^cab, W^cba of the cube live in the cubes (b, c, a), (c, a, b) and
// (c, b, a) of W) are first copied into shared memory with coalesced reads
// (the last index is contiguous in both), so that no thread gathers W at a
// stride of v or v^2.  One partial sum per block, reduced in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kTE) triples_energy_kernel(const TriplesArgs a, const T *__restrict__ W,
                                                             int i, int j, double *__restrict__ part) {
  __shared__ T cube[3][kTC][kTC][kTC + 1];
  __shared__ double red[kTE / 32];
  __shared__ T sti[kTriplesMaxV], stj[kTriplesMaxV], stk[kTriplesMaxV], sev[kTriplesMaxV];
  const int k = blockIdx.y;
  const int v = a.v, o = a.o;
  const int nc = (v + kTC - 1) / kTC;
  const int A0 = (int)(blockIdx.x / nc) * kTC, B0 = (int)(blockIdx.x % nc) * kTC;
  const long long vv = (long long)v * v, v3 = vv * v;
  const T *Wk = W + (long long)k * v3;
  const T *oovv = static_cast<const T *>(a.oovv);
  const T *Ijk = oovv + ((long long)j * o + k) * vv;  // v_jk^bc at [b][c]
  const T *Iik = oovv + ((long long)i * o + k) * vv;  // v_ik^ac at [a][c]
  const T *Iij = oovv + ((long long)i * o + j) * vv;  // v_ij^ab at [a][b]
  // terms in T (FP32 mode: the FP64 pipe is scarce on this part, so the
  // singles and orbital energies are converted once per block), sums in FP64
  for (int x = threadIdx.x; x < v; x += kTE) {
    sti[x] = (T)a.t1[(long long)i * v + x];
    stj[x] = (T)a.t1[(long long)j * v + x];
    stk[x] = (T)a.t1[(long long)k * v + x];
    sev[x] = (T)a.e_vir[x];
  }
  const T eijk = (T)(a.e_occ[i] + a.e_occ[j] + a.e_occ[k]);
  // the thread's sum: FP64 for T = double; for T = float a double-single
  // (hi, lo) kept with TwoSum on the FP32 pipe (about 48 bits), widened once
  double s = 0.0;
  float sh = 0.f, sl = 0.f;
  for (int C0 = 0; C0 < v; C0 += kTC) {
    // cube q holds W[X0 + x][Y0 + y][Z0 + z] at [x][y][z]:
    //   q = 0: (X, Y, Z) = (B, C, A);  q = 1: (C, A, B);  q = 2: (C, B, A)
    for (int t = threadIdx.x; t < 3 * kTC * kTC * kTC; t += kTE) {
      const int q = t / (kTC * kTC * kTC), r = t % (kTC * kTC * kTC);
      const int x = r / (kTC * kTC), y = (r / kTC) % kTC, z = r % kTC;
      const int X0 = q == 0 ? B0 : C0, Y0 = q == 0 ? C0 : (q == 1 ? A0 : B0), Z0 = q == 1 ? B0 : A0;
      const int X = X0 + x, Y = Y0 + y, Z = Z0 + z;
      cube[q][x][y][z] = (X < v && Y < v && Z < v) ? Wk[(long long)X * vv + (long long)Y * v + Z] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < kTC * kTC * kTC; r += kTE) {
      const int al = r / (kTC * kTC), bl = (r / kTC) % kTC, cl = r % kTC;
      const int aa = A0 + al, bb = B0 + bl, cc = C0 + cl;
      if (aa >= v || bb >= v || cc >= v) continue;
      const T wabc = Wk[(long long)aa * vv + (long long)bb * v + cc];
      const T wbca = cube[0][bl][cl][al];
      const T wcab = cube[1][cl][al][bl];
      const T wcba = cube[2][cl][bl][al];
      const T vabc = wabc + Ijk[(long long)bb * v + cc] * sti[aa] + Iik[(long long)aa * v + cc] * stj[bb] +
                     Iij[(long long)aa * v + bb] * stk[cc];
      const T vcba = wcba + Ijk[(long long)bb * v + aa] * sti[cc] + Iik[(long long)cc * v + aa] * stj[bb] +
                     Iij[(long long)cc * v + bb] * stk[aa];
      const T D = eijk - sev[aa] - sev[bb] - sev[cc];
      const T term = (T(4) * wabc + wbca + wcab) * (vabc - vcba) / (T(3) * D);
      if constexpr (std::is_same<T, float>::value) {
        const float t = __fadd_rn(sh, term), bb = __fsub_rn(t, sh);
        sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(term, bb)));
        sh = t;
      } else {
        s += (double)term;
      }
    }
    __syncthreads();
  }
  if constexpr (std::is_same<T, float>::value) s = (double)sh + (double)sl;
  // fixed-order reduction: warp shuffles, then the warps' sums in order
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kTE / 32; ++w) t += red[w];
    part[(((long long)i * o + j) * o + k) * gridDim.x + blockIdx.x] = t;
  }
}

// t2 in the GEMMs' element type (t2c, skipped when null) and with the two
// virtual indices exchanged (t2T[i][j][b][a] = t2[i][j][a][b]).
template <typename T>
__global__ void triples_t2_kernel(long long n, int v, const double *__restrict__ t2, T *__restrict__ t2c,
                                  T *__restrict__ t2T) {
  const long long vv = (long long)v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double x = t2[e];
    const long long ij = e / vv, ab = e % vv;
    if (t2c) t2c[e] = (T)x;
    t2T[ij * vv + (ab % v) * v + ab / v] = (T)x;
  }
}

template <typename T>
__global__ void triples_negate_kernel(T *__restrict__ x, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = -x[e];
}

// One block: thread t sums partials t, t + 1024, ... in order, then a tree.
// A nonzero *status (a bounded wait of the tensor-core W kernel ran out)
// makes the result NaN.
__global__ void __launch_bounds__(1024) triples_final_kernel(const double *__restrict__ part, long long n,
                                                             double *__restrict__ E, const int *status) {
  __shared__ double red[1024];
  double s = 0.0;
  for (long long q = threadIdx.x; q < n; q += 1024) s += part[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *E = (status && *status) ? __longlong_as_double(0x7ff8000000000000LL) : red[0];
}

}  // namespace

int triples_energy_blocks(int v) {
  const int nc = (v + kTC - 1) / kTC;
  return nc * nc;
}

template <typename T>
cudaError_t launch_triples_energy(const TriplesArgs &a, const T *W, int i, int j, double *part,
                                  cudaStream_t s) {
  const dim3 grid((unsigned)triples_energy_blocks(a.v), (unsigned)a.o);
  triples_energy_kernel<T><<<grid, kTE, 0, s>>>(a, W, i, j, part);
  return cudaGetLastError();
}
template cudaError_t launch_triples_energy<double>(const TriplesArgs &, const double *, int, int, double *,
                                                   cudaStream_t);
template cudaError_t launch_triples_energy<float>(const TriplesArgs &, const float *, int, int, double *,
                                                  cudaStream_t);

template <typename T>
cudaError_t launch_triples_t2(int o, int v, const double *t2, T *t2c, T *t2T, cudaStream_t s) {
  const long long n = (long long)o * o * v * v;
  const long long blocks = std::min<long long>((n + 255) / 256, 8192);
  triples_t2_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(n, v, t2, t2c, t2T);
  return cudaGetLastError();
}
template cudaError_t launch_triples_t2<double>(int, int, const double *, double *, double *, cudaStream_t);
template cudaError_t launch_triples_t2<float>(int, int, const double *, float *, float *, cudaStream_t);

template <typename T>
cudaError_t launch_triples_negate(T *x, long long n, cudaStream_t s) {
  const long long blocks = std::min<long long>((n + 255) / 256, 8192);
  if (blocks > 0) triples_negate_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(x, n);
  return cudaGetLastError();
}
template cudaError_t launch_triples_negate<double>(double *, long long, cudaStream_t);
template cudaError_t launch_triples_negate<float>(float *, long long, cudaStream_t);

cudaError_t launch_triples_final(const double *part, long long n, double *E, cudaStream_t s, const int *status) {
  triples_final_kernel<<<1, 1024, 0, s>>>(part, n, E, status);
  return cudaGetLastError();
}

}  // namespace ladder
