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

#include "kernels.h"

namespace ladder {
namespace {

constexpr int kTE = 256;       // threads per energy block
constexpr int kTPer = 16;      // abc elements per thread

template <typename T>
__global__ void __launch_bounds__(kTE) triples_energy_kernel(const TriplesArgs a, const T *__restrict__ W,
                                                             int i, int j, double *__restrict__ part) {
  __shared__ double red[kTE];
  const int k = blockIdx.y;
  const int v = a.v, o = a.o;
  const long long v3 = (long long)v * v * v;
  const T *Wk = W + (long long)k * v3;
  const T *oovv = static_cast<const T *>(a.oovv);
  const T *Ijk = oovv + ((long long)j * o + k) * v * v;  // v_jk^bc at [b][c]
  const T *Iik = oovv + ((long long)i * o + k) * v * v;  // v_ik^ac at [a][c]
  const T *Iij = oovv + ((long long)i * o + j) * v * v;  // v_ij^ab at [a][b]
  const double *ti = a.t1 + (long long)i * v, *tj = a.t1 + (long long)j * v, *tk = a.t1 + (long long)k * v;
  // terms in T (FP32 mode: the FP64 pipe is scarce on this part), sums in FP64
  const T eijk = (T)(a.e_occ[i] + a.e_occ[j] + a.e_occ[k]);
  double s = 0.0;
  const long long e0 = ((long long)blockIdx.x * kTE * kTPer);
  for (int r = 0; r < kTPer; ++r) {
    const long long e = e0 + (long long)r * kTE + threadIdx.x;
    if (e >= v3) break;
    const int aa = (int)(e / ((long long)v * v)), bb = (int)((e / v) % v), cc = (int)(e % v);
    const T wabc = Wk[e];
    const T wbca = Wk[((long long)bb * v + cc) * v + aa];
    const T wcab = Wk[((long long)cc * v + aa) * v + bb];
    const T wcba = Wk[((long long)cc * v + bb) * v + aa];
    const T vabc = wabc + Ijk[(long long)bb * v + cc] * (T)ti[aa] + Iik[(long long)aa * v + cc] * (T)tj[bb] +
                   Iij[(long long)aa * v + bb] * (T)tk[cc];
    const T vcba = wcba + Ijk[(long long)bb * v + aa] * (T)ti[cc] + Iik[(long long)cc * v + aa] * (T)tj[bb] +
                   Iij[(long long)cc * v + bb] * (T)tk[aa];
    const T D = eijk - (T)a.e_vir[aa] - (T)a.e_vir[bb] - (T)a.e_vir[cc];
    s += (double)((T(4) * wabc + wbca + wcab) * (vabc - vcba) / (T(3) * D));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kTE / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    part[(((long long)i * o + j) * o + k) * gridDim.x + blockIdx.x] = red[0];
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
  const long long v3 = (long long)v * v * v;
  return (int)((v3 + (long long)kTE * kTPer - 1) / ((long long)kTE * kTPer));
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
