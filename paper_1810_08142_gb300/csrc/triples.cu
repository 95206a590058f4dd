// Perturbative triples (Sec. II.A): the energy kernels.
//
//   E(T) = sum_ijk sum_abc (4 W_ijk^abc + W_ijk^bca + W_ijk^cab)
//                          (V_ijk^abc - V_ijk^cba) / (3 D_ijk^abc)
//   V_ijk^abc = W_ijk^abc + v_jk^bc t_i^a + v_ik^ac t_j^b + v_ij^ab t_k^c
//   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c
//
// W_ijk^abc itself (the permutation operator P over the six orderings of the
// two contractions of Sec. II.A, one two-segment GEMM per ordering) is
// accumulated by the CUDA-core GEMM of dress.cu or the tensor-core GEMM of
// triples_tc.cu, for one (i, j) with i >= j and every k <= j at a time, into
// W[k][a][b][c].  These kernels read that W, form V from it and the
// integrals v_jk^bc = (bj|ck) (stored [j][k][b][c]), and reduce the energy of
// the sorted triples in a fixed order:
//   triples_energy_kernel   one partial sum per (sorted i >= j >= k, block of abc)
//   triples_final_kernel    the partials of all (i, j, k), one block, fixed order
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace ladder {
namespace {

constexpr int kTE = 256;  // threads per energy block
constexpr int kTriplesMaxBlocks = 1024;  // energy blocks per k (each walks several orbits)
constexpr int kTC = 8;    // edge of the (a, b, c) cube of one block

// Sorted triples.  W and V are symmetric under a simultaneous permutation of
// (i, j, k) and (a, b, c), and D is symmetric in each, so the energy of a
// permuted triple is the sum over abc of the same tensors with permuted
// virtual indices.  Relabelling the sum, the factor
//   Z^abc = 4 W^abc + W^bca + W^cab
// is unchanged (the two 3-cycles are conjugate to each other), and V^cba
// becomes V with one of the three transpositions of (a, b, c) applied.  Over
// the six orderings of a triple each transposition comes twice, so
//   sum over the distinct orderings of (i, j, k) of E_ijk
//     = m_ijk sum_abc Z^abc (3 V^abc - V^acb - V^bac - V^cba) / (3 D^abc)
// with m = 2 for i > j > k, 1 for two equal indices, 1/3 for i = j = k.  The
// W contractions then run only for i >= j >= k (a sixth of the triples).
//
// Blocks over (orbits of 8-wide index blocks, k <= j), each block walking
// orbits blockIdx.x, blockIdx.x + gridDim.x, ... (at most kTriplesMaxBlocks
// blocks per k, so the partials stay bounded).  An orbit is a
// sorted block triple A0 <= B0 <= C0 with its distinct orderings (6, 3 or
// 1): the elements (a, b, c) of every ordering's 8x8x8 cube need W only at
// the six index permutations of (a, b, c), and those lie in the cubes of the
// same orbit.  The block therefore copies each of the orbit's cubes of W[k]
// into shared memory once (coalesced rows of 8) and reads every permuted W
// from there, so W is read from memory once per k instead of six times.
// One partial sum per block, reduced in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kTE) triples_energy_kernel(const TriplesArgs a, const T *__restrict__ W,
                                                             int i, int j, double *__restrict__ part) {
  constexpr int kCube = kTC * kTC * kTC;
  __shared__ double red[kTE / 32];
  __shared__ int pos[6][3];     // the orbit's distinct block orderings (X0, Y0, Z0)
  __shared__ int cid[6][6];     // cube index of permutation q of position p
  __shared__ int npos;
  // dynamic shared memory: six cubes, then t1 of i, j, k and e_vir (v each)
  extern __shared__ __align__(16) unsigned char tri_smem[];
  T(*cube)[kTC][kTC][kTC + 1] = reinterpret_cast<T(*)[kTC][kTC][kTC + 1]>(tri_smem);
  const int k = blockIdx.y;
  const int v = a.v, o = a.o;
  const int nc = (v + kTC - 1) / kTC;
  T *sti = reinterpret_cast<T *>(tri_smem) + 6 * kTC * kTC * (kTC + 1);
  T *stj = sti + v, *stk = stj + v, *sev = stk + v;
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
  // V^xyz = W^xyz + v_jk^yz t_i^x + v_ik^xz t_j^y + v_ij^xy t_k^z
  auto singles = [&](int x, int y, int z) -> T {
    return Ijk[y * v + z] * sti[x] + Iik[x * v + z] * stj[y] + Iij[x * v + y] * stk[z];
  };
  // the thread's sum: FP64 for T = double; for T = float a double-single
  // (hi, lo) kept with TwoSum on the FP32 pipe (about 48 bits), widened once
  double s = 0.0;
  float sh = 0.f, sl = 0.f;
  const int norb = nc * (nc + 1) * (nc + 2) / 6;
  for (int orb = blockIdx.x; orb < norb; orb += gridDim.x) {
    __syncthreads();  // the previous orbit's cubes and tables are no longer read
    if (threadIdx.x == 0) {
      // orbit -> sorted block triple (A, B, C), A <= B <= C
      int rem = orb, A = 0, B = 0, C = 0;
      for (A = 0; A < nc; ++A) {
        const int m = nc - A, cnt = m * (m + 1) / 2;  // pairs B <= C in [A, nc)
        if (rem < cnt) break;
        rem -= cnt;
      }
      for (B = A; B < nc; ++B) {
        const int cnt = nc - B;
        if (rem < cnt) break;
        rem -= cnt;
      }
      C = B + rem;
      const int t3[3] = {A, B, C};
      static constexpr int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
      int n = 0;
      for (int q = 0; q < 6; ++q) {
        const int x = t3[P[q][0]], y = t3[P[q][1]], z = t3[P[q][2]];
        bool seen = false;
        for (int r = 0; r < n; ++r) seen |= pos[r][0] == x && pos[r][1] == y && pos[r][2] == z;
        if (!seen) {
          pos[n][0] = x;
          pos[n][1] = y;
          pos[n][2] = z;
          ++n;
        }
      }
      npos = n;
      // for position (X, Y, Z): the cubes (X,Y,Z), (Y,Z,X), (Z,X,Y), (X,Z,Y), (Y,X,Z), (Z,Y,X)
      for (int p = 0; p < n; ++p) {
        const int X = pos[p][0], Y = pos[p][1], Z = pos[p][2];
        const int want[6][3] = {{X, Y, Z}, {Y, Z, X}, {Z, X, Y}, {X, Z, Y}, {Y, X, Z}, {Z, Y, X}};
        for (int q = 0; q < 6; ++q)
          for (int r = 0; r < n; ++r)
            if (pos[r][0] == want[q][0] && pos[r][1] == want[q][1] && pos[r][2] == want[q][2]) cid[p][q] = r;
      }
    }
    __syncthreads();
    const int n = npos;
    // the orbit's cubes: thread t copies elements t and t + 256 of each
    for (int p = 0; p < n; ++p) {
      const int X0 = pos[p][0] * kTC, Y0 = pos[p][1] * kTC, Z0 = pos[p][2] * kTC;
  #pragma unroll
      for (int h = 0; h < kCube / kTE; ++h) {
        const int e = threadIdx.x + h * kTE;
        const int x = e / (kTC * kTC), y = (e / kTC) % kTC, z = e % kTC;
        const int X = X0 + x, Y = Y0 + y, Z = Z0 + z;
        cube[p][x][y][z] = (X < v && Y < v && Z < v) ? Wk[(long long)X * vv + (long long)Y * v + Z] : T(0);
      }
    }
    __syncthreads();
    for (int p = 0; p < n; ++p) {
      const int X0 = pos[p][0] * kTC, Y0 = pos[p][1] * kTC, Z0 = pos[p][2] * kTC;
      const int c0 = cid[p][0], c1 = cid[p][1], c2 = cid[p][2], c3 = cid[p][3], c4 = cid[p][4], c5 = cid[p][5];
  #pragma unroll
      for (int h = 0; h < kCube / kTE; ++h) {
        const int e = threadIdx.x + h * kTE;
        const int al = e / (kTC * kTC), bl = (e / kTC) % kTC, cl = e % kTC;
        const int aa = X0 + al, bb = Y0 + bl, cc = Z0 + cl;
        if (aa >= v || bb >= v || cc >= v) continue;
        const T wabc = cube[c0][al][bl][cl];
        const T wbca = cube[c1][bl][cl][al];
        const T wcab = cube[c2][cl][al][bl];
        const T wacb = cube[c3][al][cl][bl];
        const T wbac = cube[c4][bl][al][cl];
        const T wcba = cube[c5][cl][bl][al];
        const T vabc = wabc + singles(aa, bb, cc);
        const T vacb = wacb + singles(aa, cc, bb);
        const T vbac = wbac + singles(bb, aa, cc);
        const T vcba = wcba + singles(cc, bb, aa);
        const T D = eijk - sev[aa] - sev[bb] - sev[cc];
        const T term = (T(4) * wabc + wbca + wcab) * (T(3) * vabc - vacb - vbac - vcba) / (T(3) * D);
        if constexpr (std::is_same<T, float>::value) {
          const float t = __fadd_rn(sh, term), bp = __fsub_rn(t, sh);
          sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(term, bp)));
          sh = t;
        } else {
          s += (double)term;
        }
      }
    }
  }  // orbits
  if constexpr (std::is_same<T, float>::value) s = (double)sh + (double)sl;
  // fixed-order reduction: warp shuffles, then the warps' sums in order
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kTE / 32; ++w) t += red[w];
    // multiplicity of the sorted triple (i >= j >= k)
    const double m = (i == k) ? 1.0 / 3.0 : (i == j || j == k) ? 1.0 : 2.0;
    part[(((long long)i * o + j) * o + k) * gridDim.x + blockIdx.x] = m * t;
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

// dst[g][x][y][d] = src[g][y][x][d]; consecutive threads take consecutive d
template <typename T>
__global__ void triples_swap12_kernel(const T *__restrict__ src, T *__restrict__ dst, long long n, int v) {
  const long long vv = (long long)v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long g = e / (vv * v), r = e % (vv * v);
    const long long x = r / vv, y = (r / v) % v, d = r % v;
    dst[e] = src[g * vv * v + (y * v + x) * v + d];
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

// dynamic shared memory of the energy kernel for v virtual orbitals
template <typename T>
size_t triples_energy_smem(int v) {
  return (6 * kTC * kTC * (kTC + 1) + 4 * (size_t)v) * sizeof(T);
}

}  // namespace

// orbits of sorted 8-wide block triples
int triples_energy_blocks(int v) {
  const int nc = (v + kTC - 1) / kTC;
  return std::min(nc * (nc + 1) * (nc + 2) / 6, kTriplesMaxBlocks);
}

template <typename T>
cudaError_t launch_triples_energy(const TriplesArgs &a, const T *W, int i, int j, double *part,
                                  cudaStream_t s) {
  // k = 0 .. j of the sorted triples i >= j >= k
  const dim3 grid((unsigned)triples_energy_blocks(a.v), (unsigned)(j + 1));
  const size_t smem = triples_energy_smem<T>(a.v);
  if (smem > 48 * 1024) {  // FP64 at large v only; set on the current device
    const cudaError_t e =
        cudaFuncSetAttribute(triples_energy_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  triples_energy_kernel<T><<<grid, kTE, smem, s>>>(a, W, i, j, part);
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
cudaError_t launch_triples_swap12(const T *src, T *dst, int G, int v, cudaStream_t s) {
  const long long n = (long long)G * v * v * v;
  const long long blocks = std::min<long long>((n + 255) / 256, 152 * 64);
  if (blocks > 0) triples_swap12_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(src, dst, n, v);
  return cudaGetLastError();
}
template cudaError_t launch_triples_swap12<double>(const double *, double *, int, int, cudaStream_t);
template cudaError_t launch_triples_swap12<float>(const float *, float *, int, int, cudaStream_t);

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
