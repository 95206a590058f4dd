// t1-dressed ladder (Eq. pp-Ladder-2 with Eq. pp-Ladder-21).
//
// The dressed integrals are
//   b^{ab}_{cd} = sum_P m^P_ac (m^P_bd - mbar^P_bd) - sum_k t_k^a v^{kb}_{cd},
//   mbar^P_bd   = sum_k m^P_kd t_k^b,
// with v^{kb}_{cd} = (kc|bd) = sum_P m^P_kc m^P_bd from the same RI factors.
// Since sum_k t_k^a v^{kb}_{cd} = sum_P mbar^P_ac m^P_bd, completing the
// square gives
//   b^{ab}_{cd} = sum_P Bd^P_ac Bd^P_bd - sum_P mbar^P_ac mbar^P_bd,   Bd = B - mbar,
// so the dressed term is the undressed ladder of Bd (the fused / two-pass
// kernels unchanged, with Bd for B) minus a correction of rank o in each
// virtual index:
//   C_ij^ab = sum_kl t_k^a t_l^b X_ij^kl,
//   X_ij^kl = sum_cd G[(k,l)][(c,d)] tau_ij^cd,   G[(k,l)][(c,d)] = (kc|ld) = sum_P m^P_kc m^P_ld.
// G costs 2 (ov)^2 N flops (half of it with its symmetry), X 2 o^4 v^2: both
// O(o^2 v^2 N + o^4 v^2), against the ladder's O(v^4 N + o^2 v^4).
//
// The GEMM kernel also serves the perturbative triples (triples.cu), whose
// W terms it accumulates with the kEpiAcc3 epilogue.
//
// This file holds the two kernels of the dressing:
//   gemm_kernel     a CUDA-core GEMM C(m,n) = sum_k A(m,k) B(n,k) with free
//                   strides, split-K / batch in z, and four epilogues; it
//                   forms Bd = B - mbar (one v x v product per P, K = o),
//                   (kc|ld), X and the two t1 contractions of the correction
//   reduce_kernel   sums split-K partials
// T is double for the FP64 path, DS (double-single on the FP32 pipe, about
// 48 bits) for the error-free mode, and float for the split-BF16 paths (the
// correction is about 1e-4 of R there, so FP32 keeps it far inside their
// tolerance).
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace ladder {
namespace {

// ---------------------------------------------------------------- double-single
// h + l, an unevaluated sum of two floats.  A product keeps the rounding error
// of h h' (an FMA gives it exactly) and the cross terms in its low word; a sum
// adds the high words with Knuth's TwoSum and collects that error and the low
// words in the low word, without renormalising: the accumulation of a dot
// product is then the compensated Dot2 of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26, 2005), as accurate as a dot product in about 48 bits.  Values
// are renormalised (Dekker's Fast2Sum) only where they are stored.
__device__ __forceinline__ DS ds_make(double x) {
  DS r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - (double)r.h);
  return r;
}
__device__ __forceinline__ DS ds_norm(float s, float e) {
  DS r;
  r.h = __fadd_rn(s, e);
  r.l = __fsub_rn(e, __fsub_rn(r.h, s));
  return r;
}
__device__ __forceinline__ DS operator*(DS a, DS b) {
  DS r;
  r.h = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -r.h);
  e = __fmaf_rn(a.h, b.l, e);
  r.l = __fmaf_rn(a.l, b.h, e);
  return r;
}
__device__ __forceinline__ DS operator+(DS a, DS b) {
  DS r;
  r.h = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(r.h, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(r.h, bb)), __fsub_rn(b.h, bb));
  r.l = __fadd_rn(__fadd_rn(a.l, b.l), e);
  return r;
}
__device__ __forceinline__ DS &operator+=(DS &a, DS b) { return a = a + b; }
__device__ __forceinline__ DS &operator*=(DS &a, DS b) { return a = a * b; }
// conversions between the GEMM's types
template <typename T> __device__ __forceinline__ T to_t(double x) { return (T)x; }
template <> __device__ __forceinline__ DS to_t<DS>(double x) { return ds_make(x); }
template <typename T> __device__ __forceinline__ T to_t(float x) { return (T)x; }
template <typename T> __device__ __forceinline__ T to_t(DS x) { return (T)((double)x.h + (double)x.l); }
template <> __device__ __forceinline__ DS to_t<DS>(DS x) { return x; }
// the value as stored: a double-single renormalised (|l| <= ulp(h) / 2)
template <typename T> __device__ __forceinline__ T ds_store(T x) { return x; }
template <> __device__ __forceinline__ DS ds_store<DS>(DS x) { return ds_norm(x.h, x.l); }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return x; }
__device__ __forceinline__ double to_double(DS x) { return (double)x.h + (double)x.l; }

// ---------------------------------------------------------------- CUDA-core GEMM
constexpr int kBM = 128, kBN = 128, kBK = 8;
constexpr int kPadF = 4;  // row padding of the shared tiles (elements)

__device__ __forceinline__ void load4(const float *p, float *r) {
  const float4 x = *reinterpret_cast<const float4 *>(p);
  r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
}
__device__ __forceinline__ void load4(const double *p, double *r) {
  const double2 x = *reinterpret_cast<const double2 *>(p);
  const double2 y = *reinterpret_cast<const double2 *>(p + 2);
  r[0] = x.x; r[1] = x.y; r[2] = y.x; r[3] = y.y;
}
__device__ __forceinline__ void load4(const DS *p, DS *r) {
  const float4 x = *reinterpret_cast<const float4 *>(p);
  const float4 y = *reinterpret_cast<const float4 *>(p + 2);
  r[0].h = x.x; r[0].l = x.y; r[1].h = x.z; r[1].l = x.w;
  r[2].h = y.x; r[2].l = y.y; r[3].h = y.z; r[3].l = y.w;
}

// Operand loader: element (row, k) of a [rows x K] operand at
// base[row * srow + k * sk].  Each thread stages four elements per K-step;
// the mapping keeps whichever index is contiguous in memory on adjacent
// threads.
template <typename TM, typename T>
__device__ __forceinline__ void gemm_fetch(const TM *__restrict__ base, long long srow,
                                           long long sk, int rows, int row0, int k0, int kend,
                                           bool kfast, T (&reg)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = threadIdx.x + 256 * r;
    const int rr = kfast ? e / kBK : e % kBM;
    const int kk = kfast ? e % kBK : e / kBM;
    const int row = row0 + rr, k = k0 + kk;
    reg[r] = (row < rows && k < kend) ? to_t<T>(base[(long long)row * srow + (long long)k * sk]) : to_t<T>(0.0);
  }
}
template <typename T>
__device__ __forceinline__ void gemm_stage(T (*tile)[kBM + kPadF], bool kfast, const T (&reg)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = threadIdx.x + 256 * r;
    const int rr = kfast ? e / kBK : e % kBM;
    const int kk = kfast ? e % kBK : e / kBM;
    tile[kk][rr] = reg[r];
  }
}

template <int N>
__device__ __forceinline__ void cp_async_n(void *smem, const void *gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(N), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename TA, typename TB, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) gemm_kernel(const GemmArgs g) {
  // Operands already in the accumulation type are copied global -> shared
  // with cp.async into a ring of kStg tiles; the others are converted in
  // registers on the way (two tiles).  One buffer holds both rings; the
  // row-major epilogue reuses it.
  constexpr bool kAsync = std::is_same<TA, T>::value && std::is_same<TB, T>::value;
  constexpr int kStg = (kAsync && sizeof(T) == 4) ? 3 : 2;
  __shared__ __align__(16) T sAB[kStg * 2 * kBK * (kBM + kPadF)];
  T(*sA)[kBK][kBM + kPadF] = reinterpret_cast<T(*)[kBK][kBM + kPadF]>(sAB);
  T(*sB)[kBK][kBN + kPadF] = reinterpret_cast<T(*)[kBK][kBN + kPadF]>(sAB + kStg * kBK * (kBM + kPadF));
  int mt, nt;
  if (g.sym) {
    // upper triangle of tiles only (mt <= nt); the epilogue mirrors
    int t = blockIdx.x, r = 0, w = g.ntn;
    while (t >= w) { t -= w; ++r; --w; }
    mt = r;
    nt = r + t;
  } else {
    mt = blockIdx.x / g.ntn;
    nt = blockIdx.x % g.ntn;
  }
  const int z = blockIdx.z + g.zoff;
  const int batch = z / g.ksplit, split = z % g.ksplit;
  const int k0 = split * g.kchunk, k1 = min(g.K, k0 + g.kchunk);
  const TA *A = static_cast<const TA *>(g.A) + (long long)batch * g.sa_batch;
  const TB *Bm = static_cast<const TB *>(g.B) + (long long)batch * g.sb_batch;
  const bool akf = g.sak == 1, bkf = g.sbk == 1;
  const int m0 = mt * kBM, n0 = nt * kBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = to_t<T>(0.0);

  // an optional second K segment (A2, B2, K2; B2 scaled by beta2) follows
  // the first in the same accumulators
  const TA *A2 = static_cast<const TA *>(g.A2) + (long long)batch * g.sa2_batch;
  const TB *B2 = static_cast<const TB *>(g.B2) + (long long)batch * g.sb2_batch;
  const bool akf2 = g.sak2 == 1, bkf2 = g.sbk2 == 1;
  T ra[4], rb[4];
  const int nkt1 = k1 > k0 ? (k1 - k0 + kBK - 1) / kBK : 0;
  const int nkt2 = g.A2 ? (g.K2 + kBK - 1) / kBK : 0;
  const int nkt = nkt1 + nkt2;
  auto fetch = [&](int kt) -> bool {  // true: a tile of the second segment
    if (kt < nkt1) {
      gemm_fetch(A, g.sam, g.sak, g.M, m0, k0 + kt * kBK, k1, akf, ra);
      gemm_fetch(Bm, g.sbn, g.sbk, g.N, n0, k0 + kt * kBK, k1, bkf, rb);
      return false;
    }
    const int kk = (kt - nkt1) * kBK;
    gemm_fetch(A2, g.sam2, g.sak2, g.M, m0, kk, g.K2, akf2, ra);
    gemm_fetch(B2, g.sbn2, g.sbk2, g.N, n0, kk, g.K2, bkf2, rb);
#pragma unroll
    for (int r = 0; r < 4; ++r) rb[r] *= to_t<T>(g.beta2);
    return true;
  };
  auto stage = [&](int buf, bool seg2) {
    gemm_stage(sA[buf], seg2 ? akf2 : akf, ra);
    gemm_stage(sB[buf], seg2 ? bkf2 : bkf, rb);
  };
  auto mma_tile = [&](int buf) {
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      T a[8], b[8];
      load4(&sA[buf][kk][ty * 4], a);
      load4(&sA[buf][kk][64 + ty * 4], a + 4);
      load4(&sB[buf][kk][tx * 4], b);
      load4(&sB[buf][kk][64 + tx * 4], b + 4);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
    }
  };
  if constexpr (kAsync) {
    // (the second segment's B is used unscaled on this path: beta2 must be 1)
    auto issue = [&](int kt, int st) {
      const bool seg2 = kt >= nkt1;
      const T *Ab = seg2 ? reinterpret_cast<const T *>(A2) : reinterpret_cast<const T *>(A);
      const T *Bb = seg2 ? reinterpret_cast<const T *>(B2) : reinterpret_cast<const T *>(Bm);
      const long long am = seg2 ? g.sam2 : g.sam, ak = seg2 ? g.sak2 : g.sak;
      const long long bn = seg2 ? g.sbn2 : g.sbn, bk = seg2 ? g.sbk2 : g.sbk;
      const bool af = seg2 ? akf2 : akf, bf = seg2 ? bkf2 : bkf;
      const int kb = seg2 ? (kt - nkt1) * kBK : k0 + kt * kBK;
      const int ke = seg2 ? g.K2 : k1;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = threadIdx.x + 256 * r;
        int rr = af ? e / kBK : e % kBM, kk = af ? e % kBK : e / kBM;
        int row = m0 + rr, k = kb + kk;
        bool ok = row < g.M && k < ke;
        cp_async_n<sizeof(T)>(&sA[st][kk][rr], ok ? Ab + (long long)row * am + (long long)k * ak : Ab,
                              ok ? (int)sizeof(T) : 0);
        rr = bf ? e / kBK : e % kBN;
        kk = bf ? e % kBK : e / kBN;
        row = n0 + rr;
        k = kb + kk;
        ok = row < g.N && k < ke;
        cp_async_n<sizeof(T)>(&sB[st][kk][rr], ok ? Bb + (long long)row * bn + (long long)k * bk : Bb,
                              ok ? (int)sizeof(T) : 0);
      }
    };
#pragma unroll
    for (int st = 0; st < kStg - 1; ++st) {
      if (st < nkt) issue(st, st);
      cp_async_commit_group();
    }
    for (int kt = 0; kt < nkt; ++kt) {
      cp_async_wait_group<kStg - 2>();  // tile kt has landed
      __syncthreads();                  // ... for every thread; tile kt - 1 is free
      const int nx = kt + kStg - 1;
      if (nx < nkt) issue(nx, nx % kStg);
      cp_async_commit_group();
      mma_tile(kt % kStg);
    }
    cp_async_wait_group<0>();
    __syncthreads();
  } else {
    if (nkt > 0) stage(0, fetch(0));
    __syncthreads();
    for (int kt = 0; kt < nkt; ++kt) {
      const int buf = kt & 1;
      bool seg2 = false;
      if (kt + 1 < nkt) seg2 = fetch(kt + 1);
      mma_tile(buf);
      if (kt + 1 < nkt) stage(buf ^ 1, seg2);
      __syncthreads();
    }
  }

  if (g.epi == kEpiAcc3 && g.s2 == 1 && g.s3 != 1) {
    // the output's contiguous index is the row's (m % pv): stage 32-row slabs
    // of the tile in shared memory and walk them rows fastest, so a warp's
    // read-modify-writes fall on consecutive addresses
    static_assert(32 * (kBN + 1) <= 2 * 2 * kBK * (kBM + kPadF), "stage fits the operand rings");
    T *stage = sAB;
    T *O = static_cast<T *>(g.Out) + (long long)batch * g.so_batch;
    const T alpha = to_t<T>(g.alpha);
    for (int sl = 0; sl < 4; ++sl) {
      // rows 32 sl .. 32 sl + 31 belong to ty in [8 (sl & 1), 8 (sl & 1) + 8), half sl >> 1
      if ((ty >> 3) == (sl & 1)) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = ((sl >> 1) ? 64 : 0) + ty * 4 + i - 32 * sl;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4);
            stage[r * (kBN + 1) + c] = ds_store(acc[(sl >> 1) ? 4 + i : i][j]);
          }
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * kBN; e += 256) {
        const int rl = e % 32, c = e / 32;
        const int m = m0 + 32 * sl + rl, n = n0 + c;
        if (m < g.M && n < g.N) {
          T *w = O + (long long)(m / g.pv) * g.s1 + (long long)(m % g.pv) + (long long)n * g.s3;
          const T x = alpha * stage[rl * (kBN + 1) + c];
          *w = g.acc ? *w + x : x;
        }
      }
      __syncthreads();
    }
    return;
  }
  // epilogue: thread rows ty*4+i (i<4) and 64+ty*4+i, columns likewise with tx
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (n >= g.N) continue;
      const T val = ds_store(acc[i][j]);
      if (g.epi == kEpiStore) {
        static_cast<T *>(g.Out)[(long long)z * g.so_batch + (long long)m * g.ldo + n] = val;
      } else if (g.epi == kEpiPerm) {
        // m = (k, c), n = (l, d) -> G[(k, l)][(c, d)]; mirrored for the symmetric product
        const int pn = g.pn ? g.pn : g.pv;
        const int k = m / g.pv, c = m % g.pv, l = n / pn, d = n % pn;
        T *G = static_cast<T *>(g.Out);
        const long long cd = (long long)g.pv * pn;
        G[((long long)k * g.po + l) * cd + (long long)c * pn + d] = val;
        if (g.sym) G[((long long)l * g.po + k) * cd + (long long)d * pn + c] = val;
      } else if (g.epi == kEpiAcc3) {
        T *O = static_cast<T *>(g.Out) + (long long)batch * g.so_batch + (long long)(m / g.pv) * g.s1 +
               (long long)(m % g.pv) * g.s2 + (long long)n * g.s3;
        const T x = to_t<T>(g.alpha) * val;
        *O = g.acc ? *O + x : x;
      } else if (g.epi == kEpiSubR) {  // R -= val (FP64 result)
        double *R = static_cast<double *>(g.Out);
        R[(long long)batch * g.so_batch + (long long)m * g.ldo + n] -= to_double(val);
      } else {  // kEpiFromSrc: Out = Src - val (FP64)
        const long long at = (long long)batch * g.so_batch + (long long)m * g.ldo + n;
        static_cast<double *>(g.Out)[at] = g.Src[at] - to_double(val);
      }
    }
  }
}

template <typename T>
__global__ void reduce_kernel(T *__restrict__ X, long long n, int parts) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    T s = X[e];
    for (int p = 1; p < parts; ++p) s += X[(long long)p * n + e];
    X[e] = ds_store(s);
  }
}

}  // namespace

template <typename TA, typename TB, typename T>
cudaError_t launch_gemm(const GemmArgs &g, int batch, cudaStream_t s) {
  GemmArgs a = g;
  a.ntm = (a.M + kBM - 1) / kBM;
  a.ntn = (a.N + kBN - 1) / kBN;
  if (a.ksplit < 1) a.ksplit = 1;
  if (a.kchunk < 1) a.kchunk = a.K;
  if (a.sym && a.M != a.N) return cudaErrorInvalidValue;
  const long long tiles = a.sym ? (long long)a.ntm * (a.ntm + 1) / 2 : (long long)a.ntm * a.ntn;
  const long long nz = (long long)batch * a.ksplit;
  if (tiles == 0 || nz == 0) return cudaSuccess;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  // z = batch * ksplit + split, launched in slices of at most 65535
  for (long long z0 = 0; z0 < nz; z0 += 65535) {
    a.zoff = (int)z0;
    const dim3 grid((unsigned)tiles, 1, (unsigned)std::min<long long>(65535, nz - z0));
    gemm_kernel<TA, TB, T><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}
template cudaError_t launch_gemm<double, double, double>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<double, double, float>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<double, float, float>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<float, double, float>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<float, float, float>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<double, double, DS>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<double, DS, DS>(const GemmArgs &, int, cudaStream_t);
template cudaError_t launch_gemm<DS, double, DS>(const GemmArgs &, int, cudaStream_t);

template <typename T>
cudaError_t launch_reduce(T *X, long long n, int parts, cudaStream_t s) {
  if (parts <= 1 || n == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  reduce_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X, n, parts);
  return cudaGetLastError();
}
template cudaError_t launch_reduce<double>(double *, long long, int, cudaStream_t);
template cudaError_t launch_reduce<float>(float *, long long, int, cudaStream_t);
template cudaError_t launch_reduce<DS>(DS *, long long, int, cudaStream_t);

}  // namespace ladder
