// Preparation and reduction kernels of the ladder path:
//   tau assembly (Eq. pp-Ladder-01), packing of tau into the symmetric and
//   antisymmetric pair combinations (FP64 or BF16 slices), slicing of the RI
//   factor into K-major BF16 slices, and the FP64 ladder energy.
// All of these are bandwidth-bound O(o^2 v^2) or O(N v^2) passes.
#include "common.cuh"
#include "kernels.h"

namespace ladder {

// ---------------------------------------------------------------- tau
// tau_ij^ab = t_ij^ab + t_i^a t_j^b, one thread per (i, j, a, b), FP64.
__global__ void tau_kernel(int o, int v, const double *__restrict__ t1,
                           const double *__restrict__ t2, double *__restrict__ tau) {
  const size_t total = (size_t)o * o * v * v;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    size_t r = idx / v;
    const int a = (int)(r % v);
    r /= v;
    const int j = (int)(r % o);
    const int i = (int)(r / o);
    tau[idx] = t2[idx] + t1[(size_t)i * v + a] * t1[(size_t)j * v + b];
  }
}

void launch_tau(int o, int v, const double *t1, const double *t2, double *tau,
                cudaStream_t s) {
  const size_t total = (size_t)o * o * v * v;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  tau_kernel<<<blocks, 256, 0, s>>>(o, v, t1, t2, tau);
}

// ---------------------------------------------------------------- slices
// x = s0 + s1 + s2 + ..., each s_k the BF16 rounding (to nearest) of what the
// earlier slices leave; the remainders are exact in FP64.
template <int S>
__device__ __forceinline__ void split_bf16(double x, __nv_bfloat16 (&out)[S]) {
#pragma unroll
  for (int k = 0; k < S; ++k) {
    out[k] = __double2bfloat16(x);
    x -= (double)__bfloat162float(out[k]);
  }
}

// ---------------------------------------------------------------- tau pm
// Packed pair combinations, rows = occupied pairs, columns = K slots:
//   Tp[lam+][p*64 + cl*8 + dl] = w_p (tau_ij^cd + tau_ij^dc) / 2   (i <= j)
//   Tm[lam-][p*64 + cl*8 + dl] = w_p (tau_ij^cd - tau_ij^dc) / 2   (i <  j)
// with block pair p = (k, l), c = 8k + cl, d = 8l + dl, w_p = 1/2 for k = l.
// Entries with c or d >= v are zero.  grid.x covers the K slots of one row in
// chunks, grid.y the rows (plus rows first, then minus rows).
// For the BF16 layout the output is [slice][row][K].
// A NaN or infinite tau element records kSiteNonFinite in *status (if given).
template <typename T, int S>
__global__ void pack_tpm_kernel(int o, int v, int K, int nlp, int nlm,
                                const double *__restrict__ tau, T *__restrict__ Tp,
                                T *__restrict__ Tm, size_t slice_stride_p,
                                size_t slice_stride_m, int *status) {
  const int row = blockIdx.y;
  const bool plus = row < nlp;
  int i, j;
  if (plus)
    lam_plus(row, i, j);
  else
    lam_minus(row - nlp, i, j);
  const double *tij = tau + ((size_t)i * o + j) * v * v;
  const int lrow = plus ? row : row - nlp;
  T *dst = plus ? Tp : Tm;
  const size_t sstride = plus ? slice_stride_p : slice_stride_m;
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < K; col += gridDim.x * blockDim.x) {
    const int p = col / SLOTS, s = col % SLOTS;
    int k, l;
    pair_of(p, k, l);
    const int c = k * CB + s / CB, d = l * CB + s % CB;
    double val = 0.0;
    if (c < v && d < v) {
      const double w = (k == l) ? 0.25 : 0.5;
      const double x = tij[(size_t)c * v + d], y = tij[(size_t)d * v + c];
      if (status && !(isfinite(x) && isfinite(y))) record_status(status, kSiteNonFinite);
      val = plus ? w * (x + y) : w * (x - y);
    }
    if constexpr (S == 0) {
      dst[(size_t)lrow * K + col] = (T)val;
    } else {
      __nv_bfloat16 sl[S];
      split_bf16<S>(val, sl);
#pragma unroll
      for (int q = 0; q < S; ++q) dst[q * sstride + (size_t)lrow * K + col] = sl[q];
    }
  }
}

void launch_pack_tpm_f64(int o, int v, int K, const double *tau, double *Tp, double *Tm,
                         cudaStream_t s) {
  const int nlp = ppos(o), nlm = pneg(o);
  dim3 grid((K + 255) / 256 < 64 ? (K + 255) / 256 : 64, nlp + nlm);
  pack_tpm_kernel<double, 0><<<grid, 256, 0, s>>>(o, v, K, nlp, nlm, tau, Tp, Tm, 0, 0, nullptr);
}

void launch_pack_tpm_bf16(int o, int v, int K, int nslices, int rows_p, int rows_m,
                          const double *tau, __nv_bfloat16 *Tp, __nv_bfloat16 *Tm,
                          cudaStream_t s, int *status) {
  const int nlp = ppos(o), nlm = pneg(o);
  dim3 grid((K + 255) / 256 < 64 ? (K + 255) / 256 : 64, nlp + nlm);
  const size_t sp = (size_t)rows_p * K, sm = (size_t)rows_m * K;
  if (nslices == 2)
    pack_tpm_kernel<__nv_bfloat16, 2><<<grid, 256, 0, s>>>(o, v, K, nlp, nlm, tau, Tp, Tm, sp, sm, status);
  else
    pack_tpm_kernel<__nv_bfloat16, 3><<<grid, 256, 0, s>>>(o, v, K, nlp, nlm, tau, Tp, Tm, sp, sm, status);
}

// ---------------------------------------------------------------- tau+- per chunk
// Chunk-major copy of the tau+- slices for the GEMM2 pass of the two-pass
// form: for chunk c, 16-slot piece x and slice s, the chunk's sc rows
// (lambda+ rows, padding, lambda- rows, padding) of 32 bytes each, stored
// contiguously and already in the 32-byte-swizzled order of shared memory
// (the two 16-byte halves of row r swapped when bit 2 of r is set), so one
// bulk copy per piece fills a GEMM2 operand.  Padding rows are zero.
__global__ void pack_t2_kernel(const __grid_constant__ T2Args a) {
  const TcChunk CH = a.chunks[blockIdx.y];
  const int sc = CH.nps + CH.nms;
  const size_t units = (size_t)(a.K / 16) * a.S * sc * 2;
  const uint4 *Tp = reinterpret_cast<const uint4 *>(a.Tp);
  const uint4 *Tm = reinterpret_cast<const uint4 *>(a.Tm);
  uint4 *dst = reinterpret_cast<uint4 *>(a.T2 + a.off[blockIdx.y]);
  const size_t K8 = (size_t)a.K / 8;  // 16-byte units per row of Tp / Tm
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(u & 1);
    size_t t = u >> 1;
    const int row = (int)(t % sc);
    t /= sc;
    const int s = (int)(t % a.S);
    const size_t xp = t / a.S;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (row < CH.np)
      val = Tp[((size_t)s * a.rows_p + CH.lp0 + row) * K8 + xp * 2 + h];
    else if (row >= CH.nps && row - CH.nps < CH.nm)
      val = Tm[((size_t)s * a.rows_m + CH.lm0 + (row - CH.nps)) * K8 + xp * 2 + h];
    dst[((xp * a.S + s) * sc + row) * 2 + (h ^ ((row >> 2) & 1))] = val;
  }
}

void launch_pack_t2(const T2Args &a, cudaStream_t s) {
  dim3 grid(1024, a.nchunks);
  pack_t2_kernel<<<grid, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- lambda-only tau per chunk
// Operand of the lambda-only GEMM2 (T2LamArgs): layout [piece x][plane j][slice
// s][row][32 bytes], rows 32-byte swizzled like pack_t2, so one bulk copy per
// piece fills both planes.  Half h of the row of piece x (block pair (k, l),
// local piece x % 4) holds slots 16 (x % 4) + 8 h + e, i.e. c = 8 k + 2 (x % 4) + h
// and d = 8 l + e for e = 0..7.
template <int S>
__global__ void pack_t2_lam_kernel(const __grid_constant__ T2LamArgs a) {
  const TcChunk CH = a.chunks[blockIdx.y];
  const int sc = CH.nps;
  const size_t units = (size_t)(a.K / 16) * 2 * sc * 2;  // (piece, plane, row, half)
  uint4 *dst = reinterpret_cast<uint4 *>(a.T2 + CH.t2off / 2);
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(u & 1);
    size_t t = u >> 1;
    const int row = (int)(t % sc);
    t /= sc;
    const int j = (int)(t & 1);
    const size_t x = t >> 1;
    int k, l;
    pair_of((int)(x / 4), k, l);
    const int c = k * CB + 2 * (int)(x % 4) + h, d0 = l * CB;
    const double w = (k == l) ? 0.5 : 1.0;
    const bool live = row < CH.np;
    const double *tij = a.tau + (size_t)(live ? CH.lp0 + row : 0) * a.v * a.v;
    __nv_bfloat16 sl[S][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int d = d0 + e;
      double val = 0.0;
      if (live && c < a.v && d < a.v) val = w * (j ? tij[(size_t)d * a.v + c] : tij[(size_t)c * a.v + d]);
      __nv_bfloat16 xs[S];
      split_bf16<S>(val, xs);
#pragma unroll
      for (int q = 0; q < S; ++q) sl[q][e] = xs[q];
    }
#pragma unroll
    for (int q = 0; q < S; ++q)
      dst[(((x * 2 + j) * S + q) * sc + row) * 2 + (h ^ ((row >> 2) & 1))] =
          *reinterpret_cast<const uint4 *>(sl[q]);
  }
}

void launch_pack_t2_lam(const T2LamArgs &a, cudaStream_t s) {
  dim3 grid(1024, a.nchunks);
  if (a.S == 2)
    pack_t2_lam_kernel<2><<<grid, 256, 0, s>>>(a);
  else
    pack_t2_lam_kernel<3><<<grid, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- B per aux chunk (two-pass dB)
// Second operand of the GEMM2 kernel in the two-pass dB: for aux chunk c,
// (b, d) block q = (Bb, Dd) and 16-slot piece, the chunk's rows P (padding
// rows zero) of 32 bytes, slot (b_l, d_l) = 8 (2 piece + h) + d_l holding
// slice s of B^P_{8 Bb + b_l, 8 Dd + d_l}, in the 32-byte-swizzled order of
// shared memory (the two 16-byte halves of row r swapped when bit 2 of r is
// set) so that one bulk copy per piece fills the operand.
template <int S>
__global__ void pack_b2_kernel(const __grid_constant__ BpackArgs a) {
  const TcChunk CH = a.chunks[blockIdx.y];
  const int nq = a.nb * a.nb, rows = CH.nps;
  const size_t units = (size_t)nq * 4 * rows * 2;  // (q, piece, row, half)
  uint4 *dst = reinterpret_cast<uint4 *>(a.T2 + CH.t2off / 2);
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < units;
       u += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(u & 1);
    size_t t = u >> 1;
    const int r = (int)(t % rows);
    t /= rows;
    const int piece = (int)(t % 4);
    const int q = (int)(t / 4);
    const int P = CH.lp0 + r;
    const int b = (q / a.nb) * CB + 2 * piece + h, d0 = (q % a.nb) * CB;
    __nv_bfloat16 sl[S][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int d = d0 + e;
      const double x = (r < CH.np && P < a.N && b < a.v && d < a.v) ? a.B[((size_t)P * a.v + b) * a.v + d] : 0.0;
      __nv_bfloat16 xs[S];
      split_bf16<S>(x, xs);
#pragma unroll
      for (int s = 0; s < S; ++s) sl[s][e] = xs[s];
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const size_t row = ((size_t)(q * 4 + piece) * S + s) * rows + r;
      dst[row * 2 + (h ^ ((r >> 2) & 1))] = *reinterpret_cast<const uint4 *>(sl[s]);
    }
  }
}

void launch_pack_b2(const BpackArgs &a, cudaStream_t s) {
  dim3 grid(1024, a.nchunks);
  if (a.S == 2)
    pack_b2_kernel<2><<<grid, 256, 0, s>>>(a);
  else
    pack_b2_kernel<3><<<grid, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- B slices
// Bt[q][a][c][P] = slice q of B[P][a][c]; a, c < vp (zero beyond v),
// P < Np (zero beyond N).  32x32 tiles through shared memory so both the
// read (c fastest) and the write (P fastest) are coalesced.
// A NaN or infinite element records kSiteNonFinite in *status (if given).
template <int S>
__global__ void split_B_kernel(int N, int v, int vp, int Np, const double *__restrict__ B,
                               __nv_bfloat16 *__restrict__ Bt, int transB, int *status) {
  __shared__ double tile[32][33];
  const int a = blockIdx.z;
  const int c0 = blockIdx.x * 32, P0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int P = P0 + r, c = c0 + tx;
    // transB: slice B^P_ca at position (a, c) (the transposed ladder of the adjoint)
    const size_t src = transB ? ((size_t)P * v + c) * v + a : ((size_t)P * v + a) * v + c;
    const double x = (P < N && c < v && a < v) ? B[src] : 0.0;
    if (status && !isfinite(x)) record_status(status, kSiteNonFinite);
    tile[r][tx] = x;
  }
  __syncthreads();
  const size_t slice = (size_t)vp * vp * Np;
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, P = P0 + tx;
    if (c < vp && P < Np) {
      __nv_bfloat16 sl[S];
      split_bf16<S>(tile[tx][r], sl);
      const size_t off = ((size_t)a * vp + c) * Np + P;
#pragma unroll
      for (int q = 0; q < S; ++q) Bt[q * slice + off] = sl[q];
    }
  }
}

void launch_split_B(int N, int v, int vp, int Np, int nslices, const double *B,
                    __nv_bfloat16 *Bt, cudaStream_t s, bool transB, int *status) {
  dim3 grid((vp + 31) / 32, (Np + 31) / 32, vp), block(32, 8);
  if (nslices == 2)
    split_B_kernel<2><<<grid, block, 0, s>>>(N, v, vp, Np, B, Bt, transB ? 1 : 0, status);
  else
    split_B_kernel<3><<<grid, block, 0, s>>>(N, v, vp, Np, B, Bt, transB ? 1 : 0, status);
}

// ---------------------------------------------------------------- energy
// E_L = sum_ijab R_ij^ab (2 t_ij^ab - t_ij^ba).  Stage 1: block (tile, ij)
// sums a 32x32 (a, b) tile with the transposed t tile staged in shared memory,
// writes one partial per block; stage 2: one block adds the partials in a
// fixed order.  Same inputs, same bits.  The grid is one-dimensional,
// blockIdx.x = ij * tiles + tile (o^2 can exceed the 65535 limit of grid.y).
constexpr int kEnergyThreads = 256;

__device__ __forceinline__ double block_sum(double x, double *red) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) red[w] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) s += red[k];
  __syncthreads();
  return s;
}

__global__ void energy_partial_kernel(int o, int v, const double *__restrict__ R,
                                      const double *__restrict__ t2, double *__restrict__ part) {
  __shared__ double tt[32][33];
  __shared__ double red[kEnergyThreads / 32];
  const int nt = (v + 31) / 32;
  const unsigned tile = blockIdx.x % (unsigned)(nt * nt);
  const int ta = (int)tile / nt, tb = (int)tile % nt;
  const size_t ij = blockIdx.x / (unsigned)(nt * nt);
  const size_t base = ij * v * v;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  // transposed tile: tt[b_local][a_local] = t_ij^{b a}
  for (int r = ty; r < 32; r += 8) {
    const int b = tb * 32 + r, a = ta * 32 + tx;
    tt[r][tx] = (a < v && b < v) ? t2[base + (size_t)b * v + a] : 0.0;
  }
  __syncthreads();
  double acc = 0.0;
  for (int r = ty; r < 32; r += 8) {
    const int a = ta * 32 + r, b = tb * 32 + tx;
    if (a < v && b < v) {
      const size_t e = base + (size_t)a * v + b;
      acc += R[e] * (2.0 * t2[e] - tt[tx][r]);
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void energy_final_kernel(size_t n, const double *__restrict__ part,
                                    double *__restrict__ E) {
  __shared__ double red[kEnergyThreads / 32];
  double acc = 0.0;
  for (size_t k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *E = s;
}

size_t energy_partials(int o, int v) {
  const int nt = (v + 31) / 32;
  return (size_t)nt * nt * o * o;
}

void launch_energy(int o, int v, const double *R, const double *t2, double *part, double *E,
                   cudaStream_t s) {
  const int nt = (v + 31) / 32;
  const unsigned blocks = (unsigned)(nt * nt) * (unsigned)(o * o);  // <= 2^30 for o <= 256, v <= 4096
  energy_partial_kernel<<<blocks, kEnergyThreads, 0, s>>>(o, v, R, t2, part);
  energy_final_kernel<<<1, kEnergyThreads, 0, s>>>(energy_partials(o, v), part, E);
}

// Y_ij^ab = alpha X_ij^ab + beta X_ij^ba.  With (alpha, beta) = (2, -1) this is
// the energy weight W = 2 t2 - t2^T (dE_L/dR) and, applied to R, the
// derivative of E_L through its weights, dE_L/dt2 = 2 R - R^T.
__global__ void pair_combine_kernel(int o, int v, double alpha, double beta,
                                    const double *__restrict__ X, double *__restrict__ Y) {
  const size_t total = (size_t)o * o * v * v;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    const size_t r = idx / v;
    const int a = (int)(r % v);
    const size_t ij = r / v;
    Y[idx] = alpha * X[idx] + beta * X[(ij * v + b) * v + a];
  }
}

void launch_pair_combine(int o, int v, double alpha, double beta, const double *X, double *Y,
                         cudaStream_t s) {
  const size_t total = (size_t)o * o * v * v;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  pair_combine_kernel<<<blocks, 256, 0, s>>>(o, v, alpha, beta, X, Y);
}

}  // namespace ladder

namespace ladder {

// ---------------------------------------------------------------- adjoint slices
// Xt[q][x][b][ij] = slice q of X_ij^{xb} (X = W or tau), K-major over the
// occupied pairs ij = i*o + j; x, b < vp (zero beyond v), ij < IJp (zero
// beyond o^2).  32x32 tiles through shared memory (read b fastest, write ij
// fastest).
template <int S>
__global__ void split_pairs_kernel(int o, int v, int vp, int IJp, const double *__restrict__ X,
                                   __nv_bfloat16 *__restrict__ Xt) {
  __shared__ double tile[32][33];
  const int x = blockIdx.z;
  const int b0 = blockIdx.x * 32, ij0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int o2 = o * o;
  for (int r = ty; r < 32; r += 8) {
    const int ij = ij0 + r, b = b0 + tx;
    tile[r][tx] = (ij < o2 && b < v && x < v) ? X[((size_t)ij * v + x) * v + b] : 0.0;
  }
  __syncthreads();
  const size_t slice = (size_t)vp * vp * IJp;
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, ij = ij0 + tx;
    if (b < vp && ij < IJp) {
      __nv_bfloat16 sl[S];
      split_bf16<S>(tile[tx][r], sl);
      const size_t off = ((size_t)x * vp + b) * IJp + ij;
#pragma unroll
      for (int q = 0; q < S; ++q) Xt[q * slice + off] = sl[q];
    }
  }
}

void launch_split_pairs(int o, int v, int vp, int IJp, int nslices, const double *X,
                        __nv_bfloat16 *Xt, cudaStream_t s) {
  dim3 grid((vp + 31) / 32, (IJp + 31) / 32, vp), block(32, 8);
  if (nslices == 2)
    split_pairs_kernel<2><<<grid, block, 0, s>>>(o, v, vp, IJp, X, Xt);
  else
    split_pairs_kernel<3><<<grid, block, 0, s>>>(o, v, vp, IJp, X, Xt);
}

// Bs[q][P][D][b][dl] = slice q of B^P_{b, 8D+dl}: for each auxiliary function
// P and each 8-block D of d, the (b, d) slots of that block with b-major order,
// so that the 16 slots (b, 8D..8D+7), (b+1, 8D..8D+7) of a GEMM piece are
// contiguous (one 32-byte TMA row).  Padded to vp (zero beyond v) and to Np
// auxiliary functions (zero beyond N).
template <int S>
__global__ void split_B_rows_kernel(int N, int v, int vp, int Np, const double *__restrict__ B,
                                    __nv_bfloat16 *__restrict__ Bs) {
  const size_t total = (size_t)Np * vp * vp;
  const size_t slice = total;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int dl = (int)(idx % CB);
    size_t r = idx / CB;
    const int b = (int)(r % vp);
    r /= vp;
    const int D = (int)(r % (vp / CB));
    const int P = (int)(r / (vp / CB));
    const int d = D * CB + dl;
    const double val = (P < N && b < v && d < v) ? B[((size_t)P * v + b) * v + d] : 0.0;
    __nv_bfloat16 sl[S];
    split_bf16<S>(val, sl);
#pragma unroll
    for (int q = 0; q < S; ++q) Bs[q * slice + idx] = sl[q];
  }
}

void launch_split_B_rows(int N, int v, int vp, int Np, int nslices, const double *B,
                         __nv_bfloat16 *Bs, cudaStream_t s) {
  const size_t total = (size_t)Np * vp * vp;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (nslices == 2)
    split_B_rows_kernel<2><<<blocks, 256, 0, s>>>(N, v, vp, Np, B, Bs);
  else
    split_B_rows_kernel<3><<<blocks, 256, 0, s>>>(N, v, vp, Np, B, Bs);
}

}  // namespace ladder
