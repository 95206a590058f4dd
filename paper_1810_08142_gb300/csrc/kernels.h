// Internal launch interface between the C ABI (ladder_api.cu) and the kernels.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace ladder {

void launch_tau(int o, int v, const double *t1, const double *t2, double *tau, cudaStream_t s);
void launch_pack_tpm_f64(int o, int v, int K, const double *tau, double *Tp, double *Tm,
                         cudaStream_t s);
// status (nullable): a NaN or infinite input element records kSiteNonFinite
void launch_pack_tpm_bf16(int o, int v, int K, int nslices, int rows_p, int rows_m,
                          const double *tau, __nv_bfloat16 *Tp, __nv_bfloat16 *Tm,
                          cudaStream_t s, int *status = nullptr);
void launch_split_B(int N, int v, int vp, int Np, int nslices, const double *B,
                    __nv_bfloat16 *Bt, cudaStream_t s, bool transB = false, int *status = nullptr);
void launch_pair_combine(int o, int v, double alpha, double beta, const double *X, double *Y,
                         cudaStream_t s);
void launch_split_pairs(int o, int v, int vp, int IJp, int nslices, const double *X,
                        __nv_bfloat16 *Xt, cudaStream_t s);
void launch_split_B_rows(int N, int v, int vp, int Np, int nslices, const double *B,
                         __nv_bfloat16 *Bs, cudaStream_t s);
size_t energy_partials(int o, int v);
void launch_energy(int o, int v, const double *R, const double *t2, double *part, double *E,
                   cudaStream_t s);

// ---- t1-dressed ladder: Bd = B - mbar and the rank-o correction (dress.cu)
// kEpiStore: Out (T) = C; kEpiPerm: Out (T) = C in the permuted (k,l)(c,d) layout;
// kEpiSubR: Out (double) -= C; kEpiFromSrc: Out (double) = Src - C;
// kEpiAcc3: Out (T) at (m / pv) s1 + (m % pv) s2 + n s3 (+ batch * so_batch)
// gets alpha C (acc = 0) or alpha C added (acc = 1).
enum : int { kEpiStore = 0, kEpiPerm = 1, kEpiSubR = 2, kEpiFromSrc = 3, kEpiAcc3 = 4 };
// C(m, n) = sum_k A(m, k) B(n, k), A(m, k) = A[m*sam + k*sak], B(n, k) = B[n*sbn + k*sbk]
// (one of the two strides of each operand is 1); z = batch * ksplit + split.
struct GemmArgs {
  const void *A, *B;
  void *Out;
  const double *Src;  // kEpiFromSrc
  long long sam, sak, sbn, sbk;
  long long sa_batch, sb_batch, so_batch;  // per batch (A, B, kEpiSubR/FromSrc) or per z (kEpiStore)
  int M, N, K;
  int ksplit, kchunk;
  int ldo;
  int epi;
  int sym;     // A == B: compute the tiles with m-tile <= n-tile, mirror in the epilogue
  int po, pv;  // kEpiPerm: m = (k, c), n = (l, d) -> Out[((k * po + l) * pv + c) * pn + d],
  int pn;      //   c = m % pv, d = n % pn (pn = 0: pn = pv)
  long long s1, s2, s3;  // kEpiAcc3 strides
  // optional second K segment in the same accumulators: A2 (m, k) = A2[m*sam2 + k*sak2],
  // B2 (n, k) = beta2 * B2[n*sbn2 + k*sbk2], k < K2 (ksplit must be 1)
  const void *A2, *B2;
  long long sam2, sak2, sbn2, sbk2, sa2_batch, sb2_batch;
  int K2;
  double beta2;
  int acc;
  double alpha;
  int ntm, ntn, zoff;  // set by the launcher
};
// Double-single number (an unevaluated sum h + l of two floats, about 48
// bits): the accumulation type of the error-free mode's dressing correction,
// which runs on the FP32 pipe (far faster than FP64 on this GPU).  Its
// arithmetic is defined where the GEMM kernel is (dress.cu).
struct DS {
  float h, l;
};
template <typename TA, typename TB, typename T>
cudaError_t launch_gemm(const GemmArgs &g, int batch, cudaStream_t s);
template <typename T>
cudaError_t launch_reduce(T *X, long long n, int parts, cudaStream_t s);

// ---- perturbative triples (triples.cu); W from launch_gemm with kEpiAcc3
constexpr int kTriplesMaxV = 1024;  // ladder_triples: v at most this (shared-memory vectors of the energy kernel)
struct TriplesArgs {
  const void *oovv;  // [j][k][b][c] = v_jk^bc = (bj|ck), element type T of the energy kernel
  const double *t1, *e_occ, *e_vir;
  int o, v;
};
int triples_energy_blocks(int v);
template <typename T>
cudaError_t launch_triples_energy(const TriplesArgs &a, const T *W, int i, int j, double *part,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_triples_t2(int o, int v, const double *t2, T *t2c, T *t2T, cudaStream_t s);
template <typename T>
cudaError_t launch_triples_negate(T *x, long long n, cudaStream_t s);
// dst[g][x][y][d] = src[g][y][x][d] for g < G, x, y, d < v (the middle two
// indices exchanged)
template <typename T>
cudaError_t launch_triples_swap12(const T *src, T *dst, int G, int v, cudaStream_t s);
cudaError_t launch_triples_final(const double *part, long long n, double *E, cudaStream_t s,
                                 const int *status = nullptr);

// ---- perturbative triples on the tensor cores (triples_tc.cu): the W
// contractions as batched split-BF16 GEMMs (three slices of the FP32
// operands, six slice products), two K segments, kEpiAcc3-style epilogue.
// Operand slices [S][g][rows][K] (rows and K zero-padded): A1 rows m over
// K = d (K1p), B1 rows n over d, A2 rows m over K = l (K2p), B2 rows n over
// l; the outer index g of each is fix + mul * batch.
struct TwArgs {
  CUtensorMap tmA1, tmB1, tmA2, tmB2;
  // nord = 2: a second ordering of P with the same output strides adds its
  // two K segments into the same accumulators (A maps tmA1b / tmA2b, outer
  // indices a1b / b1b for both of its segments)
  CUtensorMap tmA1b, tmA2b;
  float *W;
  int *status;
  int M, N, Nt, K1p, K2p, batch;
  int a1_fix, a1_mul, b1_fix, b1_mul, a2_fix, a2_mul, b2_fix, b2_mul;
  int nord, a1b_fix, a1b_mul, b1b_fix, b1b_mul;
  int pv, acc;
  long long s1, s2, s3, so_batch;
  unsigned long long timeout_ns;
};
uint32_t tw_smem_bytes(int Nt);
cudaError_t tw_init_attributes();
cudaError_t launch_tw_gemm(const TwArgs &a, int grid, cudaStream_t s);
cudaError_t launch_tw_slice(const float *src, long long sg, long long sr, long long sk, int G, int rows,
                            int rows_pad, int K, int K_pad, __nv_bfloat16 *dst, cudaStream_t s);

// ---- FP64 fused ladder (DMMA)
struct Fp64Args {
  const double *B;   // [N][v][v]
  const double *Tp;  // [ppos(o)][K]
  const double *Tm;  // [pneg(o)][K]
  double *R;         // [o][o][v][v]
  double *slab;      // spill of the V+- tiles, grid * K * 128 doubles (null if one chunk)
  int o, v, N, vp, K;
  int ntiles;        // (8-block, 8-block) ab tiles with ia <= ib
  int transB;        // read B^P_ca for B^P_ac (adjoint: transposed ladder)
  int nchunks;
  Chunk chunks[kMaxChunks];
};
constexpr int kFp64LamTile = 64;  // max lambda+ (and lambda-) rows per chunk
int fp64_grid(const Fp64Args &a, int sm_count);
size_t fp64_slab_doubles(int K, int grid);
cudaError_t launch_ladder_fp64(const Fp64Args &a, int grid, cudaStream_t s);

// ---- FP64 gradient with respect to B (adjoint, ladder_grad_fp64.cu)
constexpr int kGradPChunk = 64;  // auxiliary functions per register-accumulator chunk
struct GradArgs {
  const double *B;    // [N][v][v]
  const double *tau;  // [o][o][v][v]
  const double *W;    // [o][o][v][v]
  double *dB;         // [N][v][v]
  double *slab;       // Gamma spill, grad_fp64_slab_doubles (null if one P-chunk)
  int o, v, N, vp;
};
int grad_fp64_grid(int vp, int sm_count);
size_t grad_fp64_slab_doubles(int vp, int N, int grid);
cudaError_t launch_grad_B_fp64(const GradArgs &a, int grid, cudaStream_t s);

// ---- split-BF16 gradient with respect to B (adjoint, ladder_grad_tc.cu)
constexpr int kGradTcPChunk = 128;  // auxiliary functions per work unit (TMEM columns)
struct GradTcArgs {
  CUtensorMap tmW;   // W slices [S][x][b][ij], box (32 ij, 8 b, 16 x), 64-byte swizzle
  CUtensorMap tmT;   // tau slices [S][y][d][ij], box (32 ij, 8 d, 8 y)
  CUtensorMap tmBs;  // B slices [S][P][D][b][dl], box (16 (b,dl), 1 D, 16 P), 32-byte swizzle
  double *dB;        // [N][v][v]
  float2 *racc;      // double-single sums, [item][128 cols][128 lanes]
  __nv_bfloat16 *Gst;  // two-pass dB: Gamma planes [tile][(b,d) block][slice][128][64]
  int qsplit;          // two-pass dB: (b,d)-block ranges per tile of the storing pass
  int *status;
  int o, v, N, vp, Np, IJp, nks, nY8, ntiles, npc;
  int kc, s_pieces, flush_every;
  unsigned long long timeout_ns;
};
cudaError_t grad_tc_init_attributes(int nslices);
cudaError_t launch_grad_B_tc(const GradTcArgs &a, int nslices, cudaStream_t s);
// Two-pass dB: the Gamma tiles of every (x,y) tile and (b,d) block stored once
// (the contraction with B then runs in the GEMM2 kernel, see TcArgs::square).
cudaError_t launch_grad_gamma_store(const GradTcArgs &a, int nslices, cudaStream_t s);

// ---- split-BF16 fused ladder (tcgen05)
// An occupied-pair chunk of the tensor-core kernel: lambda+ rows [lp0, lp0+np)
// and lambda- rows [lm0, lm0+nm), padded to nps, nms (multiples of 16) TMEM
// columns; nps + nms <= kTcMaxCols.
constexpr int kTcMaxCols = 128;
// Chunks of the GEMM2 kernel of the two-pass form (TMEM holds no GEMM1 tiles):
// lambda+ or lambda- columns only, at most kTcMaxColsV each.
constexpr int kTcMaxColsV = 192;
struct TcChunk {
  int lp0, lm0, np, nm, nps, nms;
  long long t2off;  // two-pass GEMM2: byte offset of the chunk's tau+- copy (pack_t2)
};
struct TcArgs {
  CUtensorMap tmA;   // B slices [S][a][c][P] as 4-D, box (32 aux, 8 c, 16 a, S), 64-byte swizzle
  CUtensorMap tmB;   // the same, box (32 aux, 8 d, 8 b, S)
  CUtensorMap tmTp;  // tau+ slices [S][lambda+][K], box (16 slots, 16 rows, 1)
  CUtensorMap tmTm;  // tau- slices [S][lambda-][K]
  CUtensorMap tmVl;  // stored V+- planes [tile][pair][sign][slice][128 rows][64 slots],
                     // load box (16 slots, 128 rows, S): one sign, 32-byte swizzle
  __nv_bfloat16 *Vst;  // the same planes, written by the storing pass
  const uint8_t *T2; // two-pass GEMM2: chunk-major tau+- (pack_t2)
  double *R;
  float2 *racc;      // double-single accumulators, [item][col][128 lanes], racc_cols columns per item
  int *status;
  int o, v, vp, Np, K, nbp;
  int nks;           // Np / 32
  int nA, nB8;       // 16-blocks of a, 8-blocks of b
  int ntiles, nchunks, ksplit;
  int tile0;         // first (a 16-block, b 8-block) tile of the plan's range; the
                     // work units and stored planes index tiles from it
  int racc_cols;
  int kc;            // GEMM1 K-steps (of 32 aux functions) per FP32 accumulation chain
  int xy_split;      // GEMM1: separate accumulators for hi*hi and the smaller products
  int s_pieces;      // 16-slot pieces of GEMM2 per fresh S accumulator (1, 2 or 4)
  int flush_every;   // S accumulators summed in FP32 before a flush to the double-single sums
  int nplus, wplus, wminus;  // two-pass GEMM2: plus chunks first, lambda columns per chunk
  int square;        // GEMM2 kernel: tiles cover every (16-block, 8-block) pair (two-pass dB)
  int nsign;         // GEMM2 kernel: stored planes per (tile, block) = nsign * S
  int lam_only;      // the paper's lambda-only contraction (an ablation of the +- split):
                     // the storing pass keeps X = (ac|bd) and Y' = (ad|bc) instead of
                     // V+- = X +- Y', and each GEMM2 piece multiplies both planes into
                     // one accumulator, X by tau^cd and Y' by tau^dc, for all ordered ij
  unsigned long long timeout_ns;
  TcChunk chunks[kMaxChunks];
};
// Chunk-major, pre-swizzled tau+- for the GEMM2 pass (prep_kernels.cu).
struct T2Args {
  const __nv_bfloat16 *Tp, *Tm;  // [S][rows_p][K], [S][rows_m][K]
  __nv_bfloat16 *T2;
  int K, S, rows_p, rows_m, nchunks;
  TcChunk chunks[kMaxChunks];
  long long off[kMaxChunks];     // element offset of each chunk in T2
};
void launch_pack_t2(const T2Args &a, cudaStream_t s);
// lambda-only GEMM2 operand, straight from tau: for chunk c (ordered pairs
// ij = lp0 .. lp0 + np - 1, padded to nps rows), global 16-slot piece x and
// plane j, slice s of w tau_ij^cd (j = 0) or w tau_ij^dc (j = 1), w = 1/2 on
// diagonal block pairs and 1 elsewhere, 32-byte swizzled rows; chunk c starts
// at byte t2off.
struct T2LamArgs {
  const double *tau;  // [o][o][v][v]
  __nv_bfloat16 *T2;
  int o, v, K, S, nchunks;
  TcChunk chunks[kMaxChunks];
};
void launch_pack_t2_lam(const T2LamArgs &a, cudaStream_t s);

// Per-chunk, pre-swizzled copy of the B slices as the GEMM2 kernel's second
// operand: for aux chunk c, (b,d) block q and 16-slot piece, rows P of the
// chunk; slot (b_l, d_l) of block q holds slice s of B^P_{8Bb+b_l, 8Dd+d_l}.
struct BpackArgs {
  const double *B;    // [N][v][v]
  __nv_bfloat16 *T2;
  int N, v, nb, S, nchunks;
  TcChunk chunks[kMaxChunks];  // lp0 = first P, np = P count, nps = padded rows
};
void launch_pack_b2(const BpackArgs &a, cudaStream_t s);

// ---- error-free split-BF16 mode (ladder_oz.cu)
// Every operand row is carried as S fixed-point BF16 slices under one
// power-of-two scale per row: x = scale * sum_s x_s 2^(-8 s), x_0 an integer in
// [-256, 256], x_s (s >= 1) integers in [-129, 129].  Slice products are then
// exact, and a TMEM accumulator that only ever receives products of one slice
// order p + q sums integers (in units of 2^(-8 (p + q))) that stay below 2^24
// within an exactness window, so the tensor core's FP32 accumulation makes no
// rounding error there.  Orders 0, 1 and 2 each have their own accumulator,
// orders >= 3 share one (they sit 2^-24 below the result).  Windows are summed
// in double-single form (an FP32 pair, about 48 bits) by the conversion warps.
constexpr int kOzGroups = 4;      // TMEM accumulators per tile: orders 0, 1, 2, >= 3
constexpr int kOzKc = 4;          // GEMM1 window: K-steps of 32 aux functions (128)
constexpr int kOzMaxCols = 128;   // GEMM2 chunk width (four groups fill TMEM)
struct OzArgs {
  CUtensorMap tmA, tmB;  // fixed-point B slices [S][a][c][P]: boxes (32, 8, 16, S), (32, 8, 8, S)
  CUtensorMap tmVl;      // stored V+- planes [tile][pair][sign][slice][128][64], box (16, 128, S)
  __nv_bfloat16 *Vst;    // the same planes, written by pass 1
  float *sV;             // [tile][pair][sign][128 rows] scale of each stored V+- row
  const float *rsB;      // [vp][vp] scale of each B row (a, c) (0 for zero rows)
  const uint8_t *T2;     // per-chunk tau+- slices (oz_pack_t2), byte offset chunks[c].t2off
  const float *sT;       // [chunk][pair][kOzMaxCols] scale of each tau+- row
  float2 *racc;          // double-single sums, [item][col][128 lanes]
  float2 *Xs;            // symmetric B: distinct integral tiles [(r <= q)][64][64], double-single
  const int4 *xunits;    // symmetric B: (iA, kk, q0, q1) work units of the distinct tiles
  int *status;
  int o, v, vp, Np, nbp, nks;
  int nB8, ntiles, nchunks, ksplit, racc_cols;
  int tile0;             // the plan's tiles are tile0 .. tile0 + ntiles - 1 (local index t - tile0)
  int nitems;
  unsigned long long timeout_ns;
  TcChunk chunks[kMaxChunks];
};
// tau+- of every GEMM2 chunk as fixed-point slices with one scale per (row,
// block pair), in the per-chunk, pre-swizzled layout of pack_t2.
struct OzPackArgs {
  const double *tau;
  uint8_t *T2;
  float *sT;
  int *status;
  int o, v, nbp, S, nchunks;
  TcChunk chunks[kMaxChunks];
};
// Row scales of B (and a non-finite check), then the fixed-point slices.
void launch_oz_rowscale(int N, int v, int vp, const double *B, float *rs, int *status, cudaStream_t s);
void launch_oz_split_B(int N, int v, int vp, int Np, int nslices, const double *B, const float *rs,
                       __nv_bfloat16 *Bt, cudaStream_t s);
void launch_oz_pack_t2(const OzPackArgs &a, cudaStream_t s);
// One launch of an error-free pass: a single molecule (mols == nullptr, work
// units 0..nitems-1 of `one`) or a batch (work unit k is local unit items[k].y
// of molecule items[k].x, the molecules' args in device memory).  One CTA per
// work unit.  status and timeout_ns serve every molecule of the launch.
struct OzLaunch {
  OzArgs one;
  const OzArgs *mols;
  const int2 *items;
  int nitems;
  int *status;
  unsigned long long timeout_ns;
};
uint32_t oz_smem_bytes(int pass, int nslices);
cudaError_t oz_init_attributes(int nslices);
cudaError_t launch_oz_vstore(const OzLaunch &L, int nslices, cudaStream_t s);
cudaError_t launch_oz_gemm2(const OzLaunch &L, int nslices, cudaStream_t s);
// Symmetric B: the distinct integral tiles (one CTA per unit of xunits), V+-
// of a tile range formed and sliced from them (units = tiles x block pairs),
// a single molecule (`one`) or a batch (mols / items) each, and the bitwise
// check B^P_ac = B^P_ca.
cudaError_t launch_oz_xsym(const OzLaunch &L, int nslices, cudaStream_t s);
cudaError_t launch_oz_vform(const OzLaunch &L, int nslices, int sm_count, cudaStream_t s);
void launch_oz_symcheck(int N, int v, const double *B, int *status, cudaStream_t s);

// One launch of the fused kernel: a single molecule (mols == nullptr, the
// work units are 0..nitems-1 of `one`) or a batch (work unit k is local item
// items[k].y of molecule items[k].x, args in device memory).  tcs lists the
// (molecule, tile*chunk) blocks of the unpack kernel for a batch.
struct TcLaunch {
  TcArgs one;
  const TcArgs *mols;
  const int2 *items;
  const int2 *tcs;
  int nitems;
  unsigned long long timeout_ns;
};
uint32_t tc_smem_bytes(int nslices);
cudaError_t tc_init_attributes(int nslices);  // once per device, outside stream capture
cudaError_t launch_ladder_tc(const TcLaunch &a, int nslices, int grid, cudaStream_t s);
// Two-pass form (one molecule, or a batch through mols/items): GEMM1 once per
// (tile, block pair) with the V+- slices stored to global memory, then GEMM2
// from the stored tiles.
cudaError_t launch_ladder_vstore(const TcLaunch &a, int nslices, int grid, cudaStream_t s);
cudaError_t launch_ladder_gemm2(const TcLaunch &a, int nslices, int grid, cudaStream_t s);
cudaError_t launch_unpack(const TcLaunch &a, int nblocks, cudaStream_t s);
// two-pass form: nblocks = tiles x plus-chunks (a batch lists (molecule, block) in tcs)
cudaError_t launch_unpack2(const TcLaunch &a, int nblocks, cudaStream_t s);
// lambda-only form: one block per (tile, chunk); R_ij^ab and R_ji^ba from one column
cudaError_t launch_unpack_lam(const TcLaunch &a, int nblocks, cudaStream_t s);
// two-pass dB: dB[P][x][y] = 2 x the sums of the GEMM2 kernel, blocks = tiles x chunks
cudaError_t launch_grad_unpack2(const TcLaunch &a, double *dB, int N, int nblocks, cudaStream_t s);
cudaError_t launch_selftest_wait(int *status, unsigned long long timeout_ns, int site,
                                 cudaStream_t s);

}  // namespace ladder
