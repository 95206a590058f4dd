// Internal launch interface between the C ABI (ladder_api.cu) and the kernels.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace ladder {

void launch_tau(int o, int v, const double *t1, const double *t2, double *tau, cudaStream_t s);
void launch_pack_tpm_f64(int o, int v, int K, const double *tau, double *Tp, double *Tm,
                         cudaStream_t s);
void launch_pack_tpm_bf16(int o, int v, int K, int nslices, int rows_p, int rows_m,
                          const double *tau, __nv_bfloat16 *Tp, __nv_bfloat16 *Tm,
                          cudaStream_t s);
void launch_split_B(int N, int v, int vp, int Np, int nslices, const double *B,
                    __nv_bfloat16 *Bt, cudaStream_t s);
size_t energy_partials(int o, int v);
void launch_energy(int o, int v, const double *R, const double *t2, double *part, double *E,
                   cudaStream_t s);
void launch_energy_weights(int o, int v, const double *t2, double *W, cudaStream_t s);

// ---- FP64 fused ladder (DMMA)
struct Fp64Args {
  const double *B;   // [N][v][v]
  const double *Tp;  // [ppos(o)][K]
  const double *Tm;  // [pneg(o)][K]
  double *R;         // [o][o][v][v]
  double *slab;      // spill of the V+- tiles, grid * K * 128 doubles (null if one chunk)
  int o, v, N, vp, K;
  int ntiles;        // (8-block, 8-block) ab tiles with ia <= ib
  int nchunks;
  Chunk chunks[kMaxChunks];
};
constexpr int kFp64LamTile = 64;  // max lambda+ (and lambda-) rows per chunk
int fp64_grid(const Fp64Args &a, int sm_count);
size_t fp64_slab_doubles(int K, int grid);
cudaError_t launch_ladder_fp64(const Fp64Args &a, int grid, cudaStream_t s);

}  // namespace ladder
