// C ABI of the ladder library: plans, workspace layout, argument checks and
// launch sequences.  See include/ladder.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ladder.h"
#include "kernels.h"

using namespace ladder;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

struct Layout {
  size_t status = 0, energy = 0, Tp = 0, Tm = 0, slab = 0, Bt = 0, W = 0, total = 0;
};

}  // namespace

struct ladder_plan_s {
  int o = 0, v = 0, N = 0, mode = 0;
  int vp = 0, nb = 0, nbp = 0, K = 0, Np = 0;
  int nlp = 0, nlm = 0;
  int sm_count = 0, device = 0;
  // FP64 path
  std::vector<Chunk> chunks64;
  int grid64 = 0;
  Layout lay;
  void *ws = nullptr;
  size_t ws_bytes = 0;
};

namespace {

// Occupied-pair chunks: consecutive j ranges whose lambda+ and lambda- row
// counts both stay within `rows`.
std::vector<Chunk> make_chunks(int o, int rows) {
  std::vector<Chunk> out;
  int j0 = 0;
  while (j0 < o) {
    int j1 = j0 + 1;
    while (j1 < o && ppos(j1 + 1) - ppos(j0) <= rows && pneg(j1 + 1) - pneg(j0) <= rows) ++j1;
    out.push_back({j0, j1});
    j0 = j1;
  }
  return out;
}

bool dev_ptr_ok(const void *p) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
T *ws_at(const ladder_plan_s *pl, size_t off) {
  return reinterpret_cast<T *>(static_cast<char *>(pl->ws) + off);
}

ladder_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LADDER_OK;
  cudaGetLastError();
  return LADDER_ECUDA;
}

void compute_layout(ladder_plan_s *pl) {
  Layout L;
  size_t off = 0;
  L.status = off;
  off += kAlign;
  L.energy = off;
  off = align_up(off + energy_partials(pl->o, pl->v) * sizeof(double));
  if (pl->mode == LADDER_FP64) {
    L.Tp = off;
    off = align_up(off + (size_t)pl->nlp * pl->K * sizeof(double));
    L.Tm = off;
    off = align_up(off + (size_t)std::max(pl->nlm, 1) * pl->K * sizeof(double));
    L.slab = off;
    if (pl->chunks64.size() > 1) off = align_up(off + fp64_slab_doubles(pl->K, pl->grid64) * sizeof(double));
  }
  L.W = off;  // backward: energy weights / scratch copies are caller-provided
  L.total = off;
  pl->lay = L;
}

}  // namespace

extern "C" {

const char *ladder_status_string(ladder_status s) {
  switch (s) {
    case LADDER_OK: return "ok";
    case LADDER_EINVAL: return "invalid argument";
    case LADDER_ENOMEM: return "host allocation failed";
    case LADDER_ECUDA: return "CUDA call failed";
    case LADDER_ETIMEOUT: return "bounded device wait ran out";
    case LADDER_ENOTSUP: return "mode or shape not supported";
    case LADDER_EWORKSPACE: return "workspace missing or too small";
  }
  return "unknown status";
}

ladder_status ladder_plan(int o, int v, int naux, int mode, ladder_plan_t *out) {
  if (!out) return LADDER_EINVAL;
  *out = nullptr;
  if (o < 1 || o > 256 || v < 1 || v > 4096 || naux < 1 || naux > 65536) return LADDER_EINVAL;
  if (mode < LADDER_FP64 || mode > LADDER_AUTO) return LADDER_EINVAL;
  if (mode == LADDER_AUTO) mode = LADDER_BF16X6;
  if (mode != LADDER_FP64) return LADDER_ENOTSUP;
  ladder_plan_s *pl = new (std::nothrow) ladder_plan_s();
  if (!pl) return LADDER_ENOMEM;
  pl->o = o;
  pl->v = v;
  pl->N = naux;
  pl->mode = mode;
  pl->vp = (v + VPAD - 1) / VPAD * VPAD;
  pl->nb = pl->vp / CB;
  pl->nbp = ppos(pl->nb);
  pl->K = pl->nbp * SLOTS;
  pl->nlp = ppos(o);
  pl->nlm = pneg(o);
  if (cudaGetDevice(&pl->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return LADDER_ECUDA;
  }
  pl->chunks64 = make_chunks(o, kFp64LamTile);
  if ((int)pl->chunks64.size() > kMaxChunks) {
    delete pl;
    return LADDER_ENOTSUP;
  }
  Fp64Args tmp{};
  tmp.ntiles = ppos(pl->vp / CB);
  pl->grid64 = fp64_grid(tmp, pl->sm_count);
  compute_layout(pl);
  *out = pl;
  return LADDER_OK;
}

ladder_status ladder_plan_mode(ladder_plan_t pl, int *mode) {
  if (!pl || !mode) return LADDER_EINVAL;
  *mode = pl->mode;
  return LADDER_OK;
}

ladder_status ladder_workspace_size(ladder_plan_t pl, size_t *bytes) {
  if (!pl || !bytes) return LADDER_EINVAL;
  *bytes = pl->lay.total;
  return LADDER_OK;
}

ladder_status ladder_set_workspace(ladder_plan_t pl, void *dptr, size_t bytes) {
  if (!pl) return LADDER_EINVAL;
  if (bytes < pl->lay.total) return LADDER_EWORKSPACE;
  if (!dptr || (reinterpret_cast<uintptr_t>(dptr) % kAlign)) return LADDER_EINVAL;
  if (!dev_ptr_ok(dptr)) return LADDER_EINVAL;
  pl->ws = dptr;
  pl->ws_bytes = bytes;
  // the status word starts cleared; this is the plan's only synchronous copy
  if (cudaMemset(dptr, 0, sizeof(int)) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  return LADDER_OK;
}

ladder_status ladder_tau(ladder_plan_t pl, const double *t1, const double *t2, double *tau,
                         void *stream) {
  if (!pl || !dev_ptr_ok(t1) || !dev_ptr_ok(t2) || !dev_ptr_ok(tau) || tau == t2)
    return LADDER_EINVAL;
  launch_tau(pl->o, pl->v, t1, t2, tau, static_cast<cudaStream_t>(stream));
  return cuda_status(cudaGetLastError());
}

static ladder_status apply_fp64(ladder_plan_t pl, const double *B, const double *tau, double *R,
                                cudaStream_t s) {
  double *Tp = ws_at<double>(pl, pl->lay.Tp), *Tm = ws_at<double>(pl, pl->lay.Tm);
  launch_pack_tpm_f64(pl->o, pl->v, pl->K, tau, Tp, Tm, s);
  ladder_status st = cuda_status(cudaGetLastError());
  if (st != LADDER_OK) return st;
  Fp64Args a{};
  a.B = B;
  a.Tp = Tp;
  a.Tm = Tm;
  a.R = R;
  a.slab = pl->chunks64.size() > 1 ? ws_at<double>(pl, pl->lay.slab) : nullptr;
  a.o = pl->o;
  a.v = pl->v;
  a.N = pl->N;
  a.vp = pl->vp;
  a.K = pl->K;
  a.ntiles = ppos(pl->vp / CB);
  a.nchunks = (int)pl->chunks64.size();
  for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->chunks64[c];
  return cuda_status(launch_ladder_fp64(a, pl->grid64, s));
}

ladder_status ladder_apply(ladder_plan_t pl, const double *B, const double *tau, double *R,
                           void *stream) {
  if (!pl) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!dev_ptr_ok(B) || !dev_ptr_ok(tau) || !dev_ptr_ok(R) || R == B || R == tau)
    return LADDER_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pl->mode == LADDER_FP64) return apply_fp64(pl, B, tau, R, s);
  return LADDER_ENOTSUP;
}

ladder_status ladder_energy(ladder_plan_t pl, const double *R, const double *t2, double *E_dev,
                            void *stream) {
  if (!pl) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!dev_ptr_ok(R) || !dev_ptr_ok(t2) || !E_dev) return LADDER_EINVAL;
  launch_energy(pl->o, pl->v, R, t2, ws_at<double>(pl, pl->lay.energy), E_dev,
                static_cast<cudaStream_t>(stream));
  return cuda_status(cudaGetLastError());
}

ladder_status ladder_backward(ladder_plan_t pl, const double *B, const double *tau,
                              const double *W, double *dtau, double *dB, void *stream) {
  (void)pl; (void)B; (void)tau; (void)W; (void)dtau; (void)dB; (void)stream;
  return LADDER_ENOTSUP;
}

ladder_status ladder_apply_host(ladder_plan_t pl, const double *B_host, const double *tau_host,
                                double *R_host, double *d_B, double *d_tau, double *d_R,
                                void *stream) {
  if (!pl || !B_host || !tau_host || !R_host) return LADDER_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nB = (size_t)pl->N * pl->v * pl->v * sizeof(double);
  const size_t nT = (size_t)pl->o * pl->o * pl->v * pl->v * sizeof(double);
  if (!dev_ptr_ok(d_B) || !dev_ptr_ok(d_tau) || !dev_ptr_ok(d_R)) return LADDER_EINVAL;
  if (cudaMemcpyAsync(d_B, B_host, nB, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_tau, tau_host, nT, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  ladder_status st = ladder_apply(pl, d_B, d_tau, d_R, stream);
  if (st != LADDER_OK) return st;
  if (cudaMemcpyAsync(R_host, d_R, nT, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  return cuda_status(cudaStreamSynchronize(s));
}

ladder_status ladder_plan_batched(int n, const int *o, const int *v, const int *naux, int mode,
                                  ladder_plan_t *out) {
  (void)n; (void)o; (void)v; (void)naux; (void)mode;
  if (out) *out = nullptr;
  return LADDER_ENOTSUP;
}

ladder_status ladder_apply_batched(ladder_plan_t pl, const double *const *B,
                                   const double *const *tau, double *const *R, void *stream) {
  (void)pl; (void)B; (void)tau; (void)R; (void)stream;
  return LADDER_ENOTSUP;
}

ladder_status ladder_last_device_error(ladder_plan_t pl, void *stream, int *where) {
  if (!pl) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  int *d = ws_at<int>(pl, pl->lay.status);
  if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(d, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  if (where) *where = h;
  return h == 0 ? LADDER_OK : LADDER_ETIMEOUT;
}

double ladder_flops(ladder_plan_t pl) {
  if (!pl) return 0.0;
  const double g1 = 2.0 * ppos(pl->v) * (double)pl->v * pl->v * pl->N;
  const double g2 = 2.0 * ((double)ppos(pl->o) * ppos(pl->v) * (double)ppos(pl->v) +
                           (double)pneg(pl->o) * pneg(pl->v) * (double)pneg(pl->v));
  return g1 + g2;
}

void ladder_destroy(ladder_plan_t pl) { delete pl; }

}  // extern "C"
