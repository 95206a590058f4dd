// C ABI of the ladder library: plans, workspace layout, argument checks and
// launch sequences.  See include/ladder.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/ladder.h"
#include <cudaTypedefs.h>

#include "kernels.h"

using namespace ladder;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

struct Layout {
  size_t status = 0, energy = 0, Tp = 0, Tm = 0, slab = 0, Bt = 0, W = 0, gslab = 0, total = 0;
  size_t gWt = 0, gTt = 0, gBs = 0, gacc = 0;  // split-BF16 dB
  size_t Vg = 0, T2 = 0;                       // two-pass form: stored V+- tiles, tau+- per chunk
  size_t gG = 0, gT2 = 0, gacc2 = 0;           // two-pass dB: Gamma planes, B per chunk, sums
  size_t dBd = 0, dG = 0, dX = 0, dY = 0;      // t1 dressing: B - mbar, (kc|ld), X, Y
  size_t ozRs = 0, ozSV = 0, ozST = 0;         // error-free mode: B row scales, V+- and tau+- row scales
  size_t ozXs = 0, ozXu = 0;                   // symmetric B: distinct integral tiles, their work units
};

// Two-pass form: at most this many bytes of stored V+- tiles by default.
constexpr double kVStoreDefaultCap = 128.0 * (1ull << 30);
// The error-free mode has no fused form: shapes whose stored V+- slices
// exceed this are not supported.
constexpr double kVStoreOzCap = 200.0 * (1ull << 30);
constexpr int kOzDefaultSlices = 5;
// Symmetric B: at most this many bytes of distinct integral tiles (v up to
// about 550), and column block pairs per work unit of their pass.
constexpr double kXsymCap = 96.0 * (1ull << 30);
constexpr int kXsymRange = 32;

int tc_slices(int mode) { return mode == LADDER_BF16X3 ? 2 : 3; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool encode3d(CUtensorMap *m, void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
              uint32_t b1, uint32_t b2, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
  const cuuint32_t box[3] = {b0, b1, b2};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D bf16 map: dims (d0, d1, d2, d3), d0 contiguous, box (b0, b1, b2, b3).
bool encode4d(CUtensorMap *m, void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3,
              uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {d0, d1, d2, d3};
  const cuuint64_t strides[3] = {d0 * 2, d0 * d1 * 2, d0 * d1 * d2 * 2};
  const cuuint32_t box[4] = {b0, b1, b2, b3};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct ladder_plan_s {
  int o = 0, v = 0, N = 0, mode = 0;
  bool backward = false;
  bool dressed = false;  // workspace sized for ladder_apply_dressed
  int dx_ksplit = 1;     // K splits of the X_ij^kl contraction
  int grid_grad = 0;
  int vp = 0, nb = 0, nbp = 0, K = 0, Np = 0;
  int nlp = 0, nlm = 0;
  int sm_count = 0, device = 0;
  // FP64 path
  std::vector<Chunk> chunks64;
  int grid64 = 0;
  // split-BF16 tensor-core path
  int S = 0, ksplit = 1, kc = 4, s_pieces = 4, flush_every = 64, xy_split = 1, ntiles_tc = 0, racc_cols = 0;
  std::vector<TcChunk> chunks_tc;
  // two-pass form: GEMM2 chunks (up to kTcMaxColsV columns), block-pair
  // ranges per tile of the storing pass
  int two_pass = 0, vsplit = 1, racc_cols_v = 0, nplus = 0, wplus = 0, wminus = 0;
  int lam_only = 0;  // the paper's lambda-only contraction (two-pass form only)
  int oz_slices = kOzDefaultSlices;  // error-free mode: fixed-point slices per operand
  // error-free mode with symmetric B: the distinct integral tiles once, then
  // V+- formed from them (xunits: the (iA, kk, q0, q1) units of their pass)
  int sym_b = 0;
  std::vector<int4> xunits;
  // pair-tile range of the plan (multi-GPU partition): tiles tile0 ..
  // tile0 + ntiles_tc - 1 of the shape's ntiles_all
  int tile0 = 0, ntiles_all = 0;
  // two-pass and error-free forms: tiles per sequential range (0: as many as
  // keep one range's stored V+- tiles within the cap)
  int tile_chunk = 0;
  bool last_two_pass = false;
  bool last_sym = false;  // the last error-free call took the symmetric-B form in one range
  std::vector<TcChunk> chunks_v;
  CUtensorMap tmA, tmB, tmTp, tmTm, tmVl;
  CUtensorMap tmGW, tmGT, tmGBs;  // split-BF16 dB operands
  int g_IJp = 0, g_Np = 0, g_ntiles = 0, g_npc = 0;
  // two-pass dB: Gamma stored once, contraction in the GEMM2 kernel
  bool g2 = false;
  int g2_ksplit = 1, g2_qsplit = 1, g2_cols = 0;
  std::vector<TcChunk> g2_chunks;
  CUtensorMap tmGl;
  Layout lay;
  // ragged batch: one sub-plan per molecule inside this plan's workspace
  bool batched = false;
  std::vector<ladder_plan_s *> subs;
  std::vector<size_t> sub_off;
  std::vector<int2> items, tcs;  // (molecule, local work unit), (molecule, tile*chunk)
  size_t off_mols = 0, off_items = 0, off_tcs = 0;
  // two-pass members: storing-pass and GEMM2-pass work units, unpack blocks
  std::vector<int2> items1, items2, tcs2;
  size_t off_mols1 = 0, off_mols2 = 0, off_items1 = 0, off_items2 = 0, off_tcs2 = 0;
  // symmetric-B error-free members: distinct-tile and V+- formation work units
  std::vector<int2> itemsX, itemsF;
  size_t off_itemsX = 0, off_itemsF = 0;
  size_t off_oz1 = 0, off_oz2 = 0;  // error-free batch: OzArgs tables of the two passes
  cudaStream_t cap_stream = nullptr;
  // ladder_apply_host: a side stream for the tau upload and its preparation,
  // and the events that fork it from and join it into the caller's stream
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_ev[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void *> gkey;  // pointers the graph was captured with
  bool timing = false;
  // 0..3: prep / ladder / unpack boundaries, 4: between the two passes,
  // 5..7: dressed call (start, Bd done, correction done), 8: symmetric B,
  // distinct integral tiles done (their V+- formation runs from 8 to 4)
  cudaEvent_t ev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void *ws = nullptr;
  size_t ws_bytes = 0;
};

namespace {

static int range_tiles(const ladder_plan_s *pl);

// Symmetric B: bytes of the distinct integral tiles (r <= q over the block
// pairs, 64 x 64 double-single each).
size_t xsym_bytes(const ladder_plan_s *pl) {
  return (size_t)pl->nbp * (pl->nbp + 1) / 2 * 4096 * sizeof(float2);
}

// Work units of the distinct-tile pass: row tiles (iA, kk >= 2 iA) in order,
// each against its column block pairs q >= ppos(kk) + 2 iA (the first row
// block pair it holds) in ranges that end at multiples of kXsymRange, so that
// the units of neighbouring row tiles, which run at the same time, read the
// same column block pairs.
std::vector<int4> make_xunits(int nb) {
  std::vector<int4> u;
  const int nbp = ppos(nb);
  for (int iA = 0; 2 * iA < nb; ++iA)
    for (int kk = 2 * iA; kk < nb; ++kk)
      for (int q0 = ppos(kk) + 2 * iA; q0 < nbp;) {
        const int q1 = std::min(nbp, (q0 / kXsymRange + 1) * kXsymRange);
        u.push_back(make_int4(iA, kk, q0, q1));
        q0 = q1;
      }
  return u;
}

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

// Occupied-pair chunks of the tensor-core kernels (whole j ranges; padded
// column counts with nps + nms <= maxcols).
std::vector<TcChunk> make_tc_chunks_greedy(int o, int maxcols) {
  auto pad16 = [](int x) { return (x + 15) / 16 * 16; };
  auto fits = [&](int j0, int j1) {
    const int np = pad16(ppos(j1) - ppos(j0)), nm = pad16(pneg(j1) - pneg(j0));
    return np + nm <= maxcols;
  };
  std::vector<TcChunk> out;
  int j0 = 0;
  while (j0 < o) {
    int j1 = j0 + 1;
    while (j1 < o && fits(j0, j1 + 1)) ++j1;
    TcChunk c;
    c.lp0 = ppos(j0);
    c.lm0 = pneg(j0);
    c.np = ppos(j1) - ppos(j0);
    c.nm = pneg(j1) - pneg(j0);
    c.nps = pad16(c.np);
    c.nms = pad16(c.nm);
    out.push_back(c);
    j0 = j1;
  }
  return out;
}

// As few chunks as the greedy split at `maxcols` gives, with the smallest
// column cap that keeps that count (so the chunks come out even).
std::vector<TcChunk> make_tc_chunks(int o, int maxcols) {
  const size_t n = make_tc_chunks_greedy(o, maxcols).size();
  for (int m = 32; m < maxcols; m += 16) {
    auto c = make_tc_chunks_greedy(o, m);
    if (c.size() == n) return c;
  }
  return make_tc_chunks_greedy(o, maxcols);
}

// Chunks of the two-pass GEMM2 kernel: lambda+ columns in nplus chunks of
// wplus, then lambda- columns in chunks of wminus (balanced, multiples of 16,
// at most maxcols).
// Lambda-only form: the ordered occupied pairs ij = i*o + j in balanced
// chunks of at most maxcols columns (multiples of 16).
std::vector<TcChunk> make_lam_chunks(int o, int maxcols, int &n, int &w) {
  const int cols = o * o;
  n = (cols + maxcols - 1) / maxcols;
  w = (((cols + n - 1) / n) + 15) / 16 * 16;
  std::vector<TcChunk> out;
  for (int c = 0; c * w < cols; ++c) {
    TcChunk t{};
    t.lp0 = c * w;
    t.np = std::min(w, cols - t.lp0);
    t.nps = (t.np + 15) / 16 * 16;
    out.push_back(t);
  }
  n = (int)out.size();
  return out;
}

std::vector<TcChunk> make_sign_chunks(int o, int maxcols, int &nplus, int &wplus, int &wminus) {
  auto pad16 = [](int x) { return (x + 15) / 16 * 16; };
  std::vector<TcChunk> out;
  const int nlp = ppos(o), nlm = pneg(o);
  nplus = (nlp + maxcols - 1) / maxcols;
  wplus = pad16((nlp + nplus - 1) / nplus);
  for (int c = 0; c < nplus; ++c) {
    TcChunk t{};
    t.lp0 = c * wplus;
    t.np = std::min(wplus, nlp - t.lp0);
    t.nps = pad16(t.np);
    out.push_back(t);
  }
  wminus = 16;
  if (nlm > 0) {
    const int nminus = (nlm + maxcols - 1) / maxcols;
    wminus = pad16((nlm + nminus - 1) / nminus);
    for (int c = 0; c < nminus; ++c) {
      TcChunk t{};
      t.lm0 = c * wminus;
      t.nm = std::min(wminus, nlm - t.lm0);
      t.nms = pad16(t.nm);
      out.push_back(t);
    }
  }
  return out;
}

// A device (or managed) pointer aligned to `align` bytes (16 for arrays, 8 for
// a single double).
bool dev_ptr_ok(const void *p, uintptr_t align = 16) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & (align - 1))) return false;
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
  if (pl->mode == LADDER_OZAKI) {
    // fixed-point B slices and row scales, V+- planes and their row scales,
    // tau+- per GEMM2 chunk and its row scales, the double-single sums
    const size_t S = pl->S;
    L.Bt = off;
    off = align_up(off + S * pl->vp * pl->vp * pl->Np * 2, 1024);
    L.ozRs = off;
    off = align_up(off + (size_t)pl->vp * pl->vp * sizeof(float));
    const size_t rt = range_tiles(pl);  // tiles of one sequential range
    L.slab = off;
    off = align_up(off + rt * pl->chunks_v.size() * pl->ksplit * 128 * pl->racc_cols_v * sizeof(float2), 1024);
    L.Vg = off;
    off = align_up(off + rt * pl->nbp * 2 * S * 128 * SLOTS * 2, 1024);
    L.ozSV = off;
    off = align_up(off + rt * pl->nbp * 2 * 128 * sizeof(float));
    L.T2 = off;
    size_t t2 = 0;
    for (auto &c : pl->chunks_v) {
      c.t2off = (long long)t2;
      t2 += (size_t)S * (c.nps + c.nms) * pl->K * 2;
    }
    off = align_up(off + t2, 1024);
    L.ozST = off;
    off = align_up(off + pl->chunks_v.size() * pl->nbp * kOzMaxCols * sizeof(float));
    if (pl->sym_b) {
      L.ozXs = off;
      off = align_up(off + xsym_bytes(pl), 1024);
      L.ozXu = off;
      off = align_up(off + pl->xunits.size() * sizeof(int4));
    }
  } else if (pl->mode == LADDER_FP64) {
    L.Tp = off;
    off = align_up(off + (size_t)pl->nlp * pl->K * sizeof(double));
    L.Tm = off;
    off = align_up(off + (size_t)std::max(pl->nlm, 1) * pl->K * sizeof(double));
    L.slab = off;
    if (pl->chunks64.size() > 1) off = align_up(off + fp64_slab_doubles(pl->K, pl->grid64) * sizeof(double));
  } else {
    const size_t S = pl->S;
    L.Bt = off;
    off = align_up(off + S * pl->vp * pl->vp * pl->Np * 2, 1024);
    L.Tp = off;
    off = align_up(off + S * pl->nlp * pl->K * 2, 1024);
    L.Tm = off;
    off = align_up(off + S * std::max(pl->nlm, 1) * pl->K * 2, 1024);
    L.slab = off;  // double-single accumulators of the tensor-core kernels
    const size_t nch = pl->two_pass ? pl->chunks_v.size() : pl->chunks_tc.size();
    const size_t cols = pl->two_pass ? pl->racc_cols_v : pl->racc_cols;
    const size_t rt = pl->two_pass ? range_tiles(pl) : pl->ntiles_tc;  // tiles of one range
    off = align_up(off + rt * nch * pl->ksplit * 128 * cols * sizeof(double), 1024);
    if (pl->two_pass) {
      L.Vg = off;
      off = align_up(off + rt * pl->nbp * 2 * S * 128 * SLOTS * 2, 1024);
      L.T2 = off;
      size_t t2 = 0;
      for (auto &c : pl->chunks_v) {
        c.t2off = (long long)t2;
        t2 += (size_t)S * (c.nps + c.nms) * pl->K * 2 * (pl->lam_only ? 2 : 1);
      }
      off = align_up(off + t2, 1024);
    }
  }
  L.W = off;
  L.gslab = off;  // FP64 dB: spill of the Gamma tiles
  if (pl->backward && pl->mode == LADDER_FP64)
    off = align_up(off + grad_fp64_slab_doubles(pl->vp, pl->N, pl->grid_grad) * sizeof(double));
  if (pl->backward && pl->mode != LADDER_FP64) {
    const size_t S = pl->S, vp = pl->vp;
    pl->g_IJp = (pl->o * pl->o + 31) / 32 * 32;
    pl->g_Np = (pl->N + 15) / 16 * 16;
    pl->g_ntiles = (pl->vp / 16) * (pl->vp / CB);
    pl->g_npc = (pl->g_Np + kGradTcPChunk - 1) / kGradTcPChunk;
    L.gWt = align_up(off, 1024);
    off = L.gWt + S * vp * vp * pl->g_IJp * 2;
    L.gTt = align_up(off, 1024);
    off = L.gTt + S * vp * vp * pl->g_IJp * 2;
    const size_t nq = (vp / CB) * (vp / CB);
    const double gbytes = (double)pl->g_ntiles * nq * S * 128 * SLOTS * 2;
    pl->g2 = gbytes <= 64.0 * (1ull << 30) &&
             (pl->N + kTcMaxColsV - 1) / kTcMaxColsV <= kMaxChunks;
    if (pl->g2) {
      // aux chunks of up to kTcMaxColsV rows, balanced
      pl->g2_chunks.clear();
      const int n = (pl->N + kTcMaxColsV - 1) / kTcMaxColsV;
      const int w = (((pl->N + n - 1) / n) + 15) / 16 * 16;
      pl->g2_cols = 0;
      size_t t2 = 0;
      for (int c = 0; c < n; ++c) {
        TcChunk t{};
        t.lp0 = c * w;
        t.np = std::min(w, pl->N - t.lp0);
        t.nps = (t.np + 15) / 16 * 16;
        t.t2off = (long long)t2;
        t2 += (size_t)nq * 4 * S * t.nps * 32;
        pl->g2_cols = std::max(pl->g2_cols, t.nps);
        pl->g2_chunks.push_back(t);
      }
      const int items = pl->g_ntiles * n;
      pl->g2_ksplit = std::max(1, std::min((int)nq, std::max((int)nq / 160,
                                                             (2 * pl->sm_count + items - 1) / items)));
      pl->g2_qsplit = std::max(1, std::min((int)nq, std::max((int)nq / 128,
                                                             (8 * pl->sm_count + pl->g_ntiles - 1) /
                                                                 pl->g_ntiles)));
      L.gG = align_up(off, 1024);
      off = L.gG + (size_t)gbytes;
      L.gT2 = align_up(off, 1024);
      off = L.gT2 + t2;
      L.gacc2 = align_up(off, 1024);
      off = align_up(L.gacc2 + (size_t)items * pl->g2_ksplit * 128 * pl->g2_cols * sizeof(double));
    } else {
      L.gBs = align_up(off, 1024);
      off = L.gBs + S * (size_t)pl->g_Np * vp * vp * 2;
      L.gacc = align_up(off, 1024);
      off = align_up(L.gacc + (size_t)pl->g_ntiles * pl->g_npc * 128 * kGradTcPChunk * sizeof(double));
    }
  }
  if (pl->dressed) {
    // t1 dressing (dress.cu): Bd [N][v][v] f64, then the correction in T
    // (double for FP64, float for the split modes): G [(k,l)][(c,d)],
    // X partials [dx_ksplit][(i,j)][(k,l)], Y [(i,j,k)][b]
    const size_t tsz = (pl->mode == LADDER_FP64 || pl->mode == LADDER_OZAKI) ? sizeof(double) : sizeof(float);
    const size_t o = pl->o, v = pl->v, oo = o * o;
    const long long xt = (long long)((oo + 127) / 128) * ((oo + 127) / 128);
    int ks = (int)((8LL * pl->sm_count + xt - 1) / xt);
    ks = std::max(1, std::min(ks, std::min(64, (int)std::max<size_t>(1, v * v / 1024))));
    pl->dx_ksplit = ks;
    L.dBd = align_up(off);
    off = L.dBd + (size_t)pl->N * v * v * sizeof(double);
    L.dG = align_up(off);
    off = L.dG + oo * v * v * tsz;
    L.dX = align_up(off);
    off = L.dX + (size_t)ks * oo * oo * tsz;
    L.dY = align_up(off);
    off = align_up(L.dY + oo * o * v * tsz);
  }
  L.total = off;
  pl->lay = L;
}

// Block-pair ranges per tile of the storing pass (no accumulators depend on
// them): at least about eight work units per SM, and ranges of at most about
// 128 block pairs, which the kernel walks range-major.  A batch member takes
// only the range limit (the batch itself fills the SMs).
// Tiles per sequential range of the two-pass and error-free forms: the
// requested count (tile_chunk), else as many as keep one range's stored V+-
// tiles within the cap (128 GiB, 200 GiB for the error-free mode); at least
// one.  Ranges run one after the other through both passes and the unpack,
// so a shape of any size keeps GEMM1 at one evaluation per (tile, block
// pair) and re-reads only B and tau per range.
static int range_tiles(const ladder_plan_s *pl) {
  if (pl->tile_chunk > 0) return std::min(pl->tile_chunk, pl->ntiles_tc);
  const double per_tile = (double)pl->nbp * 2 * pl->S * 128 * SLOTS * 2;
  double cap = pl->mode == LADDER_OZAKI ? kVStoreOzCap : kVStoreDefaultCap;
  if (pl->sym_b) cap -= (double)xsym_bytes(pl);
  return std::max(1, (int)std::min<double>(pl->ntiles_tc, cap / per_tile));
}

static int auto_vsplit(const ladder_plan_s *pl, bool batch_member) {
  int vs = batch_member ? 1 : (8 * pl->sm_count + pl->ntiles_tc - 1) / pl->ntiles_tc;
  vs = std::max(vs, (pl->nbp + 127) / 128);
  return std::max(1, std::min(vs, pl->nbp));
}

// Correction of the dressed term (dress.cu): R -= sum_kl t_k^a t_l^b X_ij^kl with
// X_ij^kl = sum_cd (kc|ld) tau_ij^cd, (kc|ld) = sum_P Bov^P_kc Bov^P_ld.
template <typename T>
ladder_status dress_correct(const ladder_plan_s *pl, const double *Bov, const double *t1,
                                   const double *tau, double *R, cudaStream_t s) {
  const int o = pl->o, v = pl->v;
  const long long ov = (long long)o * v, vv = (long long)v * v, oo = (long long)o * o;
  T *G = ws_at<T>(pl, pl->lay.dG), *X = ws_at<T>(pl, pl->lay.dX), *Y = ws_at<T>(pl, pl->lay.dY);
  // 1. G[(k,l)][(c,d)] = sum_P Bov[P][k][c] Bov[P][l][d]: M = N = o v, K = N_aux, symmetric
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.A = Bov;
  g.B = Bov;
  g.Out = G;
  g.sam = 1;
  g.sak = ov;
  g.sbn = 1;
  g.sbk = ov;
  g.M = g.N = (int)ov;
  g.K = pl->N;
  g.ksplit = 1;
  g.kchunk = pl->N;
  g.epi = kEpiPerm;
  g.sym = 1;
  g.po = o;
  g.pv = v;
  cudaError_t e = launch_gemm<double, double, T>(g, 1, s);
  // 2. X[(i,j)][(k,l)] = sum_(c,d) tau[(i,j)][(c,d)] G[(k,l)][(c,d)], split over (c,d)
  GemmArgs x;
  std::memset(&x, 0, sizeof(x));
  const int ks = pl->dx_ksplit;
  x.A = tau;
  x.B = G;
  x.Out = X;
  x.sam = vv;
  x.sak = 1;
  x.sbn = vv;
  x.sbk = 1;
  x.M = x.N = (int)oo;
  x.K = (int)vv;
  x.ksplit = ks;
  x.kchunk = (int)((vv + ks - 1) / ks + 7) / 8 * 8;
  x.ldo = (int)oo;
  x.so_batch = oo * oo;
  x.epi = kEpiStore;
  if (e == cudaSuccess) e = launch_gemm<double, T, T>(x, 1, s);
  if (e == cudaSuccess) e = launch_reduce<T>(X, oo * oo, ks, s);
  // 3. Y[(i,j,k)][b] = sum_l X[(i,j,k)][l] t1[l][b]: M = o^3, N = v, K = o
  GemmArgs y;
  std::memset(&y, 0, sizeof(y));
  y.A = X;
  y.B = t1;
  y.Out = Y;
  y.sam = o;
  y.sak = 1;
  y.sbn = 1;
  y.sbk = v;
  y.M = (int)(oo * o);
  y.N = v;
  y.K = o;
  y.ksplit = 1;
  y.kchunk = o;
  y.ldo = v;
  y.epi = kEpiStore;
  if (e == cudaSuccess) e = launch_gemm<T, double, T>(y, 1, s);
  // 4. R[(i,j)][a][b] -= sum_k t1[k][a] Y[(i,j)][k][b]: one v x v product per (i,j), K = o
  GemmArgs c;
  std::memset(&c, 0, sizeof(c));
  c.A = t1;
  c.B = Y;
  c.Out = R;
  c.sam = 1;
  c.sak = v;
  c.sbn = 1;
  c.sbk = v;
  c.sb_batch = ov;
  c.so_batch = vv;
  c.M = c.N = v;
  c.K = o;
  c.ksplit = 1;
  c.kchunk = o;
  c.ldo = v;
  c.epi = kEpiSubR;
  if (e == cudaSuccess) e = launch_gemm<double, T, T>(c, (int)oo, s);
  return cuda_status(e);
}

// ---- perturbative triples (Sec. II.A): workspace and launch sequence
struct TriplesLayout {
  size_t status = 0;  // word of the tensor-core kernel's bounded waits
  size_t ovvv = 0, ovvvT = 0, Q = 0, oovv = 0, t2c = 0, t2T = 0, W = 0, W2 = 0, part = 0, total = 0;
  // tensor-core W contractions: BF16 slices of the GEMM operands
  size_t tA1 = 0, tA1T = 0, tB1 = 0, tA2 = 0, tA2T = 0, tB2 = 0;
  int Nt = 0, K1p = 0, K2p = 0;
};

constexpr int kTwSlices = 3;

TriplesLayout triples_layout(int o, int v, bool fp32, bool tc = false) {
  const size_t t = fp32 ? sizeof(float) : sizeof(double);
  const size_t ov = (size_t)o * v, v3 = (size_t)v * v * v;
  TriplesLayout L;
  size_t off = kAlign;  // the status word
  L.ovvv = off;
  off = align_up(off + o * v3 * t);
  L.ovvvT = off;
  off = align_up(off + o * v3 * t);
  L.Q = off;
  off = align_up(off + (size_t)o * o * ov * t);
  L.oovv = off;
  off = align_up(off + ov * ov * t);
  L.t2c = off;  // FP32 only
  if (fp32) off = align_up(off + ov * ov * t);
  L.t2T = off;
  off = align_up(off + ov * ov * t);
  L.W = off;
  off = align_up(off + o * v3 * t);
  L.W2 = off;  // the second stream's W
  off = align_up(off + o * v3 * t);
  L.part = off;
  off = align_up(off + (size_t)o * o * o * triples_energy_blocks(v) * sizeof(double));
  if (tc) {
    // operand slices of the tensor-core W GEMMs, [S][g][rows][K] bf16
    L.Nt = (v + 15) / 16 * 16;
    L.K1p = (v + 31) / 32 * 32;
    L.K2p = (o + 15) / 16 * 16;
    const size_t S = kTwSlices, vv = (size_t)v * v;
    auto region = [&](size_t &at, size_t elems) {
      at = align_up(off, 1024);
      off = at + S * elems * 2;
    };
    region(L.tA1, (size_t)o * vv * L.K1p);
    region(L.tA1T, (size_t)o * vv * L.K1p);
    region(L.tB1, (size_t)o * o * L.Nt * L.K1p);
    region(L.tA2, (size_t)o * vv * L.K2p);
    region(L.tA2T, (size_t)o * vv * L.K2p);
    region(L.tB2, (size_t)o * o * L.Nt * L.K2p);
    off = align_up(off);
  }
  L.total = off;
  return L;
}

// E(T) = sum over (i, j), i >= j, of one batched pass over k <= j (the sorted
// triples; the energy kernel weighs each by the orderings it stands for):
//   W[k] = P applied to  sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab
// as twelve GEMMs (two per ordering of P), each written into W[k][a][b][c]
// through the kEpiAcc3 epilogue, then the energy kernel on W[k].
template <typename T>
cudaError_t triples_run(int o, int v, int n, const double *B, const double *Bov, const double *Boo,
                        const double *t1, const double *t2, const double *e_occ, const double *e_vir,
                        double *E, char *ws, const TriplesLayout &L, cudaStream_t s, bool tc = false) {
  T *ovvv = reinterpret_cast<T *>(ws + L.ovvv);
  T *ovvvT = reinterpret_cast<T *>(ws + L.ovvvT);
  T *Q = reinterpret_cast<T *>(ws + L.Q);
  T *oovv = reinterpret_cast<T *>(ws + L.oovv);
  T *Wbuf[2] = {reinterpret_cast<T *>(ws + L.W), reinterpret_cast<T *>(ws + L.W2)};
  double *part = reinterpret_cast<double *>(ws + L.part);
  const long long ov = (long long)o * v, vv = (long long)v * v, v3 = vv * v;
  const int M_rows = (int)vv;  // rows (alpha, beta) of every W GEMM
  auto base = [](GemmArgs &g) {
    std::memset(&g, 0, sizeof(g));
    g.ksplit = 1;
    g.alpha = 1.0;
  };
  GemmArgs g;
  // ovvv[i][b][a][d] = (bd|ai) = v_di^ba = sum_P Bov[P][i][a] Bvv[P][b][d]
  base(g);
  g.A = Bov;
  g.B = B;
  g.Out = ovvv;
  g.sam = 1;
  g.sak = ov;
  g.sbn = 1;
  g.sbk = vv;
  g.M = (int)ov;
  g.N = (int)vv;
  g.K = n;
  g.kchunk = n;
  g.epi = kEpiPerm;
  g.po = v;
  g.pv = v;
  g.pn = v;
  cudaError_t e = launch_gemm<double, double, T>(g, 1, s);
  // the same integrals as ovvvT[i][a][b][d] (rows (a, b)), for the orderings
  // whose b-index lands on W's contiguous index: ovvv with its middle two
  // indices exchanged
  if (e == cudaSuccess) e = launch_triples_swap12<T>(ovvv, ovvvT, o, v, s);
  // Q[k][j][c][l] = (ck|jl) = v_kl^cj = sum_P Bov[P][k][c] Boo[P][j][l] (negated below)
  base(g);
  g.A = Bov;
  g.B = Boo;
  g.Out = Q;
  g.sam = 1;
  g.sak = ov;
  g.sbn = 1;
  g.sbk = (long long)o * o;
  g.M = (int)ov;
  g.N = o * o;
  g.K = n;
  g.kchunk = n;
  g.epi = kEpiPerm;
  g.po = o;
  g.pv = v;
  g.pn = o;
  if (e == cudaSuccess) e = launch_gemm<double, double, T>(g, 1, s);
  // oovv[j][k][b][c] = (bj|ck) = v_jk^bc = sum_P Bov[P][j][b] Bov[P][k][c] (symmetric)
  base(g);
  g.A = Bov;
  g.B = Bov;
  g.Out = oovv;
  g.sam = 1;
  g.sak = ov;
  g.sbn = 1;
  g.sbk = ov;
  g.M = g.N = (int)ov;
  g.K = n;
  g.kchunk = n;
  g.epi = kEpiPerm;
  g.sym = 1;
  g.po = o;
  g.pv = v;
  g.pn = v;
  if (e == cudaSuccess) e = launch_gemm<double, double, T>(g, 1, s);
  // t2 in T (FP32 only) and with a <-> b exchanged
  T *t2c = std::is_same<T, double>::value ? nullptr : reinterpret_cast<T *>(ws + L.t2c);
  T *t2T = reinterpret_cast<T *>(ws + L.t2T);
  if (e == cudaSuccess) e = launch_triples_t2<T>(o, v, t2, t2c, t2T, s);
  // the second contraction enters W with a minus sign: keep -Q, so the GEMM
  // adds both of its K segments unscaled
  if (e == cudaSuccess) e = launch_triples_negate<T>(Q, (long long)o * o * ov, s);
  const T *t2x = t2c ? t2c : reinterpret_cast<const T *>(t2);
  // tensor-core W GEMMs: BF16 slices of the FP32 operands in their GEMM
  // layouts, and one tensor map per operand (see triples_tc.cu)
  TwArgs tw;
  std::memset(&tw, 0, sizeof(tw));
  int tw_grid = 0;
  int *tstatus = reinterpret_cast<int *>(ws + L.status);
  if (tc && e == cudaSuccess) e = cudaMemsetAsync(tstatus, 0, sizeof(int), s);
  if (tc && e == cudaSuccess) {
    const float *f_ovvv = reinterpret_cast<const float *>(ovvv), *f_ovvvT = reinterpret_cast<const float *>(ovvvT);
    const float *f_t2 = reinterpret_cast<const float *>(t2x), *f_t2T = reinterpret_cast<const float *>(t2T);
    const float *f_Q = reinterpret_cast<const float *>(Q);
    auto bf = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(ws + off); };
    const int M = (int)vv;
    // A1[x][m][d] = ovvv[x][m][d] (rows (b, a)) or ovvvT[x][m][d] (rows (a, b))
    e = launch_tw_slice(f_ovvv, v3, v, 1, o, M, M, v, L.K1p, bf(L.tA1), s);
    if (e == cudaSuccess) e = launch_tw_slice(f_ovvvT, v3, v, 1, o, M, M, v, L.K1p, bf(L.tA1T), s);
    // B1[(z, y)][gamma][d] = t2[z][y][gamma][d]
    if (e == cudaSuccess) e = launch_tw_slice(f_t2, vv, v, 1, o * o, v, L.Nt, v, L.K1p, bf(L.tB1), s);
    // A2[x][m][l] = t2[x][l][m] (rows (a, b)) or t2T[x][l][m] (rows (b, a))
    if (e == cudaSuccess) e = launch_tw_slice(f_t2, (long long)o * vv, 1, vv, o, M, M, o, L.K2p, bf(L.tA2), s);
    if (e == cudaSuccess) e = launch_tw_slice(f_t2T, (long long)o * vv, 1, vv, o, M, M, o, L.K2p, bf(L.tA2T), s);
    // B2[(z, y)][gamma][l] = -(gamma z | y l) = Q[z][y][gamma][l]
    if (e == cudaSuccess) e = launch_tw_slice(f_Q, ov, o, 1, o * o, v, L.Nt, o, L.K2p, bf(L.tB2), s);
    tw.status = tstatus;
    tw.M = M;
    tw.N = v;
    tw.Nt = L.Nt;
    tw.K1p = L.K1p;
    tw.K2p = L.K2p;
    tw.pv = v;
    tw.so_batch = v3;
    tw.timeout_ns = 2000000000ull;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    tw_grid = std::min(o * ((M + 127) / 128), sms);
    if (e == cudaSuccess) e = tw_init_attributes();
  }
  CUtensorMap mA1, mA1T, mA2, mA2T;
  if (tc && e == cudaSuccess) {
    const uint64_t S = kTwSlices, M = (uint64_t)vv, uo = (uint64_t)o;
    const bool ok =
        encode4d(&mA1, ws + L.tA1, L.K1p, M, uo, S, 32, 128, 1, (uint32_t)S, CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode4d(&mA1T, ws + L.tA1T, L.K1p, M, uo, S, 32, 128, 1, (uint32_t)S, CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode4d(&tw.tmB1, ws + L.tB1, L.K1p, L.Nt, uo * uo, S, 32, (uint32_t)L.Nt, 1, (uint32_t)S,
                 CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode4d(&mA2, ws + L.tA2, L.K2p, M, uo, S, 16, 128, 1, (uint32_t)S, CU_TENSOR_MAP_SWIZZLE_32B) &&
        encode4d(&mA2T, ws + L.tA2T, L.K2p, M, uo, S, 16, 128, 1, (uint32_t)S, CU_TENSOR_MAP_SWIZZLE_32B) &&
        encode4d(&tw.tmB2, ws + L.tB2, L.K2p, L.Nt, uo * uo, S, 16, (uint32_t)L.Nt, 1, (uint32_t)S,
                 CU_TENSOR_MAP_SWIZZLE_32B);
    if (!ok) e = cudaErrorInvalidValue;
  }
  // the six orderings of P: (x, y, z) = (I[p0], I[p1], I[p2]) with I = (i, j, k),
  // and (alpha, beta, gamma) = (A[p0], A[p1], A[p2]) with A = (a, b, c)
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {2, 0, 1}, {2, 1, 0}, {1, 2, 0}, {1, 0, 2}};
  const long long wstride[3] = {vv, v, 1};  // W[k][a][b][c]
  TriplesArgs ta;
  ta.oovv = oovv;
  ta.t1 = t1;
  ta.e_occ = e_occ;
  ta.e_vir = e_vir;
  ta.o = o;
  ta.v = v;
  // partials of the triples that are not sorted stay zero
  if (e == cudaSuccess)
    e = cudaMemsetAsync(part, 0, (size_t)o * o * o * triples_energy_blocks(v) * sizeof(double), s);
  // the (i, j) pairs alternate between the caller's stream and a second one,
  // each with its own W: the small k-batches of one pair leave SMs free for
  // the other's launches
  cudaStream_t st[2] = {s, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st[1], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st[1], ev[0], 0);
  int npair = 0;
  for (int i = 0; e == cudaSuccess && i < o; ++i)
    for (int j = 0; e == cudaSuccess && j <= i; ++j, ++npair) {
      const int I[3] = {i, j, 0};
      const int nk = j + 1;  // k = 0 .. j
      cudaStream_t sq = st[npair & 1];
      T *W = Wbuf[npair & 1];
      TwArgs twq[6];
      for (int q = 0; e == cudaSuccess && q < 6; ++q) {
        const int *p = perm[q];
        // x, y, z of the ordering; the one that is k varies with the batch
        const long long x = I[p[0]], y = I[p[1]], z = I[p[2]];
        const bool xk = p[0] == 2, yk = p[1] == 2, zk = p[2] == 2;
        // One GEMM per ordering, columns gamma, two K segments into the same
        // accumulators:  sum_d (bd|ai) t_zy^{gamma d}  over d, then
        // - sum_l t_xl^{alpha beta} (gamma z|y l)  over l.  The rows are
        // (beta, alpha) when alpha is W's contiguous index c, else (alpha, beta),
        // so the epilogue's row-fastest writes stay contiguous.
        const bool rowsBA = p[0] == 2;
        base(g);
        g.A = (rowsBA ? ovvv : ovvvT) + (xk ? 0 : x * v3);
        g.sa_batch = xk ? v3 : 0;
        g.sam = v;
        g.sak = 1;
        g.B = t2x + (zk ? 0 : z * o * vv) + (yk ? 0 : y * vv);
        g.sb_batch = (zk ? (long long)o * vv : 0) + (yk ? vv : 0);
        g.sbn = v;
        g.sbk = 1;
        g.M = (int)vv;
        g.N = v;
        g.K = v;
        g.kchunk = v;
        g.A2 = (rowsBA ? (const T *)t2T : t2x) + (xk ? 0 : x * o * vv);
        g.sa2_batch = xk ? (long long)o * vv : 0;
        g.sam2 = 1;
        g.sak2 = vv;
        g.B2 = Q + (zk ? 0 : z * o * ov) + (yk ? 0 : y * ov);
        g.sb2_batch = (zk ? (long long)o * ov : 0) + (yk ? ov : 0);
        g.sbn2 = o;
        g.sbk2 = 1;
        g.K2 = o;
        g.beta2 = 1.0;  // Q holds -(ck|jl)
        g.Out = W;
        g.so_batch = v3;
        g.epi = kEpiAcc3;
        g.pv = v;
        g.s1 = wstride[rowsBA ? p[1] : p[0]];
        g.s2 = wstride[rowsBA ? p[0] : p[1]];
        g.s3 = wstride[p[2]];
        g.acc = q > 0;
        if (tc) {
          // the same contraction on the tensor cores: operand g-indices
          // fixed or the batch (k) itself, the same output strides
          tw.tmA1 = rowsBA ? mA1 : mA1T;
          tw.a1_fix = xk ? 0 : (int)x;
          tw.a1_mul = xk ? 1 : 0;
          tw.b1_fix = (zk ? 0 : (int)z * o) + (yk ? 0 : (int)y);
          tw.b1_mul = zk ? o : (yk ? 1 : 0);
          tw.tmA2 = rowsBA ? mA2T : mA2;
          tw.a2_fix = tw.a1_fix;
          tw.a2_mul = tw.a1_mul;
          tw.b2_fix = tw.b1_fix;
          tw.b2_mul = tw.b1_mul;
          tw.s1 = g.s1;
          tw.s2 = g.s2;
          tw.s3 = g.s3;
          tw.acc = g.acc;
          tw.batch = nk;
          tw.W = reinterpret_cast<float *>(W);
          tw.nord = 1;
          twq[q] = tw;
        } else {
          e = launch_gemm<T, T, T>(g, nk, sq);
        }
      }
      if (tc) {
        // orderings 1 and 2 write W through the same strides (rows (a, c),
        // columns b), and so do 3 and 4 (rows (b, c), columns a): each pair
        // runs as one launch whose second ordering adds its K segments into
        // the same accumulators, so W is read and written four times, not six
        auto same_out = [&](int x, int y) {
          return twq[x].s1 == twq[y].s1 && twq[x].s2 == twq[y].s2 && twq[x].s3 == twq[y].s3;
        };
        for (int q = 0; e == cudaSuccess && q < 6; ++q) {
          TwArgs a = twq[q];
          if ((q == 1 || q == 3) && same_out(q, q + 1)) {
            const TwArgs &b2 = twq[q + 1];
            a.nord = 2;
            a.tmA1b = b2.tmA1;
            a.tmA2b = b2.tmA2;
            a.a1b_fix = b2.a1_fix;
            a.a1b_mul = b2.a1_mul;
            a.b1b_fix = b2.b1_fix;
            a.b1b_mul = b2.b1_mul;
            ++q;
          }
          e = launch_tw_gemm(a, std::min(tw_grid, nk * ((M_rows + 127) / 128)), sq);
        }
      }
      if (e == cudaSuccess) e = launch_triples_energy<T>(ta, W, i, j, part, sq);
    }
  // join the second stream back into the caller's
  if (st[1]) {
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st[1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    cudaStreamDestroy(st[1]);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  // E = NaN if a bounded wait of the tensor-core kernel ran out
  if (e == cudaSuccess)
    e = launch_triples_final(part, (long long)o * o * o * triples_energy_blocks(v), E, s, tc ? tstatus : nullptr);
  return e;
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
    case LADDER_ENONFINITE: return "an input holds a NaN or an infinity";
  }
  return "unknown status";
}

// Block-pair ranges per (tile, chunk): enough work units that small problems
// give every SM work; in the two-pass form also ranges of about 160 block
// pairs, which the GEMM2 kernel walks range-major so that the resident CTAs
// share their tau+- and V+- reads in L2.
static int auto_ksplit(const ladder_plan_s *pl) {
  const int nch = (int)(pl->two_pass ? pl->chunks_v.size() : pl->chunks_tc.size());
  const int items = pl->ntiles_tc * nch;
  int ks = (2 * pl->sm_count + items - 1) / items;
  if (pl->two_pass) ks = std::max(ks, pl->nbp / 160);
  return std::max(1, std::min(ks, std::max(1, pl->nbp / 4)));
}

// Fills a plan for one shape; batch members get no block-pair split (the
// batch itself keeps every SM busy).
static ladder_status init_plan(ladder_plan_s *pl, int o, int v, int naux, int mode,
                               bool with_backward, bool batch_member, bool with_dressing = false) {
  if (o < 1 || o > 256 || v < 1 || v > 4096 || naux < 1 || naux > 65536) return LADDER_EINVAL;
  if (mode < LADDER_FP64 || mode > LADDER_OZAKI) return LADDER_EINVAL;
  if (mode == LADDER_AUTO) mode = LADDER_BF16X6;
  if (mode == LADDER_OZAKI && with_backward) return LADDER_ENOTSUP;
  pl->o = o;
  pl->v = v;
  pl->N = naux;
  pl->mode = mode;
  pl->backward = with_backward;
  pl->dressed = with_dressing;
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
    return LADDER_ECUDA;
  }
  pl->chunks64 = make_chunks(o, kFp64LamTile);
  if (mode == LADDER_OZAKI) {
    // error-free split: always the two-pass form, GEMM2 chunks of <= 128 pairs
    pl->S = pl->oz_slices;
    pl->Np = (naux + 31) / 32 * 32;
    pl->chunks_v = make_sign_chunks(o, kOzMaxCols, pl->nplus, pl->wplus, pl->wminus);
    pl->racc_cols_v = 0;
    for (auto &c : pl->chunks_v) pl->racc_cols_v = std::max(pl->racc_cols_v, c.nps + c.nms);
    const int nA = pl->vp / 16, nB8 = pl->vp / CB;
    pl->ntiles_tc = 0;
    for (int i = 0; i < nA; ++i) pl->ntiles_tc += nB8 - 2 * i;
    pl->ntiles_all = pl->ntiles_tc;
    pl->two_pass = 1;
    pl->ksplit = auto_ksplit(pl);
    pl->vsplit = auto_vsplit(pl, batch_member);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, pl->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, pl->device);
    if ((int)pl->chunks_v.size() > kMaxChunks || major != 10 || minor != 3) return LADDER_ENOTSUP;
  } else if (mode != LADDER_FP64) {
    pl->S = tc_slices(mode);
    pl->Np = (naux + 31) / 32 * 32;
    pl->chunks_tc = make_tc_chunks(o, kTcMaxCols);
    pl->chunks_v = make_sign_chunks(o, kTcMaxColsV, pl->nplus, pl->wplus, pl->wminus);
    pl->racc_cols = pl->racc_cols_v = 0;
    for (auto &c : pl->chunks_tc) pl->racc_cols = std::max(pl->racc_cols, c.nps + c.nms);
    for (auto &c : pl->chunks_v) pl->racc_cols_v = std::max(pl->racc_cols_v, c.nps + c.nms);
    const int nA = pl->vp / 16, nB8 = pl->vp / CB;
    pl->ntiles_tc = 0;
    for (int i = 0; i < nA; ++i) pl->ntiles_tc += nB8 - 2 * i;
    pl->ntiles_all = pl->ntiles_tc;
    // the two-pass form for every single-molecule plan: it avoids the fused
    // kernel's per-chunk GEMM1 recompute, its storing pass issues wider MMAs
    // (it measured faster even where one chunk suffices: o=10, v=120, 1.60
    // vs 2.44 ms), and shapes whose stored tiles exceed the cap run in
    // sequential tile ranges (range_tiles)
    pl->two_pass = batch_member ? 0 : 1;
    pl->ksplit = batch_member ? 1 : auto_ksplit(pl);
    pl->vsplit = auto_vsplit(pl, batch_member);
    // FP32 accumulation chains (see ladder_tc.cu).  GEMM1: with separate
    // hi*hi / small-product accumulators a chain of kc K-steps puts 2*kc MMAs
    // on the large accumulator (32 for BF16X3, 8 for BF16X6).  GEMM2: a fresh
    // S every block pair (12 MMAs, BF16X3) or every two pieces (12 MMAs,
    // BF16X6; the autotuner's choice on every shape it was run on).
    pl->xy_split = 1;
    pl->kc = pl->S == 2 ? 16 : 4;
    pl->s_pieces = pl->S == 2 ? 4 : 2;
    // GEMM2's FP32 running sum R takes flush_every S accumulators before a
    // flush into the double-single sums.  At o=34, v=400 (BF16X6, two-pass)
    // flushing every 16 / 32 / 64 / 128 S gave pass 2 113 / 101 / 94 / 91 ms
    // and R errors 5.05 / 5.07 / 5.08 / 5.29e-7: 64 keeps the error.
    pl->flush_every = 64;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, pl->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, pl->device);
    if ((int)pl->chunks_tc.size() > kMaxChunks || (int)pl->chunks_v.size() > kMaxChunks ||
        major != 10 || minor != 3)
      return LADDER_ENOTSUP;
  } else if ((int)pl->chunks64.size() > kMaxChunks) {
    return LADDER_ENOTSUP;
  }
  Fp64Args tmp{};
  tmp.ntiles = ppos(pl->vp / CB);
  pl->grid64 = fp64_grid(tmp, pl->sm_count);
  pl->grid_grad = grad_fp64_grid(pl->vp, pl->sm_count);
  compute_layout(pl);
  return LADDER_OK;
}

ladder_status ladder_plan(int o, int v, int naux, int mode, ladder_plan_t *out) {
  if (!out) return LADDER_EINVAL;
  *out = nullptr;
  const bool with_backward = (mode & LADDER_WITH_BACKWARD) != 0;
  const bool with_dressing = (mode & LADDER_WITH_DRESSING) != 0;
  mode &= ~(LADDER_WITH_BACKWARD | LADDER_WITH_DRESSING);
  ladder_plan_s *pl = new (std::nothrow) ladder_plan_s();
  if (!pl) return LADDER_ENOMEM;
  const ladder_status st = init_plan(pl, o, v, naux, mode, with_backward, false, with_dressing);
  if (st != LADDER_OK) {
    delete pl;
    return st;
  }
  *out = pl;
  return LADDER_OK;
}

ladder_status ladder_plan_shape(ladder_plan_t pl, int *o, int *v, int *naux) {
  if (!pl || pl->batched || !o || !v || !naux) return LADDER_EINVAL;
  *o = pl->o;
  *v = pl->v;
  *naux = pl->N;
  return LADDER_OK;
}

ladder_status ladder_plan_mode(ladder_plan_t pl, int *mode) {
  if (!pl || !mode) return LADDER_EINVAL;
  *mode = pl->mode;
  return LADDER_OK;
}

ladder_status ladder_get_tuning(ladder_plan_t pl, ladder_tuning *t) {
  if (!pl || !t || pl->batched) return LADDER_EINVAL;
  t->kc = pl->kc;
  t->s_pieces = pl->s_pieces;
  t->flush_every = pl->flush_every;
  t->ksplit = pl->ksplit;
  t->xy_split = pl->xy_split;
  t->two_pass = pl->two_pass;
  t->lambda_only = pl->lam_only;
  t->oz_slices = pl->mode == LADDER_OZAKI ? pl->oz_slices : 0;
  t->tile_chunk = pl->tile_chunk;
  t->sym_b = pl->sym_b;
  return LADDER_OK;
}

ladder_status ladder_set_tuning(ladder_plan_t pl, const ladder_tuning *t) {
  if (!pl || !t || pl->batched || pl->ws) return LADDER_EINVAL;
  if (pl->mode == LADDER_FP64) return LADDER_OK;
  if (pl->mode == LADDER_OZAKI) {
    // only the slice count and the block-pair split apply
    if ((t->oz_slices != 0 && t->oz_slices != 5 && t->oz_slices != 6) || t->ksplit < 0 || t->ksplit > pl->nbp ||
        t->two_pass != 1 || t->lambda_only != 0 || t->tile_chunk < 0 || (t->sym_b != 0 && t->sym_b != 1))
      return LADDER_EINVAL;
    // the distinct integral tiles serve every tile of the shape (a plan with
    // a tile range forms all of them and V+- of its own tiles), while they
    // fit their cap; B - mbar of the dressed term is not symmetric
    if (t->sym_b && (pl->dressed || (double)xsym_bytes(pl) > kXsymCap)) return LADDER_ENOTSUP;
    if (t->oz_slices) pl->oz_slices = pl->S = t->oz_slices;
    pl->tile_chunk = t->tile_chunk;
    pl->sym_b = t->sym_b;
    pl->xunits = pl->sym_b ? make_xunits(pl->nb) : std::vector<int4>();
    pl->ksplit = t->ksplit ? t->ksplit : auto_ksplit(pl);
    compute_layout(pl);
    return LADDER_OK;
  }
  if (t->sym_b != 0) return LADDER_EINVAL;
  if (t->kc < 1 || t->kc > 64 || !(t->s_pieces == 1 || t->s_pieces == 2 || t->s_pieces == 4) ||
      t->flush_every < 1 || t->flush_every > 4096 || t->ksplit < 0 || t->ksplit > pl->nbp ||
      (t->xy_split != 0 && t->xy_split != 1) || (t->two_pass != 0 && t->two_pass != 1) ||
      (t->lambda_only != 0 && t->lambda_only != 1) || (t->lambda_only && !t->two_pass) || t->tile_chunk < 0)
    return LADDER_EINVAL;
  pl->tile_chunk = t->tile_chunk;
  if (t->lambda_only != pl->lam_only) {
    pl->lam_only = t->lambda_only;
    if (pl->lam_only) {
      pl->chunks_v = make_lam_chunks(pl->o, kTcMaxColsV, pl->nplus, pl->wplus);
      pl->wminus = 16;
    } else {
      pl->chunks_v = make_sign_chunks(pl->o, kTcMaxColsV, pl->nplus, pl->wplus, pl->wminus);
    }
    if ((int)pl->chunks_v.size() > kMaxChunks) return LADDER_ENOTSUP;
    pl->racc_cols_v = 0;
    for (auto &c : pl->chunks_v) pl->racc_cols_v = std::max(pl->racc_cols_v, c.nps + c.nms);
  }
  pl->kc = t->kc;
  pl->s_pieces = t->s_pieces;
  pl->flush_every = t->flush_every;
  pl->xy_split = t->xy_split;
  pl->two_pass = t->two_pass;
  pl->ksplit = t->ksplit ? t->ksplit : auto_ksplit(pl);
  compute_layout(pl);
  return LADDER_OK;
}

ladder_status ladder_tile_count(ladder_plan_t pl, int *ntiles) {
  if (!pl || !ntiles || pl->batched) return LADDER_EINVAL;
  if (pl->mode == LADDER_FP64) return LADDER_ENOTSUP;
  *ntiles = pl->ntiles_all;
  return LADDER_OK;
}

ladder_status ladder_set_tile_range(ladder_plan_t pl, int tile_lo, int tile_hi) {
  if (!pl || pl->batched || pl->ws) return LADDER_EINVAL;
  if (pl->mode == LADDER_FP64) return LADDER_ENOTSUP;
  if (tile_lo < 0 || tile_hi > pl->ntiles_all || tile_lo >= tile_hi) return LADDER_EINVAL;
  pl->tile0 = tile_lo;
  pl->ntiles_tc = tile_hi - tile_lo;
  pl->ksplit = auto_ksplit(pl);
  pl->vsplit = auto_vsplit(pl, false);
  compute_layout(pl);
  return LADDER_OK;
}

ladder_status ladder_workspace_size(ladder_plan_t pl, size_t *bytes) {
  if (!pl || !bytes) return LADDER_EINVAL;
  *bytes = pl->lay.total;
  return LADDER_OK;
}

static ladder_status encode_maps(ladder_plan_s *pl, char *w) {
  if (pl->mode == LADDER_FP64) return LADDER_OK;
  if (pl->mode == LADDER_OZAKI) {
    const uint64_t S = pl->S;
    const uint64_t planes = (uint64_t)range_tiles(pl) * pl->nbp * 2 * S;
    const bool ok =
        encode4d(&pl->tmA, w + pl->lay.Bt, pl->Np, pl->vp, pl->vp, S, 32, 8, 16, (uint32_t)S,
                 CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode4d(&pl->tmB, w + pl->lay.Bt, pl->Np, pl->vp, pl->vp, S, 32, 8, 8, (uint32_t)S,
                 CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode3d(&pl->tmVl, w + pl->lay.Vg, SLOTS, 128, planes, 16, 128, (uint32_t)S, CU_TENSOR_MAP_SWIZZLE_32B);
    if (!ok) return LADDER_ECUDA;
    return cuda_status(oz_init_attributes(pl->S));
  }
  const uint64_t S = pl->S;
  const bool ok =
      encode4d(&pl->tmA, w + pl->lay.Bt, pl->Np, pl->vp, pl->vp, S, 32, 8, 16, (uint32_t)S,
               CU_TENSOR_MAP_SWIZZLE_64B) &&
      encode4d(&pl->tmB, w + pl->lay.Bt, pl->Np, pl->vp, pl->vp, S, 32, 8, 8, (uint32_t)S,
               CU_TENSOR_MAP_SWIZZLE_64B) &&
      encode3d(&pl->tmTp, w + pl->lay.Tp, pl->K, pl->nlp, S, 16, 16, 1, CU_TENSOR_MAP_SWIZZLE_32B) &&
      encode3d(&pl->tmTm, w + pl->lay.Tm, pl->K, std::max(pl->nlm, 1), S, 16, 16, 1,
               CU_TENSOR_MAP_SWIZZLE_32B);
  if (!ok) return LADDER_ECUDA;
  if (pl->two_pass) {
    const uint64_t planes = (uint64_t)range_tiles(pl) * pl->nbp * 2 * S;
    const bool okv = encode3d(&pl->tmVl, w + pl->lay.Vg, SLOTS, 128, planes, 16, 128, (uint32_t)S,
                              CU_TENSOR_MAP_SWIZZLE_32B);
    if (!okv) return LADDER_ECUDA;
  }
  if (pl->backward) {
    const uint64_t vp = pl->vp;
    const bool okg =
        encode3d(&pl->tmGW, w + pl->lay.gWt, pl->g_IJp, vp, vp * S, 32, 8, 16,
                 CU_TENSOR_MAP_SWIZZLE_64B) &&
        encode3d(&pl->tmGT, w + pl->lay.gTt, pl->g_IJp, vp, vp * S, 32, 8, 8,
                 CU_TENSOR_MAP_SWIZZLE_64B) &&
        (pl->g2 ? encode3d(&pl->tmGl, w + pl->lay.gG, SLOTS, 128,
                           (uint64_t)pl->g_ntiles * (vp / CB) * (vp / CB) * S, 16, 128, (uint32_t)S,
                           CU_TENSOR_MAP_SWIZZLE_32B)
                : encode3d(&pl->tmGBs, w + pl->lay.gBs, vp * CB, vp / CB, (uint64_t)pl->g_Np * S, 16, 1, 16,
                           CU_TENSOR_MAP_SWIZZLE_32B));
    if (!okg) return LADDER_ECUDA;
    const ladder_status st = cuda_status(grad_tc_init_attributes(pl->S));
    if (st != LADDER_OK) return st;
  }
  return cuda_status(tc_init_attributes(pl->S));
}

ladder_status ladder_set_workspace(ladder_plan_t pl, void *dptr, size_t bytes) {
  if (!pl) return LADDER_EINVAL;
  if (bytes < pl->lay.total) return LADDER_EWORKSPACE;
  if (!dptr || (reinterpret_cast<uintptr_t>(dptr) % kAlign)) return LADDER_EINVAL;
  if (!dev_ptr_ok(dptr)) return LADDER_EINVAL;
  char *w = static_cast<char *>(dptr);
  if (pl->batched) {
    for (size_t m = 0; m < pl->subs.size(); ++m) {
      ladder_plan_s *sp = pl->subs[m];
      sp->ws = w + pl->sub_off[m];
      sp->ws_bytes = sp->lay.total;
      const ladder_status st = encode_maps(sp, static_cast<char *>(sp->ws));
      if (st != LADDER_OK) return st;
      if (sp->sym_b && cudaMemcpy(static_cast<char *>(sp->ws) + sp->lay.ozXu, sp->xunits.data(),
                                  sp->xunits.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_status(cudaErrorUnknown);
    }
    // work lists of the batched launches
    const std::pair<size_t, const std::vector<int2> *> lists[] = {
        {pl->off_items, &pl->items},   {pl->off_tcs, &pl->tcs},     {pl->off_items1, &pl->items1},
        {pl->off_items2, &pl->items2}, {pl->off_tcs2, &pl->tcs2},   {pl->off_itemsX, &pl->itemsX},
        {pl->off_itemsF, &pl->itemsF}};
    for (const auto &li : lists)
      if (!li.second->empty() &&
          cudaMemcpy(w + li.first, li.second->data(), li.second->size() * sizeof(int2),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_status(cudaErrorUnknown);
    if (pl->gexec) {
      cudaGraphExecDestroy(pl->gexec);
      pl->gexec = nullptr;
      pl->gkey.clear();
    }
  } else {
    const ladder_status st = encode_maps(pl, w);
    if (st != LADDER_OK) return st;
    if (pl->sym_b && cudaMemcpy(w + pl->lay.ozXu, pl->xunits.data(), pl->xunits.size() * sizeof(int4),
                                cudaMemcpyHostToDevice) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
  }
  pl->ws = dptr;
  pl->ws_bytes = bytes;
  // the status word starts cleared
  if (cudaMemset(dptr, 0, sizeof(int)) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  return LADDER_OK;
}

ladder_status ladder_tau(ladder_plan_t pl, const double *t1, const double *t2, double *tau,
                         void *stream) {
  if (!pl || pl->batched || !dev_ptr_ok(t1) || !dev_ptr_ok(t2) || !dev_ptr_ok(tau) || tau == t2)
    return LADDER_EINVAL;
  launch_tau(pl->o, pl->v, t1, t2, tau, static_cast<cudaStream_t>(stream));
  return cuda_status(cudaGetLastError());
}

static void mark(ladder_plan_t pl, int k, cudaStream_t s) {
  if (pl->timing) cudaEventRecord(pl->ev[k], s);
}

static ladder_status apply_fp64(ladder_plan_t pl, const double *B, const double *tau, double *R,
                                cudaStream_t s, bool transB = false) {
  pl->last_two_pass = false;
  mark(pl, 0, s);
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
  a.transB = transB ? 1 : 0;
  a.nchunks = (int)pl->chunks64.size();
  for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->chunks64[c];
  mark(pl, 1, s);
  st = cuda_status(launch_ladder_fp64(a, pl->grid64, s));
  mark(pl, 2, s);
  mark(pl, 3, s);
  return st;
}

static double tc_timeout_ns(const ladder_plan_s *pl) {
  // generous bound on any single wait: 2 s plus 20x the estimated item time
  const double item_flops = 2.0 * pl->nbp * 2.0 * 128.0 * 64.0 * pl->Np * 6.0 / pl->ksplit;
  return 2e9 + 20.0 * item_flops / 4e12 * 1e9;
}

static TcArgs tc_args(const ladder_plan_s *pl, double *R, int *status) {
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tmA = pl->tmA;
  a.tmB = pl->tmB;
  a.tmTp = pl->tmTp;
  a.tmTm = pl->tmTm;
  a.tmVl = pl->tmVl;
  a.Vst = pl->two_pass ? ws_at<__nv_bfloat16>(pl, pl->lay.Vg) : nullptr;
  a.T2 = pl->two_pass ? ws_at<uint8_t>(pl, pl->lay.T2) : nullptr;
  a.R = R;
  a.status = status;
  a.o = pl->o;
  a.v = pl->v;
  a.vp = pl->vp;
  a.Np = pl->Np;
  a.K = pl->K;
  a.nbp = pl->nbp;
  a.nks = pl->Np / 32;
  a.nA = pl->vp / 16;
  a.nB8 = pl->vp / CB;
  a.ntiles = pl->ntiles_tc;
  a.tile0 = pl->tile0;
  a.nchunks = (int)pl->chunks_tc.size();
  a.ksplit = pl->ksplit;
  a.racc = ws_at<float2>(pl, pl->lay.slab);
  a.racc_cols = pl->racc_cols;
  a.kc = pl->kc;
  a.xy_split = pl->xy_split;
  a.s_pieces = pl->s_pieces;
  a.flush_every = pl->flush_every;
  for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->chunks_tc[c];
  a.timeout_ns = (unsigned long long)tc_timeout_ns(pl);
  a.nsign = 2;
  a.lam_only = pl->lam_only;
  return a;
}

// status: the device status word that a NaN or infinite input is reported to
static void tc_prep(ladder_plan_t pl, const double *B, const double *tau, cudaStream_t s,
                    bool transB, int *status) {
  auto *Bt = ws_at<__nv_bfloat16>(pl, pl->lay.Bt);
  auto *Tp = ws_at<__nv_bfloat16>(pl, pl->lay.Tp);
  auto *Tm = ws_at<__nv_bfloat16>(pl, pl->lay.Tm);
  launch_split_B(pl->N, pl->v, pl->vp, pl->Np, pl->S, B, Bt, s, transB, status);
  if (pl->lam_only && pl->two_pass) {
    // the lambda-only GEMM2 operand comes straight from tau (pack_t2_lam)
    T2LamArgs t;
    std::memset(&t, 0, sizeof(t));
    t.tau = tau;
    t.T2 = ws_at<__nv_bfloat16>(pl, pl->lay.T2);
    t.o = pl->o;
    t.v = pl->v;
    t.K = pl->K;
    t.S = pl->S;
    t.nchunks = (int)pl->chunks_v.size();
    for (int c = 0; c < t.nchunks; ++c) t.chunks[c] = pl->chunks_v[c];
    launch_pack_t2_lam(t, s);
    return;
  }
  launch_pack_tpm_bf16(pl->o, pl->v, pl->K, pl->S, pl->nlp, std::max(pl->nlm, 1), tau, Tp, Tm, s, status);
}

// Arguments of the storing pass (GEMM1 + V+- store) of the two-pass form.
static TcArgs pass1_args(const ladder_plan_s *pl, int *status) {
  TcArgs a = tc_args(pl, nullptr, status);
  a.nchunks = 1;
  std::memset(&a.chunks[0], 0, sizeof(TcChunk));
  a.ksplit = pl->vsplit;
  a.racc = nullptr;
  return a;
}

// Arguments of the GEMM2 pass of the two-pass form (sign-separated chunks).
static TcArgs pass2_args(const ladder_plan_s *pl, double *R, int *status) {
  TcArgs a = tc_args(pl, R, status);
  a.nchunks = (int)pl->chunks_v.size();
  for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->chunks_v[c];
  a.racc_cols = pl->racc_cols_v;
  a.nplus = pl->nplus;
  a.wplus = pl->wplus;
  a.wminus = pl->wminus;
  return a;
}

// Chunk-major, pre-swizzled copy of the tau+- slices for the GEMM2 pass.
static void pack_t2(const ladder_plan_s *pl, cudaStream_t s) {
  T2Args t2;
  std::memset(&t2, 0, sizeof(t2));
  t2.Tp = ws_at<__nv_bfloat16>(pl, pl->lay.Tp);
  t2.Tm = ws_at<__nv_bfloat16>(pl, pl->lay.Tm);
  t2.T2 = ws_at<__nv_bfloat16>(pl, pl->lay.T2);
  t2.K = pl->K;
  t2.S = pl->S;
  t2.rows_p = pl->nlp;
  t2.rows_m = std::max(pl->nlm, 1);
  t2.nchunks = (int)pl->chunks_v.size();
  for (int c = 0; c < t2.nchunks; ++c) {
    t2.chunks[c] = pl->chunks_v[c];
    t2.off[c] = pl->chunks_v[c].t2off / 2;
  }
  launch_pack_t2(t2, s);
}

static ladder_status apply_tc(ladder_plan_t pl, const double *B, const double *tau, double *R,
                              cudaStream_t s, bool transB = false) {
  mark(pl, 0, s);
  int *status = ws_at<int>(pl, pl->lay.status);
  tc_prep(pl, B, tau, s, transB, status);
  ladder_status st = cuda_status(cudaGetLastError());
  if (st != LADDER_OK) return st;
  TcLaunch L;
  std::memset(&L, 0, sizeof(L));
  if (pl->two_pass) {
    if (!pl->lam_only) pack_t2(pl, s);
    st = cuda_status(cudaGetLastError());
    if (st != LADDER_OK) return st;
    // tile ranges one after the other (one range unless the stored tiles of
    // all tiles exceed the cap): pass 1 stores GEMM1's V+- slices of every
    // (tile, block pair) of the range, pass 2 contracts them in chunks of up
    // to kTcMaxColsV occupied pairs of one sign, the unpack writes R
    const int nt = pl->ntiles_tc, rt = range_tiles(pl);
    const bool one = rt >= nt;
    pl->last_two_pass = one;
    mark(pl, 1, s);
    for (int r0 = 0; r0 < nt && st == LADDER_OK; r0 += rt) {
      const int cnt = std::min(rt, nt - r0);
      TcLaunch L1 = L;
      L1.one = pass1_args(pl, status);
      L1.one.tile0 += r0;
      L1.one.ntiles = cnt;
      L1.timeout_ns = L1.one.timeout_ns;
      L1.nitems = cnt * L1.one.ksplit;
      TcLaunch L2 = L;
      L2.one = pass2_args(pl, R, status);
      L2.one.tile0 += r0;
      L2.one.ntiles = cnt;
      L2.timeout_ns = L2.one.timeout_ns;
      L2.nitems = cnt * L2.one.nchunks * L2.one.ksplit;
      st = cuda_status(launch_ladder_vstore(L1, pl->S, L1.nitems, s));
      if (one) mark(pl, 4, s);
      if (st == LADDER_OK) st = cuda_status(launch_ladder_gemm2(L2, pl->S, L2.nitems, s));
      if (one) mark(pl, 2, s);
      if (st == LADDER_OK)
        st = cuda_status(pl->lam_only ? launch_unpack_lam(L2, cnt * L2.one.nchunks, s)
                                      : launch_unpack2(L2, cnt * L2.one.nplus, s));
    }
    if (!one) mark(pl, 2, s);
  } else {
    pl->last_two_pass = false;
    L.one = tc_args(pl, R, status);
    L.timeout_ns = L.one.timeout_ns;
    L.nitems = L.one.ntiles * L.one.nchunks * L.one.ksplit;
    mark(pl, 1, s);
    st = cuda_status(launch_ladder_tc(L, pl->S, L.nitems, s));
    mark(pl, 2, s);
    if (st == LADDER_OK) st = cuda_status(launch_unpack(L, L.one.ntiles * L.one.nchunks, s));
  }
  mark(pl, 3, s);
  return st;
}

// The error-free mode: operand preparation (B row scales and fixed-point
// slices, tau+- slices per GEMM2 chunk), the storing pass, the GEMM2 pass and
// the unpack of the two-pass form.
// Error-free preparation of one molecule: row scales and fixed-point slices
// of B (oz_prep_B, which pass 1 needs), and the tau+- slices of every GEMM2
// chunk (oz_prep_tau, which only pass 2 needs).
static void oz_prep_B(const ladder_plan_s *pl, const double *B, int *status, cudaStream_t s) {
  float *rsB = ws_at<float>(pl, pl->lay.ozRs);
  launch_oz_rowscale(pl->N, pl->v, pl->vp, B, rsB, status, s);
  launch_oz_split_B(pl->N, pl->v, pl->vp, pl->Np, pl->S, B, rsB, ws_at<__nv_bfloat16>(pl, pl->lay.Bt), s);
}
static void oz_prep_tau(const ladder_plan_s *pl, const double *tau, int *status, cudaStream_t s) {
  OzPackArgs pk;
  std::memset(&pk, 0, sizeof(pk));
  pk.tau = tau;
  pk.T2 = ws_at<uint8_t>(pl, pl->lay.T2);
  pk.sT = ws_at<float>(pl, pl->lay.ozST);
  pk.status = status;
  pk.o = pl->o;
  pk.v = pl->v;
  pk.nbp = pl->nbp;
  pk.S = pl->S;
  pk.nchunks = (int)pl->chunks_v.size();
  for (int c = 0; c < pk.nchunks; ++c) pk.chunks[c] = pl->chunks_v[c];
  launch_oz_pack_t2(pk, s);
}
static void oz_prep(const ladder_plan_s *pl, const double *B, const double *tau, int *status, cudaStream_t s) {
  oz_prep_B(pl, B, status, s);
  oz_prep_tau(pl, tau, status, s);
}

// Arguments of the error-free passes over all of a plan's tiles: pass 1
// (pass = 1: block-pair ranges vsplit, no accumulators) or pass 2 (ranges
// ksplit, accumulators in the slab).
static OzArgs oz_args(const ladder_plan_s *pl, int pass, int *status) {
  OzArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tmA = pl->tmA;
  a.tmB = pl->tmB;
  a.tmVl = pl->tmVl;
  a.Vst = ws_at<__nv_bfloat16>(pl, pl->lay.Vg);
  a.sV = ws_at<float>(pl, pl->lay.ozSV);
  a.rsB = ws_at<float>(pl, pl->lay.ozRs);
  a.T2 = ws_at<uint8_t>(pl, pl->lay.T2);
  a.sT = ws_at<float>(pl, pl->lay.ozST);
  if (pl->sym_b) {
    a.Xs = ws_at<float2>(pl, pl->lay.ozXs);
    a.xunits = ws_at<int4>(pl, pl->lay.ozXu);
  }
  a.status = status;
  a.o = pl->o;
  a.v = pl->v;
  a.vp = pl->vp;
  a.Np = pl->Np;
  a.nbp = pl->nbp;
  a.nks = pl->Np / 32;
  a.nB8 = pl->vp / CB;
  a.ntiles = pl->ntiles_tc;
  a.tile0 = pl->tile0;
  a.nchunks = (int)pl->chunks_v.size();
  for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->chunks_v[c];
  a.racc_cols = pl->racc_cols_v;
  // every single wait is far shorter than a pass; 2 s plus 20x a work unit's estimate
  const double unit_flops = 2.0 * 128.0 * 64.0 * 2.0 * pl->Np * 21.0 * ((double)pl->nbp / pl->vsplit);
  a.timeout_ns = (unsigned long long)(2e9 + 20.0 * unit_flops / 4e12 * 1e9);
  a.ksplit = pass == 1 ? pl->vsplit : pl->ksplit;
  a.nitems = pl->ntiles_tc * (pass == 1 ? 1 : a.nchunks) * a.ksplit;
  a.racc = pass == 1 ? nullptr : ws_at<float2>(pl, pl->lay.slab);
  return a;
}

static OzLaunch oz_launch(const OzArgs &a) {
  OzLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.one = a;
  L.nitems = a.nitems;
  L.status = a.status;
  L.timeout_ns = a.timeout_ns;
  return L;
}

// side: when given, tau's preparation was enqueued on another stream and
// side_done marks its end; pass 2 waits for it (pass 1 does not need tau).
// sym: the plan's symmetric-B form applies to this B (not to a dressed B).
static ladder_status apply_oz(ladder_plan_t pl, const double *B, const double *tau, double *R,
                              cudaStream_t s, cudaEvent_t side_done = nullptr, bool sym = true) {
  mark(pl, 0, s);
  int *status = ws_at<int>(pl, pl->lay.status);
  sym = sym && pl->sym_b;
  if (sym) launch_oz_symcheck(pl->N, pl->v, B, status, s);
  if (side_done)
    oz_prep_B(pl, B, status, s);
  else
    oz_prep(pl, B, tau, status, s);
  ladder_status st = cuda_status(cudaGetLastError());
  if (st != LADDER_OK) return st;
  OzArgs a1 = oz_args(pl, 1, status), a2 = oz_args(pl, 2, status);
  // tile ranges one after the other (one unless the stored tiles exceed the
  // cap): pass 1 (GEMM1 of every (tile, block pair), V+- slices and scales
  // stored; with symmetric B the distinct integral tiles once, before the
  // first range, then V+- of each range formed from them), pass 2 (GEMM2 per
  // (tile, chunk, block-pair range)), unpack
  const int nt = pl->ntiles_tc, rt = range_tiles(pl);
  const bool one = rt >= nt;
  pl->last_two_pass = one;
  pl->last_sym = sym && one;
  mark(pl, 1, s);
  if (sym) {
    OzArgs ax = a1;
    ax.nitems = (int)pl->xunits.size();
    st = cuda_status(launch_oz_xsym(oz_launch(ax), pl->S, s));
    if (one) mark(pl, 8, s);
  }
  for (int r0 = 0; r0 < nt && st == LADDER_OK; r0 += rt) {
    const int cnt = std::min(rt, nt - r0);
    a1.tile0 = a2.tile0 = pl->tile0 + r0;
    a1.ntiles = a2.ntiles = cnt;
    a1.nitems = cnt * pl->vsplit;
    a2.nitems = cnt * a2.nchunks * pl->ksplit;
    if (sym) {
      OzArgs af = a1;
      af.nitems = cnt * pl->nbp;
      st = cuda_status(launch_oz_vform(oz_launch(af), pl->S, pl->sm_count, s));
    } else {
      st = cuda_status(launch_oz_vstore(oz_launch(a1), pl->S, s));
    }
    if (one) mark(pl, 4, s);
    if (st == LADDER_OK && side_done && r0 == 0) st = cuda_status(cudaStreamWaitEvent(s, side_done, 0));
    if (st == LADDER_OK) st = cuda_status(launch_oz_gemm2(oz_launch(a2), pl->S, s));
    if (one) mark(pl, 2, s);
    if (st == LADDER_OK) {
      TcLaunch L;
      std::memset(&L, 0, sizeof(L));
      L.one = pass2_args(pl, R, status);
      L.one.tile0 = pl->tile0 + r0;
      L.one.ntiles = cnt;
      st = cuda_status(launch_unpack2(L, cnt * pl->nplus, s));
    }
  }
  if (!one) mark(pl, 2, s);
  mark(pl, 3, s);
  return st;
}

ladder_status ladder_apply(ladder_plan_t pl, const double *B, const double *tau, double *R,
                           void *stream) {
  if (!pl || pl->batched) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!dev_ptr_ok(B) || !dev_ptr_ok(tau) || !dev_ptr_ok(R) || R == B || R == tau)
    return LADDER_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pl->mode == LADDER_FP64) return apply_fp64(pl, B, tau, R, s);
  if (pl->mode == LADDER_OZAKI) return apply_oz(pl, B, tau, R, s);
  return apply_tc(pl, B, tau, R, s);
}

ladder_status ladder_apply_dressed(ladder_plan_t pl, const double *B, const double *Bov,
                                   const double *t1, const double *tau, double *R, void *stream) {
  if (!pl || pl->batched || !pl->dressed) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (pl->ntiles_tc != pl->ntiles_all) return LADDER_ENOTSUP;  // the correction spans all of R
  if (!dev_ptr_ok(B) || !dev_ptr_ok(Bov) || !dev_ptr_ok(t1) || !dev_ptr_ok(tau) || !dev_ptr_ok(R) ||
      R == B || R == tau || R == Bov || R == t1)
    return LADDER_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the error-free mode keeps FP64 for the dressing as the FP64 path does
  const bool f64 = pl->mode == LADDER_FP64 || pl->mode == LADDER_OZAKI;
  mark(pl, 5, s);
  double *Bd = ws_at<double>(pl, pl->lay.dBd);
  // Bd[P][b][d] = B[P][b][d] - sum_k t1[k][b] Bov[P][k][d]: one v x v product per P, K = o
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.A = t1;
  g.B = Bov;
  g.Out = Bd;
  g.Src = B;
  g.sam = 1;
  g.sak = pl->v;
  g.sbn = 1;
  g.sbk = pl->v;
  g.sb_batch = (long long)pl->o * pl->v;
  g.so_batch = (long long)pl->v * pl->v;
  g.M = g.N = pl->v;
  g.K = pl->o;
  g.ksplit = 1;
  g.kchunk = pl->o;
  g.ldo = pl->v;
  g.epi = kEpiFromSrc;
  ladder_status st = cuda_status(f64 ? launch_gemm<double, double, double>(g, pl->N, s)
                                     : launch_gemm<double, double, float>(g, pl->N, s));
  if (st != LADDER_OK) return st;
  mark(pl, 6, s);
  st = pl->mode == LADDER_FP64 ? apply_fp64(pl, Bd, tau, R, s)
       : pl->mode == LADDER_OZAKI ? apply_oz(pl, Bd, tau, R, s, nullptr, false)
                                  : apply_tc(pl, Bd, tau, R, s);
  if (st != LADDER_OK) return st;
  // the correction's GEMMs: FP64 for the plain method, double-single on the
  // FP32 pipe for the error-free mode, FP32 for the split-BF16 modes
  st = pl->mode == LADDER_FP64    ? dress_correct<double>(pl, Bov, t1, tau, R, s)
       : pl->mode == LADDER_OZAKI ? dress_correct<DS>(pl, Bov, t1, tau, R, s)
                                  : dress_correct<float>(pl, Bov, t1, tau, R, s);
  mark(pl, 7, s);
  return st;
}

ladder_status ladder_triples_workspace_size(int o, int v, int naux, int precision, size_t *bytes) {
  if (!bytes || o < 1 || o > 256 || v < 1 || v > kTriplesMaxV || naux < 1 || naux > 65536 ||
      (precision != LADDER_TRIPLES_FP64 && precision != LADDER_TRIPLES_FP32 && precision != LADDER_TRIPLES_BF16X6))
    return LADDER_EINVAL;
  if (precision == LADDER_TRIPLES_BF16X6 && v > 256) return LADDER_ENOTSUP;
  *bytes = triples_layout(o, v, precision != LADDER_TRIPLES_FP64, precision == LADDER_TRIPLES_BF16X6).total;
  return LADDER_OK;
}

ladder_status ladder_triples(int o, int v, int naux, int precision, const double *B, const double *Bov,
                             const double *Boo, const double *t1, const double *t2, const double *e_occ,
                             const double *e_vir, double *E_dev, void *workspace, size_t ws_bytes,
                             void *stream) {
  size_t need = 0;
  const ladder_status st = ladder_triples_workspace_size(o, v, naux, precision, &need);
  if (st != LADDER_OK) return st;
  if (!workspace || ws_bytes < need) return LADDER_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return LADDER_EINVAL;
  const void *ptrs[] = {B, Bov, Boo, t1, t2, e_occ, e_vir, E_dev, workspace};
  for (const void *q : ptrs)
    if (!dev_ptr_ok(q)) return LADDER_EINVAL;
  const bool tc = precision == LADDER_TRIPLES_BF16X6;
  const TriplesLayout L = triples_layout(o, v, precision != LADDER_TRIPLES_FP64, tc);
  char *ws = static_cast<char *>(workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return cuda_status(precision == LADDER_TRIPLES_FP64
                         ? triples_run<double>(o, v, naux, B, Bov, Boo, t1, t2, e_occ, e_vir, E_dev, ws, L, s)
                         : triples_run<float>(o, v, naux, B, Bov, Boo, t1, t2, e_occ, e_vir, E_dev, ws, L, s,
                                              tc));
}

ladder_status ladder_energy(ladder_plan_t pl, const double *R, const double *t2, double *E_dev,
                            void *stream) {
  if (!pl || pl->batched) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!dev_ptr_ok(R) || !dev_ptr_ok(t2) || !dev_ptr_ok(E_dev, 8)) return LADDER_EINVAL;
  launch_energy(pl->o, pl->v, R, t2, ws_at<double>(pl, pl->lay.energy), E_dev,
                static_cast<cudaStream_t>(stream));
  return cuda_status(cudaGetLastError());
}

ladder_status ladder_backward(ladder_plan_t pl, const double *B, const double *tau,
                              const double *W, double *dtau, double *dB, void *stream) {
  if (!pl || pl->batched) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!dev_ptr_ok(B) || !dev_ptr_ok(tau) || !dev_ptr_ok(W)) return LADDER_EINVAL;
  if (dtau && (!dev_ptr_ok(dtau) || dtau == W || dtau == tau || dtau == B)) return LADDER_EINVAL;
  if (dB && (!dev_ptr_ok(dB) || dB == B)) return LADDER_EINVAL;
  if (pl->mode == LADDER_OZAKI) {
    // with B symmetric the transposed ladder is the ladder itself, so dtau
    // comes from the error-free forward passes; this mode has no dB
    if (dB || !pl->sym_b || pl->ntiles_tc != pl->ntiles_all) return LADDER_ENOTSUP;
    return dtau ? apply_oz(pl, B, W, dtau, static_cast<cudaStream_t>(stream)) : LADDER_OK;
  }
  if (dB && !pl->backward) return LADDER_EWORKSPACE;
  if (pl->ntiles_tc != pl->ntiles_all) return LADDER_ENOTSUP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtau) {
    // transposed ladder: dtau = sum_ab W_ij^ab (ac|bd), i.e. the ladder of W
    // with every factor B^P replaced by its transpose
    const ladder_status st = pl->mode == LADDER_FP64 ? apply_fp64(pl, B, W, dtau, s, true)
                                                     : apply_tc(pl, B, W, dtau, s, true);
    if (st != LADDER_OK) return st;
  }
  if (dB && pl->mode == LADDER_FP64) {
    GradArgs g{};
    g.B = B;
    g.tau = tau;
    g.W = W;
    g.dB = dB;
    g.slab = pl->N > kGradPChunk ? ws_at<double>(pl, pl->lay.gslab) : nullptr;
    g.o = pl->o;
    g.v = pl->v;
    g.N = pl->N;
    g.vp = pl->vp;
    const ladder_status st = cuda_status(launch_grad_B_fp64(g, pl->grid_grad, s));
    if (st != LADDER_OK) return st;
  } else if (dB && pl->g2) {
    // two-pass dB: Gamma tiles stored once, then their contraction with the
    // B slices in the GEMM2 kernel (square tiles, one sign), then dB = 2 x sums
    auto *Wt = ws_at<__nv_bfloat16>(pl, pl->lay.gWt);
    auto *Tt = ws_at<__nv_bfloat16>(pl, pl->lay.gTt);
    launch_split_pairs(pl->o, pl->v, pl->vp, pl->g_IJp, pl->S, W, Wt, s);
    launch_split_pairs(pl->o, pl->v, pl->vp, pl->g_IJp, pl->S, tau, Tt, s);
    BpackArgs bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.B = B;
    bp.T2 = ws_at<__nv_bfloat16>(pl, pl->lay.gT2);
    bp.N = pl->N;
    bp.v = pl->v;
    bp.nb = pl->vp / CB;
    bp.S = pl->S;
    bp.nchunks = (int)pl->g2_chunks.size();
    for (int c = 0; c < bp.nchunks; ++c) bp.chunks[c] = pl->g2_chunks[c];
    launch_pack_b2(bp, s);
    ladder_status st = cuda_status(cudaGetLastError());
    if (st != LADDER_OK) return st;
    int *status = ws_at<int>(pl, pl->lay.status);
    GradTcArgs g;
    std::memset(&g, 0, sizeof(g));
    g.tmW = pl->tmGW;
    g.tmT = pl->tmGT;
    g.Gst = ws_at<__nv_bfloat16>(pl, pl->lay.gG);
    g.qsplit = pl->g2_qsplit;
    g.status = status;
    g.o = pl->o;
    g.v = pl->v;
    g.N = pl->N;
    g.vp = pl->vp;
    g.IJp = pl->g_IJp;
    g.nks = pl->g_IJp / 32;
    g.nY8 = pl->vp / CB;
    g.ntiles = pl->g_ntiles;
    g.kc = pl->kc;
    const int nq = (pl->vp / CB) * (pl->vp / CB);
    const double unit_flops = 2.0 * 128.0 * 64.0 * pl->g_IJp * 6.0 * ((double)nq / pl->g2_qsplit);
    g.timeout_ns = (unsigned long long)(2e9 + 20.0 * unit_flops / 4e12 * 1e9);
    st = cuda_status(launch_grad_gamma_store(g, pl->S, s));
    if (st != LADDER_OK) return st;
    TcLaunch L;
    std::memset(&L, 0, sizeof(L));
    TcArgs &a = L.one;
    a.tmVl = pl->tmGl;
    a.T2 = ws_at<uint8_t>(pl, pl->lay.gT2);
    a.status = status;
    a.o = pl->o;
    a.v = pl->v;
    a.vp = pl->vp;
    a.nbp = nq;
    a.nA = pl->vp / 16;
    a.nB8 = pl->vp / CB;
    a.ntiles = pl->g_ntiles;
    a.nchunks = (int)pl->g2_chunks.size();
    for (int c = 0; c < a.nchunks; ++c) a.chunks[c] = pl->g2_chunks[c];
    a.ksplit = pl->g2_ksplit;
    a.racc = ws_at<float2>(pl, pl->lay.gacc2);
    a.racc_cols = pl->g2_cols;
    a.s_pieces = pl->s_pieces;
    a.flush_every = pl->flush_every;
    a.square = 1;
    a.nsign = 1;
    const double item_flops = 2.0 * 128.0 * pl->g2_cols * 64.0 * 6.0 * ((double)nq / pl->g2_ksplit);
    a.timeout_ns = (unsigned long long)(2e9 + 20.0 * item_flops / 4e12 * 1e9);
    L.timeout_ns = a.timeout_ns;
    L.nitems = a.ntiles * a.nchunks * a.ksplit;
    st = cuda_status(launch_ladder_gemm2(L, pl->S, L.nitems, s));
    if (st != LADDER_OK) return st;
    return cuda_status(launch_grad_unpack2(L, dB, pl->N, a.ntiles * a.nchunks, s));
  } else if (dB) {
    auto *Wt = ws_at<__nv_bfloat16>(pl, pl->lay.gWt);
    auto *Tt = ws_at<__nv_bfloat16>(pl, pl->lay.gTt);
    auto *Bs = ws_at<__nv_bfloat16>(pl, pl->lay.gBs);
    launch_split_pairs(pl->o, pl->v, pl->vp, pl->g_IJp, pl->S, W, Wt, s);
    launch_split_pairs(pl->o, pl->v, pl->vp, pl->g_IJp, pl->S, tau, Tt, s);
    launch_split_B_rows(pl->N, pl->v, pl->vp, pl->g_Np, pl->S, B, Bs, s);
    ladder_status st = cuda_status(cudaGetLastError());
    if (st != LADDER_OK) return st;
    GradTcArgs g;
    std::memset(&g, 0, sizeof(g));
    g.tmW = pl->tmGW;
    g.tmT = pl->tmGT;
    g.tmBs = pl->tmGBs;
    g.dB = dB;
    g.racc = ws_at<float2>(pl, pl->lay.gacc);
    g.status = ws_at<int>(pl, pl->lay.status);
    g.o = pl->o;
    g.v = pl->v;
    g.N = pl->N;
    g.vp = pl->vp;
    g.Np = pl->g_Np;
    g.IJp = pl->g_IJp;
    g.nks = pl->g_IJp / 32;
    g.nY8 = pl->vp / CB;
    g.ntiles = pl->g_ntiles;
    g.npc = pl->g_npc;
    g.kc = pl->kc;
    g.s_pieces = pl->s_pieces;
    g.flush_every = pl->flush_every;
    const double item_flops = 2.0 * (pl->vp / CB) * (pl->vp / CB) * 128.0 * 64.0 *
                              (pl->g_IJp + 2.0 * kGradTcPChunk) * 6.0;
    g.timeout_ns = (unsigned long long)(2e9 + 20.0 * item_flops / 4e12 * 1e9);
    st = cuda_status(launch_grad_B_tc(g, pl->S, s));
    if (st != LADDER_OK) return st;
  }
  return LADDER_OK;
}

ladder_status ladder_pair_combine(int o, int v, double alpha, double beta, const double *X,
                                  double *Y, void *stream) {
  if (o < 1 || o > 256 || v < 1 || v > 4096) return LADDER_EINVAL;
  if (!dev_ptr_ok(X) || !dev_ptr_ok(Y) || X == Y) return LADDER_EINVAL;
  launch_pair_combine(o, v, alpha, beta, X, Y, static_cast<cudaStream_t>(stream));
  return cuda_status(cudaGetLastError());
}

ladder_status ladder_apply_host(ladder_plan_t pl, const double *B_host, const double *tau_host,
                                double *R_host, double *d_B, double *d_tau, double *d_R,
                                void *stream) {
  if (!pl || pl->batched || !B_host || !tau_host || !R_host) return LADDER_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nB = (size_t)pl->N * pl->v * pl->v * sizeof(double);
  const size_t nT = (size_t)pl->o * pl->o * pl->v * pl->v * sizeof(double);
  if (!dev_ptr_ok(d_B) || !dev_ptr_ok(d_tau) || !dev_ptr_ok(d_R) || d_R == d_B || d_R == d_tau)
    return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  ladder_status st = LADDER_OK;
  if (pl->mode == LADDER_OZAKI) {
    // tau's upload and preparation run on a side stream, overlapping B's
    // upload, B's preparation and pass 1; pass 2 waits for them
    if (!pl->side_stream &&
        (cudaStreamCreateWithFlags(&pl->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&pl->side_ev[0], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&pl->side_ev[1], cudaEventDisableTiming) != cudaSuccess))
      return cuda_status(cudaErrorUnknown);
    cudaStream_t t = pl->side_stream;
    if (cudaEventRecord(pl->side_ev[0], s) != cudaSuccess || cudaStreamWaitEvent(t, pl->side_ev[0], 0) != cudaSuccess ||
        cudaMemcpyAsync(d_tau, tau_host, nT, cudaMemcpyHostToDevice, t) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    oz_prep_tau(pl, d_tau, ws_at<int>(pl, pl->lay.status), t);
    if (cudaEventRecord(pl->side_ev[1], t) != cudaSuccess ||
        cudaMemcpyAsync(d_B, B_host, nB, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    st = apply_oz(pl, d_B, d_tau, d_R, s, pl->side_ev[1]);
    // the side stream's work is joined before R leaves the device
    if (st == LADDER_OK) st = cuda_status(cudaStreamWaitEvent(s, pl->side_ev[1], 0));
  } else {
    if (cudaMemcpyAsync(d_B, B_host, nB, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_tau, tau_host, nT, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    st = ladder_apply(pl, d_B, d_tau, d_R, stream);
  }
  if (st != LADDER_OK) return st;
  if (cudaMemcpyAsync(R_host, d_R, nT, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  return cuda_status(cudaStreamSynchronize(s));
}

// Stored V+- tiles of a batch: at most this many bytes in all (members beyond
// it use the fused form).
constexpr double kVStoreBatchCap = 128.0 * (1ull << 30);

// (Re)builds a batch plan's work lists and workspace layout from its
// members' current forms: fused members' work units cost-sorted, largest
// first; two-pass members largest first, each in its own range-major order.
static void batch_finalize(ladder_plan_s *pl) {
  struct Unit {
    double cost;
    int m, k;
  };
  std::vector<Unit> units;
  std::vector<std::pair<double, int>> twopass;  // (flops, molecule)
  pl->items.clear();
  pl->tcs.clear();
  pl->items1.clear();
  pl->items2.clear();
  pl->tcs2.clear();
  pl->sub_off.clear();
  const int n = (int)pl->subs.size();
  for (int m = 0; m < n; ++m) {
    ladder_plan_s *sp = pl->subs[m];
    if (sp->two_pass) {
      twopass.push_back({ladder_flops(sp), m});
      continue;
    }
    const int nwork = sp->ntiles_tc * (int)sp->chunks_tc.size();
    // cost of one work unit: block pairs x (GEMM1 K-steps + GEMM2 pieces)
    const double cost = (double)sp->nbp * (2.0 * (sp->Np / 32) + 4.0);
    for (int k = 0; k < nwork; ++k) {
      units.push_back({cost, m, k});
      pl->tcs.push_back(make_int2(m, k));
    }
  }
  // fused work units: largest first, ties keep molecule order
  std::stable_sort(units.begin(), units.end(),
                   [](const Unit &x, const Unit &y) { return x.cost > y.cost; });
  for (auto &u : units) pl->items.push_back(make_int2(u.m, u.k));
  std::stable_sort(twopass.begin(), twopass.end(),
                   [](const std::pair<double, int> &x, const std::pair<double, int> &y) {
                     return x.first > y.first;
                   });
  pl->itemsX.clear();
  pl->itemsF.clear();
  for (auto &t : twopass) {
    const ladder_plan_s *sp = pl->subs[t.second];
    const int m = t.second;
    if (sp->sym_b) {
      // symmetric-B error-free member: its distinct tiles and V+- formation
      // take the place of the storing pass
      for (int k = 0; k < (int)sp->xunits.size(); ++k) pl->itemsX.push_back(make_int2(m, k));
      for (int k = 0; k < sp->ntiles_tc * sp->nbp; ++k) pl->itemsF.push_back(make_int2(m, k));
    } else {
      for (int k = 0; k < sp->ntiles_tc * sp->vsplit; ++k) pl->items1.push_back(make_int2(m, k));
    }
    for (int k = 0; k < sp->ntiles_tc * (int)sp->chunks_v.size() * sp->ksplit; ++k)
      pl->items2.push_back(make_int2(m, k));
    for (int k = 0; k < sp->ntiles_tc * sp->nplus; ++k) pl->tcs2.push_back(make_int2(m, k));
  }
  size_t off = kAlign;  // status word
  pl->lay.status = 0;
  auto region = [&](size_t &at, size_t bytes) {
    at = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
  };
  region(pl->off_mols, (size_t)n * sizeof(TcArgs));
  region(pl->off_mols1, (size_t)n * sizeof(TcArgs));
  region(pl->off_mols2, (size_t)n * sizeof(TcArgs));
  const size_t noz = pl->mode == LADDER_OZAKI ? (size_t)n : 0;
  region(pl->off_oz1, noz * sizeof(OzArgs));
  region(pl->off_oz2, noz * sizeof(OzArgs));
  region(pl->off_items, pl->items.size() * sizeof(int2));
  region(pl->off_tcs, pl->tcs.size() * sizeof(int2));
  region(pl->off_items1, pl->items1.size() * sizeof(int2));
  region(pl->off_items2, pl->items2.size() * sizeof(int2));
  region(pl->off_tcs2, pl->tcs2.size() * sizeof(int2));
  region(pl->off_itemsX, pl->itemsX.size() * sizeof(int2));
  region(pl->off_itemsF, pl->itemsF.size() * sizeof(int2));
  for (auto *sp : pl->subs) {
    off = align_up(off, 1024);
    pl->sub_off.push_back(off);
    off += sp->lay.total;
  }
  pl->lay.total = align_up(off);
}

// Stored V+- bytes of a member in the two-pass form.
static double member_vbytes(const ladder_plan_s *sp) {
  return (double)sp->ntiles_tc * sp->nbp * 2 * sp->S * 128 * SLOTS * 2;
}

// A member's form: the two-pass form keeps block-pair ranges of about 160
// for its GEMM2 units; a fused member runs whole tiles.
static void set_member_form(ladder_plan_s *sp, bool two_pass) {
  sp->two_pass = two_pass ? 1 : 0;
  sp->tile_chunk = sp->ntiles_tc;  // the batch cap keeps every member's tiles in one range
  sp->ksplit = two_pass ? std::max(1, std::min(sp->nbp, sp->nbp / 160)) : 1;
  compute_layout(sp);
}

ladder_status ladder_plan_batched(int n, const int *o, const int *v, const int *naux, int mode,
                                  ladder_plan_t *out) {
  if (!out || n < 1 || n > 4096 || !o || !v || !naux) return LADDER_EINVAL;
  *out = nullptr;
  if (mode & LADDER_WITH_BACKWARD) return LADDER_ENOTSUP;
  if (mode == LADDER_AUTO) mode = LADDER_BF16X6;
  if (mode != LADDER_BF16X3 && mode != LADDER_BF16X6 && mode != LADDER_OZAKI) return LADDER_ENOTSUP;
  const bool oz = mode == LADDER_OZAKI;
  ladder_plan_s *pl = new (std::nothrow) ladder_plan_s();
  if (!pl) return LADDER_ENOMEM;
  pl->batched = true;
  pl->mode = mode;
  pl->S = oz ? kOzDefaultSlices : tc_slices(mode);
  double vsum = 0.0;
  for (int m = 0; m < n; ++m) {
    ladder_plan_s *sp = new (std::nothrow) ladder_plan_s();
    if (!sp) {
      ladder_destroy(pl);
      return LADDER_ENOMEM;
    }
    pl->subs.push_back(sp);
    const ladder_status st = init_plan(sp, o[m], v[m], naux[m], mode, false, true);
    if (st != LADDER_OK) {
      ladder_destroy(pl);
      return st;
    }
    pl->device = sp->device;
    pl->sm_count = sp->sm_count;
    if (oz) {
      // the error-free mode has only the two-pass form: every member's
      // stored slices must fit the cap together
      vsum += member_vbytes(sp);
      if (vsum > kVStoreOzCap) {
        ladder_destroy(pl);
        return LADDER_ENOTSUP;
      }
      set_member_form(sp, true);
      continue;
    }
    // members whose fused form would recompute GEMM1 per chunk take the
    // two-pass form while the batch's stored tiles fit the cap
    const double vb = member_vbytes(sp);
    const bool tp = sp->chunks_tc.size() > 1 && vsum + vb <= kVStoreBatchCap;
    if (tp) {
      vsum += vb;
      set_member_form(sp, true);
    }
  }
  batch_finalize(pl);
  *out = pl;
  return LADDER_OK;
}

ladder_status ladder_set_member_tuning(ladder_plan_t pl, int m, const ladder_tuning *t) {
  if (!pl || !t || !pl->batched || pl->ws || m < 0 || m >= (int)pl->subs.size()) return LADDER_EINVAL;
  if (pl->mode == LADDER_OZAKI) {
    // an error-free member takes only sym_b; its slices, form and splits
    // are the batch's
    if (t->sym_b != 0 && t->sym_b != 1) return LADDER_EINVAL;
    ladder_plan_s *sp = pl->subs[m];
    if (t->sym_b && (double)xsym_bytes(sp) > kXsymCap) return LADDER_ENOTSUP;
    double tot = 0.0;
    for (auto *q : pl->subs)
      tot += member_vbytes(q) + ((q == sp ? t->sym_b : q->sym_b) ? (double)xsym_bytes(q) : 0.0);
    if (tot > kVStoreOzCap) return LADDER_ENOTSUP;
    sp->sym_b = t->sym_b;
    sp->xunits = sp->sym_b ? make_xunits(sp->nb) : std::vector<int4>();
    compute_layout(sp);
    batch_finalize(pl);
    return LADDER_OK;
  }
  if (t->sym_b != 0) return LADDER_EINVAL;
  if (t->kc < 1 || t->kc > 64 || !(t->s_pieces == 1 || t->s_pieces == 2 || t->s_pieces == 4) ||
      t->flush_every < 1 || t->flush_every > 4096 || (t->xy_split != 0 && t->xy_split != 1) ||
      (t->two_pass != 0 && t->two_pass != 1) || t->lambda_only != 0)
    return LADDER_EINVAL;
  ladder_plan_s *sp = pl->subs[m];
  if (t->two_pass && !sp->two_pass) {
    double vsum = member_vbytes(sp);
    for (auto *q : pl->subs)
      if (q->two_pass) vsum += member_vbytes(q);
    if (vsum > kVStoreBatchCap) return LADDER_ENOTSUP;
  }
  sp->kc = t->kc;
  sp->s_pieces = t->s_pieces;
  sp->flush_every = t->flush_every;
  sp->xy_split = t->xy_split;
  set_member_form(sp, t->two_pass != 0);
  batch_finalize(pl);
  return LADDER_OK;
}

// Records (or replays) one batch step as a CUDA graph.  With t1, t2 and E
// given, every molecule's step starts with tau = t2 + t1 (x) t1 into tau[m]
// and ends with its ladder energy into E[m]; without them tau[m] is an input.
static ladder_status batch_run(ladder_plan_t pl, const double *const *B, const double *const *t1,
                               const double *const *t2, double *const *tau, double *const *R, double *E,
                               void *stream) {
  if (!pl || !pl->batched) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (!B || !tau || !R) return LADDER_EINVAL;
  const bool step = t1 != nullptr;
  if (step && (!t2 || !dev_ptr_ok(E, 8))) return LADDER_EINVAL;
  const size_t n = pl->subs.size();
  std::vector<const void *> key;
  for (size_t m = 0; m < n; ++m) {
    if (!dev_ptr_ok(B[m]) || !dev_ptr_ok(tau[m]) || !dev_ptr_ok(R[m]) || R[m] == B[m] ||
        R[m] == tau[m])
      return LADDER_EINVAL;
    if (step && (!dev_ptr_ok(t1[m]) || !dev_ptr_ok(t2[m]) || tau[m] == t2[m] || R[m] == t2[m]))
      return LADDER_EINVAL;
    key.push_back(B[m]);
    key.push_back(tau[m]);
    key.push_back(R[m]);
    if (step) {
      key.push_back(t1[m]);
      key.push_back(t2[m]);
    }
  }
  key.push_back(step ? E : nullptr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!pl->gexec || key != pl->gkey) {
    // (re)build: per-molecule arguments into the workspace table, then capture
    // the whole batch (tau assembly and operand preparation of every
    // molecule, the fused, storing and GEMM2 launches over all molecules, the
    // unpacks, and every molecule's energy)
    char *w = static_cast<char *>(pl->ws);
    int *status = ws_at<int>(pl, pl->lay.status);
    const bool oz = pl->mode == LADDER_OZAKI;
    std::vector<TcArgs> args(n), args1(n), args2(n);
    std::vector<OzArgs> oz1(oz ? n : 0), oz2(oz ? n : 0);
    unsigned long long tmax = 0;
    for (size_t m = 0; m < n; ++m) {
      const ladder_plan_s *sp = pl->subs[m];
      if (oz) {
        // error-free members: the passes read OzArgs; the unpack reads the
        // two-pass TcArgs of the same accumulators
        oz1[m] = oz_args(sp, 1, status);
        oz2[m] = oz_args(sp, 2, status);
        args[m] = args1[m] = args2[m] = pass2_args(sp, R[m], status);
        tmax = std::max(tmax, oz1[m].timeout_ns);
        continue;
      }
      args[m] = tc_args(sp, R[m], status);
      if (sp->two_pass) {
        args1[m] = pass1_args(sp, status);
        args2[m] = pass2_args(sp, R[m], status);
      } else {
        args1[m] = args2[m] = args[m];
      }
      tmax = std::max(tmax, args[m].timeout_ns);
    }
    if (oz && (cudaStreamSynchronize(s) != cudaSuccess ||
               cudaMemcpy(w + pl->off_oz1, oz1.data(), n * sizeof(OzArgs), cudaMemcpyHostToDevice) !=
                   cudaSuccess ||
               cudaMemcpy(w + pl->off_oz2, oz2.data(), n * sizeof(OzArgs), cudaMemcpyHostToDevice) !=
                   cudaSuccess))
      return cuda_status(cudaErrorUnknown);
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(w + pl->off_mols, args.data(), n * sizeof(TcArgs), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(w + pl->off_mols1, args1.data(), n * sizeof(TcArgs), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(w + pl->off_mols2, args2.data(), n * sizeof(TcArgs), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    if (!pl->cap_stream &&
        cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    if (pl->gexec) {
      cudaGraphExecDestroy(pl->gexec);
      pl->gexec = nullptr;
    }
    auto batch_launch = [&](size_t mols, size_t items, size_t tcs, int nitems) {
      TcLaunch L;
      std::memset(&L, 0, sizeof(L));
      L.mols = reinterpret_cast<const TcArgs *>(w + mols);
      L.items = reinterpret_cast<const int2 *>(w + items);
      L.tcs = reinterpret_cast<const int2 *>(w + tcs);
      L.nitems = nitems;
      L.timeout_ns = tmax;
      return L;
    };
    const TcLaunch L = batch_launch(pl->off_mols, pl->off_items, pl->off_tcs, (int)pl->items.size());
    const TcLaunch L1 = batch_launch(pl->off_mols1, pl->off_items1, pl->off_tcs2, (int)pl->items1.size());
    const TcLaunch L2 = batch_launch(pl->off_mols2, pl->off_items2, pl->off_tcs2, (int)pl->items2.size());
    cudaStream_t c = pl->cap_stream;
    if (cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
    for (size_t m = 0; m < n; ++m) {
      const ladder_plan_s *sp = pl->subs[m];
      if (step) launch_tau(sp->o, sp->v, t1[m], t2[m], tau[m], c);
      if (oz) {
        if (sp->sym_b) launch_oz_symcheck(sp->N, sp->v, B[m], status, c);
        oz_prep(sp, B[m], tau[m], status, c);
        continue;
      }
      tc_prep(pl->subs[m], B[m], tau[m], c, false, status);
      if (sp->two_pass) pack_t2(sp, c);
    }
    if (oz) {
      // both error-free passes over every member's work units, one CTA each
      auto oz_batch = [&](size_t mols, size_t items, int nitems) {
        OzLaunch Lz;
        std::memset(&Lz, 0, sizeof(Lz));
        Lz.mols = reinterpret_cast<const OzArgs *>(w + mols);
        Lz.items = reinterpret_cast<const int2 *>(w + items);
        Lz.nitems = nitems;
        Lz.status = status;
        Lz.timeout_ns = tmax;
        return Lz;
      };
      launch_oz_xsym(oz_batch(pl->off_oz1, pl->off_itemsX, (int)pl->itemsX.size()), pl->S, c);
      launch_oz_vform(oz_batch(pl->off_oz1, pl->off_itemsF, (int)pl->itemsF.size()), pl->S, pl->sm_count, c);
      launch_oz_vstore(oz_batch(pl->off_oz1, pl->off_items1, (int)pl->items1.size()), pl->S, c);
      launch_oz_gemm2(oz_batch(pl->off_oz2, pl->off_items2, (int)pl->items2.size()), pl->S, c);
    }
    if (L.nitems) launch_ladder_tc(L, pl->S, std::min(L.nitems, pl->sm_count), c);
    if (!oz && L1.nitems) launch_ladder_vstore(L1, pl->S, std::min(L1.nitems, pl->sm_count), c);
    if (!oz && L2.nitems) launch_ladder_gemm2(L2, pl->S, std::min(L2.nitems, pl->sm_count), c);
    if (!pl->tcs.empty()) launch_unpack(L, (int)pl->tcs.size(), c);
    if (!pl->tcs2.empty()) launch_unpack2(L2, (int)pl->tcs2.size(), c);
    if (step)
      for (size_t m = 0; m < n; ++m) {
        const ladder_plan_s *sp = pl->subs[m];
        launch_energy(sp->o, sp->v, R[m], t2[m], ws_at<double>(sp, sp->lay.energy), E + m, c);
      }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c, &graph);
    if (ce != cudaSuccess || !graph) return cuda_status(ce == cudaSuccess ? cudaErrorUnknown : ce);
    const cudaError_t ie = cudaGraphInstantiate(&pl->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      pl->gexec = nullptr;
      return cuda_status(ie);
    }
    pl->gkey = key;
  }
  pl->last_two_pass = false;
  mark(pl, 0, s);
  mark(pl, 1, s);
  const ladder_status st = cuda_status(cudaGraphLaunch(pl->gexec, s));
  mark(pl, 2, s);
  mark(pl, 3, s);
  return st;
}

ladder_status ladder_apply_batched(ladder_plan_t pl, const double *const *B,
                                   const double *const *tau, double *const *R, void *stream) {
  return batch_run(pl, B, nullptr, nullptr, const_cast<double *const *>(tau), R, nullptr, stream);
}

ladder_status ladder_step_batched(ladder_plan_t pl, const double *const *B, const double *const *t1,
                                  const double *const *t2, double *const *tau, double *const *R, double *E,
                                  void *stream) {
  if (!t1 || !t2) return LADDER_EINVAL;
  return batch_run(pl, B, t1, t2, tau, R, E, stream);
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
  if (h == kSiteNonFinite) return LADDER_ENONFINITE;
  if (h == kSiteAsymmetric) return LADDER_EINVAL;
  return h == 0 ? LADDER_OK : LADDER_ETIMEOUT;
}

ladder_status ladder_selftest_wait(ladder_plan_t pl, unsigned long long timeout_ns, void *stream) {
  if (!pl) return LADDER_EINVAL;
  if (!pl->ws) return LADDER_EWORKSPACE;
  if (timeout_ns < 1000000ull || timeout_ns > 10000000000ull) return LADDER_EINVAL;
  return cuda_status(launch_selftest_wait(ws_at<int>(pl, pl->lay.status), timeout_ns, 99,
                                          static_cast<cudaStream_t>(stream)));
}

ladder_status ladder_set_timing(ladder_plan_t pl, int on) {
  if (!pl) return LADDER_EINVAL;
  if (on && !pl->ev[0]) {
    for (auto &e : pl->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  }
  pl->timing = on != 0;
  return LADDER_OK;
}

ladder_status ladder_timing(ladder_plan_t pl, float *prep_ms, float *fused_ms, float *unpack_ms) {
  if (!pl) return LADDER_EINVAL;
  if (!pl->timing || !pl->ev[0]) return LADDER_EINVAL;
  if (cudaEventSynchronize(pl->ev[3]) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  float t[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k)
    if (cudaEventElapsedTime(&t[k], pl->ev[k], pl->ev[k + 1]) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
  if (prep_ms) *prep_ms = t[0];
  if (fused_ms) *fused_ms = t[1];
  if (unpack_ms) *unpack_ms = t[2];
  return LADDER_OK;
}

ladder_status ladder_timing_passes(ladder_plan_t pl, float *pass1_ms, float *pass2_ms) {
  if (!pl || !pl->timing || !pl->ev[0]) return LADDER_EINVAL;
  if (cudaEventSynchronize(pl->ev[3]) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  float t1 = 0.f, t2 = 0.f;
  if (pl->last_two_pass) {
    if (cudaEventElapsedTime(&t1, pl->ev[1], pl->ev[4]) != cudaSuccess ||
        cudaEventElapsedTime(&t2, pl->ev[4], pl->ev[2]) != cudaSuccess)
      return cuda_status(cudaErrorUnknown);
  } else if (cudaEventElapsedTime(&t1, pl->ev[1], pl->ev[2]) != cudaSuccess) {
    return cuda_status(cudaErrorUnknown);
  }
  if (pass1_ms) *pass1_ms = t1;
  if (pass2_ms) *pass2_ms = t2;
  return LADDER_OK;
}

ladder_status ladder_timing_sym(ladder_plan_t pl, float *xsym_ms, float *form_ms) {
  if (!pl || !pl->timing || !pl->ev[0] || !pl->last_sym) return LADDER_EINVAL;
  if (cudaEventSynchronize(pl->ev[3]) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  float t1 = 0.f, t2 = 0.f;
  if (cudaEventElapsedTime(&t1, pl->ev[1], pl->ev[8]) != cudaSuccess ||
      cudaEventElapsedTime(&t2, pl->ev[8], pl->ev[4]) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  if (xsym_ms) *xsym_ms = t1;
  if (form_ms) *form_ms = t2;
  return LADDER_OK;
}

ladder_status ladder_timing_dressing(ladder_plan_t pl, float *bd_ms, float *correction_ms) {
  if (!pl || !pl->timing || !pl->ev[0] || !pl->dressed) return LADDER_EINVAL;
  if (cudaEventSynchronize(pl->ev[7]) != cudaSuccess) return cuda_status(cudaErrorUnknown);
  float t1 = 0.f, t2 = 0.f;
  if (cudaEventElapsedTime(&t1, pl->ev[5], pl->ev[6]) != cudaSuccess ||
      cudaEventElapsedTime(&t2, pl->ev[3], pl->ev[7]) != cudaSuccess)
    return cuda_status(cudaErrorUnknown);
  if (bd_ms) *bd_ms = t1;
  if (correction_ms) *correction_ms = t2;
  return LADDER_OK;
}

double ladder_flops(ladder_plan_t pl) {
  if (!pl) return 0.0;
  if (pl->batched) {
    double f = 0.0;
    for (auto *sp : pl->subs) f += ladder_flops(sp);
    return f;
  }
  const double g1 = 2.0 * ppos(pl->v) * (double)pl->v * pl->v * pl->N;
  const double g2 = 2.0 * ((double)ppos(pl->o) * ppos(pl->v) * (double)ppos(pl->v) +
                           (double)pneg(pl->o) * pneg(pl->v) * (double)pneg(pl->v));
  return g1 + g2;
}

void ladder_destroy(ladder_plan_t pl) {
  if (!pl) return;
  for (auto &e : pl->ev)
    if (e) cudaEventDestroy(e);
  for (auto *sp : pl->subs) ladder_destroy(sp);
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (pl->side_stream) cudaStreamDestroy(pl->side_stream);
  for (auto &e : pl->side_ev)
    if (e) cudaEventDestroy(e);
  delete pl;
}

}  // extern "C"
