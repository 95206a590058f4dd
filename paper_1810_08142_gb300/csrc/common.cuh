// Shared device/host definitions of the ladder library (not used by the oracle).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace ladder {

// Virtual indices are processed in blocks of CB = 8 (the c/d blocks of the
// symmetric/antisymmetric scheme); v is padded with zeros to VPAD = 16.
constexpr int CB = 8;
constexpr int SLOTS = CB * CB;  // (c,d) slots per block pair
constexpr int VPAD = 16;

// Device status word codes (site of the first bounded wait that ran out).
enum : int {
  kStatusOk = 0,
  kSiteTmaFull = 1,
  kSiteTmaEmpty = 2,
  kSiteXYFull = 3,
  kSiteXYFree = 4,
  kSiteVFull = 5,
  kSiteVFree = 6,
  kSiteRFull = 7,
  kSiteRFree = 8,
  kSiteNonFinite = 50,  // an input element was NaN or infinite (not a wait)
  kSiteAsymmetric = 51, // B declared symmetric is not (not a wait)
};

__host__ __device__ inline int ppos(int n) { return n * (n + 1) / 2; }
__host__ __device__ inline int pneg(int n) { return n * (n - 1) / 2; }

// Block pair p <-> (k, l), k <= l, ordered p = l(l+1)/2 + k.
__host__ __device__ inline void pair_of(int p, int &k, int &l) {
  int t = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while (ppos(t + 1) <= p) ++t;
  while (ppos(t) > p) --t;
  l = t;
  k = p - ppos(t);
}

// Symmetric pair lambda+ = j(j+1)/2 + i (i <= j).
__host__ __device__ inline void lam_plus(int lam, int &i, int &j) { pair_of(lam, i, j); }

// Antisymmetric pair lambda- = j(j-1)/2 + i (i < j).
__host__ __device__ inline void lam_minus(int lam, int &i, int &j) {
  int k, l;
  pair_of(lam, k, l);  // lam = l(l+1)/2 + k with k <= l  ->  j = l + 1, i = k
  i = k;
  j = l + 1;
}

// A chunk of occupied pairs: every (i <= j) with j0 <= j < j1.  Its
// lambda+ rows are [ppos(j0), ppos(j1)) and lambda- rows [pneg(j0), pneg(j1)).
struct Chunk {
  int j0, j1;
};
constexpr int kMaxChunks = 64;

// Bounded spin budget for every device-side wait (iterations of try_wait,
// each of which may itself suspend for a hardware-defined time).
constexpr uint32_t kSpinLimit = 1u << 26;

// Value of a double-single accumulator (hi, lo).
__host__ __device__ inline double ds_value(float2 v) { return (double)v.x + (double)v.y; }

__device__ __forceinline__ void record_status(int *status, int site) {
  if (status) atomicCAS(status, 0, site);
}

}  // namespace ladder
