// Closed-shell RI-CCSD iteration (Sec. II.A): the CCSD amplitude equations
// solved by Jacobi steps accelerated with DIIS over a few stored iterates,
// with the particle-particle ladder of every step taken by the library's
// ladder kernels (ladder_apply on a caller's plan).
//
// The equations are the CCSD projections of exp(-T) H exp(T) in spin
// orbitals, organised with the one- and two-body intermediates of Stanton,
// Gauss, Watts and Bartlett (J. Chem. Phys. 94, 4334, 1991); the reference is
// canonical Hartree-Fock (diagonal Fock matrix of the orbital energies) and
// the integrals come from the RI factors, (pq|rs) = sum_P B^P_pq B^P_rs.
//
// Spin blocks.  For a closed-shell reference every spin-orbital tensor is
// unchanged when all its spins flip, and it vanishes unless spin is conserved
// along its two index pairs.  Every four-index tensor here pairs positions
// (0, 2) and (1, 3) (<pq||rs>: p-r and q-s; t_ij^ab: i-a and j-b), so it is
// held as three spatial arrays, the spin blocks aaaa, abab and abba (the
// others are their flips or zero), and a two-index tensor as one (aa).  A
// spin-orbital contraction is then the sum, over the spins of its summed
// indices, of spatial contractions of the matching blocks, for each block of
// the result: the same equations as in spin orbitals, on arrays of spatial
// size.  The closed-shell amplitudes are t_i^a (the aa block) and t_ij^ab
// (the abab block).
//
// Every contraction is a GEMM of the CUDA-core kernel of dress.cu on operands
// brought into [rows][K] order by a permutation kernel (transpose - GEMM -
// transpose), in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "ladder.h"

namespace ladder {
namespace {

// ---------------------------------------------------------------- kernels
struct PermArgs {
  const double *in;
  double *out;
  long long n;
  int nd;
  long long od[4];    // output extents
  long long istr[4];  // input stride of output dimension d
  double alpha, beta;
};

// out[e] = alpha in[perm(e)] (+ beta out[e]) over the output's row-major
// order; index arithmetic in 32 bits when the arrays allow it
template <typename I>
__global__ void permute_kernel(const PermArgs a) {
  const I n = (I)a.n;
  I od[4], is[4];
  for (int d = 0; d < 4; ++d) {
    od[d] = (I)a.od[d];
    is[d] = (I)a.istr[d];
  }
  for (I e = blockIdx.x * (I)blockDim.x + threadIdx.x; e < n; e += (I)gridDim.x * blockDim.x) {
    I r = e, off = 0;
    for (int d = a.nd - 1; d >= 0; --d) {
      const I x = r % od[d];
      r /= od[d];
      off += x * is[d];
    }
    const double v = a.alpha * a.in[off];
    a.out[e] = a.beta != 0.0 ? v + a.beta * a.out[e] : v;
  }
}

// The three spin blocks of <pq||rs> = <pq|rs> - <pq|sr> over one range of
// each index (occupied or virtual), from the spatial (pq|rs) = eri[p][q][r][s]:
//   aaaa = (pr|qs) - (ps|qr),  abab = (pr|qs),  abba = -(ps|qr).
struct IntArgs {
  const double *eri;
  double *aaaa, *abab, *abba;
  int n, o;
  int vir[4];  // 1: that index runs over the virtual orbitals
  long long ext[4];
};

__global__ void int_blocks_kernel(const IntArgs a) {
  const long long tot = a.ext[0] * a.ext[1] * a.ext[2] * a.ext[3];
  const long long n = a.n, nn = n * n, nnn = nn * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    long long orb[4];
    for (int d = 3; d >= 0; --d) {
      const long long x = r % a.ext[d];
      r /= a.ext[d];
      orb[d] = x + (a.vir[d] ? a.o : 0);
    }
    const double J = a.eri[orb[0] * nnn + orb[2] * nn + orb[1] * n + orb[3]];  // (pr|qs)
    const double K = a.eri[orb[0] * nnn + orb[3] * nn + orb[1] * n + orb[2]];  // (ps|qr)
    a.aaaa[e] = J - K;
    a.abab[e] = J;
    a.abba[e] = -K;
  }
}

// tau = t2 + t1 t1 - (t1 t1, a <-> b), tau_t the same with halves, and
// X = t2 / 2 + t_j^f t_n^b (laid out [j][n][f][b]), block by block: the
// product t_i^a t_j^b lives in the aaaa and abab blocks, t_i^b t_j^a in aaaa
// and abba.
__global__ void tau_blocks_kernel(const double *__restrict__ t1, const double *const *t2, double *const *tau,
                                  double *const *tau_t, double *const *X, int o, int v) {
  const long long n = (long long)o * o * v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % v), a = (int)((e / v) % v), j = (int)((e / v / v) % o), i = (int)(e / v / v / o);
    const double p = t1[(long long)i * v + a] * t1[(long long)j * v + b];
    const double q = t1[(long long)i * v + b] * t1[(long long)j * v + a];
    // aaaa, abab, abba
    const double pp[3] = {p, p, 0.0}, qq[3] = {q, 0.0, q};
    for (int k = 0; k < 3; ++k) {
      const double t = t2[k][e];
      tau[k][e] = t + pp[k] - qq[k];
      tau_t[k][e] = t + 0.5 * (pp[k] - qq[k]);
      X[k][e] = 0.5 * t + pp[k];
    }
  }
}

// x_new = rhs / D (D = eps_occ sums - eps_vir sums, spatial), err = x_new - x
__global__ void jacobi_kernel(const double *__restrict__ rhs, const double *__restrict__ x, const double *eps,
                              int o, int v, int rank, double *__restrict__ xn, double *__restrict__ err) {
  const long long n = rank == 1 ? (long long)o * v : (long long)o * o * v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double D;
    if (rank == 1) {
      D = eps[e / v] - eps[o + e % v];
    } else {
      const int b = (int)(e % v), a = (int)((e / v) % v), j = (int)((e / v / v) % o), i = (int)(e / v / v / o);
      D = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    }
    const double y = rhs[e] / D;
    xn[e] = y;
    err[e] = y - x[e];
  }
}

// The ladder R_ij^ab = sum_cd (ac|bd) tau_ij^cd (spatial) as the term
// 1/2 sum_ef tau_ij^ef <ab||ef> of the doubles: abab += R, abba -= R^ba,
// aaaa += R - R^ba.
__global__ void ladder_blocks_kernel(const double *__restrict__ R, double *__restrict__ aaaa,
                                     double *__restrict__ abab, double *__restrict__ abba, int o, int v) {
  const long long n = (long long)o * o * v * v, vv = (long long)v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long ij = e / vv;
    const int b = (int)(e % v), a = (int)((e / v) % v);
    const double rab = R[e], rba = R[ij * vv + (long long)b * v + a];
    aaaa[e] += rab - rba;
    abab[e] += rab;
    abba[e] -= rba;
  }
}

// partial dot products x . y over grid-strided slices, one per block (fixed order)
__global__ void dot_kernel(const double *__restrict__ x, const double *__restrict__ y, long long n,
                           double *part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s += x[e] * y[e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// y = sum_k c_k x_k over up to 8 vectors
struct CombArgs {
  const double *x[8];
  double c[8];
  int m;
  double *y;
  long long n;
};
__global__ void combine_kernel(const CombArgs a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < a.n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < a.m; ++k) s += a.c[k] * a.x[k][e];
    a.y[e] = s;
  }
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

// ---------------------------------------------------------------- tensors and contractions
struct Ten {
  double *p = nullptr;
  int nd = 0;
  long long d[4] = {1, 1, 1, 1};
  long long size() const {
    long long s = 1;
    for (int k = 0; k < nd; ++k) s *= d[k];
    return s;
  }
};

Ten ten(double *p, std::initializer_list<long long> dims) {
  Ten t;
  t.p = p;
  for (long long x : dims) t.d[t.nd++] = x;
  return t;
}

// A bump allocator over the workspace (offsets aligned to 256 bytes).
struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  double *take(long long n) {
    const size_t bytes = ((size_t)std::max<long long>(n, 1) * sizeof(double) + 255) / 256 * 256;
    if (off + bytes > cap) return nullptr;
    double *p = reinterpret_cast<double *>(base + off);
    off += bytes;
    return p;
  }
};

struct Engine {
  cudaStream_t s;
  double *ta, *tb, *tc;  // permutation and product scratch, each `scratch` doubles
  long long scratch;
  cudaError_t err = cudaSuccess;

  // out (labels lo) = alpha * in (labels li, a permutation of lo) + beta * out
  void permute(const Ten &in, const char *li, const Ten &out, const char *lo, double alpha, double beta) {
    if (err != cudaSuccess) return;
    PermArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = in.p;
    a.out = out.p;
    a.nd = out.nd;
    a.n = out.size();
    a.alpha = alpha;
    a.beta = beta;
    long long istr[4];
    long long st = 1;
    for (int k = in.nd - 1; k >= 0; --k) {
      istr[k] = st;
      st *= in.d[k];
    }
    for (int k = 0; k < out.nd; ++k) {
      a.od[k] = out.d[k];
      const char *f = std::strchr(li, lo[k]);
      a.istr[k] = istr[f - li];
    }
    if (a.n < (1ll << 31) && in.size() < (1ll << 31))
      permute_kernel<unsigned><<<grid_for(a.n), 256, 0, s>>>(a);
    else
      permute_kernel<unsigned long long><<<grid_for(a.n), 256, 0, s>>>(a);
    err = cudaGetLastError();
  }

  // C (labels lc) = alpha * sum over the labels A and B share of A B + beta * C.
  // Every label of C is in exactly one of A and B; the shared labels are summed.
  void contract(const char *la, const Ten &A, const char *lb, const Ten &B, const char *lc, const Ten &C,
                double alpha, double beta) {
    if (err != cudaSuccess) return;
    std::string M, N, K;
    for (const char *c = lc; *c; ++c) (std::strchr(la, *c) ? M : N) += *c;
    for (const char *c = la; *c; ++c)
      if (!std::strchr(lc, *c)) K += *c;
    auto extent = [&](char c) -> long long {
      const char *f = std::strchr(la, c);
      if (f) return A.d[f - la];
      return B.d[std::strchr(lb, c) - lb];
    };
    long long m = 1, n = 1, k = 1;
    for (char c : M) m *= extent(c);
    for (char c : N) n *= extent(c);
    for (char c : K) k *= extent(c);
    // split K over CTAs when the product has few 128 x 128 tiles (the FP64
    // pipe of one SM is slow): partial products side by side in tc, summed
    const long long tiles = ((m + 127) / 128) * ((n + 127) / 128);
    long long ks = 1;
    if (tiles < 2 * 152 && k >= 1024) ks = std::min<long long>((2 * 152 + tiles - 1) / tiles, k / 512);
    ks = std::max<long long>(1, std::min<long long>(ks, scratch / std::max<long long>(m * n, 1)));
    if (m * k > scratch || n * k > scratch || m * n > scratch) {
      err = cudaErrorInvalidValue;
      return;
    }
    // A -> [M][K], B -> [N][K]
    auto bring = [&](const Ten &X, const char *lx, const std::string &rows, double *dst) {
      Ten t;
      t.p = dst;
      std::string lbl = rows + K;
      for (char c : lbl) t.d[t.nd++] = extent(c);
      permute(X, lx, t, lbl.c_str(), 1.0, 0.0);
    };
    bring(A, la, M, ta);
    bring(B, lb, N, tb);
    if (err != cudaSuccess) return;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = ta;
    g.B = tb;
    g.Out = tc;
    g.sam = k;
    g.sak = 1;
    g.sbn = k;
    g.sbk = 1;
    g.M = (int)m;
    g.N = (int)n;
    g.K = (int)k;
    g.ksplit = (int)ks;
    g.kchunk = (int)((k + ks - 1) / ks);
    g.epi = kEpiStore;  // split q of K at tc + q m n, [m][n]
    g.ldo = (int)n;
    g.so_batch = m * n;
    err = launch_gemm<double, double, double>(g, 1, s);
    if (err == cudaSuccess && ks > 1) err = launch_reduce<double>(tc, m * n, (int)ks, s);
    if (err != cudaSuccess) return;
    Ten t;
    t.p = tc;
    std::string lbl = M + N;
    for (char c : lbl) t.d[t.nd++] = extent(c);
    permute(t, lbl.c_str(), C, lc, alpha, beta);
  }
};

// A closed-shell spin-orbital tensor by spin blocks: nd = 2 holds the aa
// block, nd = 4 the aaaa, abab and abba blocks (positions (0, 2) and (1, 3)
// paired); the flipped blocks are equal to these, the rest vanish.
struct ST {
  int nd = 0;
  Ten b[3];
};

// block index of the spins s[] (0 alpha, 1 beta) of a tensor's indices, -1 if zero
int st_block(int nd, const int *s) {
  if (nd == 2) return s[0] == s[1] ? 0 : -1;
  if (s[0] == s[1] && s[1] == s[2] && s[2] == s[3]) return 0;
  if (s[0] == s[2] && s[1] == s[3]) return 1;
  if (s[0] == s[3] && s[1] == s[2]) return 2;
  return -1;
}

// spins of the stored blocks, in label order
const int kBlockSpins[3][4] = {{0, 0, 0, 0}, {0, 1, 0, 1}, {0, 1, 1, 0}};

struct SpinEngine {
  Engine *e;

  void scale(const Ten &t, double beta) {
    if (beta == 1.0 || e->err != cudaSuccess) return;
    if (beta == 0.0) {
      e->err = cudaMemsetAsync(t.p, 0, (size_t)t.size() * sizeof(double), e->s);
      return;
    }
    std::string l = std::string("pqrs").substr(0, t.nd);
    e->permute(t, l.c_str(), t, l.c_str(), beta, 0.0);
  }

  // Z (labels lc) = alpha sum over the shared labels of X Y + beta Z, summed
  // over the spins of the shared labels for every stored block of Z
  void contract(const char *la, const ST &X, const char *lb, const ST &Y, const char *lc, const ST &Z,
                double alpha, double beta) {
    std::string K;
    for (const char *c = la; *c; ++c)
      if (!std::strchr(lc, *c)) K += *c;
    const int nb = Z.nd == 2 ? 1 : 3;
    for (int ob = 0; ob < nb; ++ob) {
      int spin[128];
      for (int k = 0; lc[k]; ++k) spin[(int)lc[k]] = kBlockSpins[ob][k];
      bool first = true;
      for (int mask = 0; mask < (1 << K.size()); ++mask) {
        for (size_t t = 0; t < K.size(); ++t) spin[(int)K[t]] = (mask >> t) & 1;
        int sx[4], sy[4];
        for (int k = 0; la[k]; ++k) sx[k] = spin[(int)la[k]];
        for (int k = 0; lb[k]; ++k) sy[k] = spin[(int)lb[k]];
        const int bx = st_block(X.nd, sx), by = st_block(Y.nd, sy);
        if (bx < 0 || by < 0) continue;
        e->contract(la, X.b[bx], lb, Y.b[by], lc, Z.b[ob], alpha, first ? beta : 1.0);
        first = false;
      }
      if (first) scale(Z.b[ob], beta);
    }
  }

  // Z (labels lo) = alpha X (labels li) + beta Z, block by block
  void permute(const ST &X, const char *li, const ST &Z, const char *lo, double alpha, double beta) {
    const int nb = Z.nd == 2 ? 1 : 3;
    for (int ob = 0; ob < nb; ++ob) {
      int spin[128], sx[4];
      for (int k = 0; lo[k]; ++k) spin[(int)lo[k]] = kBlockSpins[ob][k];
      for (int k = 0; li[k]; ++k) sx[k] = spin[(int)li[k]];
      const int bx = st_block(X.nd, sx);
      if (bx < 0)
        scale(Z.b[ob], beta);
      else
        e->permute(X.b[bx], li, Z.b[ob], lo, alpha, beta);
    }
  }
};

}  // namespace


// ---------------------------------------------------------------- solver
// Workspace of the solver, in doubles: the spatial (pq|rs), three spin blocks
// of each integral class, the amplitudes and intermediates by spin block, the
// contraction scratch and the DIIS history.
struct CcsdSizes {
  long long eri, ints, t1, t2, scratch;
  size_t bytes;
};

static CcsdSizes ccsd_sizes(int o, int v, int naux, int ndiis) {
  const long long n = o + v, oo = (long long)o * o, vv = (long long)v * v, ov = (long long)o * v;
  CcsdSizes z;
  z.eri = n * n * n * n;
  // oooo, ooov, oovv, ovov, ovvv, vovv, oovo, ovvo, vvvo, ovoo
  z.ints = 3 * (oo * oo + 2 * oo * ov + 3 * oo * vv + 3 * ov * vv + oo * ov);
  z.t1 = ov;
  z.t2 = oo * vv;
  z.scratch = std::max<long long>(std::max<long long>(ov * vv, oo * vv), std::max<long long>(n * n * 8, naux * ov));
  long long s = z.eri + z.ints + 3 * z.scratch + (long long)naux * n * n;
  s += 4 * z.t1 + 4 * 3 * z.t2;                                  // t, t new, rhs, step
  s += 3 * 3 * z.t2;                                              // tau, tau_t, X
  s += 3 * 3 * z.t2 + 3 * std::max<long long>(oo * oo, z.t2);    // ring, Q, W1 and W2
  s += z.t2;                                                      // the spatial ladder R
  s += vv + oo + ov + 3 * oo * oo + 3 * ov * ov + 3 * oo * ov + 3 * vv * ov;  // intermediates
  s += 2 * (long long)ndiis * (z.t1 + 3 * z.t2);                  // DIIS history
  s += 4096 + n;
  z.bytes = (size_t)s * sizeof(double) + 256 * 256;  // + the alignment of every array
  return z;
}

}  // namespace ladder

using namespace ladder;

extern "C" {

ladder_status ladder_ccsd_workspace_size(int o, int v, int naux, int ndiis, size_t *bytes) {
  if (!bytes || o < 1 || v < 1 || naux < 1 || ndiis < 0 || ndiis > 8 || o > 128 || v > 1024) return LADDER_EINVAL;
  *bytes = ccsd_sizes(o, v, naux, ndiis).bytes;
  return LADDER_OK;
}

ladder_status ladder_ccsd(ladder_plan_t plan, int o, int v, int naux, const double *B, const double *Bov,
                          const double *Boo, const double *e_occ, const double *e_vir, int max_iter, double tol,
                          int ndiis, double *t1, double *t2, double *E_host, int *iters, void *workspace,
                          size_t ws_bytes, void *stream) {
  int po = 0, pv = 0, pn = 0;
  if (!plan || ladder_plan_shape(plan, &po, &pv, &pn) != LADDER_OK || po != o || pv != v || pn != naux ||
      !B || !Bov || !Boo || !e_occ || !e_vir || !t1 || !t2 || !E_host || !iters || !workspace || max_iter < 1 ||
      !(tol > 0.0) || ndiis < 0 || ndiis > 8 || o < 1 || v < 1 || naux < 1 || o > 128 || v > 1024)
    return LADDER_EINVAL;
  const CcsdSizes z = ccsd_sizes(o, v, naux, ndiis);
  if (ws_bytes < z.bytes) return LADDER_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = o + v;
  Arena ar;
  ar.base = static_cast<char *>(workspace);
  ar.cap = ws_bytes;
  double *Bf = ar.take((long long)naux * n * n);
  double *eri = ar.take(z.eri);
  Engine eng;
  eng.s = s;
  eng.scratch = z.scratch;
  eng.ta = ar.take(z.scratch);
  eng.tb = ar.take(z.scratch);
  eng.tc = ar.take(z.scratch);
  SpinEngine se{&eng};
  auto st2 = [&](long long d0, long long d1) {
    ST t;
    t.nd = 2;
    t.b[0] = ten(ar.take(d0 * d1), {d0, d1});
    return t;
  };
  auto st4 = [&](long long d0, long long d1, long long d2, long long d3) {
    ST t;
    t.nd = 4;
    for (int k = 0; k < 3; ++k) t.b[k] = ten(ar.take(d0 * d1 * d2 * d3), {d0, d1, d2, d3});
    return t;
  };
  const long long O = o, V = v;
  const ST g_oooo = st4(O, O, O, O), g_ooov = st4(O, O, O, V), g_oovv = st4(O, O, V, V);
  const ST g_ovov = st4(O, V, O, V), g_ovvv = st4(O, V, V, V), g_vovv = st4(V, O, V, V);
  const ST g_oovo = st4(O, O, V, O), g_ovvo = st4(O, V, V, O), g_vvvo = st4(V, V, V, O);
  const ST g_ovoo = st4(O, V, O, O);
  const ST T1 = st2(O, V), T1n = st2(O, V), R1 = st2(O, V), E1 = st2(O, V);
  const ST T2 = st4(O, O, V, V), T2n = st4(O, O, V, V), R2 = st4(O, O, V, V), E2 = st4(O, O, V, V);
  const ST Tau = st4(O, O, V, V), Taut = st4(O, O, V, V), X = st4(O, O, V, V);
  const ST Ring = st4(O, O, V, V), Q = st4(O, O, V, V), W1 = st4(O, O, V, V);
  ST W2;  // Y_ijmn and the P(ij) term of Wmnij
  W2.nd = 4;
  for (int k = 0; k < 3; ++k) W2.b[k] = ten(ar.take(std::max<long long>(O * O * O * O, z.t2)), {O, O, O, O});
  double *Rsp = ar.take(z.t2);
  const ST Fae = st2(V, V), Fmi = st2(O, O), Fme = st2(O, V);
  const ST Wmnij = st4(O, O, O, O), Wmbej = st4(O, V, V, O), Zijam = st4(O, O, V, O), U = st4(V, V, V, O);
  double *eps = ar.take(n), *red = ar.take(4096);
  std::vector<double *> hv, he;
  const long long nvec = z.t1 + 3 * z.t2;
  for (int k = 0; k < ndiis; ++k) {
    hv.push_back(ar.take(nvec));
    he.push_back(ar.take(nvec));
  }
  if (!red || (ndiis && !he.back())) return LADDER_EWORKSPACE;
  // ---- integrals: B^P_pq over all orbitals, (pq|rs), spin blocks of <pq||rs>
  {
    std::vector<double> h_eps(n);
    if (cudaMemcpyAsync(h_eps.data(), e_occ, o * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h_eps.data() + o, e_vir, v * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpyAsync(eps, h_eps.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(Bf, 0, (size_t)naux * n * n * sizeof(double), s) != cudaSuccess)
      return LADDER_ECUDA;
    for (int P = 0; P < naux; ++P)
      if (cudaMemcpy2DAsync(Bf + (size_t)P * n * n, n * sizeof(double), Boo + (size_t)P * o * o, o * sizeof(double),
                            o * sizeof(double), o, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaMemcpy2DAsync(Bf + (size_t)P * n * n + o, n * sizeof(double), Bov + (size_t)P * o * v,
                            v * sizeof(double), v * sizeof(double), o, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaMemcpy2DAsync(Bf + (size_t)P * n * n + (size_t)o * n + o, n * sizeof(double), B + (size_t)P * v * v,
                            v * sizeof(double), v * sizeof(double), v, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LADDER_ECUDA;
    // the vo block: Bf[P][o + a][i] = Bov[P][i][a]
    eng.permute(ten(const_cast<double *>(Bov), {naux, o, v}), "Pia", ten(eng.ta, {naux, v, o}), "Pai", 1.0, 0.0);
    for (int P = 0; P < naux && eng.err == cudaSuccess; ++P)
      if (cudaMemcpy2DAsync(Bf + (size_t)P * n * n + (size_t)o * n, n * sizeof(double), eng.ta + (size_t)P * v * o,
                            o * sizeof(double), o * sizeof(double), v, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LADDER_ECUDA;
    // eri[(pq)][(rs)] = sum_P Bf[P][pq] Bf[P][rs]
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.A = Bf;
    g.B = Bf;
    g.Out = eri;
    g.sam = 1;
    g.sak = (long long)n * n;
    g.sbn = 1;
    g.sbk = (long long)n * n;
    g.M = g.N = n * n;
    g.K = naux;
    g.kchunk = naux;
    g.ksplit = 1;
    g.ldo = n * n;
    g.epi = kEpiStore;
    if (launch_gemm<double, double, double>(g, 1, s) != cudaSuccess) return LADDER_ECUDA;
    auto blocks = [&](const ST &t, int v0, int v1, int v2, int v3) {
      IntArgs a;
      a.eri = eri;
      a.aaaa = t.b[0].p;
      a.abab = t.b[1].p;
      a.abba = t.b[2].p;
      a.n = n;
      a.o = o;
      const int vv_[4] = {v0, v1, v2, v3};
      for (int d = 0; d < 4; ++d) {
        a.vir[d] = vv_[d];
        a.ext[d] = vv_[d] ? v : o;
      }
      int_blocks_kernel<<<grid_for(a.ext[0] * a.ext[1] * a.ext[2] * a.ext[3]), 256, 0, s>>>(a);
    };
    blocks(g_oooo, 0, 0, 0, 0);
    blocks(g_ooov, 0, 0, 0, 1);
    blocks(g_oovv, 0, 0, 1, 1);
    blocks(g_ovov, 0, 1, 0, 1);
    blocks(g_ovvv, 0, 1, 1, 1);
    blocks(g_vovv, 1, 0, 1, 1);
    blocks(g_oovo, 0, 0, 1, 0);
    blocks(g_ovvo, 0, 1, 1, 0);
    blocks(g_vvvo, 1, 1, 1, 0);
    blocks(g_ovoo, 0, 1, 0, 0);
    if (cudaGetLastError() != cudaSuccess || eng.err != cudaSuccess) return LADDER_ECUDA;
  }
  // ---- zero amplitudes
  if (cudaMemsetAsync(T1.b[0].p, 0, z.t1 * sizeof(double), s) != cudaSuccess) return LADDER_ECUDA;
  for (int k = 0; k < 3; ++k)
    if (cudaMemsetAsync(T2.b[k].p, 0, z.t2 * sizeof(double), s) != cudaSuccess) return LADDER_ECUDA;
  auto dot = [&](const double *x, const double *y, long long len, double &out) -> bool {
    dot_kernel<<<1024, 256, 0, s>>>(x, y, len, red);
    std::vector<double> h(1024);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), red, 1024 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return false;
    out = 0.0;
    for (double x_ : h) out += x_;
    return true;
  };
  // the device pointer tables of the block kernels
  double *ptrs = ar.take(64);
  if (!ptrs) return LADDER_EWORKSPACE;
  {
    const double *tab[12] = {T2.b[0].p, T2.b[1].p, T2.b[2].p, Tau.b[0].p, Tau.b[1].p, Tau.b[2].p,
                             Taut.b[0].p, Taut.b[1].p, Taut.b[2].p, X.b[0].p, X.b[1].p, X.b[2].p};
    if (cudaMemcpyAsync(ptrs, tab, sizeof(tab), cudaMemcpyHostToDevice, s) != cudaSuccess) return LADDER_ECUDA;
  }
  double *const *dT2 = reinterpret_cast<double *const *>(ptrs);
  auto tau_blocks = [&]() {
    tau_blocks_kernel<<<grid_for(z.t2), 256, 0, s>>>(T1.b[0].p, reinterpret_cast<const double *const *>(dT2), dT2 + 3,
                                                    dT2 + 6, dT2 + 9, o, v);
  };
  double E = 0.0;
  int it = 0, stored = 0;
  for (; it < max_iter; ++it) {
    tau_blocks();
    // ---- one-body intermediates (diagonal Fock parts and f_ia vanish)
    se.contract("mf", T1, "mafe", g_ovvv, "ae", Fae, 1.0, 0.0);
    se.contract("mnaf", Taut, "mnef", g_oovv, "ae", Fae, -0.5, 1.0);
    se.contract("ne", T1, "mnie", g_ooov, "mi", Fmi, 1.0, 0.0);
    se.contract("inef", Taut, "mnef", g_oovv, "mi", Fmi, 0.5, 1.0);
    se.contract("nf", T1, "mnef", g_oovv, "me", Fme, 1.0, 0.0);
    // ---- Wmnij = <mn||ij> + P(ij) t_j^e <mn||ie> + 1/4 tau_ij^ef <mn||ef>
    se.permute(g_oooo, "mnij", Wmnij, "mnij", 1.0, 0.0);
    se.contract("je", T1, "mnie", g_ooov, "mnij", W2, 1.0, 0.0);
    se.permute(W2, "mnij", Wmnij, "mnij", 1.0, 1.0);
    se.permute(W2, "mnji", Wmnij, "mnij", -1.0, 1.0);
    se.contract("ijef", Tau, "mnef", g_oovv, "mnij", Wmnij, 0.25, 1.0);
    // ---- Wmbej = <mb||ej> + t_j^f <mb||ef> - t_n^b <mn||ej> - (t_jn^fb / 2 + t_j^f t_n^b) <mn||ef>
    se.permute(g_ovvo, "mbej", Wmbej, "mbej", 1.0, 0.0);
    se.contract("jf", T1, "mbef", g_ovvv, "mbej", Wmbej, 1.0, 1.0);
    se.contract("nb", T1, "mnej", g_oovo, "mbej", Wmbej, -1.0, 1.0);
    se.contract("jnfb", X, "mnef", g_oovv, "mbej", Wmbej, -1.0, 1.0);
    // ---- singles right-hand side
    se.contract("ie", T1, "ae", Fae, "ia", R1, 1.0, 0.0);
    se.contract("ma", T1, "mi", Fmi, "ia", R1, -1.0, 1.0);
    se.contract("imae", T2, "me", Fme, "ia", R1, 1.0, 1.0);
    se.contract("nf", T1, "naif", g_ovov, "ia", R1, -1.0, 1.0);
    se.contract("imef", T2, "maef", g_ovvv, "ia", R1, -0.5, 1.0);
    se.contract("mnae", T2, "nmei", g_oovo, "ia", R1, -0.5, 1.0);
    // ---- doubles right-hand side
    se.permute(g_oovv, "ijab", R2, "ijab", 1.0, 0.0);
    // P(ab) t_ij^ae F'_be with F'_be = F_be - t_m^b F_me / 2 (formed in Fae's storage)
    se.contract("mb", T1, "me", Fme, "be", Fae, -0.5, 1.0);
    se.contract("ijae", T2, "be", Fae, "ijab", W1, 1.0, 0.0);
    se.permute(W1, "ijab", R2, "ijab", 1.0, 1.0);
    se.permute(W1, "ijba", R2, "ijab", -1.0, 1.0);
    // - P(ij) t_im^ab F'_mj with F'_mj = F_mj + t_j^e F_me / 2
    se.contract("je", T1, "me", Fme, "mj", Fmi, 0.5, 1.0);
    se.contract("imab", T2, "mj", Fmi, "ijab", W1, 1.0, 0.0);
    se.permute(W1, "ijab", R2, "ijab", -1.0, 1.0);
    se.permute(W1, "jiab", R2, "ijab", 1.0, 1.0);
    // 1/2 tau_mn^ab Wmnij
    se.contract("mnab", Tau, "mnij", Wmnij, "ijab", R2, 0.5, 1.0);
    // 1/2 tau_ij^ef Wabef without <ab||ef>: -1/2 P(ab) t_m^b Z_ijam + 1/8 tau_mn^ab Y_ijmn
    se.contract("ijef", Tau, "amef", g_vovv, "ijam", Zijam, 1.0, 0.0);
    se.contract("ijam", Zijam, "mb", T1, "ijab", Q, 1.0, 0.0);
    se.permute(Q, "ijab", R2, "ijab", -0.5, 1.0);
    se.permute(Q, "ijba", R2, "ijab", 0.5, 1.0);
    se.contract("ijef", Tau, "mnef", g_oovv, "ijmn", W2, 1.0, 0.0);
    se.contract("mnab", Tau, "ijmn", W2, "ijab", R2, 0.125, 1.0);
    // P(ij) P(ab) (t_im^ae Wmbej - t_i^e t_m^a <mb||ej>)
    se.contract("imae", T2, "mbej", Wmbej, "ijab", Ring, 1.0, 0.0);
    se.contract("ma", T1, "mbej", g_ovvo, "abej", U, 1.0, 0.0);
    se.contract("ie", T1, "abej", U, "ijab", Ring, -1.0, 1.0);
    se.permute(Ring, "ijab", R2, "ijab", 1.0, 1.0);
    se.permute(Ring, "jiab", R2, "ijab", -1.0, 1.0);
    se.permute(Ring, "ijba", R2, "ijab", -1.0, 1.0);
    se.permute(Ring, "jiba", R2, "ijab", 1.0, 1.0);
    // P(ij) t_i^e <ab||ej> - P(ab) t_m^a <mb||ij>
    se.contract("ie", T1, "abej", g_vvvo, "ijab", W1, 1.0, 0.0);
    se.permute(W1, "ijab", R2, "ijab", 1.0, 1.0);
    se.permute(W1, "jiab", R2, "ijab", -1.0, 1.0);
    se.contract("ma", T1, "mbij", g_ovoo, "ijab", W1, 1.0, 0.0);
    se.permute(W1, "ijab", R2, "ijab", -1.0, 1.0);
    se.permute(W1, "ijba", R2, "ijab", 1.0, 1.0);
    if (eng.err != cudaSuccess) return LADDER_ECUDA;
    // the ladder: 1/2 tau_ij^ef <ab||ef> from the spatial RI ladder of tau's
    // abab block (t_ij^ab + t_i^a t_j^b)
    {
      const ladder_status st = ladder_apply(plan, B, Tau.b[1].p, Rsp, s);
      if (st != LADDER_OK) return st;
    }
    ladder_blocks_kernel<<<grid_for(z.t2), 256, 0, s>>>(Rsp, R2.b[0].p, R2.b[1].p, R2.b[2].p, o, v);
    // ---- Jacobi step, DIIS
    jacobi_kernel<<<grid_for(z.t1), 256, 0, s>>>(R1.b[0].p, T1.b[0].p, eps, o, v, 1, T1n.b[0].p, E1.b[0].p);
    for (int k = 0; k < 3; ++k)
      jacobi_kernel<<<grid_for(z.t2), 256, 0, s>>>(R2.b[k].p, T2.b[k].p, eps, o, v, 2, T2n.b[k].p, E2.b[k].p);
    if (cudaGetLastError() != cudaSuccess) return LADDER_ECUDA;
    // the pieces of one DIIS vector: t1, then the three t2 blocks
    const double *pn_[4] = {T1n.b[0].p, T2n.b[0].p, T2n.b[1].p, T2n.b[2].p};
    const double *pe_[4] = {E1.b[0].p, E2.b[0].p, E2.b[1].p, E2.b[2].p};
    double *pt_[4] = {T1.b[0].p, T2.b[0].p, T2.b[1].p, T2.b[2].p};
    const long long len_[4] = {z.t1, z.t2, z.t2, z.t2}, off_[4] = {0, z.t1, z.t1 + z.t2, z.t1 + 2 * z.t2};
    bool copied = false;
    if (ndiis > 0) {
      const int slot = it % ndiis;
      for (int q = 0; q < 4; ++q)
        if (cudaMemcpyAsync(hv[slot] + off_[q], pn_[q], len_[q] * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(he[slot] + off_[q], pe_[q], len_[q] * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
          return LADDER_ECUDA;
      stored = std::min(stored + 1, ndiis);
      if (stored > 1) {
        // Pulay: minimise |sum c_k e_k| with sum c_k = 1 (the spin-orbital
        // norm counts each block twice, which scales the system uniformly)
        const int m = stored, q1 = m + 1;
        std::vector<double> A((size_t)q1 * q1, 0.0), rhs(q1, 0.0), c(q1, 0.0);
        for (int x = 0; x < m; ++x)
          for (int y = 0; y <= x; ++y) {
            double d;
            if (!dot(he[x], he[y], nvec, d)) return LADDER_ECUDA;
            A[x * q1 + y] = A[y * q1 + x] = d;
          }
        for (int x = 0; x < m; ++x) A[x * q1 + m] = A[m * q1 + x] = -1.0;
        rhs[m] = -1.0;
        // Gaussian elimination with partial pivoting
        for (int col = 0; col < q1; ++col) {
          int pr = col;
          for (int r = col + 1; r < q1; ++r)
            if (std::fabs(A[r * q1 + col]) > std::fabs(A[pr * q1 + col])) pr = r;
          if (A[pr * q1 + col] == 0.0) break;
          if (pr != col) {
            for (int k = 0; k < q1; ++k) std::swap(A[col * q1 + k], A[pr * q1 + k]);
            std::swap(rhs[col], rhs[pr]);
          }
          for (int r = col + 1; r < q1; ++r) {
            const double f = A[r * q1 + col] / A[col * q1 + col];
            for (int k = col; k < q1; ++k) A[r * q1 + k] -= f * A[col * q1 + k];
            rhs[r] -= f * rhs[col];
          }
        }
        for (int r = q1 - 1; r >= 0; --r) {
          double acc = rhs[r];
          for (int k = r + 1; k < q1; ++k) acc -= A[r * q1 + k] * c[k];
          c[r] = A[r * q1 + r] != 0.0 ? acc / A[r * q1 + r] : 0.0;
        }
        for (int q = 0; q < 4; ++q) {
          CombArgs ca;
          std::memset(&ca, 0, sizeof(ca));
          ca.m = m;
          for (int k = 0; k < m; ++k) {
            ca.x[k] = hv[k] + off_[q];
            ca.c[k] = c[k];
          }
          ca.y = pt_[q];
          ca.n = len_[q];
          combine_kernel<<<grid_for(ca.n), 256, 0, s>>>(ca);
        }
        copied = true;
      }
    }
    if (!copied)
      for (int q = 0; q < 4; ++q)
        if (cudaMemcpyAsync(pt_[q], pn_[q], len_[q] * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          return LADDER_ECUDA;
    // step size (2-norm over the stored blocks) and the energy
    // E = 1/4 sum <ij||ab> tau_ij^ab over spin orbitals = 1/2 sum over the three blocks
    double step = 0.0, En = 0.0;
    for (int q = 0; q < 4; ++q) {
      double d;
      if (!dot(pe_[q], pe_[q], len_[q], d)) return LADDER_ECUDA;
      step += d;
    }
    tau_blocks();
    for (int k = 0; k < 3; ++k) {
      double d;
      if (!dot(g_oovv.b[k].p, Tau.b[k].p, z.t2, d)) return LADDER_ECUDA;
      En += 0.5 * d;
    }
    if (!std::isfinite(En)) return LADDER_ENONFINITE;  // the iteration diverged
    const bool done = std::fabs(En - E) < tol && std::sqrt(step) < 1e3 * tol;
    E = En;
    if (done) {
      ++it;
      break;
    }
  }
  // closed-shell amplitudes: the aa block of t1 and the abab block of t2
  if (cudaMemcpyAsync(t1, T1.b[0].p, z.t1 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(t2, T2.b[1].p, z.t2 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LADDER_ECUDA;
  *E_host = E;
  *iters = it;
  return LADDER_OK;
}

}  // extern "C"
