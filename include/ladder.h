/*
 * ladder.h -- C ABI of the GB300 particle-particle ladder library.
 *
 * The library evaluates the closed-shell pp-ladder term of RI-CCSD
 * (arxiv 1810.08142, Sec. II.C):
 *
 *   R_ij^ab = sum_cd v^{ab}_{cd} tau_ij^cd                    (Eq. pp-Ladder-0)
 *   tau_ij^ab = t_ij^ab + t_i^a t_j^b                         (Eq. pp-Ladder-01)
 *   v^{ab}_{cd} = (ac|bd) = sum_P B^P_ac B^P_bd               (Eq. eri with Eq. RIM)
 *
 * with the undressed integrals (no t1 dressing of Eq. pp-Ladder-1), and the
 * ladder energy E_L = sum_ijab R_ij^ab (2 t_ij^ab - t_ij^ba).
 *
 * Conventions for every call:
 *   - Indices: o = number of occupied orbitals (i, j), v = number of virtual
 *     orbitals (a, b, c, d), naux = number of auxiliary functions (P).
 *   - Arrays are float64, C order (last index fastest), device pointers unless
 *     a name ends in _host, caller-owned, 16-byte aligned:
 *       B    [naux][v][v]    B[P][a][c] = B^P_ac (no a<->c symmetry assumed)
 *       t1   [o][v]          t_i^a
 *       t2   [o][o][v][v]    t_ij^ab
 *       tau  [o][o][v][v]    tau_ij^ab
 *       R    [o][o][v][v]    R_ij^ab
 *   - tau (and t2) must have the pair symmetry tau_ij^cd = tau_ji^dc of
 *     Sec. II.C.  Only the blocks with i <= j are read; R is written in full.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  No call synchronises the device or allocates device
 *     memory after ladder_set_workspace.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *     Errors found on the device (a bounded wait that ran out, a NaN or an
 *     infinity in B or tau) are recorded in a status word inside the
 *     workspace; ladder_last_device_error reads it.
 *   - The library reads no environment variables: every launch parameter is
 *     set through ladder_set_tuning.
 *   - A plan is not thread safe: one host thread at a time per plan, and calls
 *     that share a plan's workspace must not overlap on the device (enqueue
 *     them on one stream).
 */
#ifndef LADDER_H
#define LADDER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ladder_plan_s *ladder_plan_t;

typedef enum {
    LADDER_OK = 0,
    LADDER_EINVAL = 1,      /* bad size, null or misaligned pointer, bad mode */
    LADDER_ENOMEM = 2,      /* host allocation failed */
    LADDER_ECUDA = 3,       /* a CUDA runtime or driver call failed */
    LADDER_ETIMEOUT = 4,    /* a bounded device wait ran out (device status) */
    LADDER_ENOTSUP = 5,     /* mode or shape not supported on this device */
    LADDER_EWORKSPACE = 6,  /* workspace missing or too small */
    LADDER_ENONFINITE = 7   /* an input element was NaN or infinite (device status) */
} ladder_status;

typedef enum {
    LADDER_FP64 = 0,        /* plain method: FP64 tensor-core (DMMA) path, exact to rounding */
    LADDER_BF16X3 = 1,      /* split BF16, two slices (hi, lo), three products, FP32 accumulation */
    LADDER_BF16X6 = 2,      /* split BF16, three slices, six products, FP32 accumulation */
    LADDER_AUTO = 3,        /* let the plan pick (autotuned cache, else BF16X6) */
    LADDER_OZAKI = 4        /* error-free split BF16: FP64-class R and E_L from the tensor cores */
} ladder_mode;

/* LADDER_OZAKI follows the error-free splitting of Ozaki, Ogita, Oishi and
 * Rump (Numer. Algorithms 59, 2012) on the BF16 tensor cores.  Each operand
 * row (a row (a,c) of B over P; a row (i,j) of tau+- or (a,b) of V+- over the
 * slots of one block pair) is held as `oz_slices` (5 or 6) fixed-point BF16
 * slices under one power-of-two scale, so every slice product is exact; the
 * products of each slice order 0, 1, 2 accumulate in their own FP32 tensor-core
 * accumulator over windows short enough (128 auxiliary functions, one block
 * pair of 64 slots) that no partial sum is rounded, and the windows are
 * summed in double-single form (about 48 bits).  The only errors left are the
 * truncation of the slice expansion (about 2^-40 of each row's largest element
 * with 5 slices, 2^-48 with 6) and the double-single sums.  The mode always
 * runs the two-pass form and stores its sliced V+- tiles (S x 32 KiB per ab
 * tile and block pair: 136 GB at o=34, v=400, N_aux=1600 with 5 slices);
 * where all tiles would exceed 200 GiB it runs them in sequential ranges (see
 * tile_chunk in ladder_tuning).  With sym_b set in ladder_tuning (B^P_ac =
 * B^P_ca, the RI factors of real orbitals) it forms each distinct integral
 * tile once instead of GEMM1 per (ab tile, block pair).  ladder_backward
 * gives dtau only, with sym_b (see there).  ladder_apply_dressed runs its
 * correction in double-single FP32 arithmetic in this mode (compensated dot
 * products, about 48 bits). */

/* OR this into `mode` to size the workspace for ladder_backward as well
 * (the FP64 gradient with respect to B spills tiles of Gamma^{xb}_{yd}). */
#define LADDER_WITH_BACKWARD 16
/* OR this into `mode` to size the workspace for ladder_apply_dressed as well
 * (B - mbar in FP64, the integrals (kc|ld) and two small intermediates). */
#define LADDER_WITH_DRESSING 32

/* Create a plan for one shape.  1 <= o <= 256, 1 <= v <= 4096, 1 <= naux <= 65536.
 * The plan owns no device memory; see ladder_workspace_size.  LADDER_OZAKI
 * with LADDER_WITH_BACKWARD returns LADDER_ENOTSUP (its dtau needs no
 * backward workspace and it has no dB; see ladder_backward). */
ladder_status ladder_plan(int o, int v, int naux, int mode, ladder_plan_t *out);

/* Launch parameters of the split-BF16 kernel (ignored by LADDER_FP64):
 *   kc          GEMM1 K-steps (32 auxiliary functions each) per FP32
 *               accumulation chain, >= 1;
 *   s_pieces    16-slot GEMM2 pieces per fresh FP32 accumulator: 1, 2 or 4;
 *   flush_every FP32 accumulators summed before a flush into the
 *               double-single (FP32 pair, about 48-bit) sums, >= 1;
 *   ksplit      block-pair ranges per work unit (more CTAs for small shapes), >= 1;
 *   xy_split    1: separate GEMM1 accumulators for the hi*hi slice product and
 *               the smaller products; 0: one accumulator, two buffers;
 *   two_pass    0: one fused kernel (the integral tiles never leave the chip;
 *               GEMM1 is recomputed for every chunk of at most 128 occupied
 *               pairs); 1: GEMM1 once per (ab tile, block pair) with the
 *               sliced V+- tiles stored in the workspace (2S x 16 KiB per
 *               tile and block pair), then GEMM2 from the stored tiles in
 *               chunks of up to 192 occupied pairs.  Single-molecule plans
 *               pick 1 (LADDER_OZAKI: always 1);
 *   lambda_only 1: the paper's own contraction, which uses only the pair
 *               symmetry R_ij^ab = R_ji^ba (Sec. II.C), as an ablation of the
 *               +- split: the storing pass keeps (ac|bd) and (ad|bc) instead
 *               of their +- combinations, and GEMM2 runs over all o^2 ordered
 *               occupied pairs against both (twice the GEMM2 work).  Needs
 *               two_pass = 1; 0 (default) is the +- form.
 *   oz_slices   LADDER_OZAKI only: fixed-point slices per operand, 5 (default)
 *               or 6; 0 keeps the plan's value.  The other fields of
 *               LADDER_OZAKI plans are fixed, except ksplit and tile_chunk;
 *   tile_chunk  two-pass form and LADDER_OZAKI: tiles of 128 virtual pairs per
 *               sequential range (both passes and the unpack run range by
 *               range, reusing the stored-tile space; GEMM1 still runs once
 *               per tile and block pair, B and tau are re-read per range).
 *               0 (default): as many as keep one range's stored V+- tiles
 *               within 128 GiB (200 GiB for LADDER_OZAKI), which is all of
 *               them for o=34, v=400; >= 0.  With several ranges
 *               ladder_timing_passes reports the ladder kernels as pass 1
 *               and 0 for pass 2.
 *   sym_b       LADDER_OZAKI only (0 for the other modes, else LADDER_EINVAL):
 *               1 promises B^P_ac = B^P_ca for every P, a, c, as for the RI
 *               factors of real orbitals.  Then (ac|bd) depends only on the
 *               unordered pairs {a,c}, {b,d} and on them in either order, and
 *               the plan computes each distinct 64 x 64 integral tile (row
 *               block pair <= column block pair; about a quarter of the
 *               GEMM1 of the general form) once, in the same exact windows,
 *               keeps them in the workspace as double-single sums (32 KiB
 *               per tile: 26.7 GB at v=400), and forms and slices V+- of
 *               every ab tile from them; R agrees with the general form to
 *               the rounding of the tail slice orders (about 2^-48 of each
 *               integral).  Every ladder_apply checks
 *               the symmetry bitwise on the device; a B that breaks it makes
 *               ladder_last_device_error return LADDER_EINVAL.  A plan with
 *               a tile range (ladder_set_tile_range) forms all the distinct
 *               tiles and V+- of its own tiles.  Not with a plan made
 *               LADDER_WITH_DRESSING, or distinct tiles above 96 GiB (v
 *               above about 550): LADDER_ENOTSUP.
 * Longer chains are faster and less accurate (the tensor core's FP32
 * accumulation error grows with the MMAs per accumulator).  ladder_set_tuning
 * must come before ladder_set_workspace (the workspace size depends on
 * ksplit and two_pass); it returns LADDER_EINVAL for out-of-range values. */
typedef struct {
    int kc, s_pieces, flush_every, ksplit, xy_split, two_pass, lambda_only, oz_slices, tile_chunk, sym_b;
} ladder_tuning;
ladder_status ladder_get_tuning(ladder_plan_t plan, ladder_tuning *t);
ladder_status ladder_set_tuning(ladder_plan_t plan, const ladder_tuning *t);

/* Mode the plan resolved to (LADDER_AUTO resolves at plan time). */
ladder_status ladder_plan_mode(ladder_plan_t plan, int *mode);
/* The (o, v, naux) a single-molecule plan was made for (LADDER_EINVAL for a
 * batched plan). */
ladder_status ladder_plan_shape(ladder_plan_t plan, int *o, int *v, int *naux);

/* Multi-GPU partition of one molecule's term (the GPU analogue of the
 * paper's split of the virtual pairs over domains, Sec. II.D, Eq. pp-Ladder-3).
 * The split-BF16 and error-free modes evaluate R in tiles of 128 virtual
 * pairs {a, b} (a in a block of 16, b in a block of 8, a <= b); every tile
 * costs the same and writes R_ij^ab and R_ij^ba for all (i, j) of its pairs
 * and nothing else.  ladder_tile_count gives the shape's tile count;
 * ladder_set_tile_range (before ladder_set_workspace) restricts the plan to
 * tiles [tile_lo, tile_hi): ladder_apply then reads all of B and tau, writes
 * only those tiles' entries of R (the rest of R is left as it was) and needs
 * a workspace for those tiles only.  Ranks holding B and tau in full that
 * zero R, apply disjoint ranges covering [0, ntiles) and add their R
 * (all-reduce) assemble the full term; ladder_energy of a rank's R is its
 * share of E_L.  Tiles are enumerated a-block major: a in [16 iA, 16 iA + 16),
 * b in [8 jB, 8 jB + 8) for iA = 0, 1, ... and jB = 2 iA .. vp/8 - 1 (vp = v
 * rounded up to 16).  LADDER_FP64 plans return LADDER_ENOTSUP; a plan with a
 * partial range refuses ladder_backward and ladder_apply_dressed
 * (LADDER_ENOTSUP).  A LADDER_OZAKI plan with sym_b forms all the distinct
 * integral tiles in every range (they serve every tile) and V+- of its own
 * tiles only.  The range also sets the plan's block-pair splits (ksplit)
 * anew; set ksplit afterwards with ladder_set_tuning to match another
 * plan's. */
ladder_status ladder_tile_count(ladder_plan_t plan, int *ntiles);
ladder_status ladder_set_tile_range(ladder_plan_t plan, int tile_lo, int tile_hi);

/* Bytes of device scratch the plan needs (slices of B and tau, packed pair
 * combinations, reduction partials, the device status word).  The caller
 * allocates it and hands it over with ladder_set_workspace; the plan keeps
 * the pointer (not the memory) until ladder_destroy or the next call. */
ladder_status ladder_workspace_size(ladder_plan_t plan, size_t *bytes);
ladder_status ladder_set_workspace(ladder_plan_t plan, void *dptr, size_t bytes);

/* Eq. pp-Ladder-01: tau = t2 + t1 (x) t1 on the device, in FP64.  tau may not alias t2. */
ladder_status ladder_tau(ladder_plan_t plan, const double *t1, const double *t2,
                         double *tau, void *stream);

/* Eq. pp-Ladder-0: R_ij^ab = sum_cd (ac|bd) tau_ij^cd.  R is overwritten (not
 * accumulated); R may not alias B or tau.  The (ac|bd) integrals are formed
 * tile by tile on the tensor cores.  LADDER_FP64 and the fused split-BF16 form
 * (two_pass = 0) never write them to memory; the two-pass form (the split-BF16
 * default where it fits, and LADDER_OZAKI) writes their sliced symmetric and
 * antisymmetric combinations V+- to the workspace once and reads them back in
 * its GEMM2 pass. */
ladder_status ladder_apply(ladder_plan_t plan, const double *B, const double *tau,
                           double *R, void *stream);

/* The t1-dressed term, Eq. pp-Ladder-0 with the integrals of Eq. pp-Ladder-2:
 *   R_ij^ab = sum_cd b^{ab}_{cd} tau_ij^cd,
 *   b^{ab}_{cd} = sum_P B^P_ac (B^P_bd - mbar^P_bd) - sum_k t_k^a (kc|bd),
 *   mbar^P_bd = sum_k Bov^P_kd t_k^b   (Eq. pp-Ladder-21),
 * with (kc|bd) = sum_P Bov^P_kc B^P_bd from the same factors.
 *   B    [naux][v][v]  RI factor of the virtual block (as for ladder_apply)
 *   Bov  [naux][o][v]  RI factor of the occupied-virtual block, Bov[P][k][c]
 *   t1   [o][v]        singles t_k^a
 *   tau  [o][o][v][v]  as for ladder_apply (from ladder_tau)
 *   R    [o][o][v][v]  overwritten; may not alias an input
 * FP64, C-contiguous device arrays.  The plan must have been created with
 * LADDER_WITH_DRESSING (else LADDER_EINVAL) and is not a batch plan.  The
 * term runs as the undressed ladder of B - mbar (in the plan's mode) minus the
 * correction sum_kl t_k^a t_l^b sum_cd (kc|ld) tau_ij^cd, which costs
 * O(o^2 v^2 N + o^4 v^2) and is formed in FP64 (LADDER_FP64) or FP32. */
ladder_status ladder_apply_dressed(ladder_plan_t plan, const double *B, const double *Bov,
                                   const double *t1, const double *tau, double *R,
                                   void *stream);

/* The perturbative triples energy of Sec. II.A (no plan needed):
 *   E(T) = sum_ijk sum_abc (4 W_ijk^abc + W_ijk^bca + W_ijk^cab)
 *                          (V_ijk^abc - V_ijk^cba) / (3 D_ijk^abc),
 *   W_ijk^abc = P_ijk^abc ( sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab ),
 *   V_ijk^abc = W_ijk^abc + v_jk^bc t_i^a + v_ik^ac t_j^b + v_ij^ab t_k^c,
 *   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c,
 * P the sum over the six simultaneous orderings of (i,j,k) and (a,b,c), and
 * the integrals v^{pq}_{rs} = (pr|qs) = sum_P m^P_pr m^P_qs from the RI
 * factors of the orbital pairs (m^P_ai = m^P_ia):
 *   B [naux][v][v], Bov [naux][o][v], Boo [naux][o][o]   factors m^P
 *   t1 [o][v], t2 [o][o][v][v]                          amplitudes
 *   e_occ [o], e_vir [v]                                orbital energies
 * 1 <= o <= 256, 1 <= v <= 1024, 1 <= naux <= 65536.
 * E_dev: one double (device memory).  precision LADDER_TRIPLES_FP64 forms W
 * in FP64; LADDER_TRIPLES_FP32 forms the integrals and W in FP32 (the energy
 * sums stay FP64), both on the CUDA cores; LADDER_TRIPLES_BF16X6 forms the
 * integrals in FP32 and runs the W contractions on the tensor cores (tcgen05)
 * as split-BF16 GEMMs: three BF16 slices of each FP32 operand, the six slice
 * products p + q < 3, FP32 accumulation with the hi*hi product in its own
 * accumulator (v <= 256, else LADDER_ENOTSUP; if one of its bounded device
 * waits runs out, E_dev is NaN).  The work is 12 o^3 v^3 (v + o) flops.  The caller supplies a workspace of at least
 * ladder_triples_workspace_size bytes (256-byte aligned): the integrals
 * (o v^3 + o^3 v + o^2 v^2 elements), W for one (i, j) (o v^3) and the
 * reduction partials.  Asynchronous on `stream`; the result is reduced in a
 * fixed order (bitwise reproducible). */
#define LADDER_TRIPLES_FP64 0
#define LADDER_TRIPLES_FP32 1
#define LADDER_TRIPLES_BF16X6 2
ladder_status ladder_triples_workspace_size(int o, int v, int naux, int precision, size_t *bytes);
ladder_status ladder_triples(int o, int v, int naux, int precision, const double *B, const double *Bov,
                             const double *Boo, const double *t1, const double *t2, const double *e_occ,
                             const double *e_vir, double *E_dev, void *workspace, size_t ws_bytes,
                             void *stream);

/* E_L = sum_ijab R_ij^ab (2 t_ij^ab - t_ij^ba), reduced in FP64 in a fixed
 * order (bitwise reproducible); writes one double at E_dev (device memory). */
ladder_status ladder_energy(ladder_plan_t plan, const double *R, const double *t2,
                            double *E_dev, void *stream);

/* E_L as ladder_energy computes it, for callers that cannot allocate device
 * memory (no plan, no workspace).  The paper has no counterpart of this call.
 * The partial sums of the reduction live in a fixed 4 MiB array owned by the
 * library (524288 doubles; held on every device that loads the library until
 * the process exits).  Shapes that need more partials than that, i.e.
 * ceil(v/32)^2 * o^2 > 524288, return LADDER_ENOTSUP before any launch.
 * The first call on a device looks up the array's device address (make it
 * before any stream capture); calls that overlap on the GPU race on the
 * array.  R, t2 and E_dev are device pointers as for ladder_energy. */
ladder_status ladder_energy_noalloc(int o, int v, const double *R, const double *t2,
                                    double *E_dev, void *stream);

/* Adjoint of ladder_apply for E = sum W_ij^ab R_ij^ab with fixed weights W
 * (W must be pair symmetric, W_ij^ab = W_ji^ba; for E_L, W = 2 t2 - t2^T):
 *   dtau_ij^cd = sum_ab W_ij^ab (ac|bd)                          (transposed ladder)
 *   dB^P_xy    = sum_{ij,b,d} W_ij^{xb} tau_ij^{yd} B^P_bd
 *              + sum_{ij,a,c} W_ij^{ax} tau_ij^{cy} B^P_ac
 * Both run in the plan's mode.  dtau is the ladder of W with every factor
 * B^P transposed.  dB evaluates 2 x the first term (both terms are equal
 * under the pair symmetry of W and tau) as Gamma^{xb}_{yd} = sum_ij W_ij^{xb}
 * tau_ij^{yd} tiles contracted with B^P_bd; it needs a plan created with
 * LADDER_WITH_BACKWARD (else LADDER_EWORKSPACE).  Either output may be NULL
 * to skip it.  Outputs are overwritten.  dtau may not alias W or tau.
 * LADDER_OZAKI plans give dtau only, and only with sym_b: B^P symmetric makes
 * the transposed ladder the ladder itself, so dtau is the error-free forward
 * of W (FP64-class, no LADDER_WITH_BACKWARD needed); dB or a plan without
 * sym_b returns LADDER_ENOTSUP. */
ladder_status ladder_backward(ladder_plan_t plan, const double *B, const double *tau,
                              const double *W, double *dtau, double *dB, void *stream);

/* Closed-shell RI-CCSD (Sec. II.A): the CCSD amplitude equations for a
 * canonical Hartree-Fock reference (orbital energies e_occ, e_vir) with the
 * integrals of the RI factors B [naux][v][v], Bov [naux][o][v] and Boo
 * [naux][o][o] (device, FP64), solved from zero amplitudes by Jacobi steps
 * with DIIS over the last ndiis iterates (0 <= ndiis <= 8; 0: plain
 * Jacobi).  Stops when the energy changes by less than tol and the step's
 * 2-norm is below 1000 tol, or after max_iter steps.  The particle-particle
 * ladder of every step is ladder_apply on `plan` (a single-molecule plan of
 * the same (o, v, naux) with its workspace set; its mode decides the ladder's
 * precision, LADDER_FP64 or LADDER_OZAKI for an FP64-class solution); every
 * other term runs in FP64.  The residual is the spin-orbital one (the
 * projections of exp(-T) H exp(T) with the one- and two-body intermediates
 * of Stanton, Gauss, Watts and Bartlett 1991) held by closed-shell spin
 * blocks (three spatial arrays per four-index tensor); the workspace holds
 * the spatial (pq|rs) over all o + v orbitals, (o+v)^4 doubles, and about
 * 9 o v^3 more: small and medium molecules (o <= 128, v <= 1024;
 * ladder_ccsd_workspace_size gives the bytes).  Outputs: t1
 * [o][v], t2 [o][o][v][v] (device), the correlation energy
 * sum_ijab (2 v_ab^ij - v_ba^ij)(t_ij^ab + t_i^a t_j^b) in *E (host) and the
 * steps taken in *iters (host); LADDER_ENONFINITE if the energy stops being
 * finite (a diverging iteration).  Synchronises `stream`. */
ladder_status ladder_ccsd_workspace_size(int o, int v, int naux, int ndiis, size_t *bytes);
ladder_status ladder_ccsd(ladder_plan_t plan, int o, int v, int naux, const double *B, const double *Bov,
                          const double *Boo, const double *e_occ, const double *e_vir, int max_iter,
                          double tol, int ndiis, double *t1, double *t2, double *E, int *iters,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Y_ij^ab = alpha X_ij^ab + beta X_ij^ba over [o][o][v][v] (device arrays,
 * Y may not alias X).  (2, -1) applied to t2 gives the energy weights
 * W = dE_L/dR; applied to R it gives dE_L/dt2 through the weights. */
ladder_status ladder_pair_combine(int o, int v, double alpha, double beta, const double *X,
                                  double *Y, void *stream);

/* Host-buffer convenience path: copies B and tau from host memory (pinned
 * memory recommended), runs the ladder as ladder_apply does (no energy), and
 * copies R back to R_host.  Needs device buffers d_B, d_tau, d_R of the
 * sizes above, supplied by the caller (d_R distinct from d_B and d_tau).  In
 * the error-free mode tau's upload and preparation run on a side stream of
 * the plan, overlapping B's upload and the first pass; the side stream is
 * joined into `stream` before R is copied back.  Synchronises `stream`
 * before return; LADDER_EWORKSPACE without a workspace. */
ladder_status ladder_apply_host(ladder_plan_t plan, const double *B_host, const double *tau_host,
                                double *R_host, double *d_B, double *d_tau, double *d_R,
                                void *stream);

/* Ragged batch: n molecules with their own (o_k, v_k, naux_k), one plan and one
 * workspace; mode LADDER_BF16X3, LADDER_BF16X6 or LADDER_OZAKI (else
 * LADDER_ENOTSUP).  BF16X3 / BF16X6: molecules whose occupied pairs fit one
 * chunk of the fused kernel run in one persistent fused launch over all their
 * work units, ordered by cost (largest first); molecules that need several
 * chunks take the two-pass form (see ladder_tuning) while their stored V+-
 * tiles fit 128 GiB in all, with one storing launch and one GEMM2 launch over
 * all of them.  LADDER_OZAKI: every molecule takes the error-free two-pass
 * form (five slices), one launch of each pass over all molecules' work units;
 * the stored slices of all molecules must fit 200 GiB (else LADDER_ENOTSUP).
 * A batched plan
 * serves only ladder_apply_batched and ladder_step_batched (the other calls
 * return LADDER_EINVAL);
 * ladder_energy_noalloc gives the energy of each molecule. */
ladder_status ladder_plan_batched(int n, const int *o, const int *v, const int *naux, int mode,
                                  ladder_plan_t *out);
/* Launch parameters of member m of a batch plan (0 <= m < n), before
 * ladder_set_workspace: kc, s_pieces, flush_every, xy_split and two_pass as in
 * ladder_tuning (ksplit is the plan's own; lambda_only must be 0).  A member
 * moved to the two-pass form must keep the batch's stored tiles within the
 * batch cap (else LADDER_ENOTSUP).  The autotuner's per-shape choices are
 * applied to a batch through this call.  A member of a LADDER_OZAKI batch
 * takes only sym_b (the other fields are ignored; 0 or 1, else
 * LADDER_EINVAL): 1 promises that member's B symmetric in a <-> c, and the
 * batch then forms its distinct integral tiles once and its V+- from them
 * (checked on the device as for a single plan).  Its distinct tiles count
 * toward the 200 GiB cap with the stored slices, and above 96 GiB for one
 * member the call returns LADDER_ENOTSUP.  The other modes return
 * LADDER_EINVAL for sym_b != 0. */
ladder_status ladder_set_member_tuning(ladder_plan_t plan, int m, const ladder_tuning *t);

/* B[k], tau[k], R[k] are device pointers for molecule k (host arrays of n
 * pointers).  The first call with a given set of pointers records the whole
 * batch (operand preparation of every molecule, the fused, storing and GEMM2
 * launches, the unpacks) as a CUDA graph on a private stream; it synchronises
 * `stream` and copies the per-molecule arguments into the workspace first.
 * Calls with the same pointers replay the graph on `stream` without
 * synchronising. */
ladder_status ladder_apply_batched(ladder_plan_t plan, const double *const *B,
                                   const double *const *tau, double *const *R, void *stream);

/* One whole step per molecule of a batch, in one CUDA graph:
 *   tau[k] = t2[k] + t1[k] (x) t1[k]                       (Eq. pp-Ladder-01)
 *   R[k]_ij^ab = sum_cd (ac|bd) tau[k]_ij^cd                (Eq. pp-Ladder-0)
 *   E[k] = sum_ijab R[k]_ij^ab (2 t2[k]_ij^ab - t2[k]_ij^ba)
 * B[k], t1[k] [o_k][v_k], t2[k], tau[k] (written), R[k] (written) are device
 * pointers for molecule k (host arrays of n pointers); E is a device array of
 * n doubles.  tau[k] may not alias t2[k].  As for ladder_apply_batched, the
 * first call with a set of pointers records the graph (synchronising
 * `stream`) and later calls with the same pointers replay it; the energies
 * use each member's share of the batch workspace for their partial sums. */
ladder_status ladder_step_batched(ladder_plan_t plan, const double *const *B, const double *const *t1,
                                  const double *const *t2, double *const *tau, double *const *R,
                                  double *E, void *stream);

/* Reads and clears the device status word (synchronises `stream`).
 * Returns LADDER_OK, LADDER_ETIMEOUT (a bounded wait ran out; *where receives
 * the site code of the first one) or LADDER_ENONFINITE (the slicing or packing
 * of B or tau met a NaN or an infinity, site code 50; the tensor-core modes and
 * LADDER_OZAKI check, the FP64 path lets them propagate into R) or
 * LADDER_EINVAL (a LADDER_OZAKI plan with sym_b met a B that is not
 * symmetric, site code 51; its R is then meaningless).  *where is 0 when
 * nothing was recorded. */
ladder_status ladder_last_device_error(ladder_plan_t plan, void *stream, int *where);

/* Self-test of the device-side failure detection: one kernel waits, with the
 * same bounded wait every pipelined kernel of the library uses, on a barrier
 * that nothing ever signals.  After timeout_ns the wait gives up, records site
 * code 99 in the plan's status word and the kernel returns, leaving the
 * context usable; ladder_last_device_error then reports LADDER_ETIMEOUT. */
ladder_status ladder_selftest_wait(ladder_plan_t plan, unsigned long long timeout_ns, void *stream);

/* Stage timing of ladder_apply.  With timing on, ladder_apply records CUDA
 * events on its stream around its three stages (operand preparation: slicing
 * and packing; the ladder kernels, fused or both passes; unpacking of R).  ladder_timing waits
 * for the events of the last ladder_apply and returns the three durations in
 * milliseconds (any pointer may be NULL).  Timing is off by default; the
 * events are created by ladder_set_timing (no device memory). */
ladder_status ladder_set_timing(ladder_plan_t plan, int on);
ladder_status ladder_timing(ladder_plan_t plan, float *prep_ms, float *fused_ms, float *unpack_ms);

/* The ladder kernels of the last ladder_apply split by pass (timing on): in
 * the two-pass form the storing GEMM1 pass and the GEMM2 pass; otherwise the
 * fused kernel and 0. */
ladder_status ladder_timing_passes(ladder_plan_t plan, float *pass1_ms, float *pass2_ms);
/* The last ladder_apply_dressed (waits for it): the B - mbar product and the
 * rank-o correction after the ladder.  LADDER_EINVAL if the plan has no
 * dressing or timing is off. */
ladder_status ladder_timing_dressing(ladder_plan_t plan, float *bd_ms, float *correction_ms);
/* The last ladder_apply of a LADDER_OZAKI plan with sym_b (timing on; waits
 * for it): the distinct integral tiles and the formation of V+- from them,
 * which together make up what ladder_timing_passes reports as pass 1.
 * LADDER_EINVAL if that call did not take the symmetric-B form in one range
 * or timing is off. */
ladder_status ladder_timing_sym(ladder_plan_t plan, float *xsym_ms, float *form_ms);

/* Algorithmic flop count of one ladder_apply (two flops per multiply-add of
 * the symmetric/antisymmetric scheme; identical for every mode). */
double ladder_flops(ladder_plan_t plan);

const char *ladder_status_string(ladder_status s);

void ladder_destroy(ladder_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* LADDER_H */
