/*
 * Plain FP64 CPU oracle for the particle-particle ladder term.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Every routine is the definition written out with plain loops in double
 * precision, in the order the paper states it, with no blocking, no symmetry
 * shortcuts and no reordering beyond parallelising independent outputs.
 *
 * Notation (Sec. II): o = N_occ, v = N_vir, n = N_ABS (auxiliary functions).
 *   B   [n][v][v]      RI factor of the virtual block, B[P][a][c] = m^P_ac
 *   t1  [o][v]         singles t_i^a
 *   t2  [o][o][v][v]   doubles t_ij^ab
 *   tau [o][o][v][v]   tau_ij^ab
 *   R   [o][o][v][v]   ladder term L_ij^ab
 * All arrays are row-major (C order).
 */
#include <stddef.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX4(i, j, a, b, o, v) ((((size_t)(i) * (o) + (j)) * (v) + (a)) * (v) + (b))
#define IDX3(P, a, c, v) (((size_t)(P) * (v) + (a)) * (v) + (c))

/* Eq. pp-Ladder-01: tau_ij^ab = t_ij^ab + t_i^a t_j^b. */
void oracle_tau(int o, int v, const double *t1, const double *t2, double *tau)
{
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b)
                    tau[IDX4(i, j, a, b, o, v)] =
                        t2[IDX4(i, j, a, b, o, v)] + t1[(size_t)i * v + a] * t1[(size_t)j * v + b];
}

/* One (a,b) column of the integrals under the RI factorisation (Eq. RIM with
 * Eq. eri): V[c][d] = (ac|bd) = v^{ab}_{cd} = sum_P m^P_ac m^P_bd. */
static void integrals_ab(int v, int n, const double *B, int a, int b, double *V)
{
    memset(V, 0, sizeof(double) * (size_t)v * v);
    for (int P = 0; P < n; ++P)
        for (int c = 0; c < v; ++c) {
            const double bac = B[IDX3(P, a, c, v)];
            for (int d = 0; d < v; ++d)
                V[(size_t)c * v + d] += bac * B[IDX3(P, b, d, v)];
        }
}

/* Eq. pp-Ladder-0 with the undressed integrals b^{ab}_{cd} = v^{ab}_{cd}:
 * R_ij^ab = sum_{c,d} (ac|bd) tau_ij^cd, for every i, j, a, b. */
void oracle_ladder(int o, int v, int n, const double *B, const double *tau, double *R)
{
    #pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * (size_t)v * v);
        #pragma omp for schedule(dynamic)
        for (int ab = 0; ab < v * v; ++ab) {
            const int a = ab / v, b = ab % v;
            integrals_ab(v, n, B, a, b, V);
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += V[(size_t)c * v + d] * tau[IDX4(i, j, c, d, o, v)];
                    R[IDX4(i, j, a, b, o, v)] = s;
                }
        }
        free(V);
    }
}

/* The same result for a list of (a,b) columns only: Rsel[k][i][j] = R_ij^{a_k b_k}.
 * Used for sampled checks at sizes where the full term takes too long. */
void oracle_ladder_pairs(int o, int v, int n, const double *B, const double *tau,
                         int npairs, const int *pa, const int *pb, double *Rsel)
{
    #pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * (size_t)v * v);
        #pragma omp for schedule(dynamic)
        for (int k = 0; k < npairs; ++k) {
            integrals_ab(v, n, B, pa[k], pb[k], V);
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += V[(size_t)c * v + d] * tau[IDX4(i, j, c, d, o, v)];
                    Rsel[((size_t)k * o + i) * o + j] = s;
                }
        }
        free(V);
    }
}

/* Brute force: build the whole four-virtual integral array v^{ab}_{cd}
 * (Eq. eri under Eq. RIM) explicitly, then contract it with tau.  Only for
 * tiny v (the array has v^4 entries). */
int oracle_ladder_brute(int o, int v, int n, const double *B, const double *tau, double *R)
{
    const size_t v4 = (size_t)v * v * v * v;
    double *I = (double *)calloc(v4, sizeof(double)); /* I[a][b][c][d] = (ac|bd) */
    if (!I) return -1;
    for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
            for (int c = 0; c < v; ++c)
                for (int d = 0; d < v; ++d) {
                    double s = 0.0;
                    for (int P = 0; P < n; ++P)
                        s += B[IDX3(P, a, c, v)] * B[IDX3(P, b, d, v)];
                    I[IDX4(a, b, c, d, v, v)] = s;
                }
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += I[IDX4(a, b, c, d, v, v)] * tau[IDX4(i, j, c, d, o, v)];
                    R[IDX4(i, j, a, b, o, v)] = s;
                }
    free(I);
    return 0;
}

/* Ladder energy E_L = sum_ijab R_ij^ab (2 t_ij^ab - t_ij^ba): the
 * "twice direct minus exchange" weighting of the closed-shell CCSD energy
 * expression (Sec. II.A) applied to the ladder term. */
double oracle_energy(int o, int v, const double *R, const double *t2)
{
    /* The terms R_ij^ab (2 t_ij^ab - t_ij^ba) in index order, summed with
     * Neumaier's compensated summation: a plain running sum of o^2 v^2 terms
     * (1.85e8 at o = 34, v = 400) carries rounding errors of order
     * sqrt(n) eps |E_L|, several microhartree at E_L ~ 3e6, which is above
     * the energy bound the GPU path is held to; the compensated sum is
     * accurate to about eps |E_L| plus n eps^2 sum |terms|. */
    double s = 0.0, c = 0.0;
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b) {
                    const double x = R[IDX4(i, j, a, b, o, v)] *
                                     (2.0 * t2[IDX4(i, j, a, b, o, v)] - t2[IDX4(i, j, b, a, o, v)]);
                    const double t = s + x;
                    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
                    s = t;
                }
    return s + c;
}

/* Energy weights W_ij^ab = dE_L/dR_ij^ab = 2 t_ij^ab - t_ij^ba. */
void oracle_energy_weights(int o, int v, const double *t2, double *W)
{
    for (int i = 0; i < o; ++i)
        for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b)
                    W[IDX4(i, j, a, b, o, v)] =
                        2.0 * t2[IDX4(i, j, a, b, o, v)] - t2[IDX4(i, j, b, a, o, v)];
}

/* Gradient of E = sum_ijab W_ij^ab R_ij^ab with respect to tau, for fixed W:
 * dE/dtau_ij^cd = sum_ab W_ij^ab (ac|bd). */
void oracle_grad_tau(int o, int v, int n, const double *B, const double *W, double *dtau)
{
    const size_t total = (size_t)o * o * v * v;
    memset(dtau, 0, sizeof(double) * total);
    double *V = (double *)malloc(sizeof(double) * (size_t)v * v);
    /* Each (a,b) column adds W_ij^ab V[c][d] into every dtau_ij^cd.  The loop
     * over (a,b) stays serial so that the sum is taken in one fixed order. */
    for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b) {
            integrals_ab(v, n, B, a, b, V);
            #pragma omp parallel for
            for (int ij = 0; ij < o * o; ++ij) {
                const int i = ij / o, j = ij % o;
                const double w = W[IDX4(i, j, a, b, o, v)];
                for (int c = 0; c < v; ++c)
                    for (int d = 0; d < v; ++d)
                        dtau[IDX4(i, j, c, d, o, v)] += w * V[(size_t)c * v + d];
            }
        }
    free(V);
}

/* Gradient with respect to the RI factor, for fixed W and tau.  Each factor
 * m^P_xy enters (ac|bd) once as m^P_ac (a=x, c=y) and once as m^P_bd (b=x,
 * d=y):
 *   dE/dB[P][x][y] = sum_{ij,b,d} W_ij^{xb} tau_ij^{yd} B[P][b][d]
 *                  + sum_{ij,a,c} W_ij^{ax} tau_ij^{cy} B[P][a][c].
 * Both terms are evaluated as written; no symmetry of W or tau is assumed. */
void oracle_grad_B(int o, int v, int n, const double *B, const double *tau,
                   const double *W, double *dB)
{
    memset(dB, 0, sizeof(double) * (size_t)n * v * v);
    #pragma omp parallel
    {
        double *G = (double *)malloc(sizeof(double) * (size_t)v * v);
        #pragma omp for schedule(dynamic)
        for (int x = 0; x < v; ++x) {
            /* first term: for each b, G[y][d] = sum_ij W_ij^{xb} tau_ij^{yd} */
            for (int b = 0; b < v; ++b) {
                memset(G, 0, sizeof(double) * (size_t)v * v);
                for (int i = 0; i < o; ++i)
                    for (int j = 0; j < o; ++j) {
                        const double w = W[IDX4(i, j, x, b, o, v)];
                        for (int y = 0; y < v; ++y)
                            for (int d = 0; d < v; ++d)
                                G[(size_t)y * v + d] += w * tau[IDX4(i, j, y, d, o, v)];
                    }
                for (int P = 0; P < n; ++P)
                    for (int y = 0; y < v; ++y) {
                        double s = 0.0;
                        for (int d = 0; d < v; ++d)
                            s += G[(size_t)y * v + d] * B[IDX3(P, b, d, v)];
                        dB[IDX3(P, x, y, v)] += s;
                    }
            }
            /* second term: for each a, G[c][y] = sum_ij W_ij^{ax} tau_ij^{cy} */
            for (int a = 0; a < v; ++a) {
                memset(G, 0, sizeof(double) * (size_t)v * v);
                for (int i = 0; i < o; ++i)
                    for (int j = 0; j < o; ++j) {
                        const double w = W[IDX4(i, j, a, x, o, v)];
                        for (int c = 0; c < v; ++c)
                            for (int y = 0; y < v; ++y)
                                G[(size_t)c * v + y] += w * tau[IDX4(i, j, c, y, o, v)];
                    }
                for (int P = 0; P < n; ++P)
                    for (int y = 0; y < v; ++y) {
                        double s = 0.0;
                        for (int c = 0; c < v; ++c)
                            s += G[(size_t)c * v + y] * B[IDX3(P, a, c, v)];
                        dB[IDX3(P, x, y, v)] += s;
                    }
            }
        }
        free(G);
    }
}

/* Selected entries of dE/dtau: out[k] = sum_ab W_{i_k j_k}^{ab} (a c_k | b d_k). */
void oracle_grad_tau_entries(int o, int v, int n, const double *B, const double *W,
                             int m, const int *ei, const int *ej, const int *ec,
                             const int *ed, double *out)
{
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < m; ++k) {
        double s = 0.0;
        for (int a = 0; a < v; ++a)
            for (int b = 0; b < v; ++b) {
                double vint = 0.0;
                for (int P = 0; P < n; ++P)
                    vint += B[IDX3(P, a, ec[k], v)] * B[IDX3(P, b, ed[k], v)];
                s += W[IDX4(ei[k], ej[k], a, b, o, v)] * vint;
            }
        out[k] = s;
    }
}

/* Selected entries of dE/dB, both terms as in oracle_grad_B. */
void oracle_grad_B_entries(int o, int v, int n, const double *B, const double *tau,
                           const double *W, int m, const int *eP, const int *ex,
                           const int *ey, double *out)
{
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < m; ++k) {
        const int P = eP[k], x = ex[k], y = ey[k];
        double s = 0.0;
        for (int i = 0; i < o; ++i)
            for (int j = 0; j < o; ++j) {
                for (int b = 0; b < v; ++b) {
                    const double w = W[IDX4(i, j, x, b, o, v)];
                    double t = 0.0;
                    for (int d = 0; d < v; ++d)
                        t += tau[IDX4(i, j, y, d, o, v)] * B[IDX3(P, b, d, v)];
                    s += w * t;
                }
                for (int a = 0; a < v; ++a) {
                    const double w = W[IDX4(i, j, a, x, o, v)];
                    double t = 0.0;
                    for (int c = 0; c < v; ++c)
                        t += tau[IDX4(i, j, c, y, o, v)] * B[IDX3(P, a, c, v)];
                    s += w * t;
                }
            }
        out[k] = s;
    }
}

/* ---------------------------------------------------------------------------
 * t1-dressed ladder (Eq. pp-Ladder-0 with the dressed integrals of
 * Eq. pp-Ladder-2 and the intermediate of Eq. pp-Ladder-21):
 *
 *   mbar^P_bd      = sum_k m^P_kd t_k^b                                (Eq. pp-Ladder-21)
 *   b^{ab}_{cd}    = sum_P m^P_ac (m^P_bd - mbar^P_bd) - sum_k t_k^a v^{kb}_{cd}   (Eq. pp-Ladder-2)
 *   R_ij^ab        = sum_cd b^{ab}_{cd} tau_ij^cd                      (Eq. pp-Ladder-0)
 *
 * with m^P_pq the RI factor of the orbital pair (p,q): the virtual block
 * B[P][a][c] and the occupied-virtual block Bov[P][k][c].  The integrals with
 * one occupied index, v^{kb}_{cd} = (kc|bd), come from the same factors
 * (Eq. RIM with Eq. eri): the paper keeps them pre-stored, built from the one
 * RI tensor before the iterations.
 *
 * Extra arrays: Bov [n][o][v], t1 [o][v].
 * ------------------------------------------------------------------------- */
#define IDX3O(P, k, c, o, v) (((size_t)(P) * (o) + (k)) * (v) + (c))

/* Eq. pp-Ladder-21: mbar[P][b][d] = sum_k Bov[P][k][d] t1[k][b]. */
static void dressed_mbar(int o, int v, int n, const double *Bov, const double *t1, double *mbar)
{
    #pragma omp parallel for schedule(static)
    for (int P = 0; P < n; ++P)
        for (int b = 0; b < v; ++b)
            for (int d = 0; d < v; ++d) {
                double s = 0.0;
                for (int k = 0; k < o; ++k)
                    s += Bov[IDX3O(P, k, d, o, v)] * t1[(size_t)k * v + b];
                mbar[IDX3(P, b, d, v)] = s;
            }
}

/* One (a,b) column of b^{ab}_{cd} (Eq. pp-Ladder-2) into V[c][d].  With
 * ovvv != NULL the pre-stored v^{kb}_{cd} = ovvv[k][c][b][d] is used,
 * otherwise it is formed from the factors for this b. */
static void dressed_integrals_ab(int o, int v, int n, const double *B, const double *Bov,
                                 const double *t1, const double *mbar, const double *ovvv,
                                 int a, int b, double *V)
{
    memset(V, 0, sizeof(double) * (size_t)v * v);
    for (int P = 0; P < n; ++P)
        for (int c = 0; c < v; ++c) {
            const double mac = B[IDX3(P, a, c, v)];
            for (int d = 0; d < v; ++d)
                V[(size_t)c * v + d] += mac * (B[IDX3(P, b, d, v)] - mbar[IDX3(P, b, d, v)]);
        }
    for (int k = 0; k < o; ++k) {
        const double tka = t1[(size_t)k * v + a];
        for (int c = 0; c < v; ++c)
            for (int d = 0; d < v; ++d) {
                double vkb;
                if (ovvv) {
                    vkb = ovvv[(((size_t)k * v + c) * v + b) * v + d];
                } else {
                    vkb = 0.0;
                    for (int P = 0; P < n; ++P)
                        vkb += Bov[IDX3O(P, k, c, o, v)] * B[IDX3(P, b, d, v)];
                }
                V[(size_t)c * v + d] -= tka * vkb;
            }
    }
}

/* The dressed term for every i, j, a, b.  Returns -1 if the pre-stored
 * integrals (o v^3 doubles) cannot be allocated. */
int oracle_ladder_dressed(int o, int v, int n, const double *B, const double *Bov,
                          const double *t1, const double *tau, double *R)
{
    double *mbar = (double *)malloc(sizeof(double) * (size_t)n * v * v);
    double *ovvv = (double *)malloc(sizeof(double) * (size_t)o * v * v * v);
    if (!mbar || !ovvv) { free(mbar); free(ovvv); return -1; }
    dressed_mbar(o, v, n, Bov, t1, mbar);
    /* v^{kb}_{cd} = (kc|bd) = sum_P m^P_kc m^P_bd, stored as ovvv[k][c][b][d] */
    #pragma omp parallel for schedule(dynamic)
    for (int kc = 0; kc < o * v; ++kc) {
        const int k = kc / v, c = kc % v;
        for (int b = 0; b < v; ++b)
            for (int d = 0; d < v; ++d) {
                double s = 0.0;
                for (int P = 0; P < n; ++P)
                    s += Bov[IDX3O(P, k, c, o, v)] * B[IDX3(P, b, d, v)];
                ovvv[(((size_t)k * v + c) * v + b) * v + d] = s;
            }
    }
    #pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * (size_t)v * v);
        #pragma omp for schedule(dynamic)
        for (int ab = 0; ab < v * v; ++ab) {
            const int a = ab / v, b = ab % v;
            dressed_integrals_ab(o, v, n, B, Bov, t1, mbar, ovvv, a, b, V);
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += V[(size_t)c * v + d] * tau[IDX4(i, j, c, d, o, v)];
                    R[IDX4(i, j, a, b, o, v)] = s;
                }
        }
        free(V);
    }
    free(ovvv);
    free(mbar);
    return 0;
}

/* Selected (a,b) columns of the dressed term: Rsel[k][i][j] = R_ij^{a_k b_k},
 * forming v^{kb}_{cd} for each selected b instead of storing all of them. */
int oracle_ladder_dressed_pairs(int o, int v, int n, const double *B, const double *Bov,
                                const double *t1, const double *tau, int npairs,
                                const int *pa, const int *pb, double *Rsel)
{
    double *mbar = (double *)malloc(sizeof(double) * (size_t)n * v * v);
    if (!mbar) return -1;
    dressed_mbar(o, v, n, Bov, t1, mbar);
    #pragma omp parallel
    {
        double *V = (double *)malloc(sizeof(double) * (size_t)v * v);
        #pragma omp for schedule(dynamic)
        for (int q = 0; q < npairs; ++q) {
            dressed_integrals_ab(o, v, n, B, Bov, t1, mbar, NULL, pa[q], pb[q], V);
            for (int i = 0; i < o; ++i)
                for (int j = 0; j < o; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < v; ++c)
                        for (int d = 0; d < v; ++d)
                            s += V[(size_t)c * v + d] * tau[IDX4(i, j, c, d, o, v)];
                    Rsel[((size_t)q * o + i) * o + j] = s;
                }
        }
        free(V);
    }
    free(mbar);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Perturbative triples, closed shell (Sec. II.A, the (T) energy):
 *
 *   E(T) = sum_ijk sum_abc (4 W_ijk^abc + W_ijk^bca + W_ijk^cab)
 *                          (V_ijk^abc - V_ijk^cba) / (3 D_ijk^abc)
 *   W_ijk^abc = P_ijk^abc ( sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab )
 *   V_ijk^abc = W_ijk^abc + v_jk^bc t_i^a + v_ik^ac t_j^b + v_ij^ab t_k^c
 *   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c
 *
 * with P_ijk^abc f(ijk,abc) = f(ijk,abc) + f(ikj,acb) + f(kij,cab) +
 * f(kji,cba) + f(jki,bca) + f(jik,bac), and the integrals v^{pq}_{rs} =
 * (pr|qs) = sum_P m^P_pr m^P_qs (Eq. eri under Eq. RIM) from the RI factors
 * of the orbital pairs: Bvv[P][a][c] = m^P_ac, Bov[P][i][a] = m^P_ia = m^P_ai
 * (real orbitals), Boo[P][k][l] = m^P_kl.  The three kinds used:
 *   v_di^ba = (bd|ai),  v_kl^cj = (ck|jl),  v_jk^bc = (bj|ck).
 * Extra arrays: Boo [n][o][o], e_occ [o], e_vir [v].
 * ------------------------------------------------------------------------- */
#define IDX3OO(P, k, l, o) (((size_t)(P) * (o) + (k)) * (o) + (l))

typedef struct {
    int o, v;
    double *ovvv;  /* [i][d][b][a] = v_di^ba = (bd|ai) */
    double *ooov;  /* [k][l][c][j] = v_kl^cj = (ck|jl) */
    double *oovv;  /* [j][k][b][c] = v_jk^bc = (bj|ck) */
} TriplesInts;

static int triples_integrals(int o, int v, int n, const double *Bvv, const double *Bov,
                             const double *Boo, TriplesInts *I)
{
    I->o = o;
    I->v = v;
    I->ovvv = (double *)malloc(sizeof(double) * (size_t)o * v * v * v);
    I->ooov = (double *)malloc(sizeof(double) * (size_t)o * o * o * v);
    I->oovv = (double *)malloc(sizeof(double) * (size_t)o * o * v * v);
    if (!I->ovvv || !I->ooov || !I->oovv) return -1;
    #pragma omp parallel for schedule(dynamic)
    for (int id = 0; id < o * v; ++id) {
        const int i = id / v, d = id % v;
        for (int b = 0; b < v; ++b)
            for (int a = 0; a < v; ++a) {
                double s = 0.0;
                for (int P = 0; P < n; ++P)
                    s += Bvv[IDX3(P, b, d, v)] * Bov[IDX3O(P, i, a, o, v)];
                I->ovvv[(((size_t)i * v + d) * v + b) * v + a] = s;
            }
    }
    for (int k = 0; k < o; ++k)
        for (int l = 0; l < o; ++l)
            for (int c = 0; c < v; ++c)
                for (int j = 0; j < o; ++j) {
                    double s = 0.0;
                    for (int P = 0; P < n; ++P)
                        s += Bov[IDX3O(P, k, c, o, v)] * Boo[IDX3OO(P, j, l, o)];
                    I->ooov[(((size_t)k * o + l) * v + c) * o + j] = s;
                }
    for (int j = 0; j < o; ++j)
        for (int k = 0; k < o; ++k)
            for (int b = 0; b < v; ++b)
                for (int c = 0; c < v; ++c) {
                    double s = 0.0;
                    for (int P = 0; P < n; ++P)
                        s += Bov[IDX3O(P, j, b, o, v)] * Bov[IDX3O(P, k, c, o, v)];
                    I->oovv[(((size_t)j * o + k) * v + b) * v + c] = s;
                }
    return 0;
}

static void triples_free(TriplesInts *I)
{
    free(I->ovvv);
    free(I->ooov);
    free(I->oovv);
}

/* The unsymmetrised term sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab. */
static double triples_raw(const TriplesInts *I, const double *t2, int i, int j, int k, int a,
                          int b, int c)
{
    const int o = I->o, v = I->v;
    double s = 0.0;
    for (int d = 0; d < v; ++d)
        s += I->ovvv[(((size_t)i * v + d) * v + b) * v + a] * t2[IDX4(k, j, c, d, o, v)];
    for (int l = 0; l < o; ++l)
        s -= I->ooov[(((size_t)k * o + l) * v + c) * o + j] * t2[IDX4(i, l, a, b, o, v)];
    return s;
}

/* W_ijk^abc and V_ijk^abc for one (i,j,k), every (a,b,c): W[a][b][c], V[a][b][c]. */
static void triples_wv(const TriplesInts *I, const double *t1, const double *t2, int i, int j,
                       int k, double *W, double *V)
{
    const int o = I->o, v = I->v;
    for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
            for (int c = 0; c < v; ++c) {
                const double w = triples_raw(I, t2, i, j, k, a, b, c) +
                                 triples_raw(I, t2, i, k, j, a, c, b) +
                                 triples_raw(I, t2, k, i, j, c, a, b) +
                                 triples_raw(I, t2, k, j, i, c, b, a) +
                                 triples_raw(I, t2, j, k, i, b, c, a) +
                                 triples_raw(I, t2, j, i, k, b, a, c);
                const size_t e = ((size_t)a * v + b) * v + c;
                W[e] = w;
                V[e] = w + I->oovv[(((size_t)j * o + k) * v + b) * v + c] * t1[(size_t)i * v + a] +
                       I->oovv[(((size_t)i * o + k) * v + a) * v + c] * t1[(size_t)j * v + b] +
                       I->oovv[(((size_t)i * o + j) * v + a) * v + b] * t1[(size_t)k * v + c];
            }
}

/* W and V of one triple (i,j,k), for the tests.  Returns -1 on allocation failure. */
int oracle_triples_wv(int o, int v, int n, const double *Bvv, const double *Bov,
                      const double *Boo, const double *t1, const double *t2, int i, int j, int k,
                      double *W, double *V)
{
    TriplesInts I;
    if (triples_integrals(o, v, n, Bvv, Bov, Boo, &I) != 0) {
        triples_free(&I);
        return -1;
    }
    triples_wv(&I, t1, t2, i, j, k, W, V);
    triples_free(&I);
    return 0;
}

/* E(T); per-(i,j,k) sums in index order, the o^3 partial sums added with
 * Neumaier's compensated summation.  Returns NAN on allocation failure. */
double oracle_triples(int o, int v, int n, const double *Bvv, const double *Bov,
                      const double *Boo, const double *t1, const double *t2,
                      const double *e_occ, const double *e_vir)
{
    TriplesInts I;
    if (triples_integrals(o, v, n, Bvv, Bov, Boo, &I) != 0) {
        triples_free(&I);
        return NAN;
    }
    double *part = (double *)calloc((size_t)o * o * o, sizeof(double));
    int bad = part == NULL;
    #pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)v * v * v);
        double *V = (double *)malloc(sizeof(double) * (size_t)v * v * v);
        if (!W || !V) {
            #pragma omp atomic write
            bad = 1;
        }
        #pragma omp for schedule(dynamic)
        for (int ijk = 0; ijk < o * o * o; ++ijk) {
            if (bad) continue;
            const int i = ijk / (o * o), j = (ijk / o) % o, k = ijk % o;
            triples_wv(&I, t1, t2, i, j, k, W, V);
            double s = 0.0;
            for (int a = 0; a < v; ++a)
                for (int b = 0; b < v; ++b)
                    for (int c = 0; c < v; ++c) {
                        const double D = e_occ[i] + e_occ[j] + e_occ[k] - e_vir[a] - e_vir[b] - e_vir[c];
                        const double w = 4.0 * W[((size_t)a * v + b) * v + c] +
                                         W[((size_t)b * v + c) * v + a] + W[((size_t)c * v + a) * v + b];
                        const double y = V[((size_t)a * v + b) * v + c] - V[((size_t)c * v + b) * v + a];
                        s += w * y / (3.0 * D);
                    }
            part[ijk] = s;
        }
        free(W);
        free(V);
    }
    double s = 0.0, c = 0.0;
    if (!bad)
        for (int q = 0; q < o * o * o; ++q) {
            const double x = part[q], t = s + x;
            c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
            s = t;
        }
    free(part);
    triples_free(&I);
    return bad ? NAN : s + c;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
