"""Plain FP64 CPU oracle for the closed-shell RI-CCSD iteration of Sec. II.A.

TEST INFRASTRUCTURE ONLY: the tests may import this module; the product
library never does.  It shares no code with the CUDA path.

Sec. II.A takes the spin-adapted closed-shell CCSD of the literature, solved
by Jacobi iteration accelerated with DIIS over a few stored iterates (three
in the paper's practice, Sec. II.B), and prints the closed-shell correlation
energy
    E_CCSD = sum_ijab (2 v_ab^ij - v_ba^ij)(t_ij^ab + t_i^a t_j^b),
but not the amplitude equations.  This module solves the CCSD amplitude
equations in their spin-orbital form (the projections <Phi_i^a| and
<Phi_ij^ab| of exp(-T) H exp(T) onto the reference, organised with the
intermediates of Stanton, Gauss, Watts and Bartlett, J. Chem. Phys. 94, 4334
(1991)) on the integrals the RI factors give, (pq|rs) = sum_P B^P_pq B^P_rs,
with a canonical Hartree-Fock reference (diagonal Fock matrix of the orbital
energies).  Any spin adaptation solves the same equations, so the closed-shell
amplitudes are read off the spin-orbital ones:
    t_i^a = t_{i alpha}^{a alpha},  t_ij^ab = t_{i alpha j beta}^{a alpha b beta}.
Spin orbitals make the arrays 16 times larger, so the module is for small
systems.  Parity is pinned by tests/test_oracle_ccsd_pins.py against what
the theory fixes: CCSD is exact (full CI) for two electrons, it is size
extensive, its first Jacobi step from zero amplitudes gives MP2, and its
energy matches the closed-shell formula above.

Functions:
  full_factors       B^P_pq over all orbitals from the oo, ov and vv blocks
  so_integrals       antisymmetrised spin-orbital integrals <pq||rs>
  residuals          the CCSD amplitude equations' residuals (spin orbitals)
  energy_so          the CCSD energy from spin-orbital amplitudes
  ccsd               Jacobi iteration with DIIS; closed-shell t1, t2 and E
  closed_shell_energy  the energy formula of Sec. II.A
  fci_two_electron   the exact energy of two electrons (full CI, singlet)
"""
from __future__ import annotations

import numpy as np


def full_factors(B_vv, B_ov, B_oo):
    """B^P_pq for p, q over the o occupied then v virtual orbitals."""
    N, o, v = B_ov.shape
    Bf = np.zeros((N, o + v, o + v))
    Bf[:, :o, :o] = B_oo
    Bf[:, :o, o:] = B_ov
    Bf[:, o:, :o] = B_ov.transpose(0, 2, 1)
    Bf[:, o:, o:] = B_vv
    return Bf


def _spin_maps(o, v):
    """Spatial orbital and spin of each spin orbital; occupied first, then
    virtual, each spatial orbital as (alpha, beta)."""
    orb = np.array([p // 2 for p in range(2 * o)] + [o + q // 2 for q in range(2 * v)])
    spin = np.array([p % 2 for p in range(2 * (o + v))])
    return orb, spin


def so_integrals(Bf, o):
    """<pq||rs> = <pq|rs> - <pq|sr> with <pq|rs> = (pr|qs) times the two spin
    deltas, (pr|qs) = sum_P B^P_pr B^P_qs (chemists' notation)."""
    n = Bf.shape[1]
    v = n - o
    eri = np.einsum("Ppq,Prs->pqrs", Bf, Bf)
    orb, spin = _spin_maps(o, v)
    same = (spin[:, None] == spin[None, :]).astype(float)
    # <PQ|RS> = (p r | q s) delta(sP, sR) delta(sQ, sS)
    phys = eri[np.ix_(orb, orb, orb, orb)].transpose(0, 2, 1, 3)
    phys = phys * same[:, None, :, None] * same[None, :, None, :]
    return phys - phys.transpose(0, 1, 3, 2)


def _P(x, a, b):
    """P(ab) X = X - X with axes a and b exchanged."""
    return x - np.swapaxes(x, a, b)


def residuals(t1, t2, g, eps, no):
    """The CCSD amplitude equations as residuals r1, r2 (zero at the
    solution); the Jacobi step is t += r / D with D_ia = e_i - e_a and
    D_ijab = e_i + e_j - e_a - e_b.  Canonical reference: f = diag(eps)."""
    O, V = slice(0, no), slice(no, g.shape[0])
    eo, ev = eps[O], eps[V]
    f_ov = np.zeros_like(t1)
    oooo, ooov, oovv = g[O, O, O, O], g[O, O, O, V], g[O, O, V, V]
    ovvv, vovv, ovov = g[O, V, V, V], g[V, O, V, V], g[O, V, O, V]
    oovo, ovvo, vvvo, ovoo = g[O, O, V, O], g[O, V, V, O], g[V, V, V, O], g[O, V, O, O]
    vvvv = g[V, V, V, V]
    tt = np.einsum("ia,jb->ijab", t1, t1)
    tau_t = t2 + 0.5 * (tt - tt.transpose(0, 1, 3, 2))
    tau = t2 + tt - tt.transpose(0, 1, 3, 2)
    # one-body intermediates (diagonal Fock parts excluded)
    Fae = (-0.5 * np.einsum("me,ma->ae", f_ov, t1) + np.einsum("mf,mafe->ae", t1, ovvv)
           - 0.5 * np.einsum("mnaf,mnef->ae", tau_t, oovv))
    Fmi = (0.5 * np.einsum("ie,me->mi", t1, f_ov) + np.einsum("ne,mnie->mi", t1, ooov)
           + 0.5 * np.einsum("inef,mnef->mi", tau_t, oovv))
    Fme = f_ov + np.einsum("nf,mnef->me", t1, oovv)
    # two-body intermediates
    Wmnij = (oooo + _P(np.einsum("je,mnie->mnij", t1, ooov), 2, 3)
             + 0.25 * np.einsum("ijef,mnef->mnij", tau, oovv))
    Wabef = (vvvv - _P(np.einsum("mb,amef->abef", t1, vovv), 0, 1)
             + 0.25 * np.einsum("mnab,mnef->abef", tau, oovv))
    Wmbej = (ovvo + np.einsum("jf,mbef->mbej", t1, ovvv) - np.einsum("nb,mnej->mbej", t1, oovo)
             - np.einsum("jnfb,mnef->mbej", 0.5 * t2 + np.einsum("jf,nb->jnfb", t1, t1), oovv))
    # singles
    rhs1 = (f_ov + np.einsum("ie,ae->ia", t1, Fae) - np.einsum("ma,mi->ia", t1, Fmi)
            + np.einsum("imae,me->ia", t2, Fme) - np.einsum("nf,naif->ia", t1, ovov)
            - 0.5 * np.einsum("imef,maef->ia", t2, ovvv) - 0.5 * np.einsum("mnae,nmei->ia", t2, oovo))
    # doubles
    Fbe = Fae - 0.5 * np.einsum("mb,me->be", t1, Fme)
    Fmj = Fmi + 0.5 * np.einsum("je,me->mj", t1, Fme)
    ring = np.einsum("imae,mbej->ijab", t2, Wmbej) - np.einsum("ie,ma,mbej->ijab", t1, t1, ovvo)
    rhs2 = (oovv + _P(np.einsum("ijae,be->ijab", t2, Fbe), 2, 3)
            - _P(np.einsum("imab,mj->ijab", t2, Fmj), 0, 1)
            + 0.5 * np.einsum("mnab,mnij->ijab", tau, Wmnij)
            + 0.5 * np.einsum("ijef,abef->ijab", tau, Wabef)
            + _P(_P(ring, 0, 1), 2, 3)
            + _P(np.einsum("ie,abej->ijab", t1, vvvo), 0, 1)
            - _P(np.einsum("ma,mbij->ijab", t1, ovoo), 2, 3))
    D1 = eo[:, None] - ev[None, :]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return rhs1 - D1 * t1, rhs2 - D2 * t2, D1, D2


def energy_so(t1, t2, g, no):
    """E = sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b
    (f_ia = 0 for the canonical reference)."""
    O, V = slice(0, no), slice(no, g.shape[0])
    oovv = g[O, O, V, V]
    return float(0.25 * np.einsum("ijab,ijab->", oovv, t2) + 0.5 * np.einsum("ijab,ia,jb->", oovv, t1, t1))


def closed_shell_energy(Bf, o, t1, t2):
    """E_CCSD = sum_ijab (2 v_ab^ij - v_ba^ij)(t_ij^ab + t_i^a t_j^b),
    v_ab^ij = (ia|jb) (Sec. II.A)."""
    Bov = Bf[:, :o, o:]
    v_ = np.einsum("Pia,Pjb->ijab", Bov, Bov)
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    return float(np.sum((2.0 * v_ - v_.transpose(0, 1, 3, 2)) * tau))


def _diis(vecs, errs):
    """Extrapolated vector sum c_k vecs[k] with sum c_k = 1 minimising the
    extrapolated error (Pulay's DIIS, the least-squares system with a
    Lagrange multiplier)."""
    m = len(vecs)
    Bm = np.empty((m + 1, m + 1))
    Bm[-1, :] = Bm[:, -1] = -1.0
    Bm[-1, -1] = 0.0
    for x in range(m):
        for y in range(m):
            Bm[x, y] = float(np.dot(errs[x], errs[y]))
    rhs = np.zeros(m + 1)
    rhs[-1] = -1.0
    c = np.linalg.solve(Bm, rhs)[:m]
    return sum(ck * vk for ck, vk in zip(c, vecs))


def ccsd(Bf, e_occ, e_vir, *, tol=1e-11, max_iter=200, diis=3, iters=None):
    """Jacobi iteration with DIIS over `diis` stored iterates (0: plain
    Jacobi) from zero amplitudes.  Returns the closed-shell t1 [o][v],
    t2 [o][o][v][v], the energy and the energies of the iterates.  With
    `iters` set, exactly that many steps are taken (no convergence test)."""
    o, v = len(e_occ), len(e_vir)
    g = so_integrals(Bf, o)
    eps = np.concatenate([np.repeat(e_occ, 2), np.repeat(e_vir, 2)])
    no = 2 * o
    t1 = np.zeros((2 * o, 2 * v))
    t2 = np.zeros((2 * o, 2 * o, 2 * v, 2 * v))
    hist_v, hist_e, energies = [], [], []
    E = 0.0
    for it in range(max_iter if iters is None else iters):
        r1, r2, D1, D2 = residuals(t1, t2, g, eps, no)
        t1n, t2n = t1 + r1 / D1, t2 + r2 / D2
        if diis:
            vec = np.concatenate([t1n.ravel(), t2n.ravel()])
            err = np.concatenate([(t1n - t1).ravel(), (t2n - t2).ravel()])
            hist_v.append(vec)
            hist_e.append(err)
            hist_v, hist_e = hist_v[-diis:], hist_e[-diis:]
            if len(hist_v) > 1:
                vec = _diis(hist_v, hist_e)
                t1n = vec[:t1.size].reshape(t1.shape)
                t2n = vec[t1.size:].reshape(t2.shape)
        t1, t2 = t1n, t2n
        En = energy_so(t1, t2, g, no)
        energies.append(En)
        done = iters is None and abs(En - E) < tol and max(np.abs(r1).max(), np.abs(r2).max()) < 1e3 * tol
        E = En
        if done:
            break
    return t1[0::2, 0::2].copy(), t2[0::2, 1::2, 0::2, 1::2].copy(), E, energies


def fci_two_electron(Bf, e_occ, e_vir):
    """Exact ground-state correlation energy of two electrons in o = 1
    doubly occupied orbital and the virtual orbitals: the lowest eigenvalue
    of the Hamiltonian on spatially symmetric two-electron functions (the
    singlets) minus the reference energy.  The one-electron integrals follow
    from the canonical Fock matrix: h_pq = f_pq - [2 (pq|00) - (p0|0q)]."""
    assert len(e_occ) == 1
    n = Bf.shape[1]
    eri = np.einsum("Ppq,Prs->pqrs", Bf, Bf)
    f = np.diag(np.concatenate([e_occ, e_vir]))
    h = f - (2.0 * eri[:, :, 0, 0] - eri[:, 0, 0, :])
    # H on product functions |pq> = phi_p(1) phi_q(2)
    I = np.eye(n)
    H = (np.einsum("pr,qs->pqrs", h, I) + np.einsum("pr,qs->pqrs", I, h)
         + eri.transpose(0, 2, 1, 3)).reshape(n * n, n * n)
    # orthonormal basis of the symmetric subspace
    cols = []
    for p in range(n):
        for q in range(p, n):
            c = np.zeros((n, n))
            c[p, q] += 1.0
            c[q, p] += 1.0
            cols.append(c.ravel() / np.linalg.norm(c))
    S = np.array(cols).T
    E0 = np.linalg.eigvalsh(S.T @ H @ S)[0]
    E_ref = h[0, 0] + f[0, 0]
    return float(E0 - E_ref)
