"""Pins for the CCSD oracle (oracle/ccsd.py), from what the theory fixes
rather than from the oracle itself:
  - two electrons: CCSD is exact, so its energy equals full CI (the lowest
    singlet of the two-electron Hamiltonian, diagonalised directly);
  - size extensivity: two fragments with no integral between them (disjoint
    orbitals and auxiliary functions) give the sum of the fragments' energies,
    each a two-electron full CI;
  - the first Jacobi step from zero amplitudes is MP2,
    E = sum (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b);
  - the closed-shell energy formula of Sec. II.A equals the spin-orbital
    energy at the solution, and the amplitudes keep the pair symmetry.
No GPU."""
import numpy as np

import synthetic
from oracle import ccsd


def test_two_electrons_is_full_ci():
    for (v, n, seed) in ((6, 12, 3), (9, 20, 11)):
        x = synthetic.make_inputs(1, v, n, seed)
        Bf = ccsd.full_factors(x.B, x.B_ov, x.B_oo)
        _, _, E, _ = ccsd.ccsd(Bf, x.e_occ, x.e_vir, tol=1e-13)
        E_fci = ccsd.fci_two_electron(Bf, x.e_occ, x.e_vir)
        assert abs(E - E_fci) <= 1e-10 * abs(E_fci), (E, E_fci)


def test_size_extensive_two_fragments():
    xa = synthetic.make_inputs(1, 5, 10, 3)
    xb = synthetic.make_inputs(1, 4, 8, 4)
    Ba = ccsd.full_factors(xa.B, xa.B_ov, xa.B_oo)
    Bb = ccsd.full_factors(xb.B, xb.B_ov, xb.B_oo)
    # combined orbitals: occupied (a0, b0), virtual (A's, B's); disjoint aux
    n = 2 + 5 + 4
    ia = [0] + list(range(2, 7))
    ib = [1] + list(range(7, 11))
    Bf = np.zeros((18, n, n))
    Bf[np.ix_(range(10), ia, ia)] = Ba
    Bf[np.ix_(range(10, 18), ib, ib)] = Bb
    e_occ = np.array([xa.e_occ[0], xb.e_occ[0]])
    e_vir = np.concatenate([xa.e_vir, xb.e_vir])
    _, _, E, _ = ccsd.ccsd(Bf, e_occ, e_vir, tol=1e-13)
    Es = ccsd.fci_two_electron(Ba, xa.e_occ, xa.e_vir) + ccsd.fci_two_electron(Bb, xb.e_occ, xb.e_vir)
    assert abs(E - Es) <= 1e-10 * abs(Es), (E, Es)


def test_first_step_is_mp2():
    x = synthetic.make_inputs(3, 7, 14, 5)
    Bf = ccsd.full_factors(x.B, x.B_ov, x.B_oo)
    _, _, E1, _ = ccsd.ccsd(Bf, x.e_occ, x.e_vir, diis=0, iters=1)
    vv = np.einsum("Pia,Pjb->ijab", x.B_ov, x.B_ov)
    D = (x.e_occ[:, None, None, None] + x.e_occ[None, :, None, None] - x.e_vir[None, None, :, None]
         - x.e_vir[None, None, None, :])
    E_mp2 = float(np.sum(vv * (2.0 * vv - vv.transpose(0, 1, 3, 2)) / D))
    assert abs(E1 - E_mp2) <= 1e-13 * abs(E_mp2)


def test_closed_shell_energy_and_symmetry():
    x = synthetic.make_inputs(3, 7, 14, 5)
    Bf = ccsd.full_factors(x.B, x.B_ov, x.B_oo)
    t1, t2, E, Es = ccsd.ccsd(Bf, x.e_occ, x.e_vir, tol=1e-13)
    assert abs(ccsd.closed_shell_energy(Bf, 3, t1, t2) - E) <= 1e-12 * abs(E)
    assert np.abs(t2 - t2.transpose(1, 0, 3, 2)).max() <= 1e-12 * np.abs(t2).max()
    assert len(Es) < 100 and abs(Es[-1] - Es[-2]) < 1e-12
