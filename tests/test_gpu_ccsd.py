"""The closed-shell RI-CCSD iteration (Sec. II.A) on the GPU against the CPU
oracle (oracle/ccsd.py), whose pins (two-electron full CI, size
extensivity, MP2) sit in tests/test_oracle_ccsd_pins.py.

Both solve the same CCSD equations from zero amplitudes with DIIS over three
iterates; the converged energies agree to the convergence tolerance and the
amplitudes to its square root."""
import numpy as np
import pytest

import synthetic
from oracle import ccsd as occsd
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


SHAPES = [(1, 6, 12, 3), (2, 8, 20, 5), (3, 7, 14, 5), (4, 10, 24, 6), (5, 13, 30, 7)]


@pytest.mark.parametrize("mode", ["fp64", "ozaki"])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_ccsd_matches_oracle(lad, mode, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    Bf = occsd.full_factors(x.B, x.B_ov, x.B_oo)
    t1_o, t2_o, E_o, Es = occsd.ccsd(Bf, x.e_occ, x.e_vir, tol=1e-12)
    L = lad.Ladder(o, v, n, mode=mode)
    t1, t2, E, it = lad.ccsd(L, to_dev(x.B), to_dev(x.B_ov), to_dev(x.B_oo), to_dev(x.e_occ),
                             to_dev(x.e_vir), tol=1e-12, max_iter=200)
    L.check_device()
    t1, t2 = t1.cpu().numpy(), t2.cpu().numpy()
    e1 = np.abs(t1 - t1_o).max() / max(np.abs(t1_o).max(), 1e-300)
    e2 = np.abs(t2 - t2_o).max() / np.abs(t2_o).max()
    print("ccsd %s o=%d v=%d n=%d: E %.12e (oracle %.12e, %d / %d steps)  t1 %.1e  t2 %.1e" % (
        mode, o, v, n, E, E_o, it, len(Es), e1, e2))
    assert abs(E - E_o) <= 1e-10 * abs(E_o)
    assert e1 < 1e-7 and e2 < 1e-7
    # the closed-shell energy formula of Sec. II.A on the GPU amplitudes
    assert abs(occsd.closed_shell_energy(Bf, o, t1, t2) - E) <= 1e-10 * abs(E)
    if o == 1:
        # two electrons: CCSD is full CI
        assert abs(E - occsd.fci_two_electron(Bf, x.e_occ, x.e_vir)) <= 1e-10 * abs(E)


def test_ccsd_plain_jacobi_and_bad_arguments(lad):
    """Without DIIS the iteration reaches the same solution; a plan of
    another shape is refused."""
    o, v, n, seed = 3, 7, 14, 5
    x = synthetic.make_inputs(o, v, n, seed)
    Bf = occsd.full_factors(x.B, x.B_ov, x.B_oo)
    _, _, E_o, _ = occsd.ccsd(Bf, x.e_occ, x.e_vir, tol=1e-12)
    L = lad.Ladder(o, v, n, mode="fp64")
    args = (to_dev(x.B), to_dev(x.B_ov), to_dev(x.B_oo), to_dev(x.e_occ), to_dev(x.e_vir))
    _, _, E, it = lad.ccsd(L, *args, tol=1e-12, max_iter=500, ndiis=0)
    _, _, E3, it3 = lad.ccsd(L, *args, tol=1e-12, max_iter=500, ndiis=3)
    print("plain Jacobi %d steps, DIIS(3) %d steps" % (it, it3))
    assert abs(E - E_o) <= 1e-10 * abs(E_o) and abs(E3 - E_o) <= 1e-10 * abs(E_o)
    assert it3 < it
    L2 = lad.Ladder(o, v + 1, n, mode="fp64")
    with pytest.raises(lad.LadderError):
        lad.ccsd(L2, *args)
