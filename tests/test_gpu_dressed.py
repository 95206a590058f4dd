"""Parity of the t1-dressed ladder (Eq. pp-Ladder-2 with Eq. pp-Ladder-21)
with the CPU oracle, through ladder_apply_dressed.

The library evaluates the undressed ladder of B - mbar in the plan's mode and
subtracts the rank-o correction sum_kl t_k^a t_l^b sum_cd (kc|ld) tau_ij^cd
(FP64 for LADDER_FP64, double-single FP32 for the error-free mode, FP32
otherwise); the oracle
follows Eq. pp-Ladder-2 term by term.  Tolerances on the relative Frobenius
error of R are those of the undressed term: FP64 1e-12, the error-free split
1e-10, BF16X6 1e-6, BF16X3 2e-5.
"""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, run_dressed, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki": 1e-10, "bf16x3": 2e-5, "bf16x6": 1e-6}

SHAPES = [
    (1, 5, 3, 11),       # one occupied orbital, v below one block
    (4, 24, 96, 0),      # smallest workload
    (5, 17, 33, 12),     # ragged v and N
    (7, 41, 70, 14),     # several tiles, ragged tail
    (12, 140, 150, 21),  # (kc|ld) over two 128-row tiles, ragged everywhere
]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode", ["fp64", "ozaki", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_dressed_matches_oracle(lad, mode, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode=mode, dressed=True)
    tau_g, R_g, E_g = run_dressed(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    assert rel_err(tau_g, tau_o) < 1e-15
    R_o = oracle.ladder_dressed(x.B, x.B_ov, x.t1, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    err = rel_err(R_g, R_o)
    print("dressed %s o=%d v=%d n=%d: rel-F %.3e  |dE| %.3e  E %.6e" % (mode, o, v, n, err,
                                                                      abs(E_g - E_o), E_o))
    assert err < TOL[mode]
    if mode in ("fp64", "ozaki"):
        assert abs(E_g - E_o) <= 1e-6


@pytest.mark.parametrize("mode", ["fp64", "ozaki", "bf16x6"])
def test_dressed_dimer(lad, mode):
    """The water-dimer-sized workload (o=10, v=120, N_aux=480), every element."""
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode=mode, dressed=True)
    _, R_g, E_g = run_dressed(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder_dressed(x.B, x.B_ov, x.t1, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    err = rel_err(R_g, R_o)
    print("dressed dimer %s: rel-F %.3e  |dE| %.3e  E %.9f" % (mode, err, abs(E_g - E_o), E_o))
    assert err < TOL[mode]
    if mode == "fp64":
        assert abs(E_g - E_o) <= 1e-6


@pytest.mark.parametrize("mode", ["fp64", "bf16x6"])
def test_dressed_sampled_columns_grad_size(lad, mode):
    """o=16, v=200, N_aux=800: sampled (a,b) columns against the oracle's
    per-column evaluation, including the last virtual index."""
    w = synthetic.WORKLOADS["grad_o16_v200_n800"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode=mode, dressed=True)
    _, R_g, _ = run_dressed(L, x)
    rng = np.random.default_rng(1)
    pa = np.r_[0, w.v - 1, rng.integers(0, w.v, 8)]
    pb = np.r_[w.v - 1, w.v - 1, rng.integers(0, w.v, 8)]
    tau_o = oracle.tau(x.t1, x.t2)
    cols = oracle.ladder_dressed_pairs(x.B, x.B_ov, x.t1, tau_o, pa, pb)
    got = np.stack([R_g[:, :, a, b] for a, b in zip(pa, pb)])
    err = rel_err(got, cols)
    print("dressed grad-size %s sampled columns: rel-F %.3e" % (mode, err))
    assert err < TOL[mode]


@pytest.mark.parametrize("mode", ["fp64", "bf16x6"])
def test_dressed_without_singles_is_the_undressed_term(lad, mode):
    """t1 = 0: mbar = 0 and the correction vanishes, so the dressed call
    returns the undressed ladder_apply result bit for bit."""
    import torch
    x = synthetic.make_inputs(7, 41, 70, 14)
    L = lad.Ladder(7, 41, 70, mode=mode, dressed=True)
    t1 = torch.zeros_like(to_dev(x.t1))
    tau = L.tau(t1, to_dev(x.t2))
    B, Bov = to_dev(x.B), to_dev(x.B_ov)
    R_d = L.apply_dressed(B, Bov, t1, tau)
    R_u = L.apply(B, tau)
    torch.cuda.synchronize()
    assert torch.equal(R_d, R_u)


def test_dressed_needs_the_plan_flag(lad):
    import torch
    x = synthetic.make_inputs(4, 24, 96, 0)
    L = lad.Ladder(4, 24, 96, mode="bf16x6")
    t1, t2 = to_dev(x.t1), to_dev(x.t2)
    tau = L.tau(t1, t2)
    with pytest.raises(lad.LadderError):
        L.apply_dressed(to_dev(x.B), to_dev(x.B_ov), t1, tau)
    torch.cuda.synchronize()
