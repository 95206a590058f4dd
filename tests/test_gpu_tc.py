"""Parity of the split-BF16 tensor-core path (tcgen05 fused ladder) with the
CPU oracle, element by element.

Tolerances on the relative Frobenius error of R:
  BF16X3 (two slices, three products): 2e-5.  Dropping the lo*lo product and
      the bits below the second slice leaves about 2^-16 per product; the
      measured error is a few 1e-6.
  BF16X6 (three slices, six products): 1e-6, the stated split tolerance.
"""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, run_forward

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 2e-5, "bf16x6": 1e-6}

SHAPES = [
    (1, 5, 3, 11),       # one occupied orbital, v below one block
    (3, 10, 30, 3),      # finite-difference size
    (4, 24, 96, 0),      # smallest workload
    (5, 17, 33, 12),     # ragged v and N
    (7, 41, 70, 14),     # several tiles, ragged tail
    (12, 32, 40, 13),    # occupied pairs fill one TMEM region
    (20, 40, 50, 16),    # two occupied-pair chunks
]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("two_pass", [0, 1])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_tc_matches_oracle(lad, mode, two_pass, o, v, n, seed):
    """Both forms (fused kernel, two-pass) on every shape."""
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode=mode, tuning={"two_pass": two_pass})
    _, R_g, E_g = run_forward(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder(x.B, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    err = rel_err(R_g, R_o)
    print("%s two_pass=%d o=%d v=%d n=%d: rel-F %.3e  |dE| %.3e  E %.6e" % (mode, two_pass, o, v, n, err,
                                                                          abs(E_g - E_o), E_o))
    assert err < TOL[mode]
    # pair symmetry of the output holds by construction of the unpacking
    assert np.array_equal(R_g, R_g.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
def test_tc_dimer_full(lad, mode):
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode=mode)
    _, R_g, E_g = run_forward(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder(x.B, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    err = rel_err(R_g, R_o)
    print("%s dimer: rel-F %.3e  |dE| %.3e  E %.6e" % (mode, err, abs(E_g - E_o), E_o))
    assert err < TOL[mode]


# Shapes whose occupied pairs need several chunks of the fused kernel: both
# forms (fused with GEMM1 recomputed per chunk, and the two-pass form with the
# V+- tiles stored in the workspace) are checked against the oracle.
MULTI_CHUNK = [
    (12, 32, 40, 13),    # two chunks in the fused form, one in the two-pass form
    (20, 40, 50, 16),
    (24, 17, 33, 9),     # ragged v (one 16-block, padded)
    (34, 24, 60, 5),     # the mid workload's o: ten fused chunks, five two-pass
]


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("two_pass", [0, 1])
@pytest.mark.parametrize("o,v,n,seed", MULTI_CHUNK)
def test_tc_forms_match_oracle(lad, mode, two_pass, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode=mode, tuning={"two_pass": two_pass})
    assert lad.ladder_get_tuning(L.plan).two_pass == two_pass
    _, R_g, E_g = run_forward(L, x)
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    err = rel_err(R_g, R_o)
    print("%s two_pass=%d o=%d v=%d n=%d: rel-F %.3e" % (mode, two_pass, o, v, n, err))
    assert err < TOL[mode]
    assert np.array_equal(R_g, R_g.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("ksplit", [1, 3])
def test_two_pass_block_pair_split(lad, ksplit):
    """The GEMM2 pass with its block pairs split over work units (FP64 sums
    of the ranges in the unpack kernel) against the unsplit pass."""
    o, v, n, seed = 16, 48, 64, 21
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="bf16x6", tuning={"two_pass": 1, "ksplit": ksplit})
    _, R_g, _ = run_forward(L, x)
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    err = rel_err(R_g, R_o)
    print("two_pass ksplit=%d: rel-F %.3e" % (ksplit, err))
    assert err < TOL["bf16x6"]
