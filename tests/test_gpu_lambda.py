"""The paper's lambda-only contraction (Sec. II.C: only the pair symmetry
R_ij^ab = R_ji^ba is used) as an ablation of the +- split, against the CPU
oracle element by element.  The storing pass keeps (ac|bd) and (ad|bc)
instead of their +- combinations; GEMM2 multiplies both into one accumulator
for all o^2 ordered occupied pairs.  Same tolerances as the +- form:
BF16X3 2e-5, BF16X6 1e-6 relative Frobenius error of R.
"""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, run_forward

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 2e-5, "bf16x6": 1e-6}

SHAPES = [
    (1, 5, 3, 11),       # one occupied orbital
    (4, 24, 96, 0),      # smallest workload
    (5, 17, 33, 12),     # ragged v and N
    (7, 41, 70, 14),     # several tiles, ragged tail
    (14, 40, 50, 16),    # o^2 = 196 ordered pairs: two GEMM2 chunks
]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_lambda_only_matches_oracle(lad, mode, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode=mode, tuning={"two_pass": 1, "lambda_only": 1})
    assert lad.ladder_get_tuning(L.plan).lambda_only == 1
    _, R_g, E_g = run_forward(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder(x.B, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    err = rel_err(R_g, R_o)
    print("lambda-only %s o=%d v=%d n=%d: rel-F %.3e  |dE| %.3e" % (mode, o, v, n, err, abs(E_g - E_o)))
    assert err < TOL[mode]
    # every element of R is written from one accumulator column and mirrored
    assert np.array_equal(R_g, R_g.transpose(1, 0, 3, 2))


def test_lambda_only_dimer(lad):
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode="bf16x6", tuning={"two_pass": 1, "lambda_only": 1})
    _, R_g, _ = run_forward(L, x)
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    err = rel_err(R_g, R_o)
    print("lambda-only dimer bf16x6: rel-F %.3e" % err)
    assert err < TOL["bf16x6"]


def test_lambda_only_needs_the_two_pass_form(lad):
    plan = lad.ladder_plan(4, 24, 96, lad.LADDER_BF16X6)
    try:
        t = lad.ladder_get_tuning(plan)
        t.two_pass, t.lambda_only = 0, 1
        with pytest.raises(lad.LadderError):
            lad.ladder_set_tuning(plan, t)
    finally:
        lad.ladder_destroy(plan)
