"""Full-size workloads against stored oracle values.

tests/golden/<workload>.json holds, for the seeded synthetic inputs of each
workload, E_L, the Frobenius norm of R and a dozen full R_ij^ab columns, all
written by tests/golden/make_golden.py from the plain FP64 CPU oracle.  The
GPU path runs the same inputs through the C ABI, in the launch configuration
the benchmark times.

Bars: FP64 mode |dE_L| <= 1 microhartree and the sampled columns to 1e-12
relative; split-BF16 modes the sampled columns and ||R||_F to their relative
Frobenius tolerance (BF16X6 1e-6, BF16X3 2e-5)."""
import json
import os

import numpy as np
import pytest

import synthetic
from gpu_util import rel_fro, run_forward

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"fp64": 1e-12, "bf16x6": 1e-6, "bf16x3": 2e-5}


def _golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for " + name)
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


CASES = [("dimer_o10_v120_n480", m) for m in ("fp64", "bf16x6", "bf16x3")] + \
        [("grad_o16_v200_n800", m) for m in ("fp64", "bf16x6")] + \
        [("mid_o34_v400_n1600", m) for m in ("bf16x6", "fp64")]


@pytest.mark.parametrize("name,mode", CASES)
def test_full_size_against_stored_oracle(lad, name, mode):
    g = _golden(name)
    w = synthetic.WORKLOADS[name]
    assert (g["o"], g["v"], g["naux"], g["seed"]) == (w.o, w.v, w.naux, w.seed)
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode=mode)
    _, R, E = run_forward(L, x)
    L.close()
    got = np.stack([R[:, :, a, b] for a, b in zip(g["pairs_a"], g["pairs_b"])])
    ref = np.asarray(g["R_cols"])
    e_cols = rel_fro(got, ref)
    e_fro = abs(float(np.linalg.norm(R)) - g["R_fro"]) / g["R_fro"]
    dE = abs(E - g["E_L"])
    print("%s %s: columns rel-F %.3e  |R|_F rel %.3e  dE_L %.3e" % (name, mode, e_cols, e_fro, dE))
    assert e_cols < TOL[mode]
    assert e_fro < TOL[mode]
    if mode == "fp64":
        assert dE <= 1e-6
    # the ladder term keeps the pair symmetry R_ij^ab = R_ji^ba exactly
    assert np.array_equal(R, R.transpose(1, 0, 3, 2))
