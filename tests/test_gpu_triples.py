"""The perturbative triples energy E(T) (Sec. II.A) through ladder_triples,
against the CPU oracle.  FP64 forms W in FP64 (bar 1e-12 relative); FP32
forms the integrals and W in FP32 with FP64 energy sums (bar 1e-5 relative:
W carries FP32 rounding of sums over v + o terms); BF16X6 runs the W
contractions on the tensor cores from three BF16 slices of each FP32 operand
(bar 1e-5 relative: the slices hold the FP32 operands exactly, the six
products drop terms 2^-24 below, and the tensor core's FP32 accumulation
adds a bias of about 2e-8 per accumulation step)."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x6": 1e-5}
SHAPES = [(2, 4, 3, 11), (3, 5, 4, 7), (4, 24, 96, 0), (5, 17, 33, 12), (8, 60, 240, 21)]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


def run(lad, x, precision):
    import torch
    E = lad.triples(to_dev(x.B), to_dev(x.B_ov), to_dev(x.B_oo), to_dev(x.t1), to_dev(x.t2),
                    to_dev(x.e_occ), to_dev(x.e_vir), precision=precision)
    torch.cuda.synchronize()
    return float(E.item())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x6"])
@pytest.mark.parametrize("o,v,n,seed", SHAPES + [(3, 140, 60, 23), (17, 33, 40, 24)])
def test_triples_matches_oracle(lad, precision, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    E_g = run(lad, x, precision)
    E_o = oracle.triples(x.B, x.B_ov, x.B_oo, x.t1, x.t2, x.e_occ, x.e_vir)
    err = abs(E_g - E_o) / abs(E_o)
    print("triples %s o=%d v=%d n=%d: E(T) %.12e  rel err %.3e" % (precision, o, v, n, E_o, err))
    assert err < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x6"])
def test_triples_vanish_with_one_occupied_orbital(lad, precision):
    """o = 1: W_iii^abc is symmetric in (a, b, c) (P sums all six orderings),
    so sum_abc (4 W_abc + W_bca + W_cab)(V_abc - V_cba) = 0 up to rounding."""
    x = synthetic.make_inputs(1, 9, 12, 11)
    x2 = synthetic.make_inputs(2, 9, 12, 11)
    scale = abs(oracle.triples(x2.B, x2.B_ov, x2.B_oo, x2.t1, x2.t2, x2.e_occ, x2.e_vir))
    assert abs(run(lad, x, precision)) <= (1e-9 if precision == "fp64" else TOL[precision]) * scale
    assert abs(oracle.triples(x.B, x.B_ov, x.B_oo, x.t1, x.t2, x.e_occ, x.e_vir)) <= 1e-12 * scale


def test_triples_is_reproducible(lad):
    x = synthetic.make_inputs(5, 17, 33, 12)
    assert run(lad, x, "fp64") == run(lad, x, "fp64")


def test_triples_rejects_a_small_workspace(lad):
    import torch
    x = synthetic.make_inputs(3, 5, 4, 7)
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    E = torch.empty((), dtype=torch.float64, device="cuda")
    with pytest.raises(lad.LadderError):
        lad.ladder_triples(3, 5, 4, 0, to_dev(x.B), to_dev(x.B_ov), to_dev(x.B_oo), to_dev(x.t1),
                           to_dev(x.t2), to_dev(x.e_occ), to_dev(x.e_vir), E, ws)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x6"])
def test_triples_dimer_against_stored_oracle(lad, precision):
    """The water-dimer-sized workload (o=10, v=120, N_aux=480) against E(T)
    stored by tests/golden/make_golden.py --triples."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "dimer_o10_v120_n480_triples.json")
    if not os.path.exists(path):
        pytest.skip("no stored E(T)")
    with open(path) as f:
        g = json.load(f)
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    assert (g["o"], g["v"], g["naux"], g["seed"]) == (w.o, w.v, w.naux, w.seed)
    E_g = run(lad, synthetic.make_inputs(w.o, w.v, w.naux, w.seed), precision)
    err = abs(E_g - g["E_T"]) / abs(g["E_T"])
    print("triples dimer %s: E(T) %.12e  rel err %.3e" % (precision, g["E_T"], err))
    assert err < TOL[precision]


def test_triples_tensor_core_size_limit(lad):
    """The tensor-core W kernel holds one column tile of at most 256 virtual
    orbitals: larger v is refused before any launch."""
    with pytest.raises(lad.LadderError):
        lad.ladder_triples_workspace_size(4, 257, 40, lad.TRIPLES_PRECISION["bf16x6"])
