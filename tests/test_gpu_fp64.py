"""Parity of the FP64 path (DMMA fused ladder, tau assembly, energy) with the
CPU oracle, element by element.  Tolerances: relative Frobenius error of R at
most 1e-12 and |dE_L| at most 1e-6 Eh (the plain method is exact up to FP64
rounding)."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, run_forward

pytestmark = pytest.mark.gpu

SHAPES = [
    (1, 5, 3, 11),       # degenerate: one occupied orbital, v below one block
    (3, 10, 30, 3),      # finite-difference size
    (4, 24, 96, 0),      # smallest workload
    (5, 17, 33, 12),     # ragged v and N
    (12, 32, 40, 13),    # occupied pairs span two chunks (spill path)
    (7, 41, 70, 14),     # several tiles, ragged tail
    (17, 24, 20, 15),    # four chunks, tiny v
]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300  # noqa: F401
    return torch


@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_fp64_matches_oracle(torch_cuda, o, v, n, seed):
    import paper_1810_08142_gb300 as lad
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="fp64")
    tau_g, R_g, E_g = run_forward(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    assert rel_err(tau_g, tau_o) < 1e-15
    R_o = oracle.ladder(x.B, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    assert rel_err(R_g, R_o) < 1e-12
    assert abs(E_g - E_o) < 1e-6
    assert abs(E_g - E_o) <= 1e-12 * abs(E_o) + 1e-15


def test_fp64_general_B_and_tau(torch_cuda):
    # B without a<->c symmetry; tau pair symmetric but otherwise random
    import paper_1810_08142_gb300 as lad
    rng = np.random.default_rng(5)
    o, v, n = 6, 19, 23
    B = rng.standard_normal((n, v, v))
    tau = rng.standard_normal((o, o, v, v))
    tau = 0.5 * (tau + tau.transpose(1, 0, 3, 2))
    L = lad.Ladder(o, v, n, mode="fp64")
    import torch
    R = L.apply(torch.from_numpy(B).cuda(), torch.from_numpy(tau).cuda()).cpu().numpy()
    assert rel_err(R, oracle.ladder(B, tau)) < 1e-12


def test_fp64_dimer_full(torch_cuda):
    import paper_1810_08142_gb300 as lad
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode="fp64")
    _, R_g, E_g = run_forward(L, x)
    tau_o = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder(x.B, tau_o)
    E_o = oracle.energy(R_o, x.t2)
    assert rel_err(R_g, R_o) < 1e-12
    assert abs(E_g - E_o) < 1e-6
