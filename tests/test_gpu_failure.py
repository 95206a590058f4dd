"""Device-side failure detection without a GPU fault: a bounded wait that
nothing satisfies gives up, records its site in the status word, and the
context stays usable for the next ladder evaluation."""
import time

import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, run_forward

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    L = lad.Ladder(4, 24, 96, mode="bf16x6")
    assert lad.ladder_last_device_error(L.plan) == (0, 0)
    t0 = time.time()
    lad.ladder_selftest_wait(L.plan, 200_000_000)  # 0.2 s
    st, where = lad.ladder_last_device_error(L.plan)
    dt = time.time() - t0
    assert st == 4 and where == 99  # LADDER_ETIMEOUT at the self-test site
    assert 0.15 < dt < 10.0
    # the status word was cleared by the read, and the context still computes
    assert lad.ladder_last_device_error(L.plan) == (0, 0)
    x = synthetic.make_inputs(4, 24, 96, 0)
    _, R, _ = run_forward(L, x)
    assert rel_err(R, oracle.ladder(x.B, oracle.tau(x.t1, x.t2))) < 1e-6


def test_argument_errors_are_synchronous():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    L = lad.Ladder(4, 24, 96, mode="fp64")
    B = torch.zeros(96, 24, 24, dtype=torch.float64, device="cuda")
    tau = torch.zeros(4, 4, 24, 24, dtype=torch.float64, device="cuda")
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_apply(L.plan, B, tau, tau)          # R aliases tau
    assert e.value.status == 1
    host = torch.zeros(4, 4, 24, 24, dtype=torch.float64)
    with pytest.raises(lad.LadderError):
        lad.ladder_apply(L.plan, B, host, tau)          # host pointer
    with pytest.raises(lad.LadderError):
        lad.ladder_selftest_wait(L.plan, 1)             # limit out of range
