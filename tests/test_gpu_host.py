"""The host-buffer entry point ladder_apply_host: B and tau in host memory,
R copied back to host memory, against the CPU oracle in every mode (bars as
for ladder_apply: FP64 1e-12, the error-free split 1e-10, BF16X6 1e-6 on the
larger of the relative Frobenius error and the worst element)."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki": 1e-10, "ozaki_sym": 1e-10, "bf16x6": 1e-6}


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("mode", ["fp64", "ozaki", "ozaki_sym", "bf16x6"])
def test_apply_host_matches_oracle(lad, mode, pinned):
    """ozaki_sym: the error-free mode's symmetric-B form (the bench's e2e call)."""
    import torch
    o, v, n, seed = 7, 41, 70, 14
    x = synthetic.make_inputs(o, v, n, seed)
    tau = oracle.tau(x.t1, x.t2)
    R_o = oracle.ladder(x.B, tau)
    L = lad.Ladder(o, v, n, mode="ozaki" if mode == "ozaki_sym" else mode,
                   tuning={"sym_b": 1} if mode == "ozaki_sym" else None)
    h_B, h_tau = torch.from_numpy(x.B), torch.from_numpy(tau)
    h_R = torch.full_like(h_tau, float("nan"))
    if pinned:
        h_B, h_tau, h_R = h_B.pin_memory(), h_tau.pin_memory(), h_R.pin_memory()
    d_B = torch.empty(x.B.shape, dtype=torch.float64, device="cuda")
    d_tau = torch.empty(tau.shape, dtype=torch.float64, device="cuda")
    d_R = torch.empty_like(d_tau)
    for _ in range(2):
        lad.ladder_apply_host(L.plan, h_B, h_tau, h_R, d_B, d_tau, d_R)
        L.check_device()
        R = h_R.numpy()
        err = rel_err(R, R_o)
        print("%s pinned=%s: rel err %.3e" % (mode, pinned, err))
        assert err < TOL[mode]
        assert np.array_equal(R, d_R.cpu().numpy())
    L.close()


def test_apply_host_rejects_null_host_buffers(lad):
    import torch
    L = lad.Ladder(4, 24, 96, mode="fp64")
    d = torch.empty((4, 4, 24, 24), dtype=torch.float64, device="cuda")
    with pytest.raises(lad.LadderError):
        lad.ladder_apply_host(L.plan, None, None, None, d, d, d)
    L.close()
