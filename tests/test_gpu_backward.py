"""Adjoint of the ladder term on the GPU against the CPU oracle's analytic
gradient, and central finite differences through the autograd Function.

E = sum W_ij^ab R_ij^ab is linear in tau and quadratic in B, so central
differences have no truncation error: only rounding (about 1e-16 |E| / h)."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, to_dev

pytestmark = pytest.mark.gpu

# relative Frobenius tolerances of dtau and dB, per mode (as for R)
DTAU_TOL = {"fp64": 1e-12, "bf16x6": 1e-6, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode,two_pass", [("fp64", 0), ("bf16x6", 0), ("bf16x6", 1), ("bf16x3", 1)])
@pytest.mark.parametrize("o,v,n,seed", [(3, 10, 30, 3), (4, 24, 96, 0), (5, 17, 33, 12), (6, 40, 90, 21),
                                         (12, 24, 40, 22)])
def test_backward_matches_oracle_gradient(lad, mode, two_pass, o, v, n, seed):
    """dtau runs the transposed ladder in the plan's form (fused or two-pass)."""
    import torch
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, v, v)) * 0.1          # general B (no a<->c symmetry)
    x = synthetic.make_inputs(o, v, n, seed)
    tau = oracle.tau(x.t1, x.t2)
    W = oracle.energy_weights(x.t2)
    L = lad.Ladder(o, v, n, mode=mode, backward=True,
                   tuning=None if mode == "fp64" else {"two_pass": two_pass})
    dtau, dB = L.backward(to_dev(B), to_dev(tau), to_dev(W))
    torch.cuda.synchronize()
    L.check_device()
    e_tau = rel_err(dtau.cpu().numpy(), oracle.grad_tau(B, W))
    e_B = rel_err(dB.cpu().numpy(), oracle.grad_B(B, tau, W))
    print("%s two_pass=%d o=%d v=%d n=%d: dtau rel-F %.3e  dB rel-F %.3e" % (mode, two_pass, o, v, n, e_tau, e_B))
    assert e_tau < DTAU_TOL[mode]
    assert e_B < DTAU_TOL[mode]  # dB runs in the plan's mode as well


def test_weights_kernel_matches_oracle(lad):
    x = synthetic.make_inputs(4, 13, 20, 5)
    L = lad.Ladder(4, 13, 20, mode="fp64")
    W = L.weights(to_dev(x.t2)).cpu().numpy()
    assert np.array_equal(W, oracle.energy_weights(x.t2))


def test_autograd_central_differences_fp64(lad):
    """dE_L/dB, dE_L/dtau and dE_L/dt2 from LadderEnergy against central
    differences with step 1e-6 at o=3, v=10, N_aux=30."""
    import torch
    from paper_1810_08142_gb300.autograd import ladder_energy
    w = synthetic.WORKLOADS["fd_o3_v10_n30"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode="fp64", backward=True)
    tau0 = oracle.tau(x.t1, x.t2)
    B = to_dev(x.B).requires_grad_(True)
    tau = to_dev(tau0).requires_grad_(True)
    t2 = to_dev(x.t2).requires_grad_(True)
    E = ladder_energy(B, tau, t2, L)
    E.backward()
    gB, gtau, gt2 = B.grad.cpu().numpy(), tau.grad.cpu().numpy(), t2.grad.cpu().numpy()

    def energy(Bn, taun, t2n):
        with torch.no_grad():
            return float(ladder_energy(to_dev(Bn), to_dev(taun), to_dev(t2n), L).item())

    rng = np.random.default_rng(99)
    h = 1e-6
    for which in ("B", "tau", "t2"):
        base = {"B": x.B, "tau": tau0, "t2": x.t2}
        D = rng.standard_normal(base[which].shape)
        if which in ("tau", "t2"):
            D = 0.5 * (D + D.transpose(1, 0, 3, 2))  # stay on pair-symmetric inputs
        plus = dict(base)
        minus = dict(base)
        plus[which] = base[which] + h * D
        minus[which] = base[which] - h * D
        fd = (energy(plus["B"], plus["tau"], plus["t2"]) -
              energy(minus["B"], minus["tau"], minus["t2"])) / (2 * h)
        an = float(np.sum({"B": gB, "tau": gtau, "t2": gt2}[which] * D))
        print("FD %s: fd %.12e analytic %.12e" % (which, fd, an))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12)


@pytest.mark.parametrize("mode", ["fp64", "bf16x6"])
def test_backward_full_size_sampled(lad, mode):
    """Gradient workload o=16, v=200, N_aux=800: 1024 entries each of dtau and
    dB against the oracle's entry-wise analytic gradient, stored in
    tests/golden/grad_o16_v200_n800_grad.json by make_golden.py --grad; both
    the relative Frobenius error of the sample and its worst entry (against
    the sample's largest) stay within the mode's bar."""
    import json
    import os
    import torch
    w = synthetic.WORKLOADS["grad_o16_v200_n800"]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", w.name + "_grad.json")
    if not os.path.exists(path):
        pytest.skip("no stored gradient entries")
    with open(path) as f:
        g = json.load(f)
    assert (g["o"], g["v"], g["naux"], g["seed"]) == (w.o, w.v, w.naux, w.seed)
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    tau = oracle.tau(x.t1, x.t2)
    W = oracle.energy_weights(x.t2)
    L = lad.Ladder(w.o, w.v, w.naux, mode=mode, backward=True)
    dtau, dB = L.backward(to_dev(x.B), to_dev(tau), to_dev(W))
    torch.cuda.synchronize()
    L.check_device()
    dtau, dB = dtau.cpu().numpy(), dB.cpu().numpy()
    i, j, c, d = (np.asarray(t) for t in g["dtau_index"])
    P, xx, yy = (np.asarray(t) for t in g["dB_index"])
    e_tau = rel_err(dtau[i, j, c, d], np.asarray(g["dtau"]))
    e_B = rel_err(dB[P, xx, yy], np.asarray(g["dB"]))
    print("%s full size: dtau %d entries rel %.3e  dB %d entries rel %.3e" % (mode, len(i), e_tau, len(P), e_B))
    assert len(i) >= 1000 and len(P) >= 1000
    assert e_tau < DTAU_TOL[mode]
    assert e_B < DTAU_TOL[mode]
    # the dtau output keeps the pair symmetry of the ladder
    assert np.array_equal(dtau, dtau.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("sym_b", [0, 1])
def test_autograd_error_free_forward_split_adjoint(lad, sym_b):
    """Gradient workload o=16, v=200, N_aux=800 through the autograd Function
    with an error-free forward plan and a BF16X6 plan for the adjoint: E_L
    within 1 uEh of the stored oracle value, and 1024 stored entries each of
    dE/dtau and dE/dB within the BF16X6 bar; with sym_b the forward plan
    gives dE/dtau itself, error-free (within 1e-10)."""
    import json
    import os
    import torch
    from paper_1810_08142_gb300.autograd import ladder_energy
    w = synthetic.WORKLOADS["grad_o16_v200_n800"]
    gdir = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(gdir, w.name + ".json")) as f:
        gold = json.load(f)
    with open(os.path.join(gdir, w.name + "_grad.json")) as f:
        g = json.load(f)
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    B = to_dev(x.B).requires_grad_(True)
    tau = to_dev(oracle.tau(x.t1, x.t2)).requires_grad_(True)
    t2 = to_dev(x.t2)
    L = lad.Ladder(w.o, w.v, w.naux, mode="ozaki", tuning={"sym_b": sym_b})
    Lg = lad.Ladder(w.o, w.v, w.naux, mode="bf16x6", backward=True)
    E = ladder_energy(B, tau, t2, L, Lg)
    E.backward()
    torch.cuda.synchronize()
    L.check_device()
    Lg.check_device()
    dE = abs(float(E) - gold["E_L"])
    dtau, dB = tau.grad.cpu().numpy(), B.grad.cpu().numpy()
    i, j, c, d = (np.asarray(t) for t in g["dtau_index"])
    P, xx, yy = (np.asarray(t) for t in g["dB_index"])
    e_tau = rel_err(dtau[i, j, c, d], np.asarray(g["dtau"]))
    e_B = rel_err(dB[P, xx, yy], np.asarray(g["dB"]))
    print("ozaki (sym_b %d) forward + bf16x6 adjoint: |dE_L| %.3e  dtau rel %.3e  dB rel %.3e" % (sym_b, dE, e_tau, e_B))
    assert dE <= 1e-6
    assert e_tau < (1e-10 if sym_b else DTAU_TOL["bf16x6"]) and e_B < DTAU_TOL["bf16x6"]
    with pytest.raises(ValueError):
        ladder_energy(B, tau, t2, L, lad.Ladder(4, 24, 96, mode="bf16x6", backward=True))


@pytest.mark.parametrize("o,v,n,seed", [(3, 10, 30, 4), (7, 41, 70, 14)])
def test_error_free_dtau_with_symmetric_B(lad, o, v, n, seed):
    """ladder_backward on an error-free plan with sym_b: dE/dtau (the forward
    of W, since B is symmetric) against the oracle's gradient within 1e-10
    (worst entry included); dE/dB and plans without sym_b are refused."""
    import torch
    x = synthetic.make_inputs(o, v, n, seed)
    tau = oracle.tau(x.t1, x.t2)
    W = oracle.energy_weights(x.t2)
    g_o = oracle.grad_tau(x.B, W)
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"sym_b": 1})
    dtau, _ = L.backward(to_dev(x.B), to_dev(tau), to_dev(W), dtau=True, dB=False)
    torch.cuda.synchronize()
    L.check_device()
    got = dtau.cpu().numpy()
    err = rel_err(got, g_o)
    emax = float(np.abs(got - g_o).max() / np.abs(g_o).max())
    print("error-free dtau o=%d v=%d n=%d: rel-F %.3e  max %.3e" % (o, v, n, err, emax))
    assert err < 1e-10 and emax < 1e-10
    with pytest.raises(lad.LadderError):
        L.backward(to_dev(x.B), to_dev(tau), to_dev(W), dtau=True, dB=True)
    L.close()
    G = lad.Ladder(o, v, n, mode="ozaki")
    with pytest.raises(lad.LadderError):
        G.backward(to_dev(x.B), to_dev(tau), to_dev(W), dtau=True, dB=False)
    G.close()
