"""Ragged batch: one plan, one persistent fused launch over the work units of
all molecules, replayed as a CUDA graph.  Checked against the CPU oracle per
molecule, against single-molecule launches with the same work decomposition
(bitwise), and graph replay against the first (capturing) call (bitwise)."""
import os

import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 2e-5, "bf16x6": 1e-6}
SHAPES = [(2, 10, 20, 400), (5, 33, 60, 401), (3, 17, 40, 402), (8, 60, 120, 403),
          (1, 7, 9, 404), (6, 24, 96, 405)]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode", ["bf16x6", "bf16x3"])
def test_batch_matches_oracle_and_single_launches(lad, mode):
    import torch
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in SHAPES]
    taus = [oracle.tau(x.t1, x.t2) for x in mols]
    Bs_d = [to_dev(x.B) for x in mols]
    taus_d = [to_dev(t) for t in taus]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode=mode)
    R1 = batch.apply(Bs_d, taus_d)           # records the graph
    torch.cuda.synchronize()
    R1 = [r.cpu().numpy() for r in R1]
    outs = [torch.empty_like(t) for t in taus_d]
    batch.apply(Bs_d, taus_d, outs)          # new output pointers: records again
    R2 = batch.apply(Bs_d, taus_d, outs)     # same pointers: graph replay
    torch.cuda.synchronize()
    batch.check_device()
    R2 = [r.cpu().numpy() for r in R2]
    for k, x in enumerate(mols):
        ref = oracle.ladder(x.B, taus[k])
        err = rel_err(R1[k], ref)
        print("%s molecule %d (o=%d v=%d n=%d): rel-F %.3e" % (mode, k, x.o, x.v, x.naux, err))
        assert err < TOL[mode]
        assert np.array_equal(R1[k], R2[k])
        # these molecules fit one chunk, so the batch runs them in the fused form
        L = lad.Ladder(x.o, x.v, x.naux, mode=mode, tuning={"two_pass": 0, "ksplit": 1})
        Rs = L.apply(Bs_d[k], taus_d[k]).cpu().numpy()
        assert np.array_equal(Rs, R1[k])


def test_ragged48_sampled_columns(lad):
    """The 48-molecule ragged batch (seeds 100..147) against the oracle: every
    (a, b) column of R for the members with v <= 64, and 64 seeded columns of
    each larger member, each column set within the BF16X6 bar (relative
    Frobenius error and worst element)."""
    import torch
    mols = synthetic.ragged_batch()
    taus = [oracle.tau(x.t1, x.t2) for x in mols]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="bf16x6")
    Rs = batch.apply([to_dev(x.B) for x in mols], [to_dev(t) for t in taus])
    torch.cuda.synchronize()
    batch.check_device()
    worst, ncols = 0.0, 0
    rng = np.random.default_rng(3)
    for k, x in enumerate(mols):
        got = Rs[k].cpu().numpy()
        if x.v <= 64:
            ref = oracle.ladder(x.B, taus[k])
            err = rel_err(got, ref)
            ncols += x.v * x.v
        else:
            pa, pb = rng.integers(0, x.v, 64), rng.integers(0, x.v, 64)
            ref = oracle.ladder_pairs(x.B, taus[k], pa, pb)
            err = rel_err(np.stack([got[:, :, a, b] for a, b in zip(pa, pb)]), ref)
            ncols += 64
        worst = max(worst, err)
        assert np.array_equal(got, got.transpose(1, 0, 3, 2))
    print("ragged48: %d columns checked, worst rel err %.3e" % (ncols, worst))
    assert worst < TOL["bf16x6"]


TWO_PASS_SHAPES = [(12, 32, 40, 410), (3, 17, 40, 411), (16, 24, 48, 412), (20, 17, 33, 413),
                   (6, 24, 96, 414)]


def test_batch_with_two_pass_members(lad):
    """Molecules whose occupied pairs need several chunks run in the two-pass
    form inside the batch (one storing launch and one GEMM2 launch over all
    of them), the others in the fused launch.  Each molecule against the
    oracle, and bitwise against a single-molecule launch in the same form and
    block-pair split (the storing pass's work grouping does not change any
    value)."""
    import torch
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in TWO_PASS_SHAPES]
    taus = [oracle.tau(x.t1, x.t2) for x in mols]
    Bs_d = [to_dev(x.B) for x in mols]
    taus_d = [to_dev(t) for t in taus]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="bf16x6")
    R1 = batch.apply(Bs_d, taus_d)
    R2 = batch.apply(Bs_d, taus_d, R1)       # graph replay into the same outputs
    torch.cuda.synchronize()
    batch.check_device()
    R = [r.cpu().numpy() for r in R2]
    for k, x in enumerate(mols):
        ref = oracle.ladder(x.B, taus[k])
        err = rel_err(R[k], ref)
        multi = x.o >= 11
        print("molecule %d (o=%d v=%d n=%d, %s): rel-F %.3e" % (k, x.o, x.v, x.naux,
              "two-pass" if multi else "fused", err))
        assert err < TOL["bf16x6"]
        tun = {"two_pass": int(multi), "ksplit": 1}
        L = lad.Ladder(x.o, x.v, x.naux, mode="bf16x6", tuning=tun)
        Rs = L.apply(Bs_d[k], taus_d[k]).cpu().numpy()
        assert np.array_equal(Rs, R[k])
        L.close()


def test_batch_member_tunings(lad):
    """Per-member launch parameters and forms (what the autotuner's per-shape
    choices set): every member against the oracle, and a two-pass member
    bitwise against its single-molecule launch in the same form and split."""
    import torch
    tunings = [{"kc": 2, "s_pieces": 1, "two_pass": 1}, {"kc": 8, "s_pieces": 2, "two_pass": 0},
               {"kc": 4, "s_pieces": 4, "two_pass": 1}, {"kc": 1, "s_pieces": 2, "two_pass": 0},
               None, {"kc": 4, "s_pieces": 2, "two_pass": 1}]
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in SHAPES]
    taus = [oracle.tau(x.t1, x.t2) for x in mols]
    Bs_d = [to_dev(x.B) for x in mols]
    taus_d = [to_dev(t) for t in taus]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="bf16x6", tunings=tunings)
    R = [r.cpu().numpy() for r in batch.apply(Bs_d, taus_d)]
    torch.cuda.synchronize()
    batch.check_device()
    for k, x in enumerate(mols):
        err = rel_err(R[k], oracle.ladder(x.B, taus[k]))
        print("member %d %s: rel-F %.3e" % (k, tunings[k], err))
        assert err < TOL["bf16x6"]
    # member 0 (two-pass, kc 2, one piece per S): the batch's storing pass and
    # GEMM2 pass give the single-molecule launch's bits
    x = mols[0]
    L = lad.Ladder(x.o, x.v, x.naux, mode="bf16x6",
                   tuning={"kc": 2, "s_pieces": 1, "two_pass": 1, "ksplit": 1})
    Rs = L.apply(Bs_d[0], taus_d[0]).cpu().numpy()
    assert np.array_equal(Rs, R[0])


def test_batch_tuned_mode(lad):
    """mode="tuned": each member's choices from the autotuner's cache."""
    import torch
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in SHAPES]
    taus = [oracle.tau(x.t1, x.t2) for x in mols]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="tuned")
    assert len(batch.tunings) == len(mols)
    R = batch.apply([to_dev(x.B) for x in mols], [to_dev(t) for t in taus])
    torch.cuda.synchronize()
    batch.check_device()
    for k, x in enumerate(mols):
        assert rel_err(R[k].cpu().numpy(), oracle.ladder(x.B, taus[k])) < TOL["bf16x6"]


def _e_scale(R, t2):
    """sum |R_ij^ab (2 t_ij^ab - t_ij^ba)|: the scale of E_L's rounding."""
    return float(np.sum(np.abs(R * (2.0 * t2 - t2.transpose(0, 1, 3, 2)))))


@pytest.mark.parametrize("mode", ["bf16x6", "bf16x3"])
def test_step_batched_tau_ladder_energy(lad, mode):
    """ladder_step_batched: tau assembly, the ladder and E_L of every molecule
    in one graph, from t1 and t2 on the device.  tau against the oracle to
    rounding, R within the mode's bar, E_L within it relative to the sum of
    its terms' magnitudes, and a replay with the same pointers bitwise equal."""
    import torch
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in SHAPES + TWO_PASS_SHAPES[:2]]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode=mode)
    Bs, t1s, t2s = ([to_dev(getattr(x, a)) for x in mols] for a in ("B", "t1", "t2"))
    taus, Rs, E = batch.step(Bs, t1s, t2s)
    torch.cuda.synchronize()
    batch.check_device()
    first = ([t.cpu().numpy() for t in taus], [r.cpu().numpy() for r in Rs], E.cpu().numpy())
    batch.step(Bs, t1s, t2s, taus, Rs, E)   # replay
    torch.cuda.synchronize()
    for k, x in enumerate(mols):
        tau_o = oracle.tau(x.t1, x.t2)
        R_o = oracle.ladder(x.B, tau_o)
        E_o = oracle.energy(R_o, x.t2)
        e_tau = rel_err(first[0][k], tau_o)
        e_R = rel_err(first[1][k], R_o)
        e_E = abs(first[2][k] - E_o) / _e_scale(R_o, x.t2)
        print("%s molecule %d (o=%d v=%d n=%d): tau %.1e  R %.3e  E_L %.3e" % (mode, k, x.o, x.v, x.naux,
                                                                            e_tau, e_R, e_E))
        assert e_tau < 1e-15
        assert e_R < TOL[mode]
        assert e_E < TOL[mode]
        assert np.array_equal(Rs[k].cpu().numpy(), first[1][k])
    assert np.array_equal(E.cpu().numpy(), first[2])
    batch.close()


def test_ragged48_step_energies(lad):
    """The 48-molecule ragged batch through ladder_step_batched: every
    member's E_L against the oracle for the members with v <= 64 (the oracle
    needs the whole R), and tau of every member to rounding."""
    import torch
    mols = synthetic.ragged_batch()
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="tuned")
    Bs, t1s, t2s = ([to_dev(getattr(x, a)) for x in mols] for a in ("B", "t1", "t2"))
    taus, Rs, E = batch.step(Bs, t1s, t2s)
    torch.cuda.synchronize()
    batch.check_device()
    E = E.cpu().numpy()
    worst, nE = 0.0, 0
    for k, x in enumerate(mols):
        tau_o = oracle.tau(x.t1, x.t2)
        assert rel_err(taus[k].cpu().numpy(), tau_o) < 1e-15
        if x.v <= 64:
            R_o = oracle.ladder(x.B, tau_o)
            worst = max(worst, abs(E[k] - oracle.energy(R_o, x.t2)) / _e_scale(R_o, x.t2))
            nE += 1
    print("ragged48 step: %d energies checked, worst %.3e" % (nE, worst))
    assert nE >= 1 and worst < TOL["bf16x6"]
    batch.close()


@pytest.mark.parametrize("sym", ["general", "symmetric", "mixed"])
def test_step_batched_ozaki(lad, sym):
    """The error-free mode as a batch: every member in the two-pass form, both
    passes over all members' work units in one launch each, inside one graph
    with tau and E_L.  R within 1e-10 relative (worst element within 2e-10 of
    max |R|), |dE_L| <= 1 uEh and within 1e-12 of the sum of the energy
    terms' magnitudes, and a replay bitwise equal.  symmetric: every member
    forms its distinct integral tiles once (sym_b); mixed: every other one."""
    import torch
    shapes = SHAPES + TWO_PASS_SHAPES[:2] + [(12, 140, 150, 21)]
    mols = [synthetic.make_inputs(o, v, n, s) for o, v, n, s in shapes]
    flags = {"general": False, "symmetric": True, "mixed": [k % 2 == 1 for k in range(len(mols))]}[sym]
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="ozaki", sym_b=flags)
    Bs, t1s, t2s = ([to_dev(getattr(x, a)) for x in mols] for a in ("B", "t1", "t2"))
    taus, Rs, E = batch.step(Bs, t1s, t2s)
    torch.cuda.synchronize()
    batch.check_device()
    first = ([r.cpu().numpy() for r in Rs], E.cpu().numpy())
    batch.step(Bs, t1s, t2s, taus, Rs, E)   # replay
    torch.cuda.synchronize()
    for k, x in enumerate(mols):
        tau_o = oracle.tau(x.t1, x.t2)
        R_o = oracle.ladder(x.B, tau_o)
        E_o = oracle.energy(R_o, x.t2)
        e_R = rel_err(first[0][k], R_o)
        dE = abs(first[1][k] - E_o)
        print("ozaki molecule %d (o=%d v=%d n=%d): R %.3e  |dE_L| %.3e  E_L %.6e" % (k, x.o, x.v, x.naux,
                                                                                  e_R, dE, E_o))
        assert rel_err(taus[k].cpu().numpy(), tau_o) < 1e-15
        assert e_R < 1e-10
        assert dE <= 1e-6 and dE <= 1e-12 * _e_scale(R_o, x.t2)
        assert np.array_equal(Rs[k].cpu().numpy(), first[0][k])
    assert np.array_equal(E.cpu().numpy(), first[1])
    batch.close()


@pytest.mark.parametrize("sym_b", [False, True])
def test_ragged48_ozaki_against_stored_oracle(lad, sym_b):
    """The 48-molecule ragged batch in the error-free mode through
    ladder_step_batched: every member's E_L within 1 uEh of the stored oracle
    value (tests/golden/ragged48.json, written by make_golden.py --ragged)
    and four stored R columns per member within 1e-10; with sym_b every
    member forms its distinct integral tiles once."""
    import json
    import torch
    with open(os.path.join(os.path.dirname(__file__), "golden", "ragged48.json")) as f:
        gold = json.load(f)["molecules"]
    mols = synthetic.ragged_batch()
    assert len(gold) == len(mols)
    batch = lad.LadderBatch([(x.o, x.v, x.naux) for x in mols], mode="ozaki", sym_b=sym_b)
    Bs, t1s, t2s = ([to_dev(getattr(x, a)) for x in mols] for a in ("B", "t1", "t2"))
    taus, Rs, E = batch.step(Bs, t1s, t2s)
    torch.cuda.synchronize()
    batch.check_device()
    E = E.cpu().numpy()
    worst_E, worst_R = 0.0, 0.0
    for k, (x, g) in enumerate(zip(mols, gold)):
        assert (g["o"], g["v"], g["naux"]) == (x.o, x.v, x.naux)
        worst_E = max(worst_E, abs(E[k] - g["E_L"]))
        R = Rs[k]
        got = np.stack([R[:, :, a, b].cpu().numpy() for a, b in zip(g["pairs_a"], g["pairs_b"])])
        worst_R = max(worst_R, rel_err(got, np.array(g["R_cols"])))
    print("ragged48 ozaki (sym_b %s): worst |dE_L| %.3e Eh, worst column rel err %.3e" % (sym_b, worst_E, worst_R))
    assert worst_E <= 1e-6
    assert worst_R < 1e-10
    batch.close()
