"""Parity of the error-free split-BF16 mode (LADDER_OZAKI) with the CPU oracle.

The mode splits each operand row into S fixed-point BF16 slices under one
power-of-two scale and accumulates every slice order exactly on the tensor
cores, so its only errors are the truncation of the slice expansion (about
2^-40 of a row's largest element with S = 5, 2^-48 with S = 6) and the
double-single (about 48-bit) sums.  Bars, element by element against the FP64
oracle:
  R:    relative Frobenius error and max |dR| / max |R| <= 1e-10 (S = 5),
        1e-12 (S = 6);
  E_L:  |dE_L| <= 1 microhartree absolutely (the metric's bar) and
        |dE_L| <= 1e-12 (S = 5), 1e-13 (S = 6) times sum |R_ij^ab W_ij^ab|
        (W = 2 t - t^T), the scale of the rounding of a sum whose terms
        cancel; on the synthetic workloads E_L is coherent and that sum is
        within a few per cent of |E_L|.
A scratch simulation of the scheme with exact products (dimer size) gave
rel-F(R) 1.2e-12 / 8.9e-15 and |dE_L| / E_L 3e-14 / 7e-15 for S = 5 / 6.
"""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_fro, run_forward, to_dev

pytestmark = pytest.mark.gpu

TOL_R = {5: 1e-10, 6: 1e-12}
TOL_E = {5: 1e-12, 6: 1e-13}

SHAPES = [
    (1, 5, 3, 11),       # one occupied orbital, v below one block, N below one K-step
    (3, 10, 30, 3),      # finite-difference size
    (4, 24, 96, 0),      # smallest workload
    (5, 17, 33, 12),     # ragged v and N
    (7, 41, 70, 14),     # several tiles, ragged tail
    (12, 32, 200, 13),   # several GEMM1 windows (N = 200 > 128), ragged last window
    (20, 40, 50, 16),    # several occupied-pair chunks of each sign
    (34, 24, 60, 5),     # the mid workload's o: five plus and five minus chunks
]


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


def _check(R_g, E_g, R_o, E_o, S, tag, t2):
    err = rel_fro(R_g, R_o)
    emax = float(np.max(np.abs(R_g - R_o)) / max(np.max(np.abs(R_o)), 1e-300))
    dE = abs(E_g - E_o)
    e_abs = float(np.sum(np.abs(R_o * (2.0 * t2 - t2.transpose(0, 1, 3, 2)))))
    print("%s S=%d: rel-F %.3e  max %.3e  |dE| %.3e  |dE|/sum|RW| %.3e  E %.6e  sum|RW| %.6e" %
          (tag, S, err, emax, dE, dE / e_abs, E_o, e_abs))
    assert err <= TOL_R[S]
    assert emax <= TOL_R[S]
    assert dE <= 1e-6
    assert dE <= TOL_E[S] * e_abs
    # the unpacking writes R_ij^ab and R_ji^ba from the same sums
    assert np.array_equal(R_g, R_g.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("S", [5, 6])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_ozaki_matches_oracle(lad, S, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"oz_slices": S})
    assert lad.ladder_get_tuning(L.plan).oz_slices == S
    _, R_g, E_g = run_forward(L, x)
    L.close()
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), S, "o=%d v=%d n=%d" % (o, v, n), x.t2)


@pytest.mark.parametrize("ksplit", [1, 3])
def test_ozaki_block_pair_split(lad, ksplit):
    """GEMM2 work units over block-pair ranges (summed by the unpack kernel)."""
    o, v, n, seed = 16, 48, 64, 21
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"ksplit": ksplit})
    _, R_g, E_g = run_forward(L, x)
    L.close()
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), 5, "ksplit=%d" % ksplit, x.t2)


def test_ozaki_general_B(lad):
    """B without the a<->c symmetry of the generator (the plan assumes none)."""
    o, v, n, seed = 6, 30, 45, 31
    x = synthetic.make_inputs(o, v, n, seed)
    rng = np.random.default_rng(99)
    B = x.B + 0.02 * rng.standard_normal(x.B.shape) * synthetic.sigma(n)[:, None, None]
    x.B = np.ascontiguousarray(B)
    L = lad.Ladder(o, v, n, mode="ozaki")
    _, R_g, E_g = run_forward(L, x)
    L.close()
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), 5, "general B", x.t2)


def test_ozaki_scale_invariance(lad):
    """Scaling B by 2^k scales R by 2^2k bit for bit: the row scales absorb
    powers of two and the slices do not change."""
    import torch
    o, v, n, seed = 5, 26, 40, 8
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="ozaki")
    t1, t2 = to_dev(x.t1), to_dev(x.t2)
    tau = L.tau(t1, t2)
    R1 = L.apply(to_dev(x.B), tau).cpu().numpy()
    R2 = L.apply(to_dev(x.B * 2.0 ** 20), tau).cpu().numpy()
    torch.cuda.synchronize()
    L.check_device()
    L.close()
    assert np.array_equal(R2, R1 * 2.0 ** 40)


@pytest.mark.parametrize("what", ["B_nan", "B_inf", "tau_nan"])
def test_ozaki_nonfinite_input_reported(lad, what):
    """A NaN or infinity in B or tau is reported as LADDER_ENONFINITE by the
    device status word (inputs prepared on the host)."""
    import torch
    o, v, n, seed = 4, 24, 96, 0
    x = synthetic.make_inputs(o, v, n, seed)
    B = x.B.copy()
    tau = oracle.tau(x.t1, x.t2)
    if what == "B_nan":
        B[3, 5, 7] = np.nan
    elif what == "B_inf":
        B[0, 1, 2] = np.inf
    else:
        tau[1, 2, 3, 4] = np.nan
        tau[2, 1, 4, 3] = np.nan
    L = lad.Ladder(o, v, n, mode="ozaki")
    L.apply(to_dev(B), to_dev(tau))
    torch.cuda.synchronize()
    st, where = lad.ladder_last_device_error(L.plan)
    assert lad.STATUS[st] == "LADDER_ENONFINITE" and where == 50
    # the word was cleared by the read; a clean call reports nothing
    L.apply(to_dev(x.B), to_dev(oracle.tau(x.t1, x.t2)))
    torch.cuda.synchronize()
    assert lad.ladder_last_device_error(L.plan) == (0, 0)
    L.close()


@pytest.mark.parametrize("mode", ["bf16x6", "bf16x3"])
def test_split_modes_report_nonfinite(lad, mode):
    import torch
    x = synthetic.make_inputs(4, 24, 96, 0)
    B = x.B.copy()
    B[2, 3, 4] = np.inf
    L = lad.Ladder(4, 24, 96, mode=mode)
    L.apply(to_dev(B), to_dev(oracle.tau(x.t1, x.t2)))
    torch.cuda.synchronize()
    st, where = lad.ladder_last_device_error(L.plan)
    L.close()
    assert lad.STATUS[st] == "LADDER_ENONFINITE" and where == 50


def test_ozaki_dimer_full(lad):
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode="ozaki")
    _, R_g, E_g = run_forward(L, x)
    L.close()
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), 5, "dimer", x.t2)


# ---------------------------------------------------------------- symmetric B
# The generator's B is symmetric in a <-> c, so (ac|bd) depends only on the
# unordered pairs {a,c} and {b,d} and their order; with sym_b the plan computes
# each distinct 64 x 64 integral tile once and forms V+- from them.

@pytest.mark.parametrize("S", [5, 6])
@pytest.mark.parametrize("o,v,n,seed", SHAPES)
def test_ozaki_symmetric_B_matches_oracle(lad, S, o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    assert np.array_equal(x.B, x.B.transpose(0, 2, 1))
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"oz_slices": S, "sym_b": 1})
    assert lad.ladder_get_tuning(L.plan).sym_b == 1
    _, R_g, E_g = run_forward(L, x)
    L.close()
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), S, "sym o=%d v=%d n=%d" % (o, v, n), x.t2)
    # the general form on the same input: the two differ only in the rounding
    # of the tail slice orders' FP32 sums (about 2^-48 of an integral)
    G = lad.Ladder(o, v, n, mode="ozaki", tuning={"oz_slices": S})
    _, R_gen, _ = run_forward(G, x)
    G.close()
    scale = max(float(np.max(np.abs(R_o))), 1e-300)
    assert float(np.max(np.abs(R_g - R_gen))) <= 1e-13 * scale


def test_ozaki_symmetric_B_timing_and_dimer(lad):
    """The dimer-size workload in the symmetric-B form, with the two stages
    of its first pass timed."""
    w = synthetic.WORKLOADS["dimer_o10_v120_n480"]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    L = lad.Ladder(w.o, w.v, w.naux, mode="ozaki", tuning={"sym_b": 1})
    lad.ladder_set_timing(L.plan, True)
    _, R_g, E_g = run_forward(L, x)
    xs, fm = lad.ladder_timing_sym(L.plan)
    p1, p2 = lad.ladder_timing_passes(L.plan)
    L.close()
    print("dimer sym: distinct tiles %.3f ms, formation %.3f ms, pass 1 %.3f ms, pass 2 %.3f ms" % (xs, fm, p1, p2))
    assert xs > 0 and fm > 0 and abs(xs + fm - p1) <= 0.05 * p1 + 0.01
    R_o = oracle.ladder(x.B, oracle.tau(x.t1, x.t2))
    _check(R_g, E_g, R_o, oracle.energy(R_o, x.t2), 5, "sym dimer", x.t2)


def test_ozaki_symmetric_B_asymmetric_input_reported(lad):
    """A B that breaks the promised symmetry is reported as LADDER_EINVAL
    (site 51) by the device status word; a symmetric B then reports nothing."""
    import torch
    o, v, n, seed = 4, 24, 96, 0
    x = synthetic.make_inputs(o, v, n, seed)
    B = x.B.copy()
    B[7, 3, 17] += 1e-9
    tau = to_dev(oracle.tau(x.t1, x.t2))
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"sym_b": 1})
    L.apply(to_dev(B), tau)
    torch.cuda.synchronize()
    st, where = lad.ladder_last_device_error(L.plan)
    assert lad.STATUS[st] == "LADDER_EINVAL" and where == 51
    L.apply(to_dev(x.B), tau)
    torch.cuda.synchronize()
    assert lad.ladder_last_device_error(L.plan) == (0, 0)
    L.close()


def test_ozaki_symmetric_B_unsupported_combinations(lad):
    """sym_b is refused on a plan sized for the dressed term and outside the
    error-free mode; with a tile range it is taken, in either order."""
    o, v, n = 4, 40, 60

    def refused(plan, status):
        t = lad.ladder_get_tuning(plan)
        t.sym_b = 1
        with pytest.raises(lad.LadderError) as ei:
            lad.ladder_set_tuning(plan, t)
        assert lad.STATUS[ei.value.status] == status
        lad.ladder_destroy(plan)

    refused(lad.ladder_plan(o, v, n, lad.MODES["ozaki"] | lad.LADDER_WITH_DRESSING), "LADDER_ENOTSUP")
    refused(lad.ladder_plan(o, v, n, lad.MODES["bf16x6"]), "LADDER_EINVAL")
    for range_first in (True, False):
        P = lad.ladder_plan(o, v, n, lad.MODES["ozaki"])
        if range_first:
            lad.ladder_set_tile_range(P, 0, 2)
        t = lad.ladder_get_tuning(P)
        t.sym_b = 1
        lad.ladder_set_tuning(P, t)
        if not range_first:
            lad.ladder_set_tile_range(P, 0, 2)
        assert lad.ladder_get_tuning(P).sym_b == 1
        lad.ladder_destroy(P)


@pytest.mark.parametrize("chunk", [5, 1])
def test_ozaki_symmetric_B_tile_ranges(lad, chunk):
    """Sequential tile ranges: the distinct tiles are formed once, V+- range
    by range from them; R is bit for bit that of one range."""
    o, v, n, seed = 7, 41, 70, 14
    x = synthetic.make_inputs(o, v, n, seed)
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"sym_b": 1})
    _, R1, _ = run_forward(L, x)
    L.close()
    L = lad.Ladder(o, v, n, mode="ozaki", tuning={"sym_b": 1, "tile_chunk": chunk})
    _, R2, _ = run_forward(L, x)
    L.close()
    assert np.array_equal(R1, R2)
