"""Pair-tile ranges on one GPU (ladder_set_tile_range): two plans over
disjoint ranges write only their tiles' entries of R, and those entries are
bitwise the full plan's (same block-pair split), so the sum of the two
zero-initialised outputs is the full term; their energies add up to E_L."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"bf16x6": 1e-6, "ozaki": 1e-10}


@pytest.fixture(scope="module")
def lad():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return lad


@pytest.mark.parametrize("mode,two_pass", [("bf16x6", 1), ("bf16x6", 0), ("ozaki", 1), ("ozaki_sym", 1)])
def test_two_ranges_assemble_the_full_term(lad, mode, two_pass):
    """ozaki_sym: the error-free mode's symmetric-B form, where each range's
    plan forms all the distinct integral tiles and V+- of its own tiles."""
    import torch
    from paper_1810_08142_gb300 import partition as pt
    o, v, n, seed = 7, 41, 70, 14
    x = synthetic.make_inputs(o, v, n, seed)
    tau_h = oracle.tau(x.t1, x.t2)
    B, tau = to_dev(x.B), to_dev(tau_h)
    tun = ({"ksplit": 2, "sym_b": 1} if mode == "ozaki_sym" else {"ksplit": 2} if mode == "ozaki"
           else {"two_pass": two_pass, "ksplit": 2})
    mode = "ozaki" if mode == "ozaki_sym" else mode
    L = lad.Ladder(o, v, n, mode=mode, tuning=tun)
    ntiles = lad.ladder_tile_count(L.plan)
    assert ntiles == pt.tile_count(v)
    R_full = L.apply(B, tau)
    E_full = float(L.energy(R_full, to_dev(x.t2)).item())
    R_full = R_full.cpu().numpy()
    L.close()
    mid = ntiles * 2 // 5
    total = np.zeros_like(R_full)
    E_sum = 0.0
    for lo, hi in ((0, mid), (mid, ntiles)):
        Lr = lad.Ladder(o, v, n, mode=mode, tuning=tun, tiles=(lo, hi))
        assert lad.ladder_get_tuning(Lr.plan).ksplit == 2
        R = torch.full(tau.shape, 7.0, dtype=torch.float64, device="cuda")
        Lr.apply(B, tau, R)
        torch.cuda.synchronize()
        Lr.check_device()
        Rh = R.cpu().numpy()
        mask = np.broadcast_to(pt.pair_mask(v, lo, hi)[None, None], Rh.shape)
        assert np.all(Rh[~mask] == 7.0)                  # outside the range: untouched
        assert np.array_equal(Rh[mask], R_full[mask])  # inside: the full plan's bits
        slab = np.where(mask, Rh, 0.0)
        E_sum += float(Lr.energy(to_dev(slab), to_dev(x.t2)).item())
        total += slab
        Lr.close()
    assert np.array_equal(total, R_full)
    assert abs(E_sum - E_full) <= 1e-12 * abs(E_full)
    err = rel_err(total, oracle.ladder(x.B, tau_h))
    print("%s two_pass=%d: %d tiles in two ranges, rel err %.3e" % (mode, two_pass, ntiles, err))
    assert err < TOL[mode]


def test_tile_range_arguments(lad):
    L = lad.Ladder(4, 24, 96, mode="fp64")
    with pytest.raises(lad.LadderError):
        lad.ladder_tile_count(L.plan)                   # LADDER_ENOTSUP: FP64 has no tiles
    L.close()
    plan = lad.ladder_plan(4, 24, 96, lad.MODES["bf16x6"])
    n = lad.ladder_tile_count(plan)
    for lo, hi in ((-1, 2), (0, n + 1), (2, 2), (3, 1)):
        with pytest.raises(lad.LadderError):
            lad.ladder_set_tile_range(plan, lo, hi)
    lad.ladder_set_tile_range(plan, 0, 1)
    lad.ladder_destroy(plan)
    L = lad.Ladder(4, 24, 96, mode="bf16x6")
    with pytest.raises(lad.LadderError):
        lad.ladder_set_tile_range(L.plan, 0, 1)         # after ladder_set_workspace
    L.close()


@pytest.mark.parametrize("mode,extra", [("bf16x6", {"two_pass": 1}), ("bf16x6", {"two_pass": 1, "lambda_only": 1}),
                                        ("ozaki", {})])
def test_sequential_tile_ranges_match_one_range(lad, mode, extra):
    """tile_chunk: both passes and the unpack run over ranges of tiles one
    after the other (as a shape too large for one range does); R is bitwise
    the one-range result with the same block-pair split."""
    import torch
    o, v, n, seed = 7, 41, 70, 14
    x = synthetic.make_inputs(o, v, n, seed)
    B, tau = to_dev(x.B), to_dev(oracle.tau(x.t1, x.t2))
    outs = []
    for chunk in (0, 5, 1):
        L = lad.Ladder(o, v, n, mode=mode, tuning=dict(extra, ksplit=2, tile_chunk=chunk))
        assert lad.ladder_get_tuning(L.plan).tile_chunk == chunk
        outs.append(L.apply(B, tau).cpu().numpy())
        torch.cuda.synchronize()
        L.check_device()
        L.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
