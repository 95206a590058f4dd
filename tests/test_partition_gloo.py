"""The multi-GPU partition of one molecule's term (host side) on CPU: pair
tiles split over ranks cover every entry of R exactly once, and two gloo
ranks that each hold their tiles' entries of R (zero elsewhere) assemble the
whole term and E_L by one all-reduce.  The ranks' slabs come from the plain
FP64 oracle masked to their tiles, standing in for the GPU plans of
ladder_set_tile_range (whose tiles the GPU test compares bit for bit)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_enumeration_matches_the_shape():
    from paper_1810_08142_gb300 import partition as pt
    for v in (5, 16, 17, 24, 41, 120, 400):
        vp = (v + 15) // 16 * 16
        n = pt.tile_count(v)
        assert n == sum(vp // 8 - 2 * i for i in range(vp // 16))
        blocks = [pt.tile_blocks(v, t) for t in range(n)]
        assert len(set(blocks)) == n
        assert all(2 * iA <= jB < vp // 8 for iA, jB in blocks)


@pytest.mark.parametrize("v,world", [(41, 2), (41, 3), (120, 4), (24, 5), (17, 2)])
def test_ranges_cover_every_entry_once(v, world):
    from paper_1810_08142_gb300 import partition as pt
    n = pt.tile_count(v)
    ranges = [pt.partition_tiles(n, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    assert max(h - l for l, h in ranges) - min(h - l for l, h in ranges) <= 1
    count = sum(pt.pair_mask(v, l, h).astype(int) for l, h in ranges)
    assert np.array_equal(count, np.ones((v, v), dtype=int))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import synthetic
    from paper_1810_08142_gb300 import partition as pt
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = synthetic.make_inputs(7, 41, 70, 14)
    tau = oracle.tau(x.t1, x.t2)
    R_full = oracle.ladder(x.B, tau)
    lo, hi = pt.partition_tiles(pt.tile_count(x.v), world, rank)
    mask = pt.pair_mask(x.v, lo, hi)
    slab = np.where(mask[None, None], R_full, 0.0)       # this rank's entries only
    E_part = oracle.energy(slab, x.t2)                   # its share of E_L
    R = torch.from_numpy(slab.copy())
    pt.assemble(R)
    E = torch.tensor([E_part], dtype=torch.float64)
    dist.all_reduce(E)
    cover = torch.from_numpy(mask.astype(np.int32))
    dist.all_reduce(cover)
    dist.destroy_process_group()
    out.put((rank, bool(np.array_equal(R.numpy(), R_full)), float(E.item()), oracle.energy(R_full, x.t2),
             int(cover.min().item()), int(cover.max().item())))


def test_two_gloo_ranks_assemble_R_and_E_L():
    mp = pytest.importorskip("torch.multiprocessing")
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    for rank, same, E, E_full, cmin, cmax in sorted(q.get(timeout=10) for _ in range(2)):
        assert same                                       # disjoint slabs add up exactly
        assert (cmin, cmax) == (1, 1)                     # every entry owned by one rank
        assert abs(E - E_full) <= 1e-13 * abs(E_full)
