"""The multi-rank host logic of bench.py on CPU: two gloo ranks run the
replica bookkeeping (barrier, max over ranks of the timed region, whole-job
value) that the GPU run uses with NCCL, and the reference arm does its work
on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo")
    assert (rep.world, rep.rank) == (world, rank)
    rep.barrier()
    local_ms = 10.0 + 5.0 * rank              # rank 1 is the slowest
    ms = rep.max(local_ms)
    value = rep.job_value(1e9, ms)            # 1e9 units per rank
    rep.barrier()
    rep.close()
    out.put((rank, ms, value))


def test_two_gloo_ranks_take_the_max_over_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 15.0                    # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1e9 / 15e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))
    args = type("A", (), {"workload": "small_o4_v24_n96", "steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args) == 0
    assert called == []


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rep = bench.Replicas("gloo")
    assert rep.dist is None and rep.world == 1
    assert rep.max(3.5) == 3.5
    assert rep.job_value(2e9, 4.0) == pytest.approx(2e9 / 4e-3)
