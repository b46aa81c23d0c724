"""The multi-process path of bench.py (one process per GPU, independent tanks,
replicas): rank bookkeeping from the torchrun environment, barriers and the
maximum over ranks of a timing, exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    slowest = r.max(10.0 + 2.5 * rank, "cpu")      # each rank's own timing; the job takes the slowest
    r.barrier()
    out.put((r.rank, r.local, r.world, slowest))
    r.close()


def test_two_gloo_ranks_take_the_max_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, out)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, l, w) for r, l, w, _ in res] == [(0, 0, 2), (1, 1, 2)]
    assert all(m == pytest.approx(12.5) for *_, m in res)


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    r = bench.Ranks("gloo")
    assert (r.world, r.rank, r.local, r.dist) == (1, 0, 0, None)
    assert r.max(3.25, "cpu") == 3.25
    r.barrier()
    r.close()
