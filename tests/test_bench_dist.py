"""bench.py's multi-rank path on CPU: two gloo ranks (spawned processes) run the host logic
of `--gpus 2` replicas -- the problem built by rank 0 before the others read it, the timed
region reduced to the slowest rank, the whole-job value over all ranks' columns -- and the
reference arm does no work on ranks other than 0.  No GPU and no data-path collective."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as td
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, _ = bench.dist()
        P = bench.load_problem("plate_tiny", r, w)
        ms = 100.0 + 50.0 * r                      # the ranks' timed regions differ
        m = bench.max_over_ranks(ms, w)
        q.put((r, w, m, bench.replica_value(8, 3, w, m), P.n))
    finally:
        td.destroy_process_group()


def test_two_gloo_replicas_reduce_to_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0]
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 150.0 for g in got)                        # max over ranks, on every rank
    assert all(g[3] == pytest.approx(8 * 3 * 2 / 0.150) for g in got)   # all ranks' columns / slowest time
    assert got[0][4] == got[1][4]                                 # same problem on both ranks


def test_reference_arm_idle_on_other_ranks(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "load_problem", lambda *a: pytest.fail("rank 1 must not build the problem"))
    assert bench.run_reference(None) is None      # returns before it reads its arguments
    assert capsys.readouterr().out == ""
