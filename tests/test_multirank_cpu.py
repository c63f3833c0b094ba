"""The N > 1 path on CPU with two gloo ranks: each rank's share of the sweep
is distinct and the shares cover the finer sweep; the job time is the
slowest rank's.  No data-path collective exists (independent lattices)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        from paper_1410_2569_gb300 import inputs
        mine = [(c["fsi"], round(c["gw"], 12), c["ratio"]) for c in inputs.sweep_cases(ws, rank)]
        everyone = [None] * ws
        dist.all_gather_object(everyone, mine)
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        if rank == 0:
            q.put((everyone, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_sweep():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    everyone, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1410_2569_gb300 import inputs
    a, b = set(everyone[0]), set(everyone[1])
    assert len(a) == len(b) == 72 and not (a & b)
    full = {(c["fsi"], round(c["gw"], 12), c["ratio"]) for r in range(ws)
            for c in inputs.sweep_cases(ws, r)}
    assert a | b == full and len(full) == 144
    assert t == 2.0  # max over ranks


def test_single_rank_sweep_is_the_72_case_sweep():
    from paper_1410_2569_gb300 import inputs
    cases = inputs.sweep_cases()
    assert len(cases) == 72
    assert sorted({c["fsi"] for c in cases}) == ["density", "modified", "psi"]
    assert {c["ratio"] for c in cases} == {1.0, 10.0}
