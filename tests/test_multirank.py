"""The multi-process path on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank solves its own batch of candidates (weak
scaling: the same number of candidates per rank, no data-path collective)
and the job time is the slowest rank's.  These tests run that host logic
with the gloo backend, the FP64 oracle standing in for each rank's solve,
and check it against one process doing every rank's batch in turn.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WS = 2
ENTRIES = 24  # sequences of each rank's batch solved in the test


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_result(rank: int):
    """What one rank computes: its batch of the 4x4-RX urban block (the TX
    height differs per rank), solved and validated on the first ENTRIES
    sequences by the oracle."""
    sys.path.insert(0, ROOT)
    import bench

    sc, spec = bench.build_scene(rank, 4)
    table = oracle.enumerate_sequences(sc, 2, spec)
    n = min(len(table), ENTRIES) * sc.n_pairs
    _, ver = oracle.candidate_range(sc, table, 0, n, threads=1)
    return {"rank": rank, "candidates": len(table) * sc.n_pairs, "tx": sc.tx.tolist(),
            "valid": np.nonzero(ver.valid)[0].tolist(), "length": np.asarray(ver.length)[ver.valid.astype(bool)].tolist()}


def _worker(rank: int, port: int, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WS)
    try:
        sys.path.insert(0, ROOT)
        import bench

        # per-rank step times: the job's time is the slowest rank's
        slowest = bench.max_over_ranks(1.5 + rank)
        mine = _rank_result(rank)
        got = [None] * WS
        dist.all_gather_object(got, mine)
        if rank == 0:
            q.put({"slowest": slowest, "ranks": got})
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks():
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WS)]
    for p in procs:
        p.start()
    try:
        out = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    return out


def test_job_time_is_the_slowest_rank(two_ranks):
    assert two_ranks["slowest"] == 1.5 + (WS - 1)


def test_weak_scaling_batches_are_distinct_and_equal_in_size(two_ranks):
    ranks = sorted(two_ranks["ranks"], key=lambda r: r["rank"])
    assert [r["rank"] for r in ranks] == list(range(WS))
    assert len({r["candidates"] for r in ranks}) == 1
    assert ranks[0]["tx"] != ranks[1]["tx"]


def test_each_rank_matches_a_single_process_run(two_ranks):
    for r in two_ranks["ranks"]:
        want = _rank_result(r["rank"])
        assert r["valid"] == want["valid"]
        assert np.allclose(r["length"], want["length"], rtol=0, atol=1e-12)
        assert len(r["valid"]) > 0


def test_max_over_ranks_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5) == 2.5
