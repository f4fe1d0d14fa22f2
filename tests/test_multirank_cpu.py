"""The N > 1 path of bench.py on CPU: two gloo ranks agree on the max-over-ranks
time and the summed work (the only collectives; every rank solves its own
replica), and ranks other than 0 leave the reference arm without work."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _ = bench.dist_env()
    d = bench.init_dist(w, "gloo")
    bench.barrier(d)
    mx = bench.max_over_ranks(d, 1.5 * (r + 1))
    sm = bench.sum_over_ranks(d, 10.0 * (r + 1))
    bench.barrier(d)
    d.destroy_process_group()
    q.put((r, mx, sm))


def test_two_gloo_ranks_reduce_time_and_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        r, mx, sm = q.get(timeout=120)
        out[r] = (mx, sm)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: (3.0, 30.0), 1: (3.0, 30.0)}


def test_replicas_draw_their_own_start_blocks():
    class P:
        def __init__(self, n):
            self.n = n
    a = bench.start_block([P(50), P(30)], 2, 1)
    b = bench.start_block([P(50), P(30)], 2, 1 + 1000)       # rank 1's seed offset
    assert a.shape == (2, 80) and not np.allclose(a, b)
    np.testing.assert_array_equal(a, bench.start_block([P(50), P(30)], 2, 1))


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse_args(["--impl", "reference"]))
    assert capsys.readouterr().out == ""
