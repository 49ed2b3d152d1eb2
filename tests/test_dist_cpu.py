"""The multi-GPU bench path on CPU: two gloo ranks, barrier + MAX reduction of
the timed region and the whole-job throughput formula (no GPU needed)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1411_0519_gb300 import dist as pd
    r, w, l = pd.init("gloo")
    pd.barrier()
    elapsed = 1.0 + 0.5 * r            # rank 1 is the slow one
    mx = pd.max_over_ranks(elapsed)
    rate = pd.job_throughput(w, 1000.0, mx)
    q.put((r, w, mx, rate))
    pd.finalize()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, mx, rate in out:
        assert w == 2 and mx == 1.5
        assert rate == pytest.approx(2 * 1000.0 / 1.5)


def test_single_process_needs_no_group():
    from paper_1411_0519_gb300 import dist as pd
    assert pd.max_over_ranks(3.0) == 3.0
    assert pd.job_throughput(1, 10.0, 2.0) == 5.0
