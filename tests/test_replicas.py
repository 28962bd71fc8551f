"""Replica runs (one process per GPU, no data-path collective): the host-side
pieces with two gloo ranks on the CPU: joining the group from the launcher's
environment, the barrier, and the maximum of the ranks' times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    from paper_1808_01829_gb300 import replicas

    replicas.init("gloo")
    r, w, local = replicas.env()
    replicas.barrier()
    m = replicas.max_over_ranks(10.0 * (rank + 1) + 0.5)
    replicas.barrier()
    replicas.finalize()
    q.put((r, w, local, m))


def test_two_gloo_ranks_max_and_barrier():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == world and o[2] == o[0] for o in out)
    assert all(o[3] == 20.5 for o in out)  # the slowest rank's time


def test_single_rank_is_a_no_op():
    from paper_1808_01829_gb300 import replicas

    assert not replicas.active() or torch.distributed.get_world_size() == 1
    assert replicas.max_over_ranks(3.25) == 3.25
    replicas.barrier()
