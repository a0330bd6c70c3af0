"""The replicas path of the benchmark (one process per GPU, the time taken
as the maximum over processes) on CPU: two gloo processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2312_10044_gb300 import replicas

    w, r, local = replicas.init("gloo")
    assert (w, r, local) == (world, rank, rank)
    replicas.barrier(w)
    t = replicas.max_over_ranks(1.0 + rank, w)  # rank k took 1 + k seconds
    out.put((rank, t, replicas.whole_job_rate(100.0, w, t)))
    replicas.finish(w)


def test_max_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the rate counts both replicas' work
    assert [r[1] for r in res] == [2.0, 2.0]
    assert [r[2] for r in res] == [100.0, 100.0]


def test_single_process_needs_no_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2312_10044_gb300 import replicas

    assert replicas.init("gloo") == (1, 0, 0)
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0
