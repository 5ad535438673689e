"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) take distinct
seeded right-hand sides (replicas, no data-path collective) and agree on the
max-over-ranks step time; only rank 0 runs and prints the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import afi_workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = W.config("C1-small")
    c = W.body_force_coeffs(prob, seed=bench.replica_seed(rank))
    mx = bench.reduce_max(10.0 * (rank + 1), world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, float(c[0].sum())))


def test_two_gloo_ranks_replicas_and_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    assert res[0][2] != res[1][2]          # different right-hand sides per rank


def test_reference_arm_only_on_rank_zero(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
