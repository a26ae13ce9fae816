"""bench.py's multi-process path, on CPU with the gloo backend (world size 2):
replicas never exchange data; only the timing is reduced (max over ranks),
the whole-job rate counts every replica's steps, and only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 1.0 * rank])
    out[rank] = got
    ref = bench.run_reference_rank_gate()
    out[10 + rank] = ref
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == [11.0, 5.0, 1.0]
    assert out[10] is True and out[11] is False  # only rank 0 runs the reference arm


def test_single_process_identity_and_rate():
    import bench

    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    # 2 replicas x 16,384 envs x 1,000 steps in 100 ms
    assert bench.whole_job_rate(2, 16384, 1000, 100.0) == pytest.approx(2 * 16384 * 1000 / 0.1)
