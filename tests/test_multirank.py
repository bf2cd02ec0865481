"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

Ranks run independent replicas; the job time is the max over ranks and the
whole-job ms/frame divides it by all ranks' frames.  The reference arm runs
on rank 0 only; other ranks exit without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.aggregate_max([1.0 + rank, 10.0 * (rank + 1)], world)
    frame = bench.per_frame(got[0], 5, world)
    r, w, l = bench.dist_setup(world)

    class A:
        gpus, steps, warmup, workload = world, 1, 0, "disks64"
    printed = None
    if rank != 0:
        import io
        import contextlib
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(A())
        printed = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, frame, (r, w, l), printed))


def test_two_rank_aggregation_gloo():
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
    for rank, got, frame, ids, printed in res:
        assert got == [2.0, 20.0]            # max over ranks
        assert frame == 2.0 / (5 * 2)        # all ranks' frames in the max time
        assert ids == (rank, 2, rank)
        if rank == 1:
            assert printed == ""             # the reference arm prints on rank 0 only
