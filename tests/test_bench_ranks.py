"""The benchmark's multi-GPU bookkeeping on CPU: two gloo ranks, each a replica rendering its own
frames (weak scaling, no collective on the data path); the job time is the slowest rank's and the
frame count is the sum over ranks."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank
    e2e = 2.0 + rank
    q.put((rank, bench.combine_ranks(ms, e2e, 240, world, "cpu")))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_slowest_time_and_all_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert out[r] == (150.0, 3.0, 480)


def test_single_rank_passes_through():
    import bench
    assert bench.combine_ranks(12.5, 1.0, 240, 1) == (12.5, 1.0, 240)
