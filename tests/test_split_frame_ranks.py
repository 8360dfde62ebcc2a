"""The split frame's host logic on CPU: two gloo ranks each draw one part of a frame with the
oracle (the selected nodes with node index = rank mod 2), the product's reduce_partials sums them,
and the reduced image equals the oracle's whole frame bit for bit; the parts partition the
selected nodes."""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene():
    from paper_0811_2055_gb300 import synth
    p = synth.tiny(40000, seed=51)
    cam = synth.look_at((0.45, 0.55, -0.6), (0.5, 0.5, 0.5), width=160, height=120)
    return p, cam


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_0811_2055_gb300 import split
    p, cam = _scene()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=300)
    part, st, _, _ = O.render_lod_part(T, cam, O.rparams(lambda_px=6.0), rank, world)
    acc = torch.from_numpy(part.view(np.int64).copy())
    split.reduce_partials(acc)
    q.put((rank, st, acc.numpy().view(np.uint64).copy()))
    dist.destroy_process_group()


def test_two_ranks_sum_their_parts_to_the_whole_frame():
    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in range(2):
        r, st, img = q.get(timeout=180)
        out[r] = (st, img)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, cam = _scene()
    T = O.build_tree(p.xyz, p.mass, p.h, seed=1, n_max=300)
    rp = O.rparams(lambda_px=6.0)
    whole, st, _, _ = O.render_lod(T, cam, rp)
    assert st == 0 and whole.sum() > 0
    for r in (0, 1):
        assert out[r][0] == 0
        assert np.array_equal(out[r][1], whole)
    # each part draws its own nodes: neither part alone is the frame
    a = O.render_lod_part(T, cam, rp, 0, 2)[0]
    b = O.render_lod_part(T, cam, rp, 1, 2)[0]
    assert a.sum() > 0 and b.sum() > 0 and np.array_equal(a + b, whole)


def test_part_of_partitions_node_indices():
    from paper_0811_2055_gb300 import split
    for n in (1, 2, 3, 8):
        parts = [split.part_of(i, n) for i in range(1000)]
        assert set(parts) == set(range(n)) and all(parts[i] == i % n for i in range(1000))
