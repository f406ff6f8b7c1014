"""Host logic of the multi-process benchmark path, on CPU with the gloo
backend and two ranks: frames are independent units, so every rank of a
step decodes its own disjoint block of frames and the step time is the
maximum over ranks (no collective touches the decoded data)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        mine = [bench.frame_ids(k, rank, world, 96) for k in range(3)]
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        q.put((rank, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_max_time():
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, t in res:
        assert t == 1.5 + world - 1
        for k in range(3):
            blocks = [set(got[r][k]) for r in range(world)]
            assert all(len(b) == 96 for b in blocks)
            assert not blocks[0] & blocks[1]
            assert sorted(blocks[0] | blocks[1]) == list(range(k * 192, k * 192 + 192))
