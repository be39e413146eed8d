"""Multi-process host logic of the multi-GPU form, on CPU with gloo: the
frame shares of the ranks cover every frame exactly once, and the timing
reduction returns the slowest rank's time on every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2112_00821_b300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.frames_of_rank(11, rank, world)
        t = 0.010 * (rank + 1)                  # rank r "took" (r + 1) * 10 ms
        dist.barrier()
        tmax = shard.max_over_ranks(t)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, mine, tmax, gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_share_frames_and_agree_on_the_slowest_time(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, tmax, gathered in res:
        assert tmax == pytest.approx(0.010 * world)
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(11))
        assert mine == gathered[rank]


def test_single_process_helpers():
    from paper_2112_00821_b300 import shard
    assert shard.frames_of_rank(5, 0, 1) == [0, 1, 2, 3, 4]
    assert shard.frames_of_rank(5, 1, 2) == [1, 3]
    assert shard.max_over_ranks(0.25) == 0.25
    assert shard.whole_job_rate(100.0, 2.0, 4) == 200.0
    with pytest.raises(ValueError):
        shard.frames_of_rank(5, 2, 2)
