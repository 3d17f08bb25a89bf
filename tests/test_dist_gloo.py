"""The N>1 path on CPU: two gloo ranks split independent stacks and reduce
their timings (maximum over ranks); no collective touches the data."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2211_00645_gb300 import dist as pdist  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_items, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(pdist.shard(n_items, rank, world))
        pdist.barrier()
        t = pdist.max_over_ranks(10.0 + rank)
        q.put((rank, mine, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_items", [7, 8, 1])
def test_two_ranks_shard_and_max(n_items):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_items, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    items = out[0][1] + out[1][1]
    assert sorted(items) == list(range(n_items))      # every stack exactly once
    assert all(t == 11.0 for _, _, t in out)          # max over ranks


def test_shard_balanced():
    for n in range(0, 20):
        for w in range(1, 6):
            sizes = [len(pdist.shard(n, r, w)) for r in range(w)]
            assert sum(sizes) == n and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pdist.shard(4, 2, 2)


def test_max_without_group():
    assert pdist.max_over_ranks(3.5) == 3.5
