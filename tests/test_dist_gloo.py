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


def test_xshard_bounds():
    """Column ranges are contiguous, in rank order, cover every column once,
    start on 16-byte (8-column) boundaries and are balanced in 8-column
    blocks."""
    for n in (0, 1, 7, 8, 9, 136, 264, 2047, 2048):
        for w in (1, 2, 3, 4, 8):
            rs = [pdist.xshard(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            assert all(a % 8 == 0 or a == b == n for a, b in rs)
            blocks = [-(-(b - a) // 8) for a, b in rs]
            assert max(blocks) - min(blocks) <= 1
    with pytest.raises(ValueError):
        pdist.xshard(16, 2, 2)


def _xshard_worker(rank, world, port, q):
    """Each rank projects its own x-columns of one stack with the FP64
    oracle; the concatenation of the parts is the whole stack's view."""
    import numpy as np

    import opm_synth
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shape = (12, 10, 52, 35.0, 0.3, 0.1)
        R = opm_synth.raw_stack(opm_synth.StackConfig("x", *shape, n_blobs=6, sigma=(1.0, 2.0),
                                                      amp=(200.0, 3000.0), seed=5)).astype(np.float64)
        x0, x1 = pdist.xshard(shape[2], rank, world)
        g = O.geometry(shape[0], shape[1], max(1, x1 - x0), *shape[3:])
        zmip, _, ymip, _ = O.project(R[:, :, x0:x1], g) if x1 > x0 else (np.zeros((g.ny, 0)), 0, np.zeros((g.nz, 0)), 0)
        zfull = pdist.gather_x(torch.from_numpy(np.ascontiguousarray(zmip)), shape[2], world)
        yfull = pdist.gather_x(torch.from_numpy(np.ascontiguousarray(ymip)), shape[2], world)
        gw = O.geometry(*shape)
        zref, _, yref, _ = O.project(R, gw)
        q.put((rank, bool(np.array_equal(zfull.numpy(), zref)), bool(np.array_equal(yfull.numpy(), yref))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_xshard_reassembles_the_view():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_xshard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out == [(0, True, True), (1, True, True)]
