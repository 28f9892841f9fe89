"""Multi-rank host logic on CPU (gloo, world size 2): sharding of independent
spectra, the max-over-ranks timing and the merge give the single-process
result."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1911_01353_gb300.ranks import max_over_ranks, merge, shard  # noqa: E402


def test_shard_covers_items_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _items():
    import synth
    return [(3000 + 517 * i, 100 + i, [synth.Signal(400.25 + 97 * i, 4.0, 20.0, 30.0, 0.5)]) for i in range(5)]


def _search(item):
    import oracle
    import synth
    n, seed, sigs = item
    F = synth.spectrum(n, seed, sigs)
    p = oracle.Params(6, 2, 20, 20, stages=(1, 2), thresh=(12.0, 16.0))
    return oracle.search(F, p).candidates


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = _items()
    mine = []
    for i in shard(len(items), rank, world):
        mine += [(i,) + tuple(c) for c in _search(items[i])]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        q.put((merge(gathered), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_equal_single_process():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items = _items()
    single = merge([[(i,) + tuple(c) for c in _search(items[i])] for i in range(len(items))])
    assert merged == single and len(single) >= len(items)
    assert t == 2.0
