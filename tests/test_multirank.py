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


# ---------------------------------------------------------------------------
# One spectrum split by template range: partial max-projections (packed) and
# statistics sums from the oracle's FFT route over each rank's templates, one
# MAX and one SUM all-reduce over gloo, then thresholds and peaks on rank 0.
# ---------------------------------------------------------------------------

def _split_params(mode):
    import oracle
    import synth
    wl = synth.small_single()
    if mode == "sigma":
        return wl, oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1, 2, 3), thresh_mode="sigma",
                                 thresh=(6.0, 6.0, 5.0))
    return wl, oracle.Params(wl.zmax, wl.dz, wl.wmax, wl.dw, stages=(1, 2), thresh=(8.0, 11.0))


def _split_worker(rank, world, port, mode, q):
    import numpy as np

    import oracle
    from paper_1911_01353_gb300.ranks import pack, reduce_split, template_range, unpack
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, p = _split_params(mode)
    Fn = oracle.normalise(wl.make(), p.norm_block)
    lo, hi = template_range(p.n_templates, rank, world)
    part = oracle.fft_search(Fn, p, fund=np.arange(lo, hi), L=2048)
    ms = [torch.from_numpy(pack(np.maximum(part.maxproj[H][0], 0.0), np.where(part.maxproj[H][1] < 0, 0,
                                                                              part.maxproj[H][1])).copy())
          for H in p.stages]
    sums = torch.tensor([[part.sums[H][k] for H in p.stages] for k in range(3)], dtype=torch.float64)
    reduce_split(ms, sums, dist)
    if rank == 0:
        out = {"M": {}, "cands": [], "theta": {}}
        for si, H in enumerate(p.stages):
            v, t = unpack(ms[si].numpy())
            s1, s2, n = (float(x) for x in sums[:, si])
            if p.thresh_mode == "sigma":
                mu = s1 / n
                th = np.float32(mu + p.thresh[si] * np.sqrt(max(0.0, s2 / n - mu * mu)))
            else:
                th = np.float32(p.thresh[si])
            out["M"][H] = (v, t)
            out["theta"][H] = th
            out["cands"] += [(H, int(c), int(t[c]), float(v[c])) for c in oracle.peaks(v, th)]
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["abs", "sigma"])
def test_split_by_template_range_equals_single_process(mode):
    """Two ranks, each with half of the bank's templates (and the rows of its
    fundamentals' harmonics, made locally): after the reductions the
    max-projections (values and argmax), thresholds and candidates equal the
    single-process search."""
    import numpy as np

    import oracle
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=600)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    wl, p = _split_params(mode)
    ref = oracle.search(wl.make(), p)
    assert got["cands"] == ref.candidates and len(ref.candidates) > 0
    for H in p.stages:
        M, arg = ref.maxproj[H]
        assert np.array_equal(got["M"][H][0], M)
        fund, S = ref.sums[H]
        S32 = np.sort(S.astype(np.float32), axis=0)
        tie = S32[-1] == S32[-2]
        assert np.array_equal(got["M"][H][1][~tie], arg[~tie])
        assert abs(float(got["theta"][H]) - float(ref.theta[H])) <= 1e-6 * float(ref.theta[H])


def test_template_ranges_partition_the_bank():
    from paper_1911_01353_gb300.ranks import pack, template_range, unpack
    import numpy as np
    for T in (1, 147, 12261):
        for world in (1, 2, 3, 8):
            rs = [template_range(T, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == T
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    v = np.array([0.0, 1.5, 1.5, 3.25], dtype=np.float32)
    t = np.array([7, 3, 9, 0])
    pk = pack(v, t)
    # equal values: the larger packed entry has the lower t
    assert pk[1] > pk[2]
    vv, tt = unpack(pk)
    assert np.array_equal(vv, v) and np.array_equal(tt, t)
    with pytest.raises(ValueError):
        pack(np.array([-1.0], np.float32), np.array([0]))
