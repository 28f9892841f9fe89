"""Host logic of the server (no device): admission, batch choice, the
arrival trace and the request cost."""
import numpy as np

from paper_1911_01353_gb300 import serve


def req(k, n, zs=50, ws=0, arrival=0.0):
    return serve.Request(k, np.zeros(n, np.complex64), zs, ws, arrival=arrival)


def test_pick_batch_is_fifo_and_bounded():
    w = [req(0, 100), req(1, 300), req(2, 50), req(3, 10)]
    assert [r.rid for r in serve.pick_batch(w, 400, 8)] == [0, 1]     # 2 would exceed 400 bins
    assert [r.rid for r in serve.pick_batch(w, 10_000, 3)] == [0, 1, 2]
    assert serve.pick_batch(w, 99, 8) == []                            # the head does not fit
    assert [r.rid for r in serve.pick_batch(w, 100, 8)] == [0]
    assert serve.pick_batch([], 100, 8) == []


def test_admission_keeps_the_reserve():
    assert serve.admissible(1 << 20, (8 << 20) + 1000, 1000)
    assert not serve.admissible(1 << 20, (8 << 20) + 999, 1000)


def test_cells_of_counts_templates_and_cells():
    r = req(0, 1000, zs=4, ws=20)               # 5 z x 3 w templates at dz 2, dw 20
    assert serve.templates_in(4, 20, 2, 20) == 15
    assert serve.cells_of(r, 2, 20) == 2 * 1000 * 15
    assert serve.templates_in(300, 900, 2, 20) == 301 * 91


def test_poisson_trace_statistics():
    tr = serve.poisson_trace(20.0, 200.0, seed=5)
    t = np.array([x[0] for x in tr])
    assert np.all(np.diff(t) > 0) and t[-1] < 200.0
    assert abs(len(tr) / 200.0 - 20.0) < 3 * np.sqrt(20.0 / 200.0) + 0.5   # rate within a few sigma
    n = np.array([x[1] for x in tr])
    assert n.min() >= 1 << 18 and n.max() < 1 << 23
    lg = np.log2(n)
    assert abs(lg.mean() - 20.5) < 0.15                                   # log-uniform over [18, 23)
    assert {x[2] for x in tr} == {50, 100, 200, 300} and {x[3] for x in tr} == {0, 300, 600, 900}
    assert serve.poisson_trace(20.0, 200.0, seed=5) == tr                 # seeded


def test_summary_percentiles():
    rs = []
    for k in range(100):
        r = req(k, 1000, 0, 0, arrival=0.0)
        r.done = (k + 1) / 1000.0
        rs.append(r)
    s = serve.summary(rs, 2, 20)
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and abs(s["p99_ms"] - 99.01) < 1e-6
    assert s["cells"] == 100 * 2000 and abs(s["cells_per_s"] - 2000 * 100 / 0.1) < 1e-3


def test_next_batch_small_first_then_large_fifo():
    cost = lambda r: r.n                                     # noqa: E731  (cost = bins here)
    adm = [req(0, 500), req(1, 40), req(2, 900), req(3, 30), req(4, 20)]
    b, small = serve.next_batch(adm, cost, 50, 10_000, 8, 0, 2)
    assert small and [r.rid for r in b] == [1, 3, 4]         # small ones, oldest first, <= 2 x 50 work
    b, small = serve.next_batch(adm, cost, 35, 10_000, 8, 0, 2)
    assert small and [r.rid for r in b] == [3, 4]
    big = [req(0, 500), req(2, 900)]
    b, small = serve.next_batch(big, cost, 50, 10_000, 8, 0, 2)
    assert not small and [r.rid for r in b] == [0]           # large ones one batch at a time, oldest first
    assert serve.next_batch(big, cost, 50, 10_000, 8, 2, 2) == ([], False)   # max_large running
    b, small = serve.next_batch(adm, cost, 50, 10_000, 1, 0, 2, fifo=True)
    assert not small and [r.rid for r in b] == [0]           # plain form: the oldest, whatever its size


def test_pick_batch_cell_limit():
    cost = lambda r: r.n                                     # noqa: E731
    w = [req(0, 60), req(1, 30), req(2, 20)]
    assert [r.rid for r in serve.pick_batch(w, 1000, 8, 90, cost)] == [0, 1]
    assert [r.rid for r in serve.pick_batch(w, 1000, 8, 10, cost)] == [0]   # the first is always taken
