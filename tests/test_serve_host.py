"""Host-side logic of the serving loop (no GPU): the pixel-slot arena that
implements admission by device memory, and the request stream."""
import numpy as np

from paper_2404_16221_b300 import synthetic as sy


def _arena():
    import importlib

    serve = importlib.import_module("paper_2404_16221_b300.serve")
    return serve.Arena


def test_arena_first_fit_and_merge():
    Arena = _arena()
    a = Arena(100)
    x = a.alloc(30)
    y = a.alloc(50)
    assert (x, y) == (0, 30)
    assert a.alloc(30) == -1  # only 20 left
    a.release(x, 30)
    assert a.used == 50
    z = a.alloc(25)
    assert z == 0
    a.release(y, 50)
    a.release(z, 25)
    assert a.free == [(0, 100)]  # fully merged


def test_arena_random_workload_never_overlaps():
    Arena = _arena()
    g = np.random.default_rng(0)
    a = Arena(10_000)
    live = {}
    for step in range(2000):
        if live and g.uniform() < 0.45:
            k = list(live)[g.integers(len(live))]
            s, n = live.pop(k)
            a.release(s, n)
        else:
            n = int(g.integers(1, 900))
            s = a.alloc(n)
            if s >= 0:
                for s2, n2 in live.values():
                    assert s + n <= s2 or s2 + n2 <= s
                assert s + n <= 10_000
                live[step] = (s, n)
        assert a.used == sum(n for _, n in live.values())


def test_request_stream_shape():
    t, H, W, eye, tgt = sy.request_stream(2000, 200.0, 1004)
    assert np.all(np.diff(t) >= 0) and t[0] == 0
    assert abs(len(t) / t[-1] - 200) < 20  # Poisson rate
    assert H.min() >= 64 and H.max() <= 1080 and W.min() >= 64 and W.max() <= 1920
    assert np.all(W >= np.minimum(H, 1920))


def _shares(reqs, budget, one_at_a_time=False, policy="fair"):
    from collections import deque

    from paper_2404_16221_b300 import serve

    class Eng:
        pass

    e = Eng()
    e.one_at_a_time, e.max_items, e.max_batch, e.policy = one_at_a_time, 4096, budget, policy
    return serve.ServeEngine._shares(e, deque(reqs))


def test_fair_share_water_filling():
    """Each batch: requests needing less than an equal share get all of it,
    the rest is split evenly; nothing beyond a request's need, nothing beyond
    the batch."""
    from paper_2404_16221_b300 import serve

    g = np.random.default_rng(5)
    for trial in range(200):
        n = int(g.integers(1, 12))
        reqs = [serve.Request(i, float(i), int(g.integers(1, 60)), int(g.integers(1, 60)), (0, 0, 0), (1, 1, 1))
                for i in range(n)]
        for r in reqs:
            r.next_pixel = int(g.integers(0, r.pixels))
        budget = int(g.integers(1, 4000))
        sh = dict((r.rid, t) for r, t in _shares(reqs, budget))
        need = {r.rid: r.pixels - r.next_pixel for r in reqs}
        assert sum(sh.values()) == min(budget, sum(need.values()))
        assert all(0 < t <= need[k] for k, t in sh.items())
        level = max(sh.values())
        for r in reqs:  # below the water level a request is served in full
            got = sh.get(r.rid, 0)
            assert got == need[r.rid] or got >= level - 1


def test_small_request_not_held_behind_a_large_one():
    from paper_2404_16221_b300 import serve

    big = serve.Request(0, 0.0, 1080, 1920, (0, 0, 0), (1, 1, 1))
    small = serve.Request(1, 0.1, 64, 64, (0, 0, 0), (1, 1, 1))
    sh = dict((r.rid, t) for r, t in _shares([big, small], 1 << 18))
    assert sh[1] == small.pixels and sh[0] == (1 << 18) - small.pixels
    fifo = _shares([big, small], 1 << 18, one_at_a_time=True)
    assert [(r.rid, t) for r, t in fifo] == [(0, 1 << 18)]


def test_fifo_and_shortest_remaining_first():
    from paper_2404_16221_b300 import serve

    reqs = [serve.Request(0, 0.0, 100, 100, (0, 0, 0), (1, 1, 1)), serve.Request(1, 0.1, 10, 10, (0, 0, 0), (1, 1, 1)),
            serve.Request(2, 0.2, 20, 20, (0, 0, 0), (1, 1, 1))]
    assert [(r.rid, t) for r, t in _shares(reqs, 5000, policy="fifo")] == [(0, 5000)]
    assert [(r.rid, t) for r, t in _shares(reqs, 5000, policy="srpt")] == [(1, 100), (2, 400), (0, 4500)]
