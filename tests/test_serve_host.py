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
