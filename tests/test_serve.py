"""Host-side logic of the request loop: the arena allocator (CPU only)."""
import numpy as np

from paper_2604_27325_gb300.serve import Arena


def test_arena_first_fit_and_coalescing():
    a = Arena(1000)
    x = a.alloc(100)
    y = a.alloc(201)  # padded to 204
    z = a.alloc(300)
    assert (x, y, z) == (0, 100, 304)
    assert a.alloc(500) is None
    a.free(y, 201)
    assert a.alloc(150) == 100  # first fit reuses the hole
    a.free(100, 150)
    a.free(x, 100)
    a.free(z, 300)
    assert a.used == 0 and a.free_off == [0] and a.free_len == [1000]


def test_arena_random_traffic_never_overlaps():
    rng = np.random.default_rng(0)
    a = Arena(1 << 16)
    live = {}
    for step in range(5000):
        if live and rng.random() < 0.5:
            k = list(live)[rng.integers(len(live))]
            a.free(k, live.pop(k))
        else:
            sz = int(rng.integers(1, 2000))
            o = a.alloc(sz)
            if o is not None:
                live[o] = sz
        spans = sorted((o, o + (s + 3) // 4 * 4) for o, s in live.items())
        assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))
        assert a.used == sum((s + 3) // 4 * 4 for s in live.values())
        assert all(0 <= o and e <= a.capacity for o, e in spans)
