"""The serving pool's sub-allocator (host bookkeeping only, no GPU): random
allocate / free sequences checked against a plain Python first-fit model."""
import random

import pytest


@pytest.fixture(scope="module")
def R():
    from paper_1206_1187_gb300 import _build
    _build.build()
    from paper_1206_1187_gb300 import rng
    return rng


class FirstFit:
    """Address-ordered first fit with neighbour merging, written out plainly."""

    def __init__(self, cap, align):
        self.free = [[0, cap]]
        self.used = {}
        self.align = align

    def alloc(self, nbytes):
        need = (max(nbytes, 1) + self.align - 1) // self.align * self.align
        for i, (o, sz) in enumerate(self.free):
            if sz >= need:
                if sz == need:
                    self.free.pop(i)
                else:
                    self.free[i] = [o + need, sz - need]
                self.used[o] = need
                return o
        return None

    def release(self, o):
        sz = self.used.pop(o)
        self.free.append([o, sz])
        self.free.sort()
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1][1] += b
            else:
                merged.append([a, b])
        self.free = merged


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pool_matches_first_fit_model(R, seed):
    rnd = random.Random(seed)
    cap, align = 1 << 24, 256
    pool, model = R.Pool(cap, align), FirstFit(cap, align)
    live = []
    peak = 0
    for _ in range(4000):
        if live and rnd.random() < 0.45:
            o = live.pop(rnd.randrange(len(live)))
            pool.free(o)
            model.release(o)
        else:
            nb = int(2 ** rnd.uniform(0, 21))
            a, b = pool.alloc(nb), model.alloc(nb)
            assert a == b
            if a is not None:
                live.append(a)
        st = pool.stats()
        used = sum(model.used.values())
        peak = max(peak, used)
        assert st["in_use"] == used <= cap
        assert st["live"] == len(model.used)
        assert st["free_ranges"] == len(model.free)
        assert st["largest_free"] == max([s for _, s in model.free], default=0)
        # no two live ranges overlap
        spans = sorted((o, o + s) for o, s in model.used.items())
        assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))
    for o in live:
        pool.free(o)
    st = pool.stats()
    assert st["in_use"] == 0 and st["free_ranges"] == 1 and st["largest_free"] == cap
    assert st["peak"] == peak


def test_pool_rejects_bad_frees(R):
    pool = R.Pool(4096, 256)
    o = pool.alloc(100)
    with pytest.raises(R.RNGError):
        pool.free(o + 256)
    pool.free(o)
    with pytest.raises(R.RNGError):
        pool.free(o)
    assert pool.alloc(5000) is None


def test_pool_refuses_sizes_whose_alignment_would_wrap(R):
    # a pool near 2^64 bytes: rounding such a request up to the alignment
    # would pass 2^64 and must not come back as a tiny range
    cap = (1 << 64) - 1
    pool = R.Pool(cap, 256)
    assert pool.alloc(cap) is None
    assert pool.alloc((1 << 64) - 200) is None
    st = pool.stats()
    assert st["in_use"] == 0 and st["live"] == 0 and st["largest_free"] == cap
    o = pool.alloc(1 << 63)
    assert o == 0 and pool.stats()["in_use"] == 1 << 63
    pool.free(o)
