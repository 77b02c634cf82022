"""The fused consumer's exact totals (rng_consume_mc_totals) and their host
rounding (rng_mc_round_totals), the exchange of the paper's parallel split
(Sec. 1) when one sequence's blocks are spread over ranks.

No GPU here: the rounding of word arrays is checked against Python's exact
rational rounding (float(Fraction) rounds to nearest, ties to even), and two
gloo ranks each build the word array of their half of a block range from
the oracle's variates, add the arrays with one integer all-reduce, and round
-- which must equal the oracle's exactly rounded sums over the whole range.
"""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest

M = 3 ** 33
SUM_WORDS, SQ_WORDS = 5, 6


@pytest.fixture(scope="module")
def R():
    from paper_1206_1187_gb300 import _build
    _build.build()
    from paper_1206_1187_gb300 import rng
    return rng


def _value(words):
    return sum(int(w) << (32 * k) for k, w in enumerate(words))


def _pieces(x, nwords):
    return [(x >> (32 * k)) & 0xFFFFFFFF for k in range(nwords)]


def test_rounding_of_word_arrays_matches_exact_rationals(R):
    rnd = np.random.default_rng(5)
    for trial in range(3000):
        # words of any size below 2^52 (overlapping pieces, as after many blocks)
        bits = int(rnd.integers(1, 53))
        w = [int(rnd.integers(0, 1 << bits)) for _ in range(SUM_WORDS + SQ_WORDS)]
        if trial % 7 == 0:
            w[:SUM_WORDS] = [0] * SUM_WORDS
            w[int(rnd.integers(0, SUM_WORDS))] = int(rnd.integers(1, 1 << 20))
        s1, s2 = R.mc_round_totals(w)
        assert s1 == float(Fraction(_value(w[:SUM_WORDS]), 1 << 105)), w
        assert s2 == float(Fraction(_value(w[SUM_WORDS:]), 1 << 157)), w


def test_rounding_ties_go_to_even(R):
    for lead in (1 << 60, (1 << 60) + (1 << 8), (1 << 90) + (3 << 37)):
        top = lead.bit_length() - 1
        for low_bit in (0, 1):
            # a value exactly halfway between two doubles, kept bit even or odd
            x = lead | (low_bit << (top - 52)) | (1 << (top - 53))
            for extra in (0, 1):  # one more unit below: no longer a tie
                y = x + extra
                s1, _ = R.mc_round_totals(_pieces(y, SUM_WORDS) + [0] * SQ_WORDS)
                assert s1 == float(Fraction(y, 1 << 105))
                kept_odd = (y >> (top - 52)) & 1
                want_up = kept_odd == 1 or extra == 1  # a tie goes to the even neighbour
                base = (y >> (top - 52)) << (top - 52)
                assert s1 == float(Fraction(base + ((1 << (top - 52)) if want_up else 0),
                                            1 << 105))
    assert R.mc_round_totals([0] * 11) == (0.0, 0.0)
    with pytest.raises(ValueError):
        R.mc_round_totals([0] * 10)


def _block_words(oracle_mod, a, length, blocks):
    """The word array of the given blocks, from the oracle's variates: each
    block's exact sums as integers on the 2^-105 and 2^-157 grids, cut into
    32-bit pieces and added word by word (what the kernel's atomics do)."""
    words = [0] * (SUM_WORDS + SQ_WORDS)
    for b in blocks:
        v = oracle_mod.generate(a, int(b) * length, length, "f64")
        sq = v * v  # RN(v*v), one IEEE multiply each
        s = sum(int(Fraction(float(x)) * (1 << 105)) for x in v)
        q = sum(int(Fraction(float(x)) * (1 << 157)) for x in sq)
        for k, p in enumerate(_pieces(s, SUM_WORDS) + _pieces(q, SQ_WORDS)):
            words[k] += p
    return words


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, a, length, nblocks, result_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1206_1187_gb300 import rng
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = rank * nblocks // world, (rank + 1) * nblocks // world
    words = torch.tensor(_block_words(oracle, a, length, range(lo, hi)), dtype=torch.int64)
    dist.all_reduce(words, op=dist.ReduceOp.SUM)  # exact: every word stays below 2^63
    s1, s2 = rng.mc_round_totals(words.tolist())
    np.save(os.path.join(result_dir, f"m{rank}.npy"), np.array([s1, s2]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_merge_their_totals_exactly(tmp_path, oracle_mod, R):
    import torch.multiprocessing as mp
    a, length, nblocks, world = M + 100, 256, 12, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), a, length, nblocks, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    v = oracle_mod.generate(a, 0, nblocks * length, "f64")
    want = (oracle_mod.exact_sum(v), oracle_mod.exact_sum(v * v))
    for r in range(world):
        got = tuple(np.load(tmp_path / f"m{r}.npy"))
        assert got == want, (r, got, want)
    # the per-block sums alone, rounded first and then added, need not agree
    _, o1, _ = oracle_mod.mc(a, length, np.arange(nblocks))
    assert want[0] == pytest.approx(float(np.sum(o1)), rel=1e-14)
