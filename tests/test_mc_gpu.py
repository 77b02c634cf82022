"""GPU parity of the fused Monte-Carlo consumer against the oracle.

Per block: the hit count is an integer, and sum / sum of squares are exactly
rounded sums, so all three must match the oracle bit for bit for any launch
shape.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 3 ** 33


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng
    return rng


def _run(R, a, nblocks, length, block0=0, tune=None):
    import torch
    total, hits, s1, s2 = R.consume_mc(a, nblocks, length, block0=block0, tune=tune)
    torch.cuda.synchronize()
    return (int(total.cpu().view(torch.int64)[0]), hits.view(torch.int64).cpu().numpy(),
            s1.cpu().numpy(), s2.cpu().numpy())


@pytest.mark.parametrize("conv", ["int", "fp64"])
@pytest.mark.parametrize("length", [2, 4, 62, 64, 66, 1000, 4076, 4096, 4176, 8194])
def test_small_blocks_match_the_oracle(R, oracle_mod, length, conv):
    a = M + 100
    nblocks = 37
    total, hits, s1, s2 = _run(R, a, nblocks, length, tune=R.make_tune(conv=conv))
    oh, o1, o2 = oracle_mod.mc(a, length, np.arange(nblocks))
    assert np.array_equal(hits, oh.astype(np.int64))
    assert np.array_equal(s1.view(np.int64), o1.view(np.int64))
    assert np.array_equal(s2.view(np.int64), o2.view(np.int64))
    assert total == int(oh.sum())


def test_block_offset_and_launch_shape(R, oracle_mod):
    a, length = 2 ** 53, 2048
    block0 = 10 ** 9 + 7
    ref = _run(R, a, 64, length, block0=block0)
    for block, conv in ((32, "int"), (64, "fp64"), (256, "int"), (256, "fp64"), (96, "fp64")):
        got = _run(R, a, 64, length, block0=block0, tune=R.make_tune(block=block, conv=conv))
        assert got[0] == ref[0]
        for x, y in zip(got[1:], ref[1:]):
            assert np.array_equal(np.asarray(x).view(np.int64), np.asarray(y).view(np.int64))
    oh, o1, o2 = oracle_mod.mc(a, length, block0 + np.arange(64))
    assert np.array_equal(ref[1], oh.astype(np.int64))
    assert np.array_equal(ref[2].view(np.int64), o1.view(np.int64))
    assert np.array_equal(ref[3].view(np.int64), o2.view(np.int64))


def test_blocks_holding_tiny_variates(R, oracle_mod):
    """Blocks that contain variates below 2^-16 (which leave the branch-free
    conversion and make the warp redo their chunk exactly) still match; among
    them blocks where two lanes redo the same chunk.  Blocks of 4096 variates
    give each lane one chunk of 64 pairs (128 variates)."""
    a, length = M + 100, 4096
    states = oracle_mod.generate(a, 0, 1 << 24, "u64")
    tiny = np.nonzero(states < np.uint64(M >> 16))[0]
    lanes = {}
    for i in tiny:
        lanes.setdefault(int(i) // length, set()).add(int(i) % length // 128)
    blocks = sorted(lanes)
    multi = [b for b in blocks if len(lanes[b]) >= 2]
    assert len(blocks) >= 100 and len(multi) >= 2
    for b in blocks[:4] + multi[:3]:
        oh, o1, o2 = oracle_mod.mc(a, length, np.arange(b - 1, b + 2))
        for conv in ("int", "fp64"):
            total, hits, s1, s2 = _run(R, a, 3, length, block0=b - 1, tune=R.make_tune(conv=conv))
            assert np.array_equal(hits, oh.astype(np.int64)), (b, conv)
            assert np.array_equal(s1.view(np.int64), o1.view(np.int64)), (b, conv)
            assert np.array_equal(s2.view(np.int64), o2.view(np.int64)), (b, conv)


def test_bad_arguments(R):
    with pytest.raises(R.RNGError):
        R.consume_mc(M + 100, 4, 7)      # odd length
    with pytest.raises(R.RNGError):
        R.consume_mc(M + 99, 4, 8)       # seed below 3^33+100
    with pytest.raises(R.RNGError):
        R.consume_mc(M + 100, 4, 8, tune=R.make_tune(conv=7))


@pytest.mark.slow
def test_2_36_variates_subsample(R, oracle_mod):
    """2^36 variates in 2^20 blocks of 2^16, consumed without being stored;
    the 256 blocks b = 0 mod 4096 (2^24 variates) are checked against the
    oracle, and the total against the per-block counts."""
    a, nblocks, length = M + 100, 1 << 20, 1 << 16
    total, hits, s1, s2 = _run(R, a, nblocks, length)
    for conv in ("int", "fp64"):  # both forms of the squares on a sixteenth of the blocks
        t2, h2, u1, u2 = _run(R, a, nblocks // 16, length, tune=R.make_tune(conv=conv))
        assert np.array_equal(h2, hits[: nblocks // 16]), conv
        assert np.array_equal(u1.view(np.int64), s1[: nblocks // 16].view(np.int64)), conv
        assert np.array_equal(u2.view(np.int64), s2[: nblocks // 16].view(np.int64)), conv
    assert total == int(hits.sum())
    sub = np.arange(0, nblocks, 4096)
    oh, o1, o2 = oracle_mod.mc(a, length, sub)
    assert np.array_equal(hits[sub], oh.astype(np.int64))
    assert np.array_equal(s1[sub].view(np.int64), o1.view(np.int64))
    assert np.array_equal(s2[sub].view(np.int64), o2.view(np.int64))
    # pi/4 sanity on 2^35 pairs
    assert abs(total / (nblocks * length / 2) - np.pi / 4) < 1e-4


def test_exact_totals_of_one_call(R, oracle_mod):
    """The call's totals word array rounds to the oracle's exactly rounded sums
    over all its blocks, for any launch shape; the plain entry point's
    per-block outputs are unchanged by asking for totals."""
    import torch
    a, length, nblocks, block0 = M + 100, 2048, 48, 123457
    v = oracle_mod.generate(a, block0 * length, nblocks * length, "f64")
    want = (oracle_mod.exact_sum(v), oracle_mod.exact_sum(v * v))
    ref = _run(R, a, nblocks, length, block0=block0)
    for block, conv in ((128, "fp64"), (32, "int"), (256, "fp64")):
        total, hits, s1, s2, words = R.consume_mc_totals(
            a, nblocks, length, block0=block0, tune=R.make_tune(block=block, conv=conv))
        torch.cuda.synchronize()
        w = [int(x) for x in words.view(torch.int64).cpu().tolist()]
        assert all(0 <= x < (nblocks << 32) for x in w)
        assert R.mc_round_totals(w) == want, (block, conv)
        assert int(total.view(torch.int64).cpu()[0]) == ref[0]
        assert np.array_equal(hits.view(torch.int64).cpu().numpy(), ref[1])
        assert np.array_equal(s1.cpu().numpy().view(np.int64), ref[2].view(np.int64))
        assert np.array_equal(s2.cpu().numpy().view(np.int64), ref[3].view(np.int64))


def test_long_blocks_whose_sum_passes_2_128(R, oracle_mod):
    """Blocks of 2^25 variates: the exact sum of v * 2^105 of such a block is
    about 2^129, past 128 bits, so the block sum needs its third word.  Per
    block outputs and the call's totals match the oracle for both forms of
    the squares."""
    import torch
    a, length, block0 = M + 100, 1 << 25, 3
    oh, o1, o2 = oracle_mod.mc(a, length, block0 + np.arange(2))
    assert float(np.sum(o1)) * 2.0 ** 105 > 2.0 ** 128
    for conv in ("fp64", "int"):
        total, hits, s1, s2 = _run(R, a, 2, length, block0=block0, tune=R.make_tune(conv=conv))
        assert np.array_equal(hits, oh.astype(np.int64)), conv
        assert np.array_equal(s1.view(np.int64), o1.view(np.int64)), conv
        assert np.array_equal(s2.view(np.int64), o2.view(np.int64)), conv
        assert total == int(oh.sum())
    v = oracle_mod.generate(a, block0 * length, length, "f64")
    want = (oracle_mod.exact_sum(v), oracle_mod.exact_sum(v * v))
    _, _, _, _, words = R.consume_mc_totals(a, 1, length, block0=block0)
    torch.cuda.synchronize()
    w = [int(x) for x in words.view(torch.int64).cpu().tolist()]
    assert w[4] > 0  # the fifth piece of the sum is in use
    assert R.mc_round_totals(w) == want
