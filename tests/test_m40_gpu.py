"""GPU parity of the 3^40-modulus generator against its oracle.

Every output must equal the oracle's bit for bit: states, truncated FP64
variates and FP32 variates, for any tile depth, block, chain count, buffer
count, layout and output alignment, at offsets across the period, and at the
rare smallest states whose variates need a third quotient digit.
"""
import numpy as np
import pytest

from m40_math import M40, P40, index_of_state

pytestmark = pytest.mark.gpu

ESZ = {"f64": 8, "f32": 4, "u64": 8}


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1206_1187_gb300 import rng
    return rng


def _bits(a):
    return a.view(np.int64 if a.itemsize == 8 else np.int32)


def _dev_bits(t):
    import torch
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu().numpy()


def _check(R, oracle_mod, a, off, n, dtype, tune=None, shift=0):
    """Generate into a canary-filled buffer at element offset `shift`."""
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "u64": torch.uint64}[dtype]
    esz = ESZ[dtype]
    raw = torch.full(((n + shift + 8) * esz,), 0x5A, dtype=torch.uint8, device="cuda")
    out = raw[shift * esz: (shift + n) * esz].view(tdt)
    R.generate40_at(a, off, n, dtype, out=out, tune=tune)
    torch.cuda.synchronize()
    want = oracle_mod.generate40(a, off, n, dtype)
    got = _dev_bits(out)
    bad = np.nonzero(got != _bits(want))[0]
    assert bad.size == 0, (a, off, n, dtype, tune, shift, bad[:8])
    host = raw.cpu().numpy()
    assert np.all(host[: shift * esz] == 0x5A) and np.all(host[(shift + n) * esz:] == 0x5A)


TUNES = [None,
         dict(depth=15, block=64, chains=1),
         dict(depth=31, block=96, chains=1),
         dict(depth=31, block=128, chains=2),
         dict(depth=7, block=32),
         dict(depth=63, block=128, chains=2, buffers=2),
         dict(depth=1, block=96),
         dict(layout="direct", block=64),
         dict(depth=31, block=512, chains=2, buffers=1, grid=7)]


@pytest.mark.parametrize("dtype", ["f64", "f32", "u64"])
def test_matches_the_oracle_for_every_tuning(R, oracle_mod, dtype):
    extra = ([dict(depth=44, block=64, grid=5), dict(depth=44, block=1024),
              dict(depth=44, block=512, buffers=2)] if dtype == "f32" else [])
    for k, tune in enumerate(TUNES + extra):  # 44-deep runs: FP32 on one chain only
        for a, off, n in [(M40 + 100, 0, 1), (2 ** 64 - 1, 12345, 31 * 32 * 5 + 17),
                          (M40 + 987654321, 2 ** 40 + 7, 100003)]:
            _check(R, oracle_mod, a, off, n, dtype, tune, shift=k % 3)


def test_heads_tails_and_small_sizes(R, oracle_mod):
    a = M40 + 4242
    for n in (2, 3, 31, 32, 33, 992, 993, 31 * 32 * 3 - 1, 44 * 32 * 2 + 5):
        for shift in (0, 1, 2, 3):
            _check(R, oracle_mod, a, 77, n, "f64", dict(depth=31, block=64), shift)
            _check(R, oracle_mod, a, 77, n, "f32", dict(depth=15, block=64, chains=2), shift)
            _check(R, oracle_mod, a, 77, n, "f32", None, shift)  # 44-deep one-product runs


def test_offsets_across_the_period(R, oracle_mod):
    a = M40 + 100
    for off in (P40 - 3000, P40 // 2 - 17, 2 ** 63 + 5, 2 ** 64 - 5000):
        _check(R, oracle_mod, a, off, 20000, "f64", dict(depth=15, block=128))
        _check(R, oracle_mod, a, off, 4000, "u64")


def test_smallest_states(R, oracle_mod):
    """States 1, 2, 4, ... below 3^40/2^53 give variates below 2^-53 (a zero
    first quotient); each is placed inside tiles, at tile edges, in the head
    and in the tail of a call."""
    a = M40 + 100
    for z in (1, 2, 4, 5, 1348, 1349, 1351, M40 - 1):
        i = index_of_state(a, z)
        for lead, n, tune in [(40, 81, None), (5, 3000, dict(depth=31, block=32)),
                              (31 * 32 - 1, 31 * 32 * 4, dict(depth=31, block=32, chains=2)),
                              (16, 1000, dict(depth=15, block=64, chains=1)),
                              (0, 7, dict(layout="direct", block=1))]:
            off = (i - lead) % P40
            for dtype in ("f64", "f32", "u64"):
                _check(R, oracle_mod, a, off, n, dtype, tune, shift=1)
        v = R.generate40_at(a, i, 1, "f64").cpu().numpy()
        assert v[0] == oracle_mod.to_f64_40(z) and v[0] > 0.0


def test_oversized_tiles_shrink_the_block_by_whole_warps(R, oracle_mod):
    """Tiles too large for the default block's shared memory shrink the block
    in whole warps until they fit, and the output is unchanged."""
    import torch
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin",
                    232448)
    for dtype in ("f64", "f32"):
        for tune in (dict(depth=255, buffers=2), dict(depth=127, buffers=2),
                     dict(depth=63, buffers=2)):
            r = R.resolve_tune40(1 << 20, dtype, tune)
            assert r["block"] >= 32 and r["block"] % 32 == 0, (tune, r)
            smem = r["block"] // 32 * r["buffers"] * 32 * r["depth"] * ESZ[dtype]
            assert smem <= optin, (tune, r)
            _check(R, oracle_mod, M40 + 31337, 99, 32 * tune["depth"] * 3 + 77, dtype, tune)


def test_bad_arguments(R):
    with pytest.raises(R.RNGError) as e:
        R.generate40_at(M40 + 99, 0, 10)
    assert e.value.status == 2
    for tune in (dict(step="barrett"), dict(depth=4), dict(block=33), dict(chains=3)):
        with pytest.raises(R.RNGError) as e:
            R.generate40_at(M40 + 100, 0, 10, tune=tune)
        assert e.value.status == 1
    # depth 44 is FP32 on one chain only
    for dtype, tune in (("f64", dict(depth=44)), ("u64", dict(depth=44)),
                        ("f32", dict(depth=44, chains=2)), ("f32", dict(depth=36))):
        with pytest.raises(R.RNGError) as e:
            R.generate40_at(M40 + 100, 0, 10, dtype, tune=tune)
        assert e.value.status == 1, (dtype, tune)


def test_full_size_sampled(R, oracle_mod):
    """The 2^28-variate FP64 call in its default launch: first and last 4096
    variates and 8192 random positions against the oracle."""
    import torch
    a, n = M40 + 12345, 1 << 28
    out = R.generate40_at(a, 0, n, "f64")
    torch.cuda.synchronize()
    rnd = np.random.default_rng(40)
    idx = np.unique(np.concatenate([np.arange(4096), np.arange(n - 4096, n),
                                    rnd.integers(0, n, size=8192)])).astype(np.int64)
    got = _dev_bits(out[torch.from_numpy(idx).cuda()])
    want = _bits(oracle_mod.at40(a, idx.astype(np.uint64), "f64"))
    assert np.array_equal(got, want)
    del out
    for dtype in ("f32", "u64"):
        out = R.generate40_at(a, 0, n, dtype)
        torch.cuda.synchronize()
        iv = torch.int32 if dtype == "f32" else torch.int64
        got = out.view(iv)[torch.from_numpy(idx).cuda()].cpu().numpy()  # integer view
        assert np.array_equal(got, _bits(oracle_mod.at40(a, idx.astype(np.uint64), dtype))), dtype
        del out


def test_undecided_quotients(R, oracle_mod):
    """States whose quotient the fast estimate cannot decide (the next
    remainder within a few units of 3^40) force the exact redo of their run;
    placed inside tiles and in both chains of a lane."""
    a = M40 + 271828
    zs = []
    for shift in (53, 106):  # one step (single estimate) or two steps (pair estimate) ahead
        inv = pow(2 ** shift, -1, M40)
        zs += [(M40 - k) * inv % M40 for k in (1, 2, 4, 5, 1000, 2 ** 20 + 1)]
    for z in zs:
        i = index_of_state(a, z)
        for lead, n, tune in [(100, 5000, None), (3, 992 * 3, dict(depth=31, block=32, chains=2)),
                              (20, 992 * 3, dict(depth=31, block=32, chains=2)),
                              (7, 480 * 2, dict(depth=15, block=32, chains=1)),
                              (8, 480 * 2, dict(depth=15, block=32, chains=1)),
                              (30, 992 * 2, dict(depth=31, block=32, chains=1)),
                              (31, 992 * 2, dict(depth=31, block=32, chains=1))]:
            off = (i - lead) % P40
            for dtype in ("f64", "f32"):
                _check(R, oracle_mod, a, off, n, dtype, tune)


def test_fp32_runs_from_one_product_at_the_redo_threshold(R, oracle_mod):
    """One-chain FP32 runs are read from one product; a digit below 2^23 sends
    its run to the exact forward path.  States whose first 53-bit digit is
    just below, at and above 2^23 and 2^24 are placed at the first, a middle
    and the last element of a lane's run (the last element's field has zeros,
    not the next digit, below it), with the default and every compiled depth."""
    a = M40 + 4242
    zs = []
    for q in (2 ** 23 - 2, 2 ** 23 - 1, 2 ** 23, 2 ** 23 + 1, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1):
        z = -(-(q * M40) // 2 ** 53)        # the smallest state with this digit, if any
        while z % 3 == 0 or (z << 53) // M40 != q:
            z += 1
        assert (z << 53) // M40 == q
        zs.append(z)
    for z in zs:
        i = index_of_state(a, z)
        for k, n, tune in [(43, 1408 * 2, dict(depth=44, block=32, chains=1)),
                           (44 * 7 + 3, 1408 * 2, dict(depth=44, block=32, chains=1)),
                           (30, 992 * 2, dict(depth=31, block=32, chains=1)),
                           (0, 992 * 2, dict(depth=31, block=32, chains=1)),
                           (31 * 5 + 17, 992 * 2, dict(depth=31, block=32, chains=1)),
                           (14, 480 * 2, dict(depth=15, block=32, chains=1)),
                           (31 * 40 + 30, 5000, None),
                           (31 * 3 + 30, 992 * 2, dict(depth=31, block=32, chains=2))]:
            off = (i - k) % P40
            _check(R, oracle_mod, a, off, n, "f32", tune)


def test_fp32_one_product_runs_equal_the_backward_step_at_full_size(R, oracle_mod):
    """2^28 FP32 variates of the 3^40 stream from the default one-product runs
    and from the backward step on two chains: every element identical, and a
    sample equal to the oracle."""
    import torch
    a, n = M40 + 12345, 1 << 28
    one = R.generate40_at(a, 0, n, "f32")
    back = R.generate40_at(a, 0, n, "f32", tune=dict(depth=31, chains=2))
    torch.cuda.synchronize()
    assert torch.equal(one.view(torch.int32), back.view(torch.int32))
    idx = np.random.default_rng(4040).integers(0, n, size=4096).astype(np.int64)
    got = one.view(torch.int32)[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(got, _bits(oracle_mod.at40(a, idx.astype(np.uint64), "f32")))
