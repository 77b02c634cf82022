"""Pins for the CPU oracle (no GPU).

The paper prints no example outputs, so the oracle is pinned to what the
mathematics fixes, each check computed by a route that shares nothing with
the oracle's own arithmetic:

* the constants printed in Fig. 3 / Fig. 4 against their definitions;
* the period P = 2*3^32 of Sec. 1 as a closed form (order of 2 mod 3^33),
  and the oracle's states against it, including z(j + P/2) = m - z(j);
* Eq. 2 (skip-ahead) against Eq. 3 (iteration), the cross-check Sec. 1 names;
* the states against alpha_{2,3}'s series summed term by term (Eq. 1), which
  fixes the seed offset, the floor(3^33/2) factor and "step, then emit";
* the literal binary digits of alpha_{2,3} against the same generator built
  on a small modulus 3^M (Eq. 1 at sizes where the digits can be expanded);
* the FP64 variate against exact rational rounding of z * r3i;
* the FP32 variate against truncation of the FP64 bit pattern;
* the Monte-Carlo statistics against Python float arithmetic and Fractions.
"""
import math
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

M = 3 ** 33
P = 2 * 3 ** 32
H = M // 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, v = (s.strip() for s in line.split("=", 1))
        vals[k] = v
    return vals


def _f64_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _bits_f32(b: int) -> np.float32:
    return np.frombuffer(struct.pack("<I", b), dtype=np.float32)[0]


# ---------------------------------------------------------------- constants
def test_printed_constants_follow_their_definitions():
    g = _golden()
    m = int(g["m"])
    assert m == 3 ** 33
    k = m.bit_length()
    assert k == 53
    # Modified Barrett keeps Barrett's mu = floor(2^(2k)/m)
    assert int(g["mu"], 16) == (2 ** (2 * k)) // m
    # r3i is printed as 1.0/m; that quotient is the correctly rounded 3^-33
    assert 1.0 / float(m) == float(Fraction(1, m))
    assert float(g["r3i"].split("/")[1]) == float(m)
    assert int(g["mask53"], 16) == 2 ** 53 - 1
    assert int(g["two53"], 16) == 2 ** 53
    assert int(g["period"]) == 2 * 3 ** 32
    assert 3 ** 33 < 2 ** 53 < 2 * 3 ** 33


def test_order_of_two_is_the_period():
    # the multiplicative order of 2 mod 3^33 divides P; it is P itself iff no
    # maximal proper divisor P/q (q = 2, 3 the primes of P) is an exponent of 1
    assert pow(2, P, M) == 1
    assert pow(2, P // 2, M) == M - 1
    assert pow(2, P // 3, M) != 1
    # the step multiplier 2^53 has the same order because gcd(53, P) = 1
    assert math.gcd(53, P) == 1
    assert pow(2 ** 53, P // 2, M) != 1 and pow(2 ** 53, P // 3, M) != 1


def test_seed_range(oracle_mod):
    assert oracle_mod.seed_state(M + 99) == 0
    assert oracle_mod.seed_state(M + 100) != 0
    assert oracle_mod.seed_state(2 ** 53) != 0
    assert oracle_mod.seed_state(2 ** 53 + 1) == 0


def test_oracle_has_the_period(oracle_mod):
    rng = random.Random(1)
    for _ in range(50):
        a = rng.randint(M + 100, 2 ** 53)
        j = rng.randint(0, 2 ** 62)
        z = oracle_mod.seed_state(a, j)
        assert 0 < z < M
        assert oracle_mod.seed_state(a, j + P) == z
        # 2^(53*P/2) = (2^(P/2))^53 = (-1)^53 = -1 mod m
        assert oracle_mod.seed_state(a, j + P // 2) == M - z
        assert oracle_mod.seed_state(a, j + P // 3) != z


# ---------------------------------------------------------- skip == iterate
def test_skip_equals_iterate(oracle_mod):
    a = M + 100
    n = 20000
    states = oracle_mod.generate(a, 0, n, "u64")
    # Eq. 2 evaluated directly at every block start j reproduces Eq. 3
    idx = np.arange(n, dtype=np.uint64)
    assert np.array_equal(oracle_mod.at(a, idx, "u64"), states)
    for i in range(0, n, 997):
        assert oracle_mod.seed_state(a, i + 1) == int(states[i])
    # far-out blocks: iterate from a block seed and land on the direct value
    rng = random.Random(2)
    for _ in range(20):
        a = rng.randint(M + 100, 2 ** 53)
        j = rng.randint(0, 2 ** 60)
        z = oracle_mod.seed_state(a, j)
        for _ in range(1000):
            z = oracle_mod.step(z)
        assert z == oracle_mod.seed_state(a, j + 1000)


def test_step_is_times_two53_mod_m(oracle_mod):
    rng = random.Random(3)
    for z in [1, 2, M - 1, M - 2, H, H + 1] + [rng.randrange(1, M) for _ in range(2000)]:
        assert oracle_mod.step(z) == (z * 2 ** 53) % M


# ------------------------------------------- alpha_{2,3} (Eq. 1), two ways
def _alpha_series_state(n: int) -> int:
    """(sum over k=1..33 of (2^(n-3^k) mod 3^k) * 3^(33-k)) mod 3^33.

    {2^n alpha} = S/3^33 + tail, where the terms with 3^k > n form a tail
    below 2^-(3^34 - n); S is the exact fractional part of the first 33
    terms of alpha's series placed over the common denominator 3^33."""
    s = 0
    for k in range(1, 34):
        s += pow(2, n - 3 ** k, 3 ** k) * 3 ** (33 - k)
    return s % M


@pytest.mark.parametrize("a", [M + 100, M + 12345, 2 ** 53, 7 * 10 ** 15 + 3])
def test_states_are_windows_of_alpha(oracle_mod, a):
    count = 64
    states = oracle_mod.generate(a, 0, count, "u64")
    f64 = oracle_mod.generate(a, 0, count, "f64")
    for i in range(count):
        n = a + 53 * (i + 1)  # variate i holds binary digits n+1 .. n+53
        assert n <= 3 ** 34 - 100
        s = _alpha_series_state(n)
        assert s == int(states[i]), (a, i)
        # the FP64 variate is within 2^-52 of the digits it stands for
        assert abs(Fraction(float(f64[i])) - Fraction(s, M)) < Fraction(1, 2 ** 52)


@pytest.mark.parametrize("mexp", [5, 6, 7])
def test_literal_binary_digits_small_modulus(mexp):
    """Eq. 1 at modulus 3^mexp: the 53-bit windows of alpha's literal binary
    expansion equal floor(2^53 z / 3^mexp) of the same generator (Eq. 2, 3)
    for every window between 3^mexp + 100 and 3^(mexp+1) - 100.  This pins
    the reading the oracle uses (seed index -> digit position, step then
    emit, the floor(3^m/2) factor) where the digits can be written out."""
    mod = 3 ** mexp
    nbits = 3 ** (mexp + 1) + 200
    # floor(2^nbits * alpha): the terms with 3^k > nbits + 64 cannot reach
    # the last 64 kept bits
    frac = Fraction(0)
    k = 1
    while 3 ** k <= nbits + 64:
        frac += Fraction(1, 3 ** k * 2 ** (3 ** k))
        k += 1
    bits = math.floor(frac * 2 ** nbits)
    mism = 0
    checked = 0
    for n in range(mod + 100, 3 ** (mexp + 1) - 100 - 53):
        window = (bits >> (nbits - n - 53)) & (2 ** 53 - 1)  # digits n+1..n+53
        z = pow(2, n - mod, mod) * (mod // 2) % mod          # Eq. 2 at index n
        if window != (z * 2 ** 53) // mod:
            mism += 1
        checked += 1
        # the window 53 digits on is one step of Eq. 3 away
        assert pow(2, n + 53 - mod, mod) * (mod // 2) % mod == (z * 2 ** 53) % mod
    assert checked > 50
    assert mism == 0


# ------------------------------------------------------------ conversions
def _edge_states():
    rng = random.Random(4)
    zs = [1, 2, 3, 4, M - 1, M - 2, M - 3, H, H + 1, H - 1]
    # states whose variate sits next to a power of two (exponent changes)
    for e in range(0, 54):
        c = M >> e
        zs += [max(1, c - 1), max(1, c), min(M - 1, c + 1)]
    zs += [rng.randrange(1, M) for _ in range(20000)]
    return sorted(set(z for z in zs if 0 < z < M))


def test_f64_is_one_rounded_multiply(oracle_mod):
    r3i = 1.0 / 5559060566555523.0
    for z in _edge_states():
        want = float(Fraction(z) * Fraction(r3i))  # exact product, then RN
        got = oracle_mod.to_f64(z)
        assert _f64_bits(got) == _f64_bits(want), z
        assert 0.0 < got < 1.0


def test_f32_is_truncated_f64(oracle_mod):
    for z in _edge_states():
        b = _f64_bits(oracle_mod.to_f64(z))
        exp, mant = b >> 52, b & (2 ** 52 - 1)
        want = _bits_f32(((exp - 1023 + 127) << 23) | (mant >> 29))
        got = oracle_mod.to_f32(z)
        assert got.view(np.uint32) == want.view(np.uint32), z
        assert 0.0 < got < 1.0
        # rounding toward zero as exact rationals: got <= v < the next float up
        v = Fraction(float(oracle_mod.to_f64(z)))
        up = np.nextafter(np.float32(got), np.float32(1.0))
        assert Fraction(float(got)) <= v < Fraction(float(up)), z


def test_vector_paths_match_scalar_paths(oracle_mod):
    a = M + 777
    n = 3000
    st = oracle_mod.generate(a, 5, n, "u64")
    f64 = oracle_mod.generate(a, 5, n, "f64")
    f32 = oracle_mod.generate(a, 5, n, "f32")
    for i in range(0, n, 7):
        z = int(st[i])
        assert f64[i] == oracle_mod.to_f64(z)
        assert f32[i] == oracle_mod.to_f32(z)


def test_threaded_split_matches_single_thread(oracle_mod):
    a = M + 12345
    n = 100003
    for dt in ("f64", "f32", "u64"):
        one = oracle_mod.generate(a, 11, n, dt)
        for t in (1, 3, 8):
            assert np.array_equal(oracle_mod.generate_mt(a, 11, n, dt, t), one)


def test_strided_order_is_the_papers_indexing(oracle_mod):
    """The coalesced kernels of Sec. 2.2 write a thread's i-th variate at its
    start index plus i times the step (the number of threads); the oracle's
    strided order is checked against that indexing written out as loops."""
    a, j = M + 31337, 99
    for per, threads in ((4, 3), (8, 5), (16, 1), (1, 7)):
        n = per * threads
        seq = oracle_mod.generate(a, j, n, "u64")
        want = np.zeros(n, dtype=np.uint64)
        for t in range(threads):            # thread t: start index t, step `threads`
            for i in range(per):            # its i-th variate, number t*per + i
                want[t + i * threads] = seq[t * per + i]
        got = oracle_mod.generate_strided(a, j, n, "u64", per=per)
        assert np.array_equal(got, want), (per, threads)
        assert sorted(got.tolist()) == sorted(seq.tolist())  # a permutation
    with pytest.raises(ValueError):
        oracle_mod.generate_strided(a, j, 10, "f64", per=4)


# ------------------------------------------------------ Monte-Carlo consumer
def test_mc_matches_python_floats_and_fractions(oracle_mod):
    a = M + 100
    length = 4096
    blocks = [0, 1, 7, 4096]
    hits, s1, s2 = oracle_mod.mc(a, length, blocks)
    for t, b in enumerate(blocks):
        v = [float(x) for x in oracle_mod.generate(a, b * length, length, "f64")]
        h = sum(1 for j in range(0, length, 2) if v[j] * v[j] + v[j + 1] * v[j + 1] <= 1.0)
        assert int(hits[t]) == h
        assert s1[t] == float(sum(Fraction(x) for x in v))
        assert s2[t] == float(sum(Fraction(x * x) for x in v))


def test_exact_sum_rounds_ties_to_even(oracle_mod):
    cases = [
        [1.0, 2.0 ** -53],                        # tie -> 1.0 (even)
        [1.0, 2.0 ** -53, 2.0 ** -157],           # just above the tie -> up
        [1.0 + 2.0 ** -52, 2.0 ** -53],           # tie, odd mantissa -> up
        [0.5, 0.25, 2.0 ** -105, 2.0 ** -157],
        [2.0 ** -157] * 5,
        [0.9999999999999999] * 65536,
        [],
    ]
    rng = random.Random(5)
    cases.append([rng.random() for _ in range(5000)])
    cases.append([rng.random() ** 2 for _ in range(5000)])
    for c in cases:
        want = float(sum((Fraction(x) for x in c), Fraction(0)))
        assert oracle_mod.exact_sum(c) == want
