"""Pins for the oracle of the 3^40 modulus variant, against mathematics that
does not go through the oracle's code:

* the period 2*3^39 as the exact order of 2 (closed form), and the oracle's
  skip-ahead honouring it, including the half period that negates a state;
* skip-ahead (Eq. 2 at a + 53j) against iteration of Eq. 3;
* the states against alpha_{2,3}'s series summed term by term with 40 terms,
  which fixes the seed offset, the floor(3^40/2) factor and "step, then emit";
* the FP64 variate against exact rational bounds (the largest double not
  above z/3^40), at random states, the extreme states and states closest to
  doubles, and its digits against alpha's digits from the series;
* the FP32 variate against exact rational bounds (largest float32 not above
  z/3^40);
* the smallest states (variates below 2^-53), placed at known output indices
  with exact discrete logarithms.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

from m40_math import H40, M40, P40, dlog2, index_of_state


def test_order_of_two_is_the_period40():
    assert pow(2, P40, M40) == 1
    assert pow(2, P40 // 2, M40) == M40 - 1
    assert pow(2, P40 // 3, M40) != 1
    assert math.gcd(53, P40) == 1  # so outputs have the full period
    assert M40 < 2 ** 64 < 3 ** 41 - 100


def test_seed_range40(oracle_mod):
    assert oracle_mod.seed_state40(M40 + 99) == 0
    assert oracle_mod.seed_state40(M40 + 100) != 0
    assert oracle_mod.seed_state40(2 ** 64 - 1) != 0


def test_oracle40_has_the_period(oracle_mod):
    rnd = random.Random(40)
    for _ in range(20):
        a = rnd.randrange(M40 + 100, 2 ** 64)
        j = rnd.randrange(0, 2 ** 62)
        z = oracle_mod.seed_state40(a, j)
        assert 0 < z < M40 and z % 3 != 0
        assert oracle_mod.seed_state40(a, j + P40) == z
        # 53 * P/2 steps multiply by 2^(53 P/2) = (-1)^53 = -1
        assert oracle_mod.seed_state40(a, j + P40 // 2) == M40 - z


def test_skip_equals_iterate40(oracle_mod):
    rnd = random.Random(41)
    for a, j in [(M40 + 100, 0), (2 ** 64 - 1, 10 ** 6), (rnd.randrange(M40 + 100, 2 ** 64),
                                                         rnd.randrange(2 ** 60))]:
        z = oracle_mod.seed_state40(a, j)
        for k in range(1, 3001):
            z = oracle_mod.step40(z)
            if k in (1, 2, 3, 53, 1000, 3000):
                assert z == oracle_mod.seed_state40(a, j + k), (a, j, k)
    states = oracle_mod.generate40(M40 + 777, 5, 2000, "u64")
    ref = oracle_mod.at40(M40 + 777, np.arange(5, 2005, dtype=np.uint64), "u64")
    assert np.array_equal(states, ref)


def test_step40_is_times_two53_mod_m(oracle_mod):
    rnd = random.Random(42)
    zs = [1, 2, M40 - 1, M40 - 2, 2 ** 63, 2 ** 64 - 2 ** 11, H40, H40 + 1]
    zs += [rnd.randrange(1, M40) for _ in range(2000)]
    for z in zs:
        z %= M40
        if z == 0:
            continue
        assert oracle_mod.step40(z) == (z * 2 ** 53) % M40


def _alpha_series_state40(n: int) -> int:
    """(sum over k=1..40 of (2^(n-3^k) mod 3^k) * 3^(40-k)) mod 3^40: the
    exact fractional part of the first 40 terms of alpha's series, over the
    common denominator 3^40; the remaining terms are below 2^-(3^41 - n)."""
    return sum(pow(2, n - 3 ** k, 3 ** k) * 3 ** (40 - k) for k in range(1, 41)) % M40


@pytest.mark.parametrize("a", [M40 + 100, M40 + 12345, 2 ** 64 - 1, 15 * 10 ** 18 + 7])
def test_states40_are_windows_of_alpha(oracle_mod, a):
    count = 48
    states = oracle_mod.generate40(a, 0, count, "u64")
    for i in range(count):
        n = a + 53 * (i + 1)
        assert n <= 3 ** 41 - 100
        assert _alpha_series_state40(n) == int(states[i]), (a, i)


def _near_grid_states(count: int, rnd: random.Random):
    """States whose quotient z/3^40 lies closest to a double (just above or
    below it), over a spread of binades: where truncation and rounding part."""
    out = []
    for _ in range(count):
        e = rnd.randrange(1, 64)
        mant = rnd.randrange(2 ** 52, 2 ** 53)
        z = round(Fraction(mant, 2 ** (52 + e)) * M40)
        for d in (-1, 0, 1):
            if 0 < z + d < M40 and (z + d) % 3 != 0:
                out.append(z + d)
    return out


def _truncated_quotient(z: int) -> float:
    """The largest double not above z/3^40, from integer arithmetic: the 53
    digits of floor(z * 2^s / 3^40) from its leading one."""
    s = 53 + (M40.bit_length() - z.bit_length()) + 1
    q = (z << s) // M40                   # at least 2^53
    drop = q.bit_length() - 53
    return math.ldexp(q >> drop, drop - s)


def test_f64_40_is_the_truncated_quotient(oracle_mod):
    rnd = random.Random(43)
    zs = [1, 2, 4, 5, 7, 1349, 1350, M40 - 1, M40 - 2, H40, H40 + 1, 2 ** 63, 2 ** 53, 2 ** 53 + 1]
    zs += [2 ** k for k in range(64) if 2 ** k < M40]
    zs += [rnd.randrange(1, M40) for _ in range(3000)]
    zs += _near_grid_states(1000, rnd)
    for z in zs:
        if z % 3 == 0:
            continue
        v = oracle_mod.to_f64_40(z)
        assert v == _truncated_quotient(z), z
        # exact bounds: v <= z/m < next double above v
        assert Fraction(v) <= Fraction(z, M40) < Fraction(math.nextafter(v, 2.0)), z
    assert oracle_mod.to_f64_40(M40 - 1) == math.nextafter(1.0, 0.0)  # (0,1) stays open
    assert oracle_mod.to_f64_40(1) > 0.0
    # rounding to nearest would have reached 1.0 here
    assert (M40 - 1) / M40 == 1.0


def test_f64_40_digits_are_alpha_digits(oracle_mod):
    """The 53 significant digits of variate i are binary digits of alpha_{2,3}
    following position n = a + 53(i+1) (the series terms beyond 3^40 only
    reach digit 3^41 - n and later)."""
    a = M40 + 4242
    f64 = oracle_mod.generate40(a, 0, 16, "f64")
    for i in range(16):
        n = a + 53 * (i + 1)
        s = _alpha_series_state40(n)   # {2^n alpha} = s / 3^40 + tail
        v = float(f64[i])
        lead = -math.frexp(v)[1]       # v in [2^-(lead+1), 2^-lead)
        width = lead + 1 + 52
        digits = (s << width) // M40   # alpha's digits n+1 .. n+width
        assert Fraction(v) == Fraction(digits, 2 ** width), i


def test_f32_40_is_truncated_f64(oracle_mod):
    rnd = random.Random(44)
    zs = [1, 2, M40 - 1, M40 - 2] + [rnd.randrange(1, M40) for _ in range(3000)]
    zs += _near_grid_states(300, rnd)
    for z in zs:
        if z % 3 == 0:
            continue
        f = oracle_mod.to_f32_40(z)
        nxt = np.nextafter(f, np.float32(np.inf))
        assert Fraction(float(f)) <= Fraction(z, M40) < Fraction(float(nxt)), z
        assert 0.0 < float(f) < 1.0


def test_discrete_log_places_tiny_states(oracle_mod):
    """Outputs with the smallest states (variates below 2^-53, where the
    integer conversion needs three quotient digits) at exact indices."""
    a = M40 + 100
    for z in (1, 2, 4, 5, 1348, 1349, M40 - 1):
        i = index_of_state(a, z)
        got = oracle_mod.at40(a, np.array([i], dtype=np.uint64), "u64")
        assert int(got[0]) == z
        v = oracle_mod.at40(a, np.array([i], dtype=np.uint64), "f64")
        assert float(v[0]) == _truncated_quotient(z)
    assert pow(2, dlog2(5), M40) == 5


def test_vector_paths_match40(oracle_mod):
    a = M40 + 31337
    idx = np.arange(100, 600, dtype=np.uint64)
    for dt in ("f64", "f32", "u64"):
        assert np.array_equal(oracle_mod.generate40(a, 100, 500, dt), oracle_mod.at40(a, idx, dt))
    st = oracle_mod.generate40(a, 100, 500, "u64")
    f = oracle_mod.generate40(a, 100, 500, "f64")
    assert all(float(f[k]) == _truncated_quotient(int(st[k])) for k in range(500))
