"""The 3^40 variant's device arithmetic, restated in Python from its
derivations and checked against the definitions (no GPU).

Models: the quotient floor(2^53 z / 3^40) from the 118-bit reciprocal with
the carry rule, the remainder in 64-bit wrap-around arithmetic, the
Montgomery product with its 65-bit sum, the fixed-base skip-ahead table,
the backward step that yields the previous state with its exact quotient,
and the variate bits joined from two consecutive quotients (and from the
next two when the first is 0).  Each is compared with `//`, `%` and exact
rational truncation on random, edge and adversarial states.
"""
import math
import random
import struct
from fractions import Fraction

import pytest

from m40_math import H40, M40, P40, index_of_state

U64 = 2 ** 64 - 1
R = 2 ** 181 // M40
RHI, RLO = R >> 64, R & U64
NEG_MINV = (-pow(M40, -1, 2 ** 64)) % 2 ** 64


def hi(a, b):
    return (a * b) >> 64


def quot_model(z):
    """ahi + carry(alo + bhi): the high word of z*R / 2^128."""
    alo = (z * RHI) & U64
    ahi = hi(z, RHI)
    bhi = hi(z, RLO)
    return ahi + (1 if alo + bhi > U64 else 0)


def rem_model(z, q):
    return ((z << 53) - q * M40) & U64


def mont_model(a, b):
    tlo = (a * b) & U64
    thi = hi(a, b)
    u = (tlo * NEG_MINV) & U64
    uhi = hi(u, M40)
    s1 = thi + uhi
    c1 = s1 > U64
    s1 &= U64
    s = s1 + (1 if tlo else 0)
    c2 = s > U64
    s &= U64
    return (s - M40) & U64 if (c1 or c2 or s >= M40) else s


def clz64(x):
    return 64 - x.bit_length()


def bits_model(q0, q1):
    t = clz64(q0) - 11
    mant = ((q0 << t) & U64) | (q1 >> (53 - t))
    return (((1021 - t) << 52) + mant) & U64


def bits_small_model(z1, q1):
    q2 = quot_model(rem_model(z1, q1))
    t = clz64(q1) - 11
    mant = ((q1 << t) & U64) | (q2 >> (53 - t))
    return (((1021 - 53 - t) << 52) + mant) & U64


def f64_from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def trunc_quotient(z):
    s = 53 + (M40.bit_length() - z.bit_length()) + 1
    q = (z << s) // M40
    drop = q.bit_length() - 53
    return math.ldexp(q >> drop, drop - s)


def states(count, seed):
    rnd = random.Random(seed)
    out = [1, 2, 4, 5, 7, M40 - 1, M40 - 2, H40, H40 + 1, 2 ** 63, 2 ** 63 + 1, U64 % M40]
    out += [2 ** k for k in range(64) if 2 ** k < M40]
    out += [rnd.randrange(1, M40) for _ in range(count)]
    # states just above multiples of m / 2^53 (quotient boundaries)
    for _ in range(count // 10):
        j = rnd.randrange(1, 2 ** 53)
        out.append(-(-j * M40 // 2 ** 53))
    return [z for z in out if z % 3 and 0 < z < M40]


def test_reciprocal_constants():
    assert RHI == 2 ** 117 // M40 and RHI < 2 ** 54
    assert (M40 * NEG_MINV + 1) % 2 ** 64 == 0
    # the error bound of the quotient argument: z/2^128 < 2^-64 <= 1/m
    assert Fraction(U64, 2 ** 128) < Fraction(1, M40) * 2


def test_quotient_and_remainder_are_exact():
    for z in states(40000, 1):
        q = quot_model(z)
        assert q == (z << 53) // M40, z
        r = rem_model(z, q)
        assert r == (z << 53) % M40 and 0 < r < M40


def test_montgomery_product():
    rnd = random.Random(2)
    vals = [1, 2, M40 - 1, M40 - 2, 2 ** 63, H40] + [rnd.randrange(1, M40) for _ in range(20000)]
    minv64 = pow(2 ** 64, -1, M40)
    for k in range(len(vals) - 1):
        a, b = vals[k], vals[k + 1]
        assert mont_model(a, b) == a * b * minv64 % M40
    # with one operand in Montgomery form the product is a plain product
    for a, c in [(M40 - 1, M40 - 1), (12345, 2 ** 63 % M40), (H40, 3 ** 39 + 1)]:
        assert mont_model(a, (c << 64) % M40) == a * c % M40


def test_skip_ahead_table_model():
    rnd = random.Random(3)
    g, rows = 2, []
    for k in range(8):
        v = H40 if k == 0 else 1
        row = []
        for _ in range(256):
            row.append(v if k == 0 else (v << 64) % M40)
            v = v * g % M40
        rows.append(row)
        g = pow(g, 256, M40)
    for e in [0, 1, 255, 256, P40 - 1, P40 // 2] + [rnd.randrange(P40) for _ in range(300)]:
        z = rows[0][e & 255]
        for k in range(1, 8):
            z = mont_model(z, rows[k][(e >> (8 * k)) & 255])
        assert z == pow(2, e, M40) * H40 % M40, e


def test_variate_bits_from_two_quotients():
    for z in states(20000, 4):
        q0 = quot_model(z)
        z1 = rem_model(z, q0)
        q1 = quot_model(z1)
        b = bits_model(q0, q1) if q0 else bits_small_model(z1, q1)
        v = f64_from_bits(b)
        assert v == trunc_quotient(z), z
        assert Fraction(v) <= Fraction(z, M40) < Fraction(math.nextafter(v, 2.0))


def test_smallest_variates_take_the_second_window():
    """States below 3^40 / 2^53 (variates below 2^-53) have a zero first
    quotient; their bits come from the next two quotients."""
    small = [z for z in range(1, 1350) if z % 3] + [1349, 1348]
    for z in small:
        q0 = quot_model(z)
        assert q0 == 0
        z1 = rem_model(z, q0)
        q1 = quot_model(z1)
        assert q1 != 0
        assert f64_from_bits(bits_small_model(z1, q1)) == trunc_quotient(z), z
    assert quot_model(1349) == 0 and quot_model(1350) == 1  # 3^40/2^53 = 1349.77...
    assert index_of_state(M40 + 100, 1) >= 0


def test_backward_chain_jump_distances():
    """The tiled kernel's chains run backwards and, for variates, hold the
    state one above the next element emitted (its digit continues that
    variate); after a run of c elements at s a single chain holds element s,
    two chains (b: c-1 .. h+1, a: h .. 0) hold elements s and s+h+1.  The jump
    to the next tile (s + 32c) must land one above (plus lead) the element
    each chain emits first."""
    for c in (3, 15, 31, 63):
        h = c // 2
        s = 1000
        for lead in (0, 1):
            assert (s + 32 * c + c + lead) - s == 33 * c + lead           # one chain
            assert (s + 32 * c + h + 1 + lead) - s == 32 * c + h + 1 + lead  # chain a
            assert (s + 32 * c + c + lead) - (s + h + 1) == 33 * c - h - 1 + lead  # chain b


MASK32 = 0xFFFFFFFF
MP40 = (-pow(M40, -1, 2 ** 53)) % 2 ** 53


def back_model(z):
    """The backward step on 32-bit limbs: Q = z m' mod 2^53 and
    S = z + Q 3^40 from limb 1 up, limb 0's carry being [low word of z != 0];
    returns (S >> 53, Q)."""
    z0, z1 = z & MASK32, z >> 32
    mp0, mp1 = MP40 & MASK32, MP40 >> 32
    m0, m1 = M40 & MASK32, M40 >> 32
    t = z0 * mp0
    u0, th = t & MASK32, t >> 32
    u1 = (th + z0 * mp1 + z1 * mp0) & 0x1FFFFF
    l1 = ((u0 * m0) >> 32) + z1 + (1 if z0 else 0)
    l1 += (u0 * m1) & MASK32
    l1 += (u1 * m0) & MASK32
    l2 = (l1 >> 32) + ((u0 * m1) >> 32) + ((u1 * m0) >> 32) + ((u1 * m1) & MASK32)
    l3 = (l2 >> 32) + ((u1 * m1) >> 32)
    s = ((l3 & MASK32) << 64) | ((l2 & MASK32) << 32) | (l1 & MASK32)
    return s >> 21, (u1 << 32) | u0


def test_backward_step_and_its_digit_are_exact():
    for zk in states(60000, seed=44) + [j << 32 for j in range(1, 400)]:
        if zk % 3 == 0 or not 0 < zk < M40:
            continue
        zp, q = back_model(zk)
        assert 0 < zp < M40 and (zp << 53) % M40 == zk, zk
        assert q == (zp << 53) // M40 == quot_model(zp), zk


def test_backward_digits_join_into_the_truncated_variate():
    """Two consecutive digits from two steps back give the variate of the
    lower state exactly (fast form while its leading digit is >= 2^32)."""
    for z2 in states(20000, seed=45):
        z1, q1 = back_model(z2)
        z0, q0 = back_model(z1)
        assert q1 == quot_model(z1) and q0 == quot_model(z0)
        if q0 >> 32:
            assert f64_from_bits(bits_fast_model(q0, q1)) == trunc_quotient(z0), z2


def bits_fast_model(q0, q1):
    t = (32 - (q0 >> 32).bit_length()) - 11
    mant = ((q0 << t) & U64) | ((q1 >> 32) >> (21 - t))
    return (((1021 - t) << 52) + mant) & U64


def test_fast_conversion_matches_the_exact_one():
    for z in states(20000, 6):
        q0 = (z << 53) // M40
        if q0 < 2 ** 32:
            continue  # routed to the exact path
        z1 = (z << 53) % M40
        q1 = (z1 << 53) // M40
        assert bits_fast_model(q0, q1) == bits_model(q0, q1), z
        assert f64_from_bits(bits_fast_model(q0, q1)) == trunc_quotient(z)


def bits_fast_funnel_model(q0, q1):
    """bits40_fast on 32-bit words (the kernel's PTX form): the mantissa's
    high word is a funnel shift of q0's words by t, its low word a funnel
    shift of q0's low word over q1's high word placed at the top of a word,
    and the exponent joins the high word."""
    m32 = 0xFFFFFFFF
    q0l, q0h, q1h = q0 & m32, q0 >> 32, q1 >> 32

    def shf_l(lo, hi, s):  # high word of (hi:lo) << s, s in [0, 31]
        return (((hi << 32) | lo) << s >> 32) & m32

    c = 32 - q0h.bit_length()
    t = c - 11
    mh = shf_l(q0l, q0h, t)
    ml = shf_l((q1h << 11) & m32, q0l, t)
    hi = (mh + ((1032 - c) << 20)) & m32
    return (hi << 32) | ml


def test_fast_conversion_funnel_form_matches():
    for z in states(30000, 19):
        q0 = (z << 53) // M40
        if q0 < 2 ** 32:
            continue
        q1 = ((((z << 53) - q0 * M40)) << 53) // M40
        assert bits_fast_funnel_model(q0, q1) == bits_fast_model(q0, q1), z
    for t in range(21):  # every shift, with extreme low words
        for q0l in (0, 1, 0xFFFFFFFF, 0x80000000):
            for q1h in (0, 1, (1 << 21) - 1, 1 << 20):
                q0 = ((1 << (20 - t)) << 32) | q0l
                q1 = q1h << 32
                assert bits_fast_funnel_model(q0, q1) == bits_fast_model(q0, q1), (t, q0l, q1h)


# ---------------------------------------------- FP32 runs from one product
MASK32 = 2 ** 32 - 1


def neg_minv_words40_model(W):
    """-3^-40 mod 2^(32 W) word by word, as the kernel builds it."""
    inv = pow(M40, -1, 2 ** 32)
    A, words = 1, []
    for _ in range(W):
        n = (-A * inv) % 2 ** 32
        A += M40 * n
        assert A % 2 ** 32 == 0 and A < 2 ** 97
        words.append(n)
        A >>= 32
    return words


def rz32_bits(s):
    """Bits of s/3^40 truncated to a float (24 significant bits), exactly."""
    k = 24 + M40.bit_length() - s.bit_length()
    while (s << k) // M40 >= 2 ** 24:
        k -= 1
    while (s << k) // M40 < 2 ** 23:
        k += 1
    mant = (s << k) // M40
    return struct.unpack("<I", struct.pack("<f", math.ldexp(mant, -k)))[0]


def digit_run40_model(z, C):
    """One lane's FP32 run of C variates from the state z one past it, on
    32-bit words as the kernel forms it (three-word partial sums, V below
    2^34), with the conversion of each field and the flag (digit below 2^23).
    Returns the words, the FP32 bits of elements 0 .. C-1 and their flags."""
    W = (53 * C + 31) // 32
    N = neg_minv_words40_model(W)
    z0, z1 = z & MASK32, z >> 32
    r, V = [], 0
    for i in range(W):
        x = V + (z1 * N[i - 1] if i > 0 else 0)
        assert x < 2 ** 65
        s = x + z0 * N[i]
        assert s < 2 ** 66
        r.append(s & MASK32)
        V = s >> 32
        assert V < 2 ** 34

    def bits32(pos):
        if pos < 0:
            return (r[0] << -pos) & MASK32
        k, o = pos // 32, pos % 32
        return r[k] if o == 0 else (((r[k + 1] << 32) | r[k]) >> o) & MASK32

    bits, flags = [0] * C, [False] * C
    for i in range(C):
        u1, u0 = bits32(53 * i + 21), bits32(53 * i - 11)
        c = 32 - u1.bit_length() if u1 else MASK32
        mant = (((((u1 << 32) | u0) << c) >> 32) & MASK32) >> 8 if c < 32 else u0 >> 8
        e = (c * 0xFF800000 + 0x3E800000) & MASK32
        bits[C - 1 - i] = (mant + e) & MASK32
        flags[C - 1 - i] = u1 < 4
    return r, bits, flags


def test_run40_constant():
    for W in (2, 25, 52, 70):
        N = sum(w << (32 * i) for i, w in enumerate(neg_minv_words40_model(W)))
        assert N == (-pow(M40, -1, 2 ** (32 * W))) % 2 ** (32 * W)
    assert sum(w << (32 * i) for i, w in enumerate(neg_minv_words40_model(2))) == NEG_MINV


@pytest.mark.parametrize("C", [31, 15, 1])
def test_run40_fields_are_the_digits_and_the_floats_truncate(C):
    """Field i of z N is floor(2^53 s / 3^40) of the state i + 1 steps before
    z; the word-level product equals the big-integer one; every unflagged
    element's float is s/3^40 truncated to 24 bits, and exactly the elements
    whose digit is below 2^23 are flagged.  States with digits around 2^23
    and 2^24 are placed at every position of a run."""
    W = (53 * C + 31) // 32
    inv53 = pow(2, -53, M40)
    zs = states(300, seed=70 + C)
    rnd = random.Random(71 + C)
    for q in (2 ** 23 - 2, 2 ** 23 - 1, 2 ** 23, 2 ** 23 + 1, 2 ** 24 - 1, 2 ** 24, 3, 1):
        s = -(-(q * M40) // 2 ** 53)
        while s % 3 == 0 or (s << 53) // M40 != q:
            s += 1
        for pos in {0, C - 1, rnd.randrange(C)}:
            zs.append(s * pow(2, 53 * (C - pos), M40) % M40)   # element pos holds s
    flagged = 0
    for z in zs:
        r, bits, flags = digit_run40_model(z, C)
        P = sum(w << (32 * i) for i, w in enumerate(r))
        assert P == z * (-pow(M40, -1, 2 ** (32 * W))) % 2 ** (32 * W)
        s = z
        for e in range(C - 1, -1, -1):
            s = s * inv53 % M40                               # element e's state
            qd = (s << 53) // M40
            i = C - 1 - e
            assert (P >> (53 * i)) % 2 ** 53 == qd, (z, e)
            assert flags[e] == (qd < 2 ** 23), (z, e)
            if flags[e]:
                flagged += 1
            else:
                assert bits[e] == rz32_bits(s), (z, e)
        assert s * pow(2, 53 * C, M40) % M40 == z             # the redo's start, C steps back
    assert flagged >= 4
