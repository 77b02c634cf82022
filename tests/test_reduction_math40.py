"""The 3^40 variant's device arithmetic, restated in Python from its
derivations and checked against the definitions (no GPU).

Models: the quotient floor(2^53 z / 3^40) from the 118-bit reciprocal with
the carry rule, the remainder in 64-bit wrap-around arithmetic, the
Montgomery product with its 65-bit sum, the fixed-base skip-ahead table,
and the variate bits joined from two consecutive quotients (and from the
next two when the first is 0).  Each is compared with `//`, `%` and exact
rational truncation on random, edge and adversarial states.
"""
import math
import random
import struct
from fractions import Fraction

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


def test_two_chain_jump_distances():
    """A chain that has emitted variates [s, s+len) holds the state of
    variate s+len+1 (one quotient ahead); the jump to a run starting at s'
    is 2^(53 (s' - s - len - 1)).  Tiles of 32c, a lane's run split into
    h+1 and h variates (c = 2h+1)."""
    for c in (3, 15, 31, 63):
        h = c // 2
        s = 1000
        # chain a: variates [s, s+h+1), next run at s + 32c
        assert (s + 32 * c) - (s + h + 1) - 1 == 32 * c - h - 2
        # chain b: variates [s+h+1, s+c), next run at s+h+1 + 32c
        assert (s + h + 1 + 32 * c) - (s + c) - 1 == 31 * c + h
        # one chain: [s, s+c), next run at s + 32c
        assert (s + 32 * c) - (s + c) - 1 == 31 * c - 1


H0, H1 = RHI & 0xFFFFFFFF, RHI >> 32
RL1 = RLO >> 32


def quot_fast_model(z):
    """T = z*Rhi + z1*r1 from five 32x32-bit products; returns (floor(T/2^64),
    high word of T mod 2^64)."""
    z0, z1 = z & 0xFFFFFFFF, z >> 32
    p00, p01, p10, p11, b = z0 * H0, z0 * H1, z1 * H0, z1 * H1, z1 * RL1
    lo = p00 + b
    c0 = lo >> 64
    lo &= U64
    mid = p01 + p10
    cm = (mid >> 64) << 32
    mid &= U64
    f = lo + ((mid << 32) & U64)
    c1 = f >> 64
    f &= U64
    return p11 + (mid >> 32) + cm + c0 + c1, f >> 32


def bits_fast_model(q0, q1):
    t = (32 - (q0 >> 32).bit_length()) - 11
    mant = ((q0 << t) & U64) | ((q1 >> 32) >> (21 - t))
    return (((1021 - t) << 52) + mant) & U64


def undecided_states(count):
    """States whose next remainder is within a few units of 3^40, so that
    frac(2^53 z / 3^40) is within 2^-60 of 1: the fast quotient's fraction
    is then in the undecided band."""
    inv = pow(2 ** 53, -1, M40)
    out = []
    for k in range(1, count):
        if k % 3:
            out.append((M40 - k) * inv % M40)
    return out


def test_fast_quotient_is_exact_when_decided():
    zs = states(30000, 5) + undecided_states(300)
    flagged = 0
    for z in zs:
        q_fast, fhi = quot_fast_model(z)
        exact = (z << 53) // M40
        # T = z*Rhi + z1*r1 exactly, and it falls short of z*R/2^64 by less than 2^33+2
        full = z * R >> 64
        tt = z * RHI + (z >> 32) * RL1
        assert tt >> 64 == q_fast and 0 <= full - tt < 2 ** 33 + 2
        if fhi >= 0xFFFFFFFC:
            flagged += 1
            assert q_fast in (exact, exact - 1)
        else:
            assert q_fast == exact, z
    assert flagged >= 200
    for z in undecided_states(300):
        assert quot_fast_model(z)[1] >= 0xFFFFFFFC


def test_fast_conversion_matches_the_exact_one():
    for z in states(20000, 6):
        q0 = (z << 53) // M40
        if q0 < 2 ** 32:
            continue  # routed to the exact path
        z1 = (z << 53) % M40
        q1 = (z1 << 53) // M40
        assert bits_fast_model(q0, q1) == bits_model(q0, q1), z
        assert f64_from_bits(bits_fast_model(q0, q1)) == trunc_quotient(z)


def quot_fast_chain_model(z):
    """The same T from the same five products, summed in 32-bit limbs with
    add-with-carry chains (the kernel's PTX form): limb 0 only feeds its
    carry, limb 1 is the high word of T mod 2^64, limbs 2-3 the quotient."""
    m32 = 0xFFFFFFFF
    a0, a1 = z & m32, z >> 32
    h0, h1, r1 = H0, H1, RL1
    w = a0 * h0
    u = a1 * r1
    v = a0 * h1
    x = a1 * h0
    y = a1 * h1
    w0, w1, u0, u1 = w & m32, w >> 32, u & m32, u >> 32
    v0, v1, x0, x1, y0, y1 = v & m32, v >> 32, x & m32, x >> 32, y & m32, y >> 32

    def addc(p, q, cin):  # one 32-bit add with carry in and out
        s = p + q + cin
        return s & m32, s >> 32

    _, c = addc(w0, u0, 0)           # chain A: limb 0, limb 1, carry into limb 2
    s1, c = addc(w1, u1, c)
    c2, _ = addc(0, 0, c)
    s1, c = addc(s1, v0, 0)          # chain B: + a0*h1 at limb 1, + a1*h1 at limb 2
    s2, c = addc(v1, y0, c)
    s3, _ = addc(y1, 0, c)
    s1, c = addc(s1, x0, 0)          # chain C: + a1*h0 at limb 1
    s2, c = addc(s2, x1, c)
    s3, _ = addc(s3, 0, c)
    s2, c = addc(s2, c2, 0)          # chain D: chain A's carry into limb 2
    s3, _ = addc(s3, 0, c)
    assert s3 < 2 ** 32              # T < 2^118: no carry out of limb 3
    return (s3 << 32) | s2, s1


def test_fast_quotient_carry_chains_match():
    zs = states(40000, 17) + undecided_states(300) + [2 ** 64 - 1, M40 - 1, 2 ** 63,
                                                      (2 ** 32 - 1) << 32, 2 ** 32 - 1]
    for z in zs:
        assert quot_fast_chain_model(z) == quot_fast_model(z), z


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
