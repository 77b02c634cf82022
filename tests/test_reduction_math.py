"""The arithmetic the CUDA kernels rely on, restated in Python and checked
against the definitions (no GPU).

These are models of the reductions (Sec. 2.1) and of the integer rounding,
written from their derivations -- not imports of the CUDA code, which Python
cannot run.  Each model is checked against `%` and exact rational rounding on
random, edge and adversarial states, and the bounds its correctness argument
uses are checked directly.  The GPU parity tests then check the kernels
themselves against the oracle.
"""
import math
import random
import struct
from fractions import Fraction

import pytest

M = 3 ** 33
MU = 2 ** 106 // M
K = MU + 1
MR = K // 2
R3I = 1.0 / 5559060566555523.0
MASK32 = 2 ** 32 - 1
M0, M1 = M & MASK32, M >> 32
K0, K1 = K & MASK32, K >> 32


def f64_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def rn_bits(z: int) -> int:
    """Bits of RN(z * r3i), by exact rational arithmetic."""
    return f64_bits(float(Fraction(z) * Fraction(R3I)))


def funnel_l(lo, hi, s):
    return ((((hi << 32) | lo) << (s & 31)) >> 32) & MASK32


def funnel_r(lo, hi, s):
    return (((hi << 32) | lo) >> (s & 31)) & MASK32


def clz32(x):
    return 32 - x.bit_length()


def states(count=50000, seed=0):
    rnd = random.Random(seed)
    zs = [1, 2, 3, 4, M - 1, M - 2, M - 3, M // 2, M // 2 + 1]
    zs += [(M >> e) + d for e in range(54) for d in (-1, 0, 1)]
    zs += [2 ** k for k in range(53)] + [3 * 2 ** k for k in range(52)]
    zs += [rnd.randrange(1, M) for _ in range(count)]
    return sorted({z for z in zs if 0 < z < M})


def test_constants_relations():
    assert MU == 0x33D9481681D79D
    assert K == 2 * MR and MR == 0x19ECA40B40EBCF
    assert Fraction(R3I) == Fraction(MR, 2 ** 105)
    assert M < 2 ** 53 < 2 * M


def test_modified_barrett_never_wraps():
    """Sec. 2.1.3: q3 = floor(mu z / 2^53) in {Q-1, Q}; the 53-bit wrap of
    2^53 z - q3 m would need frac(2^53 z/m) >= 2^53/m - 1, while q3 = Q-1
    needs frac(2^53 z/m) < m/2^53.  The two thresholds do not overlap."""
    assert Fraction(M, 2 ** 53) < Fraction(2 ** 53, M) - 1
    for z in states():
        q3 = (z * MU) >> 53
        Q = (z << 53) // M
        assert q3 in (Q - 1, Q)
        r = 2 ** 53 - ((q3 * M) & (2 ** 53 - 1))
        if r >= M:
            r -= M
        assert r == (z << 53) % M


def test_montgomery_back_step():
    negminv = (-pow(M, -1, 2 ** 53)) % 2 ** 53
    for z in states():
        u = (z * negminv) & (2 ** 53 - 1)
        prev = ((u * M) >> 53) + 1
        assert 0 < prev < M
        assert (prev << 53) % M == z


def test_general_barrett_mulmod_bound():
    """x*y mod m with q1 = t >> 52, q3 = (q1 mu) >> 54: t - q3 m < 3m."""
    rnd = random.Random(1)
    for _ in range(50000):
        x, y = rnd.randrange(1, M), rnd.randrange(1, M)
        t = x * y
        q3 = ((t >> 52) * MU) >> 54
        r = t - q3 * M
        assert 0 <= r < 3 * M < 2 ** 64
        while r >= M:
            r -= M
        assert r == t % M


def shared_step_model(z):
    """Word-level model of the shared-quotient step and its conversion."""
    z0, z1 = z & MASK32, z >> 32
    t0 = z0 * K0
    t1 = z0 * K1 + (t0 >> 32)
    t1 = z1 * K0 + t1
    t2 = z1 * K1 + (t1 >> 32)
    assert t1 < 2 ** 64 and t2 < 2 ** 64
    w1, w2, w3 = t1 & MASK32, t2 & MASK32, t2 >> 32
    q0, q1 = funnel_r(w1, w2, 21), funnel_r(w2, w3, 21)
    qm = q0 * M0
    qm_hi = ((qm >> 32) + q0 * M1 + q1 * M0) & MASK32
    r = ((((z0 << 21) & MASK32) << 32) - ((qm_hi << 32) | (qm & MASK32))) % 2 ** 64
    if r >= 2 ** 63:
        r = (r + M) % 2 ** 64
    if q1 == 0:
        return r, None
    c = clz32(q1)
    s = c - 10
    lh = (w1 << 11) & MASK32
    g_hi, g_lo = funnel_l(q0, q1, s), funnel_l(lh, q0, s)
    x = ((g_hi << 32) | g_lo) + (((1032 - c) << 53) | 1)
    assert x < 2 ** 64
    return r, x >> 1


def test_shared_quotient_is_q_or_q_plus_one():
    for z in states():
        q = (z * K) >> 53
        Q = (z << 53) // M
        assert q in (Q, Q + 1)
        assert -M < (z << 53) - q * M < M


def test_no_state_rounds_on_a_tie():
    """p = z*K = 2 z M_r with M_r odd; a tie needs v2(p) = bitlen(p) - 54,
    which forces v2(z) >= bitlen(z) - 2, i.e. z = 2^k or 3*2^k."""
    assert MR % 2 == 1
    for z in [2 ** k for k in range(53)] + [3 * 2 ** k for k in range(52)]:
        if z >= M:
            continue
        p = z * K
        d = p.bit_length() - 53
        assert p % 2 ** d != 2 ** (d - 1)


def test_shared_step_model_matches_definitions():
    slow = 0
    for z in states(80000, seed=2):
        r, bits = shared_step_model(z)
        assert r == (z << 53) % M
        if bits is None:
            slow += 1
            assert z * K < 2 ** 85  # q < 2^32: the variate is below 2^-21
            continue
        assert bits == rn_bits(z), z
    assert slow > 0  # the rare path is exercised by the edge states


KB, MS = K << 1, M << 10  # the scaled chain's constants: Z = z 2^10


def shared_step_scaled_model(zz):
    """Word-level model of the PTX step on a chain holding Z = z 2^10:
    returns (next Z, FP64 bits or None for the rare path, q's top word)."""
    z0, z1 = zz & MASK32, zz >> 32
    kb0, kb1, ms0, ms1 = KB & MASK32, KB >> 32, MS & MASK32, MS >> 32
    h0 = (z0 * kb0) >> 32
    t = z0 * kb1 + h0
    w1, x = t & MASK32, t >> 32
    t = z1 * kb0 + w1
    w1, x = t & MASK32, x + (t >> 32)
    t = z1 * kb1 + x
    q0, q1 = t & MASK32, t >> 32
    assert q1 < 2 ** 32
    qm = (q0 * ms0 + (((q0 * ms1 + q1 * ms0) & MASK32) << 32)) % 2 ** 64
    r = ((((z0 << 21) & MASK32) << 32) - qm) % 2 ** 64
    if r >= 2 ** 63:
        r = (r + MS) % 2 ** 64
    if q1 == 0:
        return r, None, q1
    c = clz32(q1)
    s = c - 10
    g_hi, g_lo = funnel_l(q0, q1, s), funnel_l(w1, q0, s)
    xx = ((g_hi << 32) | g_lo) + (((1032 - c) << 53) | 1)
    return r, xx >> 1, q1


def test_scaled_step_model_matches_the_unscaled_step():
    """On Z = z 2^10 with 2K and m 2^10: the same quotient window, the next
    state scaled, the same FP64 bits, and the remainder's sign from its top
    bit (|2^53 z - q m| 2^10 < 2^63)."""
    assert KB < 2 ** 55 and 2 ** 62 <= MS < 2 ** 63
    edge = [1, 2, 3, M - 1, M - 2, ((2 ** 32) * M) >> 53, (((2 ** 32) * M) >> 53) + 1]
    slow = 0
    for z in states(60000, seed=22) + edge:
        zz = z << 10
        assert ((zz * KB) >> 64) == (z * K) >> 53
        r, bits, q1 = shared_step_scaled_model(zz)
        assert r == ((z << 53) % M) << 10, z
        assert (r, bits) == ((shared_step_model(z)[0]) << 10, shared_step_model(z)[1]), z
        if bits is None:
            slow += 1
            continue
        assert bits == rn_bits(z), z
    assert slow > 0
    # the FP64-pipe conversion from Z: exact int->double, then r3i 2^-10
    for z in states(5000, seed=24) + edge:
        assert float(z << 10) == float(z) * 1024.0
        assert f64_bits(float(z << 10) * (R3I * 2.0 ** -10)) == rn_bits(z), z


def general_conversion_model(p):
    """The general integer rounding of p * 2^-106 (any leading-zero count)."""
    q = p >> 53
    low = p & (2 ** 53 - 1)
    lz = (64 - q.bit_length()) - 11
    mant = (q << lz) | (low >> (53 - lz))
    rest = (low << (11 + lz)) % 2 ** 64
    half = 2 ** 63
    up = 1 if (rest > half or (rest == half and mant & 1)) else 0
    return ((1021 - lz) << 52) + mant + up


@pytest.mark.parametrize("seed", [3, 4])
def test_general_conversion_model(seed):
    for z in states(30000, seed=seed):
        assert general_conversion_model(z * K) == rn_bits(z)


def test_f32_from_f64_bits_is_truncation():
    for z in states(20000, seed=5):
        b = rn_bits(z)
        f = ((b >> 29) - (896 << 23)) & MASK32
        v = Fraction(struct.unpack("<d", struct.pack("<Q", b))[0])
        fv = Fraction(struct.unpack("<f", struct.pack("<I", f))[0])
        nxt = Fraction(struct.unpack("<f", struct.pack("<I", f + 1))[0])
        assert fv <= v < nxt


# ------------------------------------------------ fused consumer arithmetic
def _sq_grid(v: float):
    """RN(v*v) * 2^157 as (integer, shift k) the way the fused kernel forms it:
    RNE of mant^2 to 53 bits, then M2 << k with k = 2e + sh - 1993."""
    b = f64_bits(v)
    e, mant = b >> 52, (b & (2 ** 52 - 1)) | 2 ** 52
    sq = mant * mant
    sh = 53 if sq >= 2 ** 105 else 52
    m2, rest, half = sq >> sh, sq & (2 ** sh - 1), 2 ** (sh - 1)
    if rest > half or (rest == half and m2 & 1):
        m2 += 1
    k = 2 * e + sh - 1993
    return m2 << k, k


def test_fp64_pipe_square_lands_on_the_same_grid():
    """The FP64-pipe form takes RN(v*v) from one multiply and places its
    significand M2 at k = e2 - 918 on the 2^-157 grid; that is the integer
    form's M2 << k for every variate (down to the smallest, near 2^-53)."""
    for z in states(20000, seed=9) + [1, 2, 3, 4, M - 1]:
        v = float(Fraction(z) * Fraction(R3I))
        sq = v * v  # one round-to-nearest multiply
        b = f64_bits(sq)
        e2, m2 = b >> 52, (b & (2 ** 52 - 1)) | 2 ** 52
        k = e2 - 918
        assert k >= 0
        zi, ki = _sq_grid(v)
        assert (m2 << k, k) == (zi, ki), z


def test_fused_square_grid_and_split_hit_rule():
    """RN(v*v) is an integer on the 2^-157 grid for every variate; the hit
    test RN(RN(x^2)+RN(y^2)) <= 1 equals: exact high parts (k >= 64) plus
    ceilings of the small squares on the 2^-93 grid <= 2^93 + 2^40."""
    import math
    rnd = random.Random(7)
    vals = [float(Fraction(z) * Fraction(R3I)) for z in states(4000, seed=8)]
    pairs = [(rnd.choice(vals), rnd.choice(vals)) for _ in range(8000)]
    for _ in range(4000):  # pairs on the unit circle to within a few ulps
        x = rnd.random()
        y = math.sqrt(max(0.0, 1 - x * x))
        for d in (-2, -1, 0, 1, 2):
            if 0 < y + d * 2 ** -53 < 1:
                pairs.append((x, y + d * 2 ** -53))
    for _ in range(2000):  # one tiny partner next to x close to 1
        t = 2.0 ** -rnd.randint(20, 52) * (1 + rnd.random())
        x = math.sqrt(1 - t * t)
        for d in (-1, 0, 1):
            pairs.append((x + d * 2 ** -53, t))
    lim = (2 ** 157 + 2 ** 104) >> 64
    for x, y in pairs:
        tot = 0
        for v in (x, y):
            z, k = _sq_grid(v)
            assert Fraction(z, 2 ** 157) == Fraction(v * v)
            tot += (z >> 64) if k >= 64 else -(-z // 2 ** 64)
            if k >= 64:
                assert z % 2 ** 64 == 0
            else:
                assert z < 2 ** 117
        assert (tot <= lim) == (x * x + y * y <= 1.0), (x, y)


# ------------------------------------- the paper's other two reductions
LQ, LR = M // 2 ** 25, M % 2 ** 25   # m = a*q + r with a = 2^25 (Sec. 2.1.1)


def lecuyer_mul(s):
    """2^25 * s mod m for 0 <= s < 4m by L'Ecuyer's decomposition."""
    t = s // LQ
    v = ((s - t * LQ) << 25) - t * LR
    assert -M < v < M            # the bound Sec. 2.1.1 proves for s < 4m
    return v + M if v < 0 else v


def test_lecuyer_twice_is_the_step():
    assert LR < 2 ** 25 and 2 ** 50 < M
    for z in states(30000, seed=11):
        s = lecuyer_mul(z << 2)      # 2^27 z mod m
        s = lecuyer_mul(s << 1)      # 2^53 z mod m
        assert s == (z << 53) % M


def test_classic_barrett_step():
    """Barrett's algorithm with k = 53 on x = 2^53 z: q1 = x >> 52, q3 = (mu q1)
    >> 54, r = (x - q3 m) mod 2^54, then at most two subtractions of m."""
    for z in states(30000, seed=12):
        x = z << 53
        q3 = (MU * (x >> 52)) >> 54
        assert (x // M) - 2 <= q3 <= x // M
        r = ((x % 2 ** 54) - (q3 * M) % 2 ** 54) % 2 ** 54
        subs = 0
        while r >= M:
            r -= M
            subs += 1
        assert subs <= 2 and r == x % M


def test_precomputed_quotient_mulmod():
    """Multiplication by a fixed J mod m with J' = floor(J * 2^64 / m) (a
    precomputed-quotient modular product): q = floor(z*J'/2^64) is Q or Q-1
    for Q = floor(z*J/m), so z*J - q*m lies in [0, 2m)."""
    rnd = random.Random(13)
    for _ in range(300):
        j = rnd.randrange(1, M)
        jq = (j << 64) // M
        for z in [1, M - 1] + [rnd.randrange(1, M) for _ in range(200)]:
            q = (z * jq) >> 64
            Q = (z * j) // M
            assert q in (Q - 1, Q)
            r = (z * j - q * M) % 2 ** 64
            assert r < 2 * M
            if r >= M:
                r -= M
            assert r == (z * j) % M


def rz_f32_bits(z: int) -> int:
    """Bits of the FP32 variate: RN(z * r3i) as a double, then toward zero."""
    import numpy as np
    v = float(Fraction(z) * Fraction(R3I))
    f = np.float32(v)
    if float(f) > v:
        f = np.nextafter(f, np.float32(0.0))
    return int(np.array([f], dtype=np.float32).view(np.uint32)[0])


def rotl32(x, n):
    n &= 31
    return ((x << n) | (x >> (32 - n))) & MASK32 if n else x


def test_fused_kept_chunk_parts():
    """The fused kernel's kept-chunk arithmetic for variates v >= 2^-16:
    v * 2^105 = (mh 2^32 + lo) pj 2^32 with pj = rotl(2^22, e) = 2^(e-1002),
    RN(v*v) * 2^84 = (mh2 2^32 + ml2) pk with pk = rotl(2, e2) = 2^(e2-991),
    both powers of two below 2^32, and the pair's hit rule on the 2^-84 grid
    (S <= 2^84 + 2^31 iff RN(RN(x^2) + RN(y^2)) <= 1) with S below 2^85."""
    import math
    rnd = random.Random(14)
    vals = [float(Fraction(z) * Fraction(R3I)) for z in states(20000, seed=15)]
    vals += [2.0 ** -16, math.nextafter(1.0, 0.0), 0.5, math.nextafter(0.5, 0.0),
             math.nextafter(2.0 ** -16, 1.0)]
    vals = [v for v in vals if v >= 2.0 ** -16]

    def parts(v):
        b = f64_bits(v)
        hi, lo = b >> 32, b & MASK32
        mh = (hi & 0xFFFFF) | 0x100000
        pj = rotl32(1 << 22, hi >> 20)
        assert pj == 2 ** ((hi >> 20) - 1002) and 2 ** 5 <= pj <= 2 ** 20
        assert Fraction((mh << 32 | lo) * pj << 32, 2 ** 105) == Fraction(v), v
        sb = f64_bits(v * v)                        # one round-to-nearest multiply
        shi, slo = sb >> 32, sb & MASK32
        mh2 = (shi & 0xFFFFF) | 0x100000
        pk = rotl32(2, shi >> 20)
        assert pk == 2 ** ((shi >> 20) - 991) and 1 <= pk <= 2 ** 31
        img = (mh2 << 32 | slo) * pk
        assert Fraction(img, 2 ** 84) == Fraction(v * v) and img < 2 ** 84
        return img, slo * pk, mh2 * pk

    for v in vals:
        parts(v)
    pairs = [(rnd.choice(vals), rnd.choice(vals)) for _ in range(8000)]
    for _ in range(4000):  # pairs on the unit circle to within a few ulps
        x = rnd.uniform(2.0 ** -16, 1.0)
        y = math.sqrt(max(0.0, 1 - x * x))
        for d in (-2, -1, 0, 1, 2):
            if 2.0 ** -16 <= y + d * 2 ** -53 < 1:
                pairs.append((x, y + d * 2 ** -53))
    lim = 2 ** 84 + 2 ** 31
    for x, y in pairs:
        ix, lx, hx = parts(x)
        iy, ly, hy = parts(y)
        tl, th = lx + ly, hx + hy                   # the two 64-bit partial sums
        assert tl < 2 ** 64 and th < 2 ** 53
        S = tl + (th << 32)
        assert S == ix + iy and S < 2 ** 85
        assert (S <= lim) == (x * x + y * y <= 1.0), (x, y)


def f64_of_bits(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def test_fp64_pipe_conversion_by_one_fused_multiply_add():
    """The FP64-pipe conversion in one FMA: D = 2^52 + (z mod 2^52), whose bits
    are the high word 0x43300000 | (z1 & 0xFFFFF) over the low word z0, is an
    exact double; fma(D, r3i, off) with off = -2^52*r3i when z < 2^52 and 0
    otherwise rounds D*r3i + off = z*r3i once, so it is RN(z * r3i)."""
    off_bits = f64_bits(-(2.0 ** 52) * R3I)
    assert Fraction(f64_of_bits(off_bits)) == -Fraction(2 ** 52) * Fraction(R3I)  # exact
    extra = [2 ** 52 - 1, 2 ** 52, 2 ** 52 + 1, (2 ** 52) - (2 ** 20), 2 ** 52 + 2 ** 32,
             M - 1, 1, 2 ** 32 - 1, 2 ** 32, 2 ** 32 + 1]
    for z in states(30000, seed=21) + extra:
        z0, z1 = z & MASK32, z >> 32
        hi = 0x43300000 | (z1 & 0xFFFFF)
        d = f64_of_bits((hi << 32) | z0)
        big = z1 >= 0x100000  # z >= 2^52
        assert Fraction(d) == (z if big else 2 ** 52 + z)  # D is exact
        off = Fraction(0) if big else Fraction(f64_of_bits(off_bits))
        exact = Fraction(d) * Fraction(R3I) + off
        assert exact == Fraction(z) * Fraction(R3I)
        assert f64_bits(float(exact)) == rn_bits(z)  # one rounding of the same value


def test_fused_chunk_rule_puts_every_variate_above_2_16():
    """A fused-consumer chunk is kept when the top word of every step's 53-bit
    quotient window is at least 32 (q >= 2^37): then z*r3i >= 2^-16, so
    v = RN(z*r3i) >= 2^-16 and RN(v*v) >= 2^-32 (exponent e2 >= 991), as the
    kept-chunk parts need.  Such a variate's square is also on the fast
    2^-93 grid of the exact path (k = e2 - 918 >= 73)."""
    edge = ((2 ** 37) * M) >> 53  # states around the 2^-16 boundary
    kept = 0
    for z in states(30000, 23) + [edge + d for d in range(-3, 4)]:
        if not 0 < z < M:
            continue
        q = (z * K) >> 53  # the step's 53-bit quotient window, floor(z*K / 2^53)
        v = float(Fraction(z) * Fraction(R3I))
        e2 = f64_bits(v * v) >> 52
        if q >> 32 >= 32:
            kept += 1
            assert Fraction(z) * Fraction(R3I) >= Fraction(1, 2 ** 16)
            assert v >= 2.0 ** -16 and e2 >= 991
        elif q >> 32 < 32 and 0 < z < edge - 3:
            assert v < 2.0 ** -16 + 2.0 ** -60
    assert kept > 29000


MP = (-pow(M, -1, 2 ** 53)) % 2 ** 53  # m' = -m^-1 mod 2^53
MPX = (MP << 11) % 2 ** 64              # the step's multiplier, m' 2^11 mod 2^64


def back_step_f32_model(y):
    """The backward FP32 step on 32-bit words: y = z_k - 1 gives y_(k-1), the
    quotient Q of the state z_(k-1) (the step holds X = Q 2^11 = (u1:u0)),
    its FP32 bits and the flag v (0: the exact path is needed).
    bfind.shiftamt of 0 is 2^32 - 1."""
    y0, y1 = y & MASK32, y >> 32
    k0, k1 = MPX & MASK32, MPX >> 32
    t = (y0 * k0 + MPX) % 2 ** 64
    u0, th = t & MASK32, t >> 32
    u1 = (th + y0 * k1 + y1 * k0) & MASK32
    h0 = (u0 * M0) >> 32
    lo = u0 * M1 + h0                         # carry chain of 32-bit halves
    w1 = lo & MASK32
    x = lo >> 32
    lo = u1 * M0 + w1
    x += lo >> 32
    yp = u1 * M1 + x                          # the high 64 bits of X m
    c = clz32(u1) if u1 else MASK32
    mant = (((((u1 << 32) | u0) << c) >> 32) & MASK32) >> 8 if c < 32 else u0 >> 8
    e = (c * 0xFF800000 + 0x3E800000) & MASK32
    bits = (mant + e) & MASK32
    v = ((~(u0 | 0xFFF) & MASK32) << c) & MASK32 if c < 32 else 0
    return yp, ((u1 << 32) | u0) >> 11, bits, v


def test_backward_step_gives_the_previous_state_and_its_quotient():
    for zk in states(40000, seed=31):
        yp, q, _, _ = back_step_f32_model(zk - 1)
        zp = yp + 1
        assert 0 < zp < M and (zp << 53) % M == zk, zk
        assert q == (zp << 53) // M, zk


def test_backward_f32_from_the_quotient_is_the_truncated_double():
    """Unflagged steps give RN(z*r3i) toward zero exactly; flags are rare on
    random states.  Adversarial states: quotients whose bits below the float's
    24 are all ones, all ones but one or two, at every tail length."""
    rnd = random.Random(41)
    flagged = 0
    zs = states(60000, seed=32)
    for zk in zs:
        yp, q, bits, v = back_step_f32_model(zk - 1)
        if v == 0:
            flagged += 1
            continue
        assert bits == rz_f32_bits(yp + 1), zk
    assert flagged < 200
    checked = 0
    for tail in range(9, 30):
        for k in range(1, 5):                     # all ones minus 0, 1, 2, 3
            for _ in range(150):
                head = rnd.randrange(1 << 23, 1 << 24)
                qv = (head << tail) | ((1 << tail) - k)
                zp = -(-(qv * M) // 2 ** 53)     # smallest state with this quotient
                if not 0 < zp < M or (zp << 53) // M != qv:
                    continue
                yp, q, bits, v = back_step_f32_model(((zp << 53) % M) - 1)
                assert q == qv
                if k <= 2 or tail == 9:
                    assert v == 0, (tail, k)      # must (k <= 2) or does take the exact path
                else:                             # bit 1 of Q is zero: not flagged
                    assert v != 0 and bits == rz_f32_bits(zp), (tail, k)
                    checked += 1
    assert checked > 3000
    # variates below 2^-20 (quotient below 2^33) always take it
    for qv in (list(range(1, 5000)) + [rnd.randrange(1, 2 ** 33) for _ in range(5000)]
               + [2 ** 33 - 1 - i for i in range(100)]):
        zp = -(-(qv * M) // 2 ** 53)
        if 0 < zp < M and (zp << 53) // M == qv:
            assert back_step_f32_model(((zp << 53) % M) - 1)[3] == 0


# ---------------------------------------------- FP32 runs from one product
def neg_minv_words_model(W):
    """-m^-1 mod 2^(32 W) word by word, as the device header builds it."""
    inv = pow(M, -1, 2 ** 32)
    A, words = 1, []
    for _ in range(W):
        n = (-A * inv) % 2 ** 32
        A += M * n
        assert A % 2 ** 32 == 0 and A < 2 ** 86
        words.append(n)
        A >>= 32
    return words


def f32_from_words_model(u1, u0):
    """The conversion of X = (u1:u0) = Q 2^11 to FP32 bits and the flag (0:
    the exact path is needed), as back_step_f32_model forms them."""
    c = clz32(u1) if u1 else MASK32
    mant = (((((u1 << 32) | u0) << c) >> 32) & MASK32) >> 8 if c < 32 else u0 >> 8
    e = (c * 0xFF800000 + 0x3E800000) & MASK32
    v = ((~(u0 | 0xFFF) & MASK32) << c) & MASK32 if c < 32 else 0
    return (mant + e) & MASK32, v


def digit_run_model(z, C):
    """One lane's run of C FP32 variates from the state one past it, on 32-bit
    words as the device code forms it: the words of z N mod 2^(32 W), each from
    four 32-bit products and the running carry V, then digit i (element
    C - 1 - i) read as X = (u1:u0) from bits [53i - 11, 53i + 53).  Returns
    the words, the FP32 bits of elements 0 .. C-1 and their flags."""
    W = (53 * C + 31) // 32
    N = neg_minv_words_model(W)
    z0, z1 = z & MASK32, z >> 32
    assert z1 < 2 ** 21
    r, V = [], 0
    for i in range(W):
        x = V + (z1 * N[i - 1] if i > 0 else 0)
        assert x < 2 ** 54
        s = x + z0 * N[i]
        assert s < 2 ** 65
        r.append(s & MASK32)
        V = s >> 32
        assert V < 2 ** 33

    def bits32(pos):
        if pos < 0:
            return (r[0] << -pos) & MASK32
        k, o = pos // 32, pos % 32
        return r[k] if o == 0 else funnel_r(r[k], r[k + 1], o)

    bits, flags = [0] * C, [0] * C
    for i in range(C):
        bits[C - 1 - i], flags[C - 1 - i] = f32_from_words_model(bits32(53 * i + 21),
                                                                 bits32(53 * i - 11))
    return r, bits, flags


def test_run_constant_is_minus_the_inverse_of_m():
    for W in (2, 9, 73, 90):
        N = sum(w << (32 * i) for i, w in enumerate(neg_minv_words_model(W)))
        assert (N * M + 1) % 2 ** (32 * W) == 0
        assert N == (-pow(M, -1, 2 ** (32 * W))) % 2 ** (32 * W)
    assert sum(w << (32 * i) for i, w in enumerate(neg_minv_words_model(2))) % 2 ** 53 == MP


@pytest.mark.parametrize("C", [44, 32, 4, 12, 252])
def test_run_product_fields_are_the_runs_quotients(C):
    """Field i of z N mod 2^(53 C) is floor(2^53 s / m) of the state s that
    lies i + 1 steps before z (the 2-adic digits of -z/m); the word-level
    product equals the big-integer one; every digit's top word is distinct."""
    W = (53 * C + 31) // 32
    N = (-pow(M, -1, 2 ** (53 * C))) % 2 ** (53 * C)
    inv53 = pow(2, -53, M)
    tops = [(53 * i + 52) // 32 for i in range(C)]
    assert len(set(tops)) == C and max(tops) == W - 1
    for z in states(300 if C < 100 else 40, seed=51 + C):
        r, _, _ = digit_run_model(z, C)
        P = sum(w << (32 * i) for i, w in enumerate(r))
        assert P == z * (-pow(M, -1, 2 ** (32 * W))) % 2 ** (32 * W)
        assert P % 2 ** (53 * C) == (z * N) % 2 ** (53 * C)
        s = z
        for i in range(C):
            s = s * inv53 % M                  # one step back
            assert (P >> (53 * i)) % 2 ** 53 == (s << 53) // M, (z, i)
        # the run's element 0 (the redo's start) is z 2^(-53C): C steps forward give z
        assert s == z * pow(2, -53 * C, M) % M and s * pow(2, 53 * C, M) % M == z


def test_run_conversion_is_the_backward_steps_conversion():
    """Every digit of a run gets the float and the flag that the backward step
    gives the same state (the low 11 bits of u0 hold the next digit's bits
    instead of zeros, and neither reads them), so unflagged digits are RZ of
    the FP64 variate.  Adversarial states with quotient tails of all ones are
    placed inside runs."""
    C = 44
    rnd = random.Random(57)
    inv53 = pow(2, -53, M)
    zs = states(2000, seed=58)
    for tail in (9, 12, 20, 28, 29):
        for k in (1, 2, 3):
            for _ in range(30):
                head = rnd.randrange(1 << 23, 1 << 24)
                qv = (head << tail) | ((1 << tail) - k)
                zp = -(-(qv * M) // 2 ** 53)
                if 0 < zp < M and (zp << 53) // M == qv:
                    pos = rnd.randrange(C)       # element pos of a run holds zp
                    zs.append(zp * pow(2, 53 * (C - pos), M) % M)
                    break
    flagged = 0
    for z in zs:
        _, bits, flags = digit_run_model(z, C)
        s = z
        for e in range(C - 1, -1, -1):           # element e holds state s_e
            _, q, sbits, v = back_step_f32_model(s - 1)
            s = s * inv53 % M
            assert (flags[e] == 0) == (v == 0), (z, e)
            if v:
                assert bits[e] == sbits == rz_f32_bits(s), (z, e)
            else:
                flagged += 1
    assert flagged >= 10  # the k <= 2 tails and tail 9 must flag (11 placed)
