"""Number theory for tests of the 3^40 modulus variant (test-side only).

Exact discrete logarithms base 2 modulo 3^k by Pohlig-Hellman: the group of
units modulo 3^k is cyclic of order 2*3^(k-1) with generator 2, so a log is
found digit by digit in base 3 on the 3-part and by one power on the 2-part.
Tests use it to place a chosen state (for instance z = 1, the smallest
variate) at a known output index of a known seed.
"""
from __future__ import annotations

M40 = 3 ** 40
P40 = 2 * 3 ** 39
H40 = M40 // 2


def dlog2(t: int, k: int = 40) -> int:
    """e in [0, 2*3^(k-1)) with 2^e = t (mod 3^k); t must be prime to 3."""
    m = 3 ** k
    t %= m
    if t % 3 == 0:
        raise ValueError("not a unit modulo 3^k")
    n3 = 3 ** (k - 1)
    g = 4                       # 2^2 generates the subgroup of order 3^(k-1)
    y = t * t % m               # 2^(2e) = t^2
    gamma = pow(g, n3 // 3, m)  # an element of order 3
    x = 0
    for i in range(k - 1):
        hi = pow(y * pow(g, -x, m) % m, n3 // 3 ** (i + 1), m)
        d = next(d for d in range(3) if pow(gamma, d, m) == hi)
        x += d * 3 ** i
    b = 0 if pow(t, n3, m) == 1 else 1  # 2^(3^(k-1)) = -1
    e = x + n3 * ((b - x) % 2)
    assert pow(2, e, m) == t
    return e


def index_of_state(a: int, z: int) -> int:
    """The output index i of seed a whose state is z (modulus 3^40, step then
    emit: state of output i is 2^(a - 3^40 + 53(i+1)) * floor(3^40/2))."""
    e = dlog2(z * pow(H40, -1, M40) % M40)
    return ((e - (a - M40)) * pow(53, -1, P40) - 1) % P40
